// gf_handle: device selection, grow-only scratch and the batch graph cache.
#include <cuda_runtime.h>

#include <new>

#include "internal.h"
#include "serve.h"

namespace gb {

gf_status scratch_reserve(Scratch& s, size_t dev_bytes, size_t pinned_bytes) {
    if (dev_bytes > s.dev_bytes) {
        if (s.dev) cudaFree(s.dev);
        s.dev = nullptr;
        s.dev_bytes = 0;
        const size_t want = dev_bytes + dev_bytes / 2;
        if (cudaMalloc(&s.dev, want) != cudaSuccess) return GF_ENOMEM;
        s.dev_bytes = want;
    }
    if (pinned_bytes > s.pinned_bytes) {
        if (s.pinned) cudaFreeHost(s.pinned);
        s.pinned = nullptr;
        s.pinned_bytes = 0;
        const size_t want = pinned_bytes + pinned_bytes / 2;
        if (cudaMallocHost(&s.pinned, want) != cudaSuccess) return GF_ENOMEM;
        s.pinned_bytes = want;
    }
    return GF_OK;
}

void scratch_free(Scratch& s) {
    if (s.dev) cudaFree(s.dev);
    if (s.pinned) cudaFreeHost(s.pinned);
    s = Scratch();
}

}  // namespace gb

using namespace gb;

extern "C" {

gf_status gf_create(gf_handle* out, const gf_config* cfg) {
    if (!out) return GF_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) return GF_EUNSUPPORTED;
    gf_handle_s* h = new (std::nothrow) gf_handle_s();
    if (!h) return GF_ENOMEM;
    if (cfg) {
        if (cfg->device < 0 || cfg->device >= n) {
            delete h;
            return GF_EINVAL;
        }
        h->device = cfg->device;
        h->hbm_budget = cfg->hbm_budget_bytes;
        h->use_graphs = cfg->use_graphs;
        if (cfg->tune_cache) h->tune_cache = cfg->tune_cache;
    } else {
        cudaGetDevice(&h->device);
    }
    if (cudaSetDevice(h->device) != cudaSuccess) {
        delete h;
        return GF_ECUDA;
    }
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        delete h;
        return GF_ECUDA;
    }
    h->staged_event = ev;
    *out = h;
    return GF_OK;
}

gf_status gf_destroy(gf_handle h) {
    if (!h) return GF_OK;
    cudaSetDevice(h->device);
    server_destroy(h);
    cudaDeviceSynchronize();
    if (h->graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(h->graph_exec));
    if (h->staged_event) cudaEventDestroy(static_cast<cudaEvent_t>(h->staged_event));
    scratch_free(h->batch);
    delete h;
    return GF_OK;
}

}  // extern "C"
