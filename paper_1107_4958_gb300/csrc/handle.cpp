// gf_handle: device selection, grow-only scratch and the batch graph cache.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>

#include "internal.h"
#include "plan.h"
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
        if (cfg->wait_cycles < 0) {
            delete h;
            return GF_EINVAL;
        }
        h->device = cfg->device;
        h->hbm_budget = cfg->hbm_budget_bytes;
        h->use_graphs = cfg->use_graphs;
        h->wait_cycles = cfg->wait_cycles;
        if (cfg->tune_cache) h->tune_cache = cfg->tune_cache;
        tune_load(h);
    } else {
        cudaGetDevice(&h->device);
    }
    if (cudaSetDevice(h->device) != cudaSuccess) {
        delete h;
        return GF_ECUDA;
    }
    // the handle's own status word: its kernels report expired waits here, so
    // reading or clearing it never touches another handle's or the library's
    if (cudaMalloc(reinterpret_cast<void**>(&h->status_word), sizeof(int)) != cudaSuccess) {
        delete h;
        return GF_ENOMEM;
    }
    if (cudaMemset(h->status_word, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(h->status_word);
        delete h;
        return GF_ECUDA;
    }
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaFree(h->status_word);
        delete h;
        return GF_ECUDA;
    }
    h->staged_event = ev;
    for (int f = 0; f < kMaxFork; ++f) {
        if (cudaStreamCreateWithFlags(&h->fork.s[f], cudaStreamNonBlocking) != cudaSuccess) break;
        if (cudaEventCreateWithFlags(&h->fork.ev[1 + f], cudaEventDisableTiming) != cudaSuccess) {
            cudaStreamDestroy(h->fork.s[f]);
            h->fork.s[f] = nullptr;
            break;
        }
        h->fork.n = f + 1;
    }
    if (h->fork.n > 0 && cudaEventCreateWithFlags(&h->fork.ev[0], cudaEventDisableTiming) != cudaSuccess)
        h->fork.n = 0;
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
    for (int f = 0; f < kMaxFork; ++f) {
        if (h->fork.s[f]) cudaStreamDestroy(h->fork.s[f]);
        if (h->fork.ev[1 + f]) cudaEventDestroy(h->fork.ev[1 + f]);
    }
    if (h->fork.ev[0]) cudaEventDestroy(h->fork.ev[0]);
    scratch_free(h->batch);
    scratch_free(h->host_in);
    scratch_free(h->host_out);
    scratch_free(h->inter);
    scratch_free(h->vol);
    for (void* e : h->slab_events) cudaEventDestroy(static_cast<cudaEvent_t>(e));
    if (h->status_word) cudaFree(h->status_word);
    delete h;
    return GF_OK;
}

gf_status gf_handle_status(gf_handle h, int clear) {
    if (!h) return GF_EINVAL;
    if (cudaSetDevice(h->device) != cudaSuccess) return GF_ECUDA;
    int v = 0;
    // after all work on the device (the handle's side streams do not block on the default stream)
    if (cudaDeviceSynchronize() != cudaSuccess) return GF_ECUDA;
    if (cudaMemcpy(&v, h->status_word, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GF_ECUDA;
    if (clear && cudaMemset(h->status_word, 0, sizeof(int)) != cudaSuccess) return GF_ECUDA;
    if (clear && cudaDeviceSynchronize() != cudaSuccess) return GF_ECUDA;
    return (gf_status)v;
}

gf_status gauss_filter_host(gf_handle h, const void* h_in, size_t in_pitch, void* h_out, size_t out_pitch, int H,
                            int W, int C, int in_dtype, int out_dtype, double sigma, int K, int boundary,
                            void* stream) {
    if (!h || !h_in || !h_out || H < 1 || W < 1 || C < 1 || C > 4) return GF_EINVAL;
    const int isz = dtype_size(in_dtype), osz = dtype_size(out_dtype);
    if (!isz || !osz) return GF_EINVAL;
    const size_t irow = (size_t)W * C * isz, orow = (size_t)W * C * osz;
    if (in_pitch < irow || out_pitch < orow) return GF_EINVAL;
    if (cudaSetDevice(h->device) != cudaSuccess) return GF_ECUDA;
    HandleScope scope(h->status_word, h->wait_cycles);
    const size_t dpi = (irow + 15) / 16 * 16, dpo = (orow + 15) / 16 * 16;
    gf_status st = scratch_reserve(h->host_in, dpi * H, 0);
    if (st == GF_OK) st = scratch_reserve(h->host_out, dpo * H, 0);
    if (st != GF_OK) return st;
    gf_image_desc d{};
    d.d_in = h->host_in.dev;
    d.in_pitch = dpi;
    d.d_out = h->host_out.dev;
    d.out_pitch = dpo;
    d.H = H;
    d.W = W;
    d.C = C;
    d.in_dtype = in_dtype;
    d.out_dtype = out_dtype;
    d.sigma = sigma;
    d.K = K;
    d.boundary = boundary;
    Image im;
    BoxKernel bk;
    BatchSpan spans[2];
    st = collect_batch(&d, 1, &im, &bk, spans);
    if (st != GF_OK) return st;
    apply_tuned(h, im, bk);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* din = static_cast<unsigned char*>(h->host_in.dev);
    unsigned char* dout = static_cast<unsigned char*>(h->host_out.dev);
    const unsigned char* hin = static_cast<const unsigned char*>(h_in);
    unsigned char* hout = static_cast<unsigned char*>(h_out);
    // rows [a, b) between host and device (one flat copy when both sides are dense)
    auto copy_rows = [&](bool to_dev, int a, int b, cudaStream_t q) {
        if (to_dev)
            return in_pitch == irow && dpi == irow
                       ? cudaMemcpyAsync(din + a * dpi, hin + a * in_pitch, (b - a) * irow, cudaMemcpyHostToDevice, q)
                       : cudaMemcpy2DAsync(din + a * dpi, dpi, hin + a * in_pitch, in_pitch, irow, b - a,
                                           cudaMemcpyHostToDevice, q);
        return out_pitch == orow && dpo == orow
                   ? cudaMemcpyAsync(hout + a * out_pitch, dout + a * dpo, (b - a) * orow, cudaMemcpyDeviceToHost, q)
                   : cudaMemcpy2DAsync(hout + a * out_pitch, out_pitch, dout + a * dpo, dpo, orow, b - a,
                                       cudaMemcpyDeviceToHost, q);
    };
    FilterPlan fp;
    st = resolve_plan(im, bk, &im.plan, fp);
    if (st != GF_OK) return st;
    if (fp.path == GF_PATH_FUSED || fp.path == GF_PATH_WALK) {
        const HostRows hr{hin, hout, din, dout, in_pitch, out_pitch, dpi, dpo, irow, orow};
        st = filter_host_pipelined(h, im, bk, fp, hr, s);
        if (st != GF_EUNSUPPORTED) return st;   // else: too few row tiles to pipeline
    }
    if (copy_rows(true, 0, H, s) != cudaSuccess) return GF_ECUDA;
    st = launch_filter(im, bk, &im.plan, stream);
    if (st != GF_OK) return st;
    if (copy_rows(false, 0, H, s) != cudaSuccess) return GF_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? GF_OK : GF_ECUDA;
}

}  // extern "C"
