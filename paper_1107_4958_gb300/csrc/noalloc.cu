// Batched filtering for callers that cannot allocate device memory.
//
// gauss_filter_batch needs a few kilobytes of device scratch per call (the
// per-image kernel parameters, TMA descriptors, tile prefix sums and ticket
// counters) and takes it from a handle that allocates it with cudaMalloc.
// The entry point below uses a fixed array compiled into the library instead,
// so it allocates no device or pinned memory at all.
#include <cuda_runtime.h>

#include <mutex>

#include "batch.h"
#include "internal.h"

namespace gb {
namespace {

constexpr int kNoAllocMaxDevices = 64;

// Scratch of gauss_filter_batch_noalloc.  Every device that loads the library
// holds one copy until the process exits.  In host code this name stands for
// the symbol only; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GF_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per
// device (with that device current) and cached.
gf_status noalloc_scratch(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF_ECUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return GF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GF_ECUDA;
        g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_addr[dev];
    return GF_OK;
}

// Host bookkeeping of fixed size in static storage (no device or pinned
// memory; the planner itself still uses ordinary host containers); calls are
// serialised on the host by g_work_mu.
struct NoAllocWork {
    Image ims[GF_NOALLOC_MAX_IMAGES];
    BoxKernel bks[GF_NOALLOC_MAX_IMAGES];
    BatchSpan spans[2 * GF_NOALLOC_MAX_IMAGES];
    Prepared pr[GF_NOALLOC_MAX_IMAGES];
    int order[GF_NOALLOC_MAX_IMAGES];
    BatchClass cls[GF_NOALLOC_MAX_IMAGES];
    unsigned char block[GF_NOALLOC_SCRATCH_BYTES];
};
NoAllocWork g_work;
std::mutex g_work_mu;

}  // namespace
}  // namespace gb

using namespace gb;

extern "C" gf_status gauss_filter_batch_noalloc(const gf_image_desc* images, int n, void* stream) {
    if (n < 0 || (n > 0 && !images)) return GF_EINVAL;
    if (n > GF_NOALLOC_MAX_IMAGES) return GF_ELIMIT;
    if (n == 0) return GF_OK;
    // The parameters reach the device by a copy from the static host block
    // below, which the next call rewrites: a copy recorded into a graph would
    // read whatever a later call left there when the graph is replayed.  So
    // the call refuses a capturing stream and enqueues nothing on it.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap) != cudaSuccess) return GF_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return GF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_work_mu);
    NoAllocWork& t = g_work;
    gf_status st = collect_batch(images, n, t.ims, t.bks, t.spans);
    if (st != GF_OK) return st;
    unsigned char* dev = nullptr;
    st = noalloc_scratch(&dev);
    if (st != GF_OK) return st;
    BatchWork w;
    w.pr = t.pr;
    w.order = t.order;
    w.cls = t.cls;
    st = batch_plan(t.ims, t.bks, n, w);
    if (st != GF_OK) return st;
    if (w.total > GF_NOALLOC_SCRATCH_BYTES) return GF_ELIMIT;
    // the block also carries the ticket counters, reset to zero for this call
    batch_stage(w, n, t.block, dev);
    return batch_enqueue(w, dev, t.block, static_cast<cudaStream_t>(stream));
}
