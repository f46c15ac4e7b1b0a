// Batch planning shared by the handle-based batch call and callers that
// supply their own staging storage.  Host-only declarations.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "twopass.h"

namespace gb {

// Everything a launch needs for one image: kernel parameters, its TMA tensor
// map, shared-memory bytes, grid and tile count.
struct Prepared {
    KParams kp{};
    CUtensorMap maps[3];   // row map, 8-row map (KParams::rows8), output map (KParams::tma_store)
    size_t smem = 0;
    int twmax = 256;
    dim3 grid;
    int ntiles = 0;
};

// Fused launch of a prepared image: all row tiles, or the slab [ty0, ty1).
gf_status prepare_fused(const Image& im, const BoxKernel& bk, const StripPlan* plan, Prepared& out);
gf_status launch_prepared(const Image& im, Prepared pr, void* stream, int ty0 = 0, int ty1 = -1);

// One persistent launch: the images of one type class.
struct BatchClass {
    int first, count, key, twmax, ntiles, grid, tmem_cols, nstage;
    int in_dt, out_dt, C;
    size_t smem;
    BatchArgs ba;
};

// Batched two-pass launches: up to kTPBatchMax two-pass images that take the
// same row kernel and the same column kernel, each at the same CTAs per SM,
// run as one row launch and then one column launch on one stream.  Members
// are entries first .. first + count of tp_order.
struct TPClass {
    int first = 0, count = 0;
    long long key = 0;
    int in_dt = 0, out_dt = 0, C = 0, CW = 0, B = 0;
    int tiles_r = 0, tiles_c = 0;
    size_t smem_r = 0, smem_c = 0;
    TPRows ar{};   // launch parameters (filled by batch_stage)
    TPCols ac{};
};

// Caller-provided storage (n entries each; tp and tp_off may be null when no
// image may take the two-pass path) and the staging-block layout.
struct BatchWork {
    Prepared* pr = nullptr;
    int* order = nullptr;
    BatchClass* cls = nullptr;
    TwoPass* tp = nullptr;
    size_t* tp_off = nullptr;   // byte offset of each two-pass intermediate
    int* tp_img = nullptr;      // optional: image index of each two-pass entry
    int* wk_img = nullptr;      // images run by the register walk, one launch each (null: run them fused)
    const Image* ims = nullptr; // the planned images (set by batch_plan)
    const BoxKernel* bks = nullptr;
    int nwk = 0;
    int ncls = 0;
    int nfused = 0;             // fused images: order[0 .. nfused)
    int ntp = 0;                // two-pass images: tp[0 .. ntp)
    size_t inter_total = 0;     // bytes of all two-pass intermediates
    size_t total = 0, o_maps = 0, o_ts = 0, o_cnt = 0;
    // two-pass images in batched launches (default accumulation) grouped by
    // class, and those launched on their own
    std::vector<int> tp_order, tp_solo;
    std::vector<TPClass> tp_cls;
    size_t o_tpmr = 0, o_tpmc = 0;   // staging offsets of their tensor maps
};

// Kernel launches of a planned batch.
inline int batch_launches(const BatchWork& w) {
    return w.ncls + 2 * (int)(w.tp_cls.size() + w.tp_solo.size()) + w.nwk;
}

// Plans n images (same plans as the single-image path, or each image's own)
// into fused classes and two-pass images, and sizes the staging block
// (w.total bytes) and the intermediates (w.inter_total).  Without tp storage
// every image runs fused (an explicit two-pass plan is GF_EUNSUPPORTED).
gf_status batch_plan(const Image* ims, const BoxKernel* bks, int n, BatchWork& w);
// Points the two-pass images at their intermediates inside `inter_base`.
gf_status batch_bind(BatchWork& w, unsigned char* inter_base);
// Writes the staging block to `host_block` for a device copy at `dev_base`.
void batch_stage(BatchWork& w, int n, unsigned char* host_block, unsigned char* dev_base);
// Copies the block to the device and launches one persistent kernel per class:
// all on `q`, or (fork non-null) the first class on `q` and the others on the
// fork's side streams, joined back into `q`.
gf_status batch_enqueue(const BatchWork& w, unsigned char* dev_base, const void* host_block, cudaStream_t q,
                        const Fork* fork = nullptr);

}  // namespace gb
