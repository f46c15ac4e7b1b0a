// Batch planning shared by the handle-based batch call and callers that
// supply their own staging storage.  Host-only declarations.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "strip_kernel.cuh"

namespace gb {

// Everything a launch needs for one image: kernel parameters, its TMA tensor
// map, shared-memory bytes, grid and tile count.
struct Prepared {
    KParams kp{};
    CUtensorMap map;
    size_t smem = 0;
    int twmax = 256;
    dim3 grid;
    int ntiles = 0;
};

// One persistent launch: the images of one type class.
struct BatchClass {
    int first, count, key, twmax, ntiles, grid, tmem_cols, nstage;
    int in_dt, out_dt, C;
    size_t smem;
    BatchArgs ba;
};

// Caller-provided storage (n entries each) and the staging-block layout.
struct BatchWork {
    Prepared* pr = nullptr;
    int* order = nullptr;
    BatchClass* cls = nullptr;
    int ncls = 0;
    size_t total = 0, o_maps = 0, o_ts = 0, o_cnt = 0;
};

// Plans n images (same plans as the single-image path) into type classes and
// sizes the staging block (w.total bytes).
gf_status batch_plan(const Image* ims, const BoxKernel* bks, int n, BatchWork& w);
// Writes the staging block to `host_block` for a device copy at `dev_base`.
void batch_stage(BatchWork& w, int n, unsigned char* host_block, unsigned char* dev_base);
// Copies the block to the device and launches one persistent kernel per class.
gf_status batch_enqueue(const BatchWork& w, unsigned char* dev_base, const void* host_block, cudaStream_t q);

}  // namespace gb
