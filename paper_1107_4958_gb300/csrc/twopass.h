// Host side of the two-pass filter (row pass -> FP32 intermediate R -> column
// pass) and the plan that selects between it and the fused strip kernel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "twopass_kernel.cuh"

namespace gb {

// Both launches of one image, ready except for the intermediate's address.
struct TwoPass {
    KParams kp{};
    CUtensorMap maps_in[2];   // input row map, 8-row map
    dim3 grid_r;
    size_t smem_r = 0;
    CParams cp{};
    CUtensorMap maps_r[2];    // intermediate: row map, band map (lane sums)
    dim3 grid_c;
    size_t smem_c = 0;
    int CW = 0;
    size_t r_pitch = 0, r_bytes = 0;   // intermediate: H rows of r_pitch bytes
    int in_dt = GF_F32, out_dt = GF_F32;
    TwoPassPlan plan;
};

// Bytes of the FP32 intermediate of an image (H rows, 128-byte aligned pitch).
size_t twopass_inter_bytes(const Image& im);
// The path the resolved plan of `im` takes (its own plan or the default).
int planned_path(const Image& im, const BoxKernel& bk);
// One image on its resolved plan; a two-pass image uses the intermediate at
// `inter` (twopass_inter_bytes, 128-byte aligned), a fused one ignores it.
gf_status launch_filter_into(const Image& im, const BoxKernel& bk, void* inter, cudaStream_t s);

gf_status prepare_twopass(const Image& im, const BoxKernel& bk, const TwoPassPlan& plan, TwoPass& tp);
// Points both passes at the intermediate R (r_bytes, 128-byte aligned).
gf_status bind_twopass(TwoPass& tp, void* R);
gf_status enqueue_twopass(const TwoPass& tp, cudaStream_t s);
// prepare + R from the library's stream-ordered pool + enqueue + release on `s`.
gf_status launch_twopass(const Image& im, const BoxKernel& bk, const TwoPassPlan& plan, cudaStream_t s);

// Running sums in HBM (global_path.cu): any radius, four launches; `scratch`
// holds global_path_bytes (256-byte aligned).
size_t global_path_bytes(const Image& im, const BoxKernel& bk);
gf_status launch_global(const Image& im, const BoxKernel& bk, void* scratch, cudaStream_t s);

}  // namespace gb
