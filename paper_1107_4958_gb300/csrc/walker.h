// The register-walk fused filter (walker_kernel.cuh, walker_host.cu): single-
// channel integer images whose largest radius is at most kWalkerMaxRk.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <string>

#include "depth_walker.cuh"
#include "internal.h"
#include "walker_kernel.cuh"

namespace gb {

constexpr int kWalkerTW = 128;      // output columns per CTA (= threads per CTA)
constexpr int kWalkerMaxRk = 22;    // largest radius (register budget of the line walks)

// Shared-memory geometry of one radius: column ring length LC = 2 rk + 2, rows
// per band P (a multiple of LC), band row stride RP (floats), chunk stride CS
// (LC rows rounded up to 128 bytes, in floats), offset of the folded input copy
// inside a band row (bytes), the per-row window of edge strips (the row's first
// or last bytes, from which the pixels past the row are folded), bytes per CTA.
struct WalkerGeom {
    int LC = 0, P = 0, RP = 0, CS = 0, stage_off = 0;   // CS: floats per chunk of LC rows
    int win = 0, win_off = 0;   // bytes per row of the edge window (0: none) and its offset in shared memory
    size_t smem = 0;
};
struct WalkerPlan {
    WalkerGeom geom;
    int nb = 0;       // row chunks (of LC rows) per tile
    int th = 0;       // output rows per tile
    int grid_x = 0, grid_y = 0;
};

bool walker_geom(int in_dt, int rk, WalkerGeom& g);
bool walker_eligible(const Image& im, const BoxKernel& bk);
// Tile plan of an image, or of each slice of a stack of nz such images.
WalkerPlan walker_plan(const Image& im, const BoxKernel& bk, int nz = 1);
// Compiles (or finds in the cache) the kernels for in_dt and the radii of bk
// (single images and stacks of slices); needs no device.  GF_ECUDA with the
// compiler's log if a compilation fails.
gf_status walker_compile_check(int in_dt, const BoxKernel& bk, std::string* log);
// Compiles (first use) and loads the image's kernel on the current device and
// raises its shared-memory limit: after this, launch_walker makes no call that
// stream capture forbids.
gf_status walker_prepare(const Image& im, const BoxKernel& bk);
gf_status walker_load(const Image& im, const BoxKernel& bk, cudaKernel_t* kern, WalkerPlan* plan, int nz = 1);
// All row tiles, or the slab of row tiles [ty0, ty1) (ty1 < 0: to the last).
// nz > 1: `im` is the first of nz slices of im.H rows, each starting im.H rows
// (of its pitch) after the previous one in the input and in the output, each
// filtered as an image of its own (its rows fold within the slice).
gf_status launch_walker(const Image& im, const BoxKernel& bk, cudaStream_t s, int ty0 = 0, int ty1 = -1,
                        int nz = 1);

// Depth pass as a register walk (depth_walker.cuh) for depth radii up to
// kDepthWalkMaxRk: R holds D slices of H rows (r_pitch bytes, FP32, row
// element count W C) with |R| <= max_abs_r; out receives FP32 with its own
// row pitch, slices H rows apart.  GF_EUNSUPPORTED (nothing enqueued) when
// the radii are too large or the kernel cannot be built or loaded.
constexpr int kDepthWalkMaxRk = 10;
// Compiles (or finds in the cache) the depth walk for the radii of bz; needs
// no device.  GF_ECUDA with the compiler's log if the compilation fails.
gf_status depth_walk_compile_check(const BoxKernel& bz, std::string* log);
gf_status launch_depth_walk(const float* R, size_t r_pitch, int D, int H, int W, int C, void* out, size_t out_pitch,
                            int boundary, const BoxKernel& bz, double max_abs_r, cudaStream_t s);

}  // namespace gb
