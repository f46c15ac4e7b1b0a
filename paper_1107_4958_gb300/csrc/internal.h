// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gaussbox.h"

namespace gb {

// ---- host fitter (fit.cpp) -------------------------------------------------
gf_status fit_sigma0(int K, int err_kind, int32_t* p, double* c, double* w, double* err);
gf_status fit_boxes(double sigma, int K, int err_kind, int32_t* radii, double* weights);

// ---- element sizes ------------------------------------------------------------
inline int dtype_size(int dt) {
    switch (dt) {
        case GF_U8: return 1;
        case GF_U16: return 2;
        case GF_F32: return 4;
        case GF_BF16: return 2;
        case GF_F16: return 2;
        default: return 0;
    }
}
inline bool dtype_is_int(int dt) { return dt == GF_U8 || dt == GF_U16; }

// ---- one filter job, as the kernels see it ------------------------------------
constexpr int kMaxRadius = 4096;

struct BoxKernel {
    int K = 0;
    int r[GF_KMAX] = {0, 0, 0, 0, 0};   // inclusive radii, any order
    float w[GF_KMAX] = {0, 0, 0, 0, 0};  // slice weights (FP32)
    float sw = 0.f;                      // sum_i w_i (2 r_i + 1) in FP32
    int rk = 0;                          // max radius
};

struct Image {
    const void* in = nullptr;
    size_t in_pitch = 0;    // bytes
    void* out = nullptr;
    size_t out_pitch = 0;   // bytes
    int H = 0, W = 0, C = 0;
    int in_dt = GF_F32, out_dt = GF_F32;
    int boundary = GF_REPLICATE;
};

// Tile plan of the fused strip kernel.
struct StripPlan {
    int TWp = 0;     // strip width in pixels
    int TH = 0;      // output rows per CTA
    int nstrips = 0, nrowtiles = 0;
};

gf_status make_box_kernel(const int32_t* radii, const double* weights, int K, BoxKernel* bk);
gf_status validate_image(const Image& im);

// Fused row+column filter of one image (filter.cu).  `plan` may be null (auto).
gf_status launch_filter(const Image& im, const BoxKernel& bk, const StripPlan* plan, void* stream);
StripPlan default_plan(const Image& im, const BoxKernel& bk);
gf_status launch_row_box_sums(const void* in, size_t in_pitch, int32_t* out, size_t out_pitch,
                              size_t plane_stride, int H, int W, int C, int in_dt,
                              const BoxKernel& bk, int boundary, void* stream);

// ---- handle --------------------------------------------------------------------
struct Server;   // serving state (serve.cpp)

// Grow-only device / pinned host buffers owned by a handle.
struct Scratch {
    void* dev = nullptr;
    size_t dev_bytes = 0;
    void* pinned = nullptr;
    size_t pinned_bytes = 0;
};

}  // namespace gb

struct gf_handle_s {
    int device = 0;
    size_t hbm_budget = 0;
    int use_graphs = 1;
    std::string tune_cache;
    gb::Scratch batch;                 // work lists, per-image parameters, tensor maps
    gb::Scratch host_in, host_out;     // device images of gauss_filter_host
    void* graph_exec = nullptr;        // cudaGraphExec_t of the last batch signature
    std::string graph_sig;
    void* staged_event = nullptr;      // cudaEvent_t: pinned batch staging consumed
    gb::Server* server = nullptr;
};

namespace gb {

gf_status scratch_reserve(Scratch& s, size_t dev_bytes, size_t pinned_bytes);
void scratch_free(Scratch& s);

// Validates n batch descriptors and fits their boxes (abi.cpp); `spans` is
// caller storage for 2 n address ranges (the overlap check).
struct BatchSpan {
    uintptr_t a, b;
    int out;
};
gf_status collect_batch(const gf_image_desc* images, int n, Image* ims, BoxKernel* bks, BatchSpan* spans);

// Batched filter of n images (filter_host.cu).
gf_status launch_filter_batch(gf_handle_s* h, const Image* ims, const BoxKernel* bks, int n, void* stream);

// Device status word (filter.cu).
gf_status read_device_status(int clear, int* value);
int device_sm_count();

}  // namespace gb
