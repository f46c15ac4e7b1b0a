// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/gaussbox.h"

namespace gb {

// ---- host fitter (fit.cpp) -------------------------------------------------
gf_status fit_sigma0(int K, int err_kind, int32_t* p, double* c, double* w, double* err);
gf_status fit_boxes(double sigma, int K, int err_kind, int32_t* radii, double* weights);
gf_status fit_kernel(const double* half, int n, int K, int err_kind, int32_t* radii, double* weights, double* err);

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

// Longest column tile, in output rows, whose FP32 running sums keep the box
// differences accurate.  A difference of two running sums of the column pass
// is off by up to 2^-24 of their magnitude, which grows with the tile's
// n = rows + 2 rk values; against the smallest box (2 r_min + 1 values) that is
// about 2^-24 n / (2 r_min + 1) times the ratio of the value range to the mean.
// n <= 32 (2 r_min + 1) keeps it below ~8e-6 of the image mean (never fewer
// than 8 rows; kernels whose 2 rk alone exceed the budget get 8-row tiles).
inline int column_tile_cap(const BoxKernel& bk) {
    int rmin = bk.rk;
    for (int i = 0; i < bk.K; ++i) rmin = bk.r[i] < rmin ? bk.r[i] : rmin;
    const int cap = 32 * (2 * rmin + 1) - 2 * bk.rk;
    return cap > 8 ? cap : 8;
}
// Column tile height for `H` rows: at most `rows`, at most column_tile_cap, and
// at least H / 65535 (the launch's grid y limit).
inline int column_tile_rows(int rows, int H, const BoxKernel& bk) {
    int t = rows < column_tile_cap(bk) ? rows : column_tile_cap(bk);
    const int lo = (H + 65534) / 65535;
    t = t > lo ? t : lo;
    return t < H ? (t > 0 ? t : 1) : H;
}

struct Image {
    const void* in = nullptr;
    size_t in_pitch = 0;    // bytes
    void* out = nullptr;
    size_t out_pitch = 0;   // bytes
    int H = 0, W = 0, C = 0;
    int in_dt = GF_F32, out_dt = GF_F32;
    int boundary = GF_REPLICATE;
    gf_plan plan = {0, 0, 0, 0, 0, 0};   // requested plan (all zero: default)
    // sampled outputs (two-pass path only): out(i, j) = Y(oy + i sy, ox + j sx)
    int sy = 1, sx = 1, oy = 0, ox = 0;
};

// Output rows / columns of an image (all of them unless sampled).
inline int out_h(const Image& im) { return (im.H - im.oy + im.sy - 1) / im.sy; }
inline int out_w(const Image& im) { return (im.W - im.ox + im.sx - 1) / im.sx; }
inline bool is_sampled(const Image& im) { return im.sy > 1 || im.sx > 1; }

// Tile plan of the fused strip kernel.
struct StripPlan {
    int TWp = 0;     // strip width in pixels
    int TH = 0;      // output rows per CTA
    int nstrips = 0, nrowtiles = 0;
};

// Tile plan of the two-pass form.
struct TwoPassPlan {
    int seg_px = 0;   // row pass: output pixels per row segment
    int row_th = 0;   // row pass: rows per CTA (multiple of 8)
    int CW = 0;       // column pass: element columns per CTA (32, 64, 128, 256)
    int col_th = 0;   // column pass: output rows per CTA
    int accum = GF_ACCUM_COMPENSATED;
};

// A resolved plan of one image: the path and both paths' tile shapes.
struct FilterPlan {
    int path = GF_PATH_FUSED;
    StripPlan strip;
    TwoPassPlan two;
};

TwoPassPlan default_twopass_plan(const Image& im, const BoxKernel& bk);
// Fills every zero field of `req` (path GF_PATH_AUTO picks one) and checks the rest.
gf_status resolve_plan(const Image& im, const BoxKernel& bk, const gf_plan* req, FilterPlan& out);
void plan_to_abi(const FilterPlan& fp, gf_plan* out);

gf_status make_box_kernel(const int32_t* radii, const double* weights, int K, BoxKernel* bk);
gf_status validate_image(const Image& im);

// Fused row+column filter of one image (filter_host.cu).  `plan` may be null (default).
gf_status launch_fused(const Image& im, const BoxKernel& bk, const StripPlan* plan, void* stream);
// Host and device images of gauss_filter_host (byte pointers and pitches).
struct HostRows {
    const unsigned char* hin;
    unsigned char* hout;
    unsigned char* din;
    unsigned char* dout;
    size_t in_pitch, out_pitch, dpi, dpo, irow, orow;
};
// gauss_filter_host on the fused or register-walk path in slabs of row tiles
// (copy in, filter, copy out overlapped on two side streams of the handle);
// GF_EUNSUPPORTED if the image has too few row tiles to pipeline or takes
// another path (filter_host.cu).
gf_status filter_host_pipelined(gf_handle_s* h, const Image& im, const BoxKernel& bk, const FilterPlan& fp,
                                const HostRows& hr, cudaStream_t s);
// One image on the path `plan` selects (null: the default plan; twopass_host.cu).
gf_status launch_filter(const Image& im, const BoxKernel& bk, const gf_plan* plan, void* stream);
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

// Side streams of a handle on which the classes of a batch run concurrently.
constexpr int kMaxFork = 12;
struct Fork {
    int n = 0;
    cudaStream_t s[kMaxFork] = {};
    cudaEvent_t ev[kMaxFork + 1] = {};   // ev[0]: fork point, ev[1 + f]: side stream f done
};

}  // namespace gb

struct gf_handle_s {
    int device = 0;
    int* status_word = nullptr;        // device word the handle's kernels report expired waits in
    long long wait_cycles = 0;         // bound of each pipeline wait (0: the default)
    size_t hbm_budget = 0;
    int use_graphs = 1;
    std::string tune_cache;
    gb::Scratch batch;                 // work lists, per-image parameters, tensor maps
    gb::Scratch host_in, host_out;     // device images of gauss_filter_host
    gb::Scratch inter;                 // two-pass intermediates of a batch
    gb::Scratch vol;                   // in-plane result of a volume (FP32)
    void* graph_exec = nullptr;        // cudaGraphExec_t of the last batch signature
    std::string graph_sig;
    std::string batch_key;             // inputs of the batch the graph last ran (replay without planning)
    int batch_key_launches = 0;        // kernel launches of that batch
    void* staged_event = nullptr;      // cudaEvent_t: pinned batch staging consumed
    gb::Fork fork;                     // side streams for concurrent batch classes
    std::map<std::string, gf_plan> tuned;   // autotuned plans by shape class
    int last_launches = 0;             // kernel launches of the last batch
    std::vector<void*> slab_events;    // cudaEvent_t pool of the pipelined host call
    gb::Server* server = nullptr;
};

namespace gb {

// Autotuner (tune.cpp): shape-class key, lookup of a tuned plan for an image
// whose own plan is all zero, and the cache file.
std::string tune_key(const Image& im, const BoxKernel& bk);
void apply_tuned(const gf_handle_s* h, Image& im, const BoxKernel& bk);
void tune_load(gf_handle_s* h);

gf_status scratch_reserve(Scratch& s, size_t dev_bytes, size_t pinned_bytes);
void scratch_free(Scratch& s);

// Validates n batch descriptors and fits their boxes (abi.cpp); `spans` is
// caller storage for 2 n address ranges (the overlap check).
struct BatchSpan {
    uintptr_t a, b;
    int out;
};
gf_status collect_batch(const gf_image_desc* images, int n, Image* ims, BoxKernel* bks, BatchSpan* spans);

// True if the fused kernel's working set for strips of TWp pixels fits the device.
bool fused_fits(const Image& im, const BoxKernel& bk, int TWp);
// CTAs of the fused kernel (strips of TWp pixels, TMA staging) resident per SM.
int fused_ctas_per_sm(const Image& im, const BoxKernel& bk, int TWp);

// Batched filter of n images (filter_host.cu).
gf_status launch_filter_batch(gf_handle_s* h, const Image* ims, const BoxKernel* bks, int n, void* stream);

// Depth pass of a volume (twopass_host.cu): one column launch filtering, for
// every image row y (blockIdx.z) and element column, the line of D values
// R[z][y][e] (R: D H rows of r_pitch bytes, FP32) into out (D H rows of
// out_pitch bytes, out_dt).
// In-plane two-pass filter of D slices of H rows (twopass_host.cu): the row
// launch over all D H rows of `tall` into R1, then one column launch whose
// blockIdx.z is the slice, into R2 (FP32, r2_pitch).  R1 and R2 hold D H rows
// of the two-pass intermediate pitch (128-byte aligned).
gf_status launch_slices_twopass(const Image& tall, int D, int H, const BoxKernel& bk, const TwoPassPlan& plan,
                                void* R1, void* R2, size_t r2_pitch, cudaStream_t s);
gf_status launch_depth_pass(const float* R, size_t r_pitch, int D, int H, int W, int C, void* out, size_t out_pitch,
                            int out_dt, int boundary, const BoxKernel& bz, cudaStream_t s);

// Device status word (filter.cu).
gf_status read_device_status(int clear, int* value);
int device_sm_count();

}  // namespace gb
