// extern "C" entry points of gaussbox.h: argument validation and dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "plan.h"
#include "walker.h"

namespace gb {

gf_status make_box_kernel(const int32_t* radii, const double* weights, int K, BoxKernel* bk) {
    if (K < 1 || K > GF_KMAX) return GF_EUNSUPPORTED;
    if (!radii || !weights || !bk) return GF_EINVAL;
    BoxKernel b;
    b.K = K;
    double sw = 0.0;
    for (int i = 0; i < K; ++i) {
        if (radii[i] < 0 || radii[i] > kMaxRadius) return GF_EINVAL;
        if (!std::isfinite(weights[i])) return GF_EINVAL;
        b.r[i] = radii[i];
        b.w[i] = (float)weights[i];
        b.rk = radii[i] > b.rk ? radii[i] : b.rk;
        sw += (double)b.w[i] * (2.0 * radii[i] + 1.0);
    }
    b.sw = (float)sw;
    *bk = b;
    return GF_OK;
}

namespace {

bool ranges_overlap(const void* a, size_t alen, const void* b, size_t blen) {
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + blen && b0 < a0 + alen;
}

bool have_device() {
    int n = 0;
    return cudaGetDeviceCount(&n) == cudaSuccess && n > 0;
}

}  // namespace

gf_status validate_image(const Image& im) {
    if (im.H < 1 || im.W < 1 || im.C < 1 || im.C > 4) return GF_EINVAL;
    if (!im.in || !im.out) return GF_EINVAL;
    const int isz = dtype_size(im.in_dt), osz = dtype_size(im.out_dt);
    if (!isz || !osz) return GF_EINVAL;
    if (im.boundary < GF_REPLICATE || im.boundary > GF_REFLECT) return GF_EINVAL;
    // offered pairs: integer in -> f32 out; float in -> f32 / bf16 / f16 out
    if (im.out_dt == GF_U8 || im.out_dt == GF_U16) return GF_EUNSUPPORTED;
    if (dtype_is_int(im.in_dt) && im.out_dt != GF_F32) return GF_EUNSUPPORTED;
    if (im.sy < 1 || im.sx < 1 || im.oy < 0 || im.ox < 0 || im.oy >= im.sy || im.ox >= im.sx) return GF_EINVAL;
    if (im.oy >= im.H || im.ox >= im.W) return GF_EINVAL;
    const int Ho = out_h(im);
    const size_t in_row = (size_t)im.W * im.C * isz, out_row = (size_t)out_w(im) * im.C * osz;
    if (im.in_pitch < in_row || im.out_pitch < out_row) return GF_EINVAL;
    if ((size_t)im.W * im.C > (size_t)INT32_MAX / 4 || (size_t)im.H > (size_t)INT32_MAX / 4) return GF_EINVAL;
    if (im.in_pitch % isz || im.out_pitch % osz) return GF_EINVAL;
    if (((uintptr_t)im.in) % isz || ((uintptr_t)im.out) % osz) return GF_EINVAL;
    const size_t in_len = (size_t)(im.H - 1) * im.in_pitch + in_row;
    const size_t out_len = (size_t)(Ho - 1) * im.out_pitch + out_row;
    if (ranges_overlap(im.in, in_len, im.out, out_len)) return GF_EINVAL;
    return GF_OK;
}

}  // namespace gb

using namespace gb;

extern "C" {

gf_status gauss_fit_boxes(double sigma, int K, int err_kind, int32_t* radii_out, double* weights_out) {
    return fit_boxes(sigma, K, err_kind, radii_out, weights_out);
}

gf_status gauss_fit_kernel(const double* half, int n, int K, int err_kind, int32_t* radii_out, double* weights_out,
                           double* err_out) {
    return fit_kernel(half, n, K, err_kind, radii_out, weights_out, err_out);
}

gf_status gauss_fit_sigma0(int K, int err_kind, int32_t* p_out, double* c_out, double* w_out, double* err_out) {
    return fit_sigma0(K, err_kind, p_out, c_out, w_out, err_out);
}

gf_status gauss_filter_boxes(const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch, int H, int W, int C,
                             int in_dtype, int out_dtype, const int32_t* radii, const double* weights, int K,
                             int boundary, void* stream) {
    Image im;
    im.in = d_in;
    im.in_pitch = in_pitch;
    im.out = d_out;
    im.out_pitch = out_pitch;
    im.H = H;
    im.W = W;
    im.C = C;
    im.in_dt = in_dtype;
    im.out_dt = out_dtype;
    im.boundary = boundary;
    gf_status st = validate_image(im);
    if (st != GF_OK) return st;
    BoxKernel bk;
    st = make_box_kernel(radii, weights, K, &bk);
    if (st != GF_OK) return st;
    if (!have_device()) return GF_EUNSUPPORTED;
    return launch_filter(im, bk, nullptr, stream);
}

gf_status gauss_filter_planned(const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch, int H, int W, int C,
                               int in_dtype, int out_dtype, const int32_t* radii, const double* weights, int K,
                               int boundary, const gf_plan* plan, void* stream) {
    Image im;
    im.in = d_in;
    im.in_pitch = in_pitch;
    im.out = d_out;
    im.out_pitch = out_pitch;
    im.H = H;
    im.W = W;
    im.C = C;
    im.in_dt = in_dtype;
    im.out_dt = out_dtype;
    im.boundary = boundary;
    gf_status st = validate_image(im);
    if (st != GF_OK) return st;
    BoxKernel bk;
    st = make_box_kernel(radii, weights, K, &bk);
    if (st != GF_OK) return st;
    if (!have_device()) return GF_EUNSUPPORTED;
    return launch_filter(im, bk, plan, stream);
}

gf_status gauss_filter_sampled(const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch, int H, int W, int C,
                               int in_dtype, int out_dtype, const int32_t* radii, const double* weights, int K,
                               int boundary, int step_y, int step_x, int off_y, int off_x, const gf_plan* plan,
                               void* stream) {
    Image im;
    im.in = d_in;
    im.in_pitch = in_pitch;
    im.out = d_out;
    im.out_pitch = out_pitch;
    im.H = H;
    im.W = W;
    im.C = C;
    im.in_dt = in_dtype;
    im.out_dt = out_dtype;
    im.boundary = boundary;
    im.sy = step_y;
    im.sx = step_x;
    im.oy = off_y;
    im.ox = off_x;
    gf_status st = validate_image(im);
    if (st != GF_OK) return st;
    BoxKernel bk;
    st = make_box_kernel(radii, weights, K, &bk);
    if (st != GF_OK) return st;
    if (!have_device()) return GF_EUNSUPPORTED;
    return launch_filter(im, bk, plan, stream);
}

gf_status gauss_plan_default(int H, int W, int C, int in_dtype, int out_dtype, const int32_t* radii, int K,
                             gf_plan* out) {
    if (!out || !radii || H < 1 || W < 1 || C < 1 || C > 4) return GF_EINVAL;
    if (!dtype_size(in_dtype) || !dtype_size(out_dtype)) return GF_EINVAL;
    double ones[GF_KMAX] = {1, 1, 1, 1, 1};
    BoxKernel bk;
    gf_status st = make_box_kernel(radii, ones, K, &bk);
    if (st != GF_OK) return st;
    if (!have_device()) return GF_EUNSUPPORTED;
    Image im;
    im.H = H;
    im.W = W;
    im.C = C;
    im.in_dt = in_dtype;
    im.out_dt = out_dtype;
    FilterPlan fp;
    st = resolve_plan(im, bk, nullptr, fp);
    if (st == GF_OK) plan_to_abi(fp, out);
    return st;
}

gf_status gauss_filter(const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch, int H, int W, int C,
                       int in_dtype, int out_dtype, double sigma, int K, int boundary, void* stream) {
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return GF_EINVAL;
    if (K < 1 || K > GF_KMAX) return GF_EUNSUPPORTED;
    int32_t r[GF_KMAX];
    double w[GF_KMAX];
    gf_status st = fit_boxes(sigma, K, GF_ERR_QF, r, w);
    if (st != GF_OK) return st;
    return gauss_filter_boxes(d_in, in_pitch, d_out, out_pitch, H, W, C, in_dtype, out_dtype, r, w, K, boundary,
                              stream);
}

gf_status gauss_walker_compile(int in_dtype, const int32_t* radii, int K, char* log, size_t log_len) {
    if (!radii) return GF_EINVAL;
    double ones[GF_KMAX] = {1, 1, 1, 1, 1};
    BoxKernel bk;
    gf_status st = make_box_kernel(radii, ones, K, &bk);
    if (st != GF_OK) return st;
    std::string text;
    st = walker_compile_check(in_dtype, bk, &text);
    if (log && log_len > 0) {
        const size_t n = std::min(log_len - 1, text.size());
        std::copy(text.begin(), text.begin() + n, log);
        log[n] = '\0';
    }
    return st;
}

gf_status gauss_depth_walker_compile(const int32_t* radii, int K, char* log, size_t log_len) {
    if (!radii) return GF_EINVAL;
    double ones[GF_KMAX] = {1, 1, 1, 1, 1};
    BoxKernel bz;
    gf_status st = make_box_kernel(radii, ones, K, &bz);
    if (st != GF_OK) return st;
    std::string text;
    st = depth_walk_compile_check(bz, &text);
    if (log && log_len > 0) {
        const size_t n = std::min(log_len - 1, text.size());
        std::copy(text.begin(), text.begin() + n, log);
        log[n] = '\0';
    }
    return st;
}

gf_status gauss_row_box_sums(const void* d_in, size_t in_pitch, int32_t* d_out, size_t out_pitch,
                             size_t plane_stride_elems, int H, int W, int C, int in_dtype, const int32_t* radii,
                             int K, int boundary, void* stream) {
    if (H < 1 || W < 1 || C < 1 || C > 4 || !d_in || !d_out || !radii) return GF_EINVAL;
    if (in_dtype != GF_U8 && in_dtype != GF_U16) return GF_EUNSUPPORTED;
    if (boundary < GF_REPLICATE || boundary > GF_REFLECT) return GF_EINVAL;
    const size_t isz = dtype_size(in_dtype);
    if (in_pitch < (size_t)W * C * isz || out_pitch < (size_t)W * C * 4 || out_pitch % 4) return GF_EINVAL;
    if (K > 1 && plane_stride_elems * 4 < (size_t)(H - 1) * out_pitch + (size_t)W * C * 4) return GF_EINVAL;
    double ones[GF_KMAX] = {1, 1, 1, 1, 1};
    BoxKernel bk;
    gf_status st = make_box_kernel(radii, ones, K, &bk);
    if (st != GF_OK) return st;
    if (!have_device()) return GF_EUNSUPPORTED;
    return launch_row_box_sums(d_in, in_pitch, d_out, out_pitch, plane_stride_elems, H, W, C, in_dtype, bk,
                               boundary, stream);
}

}  // extern "C"

namespace gb {

gf_status collect_batch(const gf_image_desc* images, int n, Image* ims, BoxKernel* bks, BatchSpan* spans) {
    int ns = 0;
    for (int i = 0; i < n; ++i) {
        const gf_image_desc& d = images[i];
        Image& im = ims[i];
        im.in = d.d_in;
        im.in_pitch = d.in_pitch;
        im.out = d.d_out;
        im.out_pitch = d.out_pitch;
        im.H = d.H;
        im.W = d.W;
        im.C = d.C;
        im.in_dt = d.in_dtype;
        im.out_dt = d.out_dtype;
        im.boundary = d.boundary;
        im.plan = d.plan ? *d.plan : gf_plan{0, 0, 0, 0, 0, 0};
        gf_status st = validate_image(im);
        if (st != GF_OK) return st;
        if (d.radii && d.weights) {
            st = make_box_kernel(d.radii, d.weights, d.K, &bks[i]);
        } else {
            if (!(d.sigma > 0.0) || !std::isfinite(d.sigma)) return GF_EINVAL;
            if (d.K < 1 || d.K > GF_KMAX) return GF_EUNSUPPORTED;
            int32_t r[GF_KMAX];
            double w[GF_KMAX];
            st = fit_boxes(d.sigma, d.K, GF_ERR_QF, r, w);
            if (st == GF_OK) st = make_box_kernel(r, w, d.K, &bks[i]);
        }
        if (st != GF_OK) return st;
        const size_t ib = (size_t)(d.H - 1) * d.in_pitch + (size_t)d.W * d.C * dtype_size(d.in_dtype);
        const size_t ob = (size_t)(d.H - 1) * d.out_pitch + (size_t)d.W * d.C * dtype_size(d.out_dtype);
        spans[ns++] = {(uintptr_t)d.d_in, (uintptr_t)d.d_in + ib, 0};
        spans[ns++] = {(uintptr_t)d.d_out, (uintptr_t)d.d_out + ob, 1};
    }
    // outputs may overlap neither inputs nor other outputs (inputs may share memory)
    std::sort(spans, spans + ns, [](const BatchSpan& x, const BatchSpan& y) { return x.a < y.a; });
    uintptr_t end_any = 0, end_out = 0;
    for (int k = 0; k < ns; ++k) {
        const BatchSpan& sp = spans[k];
        if (sp.out ? sp.a < end_any : sp.a < end_out) return GF_EINVAL;
        end_any = std::max(end_any, sp.b);
        if (sp.out) end_out = std::max(end_out, sp.b);
    }
    return GF_OK;
}

}  // namespace gb

extern "C" {

gf_status gauss_filter_batch(gf_handle h, const gf_image_desc* images, int n, void* stream) {
    if (!h || n < 0 || (n > 0 && !images)) return GF_EINVAL;
    if (n == 0) return GF_OK;
    std::vector<Image> ims(n);
    std::vector<BoxKernel> bks(n);
    std::vector<BatchSpan> spans(2 * (size_t)n);
    gf_status st = collect_batch(images, n, ims.data(), bks.data(), spans.data());
    if (st != GF_OK) return st;
    for (int i = 0; i < n; ++i) apply_tuned(h, ims[i], bks[i]);
    if (cudaSetDevice(h->device) != cudaSuccess) return GF_ECUDA;
    HandleScope scope(h->status_word, h->wait_cycles);
    return launch_filter_batch(h, ims.data(), bks.data(), n, stream);
}

int gf_batch_launches(gf_handle h) { return h ? h->last_launches : -1; }

gf_status gf_get_device_status(int clear) {
    if (!have_device()) return GF_EUNSUPPORTED;
    int v = 0;
    gf_status st = read_device_status(clear, &v);
    if (st != GF_OK) return st;
    return (gf_status)v;
}

const char* gf_status_string(int status) {
    switch (status) {
        case GF_OK: return "GF_OK";
        case GF_EINVAL: return "GF_EINVAL: invalid argument";
        case GF_ENOMEM: return "GF_ENOMEM: allocation failed";
        case GF_ECUDA: return "GF_ECUDA: CUDA call failed";
        case GF_ETIMEOUT: return "GF_ETIMEOUT: bounded device wait expired";
        case GF_EUNSUPPORTED: return "GF_EUNSUPPORTED: unsupported configuration";
        case GF_EADMIT: return "GF_EADMIT: request exceeds the HBM budget";
        case GF_EBUSY: return "GF_EBUSY: busy / not finished";
        case GF_ELIMIT: return "GF_ELIMIT: request exceeds a fixed capacity of the call";
        default: return "GF_UNKNOWN";
    }
}

const char* gf_version(void) { return "gaussbox 0.1 (sm_103a)"; }

}  // extern "C"
