// Host side of the fused strip filter: tile plans, shared-memory layout, the TMA
// tensor map, and launches (the kernels are instantiated in inst_*.cu).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "strip_kernel.cuh"

namespace gb {

GB_DECLARE_STRIP(uint8_t, float)
GB_DECLARE_STRIP(uint16_t, float)
GB_DECLARE_STRIP(float, float)
GB_DECLARE_STRIP(float, __nv_bfloat16)
GB_DECLARE_STRIP(float, __half)
GB_DECLARE_STRIP(__nv_bfloat16, float)
GB_DECLARE_STRIP(__nv_bfloat16, __nv_bfloat16)
GB_DECLARE_STRIP(__nv_bfloat16, __half)
GB_DECLARE_STRIP(__half, float)
GB_DECLARE_STRIP(__half, __nv_bfloat16)
GB_DECLARE_STRIP(__half, __half)
GB_DECLARE_BOX(uint8_t)
GB_DECLARE_BOX(uint16_t)

__device__ int g_device_status = 0;

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode;
}

CUtensorMapDataType tma_dtype(int dt) {
    switch (dt) {
        case GF_U8: return CU_TENSOR_MAP_DATA_TYPE_UINT8;
        case GF_U16: return CU_TENSOR_MAP_DATA_TYPE_UINT16;
        case GF_F32: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        case GF_BF16: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        default: return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    }
}

int round_up(int a, int b) { return (a + b - 1) / b * b; }

int g_max_smem = 0;
int g_sm_smem = 0;      // shared memory per SM
int g_reserved = 0;     // shared memory the runtime reserves per CTA
int g_sms = 0;
int* g_status_ptr = nullptr;
std::once_flag g_dev_once;
void query_device() {
    std::call_once(g_dev_once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&g_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&g_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (g_max_smem <= 0) g_max_smem = 227 * 1024;
        if (g_sm_smem <= 0) g_sm_smem = 228 * 1024;
        if (g_reserved < 0) g_reserved = 1024;
        if (g_sms <= 0) g_sms = 148;
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_device_status) == cudaSuccess) g_status_ptr = static_cast<int*>(p);
    });
}

// Element columns the block is laid out for.
int tw_class(int TW, int C) { return (void)C, TW <= 64 ? 64 : 256; }

// Lane chunk (multiple of 12 with an odd number of 4-element vectors, so the
// lanes' vector accesses fall in distinct banks) covering `need` staged elements.
int chunk_for(int need) {
    int m = 12;
    while (32 * m < need) m += 24;
    return m;
}

// Fills the plan-dependent part of KParams; returns the dynamic smem bytes.
size_t layout(KParams& kp, const Image& im, const BoxKernel& bk, int TWp, bool tma) {
    const int isz = dtype_size(im.in_dt);
    const int C = im.C;
    kp.TWp = TWp;
    kp.TW = TWp * C;
    const int twmax = tw_class(kp.TW, C);
    kp.ealign = 16 / isz;
    // staged elements: from the aligned start below pixel x0 - rk - 1 to pixel x0 + TWp + rk
    const int span = (TWp + 2 * bk.rk + 1) * C + kp.ealign - 1;
    // worst-case staged index of output element 0, and the scan reach it needs
    const int sout_max = (bk.rk + 1) * C + kp.ealign - 1;
    kp.m = chunk_for(std::max(span, sout_max + kp.TW + bk.rk * C + 1));
    kp.SP = round_up(std::max(32 * kp.m, sout_max + 32 * (twmax / 32) + bk.rk * C + 1), 4);
    kp.nbox = (span + 255) / 256;
    kp.boxw = round_up((span + kp.nbox - 1) / kp.nbox, 128 / isz);
    kp.SROW = round_up(std::max(kp.nbox * kp.boxw, 32 * kp.m), 128 / isz);
    const bool in_place = im.in_dt == GF_F32;   // running sums overwrite the staged f32 row
    if (in_place) kp.SROW = round_up(std::max(kp.SROW, kp.SP), 32);
    kp.NB = (2 * bk.rk + 1 + kBand + kBand - 1) / kBand;   // live rows 2 rk + 1 + kBand
    kp.RT = (kp.NB + 1) * kBand;
    const bool tm = (twmax == 256);   // wide strips keep the column ring in TMEM
    kp.tmem_cols = 0;
    if (tm) {
        int a = 32;
        while (a < 2 * kp.RT) a <<= 1;
        if (a > 512) return (size_t)1 << 40;   // ring does not fit TMEM: use a narrow strip
        kp.tmem_cols = a;
    }
    kp.nstage = tma ? (isz >= 4 ? 2 : kStages) : 1;
    if (tma && getenv("GF_STAGES")) kp.nstage = std::max(1, std::min(kMaxStages, atoi(getenv("GF_STAGES"))));
    kp.use_tma = tma ? 1 : 0;
    size_t off = 0;
    kp.off_stage = (int)off;
    off += (size_t)kp.nstage * kBand * kp.SROW * isz;
    off = (off + 127) / 128 * 128;
    kp.off_p = (int)off;
    if (!in_place) off += (size_t)kWarps * kp.SP * 4;
    off = (off + 127) / 128 * 128;
    kp.off_rband = (int)off;
    off += (size_t)2 * kBand * twmax * 4;
    kp.off_ring = (int)off;
    if (!tm) off += (size_t)(kp.NB + 1) * kBand * twmax * 4;
    off = (off + 15) / 16 * 16;
    kp.off_bar = (int)off;
    off += (size_t)kMaxStages * 8;
    kp.off_tmem = (int)off;
    off += 16;
    return off;
}

// CTAs of `smem` bytes that fit one SM by shared memory and by TMEM.
int ctas_per_sm(size_t smem, int tmem_cols) {
    int n = (int)(g_sm_smem / (smem + (size_t)g_reserved));
    n = std::min(n, 2048 / kThreads);
    if (tmem_cols > 0) n = std::min(n, 512 / tmem_cols);
    return std::max(n, 0);
}

// Pads `smem` so that shared memory admits no more CTAs per SM than TMEM does
// (a CTA must never wait inside the TMEM allocator).
size_t pad_for_tmem(size_t smem, int tmem_cols) {
    if (tmem_cols <= 0) return smem;
    const int n = 512 / tmem_cols;
    const size_t need = (size_t)g_sm_smem / (size_t)(n + 1) - (size_t)g_reserved + 16;
    return std::max(smem, (need + 15) / 16 * 16);
}

}  // namespace

int device_sm_count() {
    query_device();
    return g_sms;
}

StripPlan default_plan(const Image& im, const BoxKernel& bk) {
    query_device();
    StripPlan pl;
    // widest strip whose working set leaves room for two CTAs per SM, else one;
    // TWp even so that output columns pair up.
    const int twp_max = std::max(1, std::min(256 / im.C, im.W));
    KParams kp{};
    const size_t two = (size_t)g_max_smem / 2 - 1024;   // budget for two CTAs per SM
    int best = 0;
    for (int t = twp_max; t >= 1; --t) {
        if (t > 2 && (t & 1)) continue;
        if (layout(kp, im, bk, t, true) <= two) { best = t; break; }
    }
    if (!best) {
        for (int t = std::min(twp_max, std::max(1, 64 / im.C)); t >= 1; --t) {
            if (layout(kp, im, bk, t, true) <= (size_t)g_max_smem) { best = t; break; }
        }
    }
    pl.TWp = std::max(best, 1);
    pl.nstrips = (im.W + pl.TWp - 1) / pl.TWp;
    // rows per CTA: enough CTAs for the resident slots, keeping the vertical
    // halo (2 rk rows recomputed per CTA) small against the tile height.
    const size_t smem = layout(kp, im, bk, pl.TWp, true);
    const int per_sm = std::max(1, ctas_per_sm(pad_for_tmem(smem, kp.tmem_cols), kp.tmem_cols));
    const int target = per_sm * g_sms;
    const int tiles_y = std::max(1, target / pl.nstrips);
    int rows = (im.H + tiles_y - 1) / tiles_y;
    rows = std::max(rows, std::min(im.H, std::max(32, 4 * bk.rk)));
    pl.TH = std::max(1, std::min(rows, im.H));
    pl.nrowtiles = (im.H + pl.TH - 1) / pl.TH;
    return pl;
}

gf_status launch_filter(const Image& im, const BoxKernel& bk, const StripPlan* plan_in, void* stream) {
    query_device();
    const StripPlan pl = plan_in ? *plan_in : default_plan(im, bk);
    if (pl.TWp < 1 || pl.TH < 1 || pl.TWp * im.C > 256) return GF_EINVAL;
    KParams kp{};
    kp.in = static_cast<const unsigned char*>(im.in);
    kp.in_pitch = (long long)im.in_pitch;
    kp.out = static_cast<unsigned char*>(im.out);
    kp.out_pitch = (long long)im.out_pitch;
    kp.status = g_status_ptr;
    kp.H = im.H;
    kp.W = im.W;
    kp.C = im.C;
    kp.boundary = im.boundary;
    kp.K = bk.K;
    for (int i = 0; i < GF_KMAX; ++i) {
        kp.r[i] = bk.r[i];
        kp.w[i] = bk.w[i];
    }
    kp.sw = bk.sw;
    kp.rk = bk.rk;
    kp.TH = pl.TH;
    const int osz = dtype_size(im.out_dt);
    // TMA needs a 16-byte aligned base and pitch and a driver entry point.
    const bool tma_ok = encode_fn() != nullptr && (reinterpret_cast<uintptr_t>(im.in) % 16 == 0) &&
                        (im.in_pitch % 16 == 0) && im.in_pitch < (1ull << 40);
    const bool tma_env = getenv("GF_NO_TMA") == nullptr;
    bool tma = tma_ok && tma_env;
    size_t smem = layout(kp, im, bk, pl.TWp, tma);
    if (smem > (size_t)g_max_smem) {
        tma = false;
        smem = layout(kp, im, bk, pl.TWp, false);
        if (smem > (size_t)g_max_smem) return GF_EUNSUPPORTED;
    }
    smem = pad_for_tmem(smem, kp.tmem_cols);
    if (smem > (size_t)g_max_smem) return GF_EUNSUPPORTED;
    kp.pair_ok = ((kp.TW & 1) == 0) && (reinterpret_cast<uintptr_t>(im.out) % (2 * osz) == 0) &&
                 (im.out_pitch % (2 * osz) == 0);
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    if (tma) {
        const cuuint64_t gdim[2] = {(cuuint64_t)im.W * im.C, (cuuint64_t)im.H};
        const cuuint64_t gstride[1] = {(cuuint64_t)im.in_pitch};
        const cuuint32_t box[2] = {(cuuint32_t)kp.boxw, 1};
        const cuuint32_t estr[2] = {1, 1};
        CUresult rc = encode_fn()(&map, tma_dtype(im.in_dt), 2, const_cast<void*>(im.in), gdim, gstride, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (rc != CUDA_SUCCESS) {
            tma = false;
            smem = layout(kp, im, bk, pl.TWp, false);
        }
    }
    dim3 grid(pl.nstrips ? pl.nstrips : (im.W + pl.TWp - 1) / pl.TWp,
              pl.nrowtiles ? pl.nrowtiles : (im.H + pl.TH - 1) / pl.TH);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int twmax = tw_class(kp.TW, im.C);
    switch (im.in_dt) {
        case GF_U8:
            if (im.out_dt != GF_F32) return GF_EUNSUPPORTED;
            return launch_strip<uint8_t, float>(kp, map, grid, smem, s, twmax);
        case GF_U16:
            if (im.out_dt != GF_F32) return GF_EUNSUPPORTED;
            return launch_strip<uint16_t, float>(kp, map, grid, smem, s, twmax);
        case GF_F32:
            if (im.out_dt == GF_F32) return launch_strip<float, float>(kp, map, grid, smem, s, twmax);
            if (im.out_dt == GF_BF16) return launch_strip<float, __nv_bfloat16>(kp, map, grid, smem, s, twmax);
            return launch_strip<float, __half>(kp, map, grid, smem, s, twmax);
        case GF_BF16:
            if (im.out_dt == GF_F32) return launch_strip<__nv_bfloat16, float>(kp, map, grid, smem, s, twmax);
            if (im.out_dt == GF_BF16) return launch_strip<__nv_bfloat16, __nv_bfloat16>(kp, map, grid, smem, s, twmax);
            return launch_strip<__nv_bfloat16, __half>(kp, map, grid, smem, s, twmax);
        case GF_F16:
            if (im.out_dt == GF_F32) return launch_strip<__half, float>(kp, map, grid, smem, s, twmax);
            if (im.out_dt == GF_BF16) return launch_strip<__half, __nv_bfloat16>(kp, map, grid, smem, s, twmax);
            return launch_strip<__half, __half>(kp, map, grid, smem, s, twmax);
        default: return GF_EUNSUPPORTED;
    }
}

gf_status launch_row_box_sums(const void* in, size_t in_pitch, int32_t* out, size_t out_pitch, size_t plane_stride,
                              int H, int W, int C, int in_dt, const BoxKernel& bk, int boundary, void* stream) {
    query_device();
    const int isz = dtype_size(in_dt);
    const int rk = bk.rk;
    int TWp = std::min(W, 512 / C);
    int m = 0, SP = 0, SROW = 0;
    auto smem_for = [&](int twp) {
        const int sout_max = (rk + 1) * C + 3;
        const int span = (twp + 2 * rk + 1) * C + 3;
        m = chunk_for(std::max(span, sout_max + twp * C + rk * C + 1));
        SP = round_up(32 * m, 4);
        SROW = round_up(32 * m, 16);
        return (((size_t)kWarps * SROW * isz + 127) & ~size_t(127)) + (size_t)kWarps * SP * 4;
    };
    while (TWp > 1 && smem_for(TWp) > (size_t)g_max_smem) TWp /= 2;
    const size_t smem = smem_for(TWp);
    if (smem > (size_t)g_max_smem) return GF_EUNSUPPORTED;
    const int nstrips = (W + TWp - 1) / TWp;
    const int ny = std::max(1, std::min((H + kWarps - 1) / kWarps, 4 * g_sms / std::max(1, nstrips) + 1));
    dim3 grid(nstrips, ny);
    const int4 r03 = make_int4(bk.r[0], bk.r[1], bk.r[2], bk.r[3]);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned char* src = static_cast<const unsigned char*>(in);
    if (in_dt == GF_U8)
        return launch_box_sums<uint8_t>(src, (long long)in_pitch, out, (long long)out_pitch, (long long)plane_stride, H,
                                        W, C, bk.K, r03, bk.r[4], rk, TWp, m, SP, SROW, boundary, grid, smem, s);
    if (in_dt == GF_U16)
        return launch_box_sums<uint16_t>(src, (long long)in_pitch, out, (long long)out_pitch, (long long)plane_stride,
                                         H, W, C, bk.K, r03, bk.r[4], rk, TWp, m, SP, SROW, boundary, grid, smem, s);
    return GF_EUNSUPPORTED;
}

gf_status read_device_status(int clear, int* value) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_device_status, sizeof(int)) != cudaSuccess) return GF_ECUDA;
    if (clear) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_device_status, &z, sizeof(int)) != cudaSuccess) return GF_ECUDA;
    }
    if (value) *value = v;
    return GF_OK;
}

}  // namespace gb
