// Host side of the fused strip filter: tile plans, shared-memory layout, the TMA
// tensor map, and launches (the kernels are instantiated in inst_*.cu).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <string>
#include <vector>
#include <cstring>
#include <mutex>

#include "batch.h"
#include "plan.h"
#include "strip_kernel.cuh"
#include "walker.h"

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
GB_DECLARE_BATCH(uint8_t, float)
GB_DECLARE_BATCH(uint16_t, float)
GB_DECLARE_BATCH(float, float)
GB_DECLARE_BATCH(float, __nv_bfloat16)
GB_DECLARE_BATCH(float, __half)
GB_DECLARE_BATCH(__nv_bfloat16, float)
GB_DECLARE_BATCH(__nv_bfloat16, __nv_bfloat16)
GB_DECLARE_BATCH(__nv_bfloat16, __half)
GB_DECLARE_BATCH(__half, float)
GB_DECLARE_BATCH(__half, __nv_bfloat16)
GB_DECLARE_BATCH(__half, __half)
GB_DECLARE_ROWPASS(uint8_t)
GB_DECLARE_ROWPASS(uint16_t)
GB_DECLARE_ROWPASS(float)
GB_DECLARE_ROWPASS(__nv_bfloat16)
GB_DECLARE_ROWPASS(__half)
GB_DECLARE_COLPASS(float)
GB_DECLARE_COLPASS(__nv_bfloat16)
GB_DECLARE_COLPASS(__half)

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

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

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

namespace {

// Limits and the status-word address of each device, looked up the first time
// the library works on that device (with it current) and kept for the process.
constexpr int kMaxDevices = 64;
DeviceInfo g_info[kMaxDevices];
bool g_info_ok[kMaxDevices] = {};
std::mutex g_info_mu;
const DeviceInfo g_no_device{};   // no current device, or an ordinal beyond the table

}  // namespace

namespace {
thread_local LaunchCtx t_launch_ctx;
}  // namespace

LaunchCtx& launch_ctx() { return t_launch_ctx; }
int* launch_status_word() { return t_launch_ctx.status ? t_launch_ctx.status : device_info().status; }
long long launch_wait_limit() { return t_launch_ctx.wait > 0 ? t_launch_ctx.wait : kWaitCycles; }

const DeviceInfo& device_info() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return g_no_device;
    std::lock_guard<std::mutex> lk(g_info_mu);
    DeviceInfo& info = g_info[dev];
    if (!g_info_ok[dev]) {
        cudaDeviceGetAttribute(&info.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&info.sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&info.reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (info.max_smem <= 0) info.max_smem = 227 * 1024;
        if (info.sm_smem <= 0) info.sm_smem = 228 * 1024;
        if (info.reserved < 0) info.reserved = 1024;
        if (info.sms <= 0) info.sms = 148;
        void* p = nullptr;
        // the device copy of the library's status word on this device
        if (cudaGetSymbolAddress(&p, g_device_status) == cudaSuccess) info.status = static_cast<int*>(p);
        info.device = dev;
        g_info_ok[dev] = true;
    }
    return info;
}

namespace {

// Element columns the block is laid out for.
int tw_class(int TW, int C) { return (void)C, TW <= 64 ? 64 : 256; }

}  // namespace

// Lane chunk (multiple of 12 with an odd number of 4-element vectors, so the
// lanes' vector accesses fall in distinct banks) covering `need` staged elements.
int chunk_for(int need) {
    int m = 12;
    while (32 * m < need) m += 24;
    return m;
}

namespace {

}  // namespace

void staging_geometry(KParams& kp, int span, int min_row, int srow_mult, int isz, bool wide) {
    kp.rows8 = 0;
    if (wide) {
        // every box and staged row starts on a 128-byte boundary of shared memory
        const int maxe = 2048 / isz;   // 256 eight-byte TMA elements per box row
        kp.nbox = (span + maxe - 1) / maxe;
        kp.boxw = round_up((span + kp.nbox - 1) / kp.nbox, 128 / isz);
        kp.SROW = round_up(std::max(kp.nbox * kp.boxw, min_row), std::max(srow_mult, 128 / isz));
        kp.xshift = isz == 1 ? 3 : (isz == 2 ? 2 : 1);
        if (kp.nbox == 1 && kp.SROW * isz <= 2048) {
            kp.boxw = kp.SROW;   // rows of the box are dense at the row stride
            kp.rows8 = 1;
        }
    } else {
        kp.nbox = (span + 255) / 256;
        kp.boxw = round_up((span + kp.nbox - 1) / kp.nbox, 128 / isz);
        kp.SROW = round_up(std::max(kp.nbox * kp.boxw, min_row), std::max(srow_mult, 128 / isz));
        kp.xshift = 0;
    }
}

bool encode_row_maps(const KParams& kp, const void* base, size_t pitch, int rowlen, int H, int in_dt,
                     CUtensorMap* maps) {
    std::memset(maps, 0, 2 * sizeof(CUtensorMap));
    const auto enc = encode_fn();
    if (!enc) return false;
    const int isz = dtype_size(in_dt);
    const bool wide = kp.xshift > 0;
    const cuuint64_t gdim[2] = {(cuuint64_t)(wide ? (size_t)rowlen * isz / 8 : (size_t)rowlen), (cuuint64_t)H};
    const cuuint64_t gstride[1] = {(cuuint64_t)pitch};
    const cuuint32_t bw = (cuuint32_t)(wide ? kp.boxw * isz / 8 : kp.boxw);
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = wide ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : tma_dtype(in_dt);
    const cuuint32_t box1[2] = {bw, 1};
    if (enc(&maps[0], dt, 2, const_cast<void*>(base), gdim, gstride, box1, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (kp.rows8) {
        const cuuint32_t box8[2] = {bw, (cuuint32_t)kBand};
        if (enc(&maps[1], dt, 2, const_cast<void*>(base), gdim, gstride, box8, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

namespace {

// TMA through 8-byte elements needs rows whose byte length is a multiple of 8.
bool wide_ok(const Image& im) { return ((size_t)im.W * im.C * dtype_size(im.in_dt)) % 8 == 0; }

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
    const bool in_place = im.in_dt == GF_F32;   // running sums overwrite the staged f32 row
    staging_geometry(kp, span, in_place ? std::max(32 * kp.m, kp.SP) : 32 * kp.m, in_place ? 32 : 1, isz,
                     tma && wide_ok(im));
    kp.NB = (2 * bk.rk + 1 + kBand + kBand - 1) / kBand;   // live rows 2 rk + 1 + kBand
    kp.RT = (kp.NB + 1) * kBand;
    const bool tm = (twmax == 256);   // wide strips keep the column ring in TMEM
    kp.tmem_cols = 0;
    if (tm) {
        // two warpgroups, each with a hi ring and a lo ring of RT columns
        int a = 32;
        while (a < 4 * kp.RT) a <<= 1;
        if (a > 512) return (size_t)1 << 40;   // ring does not fit TMEM: use a narrow strip
        kp.tmem_cols = a;
    }
    kp.nstage = tma ? (isz >= 4 ? 2 : kStages) : 1;
    kp.use_tma = tma ? 1 : 0;
    size_t off = 0;
    kp.off_stage = (int)off;
    off += (size_t)kp.nstage * kBand * kp.SROW * isz;
    off = (off + 127) / 128 * 128;
    kp.off_p = (int)off;
    if (!in_place) off += (size_t)kWarps * kp.SP * 4;
    off = (off + 127) / 128 * 128;
    kp.off_pl = (int)off;   // float rows: the residue sums (row_prefix)
    if (!dtype_is_int(im.in_dt)) off += (size_t)kWarps * kp.SP * 4;
    off = (off + 127) / 128 * 128;
    kp.off_rband = (int)off;
    off += (size_t)2 * kBand * twmax * 4;
    kp.off_ring = (int)off;
    if (!tm) off += (size_t)2 * (kp.NB + 1) * kBand * twmax * 4;   // hi ring, then lo ring
    // whole output bands leave by TMA store when the output allows 16-byte boxes
    const int osz = dtype_size(im.out_dt);
    kp.tma_store = (tma && reinterpret_cast<uintptr_t>(im.out) % 16 == 0 && im.out_pitch % 16 == 0 &&
                    ((size_t)kp.TW * osz) % 16 == 0 && kp.TW <= 256)
                       ? 1
                       : 0;
    off = (off + 127) / 128 * 128;
    kp.off_obuf = (int)off;
    if (kp.tma_store) off += (size_t)kBand * kp.TW * osz;
    off = (off + 15) / 16 * 16;
    kp.off_bar = (int)off;
    off += (size_t)kMaxStages * 8;
    kp.off_tmem = (int)off;
    off += 16;
    return off;
}

}  // namespace

// CTAs of `smem` bytes that fit one SM by shared memory and by TMEM.
int ctas_per_sm(size_t smem, int tmem_cols) {
    const DeviceInfo& di = device_info();
    int n = (int)(di.sm_smem / (smem + (size_t)di.reserved));
    n = std::min(n, 2048 / kThreads);
    if (tmem_cols > 0) n = std::min(n, 512 / tmem_cols);
    return std::max(n, 0);
}

// Pads `smem` so that shared memory admits no more CTAs per SM than TMEM does
// (a CTA must never wait inside the TMEM allocator).
size_t pad_for_tmem(size_t smem, int tmem_cols) {
    if (tmem_cols <= 0) return smem;
    const int n = 512 / tmem_cols;
    const DeviceInfo& di = device_info();
    const size_t need = (size_t)di.sm_smem / (size_t)(n + 1) - (size_t)di.reserved + 16;
    return std::max(smem, (need + 15) / 16 * 16);
}

int device_sm_count() { return device_info().sms; }

StripPlan default_plan(const Image& im, const BoxKernel& bk) {
    const DeviceInfo& di = device_info();
    StripPlan pl;
    // widest strip whose working set leaves room for two CTAs per SM, else one;
    // TWp even so that output columns pair up.
    const int twp_max = std::max(1, std::min(256 / im.C, im.W));
    KParams kp{};
    const size_t two = (size_t)di.max_smem / 2 - 1024;   // budget for two CTAs per SM
    int best = 0;
    for (int t = twp_max; t >= 1; --t) {
        if (t > 2 && (t & 1)) continue;
        if (layout(kp, im, bk, t, true) <= two) { best = t; break; }
    }
    if (!best) {
        for (int t = std::min(twp_max, std::max(1, 64 / im.C)); t >= 1; --t) {
            if (layout(kp, im, bk, t, true) <= (size_t)di.max_smem) { best = t; break; }
        }
    }
    pl.TWp = std::max(best, 1);
    pl.nstrips = (im.W + pl.TWp - 1) / pl.TWp;
    // rows per CTA: enough CTAs for the resident slots, keeping the vertical
    // halo (2 rk rows recomputed per CTA) small against the tile height.
    const size_t smem = layout(kp, im, bk, pl.TWp, true);
    const int per_sm = std::max(1, ctas_per_sm(pad_for_tmem(smem, kp.tmem_cols), kp.tmem_cols));
    const int target = per_sm * di.sms;
    const int tiles_y = std::max(1, target / pl.nstrips);
    int rows = (im.H + tiles_y - 1) / tiles_y;
    rows = std::max(rows, std::min(im.H, std::max(32, 4 * bk.rk)));
    // the column sums are exact to their own magnitude at any tile height; only
    // the grid's y limit bounds the number of row tiles
    rows = std::max(rows, (im.H + 65534) / 65535);
    pl.TH = std::max(1, std::min(rows, im.H));
    pl.nrowtiles = (im.H + pl.TH - 1) / pl.TH;
    return pl;
}

namespace {

gf_status prepare(const Image& im, const BoxKernel& bk, const StripPlan* plan_in, Prepared& out) {
    const DeviceInfo& di = device_info();
    if (!di.status) return GF_EUNSUPPORTED;
    if (is_sampled(im)) return GF_EUNSUPPORTED;   // the fused kernel stores every pixel
    const StripPlan pl = plan_in ? *plan_in : default_plan(im, bk);
    if (pl.TWp < 1 || pl.TH < 1 || pl.TWp * im.C > 256) return GF_EINVAL;
    KParams& kp = out.kp;
    kp = KParams{};
    kp.in = static_cast<const unsigned char*>(im.in);
    kp.in_pitch = (long long)im.in_pitch;
    kp.out = static_cast<unsigned char*>(im.out);
    kp.out_pitch = (long long)im.out_pitch;
    kp.status = launch_status_word();
    kp.wait_limit = launch_wait_limit();
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
    // TMA needs a 16-byte aligned base and pitch and a driver entry point.
    const bool tma_ok = encode_fn() != nullptr && (reinterpret_cast<uintptr_t>(im.in) % 16 == 0) &&
                        (im.in_pitch % 16 == 0) && im.in_pitch < (1ull << 40);
    // GF_NO_TMA (any value) forces the plain loaders: the staging-path parity test
    const bool tma_env = getenv("GF_NO_TMA") == nullptr;
    bool tma = tma_ok && tma_env;
    size_t smem = layout(kp, im, bk, pl.TWp, tma);
    if (smem > (size_t)di.max_smem) {
        tma = false;
        smem = layout(kp, im, bk, pl.TWp, false);
        if (smem > (size_t)di.max_smem) return GF_EUNSUPPORTED;
    }
    std::memset(out.maps, 0, sizeof(out.maps));
    if (tma && !encode_row_maps(kp, im.in, im.in_pitch, im.W * im.C, im.H, im.in_dt, out.maps)) {
        tma = false;
        smem = layout(kp, im, bk, pl.TWp, false);
    }
    if (kp.tma_store) {
        const cuuint64_t gdim[2] = {(cuuint64_t)im.W * im.C, (cuuint64_t)im.H};
        const cuuint64_t gstride[1] = {(cuuint64_t)im.out_pitch};
        const cuuint32_t box[2] = {(cuuint32_t)kp.TW, (cuuint32_t)kBand};
        const cuuint32_t estr[2] = {1, 1};
        if (encode_fn()(&out.maps[2], tma_dtype(im.out_dt), 2, im.out, gdim, gstride, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            kp.tma_store = 0;
    }
    out.smem = smem;
    out.twmax = tw_class(kp.TW, im.C);
    out.grid = dim3(pl.nstrips ? pl.nstrips : (im.W + pl.TWp - 1) / pl.TWp,
                    pl.nrowtiles ? pl.nrowtiles : (im.H + pl.TH - 1) / pl.TH);
    out.ntiles = (int)(out.grid.x * out.grid.y);
    return GF_OK;
}

// Launch class of a batch image: the kernel instantiation (dtypes, channels,
// strip layout) and its on-chip footprint (TMEM columns, CTAs per SM), so that
// an image with a wide column ring does not lower the occupancy of the rest.
int class_key(const Image& im, const Prepared& pr) {
    int tm = 0;
    while (tm < 6 && (pr.kp.tmem_cols >> tm) > 16) ++tm;   // 0 (SMEM ring), 1..5 for 32..512 columns
    const int per_sm = std::min(7, ctas_per_sm(pad_for_tmem(pr.smem + sizeof(KParams) + 32, pr.kp.tmem_cols),
                                               pr.kp.tmem_cols));
    return (((((im.in_dt * 8 + im.out_dt) * 8 + im.C) * 2 + (pr.twmax == 64)) * 8 + tm) * 8) + per_sm;
}

gf_status dispatch_batch(int in_dt, int out_dt, const BatchArgs& ba, int C, int twmax, int grid, size_t smem,
                         cudaStream_t s) {
    switch (in_dt) {
        case GF_U8: return launch_batch<uint8_t, float>(ba, C, twmax, grid, smem, s);
        case GF_U16: return launch_batch<uint16_t, float>(ba, C, twmax, grid, smem, s);
        case GF_F32:
            if (out_dt == GF_F32) return launch_batch<float, float>(ba, C, twmax, grid, smem, s);
            if (out_dt == GF_BF16) return launch_batch<float, __nv_bfloat16>(ba, C, twmax, grid, smem, s);
            return launch_batch<float, __half>(ba, C, twmax, grid, smem, s);
        case GF_BF16:
            if (out_dt == GF_F32) return launch_batch<__nv_bfloat16, float>(ba, C, twmax, grid, smem, s);
            if (out_dt == GF_BF16) return launch_batch<__nv_bfloat16, __nv_bfloat16>(ba, C, twmax, grid, smem, s);
            return launch_batch<__nv_bfloat16, __half>(ba, C, twmax, grid, smem, s);
        case GF_F16:
            if (out_dt == GF_F32) return launch_batch<__half, float>(ba, C, twmax, grid, smem, s);
            if (out_dt == GF_BF16) return launch_batch<__half, __nv_bfloat16>(ba, C, twmax, grid, smem, s);
            return launch_batch<__half, __half>(ba, C, twmax, grid, smem, s);
        default: return GF_EUNSUPPORTED;
    }
}

}  // namespace

gf_status launch_fused(const Image& im, const BoxKernel& bk, const StripPlan* plan_in, void* stream) {
    Prepared pr;
    gf_status st = prepare(im, bk, plan_in, pr);
    if (st != GF_OK) return st;
    return launch_prepared(im, pr, stream);
}

gf_status prepare_fused(const Image& im, const BoxKernel& bk, const StripPlan* plan, Prepared& out) {
    return prepare(im, bk, plan, out);
}

gf_status launch_prepared(const Image& im, Prepared pr, void* stream, int ty0, int ty1) {
    KParams& kp = pr.kp;
    if (pr.grid.y > 65535u) return GF_EINVAL;   // grid y limit: a plan with fewer, taller row tiles fits
    if (ty1 >= 0) {   // the slab of row tiles [ty0, ty1)
        if (ty0 < 0 || ty1 <= ty0 || ty1 > (int)pr.grid.y) return GF_EINVAL;
        kp.tile_y0 = ty0;
        pr.grid.y = (unsigned)(ty1 - ty0);
    }
    size_t smem = pad_for_tmem(pr.smem, kp.tmem_cols);
    if (smem > (size_t)device_info().max_smem) return GF_EUNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int twmax = pr.twmax;
    const dim3 grid = pr.grid;
    const CUtensorMap* map = pr.maps;
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

bool fused_fits(const Image& im, const BoxKernel& bk, int TWp) {
    KParams kp{};
    return layout(kp, im, bk, TWp, false) <= (size_t)device_info().max_smem;
}

int fused_ctas_per_sm(const Image& im, const BoxKernel& bk, int TWp) {
    KParams kp{};
    const size_t smem = layout(kp, im, bk, TWp, true);
    if (smem > (size_t)device_info().max_smem) return 0;
    return ctas_per_sm(pad_for_tmem(smem, kp.tmem_cols), kp.tmem_cols);
}

namespace {

// Two-pass images of the default accumulation go into batched launches,
// classed by (input type, channels, CTAs per SM of the row pass; output type,
// strip width, band rows, CTAs per SM of the column pass), at most
// kTPBatchMax images a class: each class is a row launch and a column launch
// sized for its largest member, and classes are independent of one another
// (they may run on different streams).  An image in a study accumulation mode
// keeps its own two launches.  Extends the staging block by the batched
// images' tensor maps: [2 row maps x nb][2 column maps x nb].
gf_status plan_twopass_classes(BatchWork& w) {
    w.tp_order.clear();
    w.tp_solo.clear();
    w.tp_cls.clear();
    if (w.ntp == 0) return GF_OK;
    std::vector<long long> key(w.ntp, 0);
    for (int t = 0; t < w.ntp; ++t) {
        const TwoPass& tp = w.tp[t];
        if (tp.plan.accum != GF_ACCUM_COMPENSATED || tp.grid_c.z > 1) {
            w.tp_solo.push_back(t);
            continue;
        }
        // 3 bits type, 3 bits channels / strip width code, 1 bit band, 4 bits CTAs per SM
        const int cw_code = tp.CW == 32 ? 0 : tp.CW == 64 ? 1 : tp.CW == 128 ? 2 : 3;
        const long long row_key = (tp.in_dt << 7) | (tp.kp.C << 4) | std::min(15, ctas_per_sm(tp.smem_r, 0));
        const long long col_key = (tp.out_dt << 8) | (cw_code << 5) | ((tp.cp.B == 32 ? 1 : 0) << 4) |
                                  std::min(15, ctas_per_sm(tp.smem_c, 0));
        key[t] = (row_key << 16) | col_key;
        w.tp_order.push_back(t);
    }
    const int nb = (int)w.tp_order.size();
    if (nb == 0) return GF_OK;
    std::stable_sort(w.tp_order.begin(), w.tp_order.end(), [&](int a, int b) { return key[a] < key[b]; });
    for (int k = 0; k < nb; ++k) {
        const TwoPass& tp = w.tp[w.tp_order[k]];
        if (w.tp_cls.empty() || w.tp_cls.back().key != key[w.tp_order[k]] || w.tp_cls.back().count == kTPBatchMax) {
            TPClass c;
            c.first = k;
            c.key = key[w.tp_order[k]];
            c.in_dt = tp.in_dt;
            c.out_dt = tp.out_dt;
            c.C = tp.kp.C;
            c.CW = tp.CW;
            c.B = tp.cp.B;
            w.tp_cls.push_back(c);
        }
        TPClass& c = w.tp_cls.back();
        c.count++;
        c.smem_r = std::max(c.smem_r, tp.smem_r);
        c.smem_c = std::max(c.smem_c, tp.smem_c);
        c.tiles_r += (int)(tp.grid_r.x * tp.grid_r.y);
        c.tiles_c += (int)(tp.grid_c.x * tp.grid_c.y);
    }
    w.o_tpmr = w.total;
    w.o_tpmc = w.o_tpmr + (size_t)2 * nb * sizeof(CUtensorMap);
    w.total = (w.o_tpmc + (size_t)2 * nb * sizeof(CUtensorMap) + 255) / 256 * 256;
    return GF_OK;
}

}  // namespace

gf_status batch_plan(const Image* ims, const BoxKernel* bks, int n, BatchWork& w) {
    w.ncls = 0;
    w.nfused = 0;
    w.ntp = 0;
    w.nwk = 0;
    w.inter_total = 0;
    w.ims = ims;
    w.bks = bks;
    if (n <= 0) return GF_OK;
    const bool two_ok = w.tp != nullptr && w.tp_off != nullptr;
    for (int i = 0; i < n; ++i) {
        FilterPlan fp;
        gf_status st = resolve_plan(ims[i], bks[i], &ims[i].plan, fp);
        if (st != GF_OK) return st;
        if (fp.path == GF_PATH_HBM) return GF_EUNSUPPORTED;   // single-image calls only
        if (fp.path == GF_PATH_WALK) {
            // the register walk: its own launch, like a two-pass image (the
            // kernel is compiled and loaded here, before any capture); callers
            // without such launches run the image fused
            if (w.wk_img && walker_prepare(ims[i], bks[i]) == GF_OK) {
                w.wk_img[w.nwk++] = i;
                continue;
            }
            if (ims[i].plan.path == GF_PATH_WALK) return GF_EUNSUPPORTED;
            fp.path = GF_PATH_FUSED;
        }
        if (fp.path == GF_PATH_TWO_PASS && !two_ok) {
            // without intermediates only the fused kernel runs: an explicit
            // two-pass plan, or an accumulation mode that exists on the
            // two-pass path only, cannot be honoured
            if (ims[i].plan.path == GF_PATH_TWO_PASS || ims[i].plan.accum != GF_ACCUM_COMPENSATED)
                return GF_EUNSUPPORTED;
            fp.path = GF_PATH_FUSED;   // default tile plan of the fused kernel
        }
        if (fp.path == GF_PATH_TWO_PASS) {
            st = prepare_twopass(ims[i], bks[i], fp.two, w.tp[w.ntp]);
            if (st != GF_OK) return st;
            w.tp_off[w.ntp] = w.inter_total;
            if (w.tp_img) w.tp_img[w.ntp] = i;
            w.inter_total += (w.tp[w.ntp].r_bytes + 255) / 256 * 256;
            w.ntp++;
        } else {
            st = prepare(ims[i], bks[i], &fp.strip, w.pr[i]);
            if (st != GF_OK) return st;
            w.order[w.nfused++] = i;
        }
    }
    // group the fused images by class, keeping the callers' order inside a class
    Prepared* pr = w.pr;
    const int nf = w.nfused;
    std::sort(w.order, w.order + nf, [&](int a, int b) {
        const int ka = class_key(ims[a], pr[a]), kb = class_key(ims[b], pr[b]);
        return ka != kb ? ka < kb : a < b;
    });
    for (int k = 0; k < nf; ++k) {
        const int i = w.order[k];
        const int key = class_key(ims[i], pr[i]);
        if (w.ncls == 0 || w.cls[w.ncls - 1].key != key) {
            BatchClass c{};
            c.first = k;
            c.key = key;
            c.twmax = pr[i].twmax;
            c.in_dt = ims[i].in_dt;
            c.out_dt = ims[i].out_dt;
            c.C = ims[i].C;
            w.cls[w.ncls++] = c;
        }
        w.cls[w.ncls - 1].count++;
    }
    // class-wide shared-memory layout: each region sized for its largest image
    for (int ci = 0; ci < w.ncls; ++ci) {
        BatchClass& c = w.cls[ci];
        size_t st_b = 0, p_b = 0, pl_b = 0, ring_b = 0, ob_b = 0;
        int tcols = 0, nst = 1;
        for (int k = c.first; k < c.first + c.count; ++k) {
            const KParams& kp = pr[w.order[k]].kp;
            const Image& im = ims[w.order[k]];
            st_b = std::max(st_b, (size_t)kp.nstage * kBand * kp.SROW * dtype_size(im.in_dt));
            if (im.in_dt != GF_F32) p_b = std::max(p_b, (size_t)kWarps * kp.SP * 4);
            if (!dtype_is_int(im.in_dt)) pl_b = std::max(pl_b, (size_t)kWarps * kp.SP * 4);
            if (c.twmax == 64) ring_b = std::max(ring_b, (size_t)2 * (kp.NB + 1) * kBand * 64 * 4);
            if (kp.tma_store) ob_b = std::max(ob_b, (size_t)kBand * kp.TW * dtype_size(im.out_dt));
            tcols = std::max(tcols, kp.tmem_cols);
            nst = std::max(nst, kp.nstage);
        }
        size_t off = 0;
        const int o_stage = 0;
        off += st_b;
        off = (off + 127) / 128 * 128;
        const int o_p = (int)off;
        off += p_b;
        off = (off + 127) / 128 * 128;
        const int o_pl = (int)off;
        off += pl_b;
        off = (off + 127) / 128 * 128;
        const int o_rb = (int)off;
        off += (size_t)2 * kBand * c.twmax * 4;
        const int o_ring = (int)off;
        off += ring_b;
        off = (off + 127) / 128 * 128;
        const int o_ob = (int)off;
        off += ob_b;
        off = (off + 15) / 16 * 16;
        const int o_bar = (int)off;
        off += (size_t)kMaxStages * 8;
        const int o_tm = (int)off;
        off += 16;
        const int o_kp = (int)off;
        off += sizeof(KParams) + 16;
        off = (off + 15) / 16 * 16;
        c.smem = pad_for_tmem(off, tcols);
        if (c.smem > (size_t)device_info().max_smem) return GF_EUNSUPPORTED;
        c.tmem_cols = tcols;
        c.nstage = nst;
        c.ntiles = 0;
        for (int k = c.first; k < c.first + c.count; ++k) {
            KParams& kp = pr[w.order[k]].kp;
            kp.off_stage = o_stage;
            kp.off_p = o_p;
            kp.off_pl = o_pl;
            kp.off_rband = o_rb;
            kp.off_ring = o_ring;
            kp.off_obuf = o_ob;
            kp.off_bar = o_bar;
            kp.off_tmem = o_tm;
            kp.tmem_cols = tcols;
            c.ntiles += pr[w.order[k]].ntiles;
        }
        const int per_sm = std::max(1, ctas_per_sm(c.smem, tcols));
        c.grid = std::max(1, std::min(c.ntiles, per_sm * device_info().sms));
        c.ba.off_bar = o_bar;
        c.ba.off_tmem = o_tm;
        c.ba.off_kp = o_kp;
        c.ba.nstage = nst;
        c.ba.tmem_cols = tcols;
        c.ba.nimg = c.count;
        c.ba.ntiles = c.ntiles;
    }
    // staging block: [KParams x n][3 tensor maps x n][tile_start (count+1) per class][counter per class]
    const size_t nkp = (size_t)n * sizeof(KParams);
    w.o_maps = (nkp + 127) / 128 * 128;
    w.o_ts = w.o_maps + (size_t)3 * n * sizeof(CUtensorMap);
    w.o_cnt = w.o_ts + (size_t)(n + w.ncls) * sizeof(int);
    w.total = (w.o_cnt + (size_t)w.ncls * sizeof(int) + 255) / 256 * 256;
    return plan_twopass_classes(w);
}

void batch_stage(BatchWork& w, int n, unsigned char* hp, unsigned char* dp) {
    int* ts = reinterpret_cast<int*>(hp + w.o_ts);
    int ts_pos = 0;
    for (int ci = 0; ci < w.ncls; ++ci) {
        BatchClass& c = w.cls[ci];
        int acc = 0;
        c.ba.descs = reinterpret_cast<const KParams*>(dp) + c.first;
        c.ba.maps = reinterpret_cast<const CUtensorMap*>(dp + w.o_maps) + 3 * c.first;
        c.ba.tile_start = reinterpret_cast<const int*>(dp + w.o_ts) + ts_pos;
        c.ba.counter = reinterpret_cast<int*>(dp + w.o_cnt) + ci;
        for (int k = c.first; k < c.first + c.count; ++k) {
            std::memcpy(hp + (size_t)k * sizeof(KParams), &w.pr[w.order[k]].kp, sizeof(KParams));
            std::memcpy(hp + w.o_maps + (size_t)3 * k * sizeof(CUtensorMap), w.pr[w.order[k]].maps,
                        3 * sizeof(CUtensorMap));
            ts[ts_pos++] = acc;
            acc += w.pr[w.order[k]].ntiles;
        }
        ts[ts_pos++] = acc;
        reinterpret_cast<int*>(hp + w.o_cnt)[ci] = 0;   // ticket counters start at zero
    }
    (void)n;
    // batched two-pass launches: per class the images' parameters and tile
    // starts (launch parameters; the intermediates are bound by now) and their
    // tensor maps in the staging block
    for (TPClass& c : w.tp_cls) {
        c.ar.nimg = c.ac.nimg = c.count;
        c.ar.maps = reinterpret_cast<const CUtensorMap*>(dp + w.o_tpmr) + 2 * c.first;
        c.ac.maps = reinterpret_cast<const CUtensorMap*>(dp + w.o_tpmc) + 2 * c.first;
        int acc_r = 0, acc_c = 0;
        for (int j = 0; j < c.count; ++j) {
            const int k = c.first + j;
            const TwoPass& tp = w.tp[w.tp_order[k]];
            c.ar.kp[j] = tp.kp;
            c.ac.cp[j] = tp.cp;
            std::memcpy(hp + w.o_tpmr + (size_t)2 * k * sizeof(CUtensorMap), tp.maps_in, 2 * sizeof(CUtensorMap));
            std::memcpy(hp + w.o_tpmc + (size_t)2 * k * sizeof(CUtensorMap), tp.maps_r, 2 * sizeof(CUtensorMap));
            c.ar.tile_start[j] = acc_r;
            c.ac.tile_start[j] = acc_c;
            acc_r += (int)(tp.grid_r.x * tp.grid_r.y);
            acc_c += (int)(tp.grid_c.x * tp.grid_c.y);
        }
        c.ar.tile_start[c.count] = acc_r;
        c.ac.tile_start[c.count] = acc_c;
    }
}

namespace {

gf_status launch_tp_class(const TPClass& c, cudaStream_t s) {
    gf_status st;
    switch (c.in_dt) {
        case GF_U8: st = launch_row_pass_batch<uint8_t>(c.ar, c.C, c.tiles_r, c.smem_r, s); break;
        case GF_U16: st = launch_row_pass_batch<uint16_t>(c.ar, c.C, c.tiles_r, c.smem_r, s); break;
        case GF_F32: st = launch_row_pass_batch<float>(c.ar, c.C, c.tiles_r, c.smem_r, s); break;
        case GF_BF16: st = launch_row_pass_batch<__nv_bfloat16>(c.ar, c.C, c.tiles_r, c.smem_r, s); break;
        case GF_F16: st = launch_row_pass_batch<__half>(c.ar, c.C, c.tiles_r, c.smem_r, s); break;
        default: return GF_EUNSUPPORTED;
    }
    if (st != GF_OK) return st;
    switch (c.out_dt) {
        case GF_F32: return launch_col_pass_batch<float>(c.ac, c.CW, c.B, c.tiles_c, c.smem_c, s);
        case GF_BF16: return launch_col_pass_batch<__nv_bfloat16>(c.ac, c.CW, c.B, c.tiles_c, c.smem_c, s);
        case GF_F16: return launch_col_pass_batch<__half>(c.ac, c.CW, c.B, c.tiles_c, c.smem_c, s);
        default: return GF_EUNSUPPORTED;
    }
}

}  // namespace

gf_status batch_bind(BatchWork& w, unsigned char* inter_base) {
    if (w.ntp > 0 && !inter_base) return GF_EINVAL;
    for (int t = 0; t < w.ntp; ++t) {
        gf_status st = bind_twopass(w.tp[t], inter_base + w.tp_off[t]);
        if (st != GF_OK) return st;
    }
    return GF_OK;
}

gf_status batch_enqueue(const BatchWork& w, unsigned char* dp, const void* hp, cudaStream_t q, const Fork* fork) {
    const int nbt = (int)w.tp_cls.size();          // batched two-pass classes
    const int ntu = nbt + (int)w.tp_solo.size();   // two-pass units
    if ((w.ncls > 0 || nbt > 0) && cudaMemcpyAsync(dp, hp, w.total, cudaMemcpyHostToDevice, q) != cudaSuccess)
        return GF_ECUDA;
    const int units = w.ncls + ntu + w.nwk;   // fused classes, two-pass units, walk images
    const int nf = (fork && units > 1) ? std::min(fork->n, units - 1) : 0;
    if (nf > 0) {
        // classes 1.. run on side streams that start after the staging copy and
        // join `q` at the end, so one class's tail overlaps the next class
        if (cudaEventRecord(fork->ev[0], q) != cudaSuccess) return GF_ECUDA;
        for (int f = 0; f < nf; ++f)
            if (cudaStreamWaitEvent(fork->s[f], fork->ev[0], 0) != cudaSuccess) return GF_ECUDA;
    }
    // Longest unit first onto the least-loaded stream (stream 0 is q), by the
    // element count times each plan's halo factors.
    std::vector<int> sorted(units), where(units, 0);
    std::vector<double> cost(units, 0.0), load(nf + 1, 0.0);
    auto factor = [](int len, int halo, int) { return (double)(len + halo) / std::max(1, len); };
    for (int u = 0; u < units; ++u) {
        sorted[u] = u;
        if (u < w.ncls) {
            const BatchClass& c = w.cls[u];
            for (int k = c.first; k < c.first + c.count; ++k) {
                const KParams& kp = w.pr[w.order[k]].kp;
                const double el = (double)kp.H * kp.W * kp.C;
                cost[u] += el * factor(kp.TWp, 2 * kp.rk + 1, kp.TWp) * factor(kp.TH, 2 * kp.rk, kp.TH);
            }
        } else if (u < w.ncls + ntu) {
            auto tp_cost = [&](const TwoPass& t) {
                const double el = (double)t.kp.H * t.kp.W * t.kp.C;
                return el * (factor(t.kp.TWp, 2 * t.kp.rk + 1, t.kp.TWp) + factor(t.cp.TH, 2 * t.cp.rk, t.cp.TH));
            };
            if (u - w.ncls < nbt) {
                const TPClass& c = w.tp_cls[u - w.ncls];
                for (int k = c.first; k < c.first + c.count; ++k) cost[u] += tp_cost(w.tp[w.tp_order[k]]);
            } else
                cost[u] = tp_cost(w.tp[w.tp_solo[u - w.ncls - nbt]]);
        } else {
            const Image& im = w.ims[w.wk_img[u - w.ncls - ntu]];
            cost[u] = (double)im.H * im.W * im.C;
        }
    }
    std::stable_sort(sorted.begin(), sorted.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int u : sorted) {
        int best = 0;
        for (int f = 1; f <= nf; ++f)
            if (load[f] < load[best]) best = f;
        where[u] = best;
        load[best] += cost[u];
    }
    for (int u : sorted) {
        const cudaStream_t sq = where[u] == 0 ? q : fork->s[where[u] - 1];
        gf_status st;
        if (u < w.ncls) {
            const BatchClass& c = w.cls[u];
            st = dispatch_batch(c.in_dt, c.out_dt, c.ba, c.C, c.twmax, c.grid, c.smem, sq);
        } else if (u < w.ncls + ntu) {
            if (u - w.ncls < nbt) {
                st = launch_tp_class(w.tp_cls[u - w.ncls], sq);
            } else {
                st = enqueue_twopass(w.tp[w.tp_solo[u - w.ncls - nbt]], sq);
            }
        } else {
            const int i = w.wk_img[u - w.ncls - ntu];
            st = launch_walker(w.ims[i], w.bks[i], sq);
        }
        if (st != GF_OK) return st;
    }
    for (int f = 0; f < nf; ++f) {
        if (cudaEventRecord(fork->ev[1 + f], fork->s[f]) != cudaSuccess) return GF_ECUDA;
        if (cudaStreamWaitEvent(q, fork->ev[1 + f], 0) != cudaSuccess) return GF_ECUDA;
    }
    return GF_OK;
}

namespace {

// Every input of a batch's plan, staging block and captured graph, field by field.
std::string batch_key(const Image* ims, const BoxKernel* bks, int n) {
    std::string k;
    k.reserve((size_t)n * 160);
    auto put = [&k](const void* p, size_t len) { k.append(static_cast<const char*>(p), len); };
    for (int i = 0; i < n; ++i) {
        const Image& im = ims[i];
        const int iv[] = {im.H, im.W, im.C, im.in_dt, im.out_dt, im.boundary, im.plan.path, im.plan.tile_w,
                          im.plan.tile_h, im.plan.col_w, im.plan.col_h, im.plan.accum, im.sy, im.sx, im.oy, im.ox};
        const void* ptrs[] = {im.in, im.out};
        const size_t pitches[] = {im.in_pitch, im.out_pitch};
        put(iv, sizeof(iv));
        put(ptrs, sizeof(ptrs));
        put(pitches, sizeof(pitches));
        const BoxKernel& b = bks[i];
        put(&b.K, sizeof(b.K));
        put(b.r, sizeof(b.r));
        put(b.w, sizeof(b.w));
        put(&b.sw, sizeof(b.sw));
    }
    return k;
}

}  // namespace

gf_status launch_filter_batch(gf_handle_s* h, const Image* ims, const BoxKernel* bks, int n, void* stream) {
    if (n <= 0) return GF_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t staged = static_cast<cudaEvent_t>(h->staged_event);
    // The same batch as the last captured one: its graph holds every launch and
    // the staging copy of an unchanged block, so it is replayed as it stands
    // (ordered after the previous batch on the device, no host planning).
    std::string key;
    if (h->use_graphs) {
        key = batch_key(ims, bks, n);
        if (h->graph_exec && key == h->batch_key) {
            if (cudaStreamWaitEvent(s, staged, 0) != cudaSuccess) return GF_ECUDA;
            if (cudaGraphLaunch(static_cast<cudaGraphExec_t>(h->graph_exec), s) != cudaSuccess) return GF_ECUDA;
            if (cudaEventRecord(staged, s) != cudaSuccess) return GF_ECUDA;
            h->last_launches = h->batch_key_launches;
            return GF_OK;
        }
    }
    h->batch_key.clear();
    std::vector<Prepared> pr(n);
    std::vector<int> order(n);
    std::vector<BatchClass> cls(n);
    std::vector<TwoPass> tps(n);
    std::vector<size_t> tp_off(n);
    std::vector<int> wk(n);
    BatchWork w;
    w.pr = pr.data();
    w.order = order.data();
    w.cls = cls.data();
    w.tp = tps.data();
    w.tp_off = tp_off.data();
    w.wk_img = wk.data();
    gf_status st = batch_plan(ims, bks, n, w);
    if (st != GF_OK) return st;
    // the previous batch must have finished (its staging, its intermediates)
    // before either is rewritten
    if (cudaEventSynchronize(staged) != cudaSuccess) return GF_ECUDA;
    if (w.total > h->batch.dev_bytes || w.total > h->batch.pinned_bytes || w.inter_total > h->inter.dev_bytes) {
        if (h->graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(h->graph_exec));
        h->graph_exec = nullptr;
        h->graph_sig.clear();
        st = scratch_reserve(h->batch, w.total, w.total);
        if (st == GF_OK) st = scratch_reserve(h->inter, w.inter_total, 0);
        if (st != GF_OK) return st;
    }
    st = batch_bind(w, static_cast<unsigned char*>(h->inter.dev));
    if (st != GF_OK) return st;
    // graph signature: everything a captured launch bakes in (fused kernels read
    // their per-image parameters from the staging block; two-pass launches take
    // theirs, buffers included, as kernel arguments)
    std::string sig = std::to_string(n);
    for (int ci = 0; ci < w.ncls; ++ci) {
        const BatchClass& c = w.cls[ci];
        sig += "|" + std::to_string(c.key) + "," + std::to_string(c.count) + "," + std::to_string(c.ntiles) + "," +
               std::to_string(c.grid) + "," + std::to_string(c.smem) + "," + std::to_string(c.tmem_cols);
    }
    for (int t = 0; t < w.ntp; ++t) {
        sig += "|t";
        sig.append(reinterpret_cast<const char*>(&w.tp[t].kp), sizeof(KParams));
        sig.append(reinterpret_cast<const char*>(&w.tp[t].cp), sizeof(CParams));
        sig.append(reinterpret_cast<const char*>(w.tp[t].maps_in), 2 * sizeof(CUtensorMap));
        sig.append(reinterpret_cast<const char*>(w.tp[t].maps_r), 2 * sizeof(CUtensorMap));
        sig += std::to_string(w.tp[t].grid_r.x) + "," + std::to_string(w.tp[t].grid_r.y) + "," +
               std::to_string(w.tp[t].grid_c.x) + "," + std::to_string(w.tp[t].grid_c.y) + "," +
               std::to_string(w.tp[t].CW) + "," + std::to_string(w.tp[t].in_dt) + "," + std::to_string(w.tp[t].out_dt);
    }
    for (int k = 0; k < w.nwk; ++k) {
        // walk launches take their arguments by value: every field is in the signature
        const Image& im = ims[w.wk_img[k]];
        const BoxKernel& b = bks[w.wk_img[k]];
        sig += "|w";
        const void* ptrs[] = {im.in, im.out};
        const size_t pitches[] = {im.in_pitch, im.out_pitch};
        const int iv[] = {im.H, im.W, im.C, im.in_dt, im.out_dt, im.boundary};
        sig.append(reinterpret_cast<const char*>(ptrs), sizeof(ptrs));
        sig.append(reinterpret_cast<const char*>(pitches), sizeof(pitches));
        sig.append(reinterpret_cast<const char*>(iv), sizeof(iv));
        sig.append(reinterpret_cast<const char*>(&b), sizeof(BoxKernel));
    }
    unsigned char* hp = static_cast<unsigned char*>(h->batch.pinned);
    unsigned char* dp = static_cast<unsigned char*>(h->batch.dev);
    batch_stage(w, n, hp, dp);
    h->last_launches = batch_launches(w);
    if (h->use_graphs) {
        if (!h->graph_exec || h->graph_sig != sig) {
            if (h->graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(h->graph_exec));
            h->graph_exec = nullptr;
            cudaStream_t cap;
            if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return GF_ECUDA;
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                cudaStreamDestroy(cap);
                return GF_ECUDA;
            }
            st = batch_enqueue(w, dp, hp, cap, &h->fork);
            const cudaError_t ce = cudaStreamEndCapture(cap, &g);
            cudaStreamDestroy(cap);
            if (st != GF_OK || ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return st != GF_OK ? st : GF_ECUDA;
            }
            cudaGraphExec_t ex = nullptr;
            const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) return GF_ECUDA;
            h->graph_exec = ex;
            h->graph_sig = sig;
        }
        if (cudaGraphLaunch(static_cast<cudaGraphExec_t>(h->graph_exec), s) != cudaSuccess) return GF_ECUDA;
        h->batch_key = key;
        h->batch_key_launches = h->last_launches;
    } else {
        st = batch_enqueue(w, dp, hp, s, &h->fork);
        if (st != GF_OK) return st;
    }
    if (cudaEventRecord(staged, s) != cudaSuccess) return GF_ECUDA;
    return GF_OK;
}

gf_status launch_row_box_sums(const void* in, size_t in_pitch, int32_t* out, size_t out_pitch, size_t plane_stride,
                              int H, int W, int C, int in_dt, const BoxKernel& bk, int boundary, void* stream) {
    const DeviceInfo& di = device_info();
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
    while (TWp > 1 && smem_for(TWp) > (size_t)di.max_smem) TWp /= 2;
    const size_t smem = smem_for(TWp);
    if (smem > (size_t)di.max_smem) return GF_EUNSUPPORTED;
    const int nstrips = (W + TWp - 1) / TWp;
    const int ny = std::max(1, std::min((H + kWarps - 1) / kWarps, 4 * di.sms / std::max(1, nstrips) + 1));
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

gf_status filter_host_pipelined(gf_handle_s* h, const Image& im, const BoxKernel& bk, const FilterPlan& fp,
                                const HostRows& hr, cudaStream_t s) {
    const int H = im.H;
    // row tiles of the launch: the fused kernel's or the register walk's
    int T = 0, TH = 0;
    Prepared pr;
    gf_status st = GF_OK;
    if (fp.path == GF_PATH_FUSED) {
        st = prepare(im, bk, &fp.strip, pr);
        if (st != GF_OK) return st;
        TH = fp.strip.TH;
    } else if (fp.path == GF_PATH_WALK) {
        cudaKernel_t kern = nullptr;
        WalkerPlan wp;
        // a kernel that cannot be compiled or loaded: the unpipelined call
        // takes the default plan's fallback
        if (walker_load(im, bk, &kern, &wp) != GF_OK) return GF_EUNSUPPORTED;
        TH = wp.th;
    } else {
        return GF_EUNSUPPORTED;
    }
    T = (H + TH - 1) / TH;
    if (T < 4 || h->fork.n < 2) return GF_EUNSUPPORTED;
    auto launch_slab = [&](int ty0, int ty1) {
        return fp.path == GF_PATH_FUSED ? launch_prepared(im, pr, s, ty0, ty1) : launch_walker(im, bk, s, ty0, ty1);
    };
    const int tps = (T + 7) / 8;   // row tiles per slab
    const int nslab = (T + tps - 1) / tps;
    const int slab_rows = tps * TH;
    const size_t need = (size_t)2 * nslab + 1;
    while (h->slab_events.size() < need) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return GF_ECUDA;
        h->slab_events.push_back(ev);
    }
    auto ev = [&](size_t i) { return static_cast<cudaEvent_t>(h->slab_events[i]); };
    // rows [a, b) between host and device (one flat copy when both sides are dense)
    auto copy_rows = [&](bool to_dev, int a, int b, cudaStream_t q) {
        const size_t ai = (size_t)a;
        if (to_dev)
            return hr.in_pitch == hr.irow && hr.dpi == hr.irow
                       ? cudaMemcpyAsync(hr.din + ai * hr.dpi, hr.hin + ai * hr.in_pitch, (b - a) * hr.irow,
                                         cudaMemcpyHostToDevice, q)
                       : cudaMemcpy2DAsync(hr.din + ai * hr.dpi, hr.dpi, hr.hin + ai * hr.in_pitch, hr.in_pitch,
                                           hr.irow, b - a, cudaMemcpyHostToDevice, q);
        return hr.out_pitch == hr.orow && hr.dpo == hr.orow
                   ? cudaMemcpyAsync(hr.hout + ai * hr.out_pitch, hr.dout + ai * hr.dpo, (b - a) * hr.orow,
                                     cudaMemcpyDeviceToHost, q)
                   : cudaMemcpy2DAsync(hr.hout + ai * hr.out_pitch, hr.out_pitch, hr.dout + ai * hr.dpo, hr.dpo,
                                       hr.orow, b - a, cudaMemcpyDeviceToHost, q);
    };
    cudaStream_t cin = h->fork.s[0], cout = h->fork.s[1];
    // both copy streams start after the work already queued on `s`
    if (cudaEventRecord(ev(2 * nslab), s) != cudaSuccess) return GF_ECUDA;
    if (cudaStreamWaitEvent(cin, ev(2 * nslab), 0) != cudaSuccess) return GF_ECUDA;
    if (cudaStreamWaitEvent(cout, ev(2 * nslab), 0) != cudaSuccess) return GF_ECUDA;
    for (int k = 0; k < nslab; ++k) {
        const int a = k * slab_rows, b = std::min(H, a + slab_rows);
        if (copy_rows(true, a, b, cin) != cudaSuccess || cudaEventRecord(ev(k), cin) != cudaSuccess) return GF_ECUDA;
    }
    for (int k = 0; k < nslab; ++k) {
        const int b = std::min(H, (k + 1) * slab_rows);
        // the slab's filter needs its rows and rk rows below (earlier slabs are in by order)
        const int last_in = std::min(nslab - 1, (std::min(H, b + bk.rk) - 1) / slab_rows);
        if (cudaStreamWaitEvent(s, ev(last_in), 0) != cudaSuccess) return GF_ECUDA;
        st = launch_slab(k * tps, std::min(T, (k + 1) * tps));
        if (st != GF_OK) return st;
        if (cudaEventRecord(ev(nslab + k), s) != cudaSuccess) return GF_ECUDA;
        if (cudaStreamWaitEvent(cout, ev(nslab + k), 0) != cudaSuccess) return GF_ECUDA;
        if (copy_rows(false, k * slab_rows, b, cout) != cudaSuccess) return GF_ECUDA;
    }
    if (cudaStreamSynchronize(cout) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return GF_ECUDA;
    return GF_OK;
}

gf_status read_device_status(int clear, int* value) {
    int v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return GF_ECUDA;
    if (cudaMemcpyFromSymbol(&v, g_device_status, sizeof(int)) != cudaSuccess) return GF_ECUDA;
    if (clear) {
        const int z = 0;
        if (cudaMemcpyToSymbol(g_device_status, &z, sizeof(int)) != cudaSuccess) return GF_ECUDA;
    }
    if (value) *value = v;
    return GF_OK;
}

}  // namespace gb
