// Host side of the two-pass filter: plans, shared-memory layouts, tensor maps,
// the intermediate's memory pool, and the fused/two-pass path choice.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "plan.h"
#include "twopass.h"
#include "walker.h"

namespace gb {

GB_DECLARE_ROWPASS(uint8_t)
GB_DECLARE_ROWPASS(uint16_t)
GB_DECLARE_ROWPASS(float)
GB_DECLARE_ROWPASS(__nv_bfloat16)
GB_DECLARE_ROWPASS(__half)
GB_DECLARE_COLPASS(float)
GB_DECLARE_COLPASS(__nv_bfloat16)
GB_DECLARE_COLPASS(__half)

namespace {

constexpr int kColStages = 3;

// Shared memory a row-pass CTA may use so that two fit an SM.
size_t row_budget() { return (size_t)device_info().max_smem / 2 - 1024; }

// Row-pass part of KParams for segments of TWp pixels; returns smem bytes.
// Two TMA stages when they fit the two-CTA budget, else one (long segments
// for large radii: the halo of 2 rk + 1 pixels per segment costs more than
// exposing the copy latency).
size_t layout_rows(KParams& kp, const Image& im, const BoxKernel& bk, int TWp, bool tma, int stages = 0) {
    const int isz = dtype_size(im.in_dt);
    const int C = im.C;
    kp.TWp = TWp;
    kp.TW = TWp * C;
    kp.ealign = 16 / isz;
    const int span = (TWp + 2 * bk.rk + 1) * C + kp.ealign - 1;
    const int sout_max = (bk.rk + 1) * C + kp.ealign - 1;
    kp.m = chunk_for(std::max(span, sout_max + kp.TW + bk.rk * C + 1));
    // the gather of the last 256-element chunk reads up to its padded end
    kp.SP = round_up(std::max(32 * kp.m, sout_max + round_up(kp.TW, 256) + bk.rk * C + 1), 4);
    const bool in_place = im.in_dt == GF_F32;   // running sums overwrite the staged f32 row
    const bool wide = tma && ((size_t)im.W * C * isz) % 8 == 0;
    staging_geometry(kp, span, in_place ? std::max(32 * kp.m, kp.SP) : 32 * kp.m, in_place ? 32 : 1, isz, wide);
    kp.NB = kp.RT = kp.tmem_cols = 0;
    kp.use_tma = tma ? 1 : 0;
    kp.tma_store = 0;
    auto place = [&](int nst) {
        kp.nstage = nst;
        size_t off = 0;
        kp.off_stage = 0;
        off += (size_t)kp.nstage * kBand * kp.SROW * isz;
        off = (off + 127) / 128 * 128;
        kp.off_p = (int)off;
        if (!in_place) off += (size_t)kWarps * kp.SP * 4;
        off = (off + 127) / 128 * 128;
        kp.off_pl = (int)off;   // float rows: the residue sums (row_prefix)
        if (!dtype_is_int(im.in_dt)) off += (size_t)kWarps * kp.SP * 4;
        off = (off + 15) / 16 * 16;
        kp.off_bar = (int)off;
        off += (size_t)kMaxStages * 8;
        kp.off_rband = kp.off_ring = kp.off_tmem = kp.off_obuf = 0;
        return off;
    };
    if (!tma) return place(1);
    if (stages) return place(stages);
    const size_t two = place(2);
    return two <= row_budget() ? two : place(1);
}

// Column-pass layout for strips of CW element columns in bands of B rows;
// returns smem bytes.
size_t layout_cols_band(CParams& cp, int CW, int rk, int B) {
    cp.B = B;
    cp.NB = (2 * rk + 1 + B + B - 1) / B;   // live rows: 2 rk + 1 + one band
    cp.nstage = kColStages;
    size_t off = 0;
    cp.off_stage = 0;
    off += (size_t)cp.nstage * B * col_stage_stride(CW) * 4;
    off = (off + 127) / 128 * 128;
    cp.off_ring = (int)off;
    off += (size_t)2 * (cp.NB + 1) * B * col_ring_stride(CW) * 4;   // hi ring + mirror, then the lo ring
    off = (off + 15) / 16 * 16;
    cp.off_coff = (int)off;
    off += (size_t)CW * 4;
    off = (off + 15) / 16 * 16;
    cp.off_bar = (int)off;
    off += (size_t)kMaxStages * 8;
    return off;
}

// Column-pass layout with the band height chosen for the strip: 32-column
// strips take 32-row bands when these keep as many CTAs per SM as 16-row
// bands (measured on 8192^2 sigma 100: +9 %; where they cost a CTA per SM,
// as for radii near 130, they are slower).
size_t layout_cols(CParams& cp, int CW, int rk) {
    int B = col_band(CW);
    if (CW == 32) {
        CParams a{}, b{};
        const size_t s16 = layout_cols_band(a, CW, rk, B), s32 = layout_cols_band(b, CW, rk, 32);
        if (s32 <= (size_t)device_info().max_smem && ctas_per_sm(s32, 0) >= ctas_per_sm(s16, 0)) B = 32;
    }
    return layout_cols_band(cp, CW, rk, B);
}

// Rows per CTA for `ncols` tiles across and `slots` resident CTAs: the tile
// count down the image that minimises waves x (rows + halo), i.e. the work of
// the slowest slot, rows rounded up to `multiple`.
int rows_for(int H, int ncols, int slots, int multiple, int halo) {
    ncols = std::max(1, ncols);
    slots = std::max(1, slots);
    int best_rows = round_up(H, multiple);
    double best = -1.0;
    const int max_ty = std::max(1, std::min(H, 4 * slots / ncols + 1));
    for (int ty = 1; ty <= max_ty; ++ty) {
        const int rows = round_up((H + ty - 1) / ty, multiple);
        const int tiles = ncols * ((H + rows - 1) / rows);
        const double waves = (double)((tiles + slots - 1) / slots);
        const double cost = waves * (rows + halo);
        if (best < 0.0 || cost < best * 0.999) {
            best = cost;
            best_rows = rows;
        }
    }
    return best_rows;
}

bool valid_cw(int cw) { return cw == 32 || cw == 64 || cw == 128 || cw == 256; }

// Widest column strip whose ring leaves room for three CTAs per SM.
int default_cw(int rk) {
    CParams cp{};
    for (int c : {256, 128, 64}) {
        if (ctas_per_sm(layout_cols(cp, c, rk), 0) >= 3) return c;
    }
    return 32;
}

// Per-device pool of the two-pass intermediates: freed blocks stay in the
// pool for the next call instead of going back to the driver.
cudaMemPool_t pool_for(int dev) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

}  // namespace

TwoPassPlan default_twopass_plan(const Image& im, const BoxKernel& bk) {
    const DeviceInfo& di = device_info();
    TwoPassPlan pl;
    const int C = im.C;
    const int rk = bk.rk;
    KParams kp{};
    // Row segments long enough that the 2 rk + 1 halo pixels stay a small
    // fraction (at least 1024 elements: measured faster than 256-element
    // segments whose scan fits the registers, even for small radii).
    int seg = std::max(1, std::min(4096, std::max(1024, 8 * (2 * rk + 1) * C)) / C);
    seg = std::min(seg, im.W);
    const int target = seg;
    // shrink until two CTAs fit an SM (with one stage if need be)
    while (seg > 8 && layout_rows(kp, im, bk, seg, true) > row_budget()) seg = seg * 3 / 4;
    // Where that leaves the halo the larger part of the walk, a segment of up
    // to 512 pixels that fits one CTA per SM wins: measured on GB300 at
    // 2000 x 3000 x 3 f32 sigma 50 (101 -> 512 px: 0.379 -> 0.312 ms per filter).
    const double span = 2.0 * rk + 1.0;
    int seg1 = std::max(seg, std::min(std::min(target, 512), im.W));
    while (seg1 > seg && layout_rows(kp, im, bk, seg1, true) > (size_t)di.max_smem) seg1 = seg1 * 3 / 4;
    if (seg1 > seg && (seg1 + span) / seg1 < 0.6 * (seg + span) / seg) seg = seg1;
    pl.seg_px = std::max(1, seg);
    // Rows per row CTA: the fewest waves for the resident CTAs, but at most 32
    // rows: the row launch has no vertical halo, so short tiles cost nothing
    // but a CTA's set-up and many of them balance the SMs (8192^2 f32 sigma
    // 100: 432 -> 32 rows, 1.29 -> 1.23 ms per filter).
    const size_t smem_r = layout_rows(kp, im, bk, pl.seg_px, true);
    const int per_sm_r = std::max(1, ctas_per_sm(smem_r, 0));
    const int nseg = (im.W + pl.seg_px - 1) / pl.seg_px;
    pl.row_th = std::min(rows_for(im.H, nseg, per_sm_r * di.sms, kBand, 0), 4 * kBand);
    // Column strips: the widest whose ring leaves room for three CTAs per SM.
    CParams cp{};
    const int cw = default_cw(rk);
    pl.CW = cw;
    const int rowlen = out_w(im) * C;   // columns of R (sampled columns only)
    const int nstrips = (rowlen + cw - 1) / cw;
    const int per_sm_c = std::max(1, ctas_per_sm(layout_cols(cp, cw, rk), 0));
    pl.col_th = rows_for(im.H, nstrips, per_sm_c * di.sms, 1, 2 * rk + 2 * cp.B);
    pl.col_th = column_tile_rows(pl.col_th, im.H, bk);
    return pl;
}

gf_status prepare_twopass(const Image& im, const BoxKernel& bk, const TwoPassPlan& plan, TwoPass& tp) {
    const DeviceInfo& di = device_info();
    if (plan.seg_px < 1 || plan.row_th < 1 || plan.col_th < 1 || !valid_cw(plan.CW)) return GF_EINVAL;
    tp = TwoPass();
    tp.plan = plan;
    tp.in_dt = im.in_dt;
    tp.out_dt = im.out_dt;
    const int C = im.C;
    const int rowlen = im.W * C;
    const int rlen = out_w(im) * C;   // element columns of R and of the output
    // ---- row pass
    KParams& kp = tp.kp;
    kp.in = static_cast<const unsigned char*>(im.in);
    kp.in_pitch = (long long)im.in_pitch;
    kp.status = launch_status_word();
    kp.wait_limit = launch_wait_limit();
    kp.H = im.H;
    kp.W = im.W;
    kp.C = C;
    kp.boundary = im.boundary;
    kp.K = bk.K;
    for (int i = 0; i < GF_KMAX; ++i) {
        kp.r[i] = bk.r[i];
        kp.w[i] = bk.w[i];
    }
    kp.sw = bk.sw;
    kp.rk = bk.rk;
    kp.TH = round_up(plan.row_th, kBand);
    kp.sx = im.sx;
    kp.ox = im.ox;
    const auto enc = tensor_map_encoder();
    bool tma = enc != nullptr && (reinterpret_cast<uintptr_t>(im.in) % 16 == 0) && (im.in_pitch % 16 == 0) &&
               im.in_pitch < (1ull << 40);
    size_t smem = layout_rows(kp, im, bk, plan.seg_px, tma);
    if (smem > (size_t)di.max_smem) {
        tma = false;
        smem = layout_rows(kp, im, bk, plan.seg_px, false);
        if (smem > (size_t)di.max_smem) return GF_EUNSUPPORTED;
    }
    std::memset(tp.maps_in, 0, sizeof(tp.maps_in));
    if (tma && !encode_row_maps(kp, im.in, im.in_pitch, rowlen, im.H, im.in_dt, tp.maps_in))
        smem = layout_rows(kp, im, bk, plan.seg_px, false);
    tp.smem_r = smem;
    tp.grid_r = dim3((im.W + plan.seg_px - 1) / plan.seg_px, (im.H + kp.TH - 1) / kp.TH);
    tp.r_pitch = (size_t)round_up(rlen * 4, 128);
    tp.r_bytes = twopass_inter_bytes(im);
    // ---- column pass
    CParams& cp = tp.cp;
    cp.out = static_cast<unsigned char*>(im.out);
    cp.out_pitch = (long long)im.out_pitch;
    cp.status = launch_status_word();
    cp.wait_limit = launch_wait_limit();
    cp.H = im.H;
    cp.rowlen = rlen;
    cp.sy = im.sy;
    cp.oy = im.oy;
    cp.boundary = im.boundary;
    cp.K = bk.K;
    for (int i = 0; i < GF_KMAX; ++i) {
        cp.r[i] = bk.r[i];
        cp.w[i] = bk.w[i];
    }
    cp.sw = bk.sw;
    cp.rk = bk.rk;
    cp.TH = plan.col_th;
    tp.CW = plan.CW;
    tp.smem_c = layout_cols(cp, plan.CW, bk.rk);
    if (tp.smem_c > (size_t)di.max_smem) return GF_EUNSUPPORTED;
    cp.use_tma = enc != nullptr ? 1 : 0;
    const size_t osz = (size_t)dtype_size(im.out_dt);
    cp.pair_ok = (reinterpret_cast<uintptr_t>(im.out) % (2 * osz) == 0) && (im.out_pitch % (2 * osz) == 0);
    tp.grid_c = dim3((rlen + plan.CW - 1) / plan.CW, (im.H + plan.col_th - 1) / plan.col_th);
    if (tp.grid_r.y > 65535u || tp.grid_c.y > 65535u) return GF_EINVAL;   // grid y limit of the launches
    return GF_OK;
}

namespace {

// Tensor maps of an FP32 intermediate for the column pass: a row map (one row
// per box) and, for lane sums, the band map (B rows, col_stage_stride
// columns).  `xext` elements per row, `rows` rows of `pitch` bytes.
bool encode_col_maps(CUtensorMap* maps, const void* R, size_t pitch, uint64_t xext, int rows, int CW, int B) {
    std::memset(maps, 0, 2 * sizeof(CUtensorMap));
    const auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t gdim[2] = {(cuuint64_t)xext, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)pitch};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint32_t box1[2] = {(cuuint32_t)CW, 1};
    const cuuint32_t boxb[2] = {(cuuint32_t)col_stage_stride(CW), (cuuint32_t)B};
    if (enc(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(R), gdim, gstride, box1, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (col_lane_sums(CW) &&
        enc(&maps[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(R), gdim, gstride, boxb, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    return true;
}

gf_status launch_cols(const CParams& cp, const CUtensorMap* maps, int CW, dim3 grid, size_t smem, int out_dt,
                      cudaStream_t s, int mode) {
    switch (out_dt) {
        case GF_F32: return launch_col_pass<float>(cp, maps, CW, grid, smem, s, mode);
        case GF_BF16: return launch_col_pass<__nv_bfloat16>(cp, maps, CW, grid, smem, s, mode);
        case GF_F16: return launch_col_pass<__half>(cp, maps, CW, grid, smem, s, mode);
        default: return GF_EUNSUPPORTED;
    }
}

}  // namespace

gf_status bind_twopass(TwoPass& tp, void* R) {
    if (!R || reinterpret_cast<uintptr_t>(R) % 128) return GF_EINVAL;
    tp.kp.out = static_cast<unsigned char*>(R);
    tp.kp.out_pitch = (long long)tp.r_pitch;
    tp.cp.rin = static_cast<const unsigned char*>(R);
    tp.cp.r_pitch = (long long)tp.r_pitch;
    if (tp.cp.use_tma && !encode_col_maps(tp.maps_r, R, tp.r_pitch, (uint64_t)tp.cp.rowlen, tp.cp.H, tp.CW, tp.cp.B))
        tp.cp.use_tma = 0;
    return GF_OK;
}

gf_status launch_slices_twopass(const Image& tall, int D, int H, const BoxKernel& bk, const TwoPassPlan& plan,
                                void* R1, void* R2, size_t r2_pitch, cudaStream_t s) {
    const DeviceInfo& di = device_info();
    if (tall.H != D * H || reinterpret_cast<uintptr_t>(R2) % 16 || r2_pitch % 16) return GF_EINVAL;
    Image im = tall;
    im.out = R2;
    im.out_pitch = r2_pitch;
    im.out_dt = GF_F32;
    TwoPass tp;
    gf_status st = prepare_twopass(im, bk, plan, tp);
    if (st == GF_OK) st = bind_twopass(tp, R1);   // R1 maps cover all D H rows
    if (st != GF_OK) return st;
    // column pass per slice: H rows folded within the slice, grid z = slice
    CParams& cp = tp.cp;
    cp.H = H;
    cp.zrow = H;
    cp.zout = (long long)((size_t)H * r2_pitch);
    const int nstrips = (cp.rowlen + tp.CW - 1) / tp.CW;
    const int per_sm = std::max(1, ctas_per_sm(tp.smem_c, 0));
    cp.TH = column_tile_rows(rows_for(H, nstrips * D, per_sm * di.sms, 1, 2 * bk.rk + 2 * cp.B), H, bk);
    tp.grid_c = dim3(nstrips, (H + cp.TH - 1) / cp.TH, D);
    return enqueue_twopass(tp, s);
}

gf_status launch_depth_pass(const float* R, size_t r_pitch, int D, int H, int W, int C, void* out, size_t out_pitch,
                            int out_dt, int boundary, const BoxKernel& bz, cudaStream_t s) {
    const DeviceInfo& di = device_info();
    if (!R || reinterpret_cast<uintptr_t>(R) % 16 || r_pitch % 16) return GF_EINVAL;
    const int rowlen = W * C;
    // element offset of image row H - 1 plus a row must stay an int (TMA x coordinate)
    if ((uint64_t)H * (r_pitch / 4) > (uint64_t)INT32_MAX - 512 || H > 65535) return GF_EUNSUPPORTED;
    CParams cp{};
    cp.rin = reinterpret_cast<const unsigned char*>(R);
    cp.r_pitch = (long long)((size_t)H * r_pitch);   // one "row" of the depth pass is a slice of R
    cp.out = static_cast<unsigned char*>(out);
    cp.out_pitch = (long long)((size_t)H * out_pitch);
    cp.status = launch_status_word();
    cp.wait_limit = launch_wait_limit();
    cp.H = D;
    cp.rowlen = rowlen;
    cp.boundary = boundary;
    cp.K = bz.K;
    for (int i = 0; i < GF_KMAX; ++i) {
        cp.r[i] = bz.r[i];
        cp.w[i] = bz.w[i];
    }
    cp.sw = bz.sw;
    cp.rk = bz.rk;
    cp.sy = 1;
    cp.oy = 0;
    cp.zcol = (int)(r_pitch / 4);            // blockIdx.z = image row y
    cp.zout = (long long)out_pitch;
    const int CW = default_cw(bz.rk);
    const size_t smem = layout_cols(cp, CW, bz.rk);
    if (smem > (size_t)di.max_smem) return GF_EUNSUPPORTED;
    const int nstrips = (rowlen + CW - 1) / CW;
    const int per_sm = std::max(1, ctas_per_sm(smem, 0));
    cp.TH = column_tile_rows(rows_for(D, nstrips * H, per_sm * di.sms, 1, 2 * bz.rk + 2 * cp.B), D, bz);
    const size_t osz = (size_t)dtype_size(out_dt);
    cp.pair_ok = (reinterpret_cast<uintptr_t>(out) % (2 * osz) == 0) && (out_pitch % (2 * osz) == 0);
    CUtensorMap maps[2];
    const uint64_t xext = (uint64_t)(H - 1) * (r_pitch / 4) + (uint64_t)rowlen;
    cp.use_tma = encode_col_maps(maps, R, (size_t)H * r_pitch, xext, D, CW, cp.B) ? 1 : 0;
    const dim3 grid(nstrips, (D + cp.TH - 1) / cp.TH, H);
    return launch_cols(cp, maps, CW, grid, smem, out_dt, s, 0);
}

gf_status enqueue_twopass(const TwoPass& tp, cudaStream_t s) {
    gf_status st;
    const int m = tp.plan.accum;
    switch (tp.in_dt) {
        case GF_U8: st = launch_row_pass<uint8_t>(tp.kp, tp.maps_in, tp.grid_r, tp.smem_r, s, m); break;
        case GF_U16: st = launch_row_pass<uint16_t>(tp.kp, tp.maps_in, tp.grid_r, tp.smem_r, s, m); break;
        case GF_F32: st = launch_row_pass<float>(tp.kp, tp.maps_in, tp.grid_r, tp.smem_r, s, m); break;
        case GF_BF16: st = launch_row_pass<__nv_bfloat16>(tp.kp, tp.maps_in, tp.grid_r, tp.smem_r, s, m); break;
        case GF_F16: st = launch_row_pass<__half>(tp.kp, tp.maps_in, tp.grid_r, tp.smem_r, s, m); break;
        default: return GF_EUNSUPPORTED;
    }
    if (st != GF_OK) return st;
    return launch_cols(tp.cp, tp.maps_r, tp.CW, tp.grid_c, tp.smem_c, tp.out_dt, s, m);
}

gf_status launch_twopass(const Image& im, const BoxKernel& bk, const TwoPassPlan& plan, cudaStream_t s) {
    TwoPass tp;
    gf_status st = prepare_twopass(im, bk, plan, tp);
    if (st != GF_OK) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF_ECUDA;
    cudaMemPool_t pool = pool_for(dev);
    if (!pool) return GF_ENOMEM;
    void* R = nullptr;
    if (cudaMallocFromPoolAsync(&R, tp.r_bytes, pool, s) != cudaSuccess) return GF_ENOMEM;
    st = bind_twopass(tp, R);
    if (st == GF_OK) st = enqueue_twopass(tp, s);
    cudaFreeAsync(R, s);
    return st;
}

// ------------------------------------------------------------------ plans
// Path choice by a cost model in units of "one row pass over the image".  The
// fused kernel redoes the row pass on both halos, (TWp + 2 rk + 1) / TWp
// across and (TH + 2 rk) / TH down, and its column work on the vertical one;
// a wide TMEM ring also cuts its resident CTAs per SM (cost grows as the
// fourth root of the lost occupancy), and with several channels its strips
// hold fewer pixels and its row scans do more per element (x 1.4).  The
// two-pass form pays each halo along one axis only, plus the write and
// re-read of the FP32 intermediate (8 bytes per element against the image's
// own in + out bytes).  The weights were fitted to GB300 timings of both
// paths over sigma 2..100, K 3..5, C 1..3, u8 / bf16 / f32 and 1..67 Mpx.
int choose_path(const Image& im, const BoxKernel& bk, const StripPlan& sp) {
    if (!fused_fits(im, bk, sp.TWp)) return GF_PATH_TWO_PASS;
    const double rk = bk.rk;
    const double fx = (sp.TWp + 2.0 * rk + 1.0) / sp.TWp;
    const double fy = (sp.TH + 2.0 * rk) / sp.TH;
    const int per_sm = std::max(1, std::min(4, fused_ctas_per_sm(im, bk, sp.TWp)));
    const double fused = (fx * fy + 0.6 * fy) * std::pow(4.0 / per_sm, 0.25) * (im.C > 1 ? 1.4 : 1.0);
    const double io = dtype_size(im.in_dt) + dtype_size(im.out_dt);
    const double two = 1.0 + 0.6 + 0.9 * 8.0 / io;
    return fused > two ? GF_PATH_TWO_PASS : GF_PATH_FUSED;
}

namespace {

// True if both launches of the two-pass form fit one CTA's shared memory.
bool twopass_fits(const Image& im, const BoxKernel& bk, const TwoPassPlan& pl) {
    const size_t max_smem = (size_t)device_info().max_smem;
    KParams kp{};
    CParams cp{};
    return layout_rows(kp, im, bk, std::max(1, std::min(pl.seg_px, im.W)), false) <= max_smem &&
           layout_cols(cp, pl.CW, bk.rk) <= max_smem;
}

}  // namespace

namespace {

gf_status resolve_plan_uncached(const Image& im, const BoxKernel& bk, const gf_plan* req, FilterPlan& out);

// What a plan depends on: the device, the image's geometry, types, sampling
// and boundary, the alignment of its pointers and pitches (TMA staging and
// stores), the radii and the requested plan.
struct PlanKey {
    long long v[24];
    bool operator==(const PlanKey& o) const { return std::memcmp(v, o.v, sizeof(v)) == 0; }
};

PlanKey plan_key(const Image& im, const BoxKernel& bk, const gf_plan* req, int dev) {
    PlanKey k;
    std::memset(&k, 0, sizeof(k));
    long long* v = k.v;
    *v++ = dev;
    *v++ = im.H;
    *v++ = im.W;
    *v++ = im.C;
    *v++ = im.in_dt;
    *v++ = im.out_dt;
    *v++ = im.boundary;
    *v++ = ((long long)im.sy << 32) | (unsigned)im.sx;
    *v++ = ((long long)im.oy << 32) | (unsigned)im.ox;
    *v++ = (long long)(reinterpret_cast<uintptr_t>(im.in) % 16) | ((long long)(reinterpret_cast<uintptr_t>(im.out) % 16) << 8);
    *v++ = (long long)im.in_pitch;
    *v++ = (long long)im.out_pitch;
    *v++ = bk.K;
    for (int i = 0; i < GF_KMAX; ++i) *v++ = bk.r[i];
    if (req) {
        *v++ = 1 + req->path;
        *v++ = ((long long)req->tile_w << 32) | (unsigned)req->tile_h;
        *v++ = ((long long)req->col_w << 32) | (unsigned)req->col_h;
        *v++ = req->accum;
    }
    return k;
}

}  // namespace

// Plans are resolved once per distinct key and thread: the host work of a
// repeated call (the same image shape on the same device) is a lookup.
gf_status resolve_plan(const Image& im, const BoxKernel& bk, const gf_plan* req, FilterPlan& out) {
    constexpr int kSlots = 8;
    struct Entry {
        PlanKey key;
        FilterPlan plan;
        gf_status st;
        bool used = false;
    };
    thread_local Entry cache[kSlots];
    thread_local int next = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    const PlanKey k = plan_key(im, bk, req, dev);
    for (int i = 0; i < kSlots; ++i)
        if (cache[i].used && cache[i].key == k) {
            out = cache[i].plan;
            return cache[i].st;
        }
    const gf_status st = resolve_plan_uncached(im, bk, req, out);
    Entry& e = cache[next];
    next = (next + 1) % kSlots;
    e.key = k;
    e.plan = out;
    e.st = st;
    e.used = true;
    return st;
}

namespace {

gf_status resolve_plan_uncached(const Image& im, const BoxKernel& bk, const gf_plan* req, FilterPlan& out) {
    gf_plan r{};
    if (req) r = *req;
    if (r.path < GF_PATH_AUTO || r.path > GF_PATH_WALK) return GF_EINVAL;
    if (r.tile_w < 0 || r.tile_h < 0 || r.col_w < 0 || r.col_h < 0) return GF_EINVAL;
    if (r.col_w && !valid_cw(r.col_w)) return GF_EINVAL;
    if (r.accum < GF_ACCUM_COMPENSATED || r.accum > GF_ACCUM_PLAIN) return GF_EINVAL;
    out = FilterPlan();
    out.strip = default_plan(im, bk);
    if (r.path == GF_PATH_WALK) {
        if (r.accum != GF_ACCUM_COMPENSATED || !walker_eligible(im, bk)) return GF_EUNSUPPORTED;
        out.path = GF_PATH_WALK;
        out.two = default_twopass_plan(im, bk);
        return GF_OK;
    }
    if (r.path == GF_PATH_HBM) {
        if (r.accum != GF_ACCUM_COMPENSATED) return GF_EUNSUPPORTED;
        out.path = GF_PATH_HBM;
        out.two = default_twopass_plan(im, bk);
        return GF_OK;
    }
    if (is_sampled(im)) {
        // sampled outputs exist on the two-pass path only
        if (r.path == GF_PATH_FUSED) return GF_EUNSUPPORTED;
        out.path = GF_PATH_TWO_PASS;
    } else if (r.accum != GF_ACCUM_COMPENSATED) {
        // the study variants exist on the two-pass path only
        if (r.path == GF_PATH_FUSED) return GF_EUNSUPPORTED;
        out.path = GF_PATH_TWO_PASS;
    } else if (r.path == GF_PATH_AUTO) {
        // single-channel integer images with small radii: the register walk
        out.path = (!r.tile_w && !r.tile_h && !r.col_w && !r.col_h && walker_eligible(im, bk))
                       ? GF_PATH_WALK
                       : choose_path(im, bk, out.strip);
        if (out.path == GF_PATH_WALK) {
            out.two = default_twopass_plan(im, bk);
            return GF_OK;
        }
    } else {
        out.path = r.path;
    }
    if (out.path == GF_PATH_FUSED) {
        if (r.tile_w) {
            if (r.tile_w * im.C > 256) return GF_EINVAL;
            out.strip.TWp = std::min(r.tile_w, im.W);
        }
        if (r.tile_h) out.strip.TH = std::min(r.tile_h, im.H);
        out.strip.nstrips = (im.W + out.strip.TWp - 1) / out.strip.TWp;
        out.strip.nrowtiles = (im.H + out.strip.TH - 1) / out.strip.TH;
        out.two = default_twopass_plan(im, bk);
    } else {
        out.two = default_twopass_plan(im, bk);
        if (r.tile_w) out.two.seg_px = std::min(r.tile_w, im.W);
        if (r.tile_h) out.two.row_th = round_up(r.tile_h, kBand);
        if (r.col_w) out.two.CW = r.col_w;
        if (r.col_h) out.two.col_th = std::min(r.col_h, im.H);
        out.two.accum = r.accum;
        // beyond the shared-memory working set: running sums in HBM
        if (r.path == GF_PATH_AUTO && r.accum == GF_ACCUM_COMPENSATED && !twopass_fits(im, bk, out.two))
            out.path = GF_PATH_HBM;
    }
    return GF_OK;
}

}  // namespace

size_t twopass_inter_bytes(const Image& im) {
    return (size_t)round_up(out_w(im) * im.C * 4, 128) * (size_t)im.H;
}

int planned_path(const Image& im, const BoxKernel& bk) {
    FilterPlan fp;
    if (resolve_plan(im, bk, &im.plan, fp) != GF_OK) return GF_PATH_FUSED;
    return fp.path;
}

gf_status launch_filter_into(const Image& im, const BoxKernel& bk, void* inter, cudaStream_t s) {
    FilterPlan fp;
    gf_status st = resolve_plan(im, bk, &im.plan, fp);
    if (st != GF_OK) return st;
    if (fp.path == GF_PATH_WALK) return launch_walker(im, bk, s);
    if (fp.path == GF_PATH_FUSED) return launch_fused(im, bk, &fp.strip, s);
    if (fp.path == GF_PATH_HBM) return GF_EUNSUPPORTED;   // its scratch is not in the caller's buffer
    TwoPass tp;
    st = prepare_twopass(im, bk, fp.two, tp);
    if (st == GF_OK) st = bind_twopass(tp, inter);
    if (st == GF_OK) st = enqueue_twopass(tp, s);
    return st;
}

namespace {

// The HBM running-sum path with its scratch from the pool (released on `s`).
gf_status launch_global_pooled(const Image& im, const BoxKernel& bk, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GF_ECUDA;
    cudaMemPool_t pool = pool_for(dev);
    if (!pool) return GF_ENOMEM;
    void* buf = nullptr;
    if (cudaMallocFromPoolAsync(&buf, global_path_bytes(im, bk), pool, s) != cudaSuccess) return GF_ENOMEM;
    const gf_status st = launch_global(im, bk, buf, s);
    cudaFreeAsync(buf, s);
    return st;
}

}  // namespace

gf_status launch_filter(const Image& im, const BoxKernel& bk, const gf_plan* req, void* stream) {
    FilterPlan fp;
    gf_status st = resolve_plan(im, bk, req, fp);
    if (st != GF_OK) return st;
    const bool automatic = !req || (req->path == GF_PATH_AUTO && req->accum == GF_ACCUM_COMPENSATED);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (fp.path == GF_PATH_HBM) return launch_global_pooled(im, bk, s);
    if (fp.path == GF_PATH_WALK) {
        st = launch_walker(im, bk, s);
        // the default plan falls back to the fused kernel if the run-time
        // compilation is unavailable
        if (st == GF_OK || !automatic) return st;
        fp.path = GF_PATH_FUSED;
    }
    if (fp.path == GF_PATH_FUSED) {
        st = launch_fused(im, bk, &fp.strip, stream);
        // a default plan whose fused working set does not fit goes two-pass
        if (st != GF_EUNSUPPORTED || !automatic) return st;
    }
    st = launch_twopass(im, bk, fp.two, s);
    // a working set the plan's fit test let through but the launch refused
    if (st == GF_EUNSUPPORTED && automatic) return launch_global_pooled(im, bk, s);
    return st;
}

void plan_to_abi(const FilterPlan& fp, gf_plan* out) {
    out->path = fp.path;
    if (fp.path == GF_PATH_HBM || fp.path == GF_PATH_WALK) {
        out->tile_w = out->tile_h = out->col_w = out->col_h = 0;
        out->accum = GF_ACCUM_COMPENSATED;
        return;
    }
    if (fp.path == GF_PATH_FUSED) {
        out->tile_w = fp.strip.TWp;
        out->tile_h = fp.strip.TH;
        out->col_w = 0;
        out->col_h = 0;
    } else {
        out->tile_w = fp.two.seg_px;
        out->tile_h = fp.two.row_th;
        out->col_w = fp.two.CW;
        out->col_h = fp.two.col_th;
    }
    out->accum = fp.path == GF_PATH_FUSED ? GF_ACCUM_COMPENSATED : fp.two.accum;
}

}  // namespace gb
