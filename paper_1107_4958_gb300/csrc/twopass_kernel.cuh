// Two-pass form of the box-sum Gaussian filter (Sec. 3.4: rows, then columns).
//
// The fused strip kernel recomputes a halo in both directions: every CTA runs
// the row pass over 2 rk + 1 extra pixels of each row and over 2 rk extra rows.
// For large radii (or many channels, which narrow the strip) that overhead
// dominates.  Here the two 1D passes are separate launches joined by an FP32
// intermediate R in HBM (H x W x C, its own pitch):
//
//   row pass     one warp per row segment of up to ~1024 elements (+ halo),
//                staged by TMA, running sums (Eq. alg1) and the K-tap
//                differences (Eq. indep) with exactly the fused kernel's
//                row code, written to R with coalesced stores;
//   column pass  one CTA per column strip of CW element columns by TH rows:
//                TMA stages bands of B rows of R (8 to 32, by strip width),
//                the compensated column running sum J goes into a ring of
//                B-row blocks in shared memory (plus a mirror block), and each
//                output is sum_i w_i (J(y + r_i) - J(y - r_i - 1)).
//
// Only the column pass has a vertical halo (2 rk rows per tile, read from R),
// only the row pass a horizontal one (2 rk + 1 pixels per segment), and both
// tiles can be long in their own direction.  The waits are the bounded
// mbarrier waits of the strip kernel.
#pragma once

#include "strip_kernel.cuh"

namespace gb {

// ------------------------------------------------------------------ row pass
// Row filter at sampled pixels only (Sec. 3.4: Eq. indep needs nothing but the
// running sum, so it may be evaluated at any subset of the pixels).  Output o
// of the row segment (o = o0 + lane + 32 k, k < NQ) is channel o mod C of the
// segment's sampled pixel o / C, whose element sits at staged index
// s_first + (o / C) sx C + o mod C; offg[c] is the offset added back for
// channel c, and wscale the unit of the running sums (row_prefix).  Lanes past
// the segment's `nout` outputs recompute the last one (their results are not
// stored), so every load stays inside the staged row.
template <typename A, int C, int NQ, bool SPLIT = false>
__device__ __forceinline__ void row_taps_sampled(const KParams& p, const A* Q, const float* QL, int s_first, int o0,
                                                 int nout, const float* offg, float2* acc, int lane,
                                                 const RowScale& rs) {
    int s[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const int o = min(o0 + lane + 32 * k, nout - 1);
        const int t = o / C, c = o - t * C;
        s[k] = s_first + t * p.sx * C + c;
    }
#pragma unroll
    for (int h = 0; h < NQ / 2; ++h) {
        const int oa = min(o0 + lane + 64 * h, nout - 1), ob = min(o0 + lane + 64 * h + 32, nout - 1);
        acc[h] = make_float2(pick<C>(offg, oa % C) * p.sw, pick<C>(offg, ob % C) * p.sw);
    }
#pragma unroll
    for (int i = 0; i < GF_KMAX; ++i) {
        if (i < p.K) {
            const int ip = p.r[i] * C, im = (p.r[i] + 1) * C;
            const float2 w2 = make_float2(p.w[i], p.w[i]);
            const uint32_t cm = (uint32_t)(2 * p.r[i] + 1) * rs.bits_m;
#pragma unroll
            for (int h = 0; h < NQ / 2; ++h) {
                const int sa = s[2 * h], sb = s[2 * h + 1];
                float2 d;
                if constexpr (SPLIT) {
                    const float2 dh = make_float2((float)(int)((uint32_t)Q[sa + ip] - (uint32_t)Q[sa - im] - cm),
                                                  (float)(int)((uint32_t)Q[sb + ip] - (uint32_t)Q[sb - im] - cm));
                    const float2 dl = sub2(make_float2(QL[sa + ip], QL[sb + ip]), make_float2(QL[sa - im], QL[sb - im]));
                    d = fma2(dh, make_float2(rs.q, rs.q), dl);
                } else if constexpr (std::is_same<A, int>::value) {   // differences modulo 2^32
                    d = make_float2((float)(int)((uint32_t)Q[sa + ip] - (uint32_t)Q[sa - im]),
                                    (float)(int)((uint32_t)Q[sb + ip] - (uint32_t)Q[sb - im]));
                } else {
                    d = sub2(make_float2(Q[sa + ip], Q[sb + ip]), make_float2(Q[sa - im], Q[sb - im]));
                }
                acc[h] = fma2(w2, d, acc[h]);
            }
        }
    }
}

// KParams fields as for the strip kernel, with `out`/`out_pitch` naming R and
// TWp the segment width; there is no vertical halo.  With p.sx > 1 only the
// pixels x = ox + j sx are filtered and R holds them densely (element column
// j C + c).
// MODE: accumulation of float rows (gf_accum): 0 int32 sums of offset,
// power-of-two scaled values (exact differences), 1 FP32 sums with offsets,
// 2 plain FP32 running sums without offsets.
template <typename InT, int C, int MODE>
__device__ __forceinline__ void row_pass_tile(const KParams& p, const CUtensorMap* tmapp, const CUtensorMap* tmap8p,
                                              int bx, int by, unsigned char* smem) {
    using A = row_acc_t<InT, MODE>;
    InT* stage = reinterpret_cast<InT*>(smem + p.off_stage);
    A* pbuf = reinterpret_cast<A*>(smem + p.off_p);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + p.off_bar);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = bx * p.TWp;
    const int y0 = by * p.TH;
    if (x0 >= p.W || y0 >= p.H) return;
    const int yend = min(y0 + p.TH, p.H);
    const int nbands = (yend - y0 + kBand - 1) / kBand;
    const int ebase = floor_div((x0 - p.rk - 1) * C, p.ealign) * p.ealign;
    const int s_out0 = x0 * C - ebase;
    const bool hedge = (x0 - p.rk - 1 < 0) || (x0 + p.TWp + p.rk > p.W);
    const bool fixup = hedge && p.boundary != GF_ZERO && p.use_tma;
    const int rowlen = p.W * C;
    const int ecol0 = x0 * C;
    const int nvalid = min(p.TW, rowlen - ecol0);
    const int row_bytes = p.nbox * p.boxw * (int)sizeof(InT);

    if (tid == 0) {
        for (int s = 0; s < p.nstage; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    __syncthreads();

    auto issue_band = [&](int b, int slot) {
        InT* dst = stage + (size_t)slot * kBand * p.SROW;
        const int yb = y0 + b * kBand;
        if (p.rows8 && yb + kBand <= p.H) {   // the band is one 2D box (rows past yend are not used)
            if (lane == 0) {
                mbar_arrive_expect_tx(&bars[slot], (uint32_t)(kBand * row_bytes));
                fence_proxy_async();
                tma_load_row(dst, tmap8p, &bars[slot], ebase >> p.xshift, yb);
            }
            return;
        }
        const int y = yb + lane;
        const bool on = lane < kBand && y < yend;
        const unsigned valid = __ballot_sync(0xffffffffu, on);
        if (lane == 0) mbar_arrive_expect_tx(&bars[slot], (uint32_t)(__popc(valid) * row_bytes));
        __syncwarp();
        if (on) {
            fence_proxy_async();
            for (int k = 0; k < p.nbox; ++k)
                tma_load_row(dst + (size_t)lane * p.SROW + (size_t)k * p.boxw, tmapp, &bars[slot],
                             (ebase + k * p.boxw) >> p.xshift, y);
        }
    };
    int sidx = 0;
    uint32_t par = 0;
    if (p.use_tma && warp == 0)
        for (int b = 0; b < min(p.nstage, nbands); ++b) issue_band(b, b);

    bool ok = true;
    int band = 0;
    for (; band < nbands; ++band) {
        InT* sband = stage + (size_t)sidx * kBand * p.SROW;
        const int yb = y0 + band * kBand;
        if (p.use_tma) {
            const bool mine = mbar_wait_bounded(&bars[sidx], par, p.wait_limit);
            ok = __syncthreads_and(mine) != 0;
            if (!ok) break;
        } else {
            // plain loader: one warp per row, boundary folded while staging
            const int y = yb + warp;
            if (y < yend) {
                const InT* src = reinterpret_cast<const InT*>(p.in + (long long)y * p.in_pitch);
                InT* srow = sband + (size_t)warp * p.SROW;
                for (int i = lane; i < p.SROW; i += 32) {
                    const int g = ebase + i;
                    const int t = floor_div(g, C);
                    const int xs = fold_index(t, p.W, p.boundary);
                    InT val;
                    if (xs >= 0) val = src[xs * C + (g - t * C)];
                    else memset(&val, 0, sizeof(InT));
                    srow[i] = val;
                }
            }
            __syncwarp();
        }
        const int y = yb + warp;
        if (y < yend) {
            InT* srow = sband + (size_t)warp * p.SROW;
            if (fixup) {
                fold_halo<InT>(srow, p.SROW, ebase, C, p.W, p.boundary, lane);
                __syncwarp();
            }
            float off[C], offg[C];
            row_offsets<InT, C>(srow, s_out0, off, offg);
            constexpr bool SPLIT = !Elem<InT>::exact && MODE == 0;   // float rows: integer part + residues
            if constexpr (MODE == 2 || SPLIT) {
#pragma unroll
                for (int c = 0; c < C; ++c) off[c] = offg[c] = 0.f;
            }
            A* Q = std::is_same<InT, float>::value ? reinterpret_cast<A*>(srow) : pbuf + (size_t)warp * p.SP;
            float* QL = reinterpret_cast<float*>(smem + p.off_pl) + (size_t)warp * p.SP;
            RowScale wsc;
            row_prefix<InT, C, MODE>(srow, Q, QL, p.m, off, lane, wsc, p.rk, s_out0 - (p.rk + 1) * C,
                                     s_out0 + nvalid + p.rk * C);
            if (p.sx > 1) {
                // sampled pixels of the segment: xf, xf + sx, ... below xend
                const int xend = min(x0 + p.TWp, p.W);
                const int xf = x0 + ((p.ox - x0) % p.sx + p.sx) % p.sx;
                const int nout = xf < xend ? ((xend - 1 - xf) / p.sx + 1) * C : 0;
                float* dst = reinterpret_cast<float*>(p.out + (long long)y * p.out_pitch) + ((xf - p.ox) / p.sx) * C;
                const int s_first = s_out0 + (xf - x0) * C;
                for (int o0 = 0; o0 < nout; o0 += 256) {
                    float2 acc[4];
                    row_taps_sampled<A, C, 8, SPLIT>(p, Q, QL, s_first, o0, nout, offg, acc, lane, wsc);
                    const int nv = nout - o0;
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int ea = lane + 64 * h;
                        if (ea < nv) dst[o0 + ea] = acc[h].x;
                        if (ea + 32 < nv) dst[o0 + ea + 32] = acc[h].y;
                    }
                }
            } else {
                float* dst = reinterpret_cast<float*>(p.out + (long long)y * p.out_pitch) + ecol0;
                for (int c0 = 0; c0 < nvalid; c0 += 256) {
                    float offc[C];   // chunk element e is segment element c0 + e
#pragma unroll
                    for (int c = 0; c < C; ++c) offc[c] = pick<C>(offg, (c0 + c) % C);
                    float2 acc[4];
                    row_taps<A, C, 8, SPLIT>(p, Q, QL, s_out0 + c0, offc, acc, lane, wsc);
                    const int nv = nvalid - c0;
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int ea = lane + 64 * h;
                        if (ea < nv) dst[c0 + ea] = acc[h].x;
                        if (ea + 32 < nv) dst[c0 + ea + 32] = acc[h].y;
                    }
                }
            }
        }
        __syncthreads();   // every warp is done with the slot
        if (p.use_tma && warp == 0 && band + p.nstage < nbands) issue_band(band + p.nstage, sidx);
        if (++sidx == p.nstage) {
            sidx = 0;
            par ^= 1u;
        }
    }
    if (!ok && tid == 0) {
        atomicCAS(p.status, 0, (int)GF_ETIMEOUT);
        int sl = sidx;
        uint32_t pa = par;
        for (int b = band; b < min(band + p.nstage, nbands); ++b) {
            (void)mbar_wait_bounded(&bars[sl], pa);
            if (++sl == p.nstage) { sl = 0; pa ^= 1u; }
        }
    }
}

template <typename InT, int C, int MODE>
__global__ void __launch_bounds__(kThreads, 3) row_pass_kernel(const __grid_constant__ CUtensorMap tmap,
                                                             const __grid_constant__ CUtensorMap tmap8,
                                                             const KParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    row_pass_tile<InT, C, MODE>(p, &tmap, &tmap8, blockIdx.x, blockIdx.y, smem);
}

// --------------------------------------------------------------- column pass
struct CParams {
    const unsigned char* rin;   // R, FP32
    long long r_pitch;
    unsigned char* out;
    long long out_pitch;
    int* status;
    long long wait_limit;   // SM clock cycles per pipeline wait
    int H, rowlen, boundary;
    int K;
    int r[GF_KMAX];
    float w[GF_KMAX];
    float sw;
    int rk;
    int TH;            // output rows per CTA
    int NB;            // ring blocks of kBand rows (a mirror block follows)
    int nstage, use_tma;
    int pair_ok;       // output base and pitch allow 2-element stores
    int B;             // rows per band (the kernel's BAND)
    int sy, oy;        // outputs only at rows y = oy + i sy, stored as row i (sy <= 1: every row)
    int zcol;          // blockIdx.z adds z zcol to the element column read from R,
    int zrow;          // z zrow to the row of R (folding stays within the H rows of a plane)
    long long zout;    // and z zout bytes to the output address (one launch over z planes)
    int off_stage, off_ring, off_coff, off_bar;
};

// Default rows per band of the column pass.  Narrow strips (large radii) take
// 16-row bands, which give every thread tap rows and amortise the per-band
// wait, barriers and ring bookkeeping; wide strips keep 8-row bands, whose
// smaller ring and stage leave room for four CTAs per SM.  32-column strips
// also exist with 32-row bands (two rows per thread), which the host takes
// when they keep as many CTAs per SM as 16-row bands do.
__host__ __device__ constexpr int col_band(int CW) { return CW <= 64 ? 16 : kBand; }

// Strips of up to 128 columns sum each band in all threads, the TPP threads of
// a column pair being consecutive lanes joined by a shuffle scan; 256-column
// strips let one thread per pair sum the band (their padded band would exceed
// the 256-element TMA box, and half the threads are pair threads anyway).
__host__ __device__ constexpr bool col_lane_sums(int CW) { return CW <= 128; }
// Row stride (floats) of the column ring: padded for lane sums, so that the
// 64-bit accesses of a half-warp, which then span TPP ring rows, fall on
// distinct bank pairs.
__host__ __device__ constexpr int col_ring_stride(int CW) {
    return col_lane_sums(CW) ? CW + (CW >= 128 ? 4 : 2) : CW;
}
// Row stride (floats) of a staged band.  With lane sums the pair's lanes read
// TPP different staged rows of the same columns: interior bands are then one
// 2D TMA box CW + 4 floats wide (rows stay 16-byte multiples; the extra
// columns are never read), so those rows do not share banks; other strips
// stage dense rows one box per row.
__host__ __device__ constexpr int col_stage_stride(int CW) { return col_lane_sums(CW) ? CW + 4 : CW; }

// N consecutive ring rows of one column pair: 64-bit loads at `addr` + j STRIDE.
template <int N, int STRIDE, int J = 0>
__device__ __forceinline__ void tap_rows(uint32_t addr, float2* v) {
    if constexpr (J < N) {
        v[J] = lds2<J * STRIDE>(addr);
        tap_rows<N, STRIDE, J + 1>(addr, v);
    }
}

// CW element columns per CTA, handled as CW / 2 column pairs (64-bit shared
// accesses, packed f32x2 arithmetic).  With lane sums a band whose rows are all
// inside the image is staged by one 2D box of the band map; a band with rows
// folded by the boundary rule is loaded by the CTA's threads (its mbarrier
// phase is completed by a plain arrive).  Thread q of the TPP = 2 kThreads / CW
// threads of a pair forms the taps of RPT = BAND / TPP rows of every band:
// rows [q RPT, (q + 1) RPT), or, with lane sums and RPT > 1, rows q, q + TPP,
// ... (so that consecutive lanes read consecutive ring rows, in distinct bank
// pairs).  With lane sums (narrow strips) the pair's threads are consecutive
// lanes: each sums its own rows and a shuffle scan over the pair's lanes
// gives it the band-local prefix (one scan per sub-band of TPP rows when the
// rows are strided).  Otherwise thread t < CW / 2 sums all rows of pair t.  The only CTA barriers are the band
// wait and the one before the taps.
template <typename OutT, int CW, int MODE, int BAND>
__device__ __forceinline__ void col_pass_tile(const CParams& p, const CUtensorMap* tmapp, const CUtensorMap* bmapp,
                                              int bx, int by, int bz, unsigned char* smem) {
    constexpr int B = BAND;
    constexpr int NP = CW / 2;                  // column pairs
    constexpr int TPP = kThreads / NP;          // threads (lanes) per pair
    constexpr int RPT = B / TPP;                // rows per thread
    constexpr int RS = col_ring_stride(CW);     // ring row stride (floats)
    constexpr int SS = col_stage_stride(CW);    // staged row stride (floats)
    constexpr bool LS = col_lane_sums(CW);
    // With lane sums and several rows per thread, thread q of a pair takes
    // rows q, q + TPP, ... of the band: consecutive lanes then read consecutive
    // ring rows, which the padded row stride puts in distinct bank pairs.
    constexpr int RSTEP = (LS && RPT > 1) ? TPP : 1;
    static_assert(CW % 2 == 0 && RPT >= 1 && RPT * TPP == B && TPP <= 32, "column strip width");
    float* stage = reinterpret_cast<float*>(smem + p.off_stage);
    float* ring = reinterpret_cast<float*>(smem + p.off_ring);
    float2* coffs = reinterpret_cast<float2*>(smem + p.off_coff);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + p.off_bar);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ecol0 = bx * CW;
    const int y0 = by * p.TH;
    if (ecol0 >= p.rowlen || y0 >= p.H) return;
    const int xcol0 = ecol0 + bz * p.zcol;   // element column of the strip in R
    const int zr = bz * p.zrow;                // row of R of the plane's row 0
    const int yend = min(y0 + p.TH, p.H);
    const int vstart = y0 - p.rk;
    const int vend = yend - 1 + p.rk;
    const int nbands = (vend - vstart + 1 + B - 1) / B;
    const int ringrows = p.NB * B;
    const int pr = LS ? tid / TPP : tid % NP;   // column pair of the taps
    const int q = LS ? tid % TPP : tid / NP;    // row group within the band
    const int j0 = RSTEP > 1 ? q : q * RPT;
    // shared address of this thread's column pair in ring row 0; the lo ring
    // (MODE 0) follows the hi ring and its mirror block
    const uint32_t ring_s = smem_addr(ring) + (uint32_t)(pr * 8);
    float* const ring_lo = ring + (p.NB + 1) * B * RS;
    const uint32_t ring_lo_s = ring_s + (uint32_t)((p.NB + 1) * B * RS * 4);

    if (tid == 0) {
        for (int s = 0; s < p.nstage; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    // J(vstart - 1) = 0 sits in the last logical ring row
    if (q == 0) {
        reinterpret_cast<float2*>(ring + (ringrows - 1) * RS)[pr] = make_float2(0.f, 0.f);
        if (MODE == 0) reinterpret_cast<float2*>(ring_lo + (ringrows - 1) * RS)[pr] = make_float2(0.f, 0.f);
    }
    __syncthreads();

    // interior band: every row in the image, so no row is folded
    auto interior = [&](int b) {
        const int vb = vstart + b * B;
        return vb >= 0 && vb + B <= p.H;
    };
    // warp 0 stages band b: lane l loads rows l, l + 32, ... (folded by the
    // boundary rule); lane 0 posts the byte count
    auto issue_band = [&](int b, int slot) {
        float* dst = stage + slot * (B * SS);
        if constexpr (LS) {
            if (lane == 0) {
                if (interior(b)) {
                    mbar_arrive_expect_tx(&bars[slot], (uint32_t)(B * SS * 4));
                    fence_proxy_async();
                    tma_load_row(dst, bmapp, &bars[slot], xcol0, zr + vstart + b * B);
                } else {
                    mbar_arrive(&bars[slot]);   // loaded by the threads when consumed
                }
            }
            return;
        }
        int yr[(B + 31) / 32];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < (B + 31) / 32; ++k) {
            const int rr = lane + 32 * k;
            const int v = vstart + b * B + rr;
            yr[k] = (rr < B && v <= vend) ? fold_index(v, p.H, p.boundary) : -1;
            cnt += __popc(__ballot_sync(0xffffffffu, yr[k] >= 0));
        }
        if (lane == 0) mbar_arrive_expect_tx(&bars[slot], (uint32_t)(cnt * CW * 4));
        __syncwarp();
#pragma unroll
        for (int k = 0; k < (B + 31) / 32; ++k) {
            if (yr[k] >= 0) {
                fence_proxy_async();
                tma_load_row(dst + (lane + 32 * k) * CW, tmapp, &bars[slot], xcol0, zr + yr[k]);
            }
        }
    };
    int sidx = 0;
    uint32_t par = 0;
    if (p.use_tma && warp == 0)
        for (int b = 0; b < min(p.nstage, nbands); ++b) issue_band(b, b);

    const int c0 = ecol0 + 2 * pr;              // first element column of the pair
    const bool pair_on = c0 + 1 < p.rowlen;
    const bool single_on = c0 < p.rowlen;
    // column carry (hi + lo) and offset: of pair pr with lane sums, of pair
    // tid (tid < CW / 2) otherwise
    float2 jh = make_float2(0.f, 0.f), jl = make_float2(0.f, 0.f), coff = make_float2(0.f, 0.f);
    unsigned char* const out0 = p.out + (long long)bz * p.zout + (long long)c0 * (long long)sizeof(OutT);
    // per-tap ring offsets relative to the band's first ring row
    int dp[GF_KMAX], dm[GF_KMAX];
    float2 w2[GF_KMAX];
#pragma unroll
    for (int i = 0; i < GF_KMAX; ++i) {
        const int r = i < p.K ? p.r[i] : 0;
        dp[i] = j0 + r - p.rk;
        dm[i] = j0 - p.rk - r - 1;
        w2[i] = make_float2(p.w[i], p.w[i]);
    }
    const unsigned gmask = 0xffffffffu;
    bool ok = true;
    int band = 0, blk = 0;
    for (; band < nbands; ++band) {
        float* const sband = stage + sidx * (B * SS);
        const int v0 = vstart + band * B;
        // plain loader: folds rows while staging (all bands without TMA, the
        // bands with folded rows under lane sums)
        auto plain_load = [&]() {
            for (int i = tid; i < B * CW; i += kThreads) {
                const int r = i / CW, c = i % CW;
                const int v = v0 + r;
                const int yr = v <= vend ? fold_index(v, p.H, p.boundary) : -1;
                float val = 0.f;
                if (yr >= 0 && ecol0 + c < p.rowlen)
                    val = reinterpret_cast<const float*>(p.rin + (long long)(zr + yr) * p.r_pitch)[xcol0 + c];
                sband[r * SS + c] = val;
            }
        };
        if (p.use_tma) {
            const bool mine = mbar_wait_bounded(&bars[sidx], par, p.wait_limit);
            ok = __syncthreads_and(mine) != 0;
            if (!ok) break;
            if (LS && !interior(band)) {
                plain_load();
                __syncthreads();
            }
        } else {
            __syncthreads();
            plain_load();
            __syncthreads();
        }
        // ---- column running sums of the band
        if constexpr (!LS) {
            if (tid < NP) {
                const bool inner = v0 >= 0 && v0 + B - 1 < p.H && v0 + B - 1 <= vend;
                const float2* xs = reinterpret_cast<const float2*>(sband) + tid;   // SS == CW here
                float2* wr = reinterpret_cast<float2*>(ring + blk * (B * RS)) + tid;
                float2* wm = reinterpret_cast<float2*>(ring + ringrows * RS) + tid;
                if (band == 0) {
                    coff = MODE != 1 ? make_float2(0.f, 0.f) : xs[0];
                    if (!inner && p.boundary == GF_ZERO && (v0 < 0 || v0 >= p.H)) coff = make_float2(0.f, 0.f);
                    coffs[tid] = coff;
                }
                float2* wrl = reinterpret_cast<float2*>(ring_lo + blk * (B * RS)) + tid;
                float2* wml = reinterpret_cast<float2*>(ring_lo + ringrows * RS) + tid;
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    float2 x = xs[j * NP];
                    if (!inner) {
                        const int v = v0 + j;
                        const bool on = v <= vend && (p.boundary != GF_ZERO || (v >= 0 && v < p.H));
                        if (!on) x = make_float2(0.f, 0.f);
                    }
                    if constexpr (MODE == 0) {
                        // J = jh + jl: FP32 running sum plus its exact rounding errors
                        float2 sum, err;
                        two_sum2(jh, x, sum, err);
                        jh = sum;
                        jl = add2(jl, err);
                        wr[j * (RS / 2)] = jh;
                        wrl[j * (RS / 2)] = jl;
                        if (blk == 0) {
                            wm[j * (RS / 2)] = jh;
                            wml[j * (RS / 2)] = jl;
                        }
                    } else {
                        jh = add2(jh, sub2(x, coff));
                        wr[j * (RS / 2)] = jh;
                        if (blk == 0) wm[j * (RS / 2)] = jh;
                    }
                }
            }
        } else {
            // rows that were not loaded (ZERO boundary, past the tile) read as 0
            const bool inner = v0 >= 0 && v0 + B - 1 < p.H && v0 + B - 1 <= vend;
            float2 x[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                x[j] = reinterpret_cast<const float2*>(sband + (j0 + j * RSTEP) * SS)[pr];
                if (!inner) {
                    const int v = v0 + j0 + j * RSTEP;
                    const bool on = v <= vend && (p.boundary != GF_ZERO || (v >= 0 && v < p.H));
                    if (!on) x[j] = make_float2(0.f, 0.f);
                }
            }
            if (band == 0) {   // the column offset (study mode 1): the pair's first staged value
                const float cx = __shfl_sync(gmask, x[0].x, 0, TPP);
                const float cy = __shfl_sync(gmask, x[0].y, 0, TPP);
                coff = MODE != 1 ? make_float2(0.f, 0.f) : make_float2(cx, cy);
            }
            if constexpr (MODE == 0 && RSTEP > 1) {
                // row j0 + j TPP: the sums of the earlier sub-bands of TPP rows
                // plus a scan over the pair's lanes of sub-band j, as (hi, lo) pairs
                float2 sh = make_float2(0.f, 0.f), sl = make_float2(0.f, 0.f);
                float2* wr = reinterpret_cast<float2*>(ring + (blk * B + j0) * RS) + pr;
                float2* wm = reinterpret_cast<float2*>(ring + (ringrows + j0) * RS) + pr;
                float2* wrl = reinterpret_cast<float2*>(ring_lo + (blk * B + j0) * RS) + pr;
                float2* wml = reinterpret_cast<float2*>(ring_lo + (ringrows + j0) * RS) + pr;
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    float2 ih = x[j], il = make_float2(0.f, 0.f);
#pragma unroll
                    for (int d = 1; d < TPP; d <<= 1) {
                        const float2 oh = make_float2(__shfl_up_sync(gmask, ih.x, d, TPP), __shfl_up_sync(gmask, ih.y, d, TPP));
                        const float2 ol = make_float2(__shfl_up_sync(gmask, il.x, d, TPP), __shfl_up_sync(gmask, il.y, d, TPP));
                        if (q >= d) dd_add2(oh, ol, ih, il, ih, il);
                    }
                    float2 bh, bl, Jh, Jl;
                    dd_add2(sh, sl, ih, il, bh, bl);   // band-local prefix up to this row
                    dd_add2(jh, jl, bh, bl, Jh, Jl);
                    wr[j * RSTEP * (RS / 2)] = Jh;
                    wrl[j * RSTEP * (RS / 2)] = Jl;
                    if (blk == 0) {
                        wm[j * RSTEP * (RS / 2)] = Jh;
                        wml[j * RSTEP * (RS / 2)] = Jl;
                    }
                    const float2 toth = make_float2(__shfl_sync(gmask, ih.x, TPP - 1, TPP), __shfl_sync(gmask, ih.y, TPP - 1, TPP));
                    const float2 totl = make_float2(__shfl_sync(gmask, il.x, TPP - 1, TPP), __shfl_sync(gmask, il.y, TPP - 1, TPP));
                    dd_add2(sh, sl, toth, totl, sh, sl);
                }
                dd_add2(jh, jl, sh, sl, jh, jl);
            } else if constexpr (MODE != 0 && RSTEP > 1) {
                // the same with plain FP32 sums (study modes)
                float2 sacc = make_float2(0.f, 0.f);
                float2* wr = reinterpret_cast<float2*>(ring + (blk * B + j0) * RS) + pr;
                float2* wm = reinterpret_cast<float2*>(ring + (ringrows + j0) * RS) + pr;
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    float2 inc = sub2(x[j], coff);
#pragma unroll
                    for (int d = 1; d < TPP; d <<= 1) {
                        const float ox = __shfl_up_sync(gmask, inc.x, d, TPP);
                        const float oy = __shfl_up_sync(gmask, inc.y, d, TPP);
                        if (q >= d) inc = add2(inc, make_float2(ox, oy));
                    }
                    const float2 J = add2(jh, add2(sacc, inc));
                    wr[j * RSTEP * (RS / 2)] = J;
                    if (blk == 0) wm[j * RSTEP * (RS / 2)] = J;
                    sacc = add2(sacc, make_float2(__shfl_sync(gmask, inc.x, TPP - 1, TPP),
                                                  __shfl_sync(gmask, inc.y, TPP - 1, TPP)));
                }
                jh = add2(jh, sacc);
            } else if constexpr (MODE == 0) {
                // band-local running sums of this lane's rows as (hi, lo) pairs,
                // joined over the pair's lanes by a scan of (hi, lo) pairs, then
                // added to the carried column sum: every ring entry is J = hi + lo
                float2 Lh[RPT], Ll[RPT];
                float2 lh = make_float2(0.f, 0.f), ll = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    float2 sum, err;
                    two_sum2(lh, x[j], sum, err);
                    lh = sum;
                    ll = add2(ll, err);
                    Lh[j] = lh;
                    Ll[j] = ll;
                }
                float2 ih = lh, il = ll;
#pragma unroll
                for (int d = 1; d < TPP; d <<= 1) {
                    const float2 oh = make_float2(__shfl_up_sync(gmask, ih.x, d, TPP), __shfl_up_sync(gmask, ih.y, d, TPP));
                    const float2 ol = make_float2(__shfl_up_sync(gmask, il.x, d, TPP), __shfl_up_sync(gmask, il.y, d, TPP));
                    if (q >= d) dd_add2(oh, ol, ih, il, ih, il);
                }
                const float2 ph0 = make_float2(__shfl_up_sync(gmask, ih.x, 1, TPP), __shfl_up_sync(gmask, ih.y, 1, TPP));
                const float2 pl0 = make_float2(__shfl_up_sync(gmask, il.x, 1, TPP), __shfl_up_sync(gmask, il.y, 1, TPP));
                const float2 preh = q == 0 ? make_float2(0.f, 0.f) : ph0;
                const float2 prel = q == 0 ? make_float2(0.f, 0.f) : pl0;
                const float2 toth = make_float2(__shfl_sync(gmask, ih.x, TPP - 1, TPP), __shfl_sync(gmask, ih.y, TPP - 1, TPP));
                const float2 totl = make_float2(__shfl_sync(gmask, il.x, TPP - 1, TPP), __shfl_sync(gmask, il.y, TPP - 1, TPP));
                float2* wr = reinterpret_cast<float2*>(ring + (blk * B + j0) * RS) + pr;
                float2* wm = reinterpret_cast<float2*>(ring + (ringrows + j0) * RS) + pr;
                float2* wrl = reinterpret_cast<float2*>(ring_lo + (blk * B + j0) * RS) + pr;
                float2* wml = reinterpret_cast<float2*>(ring_lo + (ringrows + j0) * RS) + pr;
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    float2 bh, bl, Jh, Jl;
                    dd_add2(preh, prel, Lh[j], Ll[j], bh, bl);   // band-local prefix up to this row
                    dd_add2(jh, jl, bh, bl, Jh, Jl);
                    wr[j * (RS / 2)] = Jh;
                    wrl[j * (RS / 2)] = Jl;
                    if (blk == 0) {
                        wm[j * (RS / 2)] = Jh;
                        wml[j * (RS / 2)] = Jl;
                    }
                }
                dd_add2(jh, jl, toth, totl, jh, jl);
            } else {
            float2 Lv[RPT];
            float2 loc = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                loc = add2(loc, sub2(x[j], coff));
                Lv[j] = loc;
            }
            // inclusive scan of the row-group sums over the pair's lanes
            float2 inc = loc;
#pragma unroll
            for (int d = 1; d < TPP; d <<= 1) {
                const float ox = __shfl_up_sync(gmask, inc.x, d, TPP);
                const float oy = __shfl_up_sync(gmask, inc.y, d, TPP);
                if (q >= d) inc = add2(inc, make_float2(ox, oy));
            }
            float px = __shfl_up_sync(gmask, inc.x, 1, TPP);
            float py = __shfl_up_sync(gmask, inc.y, 1, TPP);
            const float2 pre = q == 0 ? make_float2(0.f, 0.f) : make_float2(px, py);   // earlier rows of the band
            const float2 tot = make_float2(__shfl_sync(gmask, inc.x, TPP - 1, TPP),
                                           __shfl_sync(gmask, inc.y, TPP - 1, TPP));
            float2* wr = reinterpret_cast<float2*>(ring + (blk * B + j0) * RS) + pr;
            float2* wm = reinterpret_cast<float2*>(ring + (ringrows + j0) * RS) + pr;
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                const float2 J = add2(jh, add2(pre, Lv[j]));
                wr[j * (RS / 2)] = J;
                if (blk == 0) wm[j * (RS / 2)] = J;
            }
            jh = add2(jh, tot);
            }
        }
        __syncthreads();   // J rows visible, stage slot free
        if (p.use_tma && warp == 0 && band + p.nstage < nbands) issue_band(band + p.nstage, sidx);

        // ---- taps: output rows y = v0 + j - rk
        if (v0 + B - 1 - p.rk >= y0) {
            float2 acc[RPT];
            const float2 cf = LS ? coff : coffs[pr];
            const float2 base = make_float2(cf.x * p.sw, cf.y * p.sw);
#pragma unroll
            for (int j = 0; j < RPT; ++j) acc[j] = base;
            const int rb = blk * B;
#pragma unroll
            for (int i = 0; i < GF_KMAX; ++i) {
                if (i < p.K) {
                    int ap = rb + dp[i];
                    ap = ap < 0 ? ap + ringrows : ap;
                    int am = rb + dm[i];
                    am = am < 0 ? am + ringrows : am;
                    // 32-bit shared addresses; the rows of the window are immediate offsets
                    const uint32_t sp = ring_s + (uint32_t)(ap * (RS * 4));
                    const uint32_t sm = ring_s + (uint32_t)(am * (RS * 4));
                    float2 a[RPT], b[RPT];
                    tap_rows<RPT, RSTEP * RS * 4>(sp, a);
                    tap_rows<RPT, RSTEP * RS * 4>(sm, b);
                    if constexpr (MODE == 0) {
                        // (hi difference) + (lo difference): accurate to the window's own sum
                        const uint32_t off_lo = ring_lo_s - ring_s;
                        float2 al[RPT], bl[RPT];
                        tap_rows<RPT, RSTEP * RS * 4>(sp + off_lo, al);
                        tap_rows<RPT, RSTEP * RS * 4>(sm + off_lo, bl);
#pragma unroll
                        for (int j = 0; j < RPT; ++j)
                            acc[j] = fma2(w2[i], add2(sub2(a[j], b[j]), sub2(al[j], bl[j])), acc[j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < RPT; ++j) acc[j] = fma2(w2[i], sub2(a[j], b[j]), acc[j]);
                    }
                }
            }
            const int ya = v0 + j0 - p.rk;
            auto store = [&](unsigned char* o, float2 v) {
                if (pair_on && p.pair_ok) {
                    store_pair<OutT>(reinterpret_cast<OutT*>(o), v);
                } else {
                    if (single_on) *reinterpret_cast<OutT*>(o) = from_float<OutT>(v.x);
                    if (pair_on) reinterpret_cast<OutT*>(o)[1] = from_float<OutT>(v.y);
                }
            };
            if (p.sy <= 1) {
                unsigned char* o = out0 + (long long)ya * p.out_pitch;
                const bool full = ya >= y0 && ya + (RPT - 1) * RSTEP < yend;
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    if (full || (ya + j * RSTEP >= y0 && ya + j * RSTEP < yend)) store(o, acc[j]);
                    o += (long long)RSTEP * p.out_pitch;
                }
            } else {
                // sampled rows only: y = oy + i sy goes to output row i
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const int t = ya + j * RSTEP - p.oy;
                    if (ya + j * RSTEP >= y0 && ya + j * RSTEP < yend && t >= 0 && t % p.sy == 0)
                        store(out0 + (long long)(t / p.sy) * p.out_pitch, acc[j]);
                }
            }
        }
        blk = (blk + 1 == p.NB) ? 0 : blk + 1;
        if (++sidx == p.nstage) {
            sidx = 0;
            par ^= 1u;
        }
    }
    if (!ok && tid == 0) {
        atomicCAS(p.status, 0, (int)GF_ETIMEOUT);
        int sl = sidx;
        uint32_t pa = par;
        for (int b = band; b < min(band + p.nstage, nbands); ++b) {
            (void)mbar_wait_bounded(&bars[sl], pa);
            if (++sl == p.nstage) { sl = 0; pa ^= 1u; }
        }
    }
}

template <typename OutT, int CW, int MODE, int BAND>
__global__ void __launch_bounds__(kThreads, 4) col_pass_kernel(const __grid_constant__ CUtensorMap tmap,
                                                             const __grid_constant__ CUtensorMap bmap,
                                                             const CParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    col_pass_tile<OutT, CW, MODE, BAND>(p, &tmap, &bmap, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

// ---------------------------------------------------------------- launchers
template <typename InT>
gf_status launch_row_pass(const KParams& kp, const CUtensorMap* maps, dim3 grid, size_t smem, cudaStream_t s,
                          int mode) {
    void (*kern)(const CUtensorMap, const CUtensorMap, const KParams) = nullptr;
    if (Elem<InT>::exact) mode = 0;   // integer rows are exact in every mode
    if (mode == 0) {
        switch (kp.C) {
            case 1: kern = row_pass_kernel<InT, 1, 0>; break;
            case 2: kern = row_pass_kernel<InT, 2, 0>; break;
            case 3: kern = row_pass_kernel<InT, 3, 0>; break;
            case 4: kern = row_pass_kernel<InT, 4, 0>; break;
            default: return GF_EUNSUPPORTED;
        }
    } else {
        // study variants: float rows, one channel
        if constexpr (!Elem<InT>::exact) {
            if (kp.C == 1) kern = mode == 1 ? row_pass_kernel<InT, 1, 1> : row_pass_kernel<InT, 1, 2>;
        }
        if (!kern) return GF_EUNSUPPORTED;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    kern<<<grid, kThreads, smem, s>>>(maps[0], maps[1], kp);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

template <typename OutT, int MODE>
void (*col_pass_for(int CW, int B))(const CUtensorMap, const CUtensorMap, const CParams) {
    switch (CW) {
        case 32: return B == 32 ? col_pass_kernel<OutT, 32, MODE, 32> : col_pass_kernel<OutT, 32, MODE, col_band(32)>;
        case 64: return col_pass_kernel<OutT, 64, MODE, col_band(64)>;
        case 128: return col_pass_kernel<OutT, 128, MODE, col_band(128)>;
        case 256: return col_pass_kernel<OutT, 256, MODE, col_band(256)>;
        default: return nullptr;
    }
}

template <typename OutT>
gf_status launch_col_pass(const CParams& cp, const CUtensorMap* maps, int CW, dim3 grid, size_t smem,
                          cudaStream_t s, int mode) {
    void (*kern)(const CUtensorMap, const CUtensorMap, const CParams) = nullptr;
    if (mode == 0) {
        kern = col_pass_for<OutT, 0>(CW, cp.B);
    } else {
        // study variants: f32 and bf16 outputs
        if constexpr (!std::is_same<OutT, __half>::value)
            kern = mode == 1 ? col_pass_for<OutT, 1>(CW, cp.B) : col_pass_for<OutT, 2>(CW, cp.B);
    }
    if (!kern) return GF_EUNSUPPORTED;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    kern<<<grid, kThreads, smem, s>>>(maps[0], maps[1], cp);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

// ------------------------------------------------------------ batched launches
// Up to kTPBatchMax two-pass images that share a row kernel (input type,
// channels) run as one launch of row tiles, and those that share a column
// kernel (output type, strip width, band) as one launch of column tiles: one
// CTA per tile, its image found in the prefix sums of the images' tile
// counts.  The images' parameters travel in the launch's own parameter space,
// read-only for the whole launch, so the tile code reads them exactly as in
// the one-image kernels; the tensor maps stay in global memory.
constexpr int kTPBatchMax = 32;

struct TPRows {
    KParams kp[kTPBatchMax];
    const CUtensorMap* maps;          // [2 nimg]: row map, 8-row map
    int tile_start[kTPBatchMax + 1];  // prefix sums of tiles per image
    int nimg;
};

struct TPCols {
    CParams cp[kTPBatchMax];
    const CUtensorMap* maps;          // [2 nimg]: row map, band map
    int tile_start[kTPBatchMax + 1];
    int nimg;
};

static_assert(sizeof(TPRows) <= 32000 && sizeof(TPCols) <= 32000, "kernel parameter space");

// The image of tile t: the last image whose first tile is at most t (every
// thread searches; the result is uniform across the CTA).
template <typename A>
__device__ __forceinline__ int tp_batch_image(const A& a, int t) {
    int lo = 0, hi = a.nimg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.tile_start[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename InT, int C>
__global__ void __launch_bounds__(kThreads, 3) row_pass_batch_kernel(const __grid_constant__ TPRows a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int t = (int)blockIdx.x;
    const int img = tp_batch_image(a, t);
    const KParams& p = a.kp[img];
    const int local = t - a.tile_start[img];
    const int nx = (p.W + p.TWp - 1) / p.TWp;
    row_pass_tile<InT, C, 0>(p, a.maps + 2 * img, a.maps + 2 * img + 1, local % nx, local / nx, smem);
}

template <typename OutT, int CW, int BAND>
__global__ void __launch_bounds__(kThreads, 4) col_pass_batch_kernel(const __grid_constant__ TPCols a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int t = (int)blockIdx.x;
    const int img = tp_batch_image(a, t);
    const CParams& p = a.cp[img];
    const int local = t - a.tile_start[img];
    const int nx = (p.rowlen + CW - 1) / CW;
    col_pass_tile<OutT, CW, 0, BAND>(p, a.maps + 2 * img, a.maps + 2 * img + 1, local % nx, local / nx, 0, smem);
}

template <typename InT>
gf_status launch_row_pass_batch(const TPRows& a, int C, int tiles, size_t smem, cudaStream_t s) {
    void (*kern)(const TPRows) = nullptr;
    switch (C) {
        case 1: kern = row_pass_batch_kernel<InT, 1>; break;
        case 2: kern = row_pass_batch_kernel<InT, 2>; break;
        case 3: kern = row_pass_batch_kernel<InT, 3>; break;
        case 4: kern = row_pass_batch_kernel<InT, 4>; break;
        default: return GF_EUNSUPPORTED;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    kern<<<tiles, kThreads, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

template <typename OutT>
gf_status launch_col_pass_batch(const TPCols& a, int CW, int B, int tiles, size_t smem, cudaStream_t s) {
    void (*kern)(const TPCols) = nullptr;
    switch (CW) {
        case 32: kern = B == 32 ? col_pass_batch_kernel<OutT, 32, 32> : col_pass_batch_kernel<OutT, 32, col_band(32)>; break;
        case 64: kern = col_pass_batch_kernel<OutT, 64, col_band(64)>; break;
        case 128: kern = col_pass_batch_kernel<OutT, 128, col_band(128)>; break;
        case 256: kern = col_pass_batch_kernel<OutT, 256, col_band(256)>; break;
        default: return GF_EUNSUPPORTED;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    kern<<<tiles, kThreads, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

#define GB_DECLARE_ROWPASS(IN)                                                                                 \
    extern template gf_status launch_row_pass<IN>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, \
                                                  int);                                                            \
    extern template gf_status launch_row_pass_batch<IN>(const TPRows&, int, int, size_t, cudaStream_t);
#define GB_DECLARE_COLPASS(OUT)                                                                             \
    extern template gf_status launch_col_pass<OUT>(const CParams&, const CUtensorMap*, int, dim3, size_t, \
                                                   cudaStream_t, int);                                      \
    extern template gf_status launch_col_pass_batch<OUT>(const TPCols&, int, int, int, size_t, cudaStream_t);

}  // namespace gb
