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
//                TMA stages kBand-row bands of R, the compensated column
//                running sum J goes into a ring of kBand-row blocks in shared
//                memory (plus a mirror block), and each output is
//                sum_i w_i (J(y + r_i) - J(y - r_i - 1)).
//
// Only the column pass has a vertical halo (2 rk rows per tile, read from R),
// only the row pass a horizontal one (2 rk + 1 pixels per segment), and both
// tiles can be long in their own direction.  The waits are the bounded
// mbarrier waits of the strip kernel.
#pragma once

#include "strip_kernel.cuh"

namespace gb {

// ------------------------------------------------------------------ row pass
// KParams fields as for the strip kernel, with `out`/`out_pitch` naming R and
// TWp the segment width; there is no vertical halo.
// MODE: accumulation of float rows (gf_accum): 0 compensated, 1 offsets with
// plain FP32 carries, 2 plain FP32 running sums without offsets.
template <typename InT, int C, int MODE>
__global__ void __launch_bounds__(kThreads, 3) row_pass_kernel(const __grid_constant__ CUtensorMap tmap,
                                                             const KParams p) {
    using A = typename Elem<InT>::acc;
    extern __shared__ __align__(128) unsigned char smem[];
    InT* stage = reinterpret_cast<InT*>(smem + p.off_stage);
    A* pbuf = reinterpret_cast<A*>(smem + p.off_p);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + p.off_bar);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * p.TWp;
    const int y0 = blockIdx.y * p.TH;
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
        const int y = y0 + b * kBand + lane;
        const bool on = lane < kBand && y < yend;
        const unsigned valid = __ballot_sync(0xffffffffu, on);
        if (lane == 0) mbar_arrive_expect_tx(&bars[slot], (uint32_t)(__popc(valid) * row_bytes));
        __syncwarp();
        if (on) {
            fence_proxy_async();
            for (int k = 0; k < p.nbox; ++k)
                tma_load_row(dst + (size_t)lane * p.SROW + (size_t)k * p.boxw, &tmap, &bars[slot],
                             ebase + k * p.boxw, y);
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
            const bool mine = mbar_wait_bounded(&bars[sidx], par);
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
            if constexpr (MODE == 2) {
#pragma unroll
                for (int c = 0; c < C; ++c) off[c] = offg[c] = 0.f;
            }
            A* Q = std::is_same<InT, float>::value ? reinterpret_cast<A*>(srow) : pbuf + (size_t)warp * p.SP;
            row_prefix<InT, C, MODE>(srow, Q, p.m, off, lane);
            float* dst = reinterpret_cast<float*>(p.out + (long long)y * p.out_pitch) + ecol0;
            for (int c0 = 0; c0 < nvalid; c0 += 256) {
                float offc[C];   // chunk element e is segment element c0 + e
#pragma unroll
                for (int c = 0; c < C; ++c) offc[c] = pick<C>(offg, (c0 + c) % C);
                float2 acc[4];
                row_taps<A, C, 8>(p, Q, s_out0 + c0, offc, acc, lane);
                const int nv = nvalid - c0;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int ea = lane + 64 * h;
                    if (ea < nv) dst[c0 + ea] = acc[h].x;
                    if (ea + 32 < nv) dst[c0 + ea + 32] = acc[h].y;
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

// --------------------------------------------------------------- column pass
struct CParams {
    const unsigned char* rin;   // R, FP32
    long long r_pitch;
    unsigned char* out;
    long long out_pitch;
    int* status;
    int H, rowlen, boundary;
    int K;
    int r[GF_KMAX];
    float w[GF_KMAX];
    float sw;
    int rk;
    int TH;            // output rows per CTA
    int NB;            // ring blocks of kBand rows (a mirror block follows)
    int nstage, use_tma;
    int off_stage, off_ring, off_coff, off_bar;
};

// CW element columns per CTA; each thread owns column tid % CW for the column
// running sum (threads below CW) and RPT = kBand CW / kThreads output rows of
// every band for the taps.
// MODE as for the row pass: 0 compensated column sums (per-column offset and
// a hi + lo carry), 1 offset and plain FP32 carry, 2 plain FP32.
template <typename OutT, int CW, int MODE>
__global__ void __launch_bounds__(kThreads, 4) col_pass_kernel(const __grid_constant__ CUtensorMap tmap,
                                                             const CParams p) {
    constexpr int RPT = kBand * CW / kThreads;
    static_assert(RPT >= 1 && RPT <= kBand, "column strip width");
    extern __shared__ __align__(128) unsigned char smem[];
    float* stage = reinterpret_cast<float*>(smem + p.off_stage);
    float* ring = reinterpret_cast<float*>(smem + p.off_ring);
    float* coffs = reinterpret_cast<float*>(smem + p.off_coff);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + p.off_bar);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ecol0 = blockIdx.x * CW;
    const int y0 = blockIdx.y * p.TH;
    if (ecol0 >= p.rowlen || y0 >= p.H) return;
    const int yend = min(y0 + p.TH, p.H);
    const int vstart = y0 - p.rk;
    const int vend = yend - 1 + p.rk;
    const int nbands = (vend - vstart + 1 + kBand - 1) / kBand;
    const int ringrows = p.NB * kBand;

    if (tid == 0) {
        for (int s = 0; s < p.nstage; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    // J(vstart - 1) = 0 sits in the last logical ring row
    if (tid < CW) ring[(size_t)(ringrows - 1) * CW + tid] = 0.f;
    __syncthreads();

    auto issue_band = [&](int b, int slot) {
        float* dst = stage + (size_t)slot * kBand * CW;
        const int v = vstart + b * kBand + lane;
        const int yr = (lane < kBand && v <= vend) ? fold_index(v, p.H, p.boundary) : -1;
        const unsigned valid = __ballot_sync(0xffffffffu, yr >= 0);
        if (lane == 0) mbar_arrive_expect_tx(&bars[slot], (uint32_t)(__popc(valid) * CW * 4));
        __syncwarp();
        if (yr >= 0) {
            fence_proxy_async();
            tma_load_row(dst + (size_t)lane * CW, &tmap, &bars[slot], ecol0, yr);
        }
    };
    int sidx = 0;
    uint32_t par = 0;
    if (p.use_tma && warp == 0)
        for (int b = 0; b < min(p.nstage, nbands); ++b) issue_band(b, b);

    const int col = tid % CW;
    const int j0 = (tid / CW) * RPT;
    const bool col_on = ecol0 + col < p.rowlen;
    float jh = 0.f, jl = 0.f, coff = 0.f;
    OutT* const out0 = reinterpret_cast<OutT*>(p.out) + ecol0 + col;
    bool ok = true;
    int band = 0, blk = 0;
    for (; band < nbands; ++band) {
        const float* sband = stage + (size_t)sidx * kBand * CW;
        const int v0 = vstart + band * kBand;
        if (p.use_tma) {
            const bool mine = mbar_wait_bounded(&bars[sidx], par);
            ok = __syncthreads_and(mine) != 0;
            if (!ok) break;
        } else {
            __syncthreads();
            for (int i = tid; i < kBand * CW; i += kThreads) {
                const int r = i / CW, c = i % CW;
                const int v = v0 + r;
                const int yr = v <= vend ? fold_index(v, p.H, p.boundary) : -1;
                float val = 0.f;
                if (yr >= 0 && ecol0 + c < p.rowlen)
                    val = reinterpret_cast<const float*>(p.rin + (long long)yr * p.r_pitch)[ecol0 + c];
                stage[(size_t)sidx * kBand * CW + i] = val;
            }
            __syncthreads();
        }
        // ---- column running sum of the band (threads < CW)
        if (tid < CW) {
            // rows that were not loaded (ZERO boundary, past the tile) read as 0
            const bool inner = v0 >= 0 && v0 + kBand - 1 < p.H && v0 + kBand - 1 <= vend;
            float x[kBand];
#pragma unroll
            for (int j = 0; j < kBand; ++j) {
                const int v = v0 + j;
                const bool on = inner || (v <= vend && (p.boundary != GF_ZERO || (v >= 0 && v < p.H)));
                x[j] = on ? sband[j * CW + tid] : 0.f;
            }
            if (band == 0) {
                coff = MODE == 2 ? 0.f : x[0];
                coffs[tid] = coff;
            }
            float L = 0.f, Jv[kBand];
            if constexpr (MODE == 0) {
#pragma unroll
                for (int j = 0; j < kBand; ++j) {
                    L = __fadd_rn(L, __fsub_rn(x[j], coff));
                    Jv[j] = __fadd_rn(jh, __fadd_rn(jl, L));
                }
                pair_add(jh, jl, L, 0.f, jh, jl);
            } else {
#pragma unroll
                for (int j = 0; j < kBand; ++j) {
                    jh = __fadd_rn(jh, __fsub_rn(x[j], coff));
                    Jv[j] = jh;
                }
            }
            float* wr = ring + (size_t)(blk * kBand) * CW + tid;
#pragma unroll
            for (int j = 0; j < kBand; ++j) wr[j * CW] = Jv[j];
            if (blk == 0) {
                float* wm = ring + (size_t)ringrows * CW + tid;
#pragma unroll
                for (int j = 0; j < kBand; ++j) wm[j * CW] = Jv[j];
            }
        }
        __syncthreads();   // J rows visible, stage slot free
        if (p.use_tma && warp == 0 && band + p.nstage < nbands) issue_band(band + p.nstage, sidx);

        // ---- taps: output rows y = v0 + j - rk
        if (v0 + kBand - 1 - p.rk >= y0) {
            float acc[RPT];
            const float base = coffs[col] * p.sw;
#pragma unroll
            for (int j = 0; j < RPT; ++j) acc[j] = base;
            for (int i = 0; i < p.K; ++i) {
                int ap = blk * kBand + j0 + p.r[i] - p.rk;
                if (ap < 0) ap += ringrows;
                int am = blk * kBand + j0 - p.rk - p.r[i] - 1;
                if (am < 0) am += ringrows;
                const float* pp = ring + (size_t)ap * CW + col;
                const float* pm = ring + (size_t)am * CW + col;
                const float wi = p.w[i];
                if constexpr (RPT >= 2) {
                    const float2 w2 = make_float2(wi, wi);
#pragma unroll
                    for (int h = 0; h < RPT / 2; ++h) {
                        const float2 d = sub2(make_float2(pp[(2 * h) * CW], pp[(2 * h + 1) * CW]),
                                              make_float2(pm[(2 * h) * CW], pm[(2 * h + 1) * CW]));
                        const float2 r2 = fma2(w2, d, make_float2(acc[2 * h], acc[2 * h + 1]));
                        acc[2 * h] = r2.x;
                        acc[2 * h + 1] = r2.y;
                    }
                } else {
                    acc[0] = __fmaf_rn(wi, __fsub_rn(pp[0], pm[0]), acc[0]);
                }
            }
            const int ya = v0 + j0 - p.rk;
            if (col_on) {
#pragma unroll
                for (int j = 0; j < RPT; ++j)
                    if (ya + j >= y0 && ya + j < yend)
                        *reinterpret_cast<OutT*>(reinterpret_cast<unsigned char*>(out0) +
                                                 (long long)(ya + j) * p.out_pitch) = from_float<OutT>(acc[j]);
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

// ---------------------------------------------------------------- launchers
template <typename InT>
gf_status launch_row_pass(const KParams& kp, const CUtensorMap& map, dim3 grid, size_t smem, cudaStream_t s,
                          int mode) {
    void (*kern)(const CUtensorMap, const KParams) = nullptr;
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
    kern<<<grid, kThreads, smem, s>>>(map, kp);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

template <typename OutT, int MODE>
void (*col_pass_for(int CW))(const CUtensorMap, const CParams) {
    switch (CW) {
        case 32: return col_pass_kernel<OutT, 32, MODE>;
        case 64: return col_pass_kernel<OutT, 64, MODE>;
        case 128: return col_pass_kernel<OutT, 128, MODE>;
        case 256: return col_pass_kernel<OutT, 256, MODE>;
        default: return nullptr;
    }
}

template <typename OutT>
gf_status launch_col_pass(const CParams& cp, const CUtensorMap& map, int CW, dim3 grid, size_t smem,
                          cudaStream_t s, int mode) {
    void (*kern)(const CUtensorMap, const CParams) = nullptr;
    if (mode == 0) {
        kern = col_pass_for<OutT, 0>(CW);
    } else {
        // study variants: f32 and bf16 outputs
        if constexpr (!std::is_same<OutT, __half>::value)
            kern = mode == 1 ? col_pass_for<OutT, 1>(CW) : col_pass_for<OutT, 2>(CW);
    }
    if (!kern) return GF_EUNSUPPORTED;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    kern<<<grid, kThreads, smem, s>>>(map, cp);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

#define GB_DECLARE_ROWPASS(IN)                                                                                 \
    extern template gf_status launch_row_pass<IN>(const KParams&, const CUtensorMap&, dim3, size_t, cudaStream_t, \
                                                  int);
#define GB_DECLARE_COLPASS(OUT)                                                                             \
    extern template gf_status launch_col_pass<OUT>(const CParams&, const CUtensorMap&, int, dim3, size_t, \
                                                   cudaStream_t, int);

}  // namespace gb
