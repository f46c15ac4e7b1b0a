// Depth pass of a stack of integer slices as a register walk (Sec. 3.4: the
// running sums of Eq. alg1 and the differences of Eq. indep along the third
// axis).  Compiled at run time with NVRTC once per depth radius set
// (walker_host.cu prepends the DW_* constants) and cached.
//
// The in-plane result R is FP32: D slices of H rows of `rowlen` elements.
// Thread c walks the line of R at (row y, element e) = (c / rowlen, c % rowlen)
// across the slices.  Consecutive threads take consecutive elements, so each
// warp reads and writes 128 contiguous bytes per slice.  The line's running
// sum J is kept as a pair (Jh, Jl), the same scheme as the 2D walk's column
// phase: Jh sums R rounded to multiples of a power of two q, which is exact
// because every partial sum is a multiple of q below 2^24 q (the host derives
// q from the bound on |R| that an integer input gives); Jl sums the rounding
// residues.  The last DW_LC = 2 r_K + 2 values of J sit in a register ring.
// Output z is sum_i w_i (J(z + r_i) - J(z - r_i - 1)).  A tile of th output
// slices walks th + 2 r_K slices in chunks of DW_LC; the loads of the next
// chunk are issued before the current chunk is filtered.  Slices before the
// first and past the last are supplied by the boundary rule; slices beyond
// the last one an output of the tile needs read as zero.  No shared memory,
// no barriers, no waits.

#pragma once

// Kernel arguments (shared with the host, which includes this file without
// the DW_* constants and so sees only this struct).
struct DepthParams {
    const unsigned char* in;   // R
    long long in_pitch, in_z;  // bytes between rows of a slice, between slices
    unsigned char* out;        // FP32 result, same layout with its own pitches
    long long out_pitch, out_z;
    int D, H, rowlen, boundary;
    int nch;                   // chunks of DW_LC slices one tile walks
    int th;                    // output slices per tile = nch * DW_LC - 2 rk
    float w[5];
    float q, magic;            // quantum (a power of two) and 1.5 * 2^23 * q
};

#ifdef DW_LC

// Source slice of virtual slice t (-1: a zero slice) under the boundary rule
// (0 replicate, 1 zero, 2 reflect, folded as often as needed).
__device__ __forceinline__ int dw_fold(int t, int n, int boundary) {
    if (t >= 0 && t < n) return t;
    if (boundary == 1) return -1;
    if (boundary == 0) return t < 0 ? 0 : n - 1;
    if (n == 1) return 0;
    const int period = 2 * (n - 1);
    int m = t % period;
    if (m < 0) m += period;
    return m < n ? m : period - m;
}

// DW_LC slices of one line: v[s] is R at tile row u = k DW_LC + s.  FIRST: the
// tile's first chunk, whose only outputs are its last two rows.  Tile row u
// gives output slice zo0 + s, stored when below D.
template <bool FIRST>
__device__ __forceinline__ void dw_chunk(float2 (&ring)[DW_LC], const float (&v)[DW_LC], const DepthParams& p,
                                         unsigned char* dst, int zo0, bool on) {
    const float2 w0 = make_float2(p.w[0], p.w[0]);
#if DW_K > 1
    const float2 w1 = make_float2(p.w[1], p.w[1]);
#endif
#if DW_K > 2
    const float2 w2 = make_float2(p.w[2], p.w[2]);
#endif
#if DW_K > 3
    const float2 w3 = make_float2(p.w[3], p.w[3]);
#endif
#if DW_K > 4
    const float2 w4 = make_float2(p.w[4], p.w[4]);
#endif
#pragma unroll
    for (int s = 0; s < DW_LC; ++s) {
        // R = Rh + Rl (Rh the nearest multiple of q, Rl the exact residue);
        // J(u) = J(u - 1) + (Rh, Rl) as one packed addition
        const float R = v[s];
        const float Rh = __fsub_rn(__fadd_rn(R, p.magic), p.magic);
        ring[s] = __fadd2_rn(ring[(s + DW_LC - 1) % DW_LC], make_float2(Rh, __fsub_rn(R, Rh)));
        if (!FIRST || s >= 2 * DW_RK) {
            // output of tile row u = s (mod DW_LC): J(u - rk + r_i) - J(u - rk - r_i - 1)
#define DW_TAP(R_, W_)                                                                              \
    {                                                                                               \
        const float2 a = ring[((s - DW_RK + (R_)) % DW_LC + DW_LC) % DW_LC];                        \
        const float2 bb = ring[((s - DW_RK - (R_) - 1) % DW_LC + DW_LC) % DW_LC];                   \
        acc = __ffma2_rn((W_), __ffma2_rn(bb, make_float2(-1.f, -1.f), a), acc);                    \
    }
            float2 acc = make_float2(0.f, 0.f);
            DW_TAP(DW_R0, w0)
#if DW_K > 1
            DW_TAP(DW_R1, w1)
#endif
#if DW_K > 2
            DW_TAP(DW_R2, w2)
#endif
#if DW_K > 3
            DW_TAP(DW_R3, w3)
#endif
#if DW_K > 4
            DW_TAP(DW_R4, w4)
#endif
#undef DW_TAP
            const int zo = zo0 + s;
            if (on && zo < p.D) *reinterpret_cast<float*>(dst + (long long)zo * p.out_z) = __fadd_rn(acc.x, acc.y);
        }
    }
}

// Grid: x covers the H rowlen lines in blocks of DW_TW threads, y the tiles
// of th output slices.
extern "C" __global__ void __launch_bounds__(DW_TW, 4) depth_walker_kernel(const DepthParams p) {
    const long long c = (long long)blockIdx.x * DW_TW + threadIdx.x;
    const bool on = c < (long long)p.H * p.rowlen;
    const int y = on ? (int)(c / p.rowlen) : 0;
    const int e = on ? (int)(c - (long long)y * p.rowlen) : 0;
    const unsigned char* const src = p.in + (long long)y * p.in_pitch + (long long)e * 4;
    unsigned char* const dst = p.out + (long long)y * p.out_pitch + (long long)e * 4;
    const int z0 = (int)blockIdx.y * p.th;
    // R at virtual slice z0 - rk + k DW_LC + s
    auto load = [&](float (&v)[DW_LC], int k) {
#pragma unroll
        for (int s = 0; s < DW_LC; ++s) {
            const int vz = z0 - DW_RK + k * DW_LC + s;
            const int sz = (on && vz <= p.D - 1 + DW_RK) ? dw_fold(vz, p.D, p.boundary) : -1;
            v[s] = sz >= 0 ? __ldg(reinterpret_cast<const float*>(src + (long long)sz * p.in_z)) : 0.f;
        }
    };
    float2 ring[DW_LC];   // J(-1) = 0 at ring[DW_LC - 1]
#pragma unroll
    for (int i = 0; i < DW_LC; ++i) ring[i] = make_float2(0.f, 0.f);
    float cur[DW_LC], nxt[DW_LC];
    load(cur, 0);
    if (p.nch > 1) load(nxt, 1);
    dw_chunk<true>(ring, cur, p, dst, z0 - 2 * DW_RK, on);
#pragma unroll 1
    for (int k = 1; k < p.nch; ++k) {
#pragma unroll
        for (int s = 0; s < DW_LC; ++s) cur[s] = nxt[s];
        if (k + 1 < p.nch) load(nxt, k + 1);
        dw_chunk<false>(ring, cur, p, dst, z0 + k * DW_LC - 2 * DW_RK, on);
    }
}

#endif  // DW_LC
