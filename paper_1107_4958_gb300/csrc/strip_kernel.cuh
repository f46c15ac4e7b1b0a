// Device code of the fused box-sum Gaussian filter for sm_103a (Sec. 3.3-3.4).
//
// One CTA owns a strip of TWp output pixels (all C channels: TW = TWp * C
// element columns) by TH output rows.  It walks the "virtual" rows
// y0 - rk .. y0 + TH - 1 + rk of its strip (rows outside the image are mapped
// by the boundary rule) in bands of kBand rows:
//
//   1. TMA stages the band's row segments into shared memory: one 2D box per
//      8-row band through an 8-byte-element view of the image when no row of
//      the band is folded by the boundary rule, else one box per row.  Pixels
//      of a segment that fall outside the image are rewritten in place from
//      their boundary source (only the halo), so the passes below never fold
//      an index.
//   2. Row pass, one warp per row: per-channel running sums of the staged
//      elements (Eq. alg1), 12 consecutive elements per lane in registers plus a
//      warp shuffle scan, then for every output element
//      sum_i w_i (I(x + r_i) - I(x - r_i - 1)) (Eq. indep) with the taps as the
//      outer loop and the lane's outputs unrolled inside it, in packed f32x2
//      arithmetic.  uint8 rows sum exactly in FP32 (integers below 2^24), uint16
//      rows in int32, float rows in int32 after a per-row offset and a
//      power-of-two scale (exact differences; row_prefix).
//   3. Column pass, one column per thread: the column running sum J of the
//      row-filtered band (per-column offset, compensated hi + lo carry, J
//      rounded once) goes into a ring of kBand-row blocks in tensor memory,
//      one TMEM lane per thread; a mirror block after the ring makes every
//      kBand-row window at any lag contiguous, so each tap end is one
//      tcgen05.ld of kBand columns.  Outputs of the band leave through one TMA
//      store of a shared-memory tile.
//
// Every running sum starts inside the tile (it needs only +-(rk + 1) pixels of
// context), so there is no carry between CTAs and no inter-CTA wait.  The only
// waits are the mbarrier waits of the TMA pipeline; they are bounded, and on
// expiry the CTA records GF_ETIMEOUT in the device status word and leaves.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace gb {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBand = 8;
constexpr int kStages = 3;
constexpr int kMaxStages = 8;
constexpr int kGroup = 12;                       // staged elements per lane step of the row scan
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

struct KParams {
    const unsigned char* in;
    long long in_pitch;
    unsigned char* out;
    long long out_pitch;
    int* status;       // device status word
    long long wait_limit;   // SM clock cycles per pipeline wait (kWaitCycles unless shortened by the host)
    int H, W, C, boundary;
    int K;
    int r[GF_KMAX];
    float w[GF_KMAX];
    float sw;          // sum_i w_i (2 r_i + 1) in FP32
    int rk;
    int TWp, TH, TW;   // TW = TWp * C valid element columns
    int m;             // staged elements per lane in the row scan (multiple of kGroup)
    int SP;            // per-warp running-sum buffer stride (entries)
    int SROW;          // staged elements per row (>= 32 m)
    int nbox, boxw, ealign;
    int xshift;        // TMA x coordinate = element index >> xshift (8-byte TMA elements when > 0)
    int rows8;         // the 8-row tensor map loads a whole band with one box
    int tma_store;     // whole output bands leave through the output map (a TW x 8 box)
    int tile_y0;       // row tile of blockIdx.y == 0 (a launch may cover a slab of row tiles)
    int sx, ox;        // row pass: outputs only at pixels x = ox + j sx (sx = 1: every pixel)
    int off_obuf;      // output band staged for the TMA store
    int NB;            // ring blocks of kBand rows (plus one mirror block)
    int RT;            // TMEM ring columns per warpgroup: (NB + 1) * kBand
    int tmem_cols;     // TMEM columns allocated per CTA (power of two >= 32), 0 = ring in SMEM
    int nstage;        // staged bands resident at once
    int use_tma;
    int off_stage, off_p, off_rband, off_ring, off_bar, off_tmem;
    int off_pl;        // float rows: per-warp running sums of the residues (row_prefix)
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase did not complete within `limit` SM clock
// cycles.  The default bound (kWaitCycles) polls with try_wait; a bound the
// host shortened (to exercise the expiry path) polls with the non-blocking
// test_wait, so that the wait really ends after `limit` cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = kWaitCycles) {
    if (limit >= kWaitCycles) {
        if (mbar_try_wait(bar, parity)) return true;
        const long long t0 = clock64();
        while (!mbar_try_wait(bar, parity)) {
            if (clock64() - t0 > limit) return false;
        }
        return true;
    }
    const long long t0 = clock64();
    while (!mbar_test_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}
__device__ __forceinline__ void tma_load_row(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_addr(dst)), "l"(map), "r"(smem_addr(bar)), "r"(x), "r"(y)
        : "memory");
}
// 64-bit shared-memory load at a 32-bit shared address plus a compile-time
// byte offset (kept in program order with the CTA barriers).
template <int OFF>
__device__ __forceinline__ float2 lds2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(addr), "n"(OFF) : "memory");
    return v;
}

// TMA store of a box from shared memory, tracked by the bulk async-group.
__device__ __forceinline__ void tma_store_box(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];"
                 ::"l"(map), "r"(smem_addr(src)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory source of every committed store has been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed store is complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------- tensor memory
// The column ring lives in TMEM: thread e of warpgroup g owns TMEM lane e % 128
// and the columns [g RT, (g + 1) RT) of it.  Every tcgen05 op below is executed
// by whole warps.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, int ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_st1(uint32_t taddr, float v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(__float_as_uint(v)) : "memory");
}
// 8 consecutive columns starting at a multiple of 8
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr) : "memory");
    return r;
}
// column taddr + J (J a compile-time offset folded into the instruction)
template <int J>
__device__ __forceinline__ uint32_t tmem_ld1_at(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1+%2];" : "=r"(r) : "r"(taddr), "n"(J) : "memory");
    return r;
}
template <int J>
__device__ __forceinline__ void tmem_ld_window(uint32_t ta, uint32_t tb, uint32_t* u) {
    if constexpr (J < kBand) {
        u[J] = tmem_ld1_at<J>(ta);
        u[kBand + J] = tmem_ld1_at<J>(tb);
        tmem_ld_window<J + 1>(ta, tb, u);
    }
}
// Waits for this thread's outstanding TMEM loads; the 16 destination registers
// are tied to the wait so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_wait_ld16(uint32_t* v) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
                 :
                 : "memory");
}

// ---------------------------------------------------------------- packed FP32 pairs
// sm_100-family packed FP32 (one instruction for two lanes), each lane rounded once.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ---------------------------------------------------------------- element types
// `acc` is the running-sum type: exact FP32 for uint8 (sums stay below 2^24),
// int32 for uint16, FP32 with offset and carry for float inputs.
template <typename T> struct Elem;
template <> struct Elem<uint8_t> {
    using acc = float;
    static constexpr bool exact = true;
    static __device__ __forceinline__ float cvt(uint8_t v) { return (float)v; }
};
template <> struct Elem<uint16_t> {
    using acc = int;
    static constexpr bool exact = true;
    static __device__ __forceinline__ int cvt(uint16_t v) { return (int)v; }
};
template <> struct Elem<float> {
    using acc = float;
    static constexpr bool exact = false;
    static __device__ __forceinline__ float cvt(float v) { return v; }
};
template <> struct Elem<__nv_bfloat16> {
    using acc = float;
    static constexpr bool exact = false;
    static __device__ __forceinline__ float cvt(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <> struct Elem<__half> {
    using acc = float;
    static constexpr bool exact = false;
    static __device__ __forceinline__ float cvt(__half v) { return __half2float(v); }
};

// Running-sum type of a staged row for accumulation mode MODE.  Float rows of
// the default mode (0) are scaled by a power of two, rounded to integers and
// summed in int32 (row_prefix), so every box difference of the row is exact
// whatever the segment length; the precision-study modes keep FP32 sums.
template <typename T, int MODE>
using row_acc_t = typename std::conditional<!Elem<T>::exact && MODE == 0, int, typename Elem<T>::acc>::type;

template <typename T> __device__ __forceinline__ T from_float(float v);
template <> __device__ __forceinline__ float from_float<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_float<__half>(float v) { return __float2half_rn(v); }

// Two adjacent output values stored with one access where the type allows.
template <typename T> __device__ __forceinline__ void store_pair(T* dst, float2 v);
template <> __device__ __forceinline__ void store_pair<float>(float* dst, float2 v) {
    *reinterpret_cast<float2*>(dst) = v;
}
template <> __device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* dst, float2 v) {
    *reinterpret_cast<__nv_bfloat162*>(dst) = __floats2bfloat162_rn(v.x, v.y);
}
template <> __device__ __forceinline__ void store_pair<__half>(__half* dst, float2 v) {
    *reinterpret_cast<__half2*>(dst) = __floats2half2_rn(v.x, v.y);
}

// off[i] for a runtime i < C without dynamic register indexing.
template <int C> __device__ __forceinline__ float pick(const float* off, int i) {
    float v = off[0];
#pragma unroll
    for (int c = 1; c < C; ++c) v = (i == c) ? off[c] : v;
    return v;
}

// Source index of position t on an axis of length n, -1 for a zero pixel.
__device__ __forceinline__ int fold_index(int t, int n, int boundary) {
    if (t >= 0 && t < n) return t;
    if (boundary == GF_ZERO) return -1;
    if (boundary == GF_REPLICATE) return t < 0 ? 0 : n - 1;
    if (n == 1) return 0;
    const int period = 2 * (n - 1);
    int m = t % period;
    if (m < 0) m += period;
    return m < n ? m : period - m;
}
__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// ------------------------------------------------------- exact-ish float pairs
// s + e == a + b exactly (Knuth's TwoSum); operations kept un-fused.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (ah, al) + (bh, bl) as an unevaluated float pair.
__device__ __forceinline__ void pair_add(float ah, float al, float bh, float bl, float& rh, float& rl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    rh = __fadd_rn(s, e);
    rl = __fsub_rn(e, __fsub_rn(rh, s));
}

// Lane-wise TwoSum on pairs: s + e == a + b exactly in each lane.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = add2(a, b);
    const float2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// (ah + al) + (bh + bl) as rh + rl: rh = fl(ah + bh), rl collects the exact
// rounding error of that sum and the low parts (not renormalised; a difference
// of two such pairs, (h_a - h_b) + (l_a - l_b), is accurate to its own size).
__device__ __forceinline__ void dd_add2(float2 ah, float2 al, float2 bh, float2 bl, float2& rh, float2& rl) {
    float2 s, e;
    two_sum2(ah, bh, s, e);
    rh = s;
    rl = add2(add2(al, bl), e);
}

// ---------------------------------------------------------------- staging
// Rewrites the staged elements of pixels outside [0, W) from their boundary
// source (replicate / reflect), so that later reads need no index folding.
// Zero pixels are already zero (TMA out-of-bounds fill / plain loader).
// Only the staged elements left of the row (g < 0) and right of it
// (g >= W C) are visited; their sources are pixels inside the row, so the
// rewrites never read a rewritten element.
template <typename T>
__device__ __forceinline__ void fold_halo(T* srow, int nelem, int ebase, int C, int W, int boundary, int lane) {
    auto fix = [&](int s) {
        const int g = ebase + s;
        const int t = floor_div(g, C);
        const int c = g - t * C;
        const int src = fold_index(t, W, boundary) * C + c - ebase;
        srow[s] = srow[min(max(src, 0), nelem - 1)];
    };
    const int left_end = min(nelem, max(0, -ebase));
    const int right_beg = max(left_end, min(nelem, W * C - ebase));
    for (int s = lane; s < left_end; s += 32) fix(s);
    for (int s = right_beg + lane; s < nelem; s += 32) fix(s);
}

// 12 consecutive staged elements, converted (vector loads; s0 is 12-aligned).
template <typename T> struct Load12;
template <> struct Load12<uint8_t> {
    static __device__ __forceinline__ void run(const uint8_t* p, float* v) {
        const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint32_t w = q[k];
#pragma unroll
            for (int b = 0; b < 4; ++b) v[4 * k + b] = (float)((w >> (8 * b)) & 0xffu);
        }
    }
};
template <> struct Load12<uint16_t> {
    static __device__ __forceinline__ void run(const uint16_t* p, int* v) {
        const uint2* q = reinterpret_cast<const uint2*>(p);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint2 w = q[k];
            v[4 * k + 0] = (int)(w.x & 0xffffu);
            v[4 * k + 1] = (int)(w.x >> 16);
            v[4 * k + 2] = (int)(w.y & 0xffffu);
            v[4 * k + 3] = (int)(w.y >> 16);
        }
    }
};
template <> struct Load12<float> {
    static __device__ __forceinline__ void run(const float* p, float* v) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 w = q[k];
            v[4 * k + 0] = w.x;
            v[4 * k + 1] = w.y;
            v[4 * k + 2] = w.z;
            v[4 * k + 3] = w.w;
        }
    }
};
template <> struct Load12<__nv_bfloat16> {
    static __device__ __forceinline__ void run(const __nv_bfloat16* p, float* v) {
        const uint2* q = reinterpret_cast<const uint2*>(p);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint2 w = q[k];
            v[4 * k + 0] = __uint_as_float(w.x << 16);
            v[4 * k + 1] = __uint_as_float(w.x & 0xffff0000u);
            v[4 * k + 2] = __uint_as_float(w.y << 16);
            v[4 * k + 3] = __uint_as_float(w.y & 0xffff0000u);
        }
    }
};
template <> struct Load12<__half> {
    static __device__ __forceinline__ void run(const __half* p, float* v) {
        const __half2* q = reinterpret_cast<const __half2*>(p);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 f = __half22float2(q[k]);
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        }
    }
};

// ---------------------------------------------------------------- row prefix
// Per-channel running sums of one staged row (Eq. alg1), by one warp:
//   Q[s] = sum of (f[s'] - off[s' mod C]) over s' <= s, s' = s (mod C),
// for staged indices s in [0, 32 m).  Lane l owns s in [l m, (l + 1) m) and
// walks it in groups of kGroup (a multiple of C, so residues are static).
// Elements before the first needed pixel add the same constant to both ends
// of every box difference and cancel.
// MODE (float rows only): 0 splits every value f into f_h + f_l, f_h the
// nearest multiple of a power of two q and f_l = f - f_h (exact, |f_l| <= q / 2):
// Q holds the running sums of f_h / q modulo 2^32 (taken from the bits of
// f + 1.5 2^23 q, whose low mantissa bits count multiples of q) and QL the
// FP32 running sums of f_l.  q is the smallest power of two with |f| < 2^22 q
// and (2 rk + 1) |f| / q < 2^30 over the staged indices [wlo, whi) the gather
// reads, so a box difference of Q is exact (window sums of f_h / q below 2^31)
// and one of QL carries only the rounding of sums of residues no larger than
// q / 2: a box sum is accurate to its own magnitude, whatever the values
// elsewhere in the row.  The rest of the staged row may hold anything: its
// residues are taken as zero and its integer sums cancel modulo 2^32.  The
// gather gets q and the bits of 1.5 2^23 q in `rs` (every element adds those
// bits once to Q, (2 r + 1) times per window).  1 and 2
// keep FP32 running sums with a plain FP32 scan of the lane totals (the
// precision-study variants; 2 is called with zero offsets).  Integer rows
// ignore `rs` (their sums are exact as they stand).
struct RowScale {
    float q = 1.f;        // quantum of the integer part (float rows, MODE 0)
    uint32_t bits_m = 0;  // bits of 1.5 2^23 q
};
template <typename T, int C, int MODE = 0>
__device__ __forceinline__ void row_prefix(const T* srow, row_acc_t<T, MODE>* Q, float* QL, int m, const float* off,
                                           int lane, RowScale& rs, int rk = 0, int wlo = 0,
                                           int whi = 0x7fffffff) {
    using A = row_acc_t<T, MODE>;
    constexpr int G = kGroup;
    const int s0 = lane * m;
    const int ngroups = m / G;
    rs = RowScale();
    if constexpr (!Elem<T>::exact && MODE == 0) {
        (void)off;
        // pass 1: the largest |f| over the staged indices [wlo, whi) that the
        // gather reads (the rest of the staged row may hold anything)
        float v[G];
        float mx = 0.f;
        for (int g = 0; g < ngroups; ++g) {
            Load12<T>::run(srow + s0 + g * G, v);
            const int sg = s0 + g * G;
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (sg + t >= wlo && sg + t < whi) mx = fmaxf(mx, fabsf(v[t]));
        }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, d));
        // q = 2^e: mx < 2^(ex + 1) <= 2^22 q and (2 rk + 1) 2^(ex + 1) <= 2^30 q
        int e = -126;
        if (mx > 0.f) {
            const int ex = (int)((__float_as_uint(mx) >> 23) & 0xffu) - 127;
            const int lw = 32 - __clz(2 * rk + 1);   // 2 rk + 1 < 2^lw
            e = max(-126, min(100, max(ex + 1 - 22, ex + 1 + lw - 30)));
        }
        const float M = __uint_as_float(((uint32_t)(e + 23 + 127) << 23) | 0x400000u);   // 1.5 2^(e + 23)
        rs.q = __uint_as_float((uint32_t)(e + 127) << 23);
        rs.bits_m = __float_as_uint(M);
        // pass 2: lane totals of both parts
        uint32_t th[C];
        float tl[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            th[c] = 0u;
            tl[c] = 0.f;
        }
        uint32_t qh[G];
        float ql[G];
        for (int g = 0; g < ngroups; ++g) {
            Load12<T>::run(srow + s0 + g * G, v);
            const int sg = s0 + g * G;
#pragma unroll
            for (int t = 0; t < G; ++t) {
                const float tt = __fadd_rn(v[t], M);
                const float fl = (sg + t >= wlo && sg + t < whi) ? __fsub_rn(v[t], __fsub_rn(tt, M)) : 0.f;
                th[t % C] += __float_as_uint(tt);
                tl[t % C] = __fadd_rn(tl[t % C], fl);
                qh[t] = th[t % C];
                ql[t] = tl[t % C];
            }
        }
        uint32_t bh[C];
        float bl[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            uint32_t ih = th[c];
            float il = tl[c];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t oh = __shfl_up_sync(0xffffffffu, ih, d);
                const float ol = __shfl_up_sync(0xffffffffu, il, d);
                if (lane >= d) {
                    ih += oh;
                    il = __fadd_rn(ol, il);
                }
            }
            bh[c] = ih - th[c];
            const float pl = __shfl_up_sync(0xffffffffu, il, 1);
            bl[c] = lane == 0 ? 0.f : pl;
        }
        if (ngroups == 1) {
            // the lane's 12 local sums are still in registers
            int4* dh = reinterpret_cast<int4*>(Q + s0);
            float4* dl = reinterpret_cast<float4*>(QL + s0);
#pragma unroll
            for (int k = 0; k < G / 4; ++k) {
                dh[k] = make_int4((int)(qh[4 * k] + bh[(4 * k) % C]), (int)(qh[4 * k + 1] + bh[(4 * k + 1) % C]),
                                  (int)(qh[4 * k + 2] + bh[(4 * k + 2) % C]),
                                  (int)(qh[4 * k + 3] + bh[(4 * k + 3) % C]));
                dl[k] = make_float4(__fadd_rn(bl[(4 * k) % C], ql[4 * k]), __fadd_rn(bl[(4 * k + 1) % C], ql[4 * k + 1]),
                                    __fadd_rn(bl[(4 * k + 2) % C], ql[4 * k + 2]),
                                    __fadd_rn(bl[(4 * k + 3) % C], ql[4 * k + 3]));
            }
        } else {
            // pass 3: the running sums from the lane bases
            for (int g = 0; g < ngroups; ++g) {
                Load12<T>::run(srow + s0 + g * G, v);
                const int sg = s0 + g * G;
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const float tt = __fadd_rn(v[t], M);
                    const float fl = (sg + t >= wlo && sg + t < whi) ? __fsub_rn(v[t], __fsub_rn(tt, M)) : 0.f;
                    bh[t % C] += __float_as_uint(tt);
                    bl[t % C] = __fadd_rn(bl[t % C], fl);
                    qh[t] = bh[t % C];
                    ql[t] = bl[t % C];
                }
                int4* dh = reinterpret_cast<int4*>(Q + s0 + g * G);
                float4* dl = reinterpret_cast<float4*>(QL + s0 + g * G);
#pragma unroll
                for (int k = 0; k < G / 4; ++k) {
                    dh[k] = make_int4((int)qh[4 * k], (int)qh[4 * k + 1], (int)qh[4 * k + 2], (int)qh[4 * k + 3]);
                    dl[k] = make_float4(ql[4 * k], ql[4 * k + 1], ql[4 * k + 2], ql[4 * k + 3]);
                }
            }
        }
        __syncwarp();
    } else {
        A tot[C];
#pragma unroll
        for (int c = 0; c < C; ++c) tot[c] = A(0);
        A v[G];
        if (ngroups == 1) {
            // common case: the lane's 12 elements stay in registers across the scan
            Load12<T>::run(srow + s0, v);
#pragma unroll
            for (int t = 0; t < G; ++t) {
                if constexpr (!Elem<T>::exact) v[t] = __fsub_rn(v[t], off[t % C]);
                tot[t % C] += v[t];
                v[t] = tot[t % C];
            }
        } else {
            for (int g = 0; g < ngroups; ++g) {
                Load12<T>::run(srow + s0 + g * G, v);
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    if constexpr (!Elem<T>::exact) tot[t % C] = __fadd_rn(tot[t % C], __fsub_rn(v[t], off[t % C]));
                    else tot[t % C] += v[t];
                }
            }
        }
        // exclusive scan of the lane totals, per channel
        A base[C];
        if constexpr (!Elem<T>::exact) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                float hi = tot[c];
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const float oh = __shfl_up_sync(0xffffffffu, hi, d);
                    if (lane >= d) hi = __fadd_rn(oh, hi);
                }
                const float bh = __shfl_up_sync(0xffffffffu, hi, 1);
                base[c] = lane == 0 ? 0.f : bh;
            }
            if (ngroups == 1) {
#pragma unroll
                for (int t = 0; t < G; ++t) v[t] = __fadd_rn(base[t % C], v[t]);
            } else {
                float loc[C];
#pragma unroll
                for (int c = 0; c < C; ++c) loc[c] = 0.f;
                for (int g = 0; g < ngroups; ++g) {
                    Load12<T>::run(srow + s0 + g * G, v);
#pragma unroll
                    for (int t = 0; t < G; ++t) {
                        loc[t % C] = __fadd_rn(loc[t % C], __fsub_rn(v[t], off[t % C]));
                        v[t] = __fadd_rn(base[t % C], loc[t % C]);
                    }
                    float4* dst = reinterpret_cast<float4*>(Q + s0 + g * G);
#pragma unroll
                    for (int k = 0; k < G / 4; ++k)
                        dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                A inc = tot[c];
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const A o = __shfl_up_sync(0xffffffffu, inc, d);
                    if (lane >= d) inc += o;
                }
                base[c] = inc - tot[c];
            }
            if (ngroups == 1) {
#pragma unroll
                for (int t = 0; t < G; ++t) v[t] += base[t % C];
            } else {
                for (int g = 0; g < ngroups; ++g) {
                    Load12<T>::run(srow + s0 + g * G, v);
#pragma unroll
                    for (int t = 0; t < G; ++t) {
                        base[t % C] += v[t];
                        v[t] = base[t % C];
                    }
                    if constexpr (std::is_same<A, int>::value) {
                        int4* dst = reinterpret_cast<int4*>(Q + s0 + g * G);
#pragma unroll
                        for (int k = 0; k < G / 4; ++k) dst[k] = make_int4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                    } else {
                        float4* dst = reinterpret_cast<float4*>(Q + s0 + g * G);
#pragma unroll
                        for (int k = 0; k < G / 4; ++k)
                            dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                    }
                }
            }
        }
        if (ngroups == 1) {
            if constexpr (std::is_same<A, int>::value) {
                int4* dst = reinterpret_cast<int4*>(Q + s0);
#pragma unroll
                for (int k = 0; k < G / 4; ++k) dst[k] = make_int4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
            } else {
                float4* dst = reinterpret_cast<float4*>(Q + s0);
#pragma unroll
                for (int k = 0; k < G / 4; ++k) dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
            }
        }
        __syncwarp();
    }
}

// Per-row offsets of a float row.  row_prefix subtracts off[s mod C] from the
// staged element s, so off[c] is taken from an element of that residue class
// (the same channel) next to the first output; the output element e sits at
// staged index s_out0 + e, so the gather adds back offg[e mod C] =
// off[(s_out0 + e) mod C].  Integer rows use no offset.
template <typename T, int C>
__device__ __forceinline__ void row_offsets(const T* srow, int s_out0, float* off, float* offg) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int k = ((c - s_out0) % C + C) % C;   // s_out0 + k == c (mod C)
        off[c] = Elem<T>::exact ? 0.f : (float)Elem<T>::cvt(srow[s_out0 + k]);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) offg[c] = pick<C>(off, (s_out0 + c) % C);
}

// Row filter of one staged row from its running sums: for output element
// columns e = lane + 32 k (k < NQ), element e sits at staged index s_out0 + e:
//   R(e) = offg[e mod C] * sw + sum_i w_i (Q[s + r_i C] - Q[s - (r_i + 1) C]).
// Taps outer, the lane's NQ outputs inner (fixed offsets from two pointers).
// SPLIT (float rows of mode 0): the box sum is q (Q difference - (2 r + 1)
// bits_m, an exact integer) plus the QL difference (row_prefix).
template <typename A, int C, int NQ, bool SPLIT = false>
__device__ __forceinline__ void row_taps(const KParams& p, const A* Q, const float* QL, int s_out0, const float* off,
                                         float2* acc, int lane, const RowScale& rs) {
#pragma unroll
    for (int h = 0; h < NQ / 2; ++h) {
        const int ea = lane + 64 * h, eb = ea + 32;
        acc[h] = make_float2(pick<C>(off, ea % C) * p.sw, pick<C>(off, eb % C) * p.sw);
    }
    const A* qc = Q + s_out0 + lane;
    const float* qlc = QL + s_out0 + lane;
    // unrolled to GF_KMAX taps with a uniform predicate, so that the loads of
    // consecutive taps can overlap
#pragma unroll
    for (int i = 0; i < GF_KMAX; ++i) {
        if (i < p.K) {
            const int r = p.r[i];
            const float2 w2 = make_float2(p.w[i], p.w[i]);
            const A* qp = qc + r * C;
            const A* qm = qc - (r + 1) * C;
            if constexpr (SPLIT) {
                const uint32_t cm = (uint32_t)(2 * r + 1) * rs.bits_m;
                const float2 q2 = make_float2(rs.q, rs.q);
                const float* lp = qlc + r * C;
                const float* lm = qlc - (r + 1) * C;
#pragma unroll
                for (int h = 0; h < NQ / 2; ++h) {
                    // sum of f_h / q over the window (exact), then q times it plus the residues
                    const float2 dh = make_float2((float)(int)((uint32_t)qp[64 * h] - (uint32_t)qm[64 * h] - cm),
                                                  (float)(int)((uint32_t)qp[64 * h + 32] - (uint32_t)qm[64 * h + 32] - cm));
                    const float2 dl = sub2(make_float2(lp[64 * h], lp[64 * h + 32]), make_float2(lm[64 * h], lm[64 * h + 32]));
                    acc[h] = fma2(w2, fma2(dh, q2, dl), acc[h]);
                }
            } else {
#pragma unroll
                for (int h = 0; h < NQ / 2; ++h) {
                    float2 d;
                    if constexpr (std::is_same<A, int>::value) {   // differences modulo 2^32
                        d = make_float2((float)(int)((uint32_t)qp[64 * h] - (uint32_t)qm[64 * h]),
                                        (float)(int)((uint32_t)qp[64 * h + 32] - (uint32_t)qm[64 * h + 32]));
                    } else {
                        d = sub2(make_float2(qp[64 * h], qp[64 * h + 32]), make_float2(qm[64 * h], qm[64 * h + 32]));
                    }
                    acc[h] = fma2(w2, d, acc[h]);
                }
            }
        }
    }
}
template <typename A, int C, int NQ, bool SPLIT = false>
__device__ __forceinline__ void row_gather(const KParams& p, const A* Q, const float* QL, int s_out0, const float* off,
                                           float* rrow, int lane, const RowScale& rs) {
    float2 acc[NQ / 2];
    row_taps<A, C, NQ, SPLIT>(p, Q, QL, s_out0, off, acc, lane, rs);
#pragma unroll
    for (int h = 0; h < NQ / 2; ++h) {
        rrow[lane + 64 * h] = acc[h].x;
        rrow[lane + 64 * h + 32] = acc[h].y;
    }
}

// ---------------------------------------------------------------- one tile
// Filters the tile (strip bx, row tile by) of the image described by `p`.
// TWMAX: element columns the block is laid out for (256 or 64); C: channels.
// The caller has initialised the stage mbarriers and (TWMAX = 256) allocated
// TMEM at `tbase`; `gband` counts the bands this CTA has staged so far (it
// selects stage slots and mbarrier phases across tiles).  Returns false if a
// bounded wait expired (the status word is then set).
template <typename InT, typename OutT, int TWMAX, int C>
__device__ __forceinline__ bool run_tile(const KParams& p, const CUtensorMap* tmap, const CUtensorMap* tmap8,
                                         const CUtensorMap* omap, int bx, int by, unsigned char* smem,
                                         uint32_t tbase, int& gband) {
    using A = row_acc_t<InT, 0>;
    constexpr int NQ = TWMAX / 32;
    InT* stage = reinterpret_cast<InT*>(smem + p.off_stage);
    A* pbuf = reinterpret_cast<A*>(smem + p.off_p);
    float* rband = reinterpret_cast<float*>(smem + p.off_rband);
    float* ring = reinterpret_cast<float*>(smem + p.off_ring);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + p.off_bar);
    OutT* obuf = reinterpret_cast<OutT*>(smem + p.off_obuf);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = bx * p.TWp;
    const int y0 = by * p.TH;
    if (y0 >= p.H || x0 >= p.W) return true;
    const int yend = min(y0 + p.TH, p.H);
    const int vstart = y0 - p.rk;
    const int vend = yend - 1 + p.rk;
    const int nbands = (vend - vstart + 1 + kBand - 1) / kBand;
    const int ebase = floor_div((x0 - p.rk - 1) * C, p.ealign) * p.ealign;
    const int s_out0 = x0 * C - ebase;                     // staged index of output element 0
    const bool hedge = (x0 - p.rk - 1 < 0) || (x0 + p.TWp + p.rk > p.W);
    const bool fixup = hedge && p.boundary != GF_ZERO && p.use_tma;
    const int rowlen = p.W * C;
    const int ecol0 = x0 * C;
    // staged indices the gather of the strip's valid outputs reads
    const int wlo = s_out0 - (p.rk + 1) * C, whi = s_out0 + min(p.TW, rowlen - ecol0) + p.rk * C;
    const int row_bytes = p.nbox * p.boxw * (int)sizeof(InT);
    const int ringrows = p.NB * kBand;   // logical ring rows (the mirror block follows)

    // Warp 0 stages band b into stage slot `slot`.  A band of kBand image rows
    // (no row folded by the boundary rule) is one 2D box of the 8-row map;
    // otherwise lane r < kBand loads row r of the band (mapped by the boundary
    // rule), one TMA box per row piece.  Lane 0 posts the byte count on the
    // slot's mbarrier.
    auto issue_band = [&](int b, int slot) {
        InT* dst = stage + (size_t)slot * kBand * p.SROW;
        const int vb = vstart + b * kBand;
        if (p.rows8 && vb >= 0 && vb + kBand <= p.H) {
            if (lane == 0) {
                mbar_arrive_expect_tx(&bars[slot], (uint32_t)(kBand * row_bytes));
                fence_proxy_async();
                tma_load_row(dst, tmap8, &bars[slot], ebase >> p.xshift, vb);
            }
            return;
        }
        const int v = vb + lane;
        const int yr = (lane < kBand && v <= vend) ? fold_index(v, p.H, p.boundary) : -1;
        const unsigned valid = __ballot_sync(0xffffffffu, yr >= 0);
        if (lane == 0) mbar_arrive_expect_tx(&bars[slot], (uint32_t)(__popc(valid) * row_bytes));
        __syncwarp();
        if (yr >= 0) {
            fence_proxy_async();
            for (int k = 0; k < p.nbox; ++k)
                tma_load_row(dst + (size_t)lane * p.SROW + (size_t)k * p.boxw, tmap, &bars[slot],
                             (ebase + k * p.boxw) >> p.xshift, yr);
        }
    };

    constexpr bool TM = (TWMAX == 256);   // wide strips keep the column ring in TMEM
    // stage slot and mbarrier parity of this tile's first band
    int sidx = gband % p.nstage;
    uint32_t par = (uint32_t)((gband / p.nstage) & 1);
    if (p.use_tma && warp == 0) {
        int sl = sidx;
        for (int b = 0; b < min(p.nstage, nbands); ++b) {
            issue_band(b, sl);
            sl = (sl + 1 == p.nstage) ? 0 : sl + 1;
        }
    }

    // Column state: column e = tid.  J(vstart - 1) = 0 sits in the last logical
    // ring row.
    const int e = tid;
    const bool col_on = e < p.TW;
    // this thread's TMEM ring row: lane 32 (warp % 4) + lane; its warpgroup's
    // columns hold the hi ring [0, RT) and the lo ring [RT, 2 RT)
    const uint32_t trow = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 2 * p.RT);
    const uint32_t trow_lo = trow + (uint32_t)p.RT;
    // the lo ring in shared memory follows the hi ring (narrow strips)
    float* const ring_lo = ring + (size_t)(p.NB + 1) * kBand * TWMAX;
    if constexpr (TM) {
        tmem_st1(trow + (uint32_t)(ringrows - 1), 0.f);
        tmem_st1(trow_lo + (uint32_t)(ringrows - 1), 0.f);
    } else {
        if (col_on) {
            ring[(size_t)(ringrows - 1) * TWMAX + e] = 0.f;
            ring_lo[(size_t)(ringrows - 1) * TWMAX + e] = 0.f;
        }
    }
    // column running sum J before this band, as jh + jl: jh the FP32 running
    // sum, jl the exact rounding errors of its additions (TwoSum) summed
    float jh = 0.f, jl = 0.f;
    bool ok = true;
    int band = 0;
    int blk = 0;        // band % NB
    OutT* const out0 = reinterpret_cast<OutT*>(p.out) + ecol0 + e;
    // Whole output bands are staged in obuf and stored by one TMA box, issued
    // by thread 0 after the next CTA barrier; thread 0 waits for the box to
    // be read before the barrier that precedes the next write of obuf.
    int pend_y = -1;   // first output row of the staged band, -1 if none

    for (; band < nbands; ++band) {
        InT* sband = stage + (size_t)sidx * kBand * p.SROW;
        const int v0 = vstart + band * kBand;
        if (p.use_tma) {
            const bool mine = mbar_wait_bounded(&bars[sidx], par, p.wait_limit);
            ok = __syncthreads_and(mine) != 0;
            if (!ok) break;
        } else {
            // plain loader: folds rows and pixels while staging
            __syncthreads();
            for (int r = 0; r < kBand; ++r) {
                const int v = v0 + r;
                const int yr = (v <= vend) ? fold_index(v, p.H, p.boundary) : -1;
                const InT* src = reinterpret_cast<const InT*>(p.in + (long long)max(yr, 0) * p.in_pitch);
                for (int i = tid; i < p.SROW; i += kThreads) {
                    const int g = ebase + i;
                    const int t = floor_div(g, C);
                    const int xs = fold_index(t, p.W, p.boundary);
                    InT val;
                    if (yr >= 0 && xs >= 0) val = src[xs * C + (g - t * C)];
                    else memset(&val, 0, sizeof(InT));
                    stage[(size_t)r * p.SROW + i] = val;
                }
            }
            __syncthreads();
        }

        if (pend_y >= 0) {
            if (tid == 0) {
                tma_store_box(omap, obuf, ecol0, pend_y);
                bulk_commit();
            }
            pend_y = -1;
        }

        // ---------------- row pass: one warp per row of the band
        float* rb = rband + (size_t)(band & 1) * kBand * TWMAX;
        {
            const int r = warp;
            const int v = v0 + r;
            float* rrow = rb + (size_t)r * TWMAX;
            if (v <= vend) {
                if (p.boundary == GF_ZERO && (v < 0 || v >= p.H)) {
#pragma unroll
                    for (int k = 0; k < NQ; ++k) rrow[lane + 32 * k] = 0.f;
                } else {
                    InT* srow = sband + (size_t)r * p.SROW;
                    if (fixup) {
                        fold_halo<InT>(srow, p.SROW, ebase, C, p.W, p.boundary, lane);
                        __syncwarp();
                    }
                    float off[C], offg[C];
                    row_offsets<InT, C>(srow, s_out0, off, offg);
                    constexpr bool SPLIT = !Elem<InT>::exact;   // float rows: integer part + residues
                    if constexpr (SPLIT) {
#pragma unroll
                        for (int c = 0; c < C; ++c) off[c] = offg[c] = 0.f;
                    }
                    // 4-byte float rows keep the integer sums in place over the staged row
                    A* Q = std::is_same<InT, float>::value ? reinterpret_cast<A*>(srow) : pbuf + (size_t)warp * p.SP;
                    float* QL = reinterpret_cast<float*>(smem + p.off_pl) + (size_t)warp * p.SP;
                    RowScale rs;
                    row_prefix<InT, C>(srow, Q, QL, p.m, off, lane, rs, p.rk, wlo, whi);
                    row_gather<A, C, NQ, SPLIT>(p, Q, QL, s_out0, offg, rrow, lane, rs);
                    __syncwarp();
                }
            }
        }
        if (p.tma_store && tid == 0) bulk_wait_read();   // obuf free for this band's outputs
        __syncthreads();
        if (p.use_tma && warp == 0 && band + p.nstage < nbands) issue_band(band + p.nstage, sidx);

        // ---------------- column pass: one column per thread
        if (TM || col_on) {
            const float* rv = rb + e;
            // J(v0 + j) = jh + jl: each row's value is added to jh in FP32 and
            // the rounding error of that addition (exact, TwoSum) to jl, so a
            // difference of two J, (jh_a - jh_b) + (jl_a - jl_b), is accurate to
            // its own magnitude however large J has grown over the column
            float Jh[kBand], Jl[kBand];
#pragma unroll
            for (int j = 0; j < kBand; ++j) {
                float sum, err;
                two_sum(jh, rv[j * TWMAX], sum, err);
                jh = sum;
                jl = __fadd_rn(jl, err);
                Jh[j] = jh;
                Jl[j] = jl;
            }
            if constexpr (TM) {
                tmem_st8(trow + (uint32_t)(blk * kBand), Jh);
                tmem_st8(trow_lo + (uint32_t)(blk * kBand), Jl);
                if (blk == 0) {
                    tmem_st8(trow + (uint32_t)ringrows, Jh);
                    tmem_st8(trow_lo + (uint32_t)ringrows, Jl);
                }
                tmem_wait_st();
            } else {
                float* wr = ring + (size_t)(blk * kBand) * TWMAX + e;
                float* wm = ring + (size_t)ringrows * TWMAX + e;
                float* wrl = ring_lo + (size_t)(blk * kBand) * TWMAX + e;
                float* wml = ring_lo + (size_t)ringrows * TWMAX + e;
#pragma unroll
                for (int j = 0; j < kBand; ++j) {
                    wr[j * TWMAX] = Jh[j];
                    wrl[j * TWMAX] = Jl[j];
                    if (blk == 0) {
                        wm[j * TWMAX] = Jh[j];
                        wml[j * TWMAX] = Jl[j];
                    }
                }
            }
            // output rows y = v0 + j - rk, j = 0 .. kBand-1, in row pairs
            if (v0 + kBand - 1 - p.rk >= y0) {
                float2 acc[kBand / 2];
#pragma unroll
                for (int h = 0; h < kBand / 2; ++h) acc[h] = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < GF_KMAX; ++i) {
                    if (i >= p.K) break;
                    int ap = blk * kBand + p.r[i] - p.rk;
                    if (ap < 0) ap += ringrows;
                    int am = blk * kBand - p.rk - p.r[i] - 1;
                    if (am < 0) am += ringrows;
                    const float2 w2 = make_float2(p.w[i], p.w[i]);
                    float a[kBand], b[kBand], al[kBand], bl[kBand];
                    if constexpr (TM) {
                        uint32_t u[2 * kBand], ul[2 * kBand];
                        tmem_ld_window<0>(trow + (uint32_t)ap, trow + (uint32_t)am, u);
                        tmem_ld_window<0>(trow_lo + (uint32_t)ap, trow_lo + (uint32_t)am, ul);
                        tmem_wait_ld16(u);
                        tmem_wait_ld16(ul);
#pragma unroll
                        for (int j = 0; j < kBand; ++j) {
                            a[j] = __uint_as_float(u[j]);
                            b[j] = __uint_as_float(u[kBand + j]);
                            al[j] = __uint_as_float(ul[j]);
                            bl[j] = __uint_as_float(ul[kBand + j]);
                        }
                    } else {
                        const float* pp = ring + (size_t)ap * TWMAX + e;
                        const float* pm = ring + (size_t)am * TWMAX + e;
                        const float* ppl = ring_lo + (size_t)ap * TWMAX + e;
                        const float* pml = ring_lo + (size_t)am * TWMAX + e;
#pragma unroll
                        for (int j = 0; j < kBand; ++j) {
                            a[j] = pp[j * TWMAX];
                            b[j] = pm[j * TWMAX];
                            al[j] = ppl[j * TWMAX];
                            bl[j] = pml[j * TWMAX];
                        }
                    }
                    // (J_hi difference) + (J_lo difference), each rounded to its own magnitude
#pragma unroll
                    for (int h = 0; h < kBand / 2; ++h) {
                        const float2 dh = sub2(make_float2(a[2 * h], a[2 * h + 1]), make_float2(b[2 * h], b[2 * h + 1]));
                        const float2 dl =
                            sub2(make_float2(al[2 * h], al[2 * h + 1]), make_float2(bl[2 * h], bl[2 * h + 1]));
                        acc[h] = fma2(w2, add2(dh, dl), acc[h]);
                    }
                }
                const int yb = v0 - p.rk;   // output row of j = 0
                if (p.tma_store && yb >= y0 && yb + kBand <= yend) {
                    if (col_on) {
#pragma unroll
                        for (int h = 0; h < kBand / 2; ++h) {
                            obuf[(2 * h) * p.TW + e] = from_float<OutT>(acc[h].x);
                            obuf[(2 * h + 1) * p.TW + e] = from_float<OutT>(acc[h].y);
                        }
                    }
                    fence_proxy_async();   // generic writes visible to the TMA store
                } else if (col_on && ecol0 + e < rowlen && yb >= y0 && yb + kBand <= yend) {
                    unsigned char* o = reinterpret_cast<unsigned char*>(out0) + (long long)yb * p.out_pitch;
#pragma unroll
                    for (int h = 0; h < kBand / 2; ++h) {
                        *reinterpret_cast<OutT*>(o) = from_float<OutT>(acc[h].x);
                        o += p.out_pitch;
                        *reinterpret_cast<OutT*>(o) = from_float<OutT>(acc[h].y);
                        o += p.out_pitch;
                    }
                } else if (col_on && ecol0 + e < rowlen) {
#pragma unroll
                    for (int h = 0; h < kBand / 2; ++h) {
                        const int ya = v0 + 2 * h - p.rk;
                        if (ya >= y0 && ya < yend)
                            *reinterpret_cast<OutT*>(reinterpret_cast<unsigned char*>(out0) +
                                                     (long long)ya * p.out_pitch) = from_float<OutT>(acc[h].x);
                        if (ya + 1 >= y0 && ya + 1 < yend)
                            *reinterpret_cast<OutT*>(reinterpret_cast<unsigned char*>(out0) +
                                                     (long long)(ya + 1) * p.out_pitch) = from_float<OutT>(acc[h].y);
                    }
                }
            }
        }
        // the band's outputs wait in obuf for the store issued after the next
        // CTA barrier; every thread records it (the flush after the last band
        // is a CTA barrier, so the decision must not depend on the column)
        {
            const int yb = v0 - p.rk;
            if (p.tma_store && yb >= y0 && yb + kBand <= yend) pend_y = yb;
        }
        blk = (blk + 1 == p.NB) ? 0 : blk + 1;
        if (p.use_tma && ++sidx == p.nstage) {
            sidx = 0;
            par ^= 1u;
        }
    }
    if (p.use_tma) gband += nbands;
    if (pend_y >= 0 && ok) {
        __syncthreads();
        if (tid == 0) {
            tma_store_box(omap, obuf, ecol0, pend_y);
            bulk_commit();
        }
    }
    if (p.tma_store && tid == 0) bulk_wait_all();   // stores complete before obuf is reused or freed

    if (!ok) {
        if (tid == 0) {
            atomicCAS(p.status, 0, (int)GF_ETIMEOUT);
            // let the copies already in flight land before the CTA leaves
            int sl = sidx;
            uint32_t pa = par;
            for (int b = band; b < min(band + p.nstage, nbands); ++b) {
                (void)mbar_wait_bounded(&bars[sl], pa);
                if (++sl == p.nstage) { sl = 0; pa ^= 1u; }
            }
        }
    }
    __syncthreads();
    return ok;
}

// Barrier and TMEM set-up shared by the single-image and the batched kernel.
template <int TWMAX>
__device__ __forceinline__ uint32_t cta_setup(unsigned char* smem, int off_bar, int off_tmem, int nstage,
                                              int tmem_cols) {
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + off_bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + off_tmem);
    if (tid == 0) {
        for (int s = 0; s < nstage; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    if (TWMAX == 256 && warp == 0) tmem_alloc(tslot, tmem_cols);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    return TWMAX == 256 ? *tslot : 0u;
}

template <int TWMAX>
__device__ __forceinline__ void cta_teardown(uint32_t tbase, int tmem_cols) {
    if (TWMAX == 256) {
        tmem_fence_before();
        __syncthreads();
        if ((threadIdx.x >> 5) == 0) tmem_dealloc(tbase, tmem_cols);
    }
}

// One tile per CTA: grid = (strips, row tiles) of a single image.
template <typename InT, typename OutT, int TWMAX, int C>
__global__ void __launch_bounds__(kThreads, 4) strip_filter_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                const __grid_constant__ CUtensorMap tmap8,
                                                                const __grid_constant__ CUtensorMap omap,
                                                                const KParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int by = (int)blockIdx.y + p.tile_y0;
    if (by * p.TH >= p.H || (int)blockIdx.x * p.TWp >= p.W) return;
    const uint32_t tbase = cta_setup<TWMAX>(smem, p.off_bar, p.off_tmem, p.nstage, p.tmem_cols);
    int gband = 0;
    (void)run_tile<InT, OutT, TWMAX, C>(p, &tmap, &tmap8, &omap, blockIdx.x, by, smem, tbase, gband);
    cta_teardown<TWMAX>(tbase, p.tmem_cols);
}

// Persistent batched kernel: CTAs take (image, strip, row tile) tickets from an
// atomic counter until the work list is exhausted.  Each image carries its own
// KParams (its own plan, radii, weights, pointers) and TMA tensor map; the
// shared-memory offsets, stage count and TMEM columns are the batch maxima.
// A tile's arithmetic is run_tile's, so an image filtered here is bit-identical
// to the same image filtered alone with the same plan.
struct BatchArgs {
    const KParams* descs;        // [nimg]
    const CUtensorMap* maps;     // [3 nimg]: per image the row map, the 8-row map, the output map
    const int* tile_start;       // [nimg + 1] prefix sums of tiles per image
    int* counter;                // ticket counter, zero before the launch
    int nimg, ntiles;
    int off_bar, off_tmem, off_kp, nstage, tmem_cols;
};

template <typename InT, typename OutT, int TWMAX, int C>
__global__ void __launch_bounds__(kThreads, 4) batch_filter_kernel(const __grid_constant__ BatchArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    KParams* kp = reinterpret_cast<KParams*>(smem + a.off_kp);
    int* sh = reinterpret_cast<int*>(smem + a.off_kp + sizeof(KParams));   // [ticket, image, tile in image]
    const uint32_t tbase = cta_setup<TWMAX>(smem, a.off_bar, a.off_tmem, a.nstage, a.tmem_cols);
    int gband = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(a.counter, 1);
            int img = -1;
            if (t < a.ntiles) {
                int lo = 0, hi = a.nimg - 1;   // last image with tile_start <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.tile_start[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                img = lo;
            }
            sh[0] = t;
            sh[1] = img;
            sh[2] = img >= 0 ? t - a.tile_start[img] : 0;
        }
        __syncthreads();
        const int img = sh[1];
        if (img < 0) break;
        {
            const int* src = reinterpret_cast<const int*>(a.descs + img);
            int* dst = reinterpret_cast<int*>(kp);
            for (int i = threadIdx.x; i < (int)(sizeof(KParams) / sizeof(int)); i += kThreads) dst[i] = src[i];
        }
        __syncthreads();
        const int local = sh[2];
        const int nstrips = (kp->W + kp->TWp - 1) / kp->TWp;
        const bool ok = run_tile<InT, OutT, TWMAX, C>(*kp, a.maps + 3 * img, a.maps + 3 * img + 1, a.maps + 3 * img + 2,
                                                      local % nstrips, local / nstrips, smem, tbase, gband);
        __syncthreads();
        if (!ok) break;
    }
    cta_teardown<TWMAX>(tbase, a.tmem_cols);
}



// ------------------------------------------------------------ integer box sums
// K exact box-sum planes along rows, from the same row_prefix code the filter
// uses (so they are the filter's own integer sums).  One warp per row segment.
template <typename InT, int C>
__global__ void __launch_bounds__(kThreads) row_box_sums_kernel(const unsigned char* in, long long in_pitch,
                                                                int32_t* out, long long out_pitch,
                                                                long long plane_stride, int H, int W, int K,
                                                                int4 r03, int r4, int rk, int TWp, int m, int SP,
                                                                int SROW, int boundary) {
    using A = row_acc_t<InT, 0>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    InT* srow = reinterpret_cast<InT*>(smem) + (size_t)warp * SROW;
    const size_t p_off = ((size_t)kWarps * SROW * sizeof(InT) + 127) & ~size_t(127);
    A* Q = reinterpret_cast<A*>(smem + p_off) + (size_t)warp * SP;
    const int rr[GF_KMAX] = {r03.x, r03.y, r03.z, r03.w, r4};
    const int x0 = blockIdx.x * TWp;
    const int ebase = floor_div((x0 - rk - 1) * C, 4) * 4;
    const int s_out0 = x0 * C - ebase;
    const int rowlen = W * C;
    const float off[C] = {};
    for (int y = blockIdx.y * kWarps + warp; y < H; y += gridDim.y * kWarps) {
        const InT* src = reinterpret_cast<const InT*>(in + (long long)y * in_pitch);
        for (int i = lane; i < SROW; i += 32) {
            const int g = ebase + i;
            const int t = floor_div(g, C);
            const int xs = fold_index(t, W, boundary);
            srow[i] = xs >= 0 ? src[xs * C + (g - t * C)] : InT(0);
        }
        __syncwarp();
        RowScale rs;   // unused: integer rows
        row_prefix<InT, C>(srow, Q, nullptr, m, off, lane, rs);
        for (int e = lane; e < TWp * C; e += 32) {
            if (x0 * C + e >= rowlen) break;
            const int s = s_out0 + e;
            for (int i = 0; i < K; ++i) {
                int32_t* o = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(out + (long long)i * plane_stride) +
                                                        (long long)y * out_pitch);
                o[x0 * C + e] = (int32_t)(Q[s + rr[i] * C] - Q[s - (rr[i] + 1) * C]);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- launchers
template <typename InT, typename OutT, int TWMAX>
gf_status launch_strip_tw(const KParams& kp, const CUtensorMap* maps, dim3 grid, size_t smem, cudaStream_t s) {
    void (*kern)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const KParams) = nullptr;
    switch (kp.C) {
        case 1: kern = strip_filter_kernel<InT, OutT, TWMAX, 1>; break;
        case 2: kern = strip_filter_kernel<InT, OutT, TWMAX, 2>; break;
        case 3: kern = strip_filter_kernel<InT, OutT, TWMAX, 3>; break;
        case 4: kern = strip_filter_kernel<InT, OutT, TWMAX, 4>; break;
        default: return GF_EUNSUPPORTED;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    kern<<<grid, kThreads, smem, s>>>(maps[0], maps[1], maps[2], kp);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

template <typename InT, typename OutT, int TWMAX>
gf_status launch_batch_tw(const BatchArgs& ba, int C, int grid, size_t smem, cudaStream_t s) {
    void (*kern)(const BatchArgs) = nullptr;
    switch (C) {
        case 1: kern = batch_filter_kernel<InT, OutT, TWMAX, 1>; break;
        case 2: kern = batch_filter_kernel<InT, OutT, TWMAX, 2>; break;
        case 3: kern = batch_filter_kernel<InT, OutT, TWMAX, 3>; break;
        case 4: kern = batch_filter_kernel<InT, OutT, TWMAX, 4>; break;
        default: return GF_EUNSUPPORTED;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    kern<<<grid, kThreads, smem, s>>>(ba);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

template <typename InT, typename OutT>
gf_status launch_batch(const BatchArgs& ba, int C, int twmax, int grid, size_t smem, cudaStream_t s) {
    return twmax == 64 ? launch_batch_tw<InT, OutT, 64>(ba, C, grid, smem, s)
                       : launch_batch_tw<InT, OutT, 256>(ba, C, grid, smem, s);
}

template <typename InT, typename OutT>
gf_status launch_strip(const KParams& kp, const CUtensorMap* maps, dim3 grid, size_t smem, cudaStream_t s,
                       int twmax) {
    return twmax == 64 ? launch_strip_tw<InT, OutT, 64>(kp, maps, grid, smem, s)
                       : launch_strip_tw<InT, OutT, 256>(kp, maps, grid, smem, s);
}

template <typename InT>
gf_status launch_box_sums(const unsigned char* in, long long in_pitch, int32_t* out, long long out_pitch,
                          long long plane_stride, int H, int W, int C, int K, int4 r03, int r4, int rk, int TWp,
                          int m, int SP, int SROW, int boundary, dim3 grid, size_t smem, cudaStream_t s) {
    void (*kern)(const unsigned char*, long long, int32_t*, long long, long long, int, int, int, int4, int, int, int,
                 int, int, int, int) = nullptr;
    switch (C) {
        case 1: kern = row_box_sums_kernel<InT, 1>; break;
        case 2: kern = row_box_sums_kernel<InT, 2>; break;
        case 3: kern = row_box_sums_kernel<InT, 3>; break;
        case 4: kern = row_box_sums_kernel<InT, 4>; break;
        default: return GF_EUNSUPPORTED;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    kern<<<grid, kThreads, smem, s>>>(in, in_pitch, out, out_pitch, plane_stride, H, W, K, r03, r4, rk, TWp, m, SP,
                                      SROW, boundary);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

#define GB_DECLARE_STRIP(IN, OUT)                                                                       \
    extern template gf_status launch_strip<IN, OUT>(const KParams&, const CUtensorMap*, dim3, size_t, \
                                                    cudaStream_t, int);
#define GB_DECLARE_BATCH(IN, OUT) \
    extern template gf_status launch_batch<IN, OUT>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
#define GB_DECLARE_BOX(IN)                                                                                  \
    extern template gf_status launch_box_sums<IN>(const unsigned char*, long long, int32_t*, long long,   \
                                                  long long, int, int, int, int, int4, int, int, int, int, \
                                                  int, int, int, dim3, size_t, cudaStream_t);

}  // namespace gb
