// Fused box-sum Gaussian filter for sm_103a (Sec. 3.3-3.4).
//
// One CTA owns a strip of TWp output pixels (all C channels) by TH output rows.
// It walks the "virtual" rows y0 - rk .. y0 + TH - 1 + rk of its strip (rows
// outside the image are mapped by the boundary rule) in bands of kBand rows:
//
//   1. TMA stages each row segment [x0 - rk, x0 + TWp + rk) of the band into
//      shared memory (one 2D box per row piece, completion on an mbarrier).
//   2. Row pass, one warp per (row, channel): the tile-local running sum
//      I(j) = sum_{t <= j} f(t) (Eq. alg1) from lane-local sums plus a warp
//      shuffle scan, then per pixel sum_i w_i (I(x + r_i) - I(x - r_i - 1))
//      (Eq. indep).  Integer inputs use exact int32 sums; float inputs use FP32
//      with a per-tile offset and Kahan-compensated accumulation.
//   3. Column pass, one thread per column: the column running sum J of the
//      row-filtered values (Kahan, per-column offset) goes into a ring of
//      2 rk + 2 rows in shared memory, and each finished output row is
//      sum_i w_i (J(y + r_i) - J(y - r_i - 1)), stored straight to HBM.
//
// Every running sum starts inside the tile (it needs only +-(rk + 1) of
// context), so there is no carry between CTAs and no inter-CTA wait.  Only the
// mbarrier waits of the TMA pipeline are bounded waits; on expiry the CTA sets
// the device status word and leaves.
#include "internal.h"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>

namespace gb {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBand = 8;
constexpr int kStages = 3;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

__device__ int g_device_status = 0;

struct KParams {
    const unsigned char* in;
    long long in_pitch;
    unsigned char* out;
    long long out_pitch;
    int H, W, C, boundary;
    int K;
    int r[GF_KMAX];
    float w[GF_KMAX];
    float sw;
    int rk;
    int TWp, TH, TW;
    int S;       // running-sum entries per row segment: TWp + 2 rk + 1
    int m;       // entries per lane in the segment scan (odd: conflict-free)
    int SP;      // per-warp running-sum buffer stride (entries)
    int SROW;    // staged elements per row
    int nbox, boxw, ealign;
    int L;       // column ring rows: 2 rk + 2
    int nstage;  // staged bands resident at once
    int use_tma;
    int off_stage, off_p, off_rband, off_ring, off_bar;
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
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase did not complete within kWaitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}
__device__ __forceinline__ void tma_load_row(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_addr(dst)), "l"(map), "r"(smem_addr(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void set_status(int code) { atomicCAS(&g_device_status, 0, code); }

// ---------------------------------------------------------------- element types
template <typename T> struct Elem;
template <> struct Elem<uint8_t> {
    using acc = int;
    static __device__ __forceinline__ int get(const uint8_t* s, int i) { return s[i]; }
};
template <> struct Elem<uint16_t> {
    using acc = int;
    static __device__ __forceinline__ int get(const uint16_t* s, int i) { return s[i]; }
};
template <> struct Elem<float> {
    using acc = float;
    static __device__ __forceinline__ float get(const float* s, int i) { return s[i]; }
};
template <> struct Elem<__nv_bfloat16> {
    using acc = float;
    static __device__ __forceinline__ float get(const __nv_bfloat16* s, int i) { return __bfloat162float(s[i]); }
};
template <> struct Elem<__half> {
    using acc = float;
    static __device__ __forceinline__ float get(const __half* s, int i) { return __half2float(s[i]); }
};

template <typename T> __device__ __forceinline__ T from_float(float v);
template <> __device__ __forceinline__ float from_float<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_float<__half>(float v) { return __float2half_rn(v); }

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
// Kahan step: adds x to the running sum (s, c), true sum ~= s - c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// ---------------------------------------------------------------- row prefix
// Tile-local running sum of one row segment (Eq. alg1), by one warp.
// Positions j = 0 .. S-1 stand for pixels t = xs + j, xs = x0 - rk - 1; P[0] = 0
// and P[j] = sum_{xs < t <= xs + j} (f(t) - off).  `srow` holds staged elements
// ebase .. ebase + srow_len - 1 of the image row; channel c of pixel t sits at
// element t*C + c.  Returns `off` (0 for integer inputs).
template <typename T>
__device__ __forceinline__ typename Elem<T>::acc row_prefix(const T* srow, int srow_len, int ebase, int x0, int c,
                                                            int C, int W, int rk, int S, int m, int boundary,
                                                            bool hedge, typename Elem<T>::acc* P, int lane) {
    using A = typename Elem<T>::acc;
    const int xs = x0 - rk - 1;
    auto load = [&](int j) -> A {
        int t = xs + j;
        if (hedge) {
            t = fold_index(t, W, boundary);
            if (t < 0) return A(0);
        }
        int idx = t * C + c - ebase;
        idx = min(max(idx, 0), srow_len - 1);
        return Elem<T>::get(srow, idx);
    };
    A off = A(0);
    const int j0 = 1 + lane * m;
    const int j1 = min(j0 + m, S);
    if constexpr (std::is_floating_point<A>::value) {
        // ---- float path: per-tile offset + Kahan + double-float warp scan
        off = Elem<T>::get(srow, min(max(x0 * C + c - ebase, 0), srow_len - 1));
        float s = 0.f, cc = 0.f;
        for (int j = j0; j < j1; ++j) kahan_add(s, cc, __fsub_rn(load(j), off));
        float hi = s, lo = -cc;
        // inclusive scan of (hi, lo) pairs
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float oh = __shfl_up_sync(0xffffffffu, hi, d);
            const float ol = __shfl_up_sync(0xffffffffu, lo, d);
            if (lane >= d) pair_add(oh, ol, hi, lo, hi, lo);
        }
        float eh = __shfl_up_sync(0xffffffffu, hi, 1);
        float el = __shfl_up_sync(0xffffffffu, lo, 1);
        if (lane == 0) { eh = 0.f; el = 0.f; }
        s = eh;
        cc = -el;
        for (int j = j0; j < j1; ++j) {
            kahan_add(s, cc, __fsub_rn(load(j), off));
            P[j] = __fsub_rn(s, cc);
        }
    } else {
        // ---- integer path: exact int32 sums
        int tot = 0;
        for (int j = j0; j < j1; ++j) tot += load(j);
        int inc = tot;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += o;
        }
        int run = inc - tot;
        for (int j = j0; j < j1; ++j) {
            run += load(j);
            P[j] = run;
        }
    }
    if (lane == 0) P[0] = A(0);
    __syncwarp();
    return off;
}

// ---------------------------------------------------------------- fused kernel
template <typename InT, typename OutT>
__global__ void __launch_bounds__(kThreads) strip_filter_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                const KParams p) {
    using A = typename Elem<InT>::acc;
    extern __shared__ __align__(128) unsigned char smem[];
    InT* stage = reinterpret_cast<InT*>(smem + p.off_stage);
    A* pbuf = reinterpret_cast<A*>(smem + p.off_p);
    float* rband = reinterpret_cast<float*>(smem + p.off_rband);
    float* ring = reinterpret_cast<float*>(smem + p.off_ring);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + p.off_bar);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * p.TWp;
    const int y0 = blockIdx.y * p.TH;
    if (y0 >= p.H || x0 >= p.W) return;
    const int yend = min(y0 + p.TH, p.H);
    const int vstart = y0 - p.rk;
    const int vend = yend - 1 + p.rk;
    const int nbands = (vend - vstart + 1 + kBand - 1) / kBand;
    const int e0 = (x0 - p.rk) * p.C;
    const int ebase = (e0 >= 0 ? e0 / p.ealign : -((-e0 + p.ealign - 1) / p.ealign)) * p.ealign;
    const bool hedge = (x0 - p.rk < 0) || (x0 + p.TWp + p.rk > p.W);
    const int rowlen = p.W * p.C;
    const int TW = p.TW;
    const int ecol0 = x0 * p.C;
    const int row_bytes = p.nbox * p.boxw * (int)sizeof(InT);

    // Thread 0 stages band b (rows inside the band and inside the image or the
    // boundary rule) into stage slot b % nstage.
    auto issue_band = [&](int b) {
        const int slot = b % p.nstage;
        InT* dst = stage + (size_t)slot * kBand * p.SROW;
        uint32_t bytes = 0;
        int yrs[kBand];
#pragma unroll
        for (int r = 0; r < kBand; ++r) {
            const int v = vstart + b * kBand + r;
            yrs[r] = (v <= vend) ? fold_index(v, p.H, p.boundary) : -1;
            if (yrs[r] >= 0) bytes += row_bytes;
        }
        mbar_arrive_expect_tx(&bars[slot], bytes);
#pragma unroll
        for (int r = 0; r < kBand; ++r) {
            if (yrs[r] < 0) continue;
            for (int k = 0; k < p.nbox; ++k)
                tma_load_row(dst + (size_t)r * p.SROW + (size_t)k * p.boxw, &tmap, &bars[slot], ebase + k * p.boxw,
                             yrs[r]);
        }
    };

    if (p.use_tma) {
        if (tid == 0) {
            for (int s = 0; s < p.nstage; ++s) mbar_init(&bars[s], 1);
            fence_barrier_init();
        }
        __syncthreads();
        if (tid == 0) {
            for (int b = 0; b < min(p.nstage, nbands); ++b) issue_band(b);
        }
    }
    // ring slot 0 holds J(vstart - 1) = 0
    for (int e = tid; e < TW; e += kThreads) ring[e] = 0.f;

    // column-pass state (one column per thread; TW <= kThreads)
    const int e = tid;
    float js = 0.f, jc = 0.f, coff = 0.f;
    int slot_next = 1;
    bool ok = true;
    int band = 0;

    for (; band < nbands; ++band) {
        const int sidx = p.use_tma ? band % p.nstage : 0;
        const InT* sband = stage + (size_t)sidx * kBand * p.SROW;
        if (p.use_tma) {
            const bool mine = mbar_wait_bounded(&bars[sidx], (uint32_t)((band / p.nstage) & 1));
            ok = __syncthreads_and(mine) != 0;
            if (!ok) break;
        } else {
            __syncthreads();
            InT* dst = stage;
            for (int r = 0; r < kBand; ++r) {
                const int v = vstart + band * kBand + r;
                const int yr = (v <= vend) ? fold_index(v, p.H, p.boundary) : -1;
                const InT* src = reinterpret_cast<const InT*>(p.in + (long long)max(yr, 0) * p.in_pitch);
                for (int i = tid; i < p.SROW; i += kThreads) {
                    const int ee = ebase + i;
                    InT val;
                    if (yr >= 0 && ee >= 0 && ee < rowlen) val = src[ee];
                    else memset(&val, 0, sizeof(InT));
                    dst[(size_t)r * p.SROW + i] = val;
                }
            }
            __syncthreads();
        }

        // ---------------- row pass: warp per (row, channel) segment
        float* rb = rband + (size_t)(band & 1) * kBand * TW;
        A* P = pbuf + (size_t)warp * p.SP;
        for (int seg = warp; seg < kBand * p.C; seg += kWarps) {
            const int r = seg / p.C;
            const int c = seg - r * p.C;
            const int v = vstart + band * kBand + r;
            if (v > vend) continue;
            float* rrow = rb + (size_t)r * TW;
            if (p.boundary == GF_ZERO && (v < 0 || v >= p.H)) {
                for (int q = lane; q < p.TWp; q += 32) rrow[q * p.C + c] = 0.f;
                continue;
            }
            const InT* srow = sband + (size_t)r * p.SROW;
            const A off = row_prefix<InT>(srow, p.SROW, ebase, x0, c, p.C, p.W, p.rk, p.S, p.m, p.boundary, hedge, P,
                                          lane);
            for (int q = lane; q < p.TWp; q += 32) {
                const int jx = q + p.rk + 1;
                float acc;
                if constexpr (std::is_floating_point<A>::value) acc = off * p.sw;
                else acc = 0.f;
#pragma unroll
                for (int i = 0; i < GF_KMAX; ++i) {
                    if (i < p.K) {
                        const A d = P[jx + p.r[i]] - P[jx - p.r[i] - 1];
                        acc = fmaf(p.w[i], (float)d, acc);
                    }
                }
                rrow[q * p.C + c] = acc;
            }
            __syncwarp();
        }
        __syncthreads();
        if (p.use_tma && tid == 0 && band + p.nstage < nbands) {
            fence_proxy_async();
            issue_band(band + p.nstage);
        }

        // ---------------- column pass: thread per column
        if (e < TW) {
            for (int r = 0; r < kBand; ++r) {
                const int v = vstart + band * kBand + r;
                if (v > vend) break;
                const float val = rb[(size_t)r * TW + e];
                if (v == vstart) coff = val;
                kahan_add(js, jc, __fsub_rn(val, coff));
                const int cur = slot_next;
                ring[(size_t)cur * TW + e] = __fsub_rn(js, jc);
                slot_next = (cur + 1 == p.L) ? 0 : cur + 1;
                const int y = v - p.rk;
                if (y >= y0 && ecol0 + e < rowlen) {
                    float acc = coff * p.sw;
#pragma unroll
                    for (int i = 0; i < GF_KMAX; ++i) {
                        if (i < p.K) {
                            int sp = cur - (p.rk - p.r[i]);
                            if (sp < 0) sp += p.L;
                            int sm = cur - (p.rk + p.r[i] + 1);
                            if (sm < 0) sm += p.L;
                            acc = fmaf(p.w[i], __fsub_rn(ring[(size_t)sp * TW + e], ring[(size_t)sm * TW + e]), acc);
                        }
                    }
                    OutT* orow = reinterpret_cast<OutT*>(p.out + (long long)y * p.out_pitch);
                    orow[ecol0 + e] = from_float<OutT>(acc);
                }
            }
        }
    }

    if (!ok) {
        if (tid == 0) {
            set_status(GF_ETIMEOUT);
            // let the copies already in flight land before the CTA leaves
            for (int b = band; b < min(band + p.nstage, nbands); ++b)
                (void)mbar_wait_bounded(&bars[b % p.nstage], (uint32_t)((b / p.nstage) & 1));
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ integer box sums
// K exact int32 box-sum planes along rows, using the same row_prefix code.
template <typename InT>
__global__ void __launch_bounds__(kThreads) row_box_sums_kernel(const unsigned char* in, long long in_pitch,
                                                                int32_t* out, long long out_pitch,
                                                                long long plane_stride, int H, int W, int C,
                                                                int K, int4 r03, int r4, int rk, int TWp, int S,
                                                                int m, int SP, int SROW, int boundary) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    InT* srow = reinterpret_cast<InT*>(smem) + (size_t)warp * SROW;
    const size_t p_off = ((size_t)kWarps * SROW * sizeof(InT) + 15) & ~size_t(15);
    int* P = reinterpret_cast<int*>(smem + p_off) + (size_t)warp * SP;
    const int rr[GF_KMAX] = {r03.x, r03.y, r03.z, r03.w, r4};
    const int x0 = blockIdx.x * TWp;
    const int ebase = (x0 - rk - 1) * C;
    const int rowlen = W * C;
    const int nseg = H * C;
    for (int seg = blockIdx.y * kWarps + warp; seg < nseg; seg += gridDim.y * kWarps) {
        const int y = seg / C;
        const int c = seg - y * C;
        const InT* src = reinterpret_cast<const InT*>(in + (long long)y * in_pitch);
        for (int i = lane; i < SROW; i += 32) {
            const int ee = ebase + i;
            srow[i] = (ee >= 0 && ee < rowlen) ? src[ee] : InT(0);
        }
        __syncwarp();
        const bool hedge = (x0 - rk < 0) || (x0 + TWp + rk > W);
        (void)row_prefix<InT>(srow, SROW, ebase, x0, c, C, W, rk, S, m, boundary, hedge, P, lane);
        for (int q = lane; q < TWp && x0 + q < W; q += 32) {
            const int jx = q + rk + 1;
            for (int i = 0; i < K; ++i) {
                int32_t* o = out + (long long)i * plane_stride;
                o = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(o) + (long long)y * out_pitch);
                o[(x0 + q) * C + c] = P[jx + rr[i]] - P[jx - rr[i] - 1];
            }
        }
        __syncwarp();
    }
}

// ======================================================================= host
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
int g_sms = 0;
std::once_flag g_dev_once;
void query_device() {
    std::call_once(g_dev_once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_max_smem <= 0) g_max_smem = 227 * 1024;
        if (g_sms <= 0) g_sms = 148;
    });
}

// Fills the plan-dependent part of KParams; returns the dynamic smem bytes.
size_t layout(KParams& kp, const Image& im, const BoxKernel& bk, int TWp, bool tma) {
    const int isz = dtype_size(im.in_dt);
    kp.TWp = TWp;
    kp.TW = TWp * im.C;
    kp.S = TWp + 2 * bk.rk + 1;
    kp.m = ((kp.S - 1) + 31) / 32;
    kp.m |= 1;
    kp.SP = round_up(kp.S, 4);
    kp.ealign = 16 / isz;
    const int need = (TWp + 2 * bk.rk) * im.C + kp.ealign - 1;
    kp.nbox = (need + 255) / 256;
    kp.boxw = round_up((need + kp.nbox - 1) / kp.nbox, 128 / isz);
    kp.SROW = kp.nbox * kp.boxw;
    kp.L = 2 * bk.rk + 2;
    kp.nstage = tma ? kStages : 1;
    kp.use_tma = tma ? 1 : 0;
    size_t off = 0;
    kp.off_stage = (int)off;
    off += (size_t)kp.nstage * kBand * kp.SROW * isz;
    off = (off + 127) / 128 * 128;
    kp.off_p = (int)off;
    off += (size_t)kWarps * kp.SP * 4;
    off = (off + 127) / 128 * 128;
    kp.off_rband = (int)off;
    off += (size_t)2 * kBand * kp.TW * 4;
    kp.off_ring = (int)off;
    off += (size_t)kp.L * kp.TW * 4;
    off = (off + 15) / 16 * 16;
    kp.off_bar = (int)off;
    off += (size_t)kStages * 8;
    return off;
}

template <typename InT, typename OutT>
gf_status launch_typed(const KParams& kp, const CUtensorMap& map, dim3 grid, size_t smem, cudaStream_t s) {
    auto kern = strip_filter_kernel<InT, OutT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GF_ECUDA;
    kern<<<grid, kThreads, smem, s>>>(map, kp);
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

template <typename InT>
gf_status launch_out(int out_dt, const KParams& kp, const CUtensorMap& map, dim3 grid, size_t smem, cudaStream_t s) {
    switch (out_dt) {
        case GF_F32: return launch_typed<InT, float>(kp, map, grid, smem, s);
        case GF_BF16: return launch_typed<InT, __nv_bfloat16>(kp, map, grid, smem, s);
        case GF_F16: return launch_typed<InT, __half>(kp, map, grid, smem, s);
        default: return GF_EUNSUPPORTED;
    }
}

}  // namespace

int device_sm_count() {
    query_device();
    return g_sms;
}

StripPlan default_plan(const Image& im, const BoxKernel& bk) {
    query_device();
    StripPlan pl;
    int twp = std::min(kThreads / im.C, im.W);
    KParams kp{};
    while (twp > 1 && layout(kp, im, bk, twp, true) > (size_t)g_max_smem) twp = twp * 3 / 4;
    pl.TWp = std::max(twp, 1);
    pl.nstrips = (im.W + pl.TWp - 1) / pl.TWp;
    // rows per CTA: enough CTAs for two per SM, but keep the vertical halo
    // (2 rk rows recomputed per CTA) small against the tile height.
    const size_t smem = layout(kp, im, bk, pl.TWp, true);
    const int per_sm = std::max(1, std::min(2, (int)(g_max_smem / std::max<size_t>(smem, 1))));
    const int target = per_sm * g_sms;
    int rows = (im.H + std::max(1, target / pl.nstrips) - 1) / std::max(1, target / pl.nstrips);
    rows = std::max(rows, std::min(im.H, std::max(32, 2 * bk.rk)));
    pl.TH = std::max(1, std::min(rows, im.H));
    pl.nrowtiles = (im.H + pl.TH - 1) / pl.TH;
    return pl;
}

gf_status launch_filter(const Image& im, const BoxKernel& bk, const StripPlan* plan_in, void* stream) {
    query_device();
    const StripPlan pl = plan_in ? *plan_in : default_plan(im, bk);
    if (pl.TWp < 1 || pl.TH < 1 || pl.TWp * im.C > kThreads) return GF_EINVAL;
    KParams kp{};
    kp.in = static_cast<const unsigned char*>(im.in);
    kp.in_pitch = (long long)im.in_pitch;
    kp.out = static_cast<unsigned char*>(im.out);
    kp.out_pitch = (long long)im.out_pitch;
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
    const bool tma_env = getenv("GF_NO_TMA") == nullptr;
    bool tma = tma_ok && tma_env;
    size_t smem = layout(kp, im, bk, pl.TWp, tma);
    if (smem > (size_t)g_max_smem) {
        tma = false;
        smem = layout(kp, im, bk, pl.TWp, false);
        if (smem > (size_t)g_max_smem) return GF_EUNSUPPORTED;
    }
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
    switch (im.in_dt) {
        case GF_U8:
            if (im.out_dt != GF_F32) return GF_EUNSUPPORTED;
            return launch_typed<uint8_t, float>(kp, map, grid, smem, s);
        case GF_U16:
            if (im.out_dt != GF_F32) return GF_EUNSUPPORTED;
            return launch_typed<uint16_t, float>(kp, map, grid, smem, s);
        case GF_F32: return launch_out<float>(im.out_dt, kp, map, grid, smem, s);
        case GF_BF16: return launch_out<__nv_bfloat16>(im.out_dt, kp, map, grid, smem, s);
        case GF_F16: return launch_out<__half>(im.out_dt, kp, map, grid, smem, s);
        default: return GF_EUNSUPPORTED;
    }
}

gf_status launch_row_box_sums(const void* in, size_t in_pitch, int32_t* out, size_t out_pitch, size_t plane_stride,
                              int H, int W, int C, int in_dt, const BoxKernel& bk, int boundary, void* stream) {
    query_device();
    const int isz = dtype_size(in_dt);
    int TWp = std::min(W, 512);
    const int rk = bk.rk;
    auto smem_for = [&](int twp, int& S, int& m, int& SP, int& SROW) {
        S = twp + 2 * rk + 1;
        m = ((S - 1 + 31) / 32) | 1;
        SP = round_up(S, 4);
        SROW = round_up((twp + 2 * rk + 2) * C, 16);
        return (size_t)kWarps * SROW * isz + 16 + (size_t)kWarps * SP * 4;
    };
    int S, m, SP, SROW;
    while (TWp > 1 && smem_for(TWp, S, m, SP, SROW) > (size_t)g_max_smem) TWp /= 2;
    size_t smem = smem_for(TWp, S, m, SP, SROW);
    if (smem > (size_t)g_max_smem) return GF_EUNSUPPORTED;
    const int nstrips = (W + TWp - 1) / TWp;
    const int ny = std::max(1, std::min((H * C + kWarps - 1) / kWarps, 4 * g_sms / std::max(1, nstrips) + 1));
    dim3 grid(nstrips, ny);
    const int4 r03 = make_int4(bk.r[0], bk.r[1], bk.r[2], bk.r[3]);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (in_dt == GF_U8) {
        auto k = row_box_sums_kernel<uint8_t>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return GF_ECUDA;
        k<<<grid, kThreads, smem, s>>>(static_cast<const unsigned char*>(in), (long long)in_pitch, out,
                                        (long long)out_pitch, (long long)plane_stride, H, W, C, bk.K, r03, bk.r[4],
                                        rk, TWp, S, m, SP, SROW, boundary);
    } else if (in_dt == GF_U16) {
        auto k = row_box_sums_kernel<uint16_t>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return GF_ECUDA;
        k<<<grid, kThreads, smem, s>>>(static_cast<const unsigned char*>(in), (long long)in_pitch, out,
                                        (long long)out_pitch, (long long)plane_stride, H, W, C, bk.K, r03, bk.r[4],
                                        rk, TWp, S, m, SP, SROW, boundary);
    } else {
        return GF_EUNSUPPORTED;
    }
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
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
