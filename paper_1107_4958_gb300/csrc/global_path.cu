// Running sums kept in HBM: the filter for kernels whose largest radius is too
// wide for the shared-memory column ring (and row staging) of the other two
// paths.  Sec. 3.3 as written: one running sum per line (Eq. alg1) over the
// whole boundary-extended line, then Eq. indep at every (or every sampled)
// output, rows first, then columns (Sec. 3.4).
//
//   line prefix  per row (one warp per line, in 32-element chunks with a warp
//                scan) or per column (in 32 chunks of rows, one thread per
//                column and chunk, coalesced across the warp; the gather adds
//                each chunk's starting sum): the values of the extended line
//                [-rk - 1, n + rk]
//                scaled by the power of two 2^e that keeps every partial sum
//                of the line below 2^61, rounded and summed in int64 (exact
//                differences; integer inputs are summed as they are, e = 0).
//                int64 leaves ~2^-61 n of the range per value, so no offset
//                is subtracted: with huge boxes over zero-extended lines an
//                offset would come back as a large term cancelling against
//                the box sums.
//   line gather  Y = 2^-e sum_i w_i (P(x + r_i) - P(x - r_i - 1)), one thread
//                per output, into the FP32 intermediate (rows) or the output
//                (columns).
//
// Work and traffic per pixel grow with nothing but K; the extra cost against the
// two-pass form is the int64 prefix arrays (8 bytes per extended element per
// pass) written and re-read through HBM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "strip_kernel.cuh"
#include "twopass.h"

namespace gb {

namespace {

constexpr int kLineThreads = 256;

// Scale exponent for `n` values of magnitude below 2^(ex + 1): 2^e n 2^(ex+1) <= 2^61.
__device__ __forceinline__ int line_exponent(float mx, long long n) {
    if (!(mx > 0.f)) return 0;
    const int ex = (int)((__float_as_uint(mx) >> 23) & 0xffu) - 127;
    const int ln = 64 - __clzll(n - 1);   // ceil(log2 n)
    return max(-126, min(126, 61 - ln - (ex + 1)));
}

template <typename InT>
__device__ __forceinline__ float load_elem(const unsigned char* row, int e) {
    return (float)Elem<InT>::cvt(reinterpret_cast<const InT*>(row)[e]);
}

// One warp per row line (row y, channel c): P[l][t] for t in [0, N), N = W + 2 rk + 2,
// t the extended position x = t - rk - 1.
template <typename InT>
__global__ void __launch_bounds__(kLineThreads) row_prefix_kernel(const unsigned char* in, long long in_pitch,
                                                                  int H, int W, int C, int rk, int boundary,
                                                                  long long* P, float* wsc) {
    const int lane = threadIdx.x & 31;
    const long long l = (long long)blockIdx.x * (kLineThreads / 32) + (threadIdx.x >> 5);
    if (l >= (long long)H * C) return;
    const int y = (int)(l / C), c = (int)(l % C);
    const unsigned char* row = in + (long long)y * in_pitch;
    const long long N = (long long)W + 2 * rk + 2;
    auto value = [&](long long t) -> float {
        const int xs = fold_index((int)(t - rk - 1), W, boundary);
        return xs < 0 ? 0.f : load_elem<InT>(row, xs * C + c);
    };
    float sc = 1.f, inv = 1.f;
    if constexpr (!Elem<InT>::exact) {
        float mx = 0.f;
        for (long long t = lane; t < N; t += 32) mx = fmaxf(mx, fabsf(value(t)));
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, d));
        const int e = line_exponent(mx, N);
        sc = __uint_as_float((uint32_t)(e + 127) << 23);
        inv = __uint_as_float((uint32_t)(127 - e) << 23);
    }
    long long* p = P + l * N;
    long long carry = 0;
    for (long long base = 0; base < N; base += 32) {
        const long long t = base + lane;
        long long q = 0;
        if (t < N) {
            const float v = value(t);
            q = Elem<InT>::exact ? (long long)v : __float2ll_rn(__fmul_rn(v, sc));
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long o = __shfl_up_sync(0xffffffffu, q, d);
            if (lane >= d) q += o;
        }
        if (t < N) p[t] = carry + q;
        carry += __shfl_sync(0xffffffffu, q, 31);
    }
    if (lane == 0) wsc[l] = inv;
}

// Column lines in G chunks of L extended rows, one thread per (column, chunk).
// First the largest |value| of each column (atomic max on the bits of a
// non-negative float, which order like the values) ...
__global__ void __launch_bounds__(kLineThreads) col_max_kernel(const float* R, long long r_pitch_elems, int H,
                                                               int cols, int rows_per_chunk, unsigned* mxbits) {
    const int col = blockIdx.x * kLineThreads + threadIdx.x;
    if (col >= cols) return;
    const int y0 = blockIdx.y * rows_per_chunk, y1 = min(H, y0 + rows_per_chunk);
    float mx = 0.f;
    for (int y = y0; y < y1; ++y) mx = fmaxf(mx, fabsf(R[(long long)y * r_pitch_elems + col]));
    if (y0 < y1) atomicMax(&mxbits[col], __float_as_uint(mx));
}

// ... then each chunk's running sums from 0 (the extension repeats image values
// or reads 0) and its total; the column's scale is the same in every chunk.
__global__ void __launch_bounds__(kLineThreads) col_prefix_kernel(const float* R, long long r_pitch_elems, int H,
                                                                  int cols, int rk, int boundary, int L,
                                                                  const unsigned* mxbits, long long* P,
                                                                  long long* T, float* wsc) {
    const int col = blockIdx.x * kLineThreads + threadIdx.x;
    if (col >= cols) return;
    const long long N = (long long)H + 2 * rk + 2;
    const int e = line_exponent(__uint_as_float(mxbits[col]), N);
    const float sc = __uint_as_float((uint32_t)(e + 127) << 23);
    const long long t0 = (long long)blockIdx.y * L, t1 = min(N, t0 + L);
    long long run = 0;
    for (long long t = t0; t < t1; ++t) {
        const int ys = fold_index((int)(t - rk - 1), H, boundary);
        const float v = ys < 0 ? 0.f : R[(long long)ys * r_pitch_elems + col];
        run += __float2ll_rn(__fmul_rn(v, sc));
        P[t * cols + col] = run;
    }
    T[(long long)blockIdx.y * cols + col] = run;
    if (blockIdx.y == 0) wsc[col] = __uint_as_float((uint32_t)(127 - e) << 23);
}

// Chunk totals -> exclusive prefix (the running sum before each chunk), in place.
__global__ void __launch_bounds__(kLineThreads) col_chunk_scan_kernel(long long* T, int cols, int G) {
    const int col = blockIdx.x * kLineThreads + threadIdx.x;
    if (col >= cols) return;
    long long acc = 0;
    for (int g = 0; g < G; ++g) {
        const long long v = T[(long long)g * cols + col];
        T[(long long)g * cols + col] = acc;
        acc += v;
    }
}

struct Taps {
    int K, rk;
    int r[GF_KMAX];
    float w[GF_KMAX];
    float sw;
};

// Rows: R[y][j C + c] for the sampled columns x = ox + j sx.
__global__ void __launch_bounds__(kLineThreads) row_gather_kernel(const long long* P, const float* wsc, float* R,
                                                                  long long r_pitch_elems, int H, int W, int C,
                                                                  int Wo, int sx, int ox, Taps tp) {
    const long long idx = (long long)blockIdx.x * kLineThreads + threadIdx.x;
    const long long per_row = (long long)Wo * C;
    if (idx >= per_row * H) return;
    const int y = (int)(idx / per_row);
    const int e = (int)(idx % per_row);
    const int j = e / C, c = e % C;
    const int x = ox + j * sx;
    const long long l = (long long)y * C + c;
    const long long N = (long long)W + 2 * tp.rk + 2;
    const long long* p = P + l * N;
    const long long at = (long long)x + tp.rk + 1;   // P index of x
    const float s = wsc[l];
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < GF_KMAX; ++i) {
        if (i < tp.K) acc = fmaf(tp.w[i] * s, (float)(p[at + tp.r[i]] - p[at - tp.r[i] - 1]), acc);
    }
    R[(long long)y * r_pitch_elems + e] = acc;
}

// Columns: out[i][col] for the sampled rows y = oy + i sy.
template <typename OutT>
__global__ void __launch_bounds__(kLineThreads) col_gather_kernel(const long long* P, const long long* T, int L,
                                                                  const float* wsc, unsigned char* out,
                                                                  long long out_pitch, int H, int cols, int Ho,
                                                                  int sy, int oy, Taps tp) {
    const long long idx = (long long)blockIdx.x * kLineThreads + threadIdx.x;
    if (idx >= (long long)Ho * cols) return;
    const int i = (int)(idx / cols), col = (int)(idx % cols);
    const int y = oy + i * sy;
    const long long at = (long long)y + tp.rk + 1;
    const float s = wsc[col];
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < GF_KMAX; ++k) {
        if (k < tp.K) {
            const long long a = at + tp.r[k], b = at - tp.r[k] - 1;
            const long long pa = P[a * cols + col] + T[(a / L) * cols + col];
            const long long pb = P[b * cols + col] + T[(b / L) * cols + col];
            acc = fmaf(tp.w[k] * s, (float)(pa - pb), acc);
        }
    }
    reinterpret_cast<OutT*>(out + (long long)i * out_pitch)[col] = from_float<OutT>(acc);
}

unsigned grid_for(long long n) { return (unsigned)((n + kLineThreads - 1) / kLineThreads); }

template <typename InT>
void launch_row_prefix(const Image& im, int rk, long long* P, float* wsc, cudaStream_t s) {
    const long long nrow = (long long)im.H * im.C;
    row_prefix_kernel<InT><<<grid_for(nrow * 32), kLineThreads, 0, s>>>(
        static_cast<const unsigned char*>(im.in), (long long)im.in_pitch, im.H, im.W, im.C, rk, im.boundary, P, wsc);
}

template <typename OutT>
void launch_col_gather(const Image& im, const long long* P, const long long* T, int L, const float* wsc, int cols,
                       int Ho, const Taps& tp, cudaStream_t s) {
    col_gather_kernel<OutT><<<grid_for((long long)Ho * cols), kLineThreads, 0, s>>>(
        P, T, L, wsc, static_cast<unsigned char*>(im.out), (long long)im.out_pitch, im.H, cols, Ho, im.sy, im.oy, tp);
}

}  // namespace

namespace {

constexpr int kColChunks = 32;   // chunks per column line (parallel column prefix)

}  // namespace

size_t global_path_bytes(const Image& im, const BoxKernel& bk) {
    const size_t C = (size_t)im.C, rk = (size_t)bk.rk;
    const size_t Wo = (size_t)out_w(im);
    const size_t prow = (size_t)im.H * C * ((size_t)im.W + 2 * rk + 2) * 8;
    const size_t r = (size_t)im.H * Wo * C * 4;
    const size_t pcol = ((size_t)im.H + 2 * rk + 2) * Wo * C * 8;
    const size_t lines = ((size_t)im.H * C + Wo * C) * 4;              // scales
    const size_t chunks = (size_t)kColChunks * Wo * C * 8 + Wo * C * 4;   // chunk offsets, column maxima
    return std::max(prow, pcol) + r + lines + chunks + 8 * 256;
}

gf_status launch_global(const Image& im, const BoxKernel& bk, void* scratch, cudaStream_t s) {
    const int C = im.C, rk = bk.rk;
    const int Wo = out_w(im), Ho = out_h(im);
    const long long cols = (long long)Wo * C;
    const long long nrow = (long long)im.H * C;
    if ((long long)im.W + 2 * rk + 2 > INT32_MAX / 2 || (long long)im.H + 2 * rk + 2 > INT32_MAX / 2)
        return GF_EUNSUPPORTED;
    if (grid_for(nrow * 32) == 0 || (long long)grid_for(cols * im.H) > INT32_MAX) return GF_EUNSUPPORTED;
    // scratch: [prefix arrays (rows, then reused for columns)][R][line scales]
    unsigned char* base = static_cast<unsigned char*>(scratch);
    const size_t prow = (size_t)nrow * ((size_t)im.W + 2 * rk + 2) * 8;
    const size_t pcol = ((size_t)im.H + 2 * rk + 2) * (size_t)cols * 8;
    long long* P = reinterpret_cast<long long*>(base);
    float* R = reinterpret_cast<float*>(base + (std::max(prow, pcol) + 255) / 256 * 256);
    const size_t rbytes = (size_t)im.H * (size_t)cols * 4;
    float* wsc = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(R) + (rbytes + 255) / 256 * 256);
    const size_t nlines = (size_t)std::max(nrow, cols);
    long long* T = reinterpret_cast<long long*>(reinterpret_cast<unsigned char*>(wsc) + (nlines * 4 + 255) / 256 * 256);
    unsigned* mxbits = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(T) +
                                                   ((size_t)kColChunks * cols * 8 + 255) / 256 * 256);
    Taps tp{};
    tp.K = bk.K;
    tp.rk = rk;
    for (int i = 0; i < GF_KMAX; ++i) {
        tp.r[i] = bk.r[i];
        tp.w[i] = bk.w[i];
    }
    tp.sw = bk.sw;
    switch (im.in_dt) {
        case GF_U8: launch_row_prefix<uint8_t>(im, rk, P, wsc, s); break;
        case GF_U16: launch_row_prefix<uint16_t>(im, rk, P, wsc, s); break;
        case GF_F32: launch_row_prefix<float>(im, rk, P, wsc, s); break;
        case GF_BF16: launch_row_prefix<__nv_bfloat16>(im, rk, P, wsc, s); break;
        case GF_F16: launch_row_prefix<__half>(im, rk, P, wsc, s); break;
        default: return GF_EUNSUPPORTED;
    }
    row_gather_kernel<<<grid_for((long long)im.H * cols), kLineThreads, 0, s>>>(P, wsc, R, cols, im.H, im.W, C, Wo,
                                                                            im.sx, im.ox, tp);
    // column prefix in kColChunks chunks per column
    const long long ncol = (long long)im.H + 2 * rk + 2;
    const int L = (int)((ncol + kColChunks - 1) / kColChunks);
    const int G = (int)((ncol + L - 1) / L);
    const int hrows = (im.H + kColChunks - 1) / kColChunks;
    if (cudaMemsetAsync(mxbits, 0, (size_t)cols * 4, s) != cudaSuccess) return GF_ECUDA;
    col_max_kernel<<<dim3(grid_for(cols), (im.H + hrows - 1) / hrows), kLineThreads, 0, s>>>(R, cols, im.H, (int)cols,
                                                                                           hrows, mxbits);
    col_prefix_kernel<<<dim3(grid_for(cols), G), kLineThreads, 0, s>>>(R, cols, im.H, (int)cols, rk, im.boundary, L,
                                                                       mxbits, P, T, wsc);
    col_chunk_scan_kernel<<<grid_for(cols), kLineThreads, 0, s>>>(T, (int)cols, G);
    switch (im.out_dt) {
        case GF_F32: launch_col_gather<float>(im, P, T, L, wsc, (int)cols, Ho, tp, s); break;
        case GF_BF16: launch_col_gather<__nv_bfloat16>(im, P, T, L, wsc, (int)cols, Ho, tp, s); break;
        case GF_F16: launch_col_gather<__half>(im, P, T, L, wsc, (int)cols, Ho, tp, s); break;
        default: return GF_EUNSUPPORTED;
    }
    return cudaGetLastError() == cudaSuccess ? GF_OK : GF_ECUDA;
}

}  // namespace gb
