// Fused filter for single-channel integer images whose radii are compile-time
// constants (Sec. 3.3-3.4).  The library compiles this text at run time with
// NVRTC once per radius set (walker_host.cu prepends the WK_* constants) and
// caches the result.
//
// With the radii fixed at compile time, every tap of Eq. indep,
//     sum_i w_i (I(x + r_i) - I(x - r_i - 1)),
// reads a running sum at a fixed distance behind the newest one, so a thread
// that walks a line keeps the last 2 r_K + 2 running sums in registers and
// forms each output from them with no shared-memory or tensor-memory traffic.
// A CTA owns a strip of WK_TW output columns by TH output rows and repeats, per
// band of WK_P rows (WK_P / WK_LC chunks of WK_LC rows):
//
//   row phase     thread t walks row t of the band along x: it reads the
//                 WK_TW + 2 r_K + 1 input pixels the strip needs (aligned
//                 16-byte loads, or a boundary-folded copy in shared memory at
//                 the image edges), keeps the running sum I (Eq. alg1, exact:
//                 8-bit pixels are summed as the integer bits of 2^23 + I, so
//                 that the FP32 views of two such words differ by exactly the
//                 box sum; 16-bit pixels in FP32, integers below 2^24) and
//                 writes the row result R of its WK_TW outputs to the band,
//                 forming two adjacent outputs per packed FP32x2 operation;
//   column phase  thread c walks column c down the band: the column running
//                 sum J of R, kept as a pair (Jh, Jl) with Jh the sum of R
//                 rounded to multiples of a power of two q (exact: every
//                 partial sum is a multiple of q below 2^24 q) and Jl the sum
//                 of the rounding residues (tiny), so a difference of two J is
//                 Jh-exact plus a residue difference of negligible error,
//                 whatever the magnitude of J; each output is the weighted sum
//                 of WK_K such differences.  Outputs overwrite the R value the
//                 same thread has just consumed, so each chunk of the band
//                 becomes a WK_LC x WK_TW output tile in place, which leaves by
//                 one TMA box (strips inside the image, output rows 16-byte
//                 aligned) or by plain stores of the thread's own column.
//
// Barriers: after the row phase; after each group of column chunks (then
// thread 0 issues their tile stores, which proceed while the next chunks are
// computed); before the next row phase overwrites the band (thread 0 has
// waited for the stores to read it).  Rows above and below the
// image are supplied by the boundary rule, rows beyond the last one an output
// needs are zero.

#pragma once

// Kernel arguments (shared with the host code, which includes this file
// without the WK_* constants and so sees only these structs).
struct WalkParams {
    const unsigned char* in;
    long long in_pitch;
    unsigned char* out;
    long long out_pitch;
    int H, W, boundary;
    int aligned;      // input base and pitch are multiples of 16 bytes
    int nch;          // row chunks (of WK_LC rows) one tile walks
    int th;           // output rows per tile = nch * WK_LC - 2 rk
    int tma_out;      // the output map is valid: strips inside the image store tiles by TMA
    int ty0;          // row tile of blockIdx.y == 0 (a launch may cover a slab of row tiles)
    float w[5];
    float q, magic;   // column quantum (a power of two) and 1.5 * 2^23 * q
    // Stacks (kernels compiled with WK_Z = 1): blockIdx.z is the slice, an
    // image of H rows whose input starts in_z bytes and output out_z bytes
    // after the previous slice's; rows fold within the slice.
    long long in_z, out_z;
};

// A TMA tensor map (the driver's 128-byte descriptor), passed by value.  The
// output map views the image as (column within strip, strip, row) with
// extents (WK_TW, W / WK_TW, H); its box (WK_RP, 1, WK_LC) matches a chunk's
// rows in shared memory, the columns past WK_TW falling outside the view.  A
// stack's map adds the slice as a fourth dimension (extent D, box 1), so a
// chunk's rows past a slice's last row fall outside the view as well.
struct alignas(64) WalkMap {
    unsigned long long v[16];
};

#ifdef WK_TW

#ifndef WK_Z
#define WK_Z 0                                     // 1: the launch covers a stack of slices (blockIdx.z)
#endif
#define WK_EB (WK_IN == 0 ? 1 : 2)                 // input bytes per pixel
#define WK_STEPS (WK_TW + 2 * WK_RK + 1)           // row walk: pixels x0 - rk - 1 .. x0 + TW + rk - 1
// byte offset of walk step 0 inside its 16-byte chunk (x0 is a multiple of WK_TW, so it is a constant)
#define WK_SHB ((((-(WK_RK + 1) * WK_EB) % 16) + 16) % 16)
#define WK_NCH ((WK_SHB + WK_STEPS * WK_EB + 15) / 16)   // 16-byte chunks the walk reads
#define WK_G ((32 + WK_LC - 1) / WK_LC)                    // column chunks per group of tile stores
// Set by the host: WK_RP floats per band row, WK_CS floats per chunk of WK_LC
// rows (a multiple of 32: chunks start on 128-byte boundaries), WK_STAGE_OFF
// the byte offset of the folded input copy of edge strips inside a row,
// WK_WIN the bytes of each row's edge window (0: none) at byte WK_WIN_OFF of
// shared memory.

__device__ __forceinline__ int wk_fold(int t, int n, int boundary) {
    if (t >= 0 && t < n) return t;
    if (boundary == 1) return -1;             // zero
    if (boundary == 0) return t < 0 ? 0 : n - 1;   // replicate
    if (n == 1) return 0;                     // reflect, folded as often as needed
    const int period = 2 * (n - 1);
    int m = t % period;
    if (m < 0) m += period;
    return m < n ? m : period - m;
}

// The element at position k of a 32-bit word: for 8-bit input the byte,
// zero-extended; for 16-bit input 2^23 + the half-word, as FP32 bits.
__device__ __forceinline__ unsigned int wk_elem(unsigned int word, int k) {
#if WK_IN == 0
    return __byte_perm(word, 0u, 0x4440u + (unsigned)k);
#else
    return __byte_perm(word, 0x4B000000u, 0x7600u + (unsigned)(2 * k) + ((unsigned)(2 * k + 1) << 4));
#endif
}

__device__ __forceinline__ unsigned int wk_smem(const void* p) {
    return (unsigned int)__cvta_generic_to_shared(p);
}

// Column chunk: WK_LC rows of the band at `cb` (this thread's column), the
// running sums carried in `ring`.  FIRST: the tile's first chunk, whose only
// outputs are its last two rows (tile rows 2 rk, 2 rk + 1), stored to `ofirst`
// (output row y0) when `on`; otherwise every row's output replaces its R.
template <bool FIRST>
__device__ __forceinline__ void wk_chunk(float2 (&ring)[WK_LC], float* cb, const WalkParams& p,
                                         unsigned char* ofirst, int rows_left, bool on) {
    const float2 w0 = make_float2(p.w[0], p.w[0]);
#if WK_K > 1
    const float2 w1 = make_float2(p.w[1], p.w[1]);
#endif
#if WK_K > 2
    const float2 w2 = make_float2(p.w[2], p.w[2]);
#endif
#if WK_K > 3
    const float2 w3 = make_float2(p.w[3], p.w[3]);
#endif
#if WK_K > 4
    const float2 w4 = make_float2(p.w[4], p.w[4]);
#endif
#pragma unroll
    for (int s = 0; s < WK_LC; ++s) {
        const float R = cb[s * WK_RP];
        // R = Rh + Rl: Rh the nearest multiple of q, Rl the (exact) residue;
        // J(u) = J(u - 1) + (Rh, Rl) as one packed addition
        const float Rh = __fsub_rn(__fadd_rn(R, p.magic), p.magic);
        ring[s] = __fadd2_rn(ring[(s + WK_LC - 1) % WK_LC], make_float2(Rh, __fsub_rn(R, Rh)));
        if (!FIRST || s >= 2 * WK_RK) {
            // output of tile row u = s (mod LC): J(u - rk + r_i) - J(u - rk - r_i - 1)
#define WK_TAP(R_, W_)                                                                              \
    {                                                                                               \
        const float2 a = ring[((s - WK_RK + (R_)) % WK_LC + WK_LC) % WK_LC];                        \
        const float2 bb = ring[((s - WK_RK - (R_) - 1) % WK_LC + WK_LC) % WK_LC];                   \
        acc = __ffma2_rn((W_), __ffma2_rn(bb, make_float2(-1.f, -1.f), a), acc);                    \
    }
            float2 acc = make_float2(0.f, 0.f);
            WK_TAP(WK_R0, w0)
#if WK_K > 1
            WK_TAP(WK_R1, w1)
#endif
#if WK_K > 2
            WK_TAP(WK_R2, w2)
#endif
#if WK_K > 3
            WK_TAP(WK_R3, w3)
#endif
#if WK_K > 4
            WK_TAP(WK_R4, w4)
#endif
#undef WK_TAP
            const float y = __fadd_rn(acc.x, acc.y);
            if (FIRST) {
                const int r = s - 2 * WK_RK;   // 0 or 1
                if (on && r < rows_left) *reinterpret_cast<float*>(ofirst + (long long)r * p.out_pitch) = y;
            } else {
                cb[s * WK_RP] = y;
            }
        }
    }
}

extern "C" __global__ void __launch_bounds__(WK_TW, 3) walker_kernel(const __grid_constant__ WalkMap omap,
                                                                      const WalkParams p) {
    extern __shared__ __align__(128) float band[];   // WK_P / WK_LC chunks of WK_CS floats
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * WK_TW;
#if WK_Z
    const int zs = (int)blockIdx.z;                   // slice
    const unsigned char* const in_base = p.in + (long long)zs * p.in_z;
    unsigned char* const out_base = p.out + (long long)zs * p.out_z;
#else
    const unsigned char* const in_base = p.in;
    unsigned char* const out_base = p.out;
#endif
    const int xs = x0 - WK_RK - 1;          // image column of walk step 0
    // byte offset (from the row start) of the first 16-byte chunk the walk reads
    const long long cbyte = (long long)xs * WK_EB - WK_SHB;
    const bool interior = p.aligned && cbyte >= 0 && cbyte + 16LL * WK_NCH <= (long long)p.W * WK_EB;
    const int nch = p.nch;
    const int y0 = ((int)blockIdx.y + p.ty0) * p.th;
    // bit c: the walk's chunk c lies inside the row (aligned input), so it is
    // loaded straight from global memory; the others come from the folded copy
    unsigned int inmask = 0u;
#pragma unroll
    for (int c = 0; c < WK_NCH; ++c) {
        const long long cb = cbyte + 16LL * c;
        if (p.aligned && cb >= 0 && cb + 16 <= (long long)p.W * WK_EB) inmask |= 1u << c;
    }
    // output tiles by TMA: a whole strip inside the image and a valid map
    const bool tma_cta = p.tma_out && x0 + WK_TW <= p.W;
    // Edge strips of aligned images fold their pixels past the row from a
    // window of the row's first (left strip) or last bytes, copied to shared
    // memory by cp.async while the previous band's column phase runs, so the
    // folded copy waits on no global load.
    const bool use_win = WK_WIN > 0 && !interior && p.aligned && (long long)p.W * WK_EB >= WK_WIN;
    const long long wbase = cbyte < 0 ? 0 : ((long long)p.W * WK_EB - WK_WIN) / 16 * 16;
    unsigned char* const wrow = reinterpret_cast<unsigned char*>(band) + WK_WIN_OFF + t * WK_WIN;
    // The fold is the same for every row, so it is tabulated once per CTA:
    // for word w of the k-th walk chunk outside the row (at most four), the
    // two window words its bytes come from (index 63: a zero word) and the
    // byte-permute selector that assembles it.  A pixel whose source lies
    // outside the window (tiny images, repeated reflections) sends the CTA to
    // the pixel-by-pixel copy.
    __shared__ unsigned int wk_tab[16];
    __shared__ int wk_tab_ok;
    bool tab = false;
    if (use_win) {   // uniform over the CTA
        const unsigned int outmask = ~inmask & (WK_NCH >= 32 ? 0xffffffffu : ((1u << WK_NCH) - 1u));
        const int n_out = __popc(outmask);
        if (t == 0) wk_tab_ok = n_out <= 4;
        __syncthreads();
        if (t < 4 * n_out && t < 16) {
            int c = 0;
            for (int k = 0, seen = 0; k < WK_NCH; ++k)
                if ((outmask >> k) & 1u) {
                    if (seen == t / 4) c = k;
                    ++seen;
                }
            unsigned int a = 64, b = 64, sel = 0;
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int pos = c * 16 + 4 * (t % 4) + k;   // byte of the walk's chunk stream
                const int x = xs - WK_SHB / WK_EB + pos / WK_EB;
                const int xf = wk_fold(x, p.W, p.boundary);
                unsigned int word = 63, byte = 0;
                if (xf >= 0) {
                    const long long o = (long long)xf * WK_EB + pos % WK_EB - wbase;
                    if (o < 0 || o >= WK_WIN) ok = false;
                    word = (unsigned int)(o >> 2) & 63u;
                    byte = (unsigned int)(o & 3);
                }
                if (a == 64 || a == word) {
                    a = word;
                    sel |= byte << (4 * k);
                } else if (b == 64 || b == word) {
                    b = word;
                    sel |= (4u + byte) << (4 * k);
                } else {
                    ok = false;
                }
            }
            if (b == 64) b = a;
            wk_tab[t] = a | (b << 6) | (sel << 16);
            if (!ok) wk_tab_ok = 0;
        }
        __syncthreads();
        tab = wk_tab_ok != 0;
    }

    // column state: the running sums J = (Jh, Jl) of the last WK_LC rows; row
    // u of the tile sits at ring[u % WK_LC] (WK_P is a multiple of WK_LC), and
    // J(-1) = 0 at ring[WK_LC - 1]
    float2 ring[WK_LC];
#pragma unroll
    for (int i = 0; i < WK_LC; ++i) ring[i] = make_float2(0.f, 0.f);
    const int xc = x0 + t;
    const bool col_on = xc < p.W;
    unsigned char* const ocol = out_base + (long long)xc * 4;

    constexpr int CPB = WK_P / WK_LC;   // row chunks per band
    const int nbands = (nch + CPB - 1) / CPB;
    // Source row of this thread in band bb (null: a row of zeros, or no row).
    // Interior strips fetch the first two 16-byte chunks of the next band's
    // row into registers while the current band's column phase runs, and
    // prefetch the rest of it to L2, so that a walk does not start on a cold
    // load (two chunks: a third would no longer fit the register budget).
    auto row_of = [&](int bb) -> const unsigned char* {
        if (t >= min(CPB, nch - bb * CPB) * WK_LC) return nullptr;
        const int v = y0 - WK_RK + bb * WK_P + t;   // virtual image row
        if (v < -WK_RK || v > p.H - 1 + WK_RK) return nullptr;
        const int src = wk_fold(v, p.H, p.boundary);
        return src >= 0 ? in_base + (long long)src * p.in_pitch : nullptr;
    };
    uint4 pre[2];
    auto fetch_first = [&](const unsigned char* row) {
        if (!interior || row == nullptr) return;
        const uint4* g = reinterpret_cast<const uint4*>(row + cbyte);
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (c < WK_NCH) pre[c] = __ldg(g + c);
#pragma unroll
        for (int off = 32; off < 16 * WK_NCH; off += 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row + cbyte + off));
    };
    auto fetch_win = [&](const unsigned char* row) {
        if (!use_win || row == nullptr) return;
#pragma unroll
        for (int k = 0; k < WK_WIN / 16; ++k)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(wk_smem(wrow + 16 * k)),
                         "l"(row + wbase + 16 * k)
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const unsigned char* nrow = row_of(0);
    fetch_first(nrow);
    fetch_win(nrow);
    for (int b = 0; b < nbands; ++b) {
        const int nchb = min(CPB, nch - b * CPB);   // chunks in this band (the last may be short)
        const unsigned char* const row = nrow;        // this thread's source row in band b
        if (b > 0) {
            // every column of the previous band is done and its tile stores
            // have read the band
            if (tma_cta && t == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            __syncthreads();
        }
        // ------------------------------------------------ row phase
        if (t < nchb * WK_LC) {
            float* rrow = band + (t / WK_LC) * WK_CS + (t % WK_LC) * WK_RP;
            if (row == nullptr) {
#pragma unroll
                for (int o = 0; o < WK_TW; o += 4) *reinterpret_cast<float4*>(rrow + o) = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const uint4* gch = reinterpret_cast<const uint4*>(row + cbyte);
                uint4* sch = reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(rrow) + WK_STAGE_OFF);
                if (!interior) {
                    if (use_win) asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's window
                    // edge strips and unaligned input: the walk's chunks that
                    // are not inside the row (or all, unaligned) copied to the
                    // tail of this row's band slot (the row's outputs overwrite
                    // it only after the walk has read it), folded by the
                    // boundary rule: from the window by the table, else pixel
                    // by pixel
                    if (tab) {
                        const unsigned int* ww = reinterpret_cast<const unsigned int*>(wrow);
#pragma unroll 1
                        for (int c = 0, k = 0; c < WK_NCH; ++c) {
                            if ((inmask >> c) & 1u) continue;
                            unsigned int wd[4];
#pragma unroll
                            for (int w = 0; w < 4; ++w) {
                                const unsigned int e = wk_tab[4 * k + w];
                                const unsigned int ia = e & 63u, ib = (e >> 6) & 63u;
                                wd[w] = __byte_perm(ia == 63u ? 0u : ww[ia], ib == 63u ? 0u : ww[ib], e >> 16);
                            }
                            sch[c] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                            ++k;
                        }
                    }
#pragma unroll 1
                    for (int c = 0; c < WK_NCH && !tab; ++c) {
                        if ((inmask >> c) & 1u) continue;
                        // all loads of the chunk first (independent), then one 16-byte store
                        constexpr int PER = 16 / WK_EB;
                        unsigned int px[PER];
#pragma unroll
                        for (int i = 0; i < PER; ++i) {
                            const int x = xs - WK_SHB / WK_EB + c * PER + i;
                            const int xf = wk_fold(x, p.W, p.boundary);
                            const long long wo = (long long)xf * WK_EB - wbase;   // byte offset in the window
                            const bool inw = use_win && wo >= 0 && wo + WK_EB <= WK_WIN;
#if WK_IN == 0
                            px[i] = xf < 0 ? 0u : inw ? (unsigned int)wrow[wo] : (unsigned int)__ldg(row + xf);
#else
                            px[i] = xf < 0 ? 0u
                                    : inw ? (unsigned int)*reinterpret_cast<const unsigned short*>(wrow + wo)
                                          : (unsigned int)__ldg(reinterpret_cast<const unsigned short*>(row) + xf);
#endif
                        }
                        unsigned int wd[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
#if WK_IN == 0
                            wd[k] = px[4 * k] | (px[4 * k + 1] << 8) | (px[4 * k + 2] << 16) | (px[4 * k + 3] << 24);
#else
                            wd[k] = px[2 * k] | (px[2 * k + 1] << 16);
#endif
                        }
                        sch[c] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                    }
                }
                // the walk: S[j] holds the sum of the pixels at steps 0..j (for
                // 8-bit input as 2^23 + that sum); outputs o - 1 and o (o odd)
                // are formed at step o + 2 rk + 1 from S[. + rk + 1 + r_i] and
                // S[. + rk - r_i], whose difference is exact
                const float2 w0 = make_float2(p.w[0], p.w[0]);
#if WK_K > 1
                const float2 w1 = make_float2(p.w[1], p.w[1]);
#endif
#if WK_K > 2
                const float2 w2 = make_float2(p.w[2], p.w[2]);
#endif
#if WK_K > 3
                const float2 w3 = make_float2(p.w[3], p.w[3]);
#endif
#if WK_K > 4
                const float2 w4 = make_float2(p.w[4], p.w[4]);
#endif
                float S[WK_STEPS];
                uint4 ch[WK_NCH];
#pragma unroll
                for (int c = 0; c < WK_NCH && c < 3; ++c)
                    ch[c] = interior ? (c < 2 ? pre[c] : __ldg(gch + c)) : ((inmask >> c) & 1u) ? __ldg(gch + c) : sch[c];
#if WK_IN == 0
                unsigned int sb = 0x4B000000u;   // bits of 2^23
#else
                float s = 0.f;
#endif
                float2 prev = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < WK_STEPS; ++j) {
                    const int pos = WK_SHB + j * WK_EB;      // byte position in the chunk stream
                    const int c = pos >> 4;
                    // entering chunk c >= 1: fetch chunk c + 2 (chunks 0..2 are fetched up front)
                    if ((pos & 15) == 0 && c >= 1 && c + 2 < WK_NCH)
                        ch[c + 2] = ((inmask >> (c + 2)) & 1u) ? __ldg(gch + c + 2) : sch[c + 2];
                    const int wi = (pos & 15) >> 2;
                    const unsigned int word = wi == 0 ? ch[c].x : wi == 1 ? ch[c].y : wi == 2 ? ch[c].z : ch[c].w;
#if WK_IN == 0
                    sb += wk_elem(word, pos & 3);
                    S[j] = __uint_as_float(sb);
#else
                    s = __fadd_rn(s, __fsub_rn(__uint_as_float(wk_elem(word, (pos & 3) / 2)), 8388608.f));
                    S[j] = s;
#endif
                    if (j >= 2 * WK_RK + 1 && ((j - (2 * WK_RK + 1)) & 1)) {
                        const int o = j - (2 * WK_RK + 1);
                        const int ap = o + WK_RK, am = o + WK_RK - 1;   // output o - 1: S[ap + r_i] - S[am - r_i]
#define WK_RTAP(R_) make_float2(__fsub_rn(S[ap + (R_)], S[am - (R_)]), __fsub_rn(S[ap + 1 + (R_)], S[am + 1 - (R_)]))
                        float2 r2 = __fmul2_rn(w0, WK_RTAP(WK_R0));
#if WK_K > 1
                        r2 = __ffma2_rn(w1, WK_RTAP(WK_R1), r2);
#endif
#if WK_K > 2
                        r2 = __ffma2_rn(w2, WK_RTAP(WK_R2), r2);
#endif
#if WK_K > 3
                        r2 = __ffma2_rn(w3, WK_RTAP(WK_R3), r2);
#endif
#if WK_K > 4
                        r2 = __ffma2_rn(w4, WK_RTAP(WK_R4), r2);
#endif
#undef WK_RTAP
                        if ((o & 3) == 1) {
                            prev = r2;
                        } else {
                            *reinterpret_cast<float4*>(rrow + o - 3) = make_float4(prev.x, prev.y, r2.x, r2.y);
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (b + 1 < nbands) {
            nrow = row_of(b + 1);
            fetch_first(nrow);
            fetch_win(nrow);
        }
        // ------------------------------------------------ column phase
#pragma unroll 1
        for (int it = 0; it < nchb; ++it) {
            const int k = b * CPB + it;                      // chunk of the tile
            float* cb = band + it * WK_CS + t;
            const int ychunk = y0 + k * WK_LC - 2 * WK_RK;   // output row of the chunk's row 0
            if (k == 0) {
                wk_chunk<true>(ring, cb, p, ocol + (long long)y0 * p.out_pitch, p.H - y0, col_on);
            } else {
                wk_chunk<false>(ring, cb, p, nullptr, 0, false);
                if (!tma_cta && col_on) {
                    // partial strip or unaligned output: this thread's column, row by row
                    const int nr = min(WK_LC, p.H - ychunk);
                    unsigned char* o = ocol + (long long)ychunk * p.out_pitch;
#pragma unroll 1
                    for (int r = 0; r < nr; ++r) *reinterpret_cast<float*>(o + (long long)r * p.out_pitch) = cb[r * WK_RP];
                }
            }
            // every WK_G chunks (at least 32 rows) the finished tiles leave by
            // TMA while the next chunks are computed
            if (tma_cta && ((it + 1) % WK_G == 0 || it + 1 == nchb)) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // tiles visible to the TMA unit
                __syncthreads();
                if (t == 0) {
                    for (int g = it + 1 - ((it % WK_G) + 1); g <= it; ++g) {
                        const int kg = b * CPB + g;
                        const int yg = y0 + kg * WK_LC - 2 * WK_RK;
                        if (kg == 0 || yg >= p.H) continue;
#if WK_Z
                        asm volatile(
                            "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];"
                            ::"l"(&omap), "r"(wk_smem(band + g * WK_CS)), "r"(0), "r"((int)blockIdx.x), "r"(yg),
                            "r"(zs)
                            : "memory");
#else
                        asm volatile(
                            "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];"
                            ::"l"(&omap), "r"(wk_smem(band + g * WK_CS)), "r"(0), "r"((int)blockIdx.x), "r"(yg)
                            : "memory");
#endif
                    }
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
            }
        }
    }
    if (tma_cta && t == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

#endif  // WK_TW
