/*
 * Oracle: the filter's result definition on all host cores, and the paper's
 * running-sum method on the CPU for timing context.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; it is compiled into oracle/_build/ and used by the tests
 * and by bench.py's CPU baseline and reference arm.
 *
 * oracle_conv_separable: the separable convolution with the staircase kernel
 *     k(t) = sum over i with |t| <= r_i of w_i          (Sec. 3.2, Eq. ciwi)
 * written out as two direct FP64 1D convolutions, rows then columns (Sec. 3.4),
 * pixels outside the image supplied by the boundary rule (0 replicate, 1 zero,
 * 2 reflect without repeating the edge pixel, folded as often as needed).  It
 * computes exactly what oracle/filter.py's filter_separable computes (the
 * same definition, in C for speed), row blocks spread over OpenMP threads.
 *
 * oracle_boxsum_u8_f32: the paper's method for an 8-bit image (Sec. 3.3-3.4):
 * an integer running sum of each row (Eq. alg1), the K weighted box
 * differences per pixel (Eq. indep) in FP32, then the same down the columns
 * with FP32 running sums of the row results.  Its numbers are context for the
 * timing (what the method costs on this CPU); it is not a reference for the
 * GPU results.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int fold(int t, int n, int boundary) {
    if (t >= 0 && t < n) return t;
    if (boundary == 1) return -1;
    if (boundary == 0) return t < 0 ? 0 : n - 1;
    if (n == 1) return 0;
    int period = 2 * (n - 1);
    int m = t % period;
    if (m < 0) m += period;
    return m < n ? m : period - m;
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* k[0 .. 2 rk] = k(-rk .. rk) */
static void staircase(const int* radii, const double* w, int K, int rk, double* k) {
    for (int t = -rk; t <= rk; ++t) {
        double v = 0.0;
        for (int i = 0; i < K; ++i)
            if ((t < 0 ? -t : t) <= radii[i]) v += w[i];
        k[t + rk] = v;
    }
}

/*
 * in, out: H x W x C doubles (row-major, interleaved channels); out may not
 * alias in.  Returns 0, or -1 if memory for the intermediate is unavailable.
 */
int oracle_conv_separable(const double* in, int H, int W, int C, const int* radii, const double* weights, int K,
                          int boundary, double* out) {
    int rk = 0;
    for (int i = 0; i < K; ++i) rk = radii[i] > rk ? radii[i] : rk;
    double* k = (double*)malloc(sizeof(double) * (2 * rk + 1));
    double* tmp = (double*)malloc(sizeof(double) * (size_t)H * W * C);
    if (!k || !tmp) {
        free(k);
        free(tmp);
        return -1;
    }
    staircase(radii, weights, K, rk, k);
    const size_t row = (size_t)W * C;
    /* rows: R(y, x) = sum_t k(t) f(y, fold(x + t)) */
#pragma omp parallel
    {
        double* ext = (double*)malloc(sizeof(double) * (W + 2 * rk) * C);
#pragma omp for schedule(static)
        for (int y = 0; y < H; ++y) {
            const double* src = in + (size_t)y * row;
            for (int t = -rk; t < W + rk; ++t) {
                const int xs = fold(t, W, boundary);
                for (int c = 0; c < C; ++c) ext[(size_t)(t + rk) * C + c] = xs >= 0 ? src[(size_t)xs * C + c] : 0.0;
            }
            double* dst = tmp + (size_t)y * row;
            for (size_t e = 0; e < row; ++e) dst[e] = 0.0;
            for (int t = 0; t <= 2 * rk; ++t) {
                const double kv = k[t];
                if (kv == 0.0) continue;
                const double* e0 = ext + (size_t)t * C;
                for (size_t e = 0; e < row; ++e) dst[e] += kv * e0[e];
            }
        }
        free(ext);
    }
    /* columns: Y(y, x) = sum_s k(s) R(fold(y + s), x) */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        double* dst = out + (size_t)y * row;
        for (size_t e = 0; e < row; ++e) dst[e] = 0.0;
        for (int s = -rk; s <= rk; ++s) {
            const double kv = k[s + rk];
            const int ys = fold(y + s, H, boundary);
            if (kv == 0.0 || ys < 0) continue;
            const double* src = tmp + (size_t)ys * row;
            for (size_t e = 0; e < row; ++e) dst[e] += kv * src[e];
        }
    }
    free(k);
    free(tmp);
    return 0;
}

/*
 * The running-sum method on an 8-bit single-channel image: in H x W bytes
 * (pitch in_pitch), out H x W floats.  Rows: int32 running sums of the
 * boundary-extended row, out(x) = sum_i w_i (I(x + r_i) - I(x - r_i - 1)).
 * Columns: FP32 running sums of the row results, kept for the last 2 rk + 2
 * rows, and the same differences.  Row bands of the image are spread over
 * OpenMP threads (each band recomputes rk rows above and below).
 */
int oracle_boxsum_u8_f32(const uint8_t* in, long long in_pitch, int H, int W, const int* radii,
                         const float* weights, int K, int boundary, float* out) {
    int rk = 0;
    for (int i = 0; i < K; ++i) rk = radii[i] > rk ? radii[i] : rk;
    const int L = 2 * rk + 2;
    int nthreads = oracle_threads();
    int band = (H + nthreads - 1) / nthreads;
    if (band < 1) band = 1;
    const int nbands = (H + band - 1) / band;
    int fail = 0;
#pragma omp parallel for schedule(static) reduction(| : fail)
    for (int b = 0; b < nbands; ++b) {
        const int y0 = b * band, y1 = y0 + band < H ? y0 + band : H;
        int32_t* I = (int32_t*)malloc(sizeof(int32_t) * (W + 2 * rk + 2));
        float* R = (float*)malloc(sizeof(float) * W);
        float* J = (float*)calloc((size_t)L * W, sizeof(float));   /* ring of column running sums */
        float* acc = (float*)calloc((size_t)W, sizeof(float));
        if (!I || !R || !J || !acc) {
            fail = 1;
        } else {
            /* rows v = y0 - rk .. y1 - 1 + rk; J(v) at ring slot (v - y0 + rk) mod L, J(y0 - rk - 1) = 0 */
            for (int v = y0 - rk; v <= y1 - 1 + rk; ++v) {
                const int ys = fold(v, H, boundary);
                const int u = v - (y0 - rk);
                if (ys < 0) {
                    for (int x = 0; x < W; ++x) R[x] = 0.f;
                } else {
                    const uint8_t* src = in + (long long)ys * in_pitch;
                    int32_t s = 0;
                    I[0] = 0;   /* I[j + 1] = sum of extended pixels -rk - 1 .. j - rk - 1 */
                    for (int j = 0; j < W + 2 * rk + 1; ++j) {
                        const int xs = fold(j - rk - 1, W, boundary);
                        s += xs >= 0 ? src[xs] : 0;
                        I[j + 1] = s;
                    }
                    for (int x = 0; x < W; ++x) {
                        float r = 0.f;
                        for (int i = 0; i < K; ++i)
                            r += weights[i] * (float)(I[x + rk + 1 + radii[i] + 1] - I[x + rk - radii[i] + 1]);
                        R[x] = r;
                    }
                }
                float* Jn = J + (size_t)(u % L) * W;
                const float* Jp = J + (size_t)((u + L - 1) % L) * W;
                if (u == 0) {
                    for (int x = 0; x < W; ++x) Jn[x] = R[x];
                } else {
                    for (int x = 0; x < W; ++x) Jn[x] = Jp[x] + R[x];
                }
                if (u >= 2 * rk) {
                    /* output row y = v - rk: sum_i w_i (J(u - rk + r_i) - J(u - rk - r_i - 1)) */
                    const int y = v - rk;
                    float* dst = out + (size_t)y * W;
                    for (int x = 0; x < W; ++x) acc[x] = 0.f;
                    for (int i = 0; i < K; ++i) {
                        const int ua = u - rk + radii[i], ub = u - rk - radii[i] - 1;
                        const float* Ja = J + (size_t)(ua % L) * W;
                        if (ub >= 0) {
                            const float* Jb = J + (size_t)(ub % L) * W;
                            for (int x = 0; x < W; ++x) acc[x] += weights[i] * (Ja[x] - Jb[x]);
                        } else {
                            for (int x = 0; x < W; ++x) acc[x] += weights[i] * Ja[x];
                        }
                    }
                    memcpy(dst, acc, sizeof(float) * W);
                }
            }
        }
        free(I);
        free(R);
        free(J);
        free(acc);
    }
    return fail ? -1 : 0;
}
