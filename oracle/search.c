/*
 * Oracle: exhaustive partition search of Sec. 4.2 (Gaussian approximation),
 * under the quadratic-form kernel error of Sec. 4.1 (Eq. mahal).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; it is compiled into oracle/_build/ and used by the tests,
 * by __graft_entry__.smoke() and by bench.py's CPU-baseline leg.
 *
 * What it computes.  The caller passes the Gram quantities of the problem
 *     M[q][q'] = s_q^T A s_q'     (n x n, row-major)
 *     h[q]     = s_q^T A g        (n)
 *     gAg      = g^T A g
 * where s_q is the indicator of the centred box of inclusive radius q and g the
 * sampled Gaussian.  For every increasing tuple q_1 < ... < q_K drawn from
 * 0..n-1 the optimal slice weights solve the K x K normal equations
 *     M_sub w = h_sub                                   (generalised least squares)
 * and the residual quadratic-form error is  E = gAg - h_sub^T w.
 * The tuple with the smallest E wins; among equal E the lexicographically
 * smallest tuple wins.  Each K x K system is solved by plain Gaussian
 * elimination with partial pivoting: no blocking, no reuse between tuples.
 */
#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KMAX 8

/* Solve a (k x k) system in place; returns 0 on success, -1 if singular. */
static int solve_dense(int k, double a[KMAX][KMAX], double b[KMAX], double x[KMAX]) {
    for (int col = 0; col < k; ++col) {
        int piv = col;
        double best = fabs(a[col][col]);
        for (int r = col + 1; r < k; ++r) {
            if (fabs(a[r][col]) > best) { best = fabs(a[r][col]); piv = r; }
        }
        if (best == 0.0) return -1;
        if (piv != col) {
            for (int c = 0; c < k; ++c) { double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t; }
            double t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int r = col + 1; r < k; ++r) {
            double f = a[r][col] / a[col][col];
            for (int c = col; c < k; ++c) a[r][c] -= f * a[col][c];
            b[r] -= f * b[col];
        }
    }
    for (int r = k - 1; r >= 0; --r) {
        double s = b[r];
        for (int c = r + 1; c < k; ++c) s -= a[r][c] * x[c];
        x[r] = s / a[r][r];
    }
    return 0;
}

/* Lexicographic comparison of two K-tuples. */
static int lex_less(const int* a, const int* b, int k) {
    for (int i = 0; i < k; ++i) {
        if (a[i] != b[i]) return a[i] < b[i];
    }
    return 0;
}

/* Evaluate one tuple; returns its error (or +inf if the system is singular). */
static double eval_tuple(const double* M, const double* h, double gAg, int n, int k,
                         const int* q, double* w_out) {
    double a[KMAX][KMAX], b[KMAX], bb[KMAX], x[KMAX];
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) a[i][j] = M[(size_t)q[i] * n + q[j]];
        b[i] = h[q[i]];
        bb[i] = b[i];
    }
    if (solve_dense(k, a, bb, x) != 0) return INFINITY;
    double e = gAg;
    for (int i = 0; i < k; ++i) e -= b[i] * x[i];
    if (w_out) for (int i = 0; i < k; ++i) w_out[i] = x[i];
    return e;
}

/*
 * Returns 0 on success, -1 on bad arguments.  Outputs: best_q[K] (radii),
 * best_w[K] (slice weights), *best_err.
 */
int oracle_partition_search(const double* M, const double* h, double gAg, int n, int k,
                            int* best_q, double* best_w, double* best_err) {
    if (k < 1 || k > KMAX || n < k) return -1;
    double g_err = INFINITY;
    int g_q[KMAX];
    for (int i = 0; i < k; ++i) g_q[i] = i;

    /* Split the enumeration by the first radius; each worker walks its slice in
       lexicographic order and keeps the first minimum it meets. */
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        double t_err = INFINITY;
        int t_q[KMAX];
        for (int i = 0; i < k; ++i) t_q[i] = i;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int first = 0; first <= n - k; ++first) {
            int q[KMAX];
            q[0] = first;
            for (int i = 1; i < k; ++i) q[i] = first + i;
            for (;;) {
                double e = eval_tuple(M, h, gAg, n, k, q, NULL);
                if (e < t_err) { t_err = e; memcpy(t_q, q, sizeof(int) * k); }
                /* next tuple with q[0] fixed: advance the last index that can move */
                int pos = k - 1;
                while (pos >= 1 && q[pos] == n - k + pos) --pos;
                if (pos < 1) break;
                ++q[pos];
                for (int i = pos + 1; i < k; ++i) q[i] = q[i - 1] + 1;
            }
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            if (t_err < g_err || (t_err == g_err && lex_less(t_q, g_q, k))) {
                g_err = t_err;
                memcpy(g_q, t_q, sizeof(int) * k);
            }
        }
    }
    memcpy(best_q, g_q, sizeof(int) * k);
    *best_err = eval_tuple(M, h, gAg, n, k, g_q, best_w);
    return 0;
}

/* Error and weights of one given tuple (used by tests to probe the landscape). */
int oracle_tuple_error(const double* M, const double* h, double gAg, int n, int k,
                       const int* q, double* w_out, double* err_out) {
    if (k < 1 || k > KMAX) return -1;
    for (int i = 0; i < k; ++i) if (q[i] < 0 || q[i] >= n || (i && q[i] <= q[i - 1])) return -1;
    *err_out = eval_tuple(M, h, gAg, n, k, q, w_out);
    return 0;
}
