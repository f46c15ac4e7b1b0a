// Host-side kernel fit: Sec. 4.1-4.2 (quadratic-form error, exhaustive search
// at sigma0 = 100/pi) and Eq. scale1 / Eq. scale2 (rescaling to any sigma);
// the same search for any symmetric kernel given by its samples (Sec. 3.2).
//
// The search walks the tree of increasing radius tuples depth first and grows
// a Cholesky factor of the K x K Gram matrix one row per level, so each leaf
// costs one short forward substitution instead of a fresh K x K solve.  The
// residual quadratic-form error of a tuple is g^T A g - |L^{-1} h|^2.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>
#include <thread>
#include <vector>

namespace gb {
namespace {

constexpr int kSamples = 200;   // t = -100 .. 99 (integer positions, t = 0 once)
constexpr int kFirstT = -100;
constexpr int kRadii = 100;     // candidate inclusive radii 0 .. 99
constexpr double kPi = 3.14159265358979323846;

struct Problem {
    // Gram matrix of the box indicators under A, right-hand side and g^T A g.
    std::vector<double> M;      // kRadii x kRadii
    std::vector<double> h;      // kRadii
    double gAg = 0.0;
};

// Autocorrelation of the natural-image prior: the inverse DFT (period 200) of
// the folded power spectrum 1/u^2, with 16.5 at u = 0 (Sec. 4.1), evaluated as
// an explicit cosine sum.
std::vector<double> prior_autocorrelation() {
    std::vector<double> spec(kSamples), phi(kSamples);
    spec[0] = 16.5;
    for (int u = 1; u < kSamples; ++u) {
        const int f = std::min(u, kSamples - u);
        spec[u] = 1.0 / (double(f) * double(f));
    }
    for (int d = 0; d < kSamples; ++d) {
        double s = 0.0;
        for (int u = 0; u < kSamples; ++u) s += spec[u] * std::cos(2.0 * kPi * double(u) * d / kSamples);
        phi[d] = s / kSamples;
    }
    return phi;
}

// The sampled Gaussian at sigma0 = 100/pi on t = -100..99.
std::vector<double> gaussian_sigma0() {
    const double sigma0 = 100.0 / kPi;
    std::vector<double> g(kSamples);
    for (int j = 0; j < kSamples; ++j) {
        const double t = double(kFirstT + j);
        g[j] = std::exp(-t * t / (2.0 * sigma0 * sigma0));
    }
    return g;
}

// Gram quantities of the search for the kernel samples g (t = -100..99).
Problem build_problem(int err_kind, const std::vector<double>& g) {
    // a(j, k) = Phi[(j - k) mod 200] (Eq. mahal with A_jk = Phi_{j-k}) or identity.
    std::vector<double> phi;
    if (err_kind == GF_ERR_QF) phi = prior_autocorrelation();
    auto a = [&](int j, int k) -> double {
        if (err_kind == GF_ERR_L2) return j == k ? 1.0 : 0.0;
        return phi[((j - k) % kSamples + kSamples) % kSamples];
    };
    // Sample index of position t, and the box of radius q = samples with |t| <= q.
    auto idx = [](int t) { return t - kFirstT; };
    // col[q][j] = sum over the box of radius q of a(j, k): grown one ring at a time.
    std::vector<double> col((size_t)kRadii * kSamples, 0.0);
    for (int q = 0; q < kRadii; ++q) {
        double* c = &col[(size_t)q * kSamples];
        if (q > 0) std::memcpy(c, &col[(size_t)(q - 1) * kSamples], sizeof(double) * kSamples);
        for (int j = 0; j < kSamples; ++j) {
            double add = a(j, idx(q));
            if (q > 0) add += a(j, idx(-q));
            c[j] += add;
        }
    }
    Problem P;
    P.M.assign((size_t)kRadii * kRadii, 0.0);
    P.h.assign(kRadii, 0.0);
    // Ag = A g
    std::vector<double> Ag(kSamples, 0.0);
    for (int j = 0; j < kSamples; ++j) {
        double s = 0.0;
        for (int k = 0; k < kSamples; ++k) s += a(j, k) * g[k];
        Ag[j] = s;
    }
    for (int j = 0; j < kSamples; ++j) P.gAg += g[j] * Ag[j];
    for (int q2 = 0; q2 < kRadii; ++q2) {
        const double* c = &col[(size_t)q2 * kSamples];
        double run = 0.0;
        for (int q1 = 0; q1 < kRadii; ++q1) {
            run += c[idx(q1)];
            if (q1 > 0) run += c[idx(-q1)];
            P.M[(size_t)q1 * kRadii + q2] = run;
        }
    }
    double run = 0.0;
    for (int q = 0; q < kRadii; ++q) {
        run += Ag[idx(q)];
        if (q > 0) run += Ag[idx(-q)];
        P.h[q] = run;
    }
    return P;
}

struct Best {
    double err = std::numeric_limits<double>::infinity();
    int q[GF_KMAX] = {0, 0, 0, 0, 0};
};

bool better(double e, const int* q, const Best& b, int K) {
    if (e < b.err) return true;
    if (e > b.err) return false;
    return std::lexicographical_compare(q, q + K, b.q, b.q + K);
}

// Depth-first walk under a fixed first radius.  L holds the Cholesky rows of the
// current prefix, z = L^{-1} h_prefix, and zz = |z|^2.
struct Walker {
    const Problem* P;
    int K;
    double L[GF_KMAX][GF_KMAX];
    double z[GF_KMAX];
    int q[GF_KMAX];
    Best best;

    // Appends radius qn at level `lev` (0-based); returns false if numerically singular.
    bool push(int lev, int qn, double* zz_out, double zz_in) {
        if (lev < 0 || lev >= GF_KMAX) return false;
        const double* M = P->M.data();
        double s2 = 0.0, dot = 0.0;
        for (int j = 0; j < lev; ++j) {
            double v = M[(size_t)qn * kRadii + q[j]];
            for (int m = 0; m < j; ++m) v -= L[j][m] * L[lev][m];
            v /= L[j][j];
            L[lev][j] = v;
            s2 += v * v;
            dot += v * z[j];
        }
        const double d2 = M[(size_t)qn * kRadii + qn] - s2;
        if (!(d2 > 0.0)) return false;
        const double d = std::sqrt(d2);
        L[lev][lev] = d;
        z[lev] = (P->h[qn] - dot) / d;
        q[lev] = qn;
        *zz_out = zz_in + z[lev] * z[lev];
        return true;
    }

    void leaves(int lev, double zz) {
        // last level: error = gAg - zz - z_K^2 for every admissible radius
        if (lev < 1 || lev >= GF_KMAX) return;
        const double* M = P->M.data();
        for (int qn = q[lev - 1] + 1; qn < kRadii; ++qn) {
            double l[GF_KMAX];
            double s2 = 0.0, dot = 0.0;
            for (int j = 0; j < lev; ++j) {
                double v = M[(size_t)qn * kRadii + q[j]];
                for (int m = 0; m < j; ++m) v -= L[j][m] * l[m];
                v /= L[j][j];
                l[j] = v;
                s2 += v * v;
                dot += v * z[j];
            }
            const double d2 = M[(size_t)qn * kRadii + qn] - s2;
            if (!(d2 > 0.0)) continue;
            const double num = P->h[qn] - dot;
            const double e = P->gAg - zz - num * num / d2;
            q[lev] = qn;
            if (better(e, q, best, K)) {
                best.err = e;
                std::memcpy(best.q, q, sizeof(int) * K);
            }
        }
    }

    void descend(int lev, double zz) {
        if (lev == K - 1) { leaves(lev, zz); return; }
        const int remaining = K - lev;   // radii still to place, including this level
        for (int qn = q[lev - 1] + 1; qn <= kRadii - remaining; ++qn) {
            double zz2;
            if (!push(lev, qn, &zz2, zz)) continue;
            descend(lev + 1, zz2);
        }
    }
};

// Weights of the chosen tuple: solve the K x K normal equations by Cholesky.
void solve_weights(const Problem& P, const int* q, int K, double* w) {
    double L[GF_KMAX][GF_KMAX] = {};
    double z[GF_KMAX];
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j <= i; ++j) {
            double v = P.M[(size_t)q[i] * kRadii + q[j]];
            for (int m = 0; m < j; ++m) v -= L[i][m] * L[j][m];
            if (i == j) L[i][i] = std::sqrt(v);
            else L[i][j] = v / L[j][j];
        }
    }
    for (int i = 0; i < K; ++i) {
        double v = P.h[q[i]];
        for (int m = 0; m < i; ++m) v -= L[i][m] * z[m];
        z[i] = v / L[i][i];
    }
    for (int i = K - 1; i >= 0; --i) {
        double v = z[i];
        for (int m = i + 1; m < K; ++m) v -= L[m][i] * w[m];
        w[i] = v / L[i][i];
    }
}

struct Sigma0Fit {
    int K = 0;
    int p[GF_KMAX];
    double w[GF_KMAX];
    double c[GF_KMAX];
    double err;
};

Sigma0Fit run_search(int K, const Problem& P) {
    const int n_first = kRadii - K + 1;
    unsigned hw = std::thread::hardware_concurrency();
    const int nthreads = (int)std::max(1u, std::min(hw ? hw : 4u, 64u));
    std::vector<Best> bests(nthreads);
    std::mutex mu;
    int next_first = 0;
    auto work = [&](int tid) {
        Walker W;
        W.P = &P;
        W.K = K;
        for (;;) {
            int f;
            {
                std::lock_guard<std::mutex> lk(mu);
                f = next_first++;
            }
            if (f >= n_first) break;
            double zz;
            if (!W.push(0, f, &zz, 0.0)) continue;
            if (K == 1) {
                const double e = P.gAg - zz;
                if (better(e, W.q, W.best, K)) { W.best.err = e; W.best.q[0] = f; }
                continue;
            }
            W.descend(1, zz);
        }
        bests[tid] = W.best;
    };
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
    for (auto& t : th) t.join();
    Best b;
    for (auto& x : bests)
        if (better(x.err, x.q, b, K)) b = x;
    Sigma0Fit F;
    F.K = K;
    F.err = b.err;
    std::memcpy(F.p, b.q, sizeof(int) * K);
    solve_weights(P, F.p, K, F.w);
    double acc = 0.0;
    for (int i = K - 1; i >= 0; --i) { acc += F.w[i]; F.c[i] = acc; }
    return F;
}

std::mutex g_fit_mu;
Sigma0Fit g_fits[2][GF_KMAX + 1];
bool g_have[2][GF_KMAX + 1] = {};

const Sigma0Fit& sigma0_fit(int K, int err_kind) {
    std::lock_guard<std::mutex> lk(g_fit_mu);
    if (!g_have[err_kind][K]) {
        g_fits[err_kind][K] = run_search(K, build_problem(err_kind, gaussian_sigma0()));
        g_have[err_kind][K] = true;
    }
    return g_fits[err_kind][K];
}

}  // namespace

gf_status fit_sigma0(int K, int err_kind, int32_t* p, double* c, double* w, double* err) {
    if (K < 1 || K > GF_KMAX) return GF_EUNSUPPORTED;
    if (err_kind != GF_ERR_QF && err_kind != GF_ERR_L2) return GF_EINVAL;
    const Sigma0Fit& F = sigma0_fit(K, err_kind);
    for (int i = 0; i < K; ++i) {
        if (p) p[i] = F.p[i];
        if (c) c[i] = F.c[i];
        if (w) w[i] = F.w[i];
    }
    if (err) *err = F.err;
    return GF_OK;
}

gf_status fit_kernel(const double* half, int n, int K, int err_kind, int32_t* radii, double* weights, double* err) {
    if (!half || n < 1 || n > kRadii + 1) return GF_EINVAL;
    if (K < 1 || K > GF_KMAX) return GF_EUNSUPPORTED;
    if (err_kind != GF_ERR_QF && err_kind != GF_ERR_L2) return GF_EINVAL;
    if (!radii || !weights) return GF_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(half[i])) return GF_EINVAL;
    // the symmetric kernel on the search grid: g(t) = half[|t|], 0 beyond
    std::vector<double> g(kSamples, 0.0);
    for (int j = 0; j < kSamples; ++j) {
        const int a = std::abs(kFirstT + j);
        if (a < n) g[j] = half[a];
    }
    const Sigma0Fit F = run_search(K, build_problem(err_kind, g));
    if (!std::isfinite(F.err)) return GF_EINVAL;
    for (int i = 0; i < K; ++i) {
        radii[i] = F.p[i];
        weights[i] = F.w[i];
    }
    if (err) *err = F.err;
    return GF_OK;
}

gf_status fit_boxes(double sigma, int K, int err_kind, int32_t* radii, double* weights) {
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return GF_EINVAL;
    if (K < 1 || K > GF_KMAX) return GF_EUNSUPPORTED;
    if (err_kind != GF_ERR_QF && err_kind != GF_ERR_L2) return GF_EINVAL;
    if (!radii || !weights) return GF_EINVAL;
    const Sigma0Fit& F = sigma0_fit(K, err_kind);
    double mass = 0.0;
    double ws[GF_KMAX];
    int32_t rs[GF_KMAX];
    for (int i = 0; i < K; ++i) {
        // Eq. scale1: floor((sigma / sigma0) p_i), with sigma0 = 100/pi
        const double scaled = sigma * kPi * double(F.p[i]) / 100.0;
        if (scaled > 1.0e6) return GF_EUNSUPPORTED;
        rs[i] = (int32_t)std::floor(scaled);
        // Eq. scale2: p_i / (2 r_i + 1) * w_i
        ws[i] = double(F.p[i]) / (2.0 * rs[i] + 1.0) * F.w[i];
        mass += ws[i] * (2.0 * rs[i] + 1.0);
    }
    for (int i = 0; i < K; ++i) {
        radii[i] = rs[i];
        weights[i] = ws[i] / mass;
    }
    return GF_OK;
}

}  // namespace gb
