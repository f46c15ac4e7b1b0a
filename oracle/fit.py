"""Oracle for the kernel fit (Sec. 4) and its per-sigma rescaling (Eq. scale1/scale2).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py; never by the product path.  Shares no code with
the library's own fitter.

Steps, in the paper's order:

1. Sample the standard Gaussian at sigma0 = 100/pi (Sec. 4.2).  Reading: integer
   positions t = -100..99 (200 samples, t = 0 once) of the peak-1 Gaussian
   exp(-t^2 / (2 sigma0^2)); the sign of the printed exponent is a typo.
2. Natural-image prior (Sec. 4.1): power spectrum 1/u^2, with the undefined
   u = 0 value set to 16.5 so that Phi_0 / Phi_r is close to 4/3.  Reading: a
   period-200 DFT with the folded spectrum S(u) = 1/min(u, 200-u)^2, Phi the
   inverse DFT of S, and A_jk = Phi[(j-k) mod 200] (Eq. mahal).
3. Exhaustive search over partitions (Sec. 4.2): every increasing tuple of
   inclusive radii q_1 < ... < q_K in 0..99; for each, the weights minimising
   the quadratic-form error (g - S w)^T A (g - S w) (closed-form generalised
   least squares).  Ties go to the lexicographically smallest tuple.  The
   search itself runs in oracle/search.c.
4. Segment constants c_i = sum_{j >= i} w_j (Eq. ciwi with w_i = c_i - c_{i+1}).
5. Rescaling to sigma: r_i = floor(sigma * pi * p_i / 100) (Eq. scale1) and
   w_i(sigma) = p_i / (2 r_i + 1) * w_i (Eq. scale2), then divided by
   sum_i w_i(sigma) (2 r_i + 1) so that a constant image is preserved.

The l2 variant (Sec. 5, "second set of parameters") replaces A by the identity.

fit_kernel runs steps 2-3 on any symmetric kernel given by its samples at
t = 0, 1, ... (Sec. 3.2, Sec. 4), returning the optimal unnormalised weights.
"""
import ctypes
import math

import numpy as np

from . import _native

N_SAMPLES = 200          # t = -100 .. 99
T_FIRST = -100
N_RADII = 100            # candidate inclusive radii 0 .. 99
SIGMA0 = 100.0 / math.pi
DC_VALUE = 16.5          # Sec. 4.1: the value given to the undefined u = 0 term


def sample_positions():
    return np.arange(T_FIRST, T_FIRST + N_SAMPLES, dtype=np.float64)


def gaussian_samples():
    """Peak-1 Gaussian at sigma0 = 100/pi on the sample grid (Sec. 4.2)."""
    t = sample_positions()
    return np.exp(-t * t / (2.0 * SIGMA0 * SIGMA0))


def prior_spectrum(dc=DC_VALUE, n=N_SAMPLES):
    """Folded 1/u^2 power spectrum of natural images (Sec. 4.1), S(0) = dc."""
    u = np.arange(n)
    s = np.empty(n, dtype=np.float64)
    fold = np.minimum(u[1:], n - u[1:]).astype(np.float64)
    s[1:] = 1.0 / (fold * fold)
    s[0] = dc
    return s


def prior_autocorrelation(dc=DC_VALUE, n=N_SAMPLES):
    """Phi: inverse Fourier transform of the prior spectrum (Sec. 4.1)."""
    return np.real(np.fft.ifft(prior_spectrum(dc, n)))


def error_matrix(err="qf", dc=DC_VALUE):
    """A of Eq. mahal: circulant Phi for 'qf', the identity for 'l2'."""
    if err == "l2":
        return np.eye(N_SAMPLES)
    if err != "qf":
        raise ValueError("err must be 'qf' or 'l2'")
    phi = prior_autocorrelation(dc)
    j = np.arange(N_SAMPLES)
    return phi[(j[:, None] - j[None, :]) % N_SAMPLES]


def box_indicators():
    """Column q is the indicator of the centred box |t| <= q (inclusive radius)."""
    t = sample_positions()
    q = np.arange(N_RADII)
    return (np.abs(t)[:, None] <= q[None, :]).astype(np.float64)


def gram(err="qf", dc=DC_VALUE, g=None):
    """M = S^T A S, h = S^T A g and g^T A g for the search (g: the sampled
    Gaussian at sigma0 unless given, on the same 200-sample grid)."""
    a = error_matrix(err, dc)
    s = box_indicators()
    g = gaussian_samples() if g is None else np.asarray(g, dtype=np.float64)
    m = s.T @ a @ s
    h = s.T @ (a @ g)
    gag = float(g @ (a @ g))
    return np.ascontiguousarray(m), np.ascontiguousarray(h), gag


def quadratic_form_error(radii, w, err="qf", dc=DC_VALUE):
    """Direct (g - S w)^T A (g - S w) for given inclusive radii and slice weights."""
    a = error_matrix(err, dc)
    t = sample_positions()
    approx = np.zeros(N_SAMPLES)
    for r, wi in zip(radii, w):
        approx += wi * (np.abs(t) <= r)
    d = gaussian_samples() - approx
    return float(d @ (a @ d))


def _search(m, h, gag, k):
    lib = _native.lib()
    n = m.shape[0]
    q = (ctypes.c_int * k)()
    w = (ctypes.c_double * k)()
    e = ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.oracle_partition_search(m.ctypes.data_as(dp), h.ctypes.data_as(dp), gag, n, k,
                                     q, w, ctypes.byref(e))
    if rc != 0:
        raise ValueError("bad search arguments")
    return np.array(list(q), dtype=np.int64), np.array(list(w)), e.value


def tuple_error(radii, err="qf", dc=DC_VALUE):
    """Closed-form GLS weights and error for one fixed tuple of radii."""
    m, h, gag = gram(err, dc)
    k = len(radii)
    lib = _native.lib()
    q = (ctypes.c_int * k)(*[int(r) for r in radii])
    w = (ctypes.c_double * k)()
    e = ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.oracle_tuple_error(m.ctypes.data_as(dp), h.ctypes.data_as(dp), gag, m.shape[0], k,
                                q, w, ctypes.byref(e))
    if rc != 0:
        raise ValueError("bad tuple")
    return np.array(list(w)), e.value


_cache = {}


def fit_sigma0(k, err="qf", dc=DC_VALUE):
    """Exhaustive search at sigma0.  Returns (p, c, w, error):
    p inclusive radii, c segment constants (Table 1), w slice weights."""
    key = (k, err, dc)
    if key not in _cache:
        m, h, gag = gram(err, dc)
        p, w, e = _search(m, h, gag, k)
        c = np.cumsum(w[::-1])[::-1].copy()
        _cache[key] = (p, c, w, e)
    p, c, w, e = _cache[key]
    return p.copy(), c.copy(), w.copy(), e


def slice_weights_from_constants(c):
    """w_i = c_i - c_{i+1}, c_{K+1} = 0 (Eq. ciwi; the printed c_i - c_{i-1} is a typo)."""
    c = np.asarray(c, dtype=np.float64)
    return c - np.append(c[1:], 0.0)


def scale_radii(p, sigma):
    """Eq. scale1: r_i = floor((sigma / sigma0) p_i), evaluated as sigma*pi*p/100."""
    return np.array([math.floor(sigma * math.pi * int(pi_) / 100.0) for pi_ in p], dtype=np.int64)


def scale_weights(p, w, r):
    """Eq. scale2 literally: w_i(sigma) = p_i / (2 r_i + 1) * w_i (unnormalised)."""
    p = np.asarray(p, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    return p / (2.0 * r + 1.0) * np.asarray(w, dtype=np.float64)


def fit_gaussian_boxes(sigma, k, err="qf"):
    """Radii and normalised slice weights for a given sigma (what gauss_fit_boxes returns)."""
    if not (sigma > 0 and math.isfinite(sigma)):
        raise ValueError("sigma must be positive and finite")
    p, _c, w, _e = fit_sigma0(k, err)
    r = scale_radii(p, sigma)
    ws = scale_weights(p, w, r)
    ws = ws / np.sum(ws * (2 * r + 1))
    return r, ws


def kernel_samples(half):
    """A symmetric kernel on the sample grid t = -100..99: g(t) = half[|t|] for
    |t| < len(half), 0 elsewhere (Sec. 3.2: a symmetric kernel on [-r, r] is approximated on
    [0, r] and mirrored)."""
    half = np.asarray(half, dtype=np.float64)
    if half.ndim != 1 or not (1 <= half.size <= N_RADII + 1):
        raise ValueError("half kernel must hold 1..101 samples (t = 0..100)")
    t = np.abs(sample_positions()).astype(np.int64)
    g = np.zeros(N_SAMPLES)
    inside = t < half.size
    g[inside] = half[t[inside]]
    return g


def fit_kernel(half, k, err="qf", dc=DC_VALUE):
    """Approximation of an arbitrary symmetric kernel by k weighted slices
    (Sec. 3.2 and Sec. 4: the same exhaustive search over increasing radii
    0..99 with closed-form weights under the chosen error).  Returns
    (radii, weights, error); the weights are the optimal ones, unnormalised."""
    m, h, gag = gram(err, dc, kernel_samples(half))
    p, w, e = _search(m, h, gag, k)
    return p, w, e


def kernel_error(half, radii, w, err="qf", dc=DC_VALUE):
    """Direct (g - S w)^T A (g - S w) of slices (radii, w) against the kernel `half`."""
    a = error_matrix(err, dc)
    t = sample_positions()
    approx = np.zeros(N_SAMPLES)
    for r, wi in zip(radii, w):
        approx += wi * (np.abs(t) <= r)
    d = kernel_samples(half) - approx
    return float(d @ (a @ d))
