"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds none of the filter's arithmetic: it only draws images and
workload descriptions.  Natural images have a Fourier amplitude close to 1/f
(Field's observation, the prior of Sec. 4.1), so the stand-in for the paper's
photographs is a 1/f-amplitude random field:

1. complex white Gaussian noise from numpy's PCG64 with a fixed seed;
2. multiplied by 1/|f| (the DC term set to 0);
3. real part of the inverse 2D FFT;
4. min-max rescaled to [0, 255]; rounded half-to-even for uint8/uint16 inputs.
"""
import math

import numpy as np


def field_1overf(h, w, seed, c=1):
    """(h, w) float64 field in [0, 255] (or (h, w, c) with independent channels)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((h, w, c), dtype=np.float64)
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.fftfreq(w)[None, :]
    mag = np.sqrt(fy * fy + fx * fx)
    amp = np.zeros_like(mag)
    amp[mag > 0] = 1.0 / mag[mag > 0]
    for ch in range(c):
        noise = rng.standard_normal((h, w)) + 1j * rng.standard_normal((h, w))
        f = np.real(np.fft.ifft2(noise * amp))
        lo, hi = f.min(), f.max()
        out[:, :, ch] = (f - lo) * (255.0 / (hi - lo)) if hi > lo else 0.0
    return out[:, :, 0] if c == 1 else out


def image(h, w, seed, dtype="f32", c=1, offset=0.0):
    """Synthetic image as a numpy array: dtype 'u8', 'u16', 'f32' (bf16/f16 inputs are
    produced by rounding the 'f32' image on the device side of the test)."""
    f = field_1overf(h, w, seed, c)
    if dtype == "u8":
        return np.rint(f).astype(np.uint8)
    if dtype == "u16":
        return np.rint(f * 257.0).astype(np.uint16)
    if dtype in ("f32", "bf16", "f16"):
        return (f + offset).astype(np.float32)
    raise ValueError(dtype)


def log_uniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def uneven_batch(n=64, seed=3, side_lo=256, side_hi=4096, sigma_lo=1.0, sigma_hi=50.0,
                 ks=(3, 4, 5), c=3):
    """Image descriptions for a batch of uneven images: list of dicts with
    h, w, c, sigma, K, seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hs = np.rint(log_uniform(rng, side_lo, side_hi, n)).astype(int)
    ws = np.rint(log_uniform(rng, side_lo, side_hi, n)).astype(int)
    sig = log_uniform(rng, sigma_lo, sigma_hi, n)
    kk = rng.choice(np.array(ks), n)
    return [dict(h=int(hs[i]), w=int(ws[i]), c=c, sigma=float(sig[i]), K=int(kk[i]),
                 seed=1000 + seed * 100000 + i) for i in range(n)]


def request_stream(n=10000, seed=5, rate_hz=1000.0, side_lo=128, side_hi=8192,
                   sigma_lo=0.5, sigma_hi=64.0, ks=(3, 4, 5), dtypes=("u8", "f32", "bf16"),
                   channels=(1, 3)):
    """Poisson arrivals of filter requests: list of dicts with t_arrive (s), h, w, c,
    dtype, sigma, K."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, n)
    t = np.cumsum(gaps) - gaps[0]
    hs = np.rint(log_uniform(rng, side_lo, side_hi, n)).astype(int)
    ws = np.rint(log_uniform(rng, side_lo, side_hi, n)).astype(int)
    cs = rng.choice(np.array(channels), n)
    dts = rng.choice(np.array(dtypes), n)
    sig = log_uniform(rng, sigma_lo, sigma_hi, n)
    kk = rng.choice(np.array(ks), n)
    return [dict(t_arrive=float(t[i]), h=int(hs[i]), w=int(ws[i]), c=int(cs[i]),
                 dtype=str(dts[i]), sigma=float(sig[i]), K=int(kk[i])) for i in range(n)]


# ------------------------------------------------------------------ inputs whose mean is far below their range
# Natural-image fields keep every pixel within a few times the image mean.
# The inputs below do not: most pixels are 0 and a few are bright, so many
# outputs are far smaller than the image's mean output.  They probe the error
# of differences of running sums near dark pixels.

def sparse_points(h, w, seed, density=0.01, c=1, dtype="u8", peak=255.0):
    """Black image with a fraction `density` of pixels set to a bright value
    (uniform in [peak / 2, peak]; integer for integer dtypes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    on = rng.random((h, w, c)) < density
    val = rng.uniform(0.5 * peak, peak, (h, w, c))
    f = np.where(on, val, 0.0)
    f = f[:, :, 0] if c == 1 else f
    return _cast(f, dtype)


def step_edge(h, w, kind="horizontal", c=1, dtype="u8", lo=0.0, hi=255.0, at=0.5):
    """A step of height hi - lo: 'horizontal' (bright rows above row at*h),
    'vertical' (bright columns left of column at*w), 'diagonal' (bright where
    x + y < at (h + w)), or 'corner' (bright only in the top-left quadrant)."""
    y = np.arange(h)[:, None]
    x = np.arange(w)[None, :]
    if kind == "horizontal":
        m = np.broadcast_to(y < int(at * h), (h, w))
    elif kind == "vertical":
        m = np.broadcast_to(x < int(at * w), (h, w))
    elif kind == "diagonal":
        m = (x + y) < int(at * (h + w))
    elif kind == "corner":
        m = (y < int(at * h)) & (x < int(at * w))
    else:
        raise ValueError(kind)
    f = np.where(m, hi, lo).astype(np.float64)
    if c > 1:
        f = np.repeat(f[:, :, None], c, axis=2)
    return _cast(f, dtype)


def _cast(f, dtype):
    if dtype == "u8":
        return np.rint(f).astype(np.uint8)
    if dtype == "u16":
        return np.rint(f * 257.0).astype(np.uint16)
    if dtype in ("f32", "bf16", "f16"):
        return f.astype(np.float32)
    raise ValueError(dtype)
