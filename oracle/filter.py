"""Oracle for the filter itself (Sec. 3.1-3.4): what the running-sum method computes.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 / int64 numpy.

Result definition.  With inclusive radii r_i and slice weights w_i, the 1D
kernel is the staircase k(t) = sum over i with |t| <= r_i of w_i (the sum of
K centred slices, Eq. S_i / Eq. ciwi).  The running-sum algorithm
(Eq. alg1 then Eq. indep) evaluates exactly the convolution with k, so the
oracle writes that convolution out directly:

    rows:     R(y, x) = sum_t k_x(t) f(y, x + t)          (Sec. 3.4)
    columns:  Y(y, x) = sum_s k_y(s) R(y + s, x)

Pixels outside the image are supplied by the boundary rule (the paper does
not give one): 'replicate' (edge pixel repeated), 'zero', or 'reflect'
(mirror about the edge pixel without repeating it, folded again as often as
needed when the radius exceeds the image).

Images are (H, W) or (H, W, C) arrays; channels are filtered independently.
The sampled form (filter_sampled) is Y on a regular grid of pixels; the 3D
form (filter_volume) applies the same 1D convolution along a third axis of a
(D, H, W[, C]) volume (Sec. 3.4, the d-dimensional case).
"""
import math

import numpy as np

BOUNDARIES = ("replicate", "zero", "reflect")


def fold_index(t, n, boundary):
    """Source index for position t on an axis of length n, or -1 for a zero pixel."""
    if 0 <= t < n:
        return t
    if boundary == "zero":
        return -1
    if boundary == "replicate":
        return 0 if t < 0 else n - 1
    if boundary == "reflect":
        if n == 1:
            return 0
        period = 2 * (n - 1)
        m = t % period
        return m if m < n else period - m
    raise ValueError("unknown boundary %r" % (boundary,))


def extend_axis(a, axis, before, after, boundary):
    """Pads `a` along `axis` by `before`/`after` samples using fold_index."""
    n = a.shape[axis]
    idx = [fold_index(t, n, boundary) for t in range(-before, n + after)]
    idx = np.array(idx, dtype=np.int64)
    out = np.take(a, np.maximum(idx, 0), axis=axis)
    if boundary == "zero":
        shape = [1] * a.ndim
        shape[axis] = idx.size
        out = out * (idx >= 0).reshape(shape)
    return out


def staircase_kernel(radii, weights):
    """k(t) for t = -r_K .. r_K: sum of the slices with |t| <= r_i (Eq. ciwi)."""
    radii = [int(r) for r in radii]
    rk = max(radii)
    t = np.arange(-rk, rk + 1)
    k = np.zeros(t.size, dtype=np.float64)
    for r, w in zip(radii, weights):
        k += float(w) * (np.abs(t) <= r)
    return k


def _as3d(f):
    f = np.asarray(f)
    if f.ndim == 2:
        return f[:, :, None], True
    if f.ndim != 3:
        raise ValueError("image must be (H, W) or (H, W, C)")
    return f, False


def conv1d_axis(f, k, axis, boundary):
    """Direct FP64 correlation of f with the symmetric kernel k along `axis`."""
    f = np.asarray(f, dtype=np.float64)
    rk = (k.size - 1) // 2
    g = extend_axis(f, axis, rk, rk, boundary)
    n = f.shape[axis]
    out = np.zeros(f.shape, dtype=np.float64)
    for j, kv in enumerate(k):
        if kv == 0.0:
            continue
        out += kv * np.take(g, np.arange(j, j + n), axis=axis)
    return out


def filter_separable(f, radii, weights, boundary="replicate", radii_y=None, weights_y=None):
    """Rows with k_x, then columns with k_y (Sec. 3.4), each a direct 1D convolution."""
    kx = staircase_kernel(radii, weights)
    ky = kx if radii_y is None else staircase_kernel(radii_y, weights_y)
    f3, squeeze = _as3d(f)
    r = conv1d_axis(f3, kx, 1, boundary)
    y = conv1d_axis(r, ky, 0, boundary)
    return y[:, :, 0] if squeeze else y


def filter_direct2d(f, radii, weights, boundary="replicate"):
    """Direct 2D convolution with the outer-product kernel k_y k_x^T (tiny inputs only)."""
    k = staircase_kernel(radii, weights)
    rk = (k.size - 1) // 2
    f3, squeeze = _as3d(np.asarray(f, dtype=np.float64))
    h, w, _ = f3.shape
    g = extend_axis(extend_axis(f3, 0, rk, rk, boundary), 1, rk, rk, boundary)
    out = np.zeros(f3.shape, dtype=np.float64)
    for s in range(k.size):
        for t in range(k.size):
            out += k[s] * k[t] * g[s:s + h, t:t + w, :]
    return out[:, :, 0] if squeeze else out


def box_sums_int64(f, radii, boundary="replicate", axis=1):
    """Integer box sums B_i = I(x + r_i) - I(x - r_i - 1) along `axis` (Eq. alg1,
    Eq. indep without the weights), from an int64 running sum of the extended
    signal.  Returns an int64 array of shape (K,) + f.shape."""
    f = np.asarray(f)
    if f.dtype.kind not in "ui":
        raise ValueError("integer input expected")
    rk = max(int(r) for r in radii)
    g = extend_axis(f.astype(np.int64), axis, rk + 1, rk, boundary)
    # running sum I along the extended axis; position j of g is pixel j - rk - 1
    cs = np.cumsum(g, axis=axis, dtype=np.int64)
    n = f.shape[axis]
    x = np.arange(n)
    out = []
    for r in radii:
        r = int(r)
        hi = np.take(cs, x + r + rk + 1, axis=axis)
        lo = np.take(cs, x - r + rk, axis=axis)
        out.append(hi - lo)
    return np.stack(out)


def true_gaussian_kernel(sigma):
    """Sampled exp(-t^2/(2 sigma^2)) for |t| <= ceil(4 sigma), normalised to sum 1:
    the exact filter that the approximation is measured against (Sec. 5)."""
    rk = int(math.ceil(4.0 * sigma))
    t = np.arange(-rk, rk + 1, dtype=np.float64)
    k = np.exp(-t * t / (2.0 * sigma * sigma))
    return k / k.sum()


def filter_true_gaussian(f, sigma, boundary="replicate"):
    k = true_gaussian_kernel(sigma)
    f3, squeeze = _as3d(f)
    y = conv1d_axis(conv1d_axis(f3, k, 1, boundary), k, 0, boundary)
    return y[:, :, 0] if squeeze else y


def psnr(a, b, peak=1.0):
    """-10 log10(MSE) with values scaled to [0, peak] (Sec. 5)."""
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else -10.0 * math.log10(mse / (peak * peak))


def filter_rows_at(f, radii, weights, boundary, ys):
    """Y at the output rows `ys` only (same definition as filter_separable):
    the row convolution of the 2 r_K + 1 source rows each output row needs,
    then the column convolution at that row.  For sampling large images."""
    kx = staircase_kernel(radii, weights)
    rk = (kx.size - 1) // 2
    f3, squeeze = _as3d(f)
    h = f3.shape[0]
    out = []
    for y in ys:
        rows = [fold_index(y + s, h, boundary) for s in range(-rk, rk + 1)]
        acc = np.zeros(f3.shape[1:], dtype=np.float64)
        for kv, src in zip(kx, rows):
            if src < 0 or kv == 0.0:
                continue
            acc += kv * conv1d_axis(f3[src:src + 1].astype(np.float64), kx, 1, boundary)[0]
        out.append(acc)
    out = np.stack(out)
    return out[:, :, 0] if squeeze else out


def filter_window_at(f, radii, weights, boundary, y0, y1, x0, x1):
    """Y on the window rows [y0, y1) x columns [x0, x1) only (same definition as
    filter_separable): the source rows y0 - r_K .. y1 - 1 + r_K and columns
    x0 - r_K .. x1 - 1 + r_K, extended by the boundary rule, row-convolved on
    the window's columns, then column-convolved on its rows.  For sampling
    large images."""
    kx = staircase_kernel(radii, weights)
    rk = (kx.size - 1) // 2
    f3, squeeze = _as3d(f)
    h, w = f3.shape[0], f3.shape[1]
    rows = np.array([fold_index(t, h, boundary) for t in range(y0 - rk, y1 + rk)])
    cols = np.array([fold_index(t, w, boundary) for t in range(x0 - rk, x1 + rk)])
    g = f3[np.maximum(rows, 0)][:, np.maximum(cols, 0)].astype(np.float64)
    g[rows < 0] = 0.0          # zero-boundary pixels
    g[:, cols < 0] = 0.0
    nx, ny = x1 - x0, y1 - y0
    r = np.zeros((len(rows), nx, f3.shape[2]), dtype=np.float64)
    for j, kv in enumerate(kx):
        if kv != 0.0:
            r += kv * g[:, j:j + nx]
    out = np.zeros((ny, nx, f3.shape[2]), dtype=np.float64)
    for i, kv in enumerate(kx):
        if kv != 0.0:
            out += kv * r[i:i + ny]
    return out[:, :, 0] if squeeze else out


def filter_sampled(f, radii, weights, boundary, step, offset=(0, 0)):
    """The filter's response on the grid of pixels (oy + i sy, ox + j sx) only
    (Sec. 3.4: Eq. indep may be evaluated at any subset of the pixels, e.g. for
    downscaling).  By definition these are the pixels of filter_separable's
    output Y at those positions; `step` = (sy, sx), `offset` = (oy, ox)."""
    sy, sx = int(step[0]), int(step[1])
    oy, ox = int(offset[0]), int(offset[1])
    if sy < 1 or sx < 1 or not (0 <= oy < sy) or not (0 <= ox < sx):
        raise ValueError("bad sampling grid")
    y = filter_separable(f, radii, weights, boundary)
    return y[oy::sy, ox::sx]


def _as4d(f):
    f = np.asarray(f)
    if f.ndim == 3:
        return f[..., None], True
    if f.ndim != 4:
        raise ValueError("volume must be (D, H, W) or (D, H, W, C)")
    return f, False


def filter_volume(f, radii, weights, boundary="replicate", radii_z=None, weights_z=None):
    """3D separable filter (Sec. 3.4, the d-dimensional case): the staircase
    kernel k_x along the rows (axis 2), k_x along the columns (axis 1), and k_z
    (k_x unless given) along the slices (axis 0), each a direct FP64 1D
    convolution with the boundary rule on its own axis.  f is (D, H, W[, C])."""
    kx = staircase_kernel(radii, weights)
    kz = kx if radii_z is None else staircase_kernel(radii_z, weights_z)
    f4, squeeze = _as4d(f)
    r = conv1d_axis(f4, kx, 2, boundary)
    r = conv1d_axis(r, kx, 1, boundary)
    r = conv1d_axis(r, kz, 0, boundary)
    return r[..., 0] if squeeze else r


def filter_direct3d(f, radii, weights, boundary="replicate", radii_z=None, weights_z=None):
    """Direct 3D convolution with the kernel k_z(a) k_x(b) k_x(c) summed over every
    offset (a, b, c) of the extended volume (tiny volumes only)."""
    kx = staircase_kernel(radii, weights)
    kz = kx if radii_z is None else staircase_kernel(radii_z, weights_z)
    rx = (kx.size - 1) // 2
    rz = (kz.size - 1) // 2
    f4, squeeze = _as4d(np.asarray(f, dtype=np.float64))
    d, h, w, _ = f4.shape
    g = extend_axis(f4, 0, rz, rz, boundary)
    g = extend_axis(g, 1, rx, rx, boundary)
    g = extend_axis(g, 2, rx, rx, boundary)
    out = np.zeros(f4.shape, dtype=np.float64)
    for a in range(kz.size):
        for b in range(kx.size):
            for c in range(kx.size):
                out += kz[a] * kx[b] * kx[c] * g[a:a + d, b:b + h, c:c + w]
    return out[..., 0] if squeeze else out


# ------------------------------------------------------------------ all host cores (C helper)
_BOUNDARY_CODE = {"replicate": 0, "zero": 1, "reflect": 2}


def filter_separable_c(f, radii, weights, boundary="replicate"):
    """filter_separable by the C helper (oracle/conv.c: the same FP64 direct
    convolutions, rows then columns, spread over the host's cores)."""
    import ctypes
    from oracle import _native
    f3, squeeze = _as3d(np.ascontiguousarray(f, dtype=np.float64))
    f3 = np.ascontiguousarray(f3)
    h, w, c = f3.shape
    out = np.empty_like(f3)
    r = (ctypes.c_int * len(radii))(*[int(v) for v in radii])
    wt = (ctypes.c_double * len(weights))(*[float(v) for v in weights])
    dp = ctypes.POINTER(ctypes.c_double)
    rc = _native.conv_lib().oracle_conv_separable(f3.ctypes.data_as(dp), h, w, c, r, wt, len(radii),
                                                   _BOUNDARY_CODE[boundary], out.ctypes.data_as(dp))
    if rc != 0:
        raise MemoryError("oracle_conv_separable")
    return out[:, :, 0] if squeeze else out


def host_threads():
    """OpenMP threads the C helper uses."""
    from oracle import _native
    return int(_native.conv_lib().oracle_threads())
