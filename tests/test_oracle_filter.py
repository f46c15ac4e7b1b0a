"""Pins for the oracle's filter definition (Sec. 3): boundary extension against
numpy.pad, separable == direct 2D, the running-sum algorithm (Eq. alg1 then
Eq. indep) against the direct staircase convolution, impulse response,
constant preservation, symmetry, linearity and exact integer box sums."""
import numpy as np
import pytest

from oracle import filter as of
from oracle import fit

NP_MODE = {"replicate": "edge", "zero": "constant", "reflect": "reflect"}


@pytest.mark.parametrize("boundary", of.BOUNDARIES)
@pytest.mark.parametrize("n,before,after", [(5, 2, 3), (4, 9, 11), (1, 3, 2), (2, 5, 5), (7, 0, 0)])
def test_extension_matches_numpy_pad(boundary, n, before, after):
    a = np.arange(1, n + 1, dtype=np.float64) * 1.5
    got = of.extend_axis(a, 0, before, after, boundary)
    if boundary == "reflect" and n == 1:
        want = np.full(n + before + after, a[0])   # numpy refuses; a 1-pixel mirror repeats it
    else:
        want = np.pad(a, (before, after), mode=NP_MODE[boundary])
    assert np.array_equal(got, want)


def _running_sum_filter_1d(row, radii, weights, boundary):
    """Sec. 3.3 written out in plain Python: I(x) = sum_{x'<=x} f(x'), then
    sum_i w_i (I(x + r_i) - I(x - r_i - 1)), on the boundary-extended row."""
    rk = max(radii)
    n = len(row)
    ext = [row[of.fold_index(t, n, boundary)] if of.fold_index(t, n, boundary) >= 0 else 0.0
           for t in range(-rk - 1, n + rk)]
    run = []
    acc = 0.0
    for v in ext:
        acc += v
        run.append(acc)
    out = []
    for x in range(n):
        j = x + rk + 1
        out.append(sum(w * (run[j + r] - run[j - r - 1]) for r, w in zip(radii, weights)))
    return np.array(out)


@pytest.mark.parametrize("boundary", of.BOUNDARIES)
def test_running_sum_algorithm_equals_staircase_convolution(boundary):
    rng = np.random.default_rng(1)
    radii, weights = fit.fit_gaussian_boxes(5.0, 3)
    for n in (1, 3, 17, 40):
        row = rng.uniform(0, 255, n)
        want = of.conv1d_axis(row, of.staircase_kernel(radii, weights), 0, boundary)
        got = _running_sum_filter_1d(list(row), list(radii), list(weights), boundary)
        assert np.max(np.abs(got - want)) <= 1e-12 * 255 * 40


@pytest.mark.parametrize("boundary", of.BOUNDARIES)
def test_separable_equals_direct_2d(boundary):
    rng = np.random.default_rng(2)
    radii, weights = fit.fit_gaussian_boxes(2.0, 4)
    for shape in [(9, 13), (1, 6), (6, 1), (11, 7, 3)]:
        f = rng.uniform(0, 255, shape)
        a = of.filter_separable(f, radii, weights, boundary)
        b = of.filter_direct2d(f, radii, weights, boundary)
        assert np.max(np.abs(a - b)) <= 1e-12 * 255


def test_impulse_response_is_outer_product_of_staircases():
    radii, weights = fit.fit_gaussian_boxes(8.0, 4)     # radii 4, 9, 14, 20
    k = of.staircase_kernel(radii, weights)
    n = 2 * 20 + 1 + 10
    f = np.zeros((n, n))
    f[n // 2, n // 2] = 1.0
    y = of.filter_separable(f, radii, weights, "zero")
    c = n // 2
    got = y[c - 20:c + 21, c - 20:c + 21]
    assert np.allclose(got, np.outer(k, k), atol=1e-15)
    assert abs(y.sum() - 1.0) < 1e-12
    # nothing outside the support
    assert np.all(y[:c - 20] == 0) and np.all(y[c + 21:] == 0)


@pytest.mark.parametrize("boundary", ["replicate", "reflect"])
def test_constant_image_preserved(boundary):
    radii, weights = fit.fit_gaussian_boxes(3.0, 5)
    f = np.full((7, 12), 42.0)
    y = of.filter_separable(f, radii, weights, boundary)
    assert np.max(np.abs(y - 42.0)) < 1e-12


def test_constant_image_interior_with_zero_boundary():
    radii, weights = fit.fit_gaussian_boxes(3.0, 5)
    rk = max(radii)
    f = np.full((2 * rk + 5, 2 * rk + 6), 42.0)
    y = of.filter_separable(f, radii, weights, "zero")
    inner = y[rk:-rk, rk:-rk]
    assert np.max(np.abs(inner - 42.0)) < 1e-12
    assert y[0, 0] < 42.0


@pytest.mark.parametrize("boundary", of.BOUNDARIES)
def test_flip_symmetry_and_linearity(boundary):
    rng = np.random.default_rng(3)
    radii, weights = fit.fit_gaussian_boxes(4.0, 3)
    f = rng.uniform(0, 1, (10, 15))
    g = rng.uniform(0, 1, (10, 15))
    y = of.filter_separable(f, radii, weights, boundary)
    assert np.allclose(of.filter_separable(f[::-1, ::-1], radii, weights, boundary), y[::-1, ::-1],
                       atol=1e-13)
    yl = of.filter_separable(2.0 * f - 3.0 * g, radii, weights, boundary)
    assert np.allclose(yl, 2.0 * y - 3.0 * of.filter_separable(g, radii, weights, boundary),
                       atol=1e-12)


@pytest.mark.parametrize("boundary", of.BOUNDARIES)
@pytest.mark.parametrize("axis", [0, 1])
def test_int_box_sums_equal_brute_force(boundary, axis):
    rng = np.random.default_rng(4)
    f = rng.integers(0, 256, (6, 9), dtype=np.uint8)
    radii = [0, 1, 3, 11]
    got = of.box_sums_int64(f, radii, boundary, axis)
    for i, r in enumerate(radii):
        want = np.zeros(f.shape, dtype=np.int64)
        for y in range(f.shape[0]):
            for x in range(f.shape[1]):
                s = 0
                for t in range(-r, r + 1):
                    if axis == 1:
                        j = of.fold_index(x + t, f.shape[1], boundary)
                        s += int(f[y, j]) if j >= 0 else 0
                    else:
                        j = of.fold_index(y + t, f.shape[0], boundary)
                        s += int(f[j, x]) if j >= 0 else 0
                want[y, x] = s
        assert np.array_equal(got[i], want)


def test_int_box_sums_weighted_equal_row_filter():
    rng = np.random.default_rng(5)
    f = rng.integers(0, 65536, (5, 33), dtype=np.uint16)
    radii, weights = fit.fit_gaussian_boxes(6.0, 4)
    b = of.box_sums_int64(f, radii, "reflect", 1)
    r_from_boxes = np.tensordot(weights, b.astype(np.float64), axes=1)
    want = of.conv1d_axis(f.astype(np.float64), of.staircase_kernel(radii, weights), 1, "reflect")
    assert np.max(np.abs(r_from_boxes - want)) < 1e-12 * 65535 * 10


def test_true_gaussian_kernel():
    for sigma in (0.7, 3.0, 10.0):
        k = of.true_gaussian_kernel(sigma)
        assert abs(k.sum() - 1.0) < 1e-15
        assert np.allclose(k, k[::-1])
        t = np.arange(k.size) - (k.size - 1) // 2
        if sigma >= 3:
            assert abs((k * t * t).sum() / sigma ** 2 - 1.0) < 1e-3


def test_psnr_definition():
    a = np.zeros((4, 4))
    b = np.full((4, 4), 0.1)
    assert abs(of.psnr(a, b) - 20.0) < 1e-12


@pytest.mark.parametrize("boundary", of.BOUNDARIES)
def test_rows_at_equals_full_filter(boundary):
    rng = np.random.default_rng(6)
    f = rng.uniform(0, 255, (23, 19, 2))
    radii, weights = fit.fit_gaussian_boxes(4.0, 4)
    full = of.filter_separable(f, radii, weights, boundary)
    ys = [0, 1, 11, 21, 22]
    assert np.max(np.abs(of.filter_rows_at(f, radii, weights, boundary, ys) - full[ys])) < 1e-10


def test_window_equals_full_filter():
    # the window evaluation is the full definition restricted to a window:
    # windows at corners, edges and inside, every boundary, radius > image side
    rng = np.random.default_rng(41)
    f = rng.uniform(0, 255, size=(23, 31, 2))
    for radii, weights in (([0, 2, 5], [0.2, 0.05, 0.01]), ([1, 4, 9, 30], [0.1, 0.04, 0.02, 0.003])):
        for boundary in ("replicate", "zero", "reflect"):
            full = of.filter_separable(f, radii, weights, boundary)
            for (y0, y1, x0, x1) in ((0, 5, 0, 7), (18, 23, 24, 31), (7, 16, 3, 29), (0, 23, 0, 31)):
                win = of.filter_window_at(f, radii, weights, boundary, y0, y1, x0, x1)
                assert np.allclose(win, full[y0:y1, x0:x1], rtol=1e-12, atol=1e-9), (boundary, y0, x0)
