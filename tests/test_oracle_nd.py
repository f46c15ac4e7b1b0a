"""Pins for the oracle's sampled-output and 3D forms (Sec. 3.4): sampled
outputs against the brute-force 2D convolution at the grid points, the 3D
separable filter against the brute-force triple sum, its impulse response (the
outer product of three staircases), constant preservation, the D = 1 case
reducing to the 2D filter, and the symmetry of axis exchange."""
import numpy as np
import pytest

from oracle import filter as of


@pytest.mark.parametrize("boundary", of.BOUNDARIES)
@pytest.mark.parametrize("step,offset", [((2, 2), (0, 0)), ((3, 2), (2, 1)), ((1, 4), (0, 3)), ((5, 1), (4, 0)),
                                         ((7, 9), (6, 8))])
def test_sampled_equals_direct_2d_at_grid(boundary, step, offset):
    rng = np.random.default_rng(11)
    f = rng.integers(0, 256, (13, 17, 2)).astype(np.float64)
    radii, w = [0, 2, 5], [0.09, 0.04, 0.02]
    got = of.filter_sampled(f, radii, w, boundary, step, offset)
    full = of.filter_direct2d(f, radii, w, boundary)
    want = full[offset[0]::step[0], offset[1]::step[1]]
    assert got.shape == want.shape
    assert got.shape[0] == -(-(13 - offset[0]) // step[0]) and got.shape[1] == -(-(17 - offset[1]) // step[1])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)


def test_sampled_rejects_bad_grid():
    f = np.zeros((4, 4))
    for step, offset in [((0, 1), (0, 0)), ((2, 2), (2, 0)), ((2, 2), (0, -1))]:
        with pytest.raises(ValueError):
            of.filter_sampled(f, [1], [1 / 3], "replicate", step, offset)


@pytest.mark.parametrize("boundary", of.BOUNDARIES)
@pytest.mark.parametrize("shape", [(4, 5, 6), (1, 3, 7), (6, 2, 3), (3, 4, 5, 2)])
def test_volume_equals_direct_3d(boundary, shape):
    rng = np.random.default_rng(12)
    f = rng.integers(0, 256, shape).astype(np.float64)
    # radii up to 4 exceed several axes, so the boundary rule folds repeatedly
    args = ([0, 1, 4], [0.2, 0.1, 0.03])
    got = of.filter_volume(f, *args, boundary, radii_z=[1, 3], weights_z=[0.1, 0.05])
    want = of.filter_direct3d(f, *args, boundary, radii_z=[1, 3], weights_z=[0.1, 0.05])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)


def test_volume_impulse_is_outer_product_of_staircases():
    radii, w = [1, 2], [0.3, 0.1]
    rz, wz = [0, 3], [0.25, 0.07]
    f = np.zeros((9, 7, 7))
    f[4, 3, 3] = 1.0
    y = of.filter_volume(f, radii, w, "zero", radii_z=rz, weights_z=wz)
    kx = of.staircase_kernel(radii, w)
    kz = of.staircase_kernel(rz, wz)
    want = np.zeros_like(f)
    want[1:8, 1:6, 1:6] = kz[:, None, None] * kx[None, :, None] * kx[None, None, :]
    np.testing.assert_allclose(y, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("boundary", ["replicate", "reflect"])
def test_volume_constant_preserved(boundary):
    radii = np.array([1, 3, 6])
    w = np.array([0.5, 0.3, 0.2])
    w = w / np.sum(w * (2 * radii + 1))
    f = np.full((5, 6, 4), 7.25)
    np.testing.assert_allclose(of.filter_volume(f, radii, w, boundary), f, rtol=1e-13)


@pytest.mark.parametrize("boundary", ["replicate", "reflect"])
def test_single_slice_volume_is_the_2d_filter(boundary):
    # one slice: every depth tap reads the slice itself, and sum_z k_z = 1
    rng = np.random.default_rng(13)
    f = rng.random((9, 11, 3))
    radii = np.array([0, 2, 4])
    w = np.array([0.3, 0.2, 0.1])
    w = w / np.sum(w * (2 * radii + 1))
    got = of.filter_volume(f[None], radii, w, boundary)[0]
    np.testing.assert_allclose(got, of.filter_separable(f, radii, w, boundary), rtol=0, atol=1e-12)


def test_volume_axis_exchange_symmetry():
    # with the same kernel on every axis, exchanging depth and rows commutes with the filter
    rng = np.random.default_rng(14)
    f = rng.random((5, 8, 6))
    radii, w = [1, 3], [0.2, 0.05]
    a = of.filter_volume(f, radii, w, "reflect")
    b = of.filter_volume(np.swapaxes(f, 0, 1).copy(), radii, w, "reflect")
    np.testing.assert_allclose(np.swapaxes(b, 0, 1), a, rtol=0, atol=1e-12)
