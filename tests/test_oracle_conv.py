"""The oracle's C helpers (oracle/conv.c): the FP64 separable direct
convolution spread over the host cores must equal the plain numpy
definition (filter_separable, itself pinned by brute force and the paper's
invariants in test_oracle_filter.py) for every boundary, channel count and
radius beyond the image; the CPU running-sum method (Sec. 3.3-3.4), timed as
context by the benchmark, must agree with it within FP32 rounding."""
import ctypes

import numpy as np
import pytest

from oracle import _native
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth


@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
@pytest.mark.parametrize("shape", [(1, 1), (9, 1), (1, 13), (37, 61), (64, 40, 3)])
def test_c_oracle_equals_numpy_definition(boundary, shape):
    f = synth.image(shape[0], shape[1], seed=21, dtype="f32", c=shape[2] if len(shape) == 3 else 1)
    for sigma, K in ((0.5, 3), (3.0, 4), (30.0, 5)):          # the last: radii beyond the image
        r, w = ofit.fit_gaussian_boxes(sigma, K)
        want = of.filter_separable(f.astype(np.float64), r, w, boundary)
        got = of.filter_separable_c(f, r, w, boundary)
        assert np.array_equal(got, want), (boundary, shape, sigma)


def test_c_oracle_explicit_boxes_and_threads():
    f = synth.image(50, 77, seed=22, dtype="f32")
    r = [0, 2, 2, 9]
    w = [0.3, 0.05, 0.02, 0.001]
    assert np.array_equal(of.filter_separable_c(f, r, w, "reflect"),
                          of.filter_separable(f.astype(np.float64), r, w, "reflect"))
    assert of.host_threads() >= 1


def _boxsum(f, r, w, boundary):
    lib = _native.conv_lib()
    f = np.ascontiguousarray(f, dtype=np.uint8)
    out = np.empty(f.shape, dtype=np.float32)
    rr = (ctypes.c_int * len(r))(*[int(v) for v in r])
    ww = (ctypes.c_float * len(w))(*[float(v) for v in w])
    rc = lib.oracle_boxsum_u8_f32(f.ctypes.data, f.shape[1], f.shape[0], f.shape[1], rr, ww, len(r),
                                  {"replicate": 0, "zero": 1, "reflect": 2}[boundary],
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    assert rc == 0
    return out


@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
def test_cpu_running_sum_method_agrees_with_the_definition(boundary):
    f = synth.image(150, 230, seed=23, dtype="u8")
    for sigma, K in ((1.0, 3), (6.0, 4), (20.0, 5)):
        r, w = ofit.fit_gaussian_boxes(sigma, K)
        w32 = np.float32(w)
        ref = of.filter_separable(f.astype(np.float64), r, w32.astype(np.float64), boundary)
        got = _boxsum(f, r, w32, boundary)
        # FP32 column running sums over a band of rows: a few ulps of the sums
        assert float(np.max(np.abs(got - ref))) <= 1e-3 * float(np.max(np.abs(ref))), (boundary, sigma)
