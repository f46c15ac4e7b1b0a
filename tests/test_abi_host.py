"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/gaussbox.h declares, its own fitter reproduces Table 1
and agrees with the oracle's fitter, and argument errors are reported before
anything touches a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from golden_tables import read_param_table
from oracle import fit as ofit

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gb():
    from paper_1107_4958_gb300 import build
    build.build()
    from paper_1107_4958_gb300 import gaussbox
    return gaussbox


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:gf_status|const char\s*\*|int|void)\s+(\w+)\s*\(", text, flags=re.M)
    return names


def test_exports_every_declared_symbol(gb):
    names = declared_functions()
    assert "gauss_filter" in names and "gauss_fit_boxes" in names
    for n in names:
        assert hasattr(gb.lib(), n), n


def test_version_and_status_strings(gb):
    assert "sm_103a" in gb.gf_version()
    assert gb.gf_status_string(0) == "GF_OK"
    assert "invalid" in gb.gf_status_string(1)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_library_fitter_reproduces_table1(gb, k):
    p, c, w, _e = gb.gauss_fit_sigma0(k)
    p_paper, c_paper = read_param_table("table1_quadratic_form.txt")[k]
    assert list(p) == p_paper
    assert np.max(np.abs(c - np.array(c_paper))) <= 2e-4


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("err", [0, 1])
def test_library_fitter_matches_oracle(gb, k, err):
    p, c, w, e = gb.gauss_fit_sigma0(k, err)
    op, oc, ow, oe = ofit.fit_sigma0(k, "qf" if err == 0 else "l2")
    assert list(p) == list(op)
    assert np.allclose(w, ow, rtol=1e-9, atol=1e-12)
    assert abs(e - oe) <= 1e-9 * max(1.0, abs(oe))


@pytest.mark.parametrize("sigma", [0.3, 0.5, 1.0, 2.0, 5.0, 8.0, 31.83, 32.0, 50.0, 100.0, 137.0])
@pytest.mark.parametrize("k", [3, 4, 5])
def test_library_scaling_matches_oracle(gb, sigma, k):
    r, w = gb.gauss_fit_boxes(sigma, k)
    orr, ow = ofit.fit_gaussian_boxes(sigma, k)
    assert list(r) == list(orr)
    assert np.allclose(w, ow, rtol=1e-9, atol=0)


def test_fit_argument_errors(gb):
    from paper_1107_4958_gb300 import abi_types as T
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(gb.GaussboxError) as ei:
            gb.gauss_fit_boxes(bad, 3)
        assert ei.value.status == T.GF_EINVAL
    # raw calls return the code
    assert gb.lib().gauss_fit_boxes(2.0, 6, 0, None, None) == T.GF_EUNSUPPORTED
    assert gb.lib().gauss_fit_boxes(2.0, 3, 7, None, None) == T.GF_EINVAL


def test_filter_argument_errors_before_any_device_work(gb):
    from paper_1107_4958_gb300 import abi_types as T
    L = gb.lib()
    base = 1 << 20

    def call(d_in=base, in_pitch=64, d_out=base * 4, out_pitch=64, H=16, W=16, C=1, idt=T.GF_F32,
             odt=T.GF_F32, sigma=2.0, K=3, b=T.GF_REPLICATE):
        return L.gauss_filter(ctypes.c_void_p(d_in), in_pitch, ctypes.c_void_p(d_out), out_pitch, H, W, C,
                              idt, odt, sigma, K, b, None)

    assert call(H=0) == T.GF_EINVAL
    assert call(W=-3) == T.GF_EINVAL
    assert call(C=5) == T.GF_EINVAL
    assert call(in_pitch=32) == T.GF_EINVAL                  # pitch < W*C*4
    assert call(sigma=0.0) == T.GF_EINVAL
    assert call(sigma=float("nan")) == T.GF_EINVAL
    assert call(K=0) == T.GF_EUNSUPPORTED
    assert call(K=6) == T.GF_EUNSUPPORTED
    assert call(b=3) == T.GF_EINVAL
    assert call(idt=T.GF_U8, odt=T.GF_BF16, in_pitch=16) == T.GF_EUNSUPPORTED
    assert call(odt=T.GF_U8) == T.GF_EUNSUPPORTED
    assert call(d_out=base + 128) == T.GF_EINVAL            # overlapping buffers
    assert call(d_in=0) == T.GF_EINVAL
    # radii outside 0..4096 through the explicit-kernel call
    r = (ctypes.c_int32 * 2)(1, 5000)
    w = (ctypes.c_double * 2)(0.1, 0.1)
    assert L.gauss_filter_boxes(ctypes.c_void_p(base), 64, ctypes.c_void_p(base * 4), 64, 16, 16, 1,
                                T.GF_F32, T.GF_F32, r, w, 2, 0, None) == T.GF_EINVAL


# ---- fit of arbitrary symmetric kernels (gauss_fit_kernel) -------------------------
def _kernels():
    t = np.arange(80, dtype=np.float64)
    return {
        "tent": np.maximum(0.0, 1.0 - t / 35.0),
        "laplace": np.exp(-t / 9.0),
        "dog": np.exp(-t ** 2 / (2 * 14.0 ** 2)) - 0.3 * np.exp(-t ** 2 / (2 * 30.0 ** 2)),
        "cosine": np.cos(np.minimum(t, 29) * np.pi / 60.0) * (t < 30),
    }


@pytest.mark.parametrize("name", ["tent", "laplace", "dog", "cosine"])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("err", [0, 1])
def test_library_kernel_fit_matches_oracle(gb, name, k, err):
    half = _kernels()[name]
    r, w, e = gb.gauss_fit_kernel(half, k, err)
    ro, wo, eo = ofit.fit_kernel(half, k, "qf" if err == 0 else "l2")
    assert r == [int(v) for v in ro]
    np.testing.assert_allclose(w, wo, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(e, eo, rtol=1e-8, atol=1e-13)


def test_library_kernel_fit_k5_and_sigma0_gaussian(gb):
    half = _kernels()["dog"]
    r, w, _e = gb.gauss_fit_kernel(half, 5)
    ro, wo, _eo = ofit.fit_kernel(half, 5)
    assert r == [int(v) for v in ro]
    np.testing.assert_allclose(w, wo, rtol=1e-9)
    # the Gaussian at sigma0 sampled on t = 0..100 is the Table 1 problem itself
    g = np.exp(-np.arange(101) ** 2 / (2.0 * ofit.SIGMA0 ** 2))
    for k in (3, 4, 5):
        r, w, _e = gb.gauss_fit_kernel(g, k)
        p, _c, w0, _e0 = gb.gauss_fit_sigma0(k)
        assert r == list(p)
        np.testing.assert_allclose(w, w0, rtol=1e-12)


def test_library_kernel_fit_recovers_staircase(gb):
    half = np.zeros(70)
    for r, wi in zip([2, 9, 33, 64], [0.4, -0.1, 0.25, 0.05]):
        half[:r + 1] += wi
    for err in (0, 1):
        r, w, e = gb.gauss_fit_kernel(half, 4, err)
        assert r == [2, 9, 33, 64]
        np.testing.assert_allclose(w, [0.4, -0.1, 0.25, 0.05], rtol=1e-9, atol=1e-12)
        assert abs(e) < 1e-10


def test_library_kernel_fit_argument_errors(gb):
    from paper_1107_4958_gb300.gaussbox import GaussboxError
    with pytest.raises(GaussboxError):
        gb.gauss_fit_kernel(np.ones(102), 3)           # more than t = 0..100
    with pytest.raises(GaussboxError):
        gb.gauss_fit_kernel([], 3)
    with pytest.raises(GaussboxError):
        gb.gauss_fit_kernel(np.ones(10), 6)
    with pytest.raises(GaussboxError):
        gb.gauss_fit_kernel([1.0, float("nan")], 2)


def test_sampled_and_volume_argument_errors_before_any_device_work(gb):
    from paper_1107_4958_gb300 import abi_types as T
    L = gb.lib()
    base = 1 << 20
    r = (ctypes.c_int32 * 2)(1, 3)
    w = (ctypes.c_double * 2)(0.1, 0.05)

    def sampled(sy=2, sx=2, oy=0, ox=0, H=16, W=16, out_pitch=32):
        return L.gauss_filter_sampled(ctypes.c_void_p(base), 64, ctypes.c_void_p(base * 4), out_pitch, H, W, 1,
                                      T.GF_F32, T.GF_F32, r, w, 2, 0, sy, sx, oy, ox, None, None)

    assert sampled(sy=0) == T.GF_EINVAL
    assert sampled(sx=-1) == T.GF_EINVAL
    assert sampled(oy=2) == T.GF_EINVAL                   # offset >= step
    assert sampled(ox=-1) == T.GF_EINVAL
    assert sampled(sy=20, oy=17) == T.GF_EINVAL           # offset beyond the image
    assert sampled(out_pitch=28) == T.GF_EINVAL           # pitch below Wo = 8 floats
    # no handle, no volume; no batch either
    rz = ctypes.POINTER(ctypes.c_int32)()
    wz = ctypes.POINTER(ctypes.c_double)()
    assert L.gauss_filter_volume(None, ctypes.c_void_p(base), 64, ctypes.c_void_p(base * 4), 64, 4, 16, 16, 1,
                                 T.GF_F32, T.GF_F32, r, w, 2, rz, wz, 0, 0, None) == T.GF_EINVAL
    assert L.gauss_filter_batch(None, None, 0, None) == T.GF_EINVAL


def test_run_time_kernels_compile_without_a_device(gb):
    # the kernels compiled at run time (NVRTC) for each radius set: the 2D
    # register walk (single images and stacks of slices) and the volumes'
    # depth walk, at the smallest and largest radii each takes
    from paper_1107_4958_gb300.abi_types import GF_EUNSUPPORTED, GF_F32, GF_U8, GF_U16
    for dt, radii in ((GF_U8, [0]), (GF_U8, [4, 9, 14, 20]), (GF_U16, [1, 3, 6, 10, 22])):
        st, log = gb.gauss_walker_compile(dt, radii)
        assert st == 0, (dt, radii, log)
    assert gb.gauss_walker_compile(GF_U8, [4, 23])[0] == GF_EUNSUPPORTED
    assert gb.gauss_walker_compile(GF_F32, [4, 9])[0] == GF_EUNSUPPORTED
    for radii in ([0], [2, 5, 9], [1, 3, 5, 8, 10]):
        st, log = gb.gauss_depth_walker_compile(radii)
        assert st == 0, (radii, log)
    assert gb.gauss_depth_walker_compile([3, 11])[0] == GF_EUNSUPPORTED
