"""GPU parity: the CUDA filter (through the C ABI) against the FP64 oracle, and
the integer row box sums bit-exact against the oracle's int64 sums."""
import os

import numpy as np
import pytest

from gpu_helpers import TOL, oracle_input, rel_err, rms_rel, to_device, to_host
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import BOUNDARY_CODE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4958_gb300 import build
    build.build()
    from paper_1107_4958_gb300 import gaussbox
    gaussbox.gf_get_device_status(clear=True)
    yield gaussbox
    assert gaussbox.gf_get_device_status() == 0


def run_filter(gb, arr, in_name, sigma, K, boundary, out_name=None, pad=0, radii=None, weights=None):
    import torch
    from gpu_helpers import torch_dtype
    x = to_device(arr, in_name, pad)
    od = torch_dtype(out_name) if out_name else None
    y = gb.filter_tensor(x, sigma=sigma, K=K, boundary=BOUNDARY_CODE[boundary], out_dtype=od,
                         radii=radii, weights=weights)
    torch.cuda.synchronize()
    return to_host(y)


def oracle(arr, in_name, sigma, K, boundary):
    r, w = ofit.fit_gaussian_boxes(sigma, K)
    return of.filter_separable(oracle_input(arr, in_name), r, w, boundary)


def test_config1_512_f32_sigma5_k3(gb):
    # 512 x 512 fp32 1/f field, sigma = 5, K = 3 (radii 3, 7, 11), replicate
    f = synth.image(512, 512, seed=1, dtype="f32")
    got = run_filter(gb, f, "f32", 5.0, 3, "replicate")
    ref = oracle(f, "f32", 5.0, 3, "replicate")
    assert rel_err(got, ref) <= TOL["f32"], (rel_err(got, ref), rms_rel(got, ref))


@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (13, 17), (37, 300), (300, 37), (70, 530)])
@pytest.mark.parametrize("in_name", ["u8", "f32"])
def test_shapes_and_boundaries(gb, boundary, shape, in_name):
    f = synth.image(shape[0], shape[1], seed=11, dtype=in_name)
    for sigma, K in ((0.5, 3), (2.0, 4), (8.0, 5)):
        got = run_filter(gb, f, in_name, sigma, K, boundary)
        ref = oracle(f, in_name, sigma, K, boundary)
        assert rel_err(got, ref) <= TOL["f32"], (sigma, K, rel_err(got, ref))


@pytest.mark.parametrize("C", [2, 3, 4])
@pytest.mark.parametrize("boundary", ["replicate", "reflect"])
def test_channels(gb, C, boundary):
    f = synth.image(45, 333, seed=12, dtype="f32", c=C)
    got = run_filter(gb, f, "f32", 3.0, 4, boundary)
    ref = oracle(f, "f32", 3.0, 4, boundary)
    assert rel_err(got, ref) <= TOL["f32"]


@pytest.mark.parametrize("in_name,out_name", [("u16", "f32"), ("bf16", "f32"), ("f16", "f32"),
                                              ("f32", "bf16"), ("f32", "f16"), ("bf16", "bf16"),
                                              ("f16", "f16")])
def test_dtypes(gb, in_name, out_name):
    f = synth.image(130, 270, seed=13, dtype="u16" if in_name == "u16" else "f32")
    got = run_filter(gb, f, in_name, 4.0, 4, "reflect", out_name=out_name)
    ref = oracle(f, in_name, 4.0, 4, "reflect")
    assert rel_err(got, ref) <= TOL[out_name], rel_err(got, ref)


def test_radius_larger_than_image(gb):
    f = synth.image(20, 24, seed=14, dtype="f32")
    for boundary in ("replicate", "zero", "reflect"):
        got = run_filter(gb, f, "f32", 30.0, 5, boundary)     # radii up to 81
        ref = oracle(f, "f32", 30.0, 5, boundary)
        assert rel_err(got, ref) <= TOL["f32"], boundary


def test_constant_image_and_identity(gb):
    f = np.full((64, 96), 77.25, dtype=np.float32)
    got = run_filter(gb, f, "f32", 6.0, 4, "replicate")
    assert np.max(np.abs(got - 77.25)) <= 1e-5 * 77.25
    g = synth.image(33, 47, seed=15, dtype="f32")
    got = run_filter(gb, g, "f32", 0.1, 3, "zero")            # radii all 0: identity
    assert rel_err(got, g) <= TOL["f32"]


def test_pitched_and_unaligned_rows(gb):
    f = synth.image(90, 201, seed=16, dtype="f32")
    ref = oracle(f, "f32", 3.0, 3, "replicate")
    for pad in (3, 16, 35):      # 3: pitch not a multiple of 16 bytes (non-TMA path)
        got = run_filter(gb, f, "f32", 3.0, 3, "replicate", pad=pad)
        assert rel_err(got, ref) <= TOL["f32"], pad


def test_tma_and_plain_staging_agree_bitwise(gb):
    f = synth.image(150, 700, seed=17, dtype="u8")
    a = run_filter(gb, f, "u8", 5.0, 4, "reflect")
    os.environ["GF_NO_TMA"] = "1"
    try:
        b = run_filter(gb, f, "u8", 5.0, 4, "reflect")
    finally:
        del os.environ["GF_NO_TMA"]
    assert np.array_equal(a, b)


def test_explicit_boxes(gb):
    f = synth.image(50, 77, seed=18, dtype="f32")
    radii = [0, 2, 2, 9]
    weights = [0.3, 0.05, 0.02, 0.001]
    got = run_filter(gb, f, "f32", None, None, "reflect", radii=radii, weights=weights)
    ref = of.filter_separable(f.astype(np.float64), radii, np.float32(weights).astype(np.float64), "reflect")
    assert rel_err(got, ref) <= TOL["f32"]


@pytest.mark.parametrize("sigma", [2.0, 8.0, 32.0])
def test_config2_4096_u8_sampled_rows(gb, sigma):
    # 4096 x 4096 uint8 1/f field, K = 4: sampled output rows against the oracle
    f = synth.image(4096, 4096, seed=2, dtype="u8")
    got = run_filter(gb, f, "u8", sigma, 4, "replicate")
    r, w = ofit.fit_gaussian_boxes(sigma, 4)
    ys = [0, 1, 2, 217, 1000, 2048, 4000, 4094, 4095]
    ref = of.filter_rows_at(f.astype(np.float64), r, w, "replicate", ys)
    assert rel_err(got[ys], ref) <= TOL["f32"], rel_err(got[ys], ref)


@pytest.mark.parametrize("in_name", ["u8", "u16"])
@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
def test_row_box_sums_bit_exact(gb, in_name, boundary):
    import torch
    for shape, radii in (((17, 31), [0, 1, 3, 7]), ((5, 700), [2, 9, 14, 20]), ((3, 40), [0, 50, 61, 85]),
                         ((9, 1000, 3), [5, 47, 69, 95, 133])):
        f = synth.image(shape[0], shape[1], seed=19, dtype=in_name, c=shape[2] if len(shape) == 3 else 1)
        x = to_device(f, in_name)
        got = gb.row_box_sums_tensor(x, radii, BOUNDARY_CODE[boundary])
        torch.cuda.synchronize()
        want = of.box_sums_int64(f, radii, boundary, axis=1)
        assert np.array_equal(got.cpu().numpy().astype(np.int64), want), (shape, radii)
