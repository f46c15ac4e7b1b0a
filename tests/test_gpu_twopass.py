"""GPU parity of the two-pass form (row launch -> FP32 intermediate -> column
launch) against the FP64 oracle, both execution paths against each other, and
the plan interface of the C ABI.

Cases are chosen so that every tile dimension has several tiles and a ragged
tail (segment width, rows per CTA, column strip width and height are forced
through explicit plans), and so that the first output element of a row
segment falls on every residue modulo C (3 channels)."""
import numpy as np
import pytest

from gpu_helpers import TOL, oracle_input, rel_err, to_device, to_host, torch_dtype
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import (BOUNDARY_CODE, GF_EINVAL, GF_EUNSUPPORTED, GF_PATH_AUTO,
                                             GF_PATH_FUSED, GF_PATH_TWO_PASS, GF_PATH_WALK)

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


def run(gb, arr, in_name, radii, weights, boundary, plan, out_name=None, pad=0):
    import torch
    x = to_device(arr, in_name, pad)
    od = torch_dtype(out_name) if out_name else None
    y = gb.filter_tensor(x, radii=radii, weights=weights, boundary=BOUNDARY_CODE[boundary], out_dtype=od,
                         plan=plan)
    torch.cuda.synchronize()
    return to_host(y)


def oracle(arr, in_name, radii, weights, boundary):
    return of.filter_separable(oracle_input(arr, in_name), radii, np.float32(weights).astype(np.float64),
                               boundary)


@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
@pytest.mark.parametrize("in_name", ["u8", "f32", "bf16"])
@pytest.mark.parametrize("sigma,K", [(1.5, 3), (6.0, 4), (21.0, 5)])
def test_two_pass_vs_oracle(gb, boundary, in_name, sigma, K):
    f = synth.image(97, 211, seed=31, dtype="u8" if in_name == "u8" else "f32")
    r, w = ofit.fit_gaussian_boxes(sigma, K)
    ref = oracle(f, in_name, r, w, boundary)
    for cw in (32, 64, 128, 256):
        plan = gb.make_plan(GF_PATH_TWO_PASS, tile_w=70, tile_h=16, col_w=cw, col_h=23)
        if cw == 256 and max(r) > 39:
            # the hi and lo column rings of 256 columns and 2 r + 17 rows exceed
            # one CTA's shared memory beyond radius 39: refused, not truncated
            with pytest.raises(gb.GaussboxError) as ei:
                run(gb, f, in_name, r, w, boundary, plan, out_name="f32")
            assert ei.value.status == GF_EUNSUPPORTED
            continue
        got = run(gb, f, in_name, r, w, boundary, plan, out_name="f32")
        assert rel_err(got, ref) <= TOL["f32"], (cw, rel_err(got, ref))


@pytest.mark.parametrize("path", [GF_PATH_FUSED, GF_PATH_TWO_PASS])
@pytest.mark.parametrize("in_name", ["f32", "bf16"])
def test_three_channels_every_residue(gb, path, in_name):
    # float rows with a large DC: a per-channel offset taken from the wrong
    # channel shows up at once.  Radii 1..12 put the first staged element at
    # every offset modulo 3.
    f = synth.image(40, 150, seed=32, dtype="f32", c=3)
    f[..., 1] += 600.0
    f[..., 2] -= 300.0
    for rk in range(1, 13):
        r, w = [0, rk // 2, rk], [0.05, 0.03, 0.02]
        tw = 0 if path == GF_PATH_FUSED else 37
        got = run(gb, f, in_name, r, w, "replicate", gb.make_plan(path, tile_w=tw), out_name="f32")
        ref = oracle(f, in_name, r, w, "replicate")
        assert rel_err(got, ref) <= TOL["f32"], (rk, rel_err(got, ref))


@pytest.mark.parametrize("C", [1, 2, 3, 4])
def test_two_pass_channels_and_pitch(gb, C):
    f = synth.image(61, 130, seed=33, dtype="f32", c=C)
    r, w = ofit.fit_gaussian_boxes(9.0, 4)
    ref = oracle(f, "f32", r, w, "reflect")
    got = run(gb, f, "f32", r, w, "reflect", gb.make_plan(GF_PATH_TWO_PASS), pad=5)
    assert rel_err(got, ref) <= TOL["f32"]


def test_two_pass_radius_larger_than_image(gb):
    f = synth.image(33, 45, seed=34, dtype="f32")
    r, w = ofit.fit_gaussian_boxes(40.0, 5)
    for boundary in ("replicate", "zero", "reflect"):
        got = run(gb, f, "f32", r, w, boundary, gb.make_plan(GF_PATH_TWO_PASS, col_w=32))
        ref = oracle(f, "f32", r, w, boundary)
        assert rel_err(got, ref) <= TOL["f32"], boundary


@pytest.mark.parametrize("out_name", ["f32", "bf16", "f16"])
def test_two_pass_output_types(gb, out_name):
    f = synth.image(80, 300, seed=35, dtype="f32")
    r, w = ofit.fit_gaussian_boxes(12.0, 4)
    ref = oracle(f, "f32", r, w, "replicate")
    got = run(gb, f, "f32", r, w, "replicate", gb.make_plan(GF_PATH_TWO_PASS), out_name=out_name)
    assert rel_err(got, ref) <= TOL[out_name]


def test_paths_agree_on_u8(gb):
    # both paths see exact integer row sums; they may differ only in the FP32
    # rounding of the weighted sums and the column pass
    f = synth.image(300, 517, seed=36, dtype="u8")
    for sigma in (2.0, 8.0, 32.0):
        r, w = ofit.fit_gaussian_boxes(sigma, 4)
        a = run(gb, f, "u8", r, w, "replicate", gb.make_plan(GF_PATH_FUSED))
        b = run(gb, f, "u8", r, w, "replicate", gb.make_plan(GF_PATH_TWO_PASS))
        ref = oracle(f, "u8", r, w, "replicate")
        assert rel_err(a, ref) <= TOL["f32"] and rel_err(b, ref) <= TOL["f32"]
        assert rel_err(a, b) <= 2 * TOL["f32"]


@pytest.mark.parametrize("sigma", [8.0, 32.0])
def test_two_pass_4096_u8_sampled_rows(gb, sigma):
    f = synth.image(4096, 4096, seed=2, dtype="u8")
    r, w = ofit.fit_gaussian_boxes(sigma, 4)
    got = run(gb, f, "u8", r, w, "replicate", gb.make_plan(GF_PATH_TWO_PASS))
    ys = [0, 1, 5, 333, 2047, 2048, 4001, 4095]
    ref = of.filter_rows_at(f.astype(np.float64), r, np.float32(w).astype(np.float64), "replicate", ys)
    assert rel_err(got[ys], ref) <= TOL["f32"]


def test_default_plan_is_complete(gb):
    from paper_1107_4958_gb300.abi_types import GF_F32, GF_U8
    for (H, W, C, sigma, K) in ((4096, 4096, 1, 8.0, 4), (512, 512, 1, 5.0, 3), (2000, 3000, 3, 50.0, 5),
                                (8192, 8192, 1, 100.0, 5)):
        r, _ = ofit.fit_gaussian_boxes(sigma, K)
        p = gb.gauss_plan_default(H, W, C, GF_U8 if C == 1 else GF_F32, GF_F32, r).as_dict()
        if p["path"] == GF_PATH_WALK:        # the register walk has no tile parameters
            assert C == 1 and max(r) <= 22
            continue
        assert p["path"] in (GF_PATH_FUSED, GF_PATH_TWO_PASS)
        assert p["tile_w"] >= 1 and p["tile_h"] >= 1
        if p["path"] == GF_PATH_TWO_PASS:
            assert p["col_w"] in (32, 64, 128, 256) and p["col_h"] >= 1


def test_auto_plan_matches_oracle_large_sigma(gb):
    f = synth.image(700, 900, seed=37, dtype="f32", c=3)
    r, w = ofit.fit_gaussian_boxes(50.0, 5)
    got = run(gb, f, "f32", r, w, "replicate", gb.make_plan(GF_PATH_AUTO))
    ref = oracle(f, "f32", r, w, "replicate")
    assert rel_err(got, ref) <= TOL["f32"]


def test_bad_plans_rejected(gb):
    import torch
    x = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    for plan in (gb.make_plan(7), gb.make_plan(GF_PATH_TWO_PASS, col_w=48),
                 gb.make_plan(GF_PATH_FUSED, tile_w=300), gb.make_plan(GF_PATH_TWO_PASS, tile_h=-1)):
        with pytest.raises(gb.GaussboxError) as e:
            gb.filter_tensor(x, radii=[1, 2], weights=[0.1, 0.1], out=y, plan=plan)
        assert e.value.status == GF_EINVAL
