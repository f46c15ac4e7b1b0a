"""GPU parity of the sampled-output filter (gauss_filter_sampled: Eq. indep at
a regular grid of pixels only, Sec. 3.4) against the FP64 oracle, bit-identity
with the full filter's pixels under the same two-pass plan, edge grids, a full
4096 x 4096 case on sampled rows, and argument errors."""
import numpy as np
import pytest

from gpu_helpers import TOL, oracle_input, rel_err, to_device, to_host, torch_dtype
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import BOUNDARY_CODE, GF_EINVAL, GF_EUNSUPPORTED, GF_PATH_FUSED, GF_PATH_TWO_PASS

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


def sampled(gb, arr, in_name, r, w, boundary, step, offset, plan=None, out_name="f32", pad=0):
    import torch
    x = to_device(arr, in_name, pad)
    y = gb.filter_sampled_tensor(x, step, offset, radii=r, weights=w, boundary=BOUNDARY_CODE[boundary],
                                 out_dtype=torch_dtype(out_name), plan=plan)
    torch.cuda.synchronize()
    return to_host(y)


def oracle(arr, in_name, r, w, boundary, step, offset):
    return of.filter_sampled(oracle_input(arr, in_name), r, np.float32(w).astype(np.float64), boundary, step,
                             offset)


@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
@pytest.mark.parametrize("in_name", ["u8", "f32", "bf16"])
@pytest.mark.parametrize("sigma,K", [(1.5, 3), (6.0, 4), (21.0, 5)])
def test_sampled_vs_oracle(gb, boundary, in_name, sigma, K):
    f = synth.image(97, 211, seed=41, dtype="u8" if in_name == "u8" else "f32")
    r, w = ofit.fit_gaussian_boxes(sigma, K)
    for step, offset in (((2, 2), (0, 0)), ((3, 5), (2, 4)), ((1, 3), (0, 1)), ((4, 1), (3, 0))):
        # several row segments, column strips and column tiles, ragged tails
        plan = gb.make_plan(GF_PATH_TWO_PASS, tile_w=70, tile_h=16, col_w=32, col_h=23)
        got = sampled(gb, f, in_name, r, w, boundary, step, offset, plan)
        ref = oracle(f, in_name, r, w, boundary, step, offset)
        assert got.shape == ref.shape
        assert rel_err(got, ref) <= TOL["f32"], (step, offset, rel_err(got, ref))


@pytest.mark.parametrize("C", [1, 2, 3, 4])
def test_sampled_channels_and_pitch(gb, C):
    f = synth.image(61, 130, seed=42, dtype="f32", c=C)
    f[..., 0] += 500.0        # a per-channel offset taken from the wrong channel shows at once
    r, w = ofit.fit_gaussian_boxes(5.0, 4)
    for step, offset in (((2, 3), (1, 2)), ((5, 2), (0, 1))):
        got = sampled(gb, f, "f32", r, w, "reflect", step, offset, pad=5)
        ref = oracle(f, "f32", r, w, "reflect", step, offset)
        assert rel_err(got, ref) <= TOL["f32"], (step, offset)


@pytest.mark.parametrize("cw", [32, 64, 128, 256])
def test_sampled_equals_full_filter_pixels_bitwise(gb, cw):
    # same plan: same row segments, column strips and tiles, so every sampled
    # value is computed by the same operations as the full filter's pixel
    import torch
    f = synth.image(150, 301, seed=43, dtype="u8", c=3)
    r, w = ofit.fit_gaussian_boxes(7.0, 4)
    plan = gb.make_plan(GF_PATH_TWO_PASS, tile_w=90, tile_h=24, col_w=cw, col_h=37)
    x = to_device(f, "u8")
    full = gb.filter_tensor(x, radii=r, weights=w, plan=plan)
    for step, offset in (((2, 2), (0, 1)), ((3, 7), (2, 6)), ((1, 2), (0, 0))):
        y = gb.filter_sampled_tensor(x, step, offset, radii=r, weights=w, plan=plan)
        torch.cuda.synchronize()
        want = full[offset[0]::step[0], offset[1]::step[1]]
        assert torch.equal(y, want), (cw, step, offset)


def test_sampled_edge_grids(gb):
    f = synth.image(33, 45, seed=44, dtype="f32")
    r, w = ofit.fit_gaussian_boxes(40.0, 5)     # radii larger than the image
    for boundary in ("replicate", "zero", "reflect"):
        for step, offset in (((33, 45), (32, 44)), ((100, 100), (0, 0)), ((1, 1), (0, 0)), ((2, 50), (1, 44))):
            got = sampled(gb, f, "f32", r, w, boundary, step, offset)
            ref = oracle(f, "f32", r, w, boundary, step, offset)
            assert got.shape == ref.shape
            assert rel_err(got, ref) <= TOL["f32"], (boundary, step, offset)


@pytest.mark.parametrize("out_name", ["bf16", "f16"])
def test_sampled_half_outputs(gb, out_name):
    f = synth.image(80, 300, seed=45, dtype="f32")
    r, w = ofit.fit_gaussian_boxes(3.0, 3)
    got = sampled(gb, f, "f32", r, w, "replicate", (2, 2), (1, 1), out_name=out_name)
    ref = oracle(f, "f32", r, w, "replicate", (2, 2), (1, 1))
    assert rel_err(got, ref) <= TOL[out_name]


@pytest.mark.parametrize("sigma", [2.0, 8.0])
def test_sampled_4096_u8_rows(gb, sigma):
    # the full-size image on its default plan; oracle rows one by one
    f = synth.image(4096, 4096, seed=2, dtype="u8")
    r, w = ofit.fit_gaussian_boxes(sigma, 4)
    got = sampled(gb, f, "u8", r, w, "replicate", (2, 2), (0, 0))
    assert got.shape == (2048, 2048)
    idx = [0, 1, 2, 700, 1023, 1024, 2000, 2047]
    ref = of.filter_rows_at(f.astype(np.float64), r, np.float32(w).astype(np.float64), "replicate",
                            [2 * i for i in idx])[:, 0::2]
    assert rel_err(got[idx], ref) <= TOL["f32"]


def test_sampled_argument_errors(gb):
    import torch
    x = torch.zeros((16, 20), dtype=torch.float32, device="cuda")
    y = torch.empty((8, 10), dtype=torch.float32, device="cuda")
    r, w = [1, 2], [0.1, 0.1]
    with pytest.raises(gb.GaussboxError) as e:
        gb.filter_sampled_tensor(x, (2, 2), radii=r, weights=w, out=y, plan=gb.make_plan(GF_PATH_FUSED))
    assert e.value.status == GF_EUNSUPPORTED
    for step, offset in (((2, 2), (2, 0)), ((0, 2), (0, 0)), ((2, 2), (0, -1))):
        with pytest.raises(gb.GaussboxError) as e:
            gb.gauss_filter_sampled(x.data_ptr(), 80, y.data_ptr(), 40, 16, 20, 1, 2, 2, r, w, 0, step[0], step[1],
                                    offset[0], offset[1], None, 0)
        assert e.value.status == GF_EINVAL
    with pytest.raises(gb.GaussboxError) as e:   # output pitch below Wo = 10 elements
        gb.gauss_filter_sampled(x.data_ptr(), 80, y.data_ptr(), 36, 16, 20, 1, 2, 2, r, w, 0, 2, 2, 0, 0, None, 0)
    assert e.value.status == GF_EINVAL
