"""GPU parity on inputs without the smoothness of natural images: white
noise, ramps across whole tiles and large DC offsets, at small sigma (where
the smallest box holds one to a few pixels), on both paths with default and
long tiles.  These are the inputs for which running sums kept in FP32 lose
accuracy with the tile length; the kernels' integer row sums and bounded
column tiles keep the 1e-5 bound."""
import numpy as np
import pytest

from gpu_helpers import TOL, oracle_input, rel_err, to_device, to_host, torch_dtype
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300.abi_types import BOUNDARY_CODE, GF_PATH_AUTO, GF_PATH_FUSED, GF_PATH_TWO_PASS

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


def noise(shape, seed, kind):
    rng = np.random.default_rng(seed)
    if kind == "white":
        return rng.uniform(0.0, 255.0, shape).astype(np.float32)
    if kind == "white+1e4":
        return (rng.uniform(0.0, 255.0, shape) + 1.0e4).astype(np.float32)
    if kind == "ramp":                     # 0 -> 255 along rows and columns, plus noise
        h, w = shape[:2]
        r = np.add.outer(np.linspace(0, 127.5, h), np.linspace(0, 127.5, w))
        return (r + rng.uniform(-8, 8, shape)).astype(np.float32)
    raise ValueError(kind)


def check(gb, f, in_name, r, w, boundary, plan):
    import torch
    x = to_device(f, in_name)
    y = gb.filter_tensor(x, radii=r, weights=w, boundary=BOUNDARY_CODE[boundary], out_dtype=torch.float32,
                         plan=plan)
    torch.cuda.synchronize()
    ref = of.filter_separable(oracle_input(f, in_name), r, np.float32(w).astype(np.float64), boundary)
    return rel_err(to_host(y), ref)


@pytest.mark.parametrize("kind", ["white", "white+1e4", "ramp"])
@pytest.mark.parametrize("sigma,K", [(0.5, 3), (1.0, 4), (2.0, 4), (3.0, 5), (8.0, 4)])
def test_noise_default_plans(gb, kind, sigma, K):
    f = noise((700, 2300), 71, kind)
    r, w = ofit.fit_gaussian_boxes(sigma, K)
    for path in (GF_PATH_AUTO, GF_PATH_FUSED, GF_PATH_TWO_PASS):
        e = check(gb, f, "f32", r, w, "reflect", gb.make_plan(path))
        assert e <= TOL["f32"], (path, e)


@pytest.mark.parametrize("kind", ["white", "ramp"])
def test_noise_longest_row_segments(gb, kind):
    # two-pass row segments of 2048 pixels: one running sum over > 2 K staged values
    f = noise((64, 9000), 72, kind)
    for sigma, K in ((0.5, 3), (1.0, 5)):
        r, w = ofit.fit_gaussian_boxes(sigma, K)
        e = check(gb, f, "f32", r, w, "replicate", gb.make_plan(GF_PATH_TWO_PASS, tile_w=2048))
        assert e <= TOL["f32"], (sigma, e)


@pytest.mark.parametrize("in_name", ["f32", "bf16", "u8"])
def test_noise_single_tall_column(gb, in_name):
    # one column of 200 000 pixels: the default column tiles stay short enough
    f = noise((200_000, 1), 73, "white")
    if in_name == "u8":
        f = np.rint(f).astype(np.uint8)
    r, w = ofit.fit_gaussian_boxes(3.0, 4)
    for path in (GF_PATH_FUSED, GF_PATH_TWO_PASS):
        e = check(gb, f, in_name, r, w, "reflect", gb.make_plan(path))
        assert e <= TOL["f32"], (path, e)


def test_noise_three_channels(gb):
    f = noise((300, 900, 3), 74, "white")
    f[..., 1] += 5000.0
    r, w = ofit.fit_gaussian_boxes(1.0, 3)
    for path in (GF_PATH_FUSED, GF_PATH_TWO_PASS):
        e = check(gb, f, "f32", r, w, "zero", gb.make_plan(path))
        assert e <= TOL["f32"], (path, e)
