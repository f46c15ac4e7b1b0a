"""GPU parity at the limits of the interface: the largest radius (4096, folded
many times over a small image), single rows and columns millions of pixels
long, the full uint16 range, and images whose byte offsets pass 2^31 on both
paths (sampled output rows checked against the oracle one by one)."""
import numpy as np
import pytest

from gpu_helpers import TOL, rel_err, to_device, to_host
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import BOUNDARY_CODE, GF_PATH_FUSED, GF_PATH_TWO_PASS

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


def run(gb, x, r, w, boundary, plan=None):
    import torch
    y = gb.filter_tensor(x, radii=r, weights=w, boundary=BOUNDARY_CODE[boundary], out_dtype=torch.float32,
                         plan=plan)
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
def test_largest_radius(gb, boundary):
    # radius 380: the column rings of 2 r + 1 running sums, high and low parts
    # (32-column strips), nearly fill the 227 KB of shared memory a CTA may
    # hold; the radii fold many times over the 40 x 300 image
    from paper_1107_4958_gb300.abi_types import GF_PATH_TWO_PASS
    f = synth.image(40, 300, seed=61, dtype="f32")
    r = [150, 300, 380]
    w = np.array([0.5, 0.3, 0.2])
    w = w / np.sum(w * (2 * np.array(r) + 1))
    got = to_host(run(gb, to_device(f, "f32"), r, w, boundary, plan=gb.make_plan(GF_PATH_TWO_PASS)))
    ref = of.filter_separable(f.astype(np.float64), r, np.float32(w).astype(np.float64), boundary)
    assert rel_err(got, ref) <= TOL["f32"]


@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
@pytest.mark.parametrize("in_name,C", [("f32", 1), ("u8", 3), ("bf16", 2), ("u16", 1)])
def test_radius_4096_running_sums_in_hbm(gb, boundary, in_name, C):
    # beyond the shared-memory column ring the default plan keeps the running
    # sums in HBM (any radius); radii fold many times over the image
    f = synth.image(37, 301, seed=65, dtype="u8" if in_name in ("u8", "u16") else "f32", c=C)
    if in_name == "u16":
        f = f.astype(np.uint16) * 257
    r = [0, 777, 4096]
    w = np.array([0.5, 0.3, 0.2])
    w = w / np.sum(w * (2 * np.array(r) + 1))
    x = to_device(f, in_name)
    got = to_host(run(gb, x, r, w, boundary))
    from gpu_helpers import oracle_input
    ref = of.filter_separable(oracle_input(f, in_name), r, np.float32(w).astype(np.float64), boundary)
    assert rel_err(got, ref) <= TOL["f32"]


def test_radius_beyond_the_column_ring_sampled_and_half_output(gb):
    import torch
    from gpu_helpers import oracle_input
    f = synth.image(120, 90, seed=66, dtype="f32")
    r = [5, 1500]
    w = np.array([0.02, 0.0003])
    x = to_device(f, "f32")
    y = gb.filter_sampled_tensor(x, (3, 2), (1, 1), radii=r, weights=w, out_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    ref = of.filter_sampled(oracle_input(f, "f32"), r, np.float32(w).astype(np.float64), "replicate", (3, 2),
                            (1, 1))
    assert rel_err(to_host(y), ref) <= TOL["bf16"]


def test_radius_beyond_the_column_ring_explicit_two_pass_refused(gb):
    import torch
    from paper_1107_4958_gb300.abi_types import GF_EUNSUPPORTED
    x = torch.zeros((40, 300), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    for rk in (1000, 4096):
        with pytest.raises(gb.GaussboxError) as e:
            gb.filter_tensor(x, radii=[10, rk], weights=[1e-3, 1e-4], out=y, plan=gb.make_plan(GF_PATH_TWO_PASS))
        assert e.value.status == GF_EUNSUPPORTED


@pytest.mark.parametrize("shape", [(1, 2_000_003), (2_000_003, 1), (3, 700_001)])
def test_very_long_rows_and_columns(gb, shape):
    f = np.tile(synth.image(64, 64, seed=62, dtype="u8").ravel(), shape[0] * shape[1] // 4096 + 1)
    f = f[:shape[0] * shape[1]].reshape(shape)
    r, w = ofit.fit_gaussian_boxes(3.0, 4)
    for path in (GF_PATH_FUSED, GF_PATH_TWO_PASS):
        got = to_host(run(gb, to_device(f, "u8"), r, w, "reflect", gb.make_plan(path)))
        ref = of.filter_separable(f.astype(np.float64), r, np.float32(w).astype(np.float64), "reflect")
        assert rel_err(got, ref) <= TOL["f32"], path


def test_full_uint16_range(gb):
    rng = np.random.default_rng(63)
    f = rng.integers(0, 65536, (300, 500)).astype(np.uint16)
    f[:, :50] = 65535
    for sigma, K in ((2.0, 3), (50.0, 5)):
        r, w = ofit.fit_gaussian_boxes(sigma, K)
        got = to_host(run(gb, to_device(f, "u16"), r, w, "replicate"))
        ref = of.filter_separable(f.astype(np.float64), r, np.float32(w).astype(np.float64), "replicate")
        assert rel_err(got, ref) <= TOL["f32"], sigma


@pytest.mark.parametrize("path", [GF_PATH_FUSED, GF_PATH_TWO_PASS])
def test_output_offsets_past_2_31_bytes(gb, path):
    # 24000 x 24000 u8 -> f32: the output is 2.3 GB, rows near the end lie past
    # 2^31 bytes (and so does the two-pass intermediate)
    import torch
    N = 24000
    tile = synth.image(1000, 1000, seed=64, dtype="u8")
    f = np.tile(tile, (N // 1000, N // 1000))
    f[N - 7:, :] = 255 - f[N - 7:, :]          # rows at the end differ from the tiling
    r, w = ofit.fit_gaussian_boxes(8.0, 4)
    x = to_device(f, "u8")
    y = run(gb, x, r, w, "replicate", gb.make_plan(path))
    ys = [0, 12345, N - 30, N - 4, N - 1]
    got = y[ys].to(torch.float64).cpu().numpy()
    del y, x
    torch.cuda.empty_cache()
    ref = of.filter_rows_at(f, r, np.float32(w).astype(np.float64), "replicate", ys)
    assert rel_err(got, ref) <= TOL["f32"]


def test_plans_beyond_the_grid_limit_are_rejected(gb):
    # 70000 rows in row tiles of 1 (fused) or column tiles of 1 (two-pass) would
    # need more than 65535 CTAs down the image: refused before any launch
    import torch
    from paper_1107_4958_gb300.abi_types import GF_EINVAL
    x = torch.zeros((70000, 8), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    for plan in (gb.make_plan(GF_PATH_FUSED, tile_h=1), gb.make_plan(GF_PATH_TWO_PASS, col_h=1)):
        with pytest.raises(gb.GaussboxError) as e:
            gb.filter_tensor(x, radii=[1], weights=[1 / 3], out=y, plan=plan)
        assert e.value.status == GF_EINVAL
    # the default plans of the same image run
    gb.filter_tensor(x, radii=[1], weights=[1 / 3], out=y)
    torch.cuda.synchronize()


@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
@pytest.mark.parametrize("in_name,C,sigma", [("u8", 1, 2.0), ("f32", 3, 8.0), ("bf16", 1, 5.0), ("u16", 2, 3.0)])
def test_hbm_path_at_ordinary_radii(gb, boundary, in_name, C, sigma):
    # the running sums in HBM, forced by the plan, against the oracle
    from paper_1107_4958_gb300.abi_types import GF_PATH_HBM
    from gpu_helpers import oracle_input
    f = synth.image(97, 211, seed=67, dtype="u8" if in_name in ("u8", "u16") else "f32", c=C)
    if in_name == "u16":
        f = f.astype(np.uint16) * 257
    r, w = ofit.fit_gaussian_boxes(sigma, 4)
    got = to_host(run(gb, to_device(f, in_name), r, w, boundary, gb.make_plan(GF_PATH_HBM)))
    ref = of.filter_separable(oracle_input(f, in_name), r, np.float32(w).astype(np.float64), boundary)
    assert rel_err(got, ref) <= TOL["f32"]


def test_hbm_path_sampled_grid(gb):
    import torch
    from paper_1107_4958_gb300.abi_types import GF_PATH_HBM
    f = synth.image(130, 170, seed=68, dtype="f32", c=2)
    r, w = ofit.fit_gaussian_boxes(6.0, 5)
    y = gb.filter_sampled_tensor(to_device(f, "f32"), (3, 4), (2, 1), radii=r, weights=w, boundary=2,
                                 plan=gb.make_plan(GF_PATH_HBM))
    torch.cuda.synchronize()
    ref = of.filter_sampled(f.astype(np.float64), r, np.float32(w).astype(np.float64), "reflect", (3, 4), (2, 1))
    assert rel_err(to_host(y), ref) <= TOL["f32"]


def test_default_plan_names_the_hbm_path_beyond_the_ring(gb):
    from paper_1107_4958_gb300.abi_types import GF_F32, GF_PATH_HBM, GF_PATH_TWO_PASS, GF_U8
    assert gb.gauss_plan_default(4096, 4096, 1, GF_U8, GF_F32, [150, 300, 380]).as_dict()["path"] == GF_PATH_TWO_PASS
    p = gb.gauss_plan_default(4096, 4096, 1, GF_U8, GF_F32, [10, 1030]).as_dict()
    assert p["path"] == GF_PATH_HBM and p["tile_w"] == 0 and p["col_w"] == 0


def test_hbm_path_refused_by_batches_and_volumes(gb):
    import torch
    from paper_1107_4958_gb300.abi_types import GF_EUNSUPPORTED, GF_PATH_HBM
    x = torch.zeros((40, 300), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    h = gb.gf_create()
    try:
        for desc in (gb.image_desc(x, y, radii=[10, 1500], weights=[1e-3, 1e-4]),
                     gb.image_desc(x, y, radii=[1, 2], weights=[0.1, 0.1], plan=gb.make_plan(GF_PATH_HBM))):
            with pytest.raises(gb.GaussboxError) as e:
                gb.gauss_filter_batch(h, [desc])
            assert e.value.status == GF_EUNSUPPORTED
        v = torch.zeros((3, 40, 30), dtype=torch.float32, device="cuda")
        with pytest.raises(gb.GaussboxError) as e:
            gb.filter_volume_tensor(h, v, radii=[10, 1500], weights=[1e-3, 1e-4])
        assert e.value.status == GF_EUNSUPPORTED
    finally:
        gb.gf_destroy(h)
