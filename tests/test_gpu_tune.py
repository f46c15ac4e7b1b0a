"""GPU: the plan autotuner (gf_tune).  The tuned plan is a complete, valid
plan; images of the tuned class then run on it in batches and on the server,
bit-identical to gauss_filter_planned with the same plan; the cache file
round-trips through a new handle."""
import os

import numpy as np
import pytest

from gpu_helpers import TOL, rel_err, to_device, to_host
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import GF_PATH_FUSED, GF_PATH_TWO_PASS

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


def _img(H, W, C, sigma, K, seed=60):
    import torch
    x = to_device(synth.image(H, W, seed=seed, dtype="f32", c=C), "f32")
    y = torch.empty_like(x)
    return x, y, sigma, K


@pytest.mark.parametrize("H,W,C,sigma,K", [(700, 900, 3, 6.0, 4), (600, 640, 1, 40.0, 5)])
def test_tuned_plan_valid_and_used_by_batch(gb, tmp_path, H, W, C, sigma, K):
    import torch
    cache = str(tmp_path / "tune.json")
    h = gb.gf_create(tune_cache=cache)
    try:
        x, y, s, k = _img(H, W, C, sigma, K)
        d = gb.image_desc(x, y, s, k)
        p = gb.gf_tune(h, d, torch.cuda.current_stream().cuda_stream)
        assert p.path in (GF_PATH_FUSED, GF_PATH_TWO_PASS) and p.tile_w >= 1 and p.tile_h >= 1
        if p.path == GF_PATH_TWO_PASS:
            assert p.col_w in (32, 64, 128, 256)
        assert gb.gf_tuned_plan(h, d).as_dict() == p.as_dict()
        # the batch runs the tuned plan: same bits as the planned single call
        yb = torch.empty_like(x)
        gb.gauss_filter_batch(h, [gb.image_desc(x, yb, s, k)], torch.cuda.current_stream().cuda_stream)
        ya = gb.filter_tensor(x, sigma=s, K=k, out=torch.empty_like(x), plan=p)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(yb), to_host(ya))
        r, w = ofit.fit_gaussian_boxes(s, k)
        ref = of.filter_separable(to_host(x), r, np.float32(w).astype(np.float64), "replicate")
        assert rel_err(to_host(yb), ref) <= TOL["f32"]
    finally:
        gb.gf_destroy(h)
    # the cache file reloads into a new handle
    assert os.path.exists(cache)
    h2 = gb.gf_create(tune_cache=cache)
    try:
        assert gb.gf_tuned_plan(h2, d).as_dict() == p.as_dict()
    finally:
        gb.gf_destroy(h2)


def test_untuned_class_has_no_plan(gb):
    h = gb.gf_create()
    try:
        x, y, s, k = _img(64, 64, 1, 2.0, 3)
        assert gb.gf_tuned_plan(h, gb.image_desc(x, y, s, k)) is None
    finally:
        gb.gf_destroy(h)


def test_tuner_falls_back_to_hbm_running_sums_beyond_the_ring(gb):
    # a radius no shared-memory plan can hold: the tuner times the HBM path
    import torch
    from paper_1107_4958_gb300.abi_types import GF_PATH_HBM
    h = gb.gf_create()
    try:
        x = to_device(synth.image(200, 300, seed=61, dtype="f32"), "f32")
        y = torch.empty_like(x)
        d = gb.image_desc(x, y, radii=[3, 1200], weights=[0.05, 1e-4])
        p = gb.gf_tune(h, d, torch.cuda.current_stream().cuda_stream)
        assert p.path == GF_PATH_HBM
    finally:
        gb.gf_destroy(h)
