"""Fused-kernel tile shapes around the staged output band (Sec. 3.4 column
pass, one band of 8 output rows leaving by one TMA box).

A tile whose height plus 2 r_K is a multiple of the band height ends on a
whole staged band, which the kernel flushes after its last band behind a CTA
barrier.  Strips narrower than a warp (1 to 24 pixels: a partial warp of
columns) must take that barrier on every thread; these cases run each such
shape on every boundary against the FP64 oracle, next to tiles whose last
band is partial."""
import numpy as np
import pytest

from gpu_helpers import TOL, oracle_input, rel_err, to_device, to_host
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import BOUNDARY_CODE, GF_PATH_FUSED

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


@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
@pytest.mark.parametrize("in_name", ["u8", "f32"])
@pytest.mark.parametrize("twp", [1, 8, 16, 24, 40])
def test_narrow_strips_whole_and_partial_last_band(gb, boundary, in_name, twp):
    import torch
    f = synth.image(203, 336, seed=91, dtype="u8" if in_name == "u8" else "f32")
    x = to_device(f, in_name)
    for sigma, K in ((2.0, 3), (9.0, 4)):
        r, w = ofit.fit_gaussian_boxes(sigma, K)
        rk = int(max(r))
        ref = of.filter_separable(oracle_input(f, in_name), r, np.float32(w).astype(np.float64), boundary)
        whole = 8 * ((40 + 2 * rk) // 8 + 1) - 2 * rk          # (TH + 2 rk) % 8 == 0
        for th in (whole, whole + 3, 2 * whole):
            y = gb.filter_tensor(x, radii=r, weights=w, boundary=BOUNDARY_CODE[boundary], out_dtype=torch.float32,
                                 plan=gb.make_plan(GF_PATH_FUSED, tile_w=twp, tile_h=th))
            torch.cuda.synchronize()
            assert rel_err(to_host(y), ref) <= TOL["f32"], (sigma, th)


def test_sixteen_column_strips_at_radius_106(gb):
    # the shape that first showed the divergent flush: f32, radius 106,
    # 16-column strips and row tiles of 212 rows (a whole last band)
    import torch
    f = synth.image(600, 640, seed=60, dtype="f32")
    r, w = ofit.fit_gaussian_boxes(40.0, 5)
    y = gb.filter_tensor(to_device(f, "f32"), radii=r, weights=w, plan=gb.make_plan(GF_PATH_FUSED, tile_w=16,
                                                                                      tile_h=212))
    torch.cuda.synchronize()
    ys = [0, 1, 211, 212, 300, 423, 424, 599]
    ref = of.filter_rows_at(f.astype(np.float64), r, np.float32(w).astype(np.float64), "replicate", ys)
    assert rel_err(to_host(y)[ys], ref) <= TOL["f32"]
