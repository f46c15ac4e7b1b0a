"""GPU precision study on 8192 x 8192 inputs, sigma = 100, K = 5 (radii up to
267): FP32 running sums of a 1/f field plus a DC offset of 1e4 (and bf16
storage of the field) against the FP64 oracle, on windows at the corners,
the edges and the inside of the image.

Variants (gf_plan.accum, two-pass path):
  default      rows: the integer part of each value on a power-of-two grid
               summed in int32 (exact differences) plus FP32 sums of the
               residues; columns: two-word (hi, lo) running sums, the lo word
               collecting the exact rounding error of every hi addition
  offset       FP32 rows and columns: per-tile offsets, plain FP32 carries
  plain        plain FP32 running sums from the tile start, default tiles
  plain-long   plain FP32 with 2048-pixel row segments and whole columns
Run as a script to print the table of max / RMS errors."""
import os
import sys

if __name__ == "__main__":   # script mode: the paths conftest.py sets up for pytest
    _here = os.path.dirname(os.path.abspath(__file__))
    sys.path[:0] = [os.path.dirname(_here), _here]

import numpy as np
import pytest

from gpu_helpers import TOL, rel_err, rms_rel, to_device, to_host
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import (GF_ACCUM_COMPENSATED, GF_ACCUM_OFFSET, GF_ACCUM_PLAIN,
                                             GF_PATH_AUTO, GF_PATH_TWO_PASS)

pytestmark = pytest.mark.gpu

N = 8192
SIGMA, K = 100.0, 5
WINDOWS = [(0, 48, 0, 48), (0, 48, N - 48, N), (N - 48, N, 0, 48), (N - 48, N, N - 48, N),
           (N // 2 - 24, N // 2 + 24, N // 2 - 24, N // 2 + 24), (1000, 1048, 6000, 6048), (7000, 7048, 333, 381)]
VARIANTS = [("default", dict(path=GF_PATH_AUTO, accum=GF_ACCUM_COMPENSATED)),
            ("offset", dict(path=GF_PATH_TWO_PASS, accum=GF_ACCUM_OFFSET)),
            ("plain", dict(path=GF_PATH_TWO_PASS, accum=GF_ACCUM_PLAIN)),
            ("plain-long", dict(path=GF_PATH_TWO_PASS, accum=GF_ACCUM_PLAIN, tile_w=2048, col_w=32, col_h=N))]


def field(offset):
    # a 4096^2 1/f field tiled 2 x 2 (an 8192^2 FFT would dominate the run time)
    base = synth.image(4096, 4096, seed=4, dtype="f32")
    return (np.tile(base, (2, 2)).astype(np.float64) + offset).astype(np.float32)


def window_errors(y, ref_windows):
    got = np.concatenate([y[a:b, c:d].ravel() for (a, b, c, d) in WINDOWS])
    ref = np.concatenate([r.ravel() for r in ref_windows])
    return rel_err(got, ref), rms_rel(got, ref)


def oracle_windows(inp, r, w):
    return [of.filter_window_at(inp, r, w, "replicate", *win) for win in WINDOWS]


def run(gb, x, out_dtype, r, w, **plan):
    import torch
    y = gb.filter_tensor(x, radii=r, weights=w, out_dtype=out_dtype, plan=gb.make_plan(**plan))
    torch.cuda.synchronize()
    return to_host(y)


def study(gb):
    import torch
    r, w = ofit.fit_gaussian_boxes(SIGMA, K)
    w32 = np.float32(w).astype(np.float64)       # the weights the kernels use
    rows = []
    f = field(1.0e4)
    ref = oracle_windows(f.astype(np.float64), r, w32)
    x = to_device(f, "f32")
    for name, plan in VARIANTS:
        y = run(gb, x, torch.float32, r, w, **plan)
        rows.append(("f32 + 1e4", name, "f32") + window_errors(y, ref))
    del x
    g = field(0.0)
    x = to_device(g, "bf16")                      # bf16 storage of the field
    xin = x.to(torch.float64).cpu().numpy()
    ref_b = oracle_windows(xin, r, w32)           # the values the device holds
    ref_f = oracle_windows(g.astype(np.float64), r, w32)
    for out_name, od in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        y = run(gb, x, od, r, w, path=GF_PATH_AUTO)
        rows.append(("bf16 storage", "default", out_name) + window_errors(y, ref_b))
        rows.append(("bf16 storage", "vs f32 field", out_name) + window_errors(y, ref_f))
    return rows


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


def test_precision_study(gb):
    rows = {(a, b, c): (m, q) for a, b, c, m, q in study(gb)}
    comp = rows[("f32 + 1e4", "default", "f32")]
    assert comp[0] <= TOL["f32"], comp                      # the stated FP32 bound
    assert rows[("f32 + 1e4", "offset", "f32")][0] <= 1e-3
    # the default sums never lose to the plain FP32 sums they replace
    assert comp[0] <= rows[("f32 + 1e4", "plain", "f32")][0]
    assert comp[0] <= rows[("f32 + 1e4", "plain-long", "f32")][0]
    assert rows[("bf16 storage", "default", "f32")][0] <= TOL["f32"]
    assert rows[("bf16 storage", "default", "bf16")][0] <= TOL["bf16"]


if __name__ == "__main__":
    from paper_1107_4958_gb300 import build
    build.build()
    from paper_1107_4958_gb300 import gaussbox
    print("%-14s %-14s %-5s %12s %12s" % ("input", "variant", "out", "max rel", "rms rel"))
    for a, b, c, m, q in study(gaussbox):
        print("%-14s %-14s %-5s %12.3e %12.3e" % (a, b, c, m, q))
