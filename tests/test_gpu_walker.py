"""GPU parity of the register-walk path (GF_PATH_WALK): the kernel compiled at
run time for the image's radii, against the FP64 oracle (Sec. 3.3-3.4).

Covers both integer input types, every boundary, shapes with ragged strips
and row tiles (widths around the 128-column strip, heights around a tile),
images narrower or shorter than one strip or tile, radii up to the path's
largest, inputs whose base or pitch are not 16-byte multiples (the folded
copy instead of vector loads), the headline 4096 x 4096 image on sampled
rows, and the refusal of images the path does not take."""
import numpy as np
import pytest

from gpu_helpers import TOL, rel_err, rms_rel, to_device, to_host
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import (BOUNDARY_CODE, GF_EUNSUPPORTED, GF_PATH_AUTO, GF_PATH_WALK, GF_U8,
                                             GF_U16)

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


def walk(gb, x, r, w, boundary, path=GF_PATH_WALK):
    import torch
    y = gb.filter_tensor(x, radii=r, weights=w, boundary=BOUNDARY_CODE[boundary], out_dtype=torch.float32,
                         plan=gb.make_plan(path))
    torch.cuda.synchronize()
    return to_host(y)


def oracle(f, r, w, boundary):
    return of.filter_separable(f.astype(np.float64), r, np.float32(w).astype(np.float64), boundary)


@pytest.mark.parametrize("dtype", ["u8", "u16"])
@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
@pytest.mark.parametrize("shape", [(1, 1), (1, 200), (300, 1), (7, 9), (37, 127), (131, 129), (400, 385),
                                   (513, 1000)])
def test_walk_shapes_and_boundaries(gb, dtype, boundary, shape):
    f = synth.image(shape[0], shape[1], seed=81, dtype=dtype)
    x = to_device(f, dtype)
    for sigma, K in ((0.5, 3), (2.0, 4), (5.0, 3), (8.0, 4), (8.5, 5)):
        r, w = ofit.fit_gaussian_boxes(sigma, K)
        if max(r) > 22:
            continue
        got = walk(gb, x, r, w, boundary)
        ref = oracle(f, r, w, boundary)
        assert rel_err(got, ref) <= TOL["f32"], (sigma, K, rel_err(got, ref), rms_rel(got, ref))


def test_walk_is_the_default_for_eligible_images(gb):
    r, _ = ofit.fit_gaussian_boxes(8.0, 4)
    assert gb.gauss_plan_default(4096, 4096, 1, GF_U8, 2, r).path == GF_PATH_WALK
    assert gb.gauss_plan_default(100, 70, 1, GF_U16, 2, r).path == GF_PATH_WALK
    assert gb.gauss_plan_default(100, 70, 3, GF_U8, 2, r).path != GF_PATH_WALK       # three channels
    assert gb.gauss_plan_default(100, 70, 1, 2, 2, r).path != GF_PATH_WALK           # float input
    r32, _ = ofit.fit_gaussian_boxes(32.0, 4)
    assert gb.gauss_plan_default(4096, 4096, 1, GF_U8, 2, r32).path != GF_PATH_WALK  # radius beyond 22


@pytest.mark.parametrize("boundary", ["replicate", "reflect"])
def test_walk_unaligned_rows(gb, boundary):
    # pitches that are not multiples of 16 bytes, and a base 1 byte into an
    # allocation: the walk reads through its boundary-folded copy everywhere
    import torch
    f = synth.image(150, 700, seed=82, dtype="u8")
    r, w = ofit.fit_gaussian_boxes(6.0, 4)
    ref = oracle(f, r, w, boundary)
    for pad in (3, 16, 35):
        got = walk(gb, to_device(f, "u8", pad), r, w, boundary)
        assert rel_err(got, ref) <= TOL["f32"], pad
    buf = torch.zeros(150 * 700 + 1, dtype=torch.uint8, device="cuda")
    buf[1:] = torch.from_numpy(f).cuda().reshape(-1)
    got = walk(gb, buf[1:].view(150, 700), r, w, boundary)
    assert rel_err(got, ref) <= TOL["f32"]


def test_walk_full_u16_range_and_noise(gb):
    rng = np.random.default_rng(83)
    f = rng.integers(0, 65536, (333, 1030)).astype(np.uint16)
    for sigma, K in ((1.0, 4), (8.0, 5)):
        r, w = ofit.fit_gaussian_boxes(sigma, K)
        got = walk(gb, to_device(f, "u16"), r, w, "reflect")
        assert rel_err(got, oracle(f, r, w, "reflect")) <= TOL["f32"], sigma
    g = rng.integers(0, 256, (333, 1030)).astype(np.uint8)
    r, w = ofit.fit_gaussian_boxes(0.5, 3)
    got = walk(gb, to_device(g, "u8"), r, w, "zero")
    assert rel_err(got, oracle(g, r, w, "zero")) <= TOL["f32"]


def test_walk_explicit_boxes_with_negative_weights(gb):
    # A difference of boxes (band-pass): negative weights, outputs of both
    # signs.  Near a zero crossing an output is the cancellation of terms as
    # large as the response of the absolute kernel, so FP32 arithmetic is held
    # to that response: error / max(|Y|, (|k| * f)(x)) <= 1e-5.
    f = synth.image(260, 530, seed=84, dtype="u8")
    r = [1, 4, 9, 17]
    w = [0.05, 0.02, -0.01, -0.002]
    got = walk(gb, to_device(f, "u8"), r, w, "replicate")
    ref = oracle(f, r, w, "replicate")
    ref_abs = oracle(f, r, np.abs(w), "replicate")
    assert float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), ref_abs))) <= TOL["f32"]


@pytest.mark.parametrize("sigma", [2.0, 8.0])
def test_walk_4096_u8_sampled_rows(gb, sigma):
    f = synth.image(4096, 4096, seed=2, dtype="u8")
    r, w = ofit.fit_gaussian_boxes(sigma, 4)
    got = walk(gb, to_device(f, "u8"), r, w, "replicate", path=GF_PATH_AUTO)
    ys = [0, 1, 2, 20, 337, 338, 339, 1000, 2048, 4000, 4094, 4095]
    ref = of.filter_rows_at(f.astype(np.float64), r, w, "replicate", ys)
    assert rel_err(got[ys], ref) <= TOL["f32"]


def test_walk_refuses_what_it_does_not_take(gb):
    import torch
    x3 = torch.zeros((40, 50, 3), dtype=torch.uint8, device="cuda")
    xf = torch.zeros((40, 50), dtype=torch.float32, device="cuda")
    r, w = ofit.fit_gaussian_boxes(3.0, 3)
    for x in (x3, xf):
        with pytest.raises(gb.GaussboxError) as ei:
            gb.filter_tensor(x, radii=r, weights=w, out_dtype=torch.float32, plan=gb.make_plan(GF_PATH_WALK))
        assert ei.value.status == GF_EUNSUPPORTED
    r40, w40 = ofit.fit_gaussian_boxes(16.0, 4)                       # radius 41
    with pytest.raises(gb.GaussboxError) as ei:
        gb.filter_tensor(torch.zeros((40, 50), dtype=torch.uint8, device="cuda"), radii=r40, weights=w40,
                         out_dtype=torch.float32, plan=gb.make_plan(GF_PATH_WALK))
    assert ei.value.status == GF_EUNSUPPORTED
    # a handle's batch runs an explicit walk request in a launch of its own;
    # the batch call on caller storage has no such launch and refuses it
    f = synth.image(40, 50, seed=85, dtype="u8")
    h = gb.gf_create()
    try:
        x = to_device(f, "u8")
        y = torch.empty((40, 50), dtype=torch.float32, device="cuda")
        gb.gauss_filter_batch(h, [gb.image_desc(x, y, 3.0, 3, plan=gb.make_plan(GF_PATH_WALK))])
        torch.cuda.synchronize()
        r3, w3 = ofit.fit_gaussian_boxes(3.0, 3)
        assert rel_err(to_host(y), oracle(f, r3, w3, "replicate")) <= TOL["f32"]
        with pytest.raises(gb.GaussboxError) as ei:
            gb.gauss_filter_batch_noalloc([gb.image_desc(x, y, 3.0, 3, plan=gb.make_plan(GF_PATH_WALK))])
        assert ei.value.status == GF_EUNSUPPORTED
    finally:
        gb.gf_destroy(h)


def test_walker_compile_needs_no_launch(gb):
    st, log = gb.gauss_walker_compile(GF_U8, [4, 9, 14, 20])
    assert st == 0, log
    st, _ = gb.gauss_walker_compile(GF_U8, [4, 9, 14, 40])
    assert st == GF_EUNSUPPORTED
