"""GPU: the persistent batched launch (gauss_filter_batch).  Every image of a
batch must be bit-identical to the same image filtered alone, for uneven
sizes, per-image sigma/K, mixed dtypes and channel counts, with and without
CUDA-graph replay; and within tolerance of the FP64 oracle."""
import numpy as np
import pytest

from gpu_helpers import TOL, oracle_input, rel_err, to_device, to_host, torch_dtype
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth

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


def _images(specs):
    out = []
    for i, (h, w, c, dt, sigma, k) in enumerate(specs):
        base = "u8" if dt in ("u8", "u16") else "f32"
        arr = synth.image(h, w, seed=100 + i, dtype=base, c=c)
        out.append((arr, dt, sigma, k))
    return out


def _run(gb, handle, imgs, out_dt=None, boundary=0):
    import torch
    xs = [to_device(a, dt) for a, dt, _, _ in imgs]
    outs = [torch.empty(x.shape, dtype=torch_dtype(out_dt or ("f32" if dt in ("u8", "u16") else dt)),
                        device="cuda") for x, (_, dt, _, _) in zip(xs, imgs)]
    gb.filter_batch_tensors(handle, xs, outs, [s for _, _, s, _ in imgs], [k for _, _, _, k in imgs], boundary)
    torch.cuda.synchronize()
    alone = [gb.filter_tensor(x, sigma=s, K=k, boundary=boundary, out_dtype=o.dtype)
             for x, o, (_, _, s, k) in zip(xs, outs, imgs)]
    torch.cuda.synchronize()
    return [to_host(o) for o in outs], [to_host(a) for a in alone]


UNEVEN = [(257, 411, 3, "f32", 1.3, 3), (96, 1000, 3, "f32", 7.5, 4), (700, 130, 3, "f32", 22.0, 5),
          (333, 333, 3, "f32", 2.0, 4), (64, 64, 3, "f32", 40.0, 5), (1200, 900, 3, "f32", 11.0, 3)]


@pytest.mark.parametrize("graphs", [True, False])
def test_batch_bit_identical_to_alone_uneven(gb, graphs):
    h = gb.gf_create(use_graphs=graphs)
    try:
        imgs = _images(UNEVEN)
        for _rep in range(2):            # second call replays the captured graph
            got, alone = _run(gb, h, imgs)
            for g, a in zip(got, alone):
                assert np.array_equal(g, a)
    finally:
        gb.gf_destroy(h)


def test_batch_mixed_classes(gb):
    specs = [(120, 300, 1, "u8", 3.0, 4), (300, 120, 3, "f32", 5.0, 3), (77, 200, 3, "bf16", 2.5, 5),
             (250, 250, 1, "f32", 30.0, 4), (40, 700, 1, "u8", 9.0, 3), (128, 128, 4, "f16", 4.0, 4)]
    h = gb.gf_create()
    try:
        imgs = _images(specs)
        got, alone = _run(gb, h, imgs)
        for g, a in zip(got, alone):
            assert np.array_equal(g, a)
    finally:
        gb.gf_destroy(h)


def test_batch_matches_oracle(gb):
    specs = [(130, 250, 3, "f32", 6.0, 4), (90, 70, 1, "u8", 13.0, 5), (200, 180, 3, "f32", 1.1, 3)]
    h = gb.gf_create()
    try:
        imgs = _images(specs)
        got, _ = _run(gb, h, imgs, boundary=2)
        for g, (arr, dt, s, k) in zip(got, imgs):
            r, w = ofit.fit_gaussian_boxes(s, k)
            ref = of.filter_separable(oracle_input(arr, dt), r, w, "reflect")
            assert rel_err(g, ref) <= TOL["f32"]
    finally:
        gb.gf_destroy(h)


def test_batch_rejects_overlapping_outputs(gb):
    import torch
    h = gb.gf_create()
    try:
        x = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
        y = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
        with pytest.raises(gb.GaussboxError) as ei:
            gb.filter_batch_tensors(h, [x, x], [y, y], [2.0, 2.0], [3, 3])
        assert ei.value.status == 1
        with pytest.raises(gb.GaussboxError):
            gb.filter_batch_tensors(h, [x, y], [y, x], [2.0, 2.0], [3, 3])
    finally:
        gb.gf_destroy(h)


def test_batch_with_forced_paths_bit_identical(gb):
    # each image runs on the plan its descriptor names; alone with the same
    # plan it gives the same bits (two-pass images use the handle's intermediates)
    import torch
    from paper_1107_4958_gb300.abi_types import GF_PATH_FUSED, GF_PATH_TWO_PASS
    imgs = _images(UNEVEN + [(500, 800, 1, "u8", 30.0, 4), (129, 257, 3, "bf16", 60.0, 5)])
    plans = [gb.make_plan(GF_PATH_TWO_PASS if i % 2 else GF_PATH_FUSED) for i in range(len(imgs))]
    plans[2] = gb.make_plan(GF_PATH_TWO_PASS, tile_w=100, tile_h=24, col_w=64, col_h=90)
    xs = [to_device(a, dt) for a, dt, _, _ in imgs]
    outs = [torch.empty(x.shape, dtype=torch.float32, device="cuda") for x in xs]
    h = gb.gf_create(use_graphs=True)
    try:
        for _rep in range(2):
            gb.filter_batch_tensors(h, xs, outs, [s for _, _, s, _ in imgs], [k for _, _, _, k in imgs], 0,
                                    plans=plans)
            torch.cuda.synchronize()
            for x, o, p, (a, dt, s, k) in zip(xs, outs, plans, imgs):
                alone = gb.filter_tensor(x, sigma=s, K=k, out_dtype=torch.float32, plan=p)
                torch.cuda.synchronize()
                assert np.array_equal(to_host(o), to_host(alone))
                r, w = ofit.fit_gaussian_boxes(s, k)
                ref = of.filter_separable(oracle_input(a, dt), r, np.float32(w).astype(np.float64), "replicate")
                assert rel_err(to_host(o), ref) <= TOL["f32"]
    finally:
        gb.gf_destroy(h)


def test_batch_launch_count(gb):
    # one persistent launch per fused class; the two-pass images of the
    # default accumulation share one row launch and one column launch per
    # kernel class, an image in a study accumulation mode keeps its own two
    import torch
    from paper_1107_4958_gb300.abi_types import GF_ACCUM_OFFSET, GF_PATH_FUSED, GF_PATH_TWO_PASS
    specs = [(100, 200, 1, "f32", 3.0, 4), (100, 200, 1, "f32", 3.0, 4), (90, 300, 3, "f32", 2.0, 3),
             (150, 160, 1, "f32", 30.0, 5), (150, 160, 1, "f32", 30.0, 5), (150, 160, 1, "f32", 30.0, 5)]
    imgs = _images(specs)
    two = gb.make_plan(GF_PATH_TWO_PASS)
    plans = [gb.make_plan(GF_PATH_FUSED)] * 3 + [two, two]
    h = gb.gf_create()
    try:
        # the two C=1 fused images (same size and radii, other pixels) share a
        # class, the C=3 one has its own; the two-pass pair is one class each way
        xs = [to_device(a, dt) for a, dt, _, _ in imgs[:5]]
        outs = [torch.empty_like(x) for x in xs]
        gb.filter_batch_tensors(h, xs, outs, [s for *_, s, _ in imgs[:5]], [k for *_, k in imgs[:5]], 0, plans=plans)
        torch.cuda.synchronize()
        assert gb.gf_batch_launches(h) == 2 + 2
        for x, o, p, (_, _, s, k) in zip(xs, outs, plans, imgs):
            alone = gb.filter_tensor(x, sigma=s, K=k, out_dtype=torch.float32, plan=p)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(o), to_host(alone))
        # a study-mode image beside them: two more launches of its own
        xs = [to_device(a, dt) for a, dt, _, _ in imgs]
        outs = [torch.empty_like(x) for x in xs]
        plans6 = plans + [gb.make_plan(GF_PATH_TWO_PASS, accum=GF_ACCUM_OFFSET)]
        gb.filter_batch_tensors(h, xs, outs, [s for *_, s, _ in imgs], [k for *_, k in imgs], 0, plans=plans6)
        torch.cuda.synchronize()
        assert gb.gf_batch_launches(h) == 2 + 2 + 2
        for x, o, p, (_, _, s, k) in zip(xs, outs, plans6, imgs):
            alone = gb.filter_tensor(x, sigma=s, K=k, out_dtype=torch.float32, plan=p)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(o), to_host(alone))
    finally:
        gb.gf_destroy(h)


def test_batch_twopass_class_split(gb):
    # a class holds at most 32 images: 40 two-pass images of one shape and
    # kernel take two row and two column launches, each image as filtered alone
    import torch
    from paper_1107_4958_gb300.abi_types import GF_PATH_TWO_PASS
    imgs = _images([(70, 90, 1, "f32", 20.0, 4)] * 40)
    plan = gb.make_plan(GF_PATH_TWO_PASS)
    xs = [to_device(a, dt) for a, dt, _, _ in imgs]
    outs = [torch.empty_like(x) for x in xs]
    h = gb.gf_create()
    try:
        gb.filter_batch_tensors(h, xs, outs, [20.0] * 40, [4] * 40, 0, plans=[plan] * 40)
        torch.cuda.synchronize()
        assert gb.gf_batch_launches(h) == 4
        for x, o in zip(xs, outs):
            alone = gb.filter_tensor(x, sigma=20.0, K=4, out_dtype=torch.float32, plan=plan)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(o), to_host(alone))
    finally:
        gb.gf_destroy(h)


def test_batch_twopass_classes_bit_identical(gb):
    # many two-pass images across input types, channel counts, output types,
    # strip widths and sizes (several row and column classes, tiles of
    # different images side by side in one launch): each as filtered alone
    import torch
    from paper_1107_4958_gb300.abi_types import GF_PATH_TWO_PASS
    specs = [(300, 500, 1, "u8", 30.0, 4), (77, 1030, 1, "u8", 12.0, 3), (500, 90, 3, "f32", 45.0, 5),
             (129, 257, 3, "f32", 60.0, 5), (64, 64, 1, "f32", 20.0, 4), (1000, 700, 4, "bf16", 25.0, 4),
             (33, 2000, 2, "f16", 18.0, 5), (400, 400, 3, "f32", 10.0, 5), (250, 31, 1, "u16", 14.0, 3),
             (300, 500, 1, "u8", 30.0, 4)]
    imgs = _images(specs)
    plans = [gb.make_plan(GF_PATH_TWO_PASS)] * len(imgs)
    plans[4] = gb.make_plan(GF_PATH_TWO_PASS, tile_w=40, tile_h=24, col_w=32, col_h=50)
    plans[7] = gb.make_plan(GF_PATH_TWO_PASS, col_w=256)   # 256-column strips hold radii up to 39
    xs = [to_device(a, dt) for a, dt, _, _ in imgs]
    # integer inputs give FP32 outputs
    out_dts = [torch.float32, torch.float32, torch.bfloat16, torch.float16, torch.float32, torch.bfloat16,
               torch.float32, torch.float32, torch.float32, torch.float32]
    outs = [torch.empty(x.shape, dtype=o, device="cuda") for x, o in zip(xs, out_dts)]
    h = gb.gf_create()
    try:
        for _rep in range(2):
            gb.filter_batch_tensors(h, xs, outs, [s for *_, s, _ in imgs], [k for *_, k in imgs], 1, plans=plans)
            torch.cuda.synchronize()
            # the first and last images (same shape and radii) share their two launches
            assert gb.gf_batch_launches(h) <= 2 * (len(imgs) - 1)
            for x, o, p, (_, _, s, k) in zip(xs, outs, plans, imgs):
                alone = gb.filter_tensor(x, sigma=s, K=k, boundary=1, out_dtype=o.dtype, plan=p)
                torch.cuda.synchronize()
                assert np.array_equal(to_host(o), to_host(alone))
    finally:
        gb.gf_destroy(h)


def test_identical_batch_replays_with_new_pixels(gb):
    # the same descriptors again: the captured graph runs as it stands, so new
    # pixel values in the same buffers must come out filtered; a changed
    # buffer or kernel plans the batch anew
    import torch
    imgs = _images(UNEVEN[:4])
    xs = [to_device(a, dt) for a, dt, _, _ in imgs]
    outs = [torch.empty_like(x) for x in xs]
    sig = [s for _, _, s, _ in imgs]
    ks = [k for _, _, _, k in imgs]
    h = gb.gf_create()
    try:
        for rep in range(4):
            if rep == 2:
                outs[1] = torch.empty_like(xs[1])       # another output buffer
            if rep == 3:
                sig[0] = sig[0] * 1.5                   # another kernel
            for x in xs:
                x.mul_(0.5).add_(float(rep))            # new pixels in the same buffers
            gb.filter_batch_tensors(h, xs, outs, sig, ks, 0)
            torch.cuda.synchronize()
            for x, o, s, k in zip(xs, outs, sig, ks):
                alone = gb.filter_tensor(x, sigma=s, K=k)
                torch.cuda.synchronize()
                assert torch.equal(o, alone), rep
    finally:
        gb.gf_destroy(h)


def test_empty_batch_is_a_no_op(gb):
    h = gb.gf_create()
    try:
        gb.gauss_filter_batch(h, [], 0)
    finally:
        gb.gf_destroy(h)
