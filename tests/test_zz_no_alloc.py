"""GPU: gauss_filter_batch_noalloc, the batch call for code that may not
allocate device memory (a plug-in whose host owns every device buffer, a
server that reserves HBM once at start-up, a latency-critical path that must
not pay for cudaMalloc/cudaFree).  It takes its scratch from a fixed array
built into the library, so its results must match the handle-based
gauss_filter_batch, which allocates its scratch.  Two calls in a row check
that the shared array, which keeps the previous call's contents, is rewritten
and its ticket counters reset each time.

This file is collected last on purpose; it also passes when run on its own in
a fresh process."""
import ctypes

import numpy as np
import pytest

from gpu_helpers import TOL, oracle_input, rel_err, to_device, to_host, torch_dtype
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


def _batch(seed):
    specs = [(130, 250, 1, "u8", 3.0 + seed, 4), (96, 300, 3, "f32", 6.5, 3), (77, 200, 3, "bf16", 2.5, 5),
             (200, 190, 1, "f32", 17.0, 4), (64, 512, 4, "f16", 4.0 + seed, 3)]
    out = []
    for i, (h, w, c, dt, sigma, k) in enumerate(specs):
        base = "u8" if dt == "u8" else "f32"
        out.append((synth.image(h, w, seed=seed * 100 + i, dtype=base, c=c), dt, sigma, k))
    return out


def _filter_both(gb, imgs):
    import torch
    xs = [to_device(a, dt) for a, dt, _, _ in imgs]
    odt = [torch_dtype("f32" if dt == "u8" else dt) for _, dt, _, _ in imgs]
    outs_na = [torch.full(x.shape, float("nan"), dtype=o, device="cuda") for x, o in zip(xs, odt)]
    outs_ref = [torch.empty(x.shape, dtype=o, device="cuda") for x, o in zip(xs, odt)]
    stream = torch.cuda.current_stream().cuda_stream
    # the no-alloc call runs every image fused; the allocating batch is given
    # the same fused plans
    fused = gb.make_plan(GF_PATH_FUSED)
    gb.gauss_filter_batch_noalloc([gb.image_desc(x, o, s, k) for x, o, (_, _, s, k) in zip(xs, outs_na, imgs)],
                                  stream)
    h = gb.gf_create()
    try:
        gb.gauss_filter_batch(h, [gb.image_desc(x, o, s, k, plan=fused)
                                  for x, o, (_, _, s, k) in zip(xs, outs_ref, imgs)], stream)
        torch.cuda.synchronize()
    finally:
        gb.gf_destroy(h)
    return [to_host(o) for o in outs_na], [to_host(o) for o in outs_ref]


def test_noalloc_matches_allocating_batch_twice(gb):
    for call in range(2):                       # two calls in a row on the shared array
        imgs = _batch(seed=call + 1)
        got, ref = _filter_both(gb, imgs)
        for g, r in zip(got, ref):
            assert not np.isnan(g).any()
            tol = TOL["f32"]
            assert rel_err(g, r) <= tol
            assert np.array_equal(g, r)         # same plans, same arithmetic: identical
        # one image of each call against the FP64 oracle, so that a staging
        # fault shared by both calls cannot pass unnoticed
        f, dt, sigma, k = imgs[call]
        rr, ww = ofit.fit_gaussian_boxes(sigma, k)
        want = of.filter_separable(oracle_input(f, dt), rr, np.float32(ww).astype(np.float64), "replicate")
        out_name = "f32" if dt in ("u8", "f32") else dt
        assert rel_err(got[call], want) <= TOL[out_name], (call, dt)


def test_noalloc_rejects_an_explicit_two_pass_plan(gb):
    import torch
    from paper_1107_4958_gb300 import abi_types as T
    x = torch.zeros((32, 32), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    d = gb.image_desc(x, y, 2.0, 3, plan=gb.make_plan(GF_PATH_TWO_PASS))
    arr = (gb.gf_image_desc * 1)(d)
    rc = gb.lib().gauss_filter_batch_noalloc(arr, 1, ctypes.c_void_p(0))
    assert rc == T.GF_EUNSUPPORTED


def test_noalloc_rejects_more_than_its_capacity(gb):
    from paper_1107_4958_gb300 import abi_types as T
    d = gb.gf_image_desc()
    arr = (gb.gf_image_desc * (T.GF_NOALLOC_MAX_IMAGES + 1))(*([d] * (T.GF_NOALLOC_MAX_IMAGES + 1)))
    rc = gb.lib().gauss_filter_batch_noalloc(arr, T.GF_NOALLOC_MAX_IMAGES + 1, ctypes.c_void_p(0))
    assert rc == T.GF_ELIMIT
    assert "capacity" in gb.gf_status_string(rc)


def test_noalloc_refuses_a_capturing_stream(gb):
    # its parameters come from host storage that the next call rewrites, so a
    # graph recorded around it would replay stale parameters: it enqueues
    # nothing and says so
    import torch
    from paper_1107_4958_gb300 import abi_types as T
    x = to_device(synth.image(40, 64, seed=5, dtype="f32"), "f32")
    y = torch.empty_like(x)
    arr = (gb.gf_image_desc * 1)(gb.image_desc(x, y, 2.0, 3))
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        y.fill_(1.0)                                   # keep the captured graph non-empty
        rc = gb.lib().gauss_filter_batch_noalloc(arr, 1, ctypes.c_void_p(side.cuda_stream))
    assert rc == T.GF_EUNSUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert bool((y == 1.0).all())                      # nothing of the call was recorded
    # outside the capture the same call runs
    rc = gb.lib().gauss_filter_batch_noalloc(arr, 1, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == T.GF_OK
    torch.cuda.synchronize()
    assert not bool((y == 1.0).all())


def test_noalloc_rejects_two_pass_only_accumulation(gb):
    # the precision-study accumulation modes exist on the two-pass path only
    import torch
    from paper_1107_4958_gb300 import abi_types as T
    x = torch.zeros((32, 32), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    for accum in (T.GF_ACCUM_OFFSET, T.GF_ACCUM_PLAIN):
        d = gb.image_desc(x, y, 2.0, 3, plan=gb.make_plan(T.GF_PATH_AUTO, accum=accum))
        arr = (gb.gf_image_desc * 1)(d)
        assert gb.lib().gauss_filter_batch_noalloc(arr, 1, ctypes.c_void_p(0)) == T.GF_EUNSUPPORTED
