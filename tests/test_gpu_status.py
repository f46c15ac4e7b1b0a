"""GPU: status words and the bounded-wait expiry path.

Every pipeline wait of the kernels is bounded.  When a bound runs out, the CTA
records GF_ETIMEOUT in a status word, waits (with the full bound) for its
copies in flight, frees its tensor memory and returns; nothing traps.  A
handle created with a bound of one SM clock cycle makes its kernels' waits
expire for real (the first staged band is never there one cycle after it was
requested), without faulting or hanging anything.

Each handle has a status word of its own, separate from every other handle's
and from the word of the handle-less calls, so that clearing one never
erases another caller's GF_ETIMEOUT."""
import numpy as np
import pytest

from gpu_helpers import TOL, rel_err, to_device, to_host
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import GF_ETIMEOUT, GF_OK, GF_PATH_FUSED, GF_PATH_TWO_PASS

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


def _batch(gb, xs, ys, plans):
    return [gb.image_desc(x, y, 4.0, 4, plan=gb.make_plan(p)) for x, y, p in zip(xs, ys, plans)]


def test_two_handles_keep_separate_status_words(gb):
    import torch
    fs = [synth.image(300, 520, seed=61, dtype="u8"), synth.image(260, 400, seed=62, dtype="u8")]
    xs = [to_device(f, "u8") for f in fs]
    ya = [torch.empty(x.shape, dtype=torch.float32, device="cuda") for x in xs]
    yb = [torch.empty(x.shape, dtype=torch.float32, device="cuda") for x in xs]
    plans = [GF_PATH_FUSED, GF_PATH_TWO_PASS]
    ha = gb.gf_create(wait_cycles=1)     # every pipeline wait of ha's kernels expires
    hb = gb.gf_create()
    s = torch.cuda.current_stream().cuda_stream
    try:
        gb.gauss_filter_batch(ha, _batch(gb, xs, ya, plans), s)    # fused class + two-pass launches
        gb.gauss_filter_batch(hb, _batch(gb, xs, yb, plans), s)
        torch.cuda.synchronize()
        assert gb.gf_handle_status(ha) == GF_ETIMEOUT
        assert gb.gf_handle_status(hb) == GF_OK
        assert gb.gf_get_device_status() == GF_OK          # the handle-less word is untouched
        r, w = ofit.fit_gaussian_boxes(4.0, 4)
        for f, y in zip(fs, yb):                            # hb's results are the filter
            ref = of.filter_separable(f.astype(np.float64), r, w, "replicate")
            assert rel_err(to_host(y), ref) <= TOL["f32"]
        # clearing one handle's word leaves the other's
        assert gb.gf_handle_status(hb, clear=True) == GF_OK
        assert gb.gf_handle_status(ha) == GF_ETIMEOUT
        assert gb.gf_handle_status(ha, clear=True) == GF_ETIMEOUT
        assert gb.gf_handle_status(ha) == GF_OK
        # a volume through the expiring handle times out too, and only there
        v = np.stack([fs[0][:64, :96]] * 5)
        vx = to_device(v, "u8")
        gb.filter_volume_tensor(ha, vx, radii=r, weights=w)
        torch.cuda.synchronize()
        assert gb.gf_handle_status(ha, clear=True) == GF_ETIMEOUT
        assert gb.gf_handle_status(hb) == GF_OK
    finally:
        gb.gf_destroy(ha)
        gb.gf_destroy(hb)
    # the device stays usable: the next ordinary call is clean and correct
    y = gb.filter_tensor(xs[0], sigma=4.0, K=4)
    torch.cuda.synchronize()
    r, w = ofit.fit_gaussian_boxes(4.0, 4)
    assert rel_err(to_host(y), of.filter_separable(fs[0].astype(np.float64), r, w, "replicate")) <= TOL["f32"]
    assert gb.gf_get_device_status() == GF_OK


def test_negative_wait_bound_is_rejected(gb):
    with pytest.raises(gb.GaussboxError) as ei:
        gb.gf_create(wait_cycles=-1)
    assert ei.value.status == 1
