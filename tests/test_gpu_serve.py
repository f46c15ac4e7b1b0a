"""GPU: the continuous-batching server.  Every served result matches the FP64
oracle (the separable staircase convolution of Sec. 3.3-3.4) within the
parity bar of its output type, and equals gauss_filter on the same image
whether a request runs alone or in a mix that arrives while other steps are on
the device; admission respects the HBM budget; oversized requests are
refused; release times are honoured."""
import numpy as np
import pytest

from gpu_helpers import TOL, oracle_input, rel_err, to_device, torch_dtype
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


MIX = [(120, 300, 1, "u8", 3.0, 4), (300, 120, 3, "f32", 5.0, 3), (77, 200, 3, "bf16", 2.5, 5),
       (250, 250, 1, "f32", 12.0, 4), (40, 700, 1, "u8", 9.0, 3), (128, 130, 3, "f32", 1.2, 5),
       (513, 257, 1, "bf16", 7.0, 4), (64, 64, 3, "u8", 20.0, 5),
       # large radii: the default plan takes the two-pass path, whose
       # intermediate the server holds in its arena while the step runs
       (300, 400, 3, "f32", 40.0, 5), (200, 900, 1, "u8", 60.0, 4)]


def _inputs():
    out = []
    for i, (h, w, c, dt, sigma, k) in enumerate(MIX * 3):
        base = "u8" if dt == "u8" else "f32"
        f = synth.image(h, w, seed=500 + i, dtype=base, c=c)
        out.append((to_device(f, dt), dt, sigma, k, f))
    return out


def _oracle(f, dt, sigma, k):
    r, w = ofit.fit_gaussian_boxes(sigma, k)
    return of.filter_separable(oracle_input(f, dt), r, np.float32(w).astype(np.float64), "replicate")


def _read(gb, comp, x, dt):
    import torch
    H, W = x.shape[0], x.shape[1]
    C = x.shape[2] if x.dim() == 3 else 1
    t = gb.completion_tensor(comp, H, W, C, torch_dtype("f32" if dt == "u8" else dt))
    return t.to(torch.float64).cpu().numpy()


def _alone(gb, x, dt, sigma, k):
    import torch
    y = gb.filter_tensor(x, sigma=sigma, K=k, out_dtype=torch_dtype("f32" if dt == "u8" else dt))
    torch.cuda.synchronize()
    return y.to(torch.float64).cpu().numpy()


@pytest.mark.parametrize("plain", [False, True])
def test_served_results_equal_alone(gb, plain):
    h = gb.gf_create()
    try:
        gb.gf_server_start(h, hbm_budget_bytes=256 << 20, max_batch=5, max_inflight=3, plain=plain)
        ins = _inputs()
        t0 = gb.gf_clock_now()
        tickets = []
        for i, (x, dt, sigma, k, _f) in enumerate(ins):
            d = gb.request_desc(x, torch_dtype("f32" if dt == "u8" else dt), sigma, k)
            # bursts of six arrivals every 2 ms: a burst forms batched steps, and
            # later bursts join while earlier steps are still on the device
            tickets.append(gb.gf_server_submit(h, d, release_time=t0 + 0.002 * (i // 6)))
        for (x, dt, sigma, k, f), t in zip(ins, tickets):
            c = gb.gf_server_wait(h, t, 60.0)
            assert c.status == 0
            assert c.t_admit >= c.t_release and c.t_done >= c.t_admit
            got = _read(gb, c, x, dt)
            # against the definition (fused, two-pass and bf16 requests alike)
            out_name = "bf16" if dt == "bf16" else "f32"
            assert rel_err(got, _oracle(f, dt, sigma, k)) <= TOL[out_name], (x.shape, dt, sigma, k)
            # and bit-identical to the same request filtered alone
            assert np.array_equal(got, _alone(gb, x, dt, sigma, k))
            gb.gf_server_release(h, t)
        st = gb.gf_server_stats_get(h)
        assert st.completed == len(ins) and st.arena_peak <= st.arena_bytes
        if not plain:
            assert st.steps < len(ins)          # requests were batched
    finally:
        gb.gf_server_stop(h)
        gb.gf_destroy(h)


def test_admission_by_budget_and_rejection(gb):
    import torch
    h = gb.gf_create()
    try:
        budget = 2 * 300 * 300 * 4 + 4096               # room for two 300x300 f32 outputs
        gb.gf_server_start(h, hbm_budget_bytes=budget, max_batch=8, max_inflight=2)
        x = to_device(synth.image(300, 300, seed=9, dtype="f32"), "f32")
        fused = gb.make_plan(GF_PATH_FUSED)             # no intermediate: outputs only
        ts = [gb.gf_server_submit(h, gb.request_desc(x, torch.float32, 4.0, 4, plan=fused), auto_release=True)
              for _ in range(9)]
        gb.gf_server_drain(h, 60.0)
        st = gb.gf_server_stats_get(h)
        assert st.completed == 9 and st.arena_peak <= budget
        big = to_device(synth.image(700, 700, seed=10, dtype="f32"), "f32")
        with pytest.raises(gb.GaussboxError) as ei:
            gb.gf_server_submit(h, gb.request_desc(big, torch.float32, 4.0, 4, plan=fused))
        assert ei.value.status == 6
        del ts
    finally:
        gb.gf_server_stop(h)
        gb.gf_destroy(h)


def test_two_pass_requests_budget_their_intermediate(gb):
    # a two-pass request holds its output (rows padded to 16 bytes) and its
    # FP32 intermediate (rows of W*C*4 bytes padded to 128) in the arena, each
    # rounded up to the arena's 256-byte granule
    import torch
    H, W = 200, 333
    out_b = -(-(H * (-(-(W * 4) // 16) * 16)) // 256) * 256
    inter_b = -(-(H * (-(-(W * 4) // 128) * 128)) // 256) * 256
    x = to_device(synth.image(H, W, seed=11, dtype="f32"), "f32")
    two = gb.make_plan(GF_PATH_TWO_PASS)
    for budget, ok in ((out_b + inter_b, True), (out_b + inter_b - 256, False)):
        h = gb.gf_create()
        try:
            gb.gf_server_start(h, hbm_budget_bytes=budget, max_batch=4, max_inflight=2)
            if ok:
                ts = [gb.gf_server_submit(h, gb.request_desc(x, torch.float32, 6.0, 4, plan=two), auto_release=True)
                      for _ in range(4)]
                gb.gf_server_drain(h, 60.0)
                st = gb.gf_server_stats_get(h)
                assert st.completed == 4 and st.arena_peak <= budget
                del ts
            else:
                with pytest.raises(gb.GaussboxError) as ei:
                    gb.gf_server_submit(h, gb.request_desc(x, torch.float32, 6.0, 4, plan=two))
                assert ei.value.status == 6
        finally:
            gb.gf_server_stop(h)
            gb.gf_destroy(h)
