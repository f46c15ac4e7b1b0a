"""GPU: gauss_filter_host (host images in, host images out).  Large images on
the fused or the register-walk path are pipelined in slabs of row tiles (copy
in, filter, copy out overlapped); every result must equal gauss_filter on
device copies of the same image bit for bit, pipelined or not, dense or
pitched host rows."""
import numpy as np
import pytest

from gpu_helpers import TOL, rel_err, torch_dtype
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import BOUNDARY_CODE, GF_EINVAL, dtype_code

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


def host_filter(gb, h, arr, in_name, out_name, sigma, K, boundary="replicate", pad=0):
    import torch
    H, W = arr.shape[0], arr.shape[1]
    C = arr.shape[2] if arr.ndim == 3 else 1
    src = torch.from_numpy(np.ascontiguousarray(arr)).to(torch_dtype(in_name))
    isz, osz = src.element_size(), torch.empty(0, dtype=torch_dtype(out_name)).element_size()
    row_in = W * C
    hin = torch.zeros((H, row_in + pad), dtype=src.dtype).pin_memory()
    hin[:, :row_in] = src.reshape(H, row_in)
    hout = torch.full((H, row_in + pad), float("nan"), dtype=torch_dtype(out_name)).pin_memory()
    stream = torch.cuda.current_stream().cuda_stream
    gb.gauss_filter_host(h, hin.data_ptr(), (row_in + pad) * isz, hout.data_ptr(), (row_in + pad) * osz, H, W, C,
                         dtype_code(src.dtype), dtype_code(hout.dtype), sigma, K, BOUNDARY_CODE[boundary], stream)
    return hout[:, :row_in].reshape(arr.shape).to(torch.float64).numpy()


def device_filter(gb, arr, in_name, out_name, sigma, K, boundary="replicate"):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(arr)).to(torch_dtype(in_name)).cuda()
    y = gb.filter_tensor(x, sigma=sigma, K=K, boundary=BOUNDARY_CODE[boundary], out_dtype=torch_dtype(out_name))
    torch.cuda.synchronize()
    return y.to(torch.float64).cpu().numpy()


@pytest.mark.parametrize("H,W,C,in_name,sigma,K,pad", [
    (4096, 4096, 1, "u8", 8.0, 4, 0),      # register walk, pipelined in slabs
    (3001, 2050, 1, "u16", 3.0, 4, 40),    # register walk, pipelined, pitched host rows, ragged strip
    (2500, 3000, 1, "f32", 5.0, 3, 24),    # fused, pipelined, pitched host rows
    (120, 333, 3, "f32", 3.0, 4, 0),       # few row tiles: one copy each way
    (700, 900, 3, "f32", 40.0, 5, 8),      # two-pass path
])
def test_host_call_equals_device_call(gb, H, W, C, in_name, sigma, K, pad):
    arr = synth.image(H, W, seed=81, dtype=in_name if in_name in ("u8", "u16") else "f32", c=C)
    h = gb.gf_create()
    try:
        for _rep in range(2):      # the second call reuses the handle's buffers and events
            got = host_filter(gb, h, arr, in_name, "f32", sigma, K, pad=pad)
            assert np.array_equal(got, device_filter(gb, arr, in_name, "f32", sigma, K))
    finally:
        gb.gf_destroy(h)


def test_host_call_matches_oracle_sampled_rows(gb):
    arr = synth.image(3000, 2048, seed=82, dtype="u8")
    h = gb.gf_create()
    try:
        got = host_filter(gb, h, arr, "u8", "f32", 6.0, 4)
    finally:
        gb.gf_destroy(h)
    r, w = ofit.fit_gaussian_boxes(6.0, 4)
    ys = [0, 1, 700, 1499, 1500, 2999]
    ref = of.filter_rows_at(arr.astype(np.float64), r, np.float32(w).astype(np.float64), "replicate", ys)
    assert rel_err(got[ys], ref) <= TOL["f32"]


def test_host_call_argument_errors(gb):
    h = gb.gf_create()
    try:
        with pytest.raises(gb.GaussboxError) as e:
            gb.gauss_filter_host(h, 1, 10, 1, 10, 4, 4, 1, 2, 2, 2.0, 3, 0, 0)   # pitches below a row
        assert e.value.status == GF_EINVAL
    finally:
        gb.gf_destroy(h)


def test_host_call_beyond_the_column_ring(gb):
    # sigma 400 (r_K 1030): the host call runs the HBM running sums
    arr = synth.image(300, 500, seed=82, dtype="u8")
    h = gb.gf_create()
    try:
        got = host_filter(gb, h, arr, "u8", "f32", 400.0, 4)
        assert np.array_equal(got, device_filter(gb, arr, "u8", "f32", 400.0, 4))
    finally:
        gb.gf_destroy(h)
