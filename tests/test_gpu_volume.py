"""GPU parity of the 3D filter (gauss_filter_volume: in-plane running-sum
filter of every slice, then the same along the slices, Sec. 3.4) against the
FP64 oracle: dtypes, boundaries, channels, anisotropic depth kernels, radii
beyond the volume, several tiles on every axis, a large volume checked on
voxel lines the oracle computes one by one, and argument errors."""
import numpy as np
import pytest

from gpu_helpers import TOL, oracle_input, rel_err, to_host, torch_dtype
from oracle import filter as of
from oracle import fit as ofit
from paper_1107_4958_gb300 import synth
from paper_1107_4958_gb300.abi_types import BOUNDARY_CODE, GF_EINVAL, GF_F32, GF_U8

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
    h = gaussbox.gf_create()
    yield gaussbox, h
    gaussbox.gf_destroy(h)
    assert gaussbox.gf_get_device_status() == 0


def volume(D, H, W, C, seed, in_name):
    v = np.stack([synth.image(H, W, seed=seed + z, dtype="u8" if in_name == "u8" else "f32", c=C)
                  for z in range(D)])
    return v


def to_dev(v, name):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(v))
    if name in ("bf16", "f16"):
        t = t.to(torch_dtype(name))
    return t.cuda()


def run(gbh, v, in_name, r, w, boundary, rz=None, wz=None, out_name="f32"):
    import torch
    gb, h = gbh
    x = to_dev(v, in_name)
    y = gb.filter_volume_tensor(h, x, radii=r, weights=w, radii_z=rz, weights_z=wz,
                                boundary=BOUNDARY_CODE[boundary], out_dtype=torch_dtype(out_name))
    torch.cuda.synchronize()
    return to_host(y)


def oracle(v, in_name, r, w, boundary, rz=None, wz=None):
    f32 = lambda a: None if a is None else np.float32(a).astype(np.float64)  # noqa: E731
    return of.filter_volume(oracle_input(v, in_name), r, f32(w), boundary, radii_z=rz, weights_z=f32(wz))


@pytest.mark.parametrize("boundary", ["replicate", "zero", "reflect"])
@pytest.mark.parametrize("in_name", ["u8", "f32", "bf16"])
def test_volume_vs_oracle(gb, boundary, in_name):
    # 300 columns: two fused strips and several depth strips; 130 rows: two row tiles
    v = volume(11, 130, 300, 1, 51, in_name)
    for sigma, K in ((1.0, 3), (4.0, 4)):
        r, w = ofit.fit_gaussian_boxes(sigma, K)
        got = run(gb, v, in_name, r, w, boundary)
        ref = oracle(v, in_name, r, w, boundary)
        assert rel_err(got, ref) <= TOL["f32"], (sigma, rel_err(got, ref))


@pytest.mark.parametrize("C", [1, 3, 4])
def test_volume_channels_anisotropic(gb, C):
    v = volume(9, 40, 70, C, 52, "f32")
    v[..., 0] += 800.0
    r, w = ofit.fit_gaussian_boxes(3.0, 3)
    rz, wz = ofit.fit_gaussian_boxes(1.5, 4)
    got = run(gb, v, "f32", r, w, "reflect", rz, wz)
    ref = oracle(v, "f32", r, w, "reflect", rz, wz)
    assert rel_err(got, ref) <= TOL["f32"]


def test_volume_large_radii_and_two_pass_slices(gb):
    # sigma 20: the stack's plan is two-pass (row launch over all rows, column
    # launch over the slices, depth launch: 3 launches); depth radii exceed the 6 slices
    gbm, h = gb
    v = volume(6, 90, 120, 1, 53, "f32")
    r, w = ofit.fit_gaussian_boxes(20.0, 5)
    for boundary in ("replicate", "zero", "reflect"):
        got = run(gb, v, "f32", r, w, boundary)
        assert gbm.gf_batch_launches(h) == 3
        ref = oracle(v, "f32", r, w, boundary)
        assert rel_err(got, ref) <= TOL["f32"], boundary


@pytest.mark.parametrize("in_name", ["u8", "u16"])
def test_volume_walk_route(gb, in_name):
    # single-channel integer stacks with radii the register walk holds: one
    # walk launch over all slices (blockIdx.z) + the depth launch.  37-row
    # slices end inside a chunk of the walk (its rows past a slice fall outside
    # the output view); 300 columns: two whole strips and a partial one
    import torch
    gbm, h = gb
    D, H, W = 7, 37, 300
    v = volume(D, H, W, 1, 59, "u8").astype(np.int32)
    if in_name == "u16":
        v = v * 251 + 3
    r, w = ofit.fit_gaussian_boxes(3.0, 4)
    tdt = torch.uint8 if in_name == "u8" else torch.uint16
    x = torch.from_numpy(v).to(tdt).cuda()
    for boundary in ("replicate", "zero", "reflect"):
        y = gbm.filter_volume_tensor(h, x, radii=r, weights=w, boundary=BOUNDARY_CODE[boundary])
        torch.cuda.synchronize()
        assert gbm.gf_batch_launches(h) == 2
        ref = of.filter_volume(v.astype(np.float64), r, np.float32(w).astype(np.float64), boundary)
        assert rel_err(to_host(y), ref) <= TOL["f32"], boundary


def test_volume_walk_route_pitched_input(gb):
    # rows padded to an odd pitch (the walk's unaligned loads) and slices of
    # one row each
    import torch
    gbm, h = gb
    D, H, W = 5, 1, 130
    v = volume(D, H, W, 1, 60, "u8")
    buf = torch.zeros((D * H, W + 3), dtype=torch.uint8, device="cuda")
    buf[:, :W] = torch.from_numpy(v.reshape(D * H, W)).cuda()
    r, w = ofit.fit_gaussian_boxes(2.0, 3)
    y = torch.empty((D, H, W), dtype=torch.float32, device="cuda")
    gbm.gauss_filter_volume(h, buf.data_ptr(), W + 3, y.data_ptr(), W * 4, D, H, W, 1, GF_U8, GF_F32, r, w, 0)
    torch.cuda.synchronize()
    ref = of.filter_volume(v.astype(np.float64), r, np.float32(w).astype(np.float64), "replicate")
    assert rel_err(to_host(y), ref) <= TOL["f32"]


def test_volume_fused_route_repeats_with_new_voxels(gb):
    # small sigma: one persistent launch over the slices + the depth launch; the
    # second call with the same buffers replays the captured batch
    import torch
    gbm, h = gb
    v = volume(10, 70, 90, 1, 58, "f32")
    r, w = ofit.fit_gaussian_boxes(2.0, 3)
    x = to_dev(v, "f32")
    y = torch.empty_like(x)
    for rep in range(3):
        x.mul_(0.5).add_(float(rep))
        gbm.filter_volume_tensor(h, x, radii=r, weights=w, out=y)
        torch.cuda.synchronize()
        assert gbm.gf_batch_launches(h) == 2
        ref = oracle(x.cpu().numpy(), "f32", r, w, "replicate")
        assert rel_err(to_host(y), ref) <= TOL["f32"], rep


def test_volume_single_slice_and_deep_stack(gb):
    r, w = ofit.fit_gaussian_boxes(2.0, 3)
    v1 = volume(1, 50, 64, 1, 54, "u8")
    got = run(gb, v1, "u8", r, w, "replicate")
    assert rel_err(got, oracle(v1, "u8", r, w, "replicate")) <= TOL["f32"]
    # many slices: several depth tiles
    vd = volume(700, 8, 40, 1, 55, "u8")
    rz, wz = ofit.fit_gaussian_boxes(12.0, 4)
    got = run(gb, vd, "u8", r, w, "reflect", rz, wz)
    assert rel_err(got, oracle(vd, "u8", r, w, "reflect", rz, wz)) <= TOL["f32"]


@pytest.mark.parametrize("out_name", ["bf16", "f16"])
def test_volume_half_outputs(gb, out_name):
    v = volume(5, 33, 80, 1, 56, "f32")
    r, w = ofit.fit_gaussian_boxes(2.5, 3)
    got = run(gb, v, "f32", r, w, "replicate", out_name=out_name)
    assert rel_err(got, oracle(v, "f32", r, w, "replicate")) <= TOL[out_name]


def test_volume_large_voxel_lines(gb):
    # 128 x 512 x 512 u8 on the default plans; the oracle filters a few (y, x)
    # lines: the in-plane window of each slice, then the depth convolution
    D, H, W = 128, 512, 512
    v = volume(D, H, W, 1, 57, "u8")
    r, w = ofit.fit_gaussian_boxes(4.0, 3)
    got = run(gb, v, "u8", r, w, "replicate")
    w64 = np.float32(w).astype(np.float64)
    kz = of.staircase_kernel(r, w64)
    for (y, x) in ((0, 0), (255, 301), (511, 511), (17, 490)):
        plane = np.array([of.filter_window_at(v[z].astype(np.float64), r, w64, "replicate", y, y + 1, x, x + 1)[0, 0]
                          for z in range(D)])
        line = of.conv1d_axis(plane, kz, 0, "replicate")
        assert rel_err(got[:, y, x], line) <= TOL["f32"], (y, x)


def test_volume_argument_errors(gb):
    import torch
    gbm, h = gb
    x = torch.zeros((4, 8, 8), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    r, w = [1, 2], [0.1, 0.1]
    for args in ((0, 8, 8), (4, 0, 8)):
        with pytest.raises(gbm.GaussboxError) as e:
            gbm.gauss_filter_volume(h, x.data_ptr(), 32, y.data_ptr(), 32, *args, 1, 2, 2, r, w, 0)
        assert e.value.status == GF_EINVAL
    with pytest.raises(gbm.GaussboxError) as e:       # in and out overlap
        gbm.gauss_filter_volume(h, x.data_ptr(), 32, x.data_ptr(), 32, 4, 8, 8, 1, 2, 2, r, w, 0)
    assert e.value.status == GF_EINVAL
