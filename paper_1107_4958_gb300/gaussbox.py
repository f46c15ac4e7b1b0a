"""Thin Python binding of the gaussbox C ABI (include/gaussbox.h).

Functions keep the C names and only marshal arguments; every step of the
filter runs in libgaussbox.so.  There is no Python or CPU fallback: if the
shared library is missing, importing this module fails.

Raw entry points take integer device addresses and a stream handle (int);
the ``*_tensor`` helpers marshal torch CUDA tensors into those calls.
"""
import ctypes
import os

import numpy as np

from . import abi_types as T

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgaussbox.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libgaussbox.so is not built (run __graft_entry__.build() or "
                      "python -m paper_1107_4958_gb300.build)")

_lib = ctypes.CDLL(LIB_PATH)

_c_int, _c_size, _vp, _c_double = ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_double
_i32p = ctypes.POINTER(ctypes.c_int32)
_dblp = ctypes.POINTER(ctypes.c_double)


def _sig(name, restype, *argtypes):
    fn = getattr(_lib, name)
    fn.restype = restype
    fn.argtypes = list(argtypes)
    return fn


_sig("gauss_fit_boxes", _c_int, _c_double, _c_int, _c_int, _i32p, _dblp)
_sig("gauss_fit_sigma0", _c_int, _c_int, _c_int, _i32p, _dblp, _dblp, _dblp)
_sig("gauss_fit_kernel", _c_int, _dblp, _c_int, _c_int, _c_int, _i32p, _dblp, _dblp)
_sig("gauss_filter", _c_int, _vp, _c_size, _vp, _c_size, _c_int, _c_int, _c_int, _c_int, _c_int,
     _c_double, _c_int, _c_int, _vp)
_sig("gauss_filter_boxes", _c_int, _vp, _c_size, _vp, _c_size, _c_int, _c_int, _c_int, _c_int, _c_int,
     _i32p, _dblp, _c_int, _c_int, _vp)
_sig("gauss_row_box_sums", _c_int, _vp, _c_size, _vp, _c_size, _c_size, _c_int, _c_int, _c_int, _c_int,
     _i32p, _c_int, _c_int, _vp)
class gf_plan(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("col_w", ctypes.c_int),
                ("col_h", ctypes.c_int), ("accum", ctypes.c_int)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_sig("gauss_filter_planned", _c_int, _vp, _c_size, _vp, _c_size, _c_int, _c_int, _c_int, _c_int, _c_int,
     _i32p, _dblp, _c_int, _c_int, ctypes.POINTER(gf_plan), _vp)
_sig("gauss_plan_default", _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _i32p, _c_int, ctypes.POINTER(gf_plan))
_sig("gauss_walker_compile", _c_int, _c_int, _i32p, _c_int, ctypes.c_char_p, _c_size)
_sig("gauss_depth_walker_compile", _c_int, _i32p, _c_int, ctypes.c_char_p, _c_size)
_sig("gauss_filter_sampled", _c_int, _vp, _c_size, _vp, _c_size, _c_int, _c_int, _c_int, _c_int, _c_int,
     _i32p, _dblp, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, ctypes.POINTER(gf_plan), _vp)


class gf_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t), ("use_graphs", ctypes.c_int),
                ("tune_cache", ctypes.c_char_p), ("wait_cycles", ctypes.c_longlong)]


class gf_image_desc(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("in_pitch", ctypes.c_size_t), ("d_out", ctypes.c_void_p),
                ("out_pitch", ctypes.c_size_t), ("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int),
                ("in_dtype", ctypes.c_int), ("out_dtype", ctypes.c_int), ("sigma", ctypes.c_double),
                ("K", ctypes.c_int), ("boundary", ctypes.c_int), ("radii", _i32p), ("weights", _dblp),
                ("plan", ctypes.POINTER(gf_plan))]


_sig("gf_create", _c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(gf_config))
_sig("gf_destroy", _c_int, ctypes.c_void_p)
_sig("gf_handle_status", _c_int, ctypes.c_void_p, _c_int)
_sig("gauss_filter_batch", _c_int, ctypes.c_void_p, ctypes.POINTER(gf_image_desc), _c_int, _vp)
_sig("gauss_filter_batch_noalloc", _c_int, ctypes.POINTER(gf_image_desc), _c_int, _vp)
_sig("gauss_filter_volume", _c_int, _vp, _vp, _c_size, _vp, _c_size, _c_int, _c_int, _c_int, _c_int, _c_int,
     _c_int, _i32p, _dblp, _c_int, _i32p, _dblp, _c_int, _c_int, _vp)


class gf_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int), ("max_inflight", ctypes.c_int),
                ("plain", ctypes.c_int)]


class gf_completion(ctypes.Structure):
    _fields_ = [("d_out", ctypes.c_void_p), ("out_pitch", ctypes.c_size_t), ("t_release", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("status", ctypes.c_int)]


class gf_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("rejected", ctypes.c_longlong),
                ("steps", ctypes.c_longlong), ("sum_batch", ctypes.c_double), ("arena_bytes", ctypes.c_size_t),
                ("arena_peak", ctypes.c_size_t), ("busy_first_release", ctypes.c_double),
                ("busy_last_done", ctypes.c_double), ("launches", ctypes.c_longlong)]


_llp = ctypes.POINTER(ctypes.c_longlong)
_sig("gf_clock_now", ctypes.c_double)
_sig("gf_server_start", _c_int, _vp, ctypes.POINTER(gf_server_config))
_sig("gf_server_submit", _c_int, _vp, ctypes.POINTER(gf_image_desc), ctypes.c_double, _c_int, _llp)
_sig("gf_server_poll", _c_int, _vp, ctypes.c_longlong, ctypes.POINTER(gf_completion))
_sig("gf_server_wait", _c_int, _vp, ctypes.c_longlong, ctypes.c_double, ctypes.POINTER(gf_completion))
_sig("gf_server_release", _c_int, _vp, ctypes.c_longlong)
_sig("gf_server_drain", _c_int, _vp, ctypes.c_double)
_sig("gf_server_stats_get", _c_int, _vp, ctypes.POINTER(gf_server_stats))
_sig("gf_server_stop", _c_int, _vp)
_sig("gauss_filter_host", _c_int, _vp, _vp, _c_size, _vp, _c_size, _c_int, _c_int, _c_int, _c_int, _c_int,
     _c_double, _c_int, _c_int, _vp)
_sig("gf_tune", _c_int, _vp, ctypes.POINTER(gf_image_desc), _vp, ctypes.POINTER(gf_plan))
_sig("gf_tuned_plan", _c_int, _vp, ctypes.POINTER(gf_image_desc), ctypes.POINTER(gf_plan))
_sig("gf_batch_launches", _c_int, _vp)
_sig("gf_get_device_status", _c_int, _c_int)
_sig("gf_status_string", ctypes.c_char_p, _c_int)
_sig("gf_version", ctypes.c_char_p)


class GaussboxError(RuntimeError):
    def __init__(self, status, where):
        self.status = int(status)
        super().__init__("%s: %s" % (where, gf_status_string(status)))


def _check(status, where):
    if status != T.GF_OK:
        raise GaussboxError(status, where)
    return status


def lib():
    """The loaded ctypes handle (for tests that check exported symbols)."""
    return _lib


def gf_create(device=0, hbm_budget_bytes=0, use_graphs=True, tune_cache=None, wait_cycles=0):
    cfg = gf_config(int(device), int(hbm_budget_bytes), 1 if use_graphs else 0,
                    tune_cache.encode() if tune_cache else None, int(wait_cycles))
    h = ctypes.c_void_p()
    _check(_lib.gf_create(ctypes.byref(h), ctypes.byref(cfg)), "gf_create")
    return h.value


def gf_destroy(handle):
    return _check(_lib.gf_destroy(ctypes.c_void_p(handle)), "gf_destroy")


def gauss_filter_batch(handle, descs, stream=0):
    """descs: sequence of gf_image_desc."""
    n = len(descs)
    arr = (gf_image_desc * max(n, 1))(*descs)
    return _check(_lib.gauss_filter_batch(ctypes.c_void_p(handle), arr, n, _vp(stream)), "gauss_filter_batch")


def gf_batch_launches(handle):
    return int(_lib.gf_batch_launches(_vp(handle)))


def gauss_filter_batch_noalloc(descs, stream=0):
    """Batch without device allocation (fixed library-owned scratch); descs: gf_image_desc."""
    n = len(descs)
    arr = (gf_image_desc * max(n, 1))(*descs)
    return _check(_lib.gauss_filter_batch_noalloc(arr, n, _vp(stream)), "gauss_filter_batch_noalloc")


def gauss_filter_host(handle, h_in, in_pitch, h_out, out_pitch, H, W, C, in_dtype, out_dtype, sigma, K, boundary,
                      stream=0):
    return _check(_lib.gauss_filter_host(_vp(handle), _vp(h_in), in_pitch, _vp(h_out), out_pitch, H, W, C, in_dtype,
                                         out_dtype, float(sigma), K, boundary, _vp(stream)), "gauss_filter_host")


def gf_clock_now():
    return float(_lib.gf_clock_now())


def gf_server_start(handle, hbm_budget_bytes=0, max_batch=0, max_inflight=0, plain=False):
    cfg = gf_server_config(int(hbm_budget_bytes), int(max_batch), int(max_inflight), 1 if plain else 0)
    return _check(_lib.gf_server_start(_vp(handle), ctypes.byref(cfg)), "gf_server_start")


def gf_server_submit(handle, desc, release_time=0.0, auto_release=False):
    t = ctypes.c_longlong()
    _check(_lib.gf_server_submit(_vp(handle), ctypes.byref(desc), float(release_time), 1 if auto_release else 0,
                                 ctypes.byref(t)), "gf_server_submit")
    return t.value


def gf_server_wait(handle, ticket, timeout_s=60.0):
    c = gf_completion()
    _check(_lib.gf_server_wait(_vp(handle), int(ticket), float(timeout_s), ctypes.byref(c)), "gf_server_wait")
    return c


def gf_server_release(handle, ticket):
    return _check(_lib.gf_server_release(_vp(handle), int(ticket)), "gf_server_release")


def gf_server_drain(handle, timeout_s=600.0):
    return _check(_lib.gf_server_drain(_vp(handle), float(timeout_s)), "gf_server_drain")


def gf_server_stats_get(handle):
    st = gf_server_stats()
    _check(_lib.gf_server_stats_get(_vp(handle), ctypes.byref(st)), "gf_server_stats_get")
    return st


def gf_server_stop(handle):
    return _check(_lib.gf_server_stop(_vp(handle)), "gf_server_stop")


def gf_tune(handle, desc, stream=0):
    """Runs the plan autotuner on one image (synchronous; its output is
    overwritten) and returns the chosen gf_plan."""
    p = gf_plan()
    _check(_lib.gf_tune(_vp(handle), ctypes.byref(desc), _vp(stream), ctypes.byref(p)), "gf_tune")
    return p


def gf_tuned_plan(handle, desc):
    """The plan tuned for desc's shape class, or None."""
    p = gf_plan()
    rc = _lib.gf_tuned_plan(_vp(handle), ctypes.byref(desc), ctypes.byref(p))
    return p if rc == T.GF_OK else None


def gf_status_string(status):
    return _lib.gf_status_string(int(status)).decode()


def gf_version():
    return _lib.gf_version().decode()


def gf_get_device_status(clear=False):
    """Sticky status word of the handle-less calls on the current device (0 = OK);
    the raw code, not raised."""
    return int(_lib.gf_get_device_status(1 if clear else 0))


def gf_handle_status(handle, clear=False):
    """Sticky status word of one handle's kernels (0 = OK); the raw code, not raised."""
    return int(_lib.gf_handle_status(ctypes.c_void_p(handle), 1 if clear else 0))


def gauss_fit_boxes(sigma, K, err_kind=T.GF_ERR_QF):
    r = (ctypes.c_int32 * K)()
    w = (ctypes.c_double * K)()
    _check(_lib.gauss_fit_boxes(float(sigma), int(K), int(err_kind), r, w), "gauss_fit_boxes")
    return np.array(list(r), dtype=np.int32), np.array(list(w), dtype=np.float64)


def gauss_fit_sigma0(K, err_kind=T.GF_ERR_QF):
    p = (ctypes.c_int32 * K)()
    c = (ctypes.c_double * K)()
    w = (ctypes.c_double * K)()
    e = ctypes.c_double()
    _check(_lib.gauss_fit_sigma0(int(K), int(err_kind), p, c, w, ctypes.byref(e)), "gauss_fit_sigma0")
    return (np.array(list(p), dtype=np.int32), np.array(list(c)), np.array(list(w)), e.value)


def gauss_fit_kernel(half, K, err_kind=T.GF_ERR_QF):
    """Radii, optimal (unnormalised) slice weights and residual error of the K-slice
    fit of the symmetric kernel with samples `half` at t = 0, 1, ..."""
    n = len(half)
    h = (ctypes.c_double * n)(*[float(v) for v in half])
    r = (ctypes.c_int32 * K)()
    w = (ctypes.c_double * K)()
    e = ctypes.c_double()
    _check(_lib.gauss_fit_kernel(h, n, K, err_kind, r, w, ctypes.byref(e)), "gauss_fit_kernel")
    return list(r), list(w), e.value


def gauss_filter(d_in, in_pitch, d_out, out_pitch, H, W, C, in_dtype, out_dtype, sigma, K, boundary,
                 stream=0):
    return _check(_lib.gauss_filter(_vp(d_in), in_pitch, _vp(d_out), out_pitch, H, W, C, in_dtype,
                                    out_dtype, float(sigma), K, boundary, _vp(stream)), "gauss_filter")


def gauss_filter_boxes(d_in, in_pitch, d_out, out_pitch, H, W, C, in_dtype, out_dtype, radii, weights,
                       boundary, stream=0):
    K = len(radii)
    r = (ctypes.c_int32 * K)(*[int(v) for v in radii])
    w = (ctypes.c_double * K)(*[float(v) for v in weights])
    return _check(_lib.gauss_filter_boxes(_vp(d_in), in_pitch, _vp(d_out), out_pitch, H, W, C, in_dtype,
                                          out_dtype, r, w, K, boundary, _vp(stream)),
                  "gauss_filter_boxes")


def make_plan(path=T.GF_PATH_AUTO, tile_w=0, tile_h=0, col_w=0, col_h=0, accum=T.GF_ACCUM_COMPENSATED):
    return gf_plan(int(path), int(tile_w), int(tile_h), int(col_w), int(col_h), int(accum))


def gauss_walker_compile(in_dtype, radii):
    """Compiles the GF_PATH_WALK kernels for these radii (no device needed).
    Returns (status, compiler log)."""
    r = (ctypes.c_int32 * len(radii))(*[int(v) for v in radii])
    buf = ctypes.create_string_buffer(1 << 16)
    st = int(_lib.gauss_walker_compile(int(in_dtype), r, len(radii), buf, len(buf)))
    return st, buf.value.decode(errors="replace")


def gauss_depth_walker_compile(radii):
    """Compiles the volumes' depth walk for these depth radii (no device
    needed).  Returns (status, compiler log)."""
    r = (ctypes.c_int32 * len(radii))(*[int(v) for v in radii])
    buf = ctypes.create_string_buffer(1 << 16)
    st = int(_lib.gauss_depth_walker_compile(r, len(radii), buf, len(buf)))
    return st, buf.value.decode(errors="replace")


def gauss_plan_default(H, W, C, in_dtype, out_dtype, radii):
    K = len(radii)
    r = (ctypes.c_int32 * K)(*[int(v) for v in radii])
    p = gf_plan()
    _check(_lib.gauss_plan_default(H, W, C, in_dtype, out_dtype, r, K, ctypes.byref(p)), "gauss_plan_default")
    return p


def gauss_filter_planned(d_in, in_pitch, d_out, out_pitch, H, W, C, in_dtype, out_dtype, radii, weights,
                         boundary, plan=None, stream=0):
    K = len(radii)
    r = (ctypes.c_int32 * K)(*[int(v) for v in radii])
    w = (ctypes.c_double * K)(*[float(v) for v in weights])
    pp = ctypes.byref(plan) if plan is not None else None
    return _check(_lib.gauss_filter_planned(_vp(d_in), in_pitch, _vp(d_out), out_pitch, H, W, C, in_dtype,
                                            out_dtype, r, w, K, boundary, pp, _vp(stream)),
                  "gauss_filter_planned")


def gauss_filter_sampled(d_in, in_pitch, d_out, out_pitch, H, W, C, in_dtype, out_dtype, radii, weights,
                         boundary, step_y, step_x, off_y=0, off_x=0, plan=None, stream=0):
    K = len(radii)
    r = (ctypes.c_int32 * K)(*[int(v) for v in radii])
    w = (ctypes.c_double * K)(*[float(v) for v in weights])
    pp = ctypes.byref(plan) if plan is not None else None
    return _check(_lib.gauss_filter_sampled(_vp(d_in), in_pitch, _vp(d_out), out_pitch, H, W, C, in_dtype,
                                            out_dtype, r, w, K, boundary, int(step_y), int(step_x), int(off_y),
                                            int(off_x), pp, _vp(stream)),
                  "gauss_filter_sampled")


def gauss_filter_volume(handle, d_in, in_pitch, d_out, out_pitch, D, H, W, C, in_dtype, out_dtype, radii,
                        weights, boundary, radii_z=None, weights_z=None, stream=0):
    K = len(radii)
    r = (ctypes.c_int32 * K)(*[int(v) for v in radii])
    w = (ctypes.c_double * K)(*[float(v) for v in weights])
    if radii_z is None:
        rz, wz, Kz = None, None, 0
    else:
        Kz = len(radii_z)
        rz = (ctypes.c_int32 * Kz)(*[int(v) for v in radii_z])
        wz = (ctypes.c_double * Kz)(*[float(v) for v in weights_z])
    return _check(_lib.gauss_filter_volume(handle, _vp(d_in), in_pitch, _vp(d_out), out_pitch, D, H, W, C,
                                           in_dtype, out_dtype, r, w, K, rz, wz, Kz, boundary, _vp(stream)),
                  "gauss_filter_volume")


def gauss_row_box_sums(d_in, in_pitch, d_out, out_pitch, plane_stride_elems, H, W, C, in_dtype, radii,
                       boundary, stream=0):
    K = len(radii)
    r = (ctypes.c_int32 * K)(*[int(v) for v in radii])
    return _check(_lib.gauss_row_box_sums(_vp(d_in), in_pitch, _vp(d_out), out_pitch, plane_stride_elems,
                                          H, W, C, in_dtype, r, K, boundary, _vp(stream)),
                  "gauss_row_box_sums")


# ---------------------------------------------------------------- torch marshalling
def _torch():
    import torch  # noqa: PLC0415  (torch only marshals device memory and streams)
    return torch


def _geom(x):
    if x.dim() == 2:
        return x.shape[0], x.shape[1], 1
    if x.dim() == 3:
        return x.shape[0], x.shape[1], x.shape[2]
    raise ValueError("expected (H, W) or (H, W, C)")


def _pitch(x):
    """Row pitch in bytes of an (H, W[, C]) tensor whose rows may be padded."""
    H, W, C = _geom(x)
    if x.dim() == 3 and (x.stride(2) != 1 or x.stride(1) != C):
        raise ValueError("pixels must be contiguous within a row")
    if x.dim() == 2 and x.stride(1) != 1:
        raise ValueError("pixels must be contiguous within a row")
    return x.stride(0) * x.element_size()


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def filter_tensor(x, sigma=None, K=4, boundary=T.GF_REPLICATE, out_dtype=None, out=None, radii=None,
                  weights=None, stream=None, plan=None):
    """Filters a CUDA tensor (H, W) or (H, W, C) into `out` (allocated if None).
    `plan` (a gf_plan) forces a path / tile shapes; the boxes then come from
    `radii`/`weights` or from fitting `sigma`, K."""
    torch = _torch()
    H, W, C = _geom(x)
    in_dt = T.dtype_code(x.dtype)
    if out is None:
        od = out_dtype if out_dtype is not None else (torch.float32 if in_dt in (T.GF_U8, T.GF_U16)
                                                      else x.dtype)
        out = torch.empty(x.shape, dtype=od, device=x.device)
    s = _stream_handle(stream)
    if plan is not None:
        if radii is None:
            radii, weights = gauss_fit_boxes(sigma, K)
        gauss_filter_planned(x.data_ptr(), _pitch(x), out.data_ptr(), _pitch(out), H, W, C, in_dt,
                             T.dtype_code(out.dtype), radii, weights, boundary, plan, s)
    elif radii is not None:
        gauss_filter_boxes(x.data_ptr(), _pitch(x), out.data_ptr(), _pitch(out), H, W, C, in_dt,
                           T.dtype_code(out.dtype), radii, weights, boundary, s)
    else:
        gauss_filter(x.data_ptr(), _pitch(x), out.data_ptr(), _pitch(out), H, W, C, in_dt,
                     T.dtype_code(out.dtype), sigma, K, boundary, s)
    return out


def sampled_shape(H, W, step_y, step_x, off_y=0, off_x=0):
    """Output rows and columns of gauss_filter_sampled."""
    return (H - off_y + step_y - 1) // step_y, (W - off_x + step_x - 1) // step_x


def filter_sampled_tensor(x, step, offset=(0, 0), sigma=None, K=4, boundary=T.GF_REPLICATE, out_dtype=None,
                          out=None, radii=None, weights=None, stream=None, plan=None):
    """The filter of `x` (H, W[, C]) at pixels (off_y + i step_y, off_x + j step_x)
    only; `step` and `offset` are (y, x) pairs.  Returns the (Ho, Wo[, C]) result."""
    torch = _torch()
    H, W, C = _geom(x)
    sy, sx = int(step[0]), int(step[1])
    oy, ox = int(offset[0]), int(offset[1])
    in_dt = T.dtype_code(x.dtype)
    if radii is None:
        radii, weights = gauss_fit_boxes(sigma, K)
    Ho, Wo = sampled_shape(H, W, sy, sx, oy, ox)
    if out is None:
        od = out_dtype if out_dtype is not None else (torch.float32 if in_dt in (T.GF_U8, T.GF_U16)
                                                      else x.dtype)
        shape = (Ho, Wo) if x.dim() == 2 else (Ho, Wo, C)
        out = torch.empty(shape, dtype=od, device=x.device)
    gauss_filter_sampled(x.data_ptr(), _pitch(x), out.data_ptr(), _pitch(out), H, W, C, in_dt,
                         T.dtype_code(out.dtype), radii, weights, boundary, sy, sx, oy, ox, plan,
                         _stream_handle(stream))
    return out


def _volume_geom(x):
    if x.dim() == 3:
        return x.shape[0], x.shape[1], x.shape[2], 1
    if x.dim() == 4:
        return x.shape[0], x.shape[1], x.shape[2], x.shape[3]
    raise ValueError("expected (D, H, W) or (D, H, W, C)")


def _volume_pitch(x):
    """Row pitch of a (D, H, W[, C]) tensor whose slices are stacked rows of one pitch."""
    D, H, W, C = _volume_geom(x)
    if x.stride(-1) != 1 or (x.dim() == 4 and x.stride(2) != C):
        raise ValueError("pixels must be contiguous within a row")
    if x.stride(0) != H * x.stride(1):
        raise ValueError("slices must follow each other row after row (slice stride = H x row stride)")
    return x.stride(1) * x.element_size()


def filter_volume_tensor(handle, x, sigma=None, K=4, boundary=T.GF_REPLICATE, out_dtype=None, out=None,
                         radii=None, weights=None, sigma_z=None, radii_z=None, weights_z=None, stream=None):
    """3D filter of a CUDA tensor (D, H, W) or (D, H, W, C): in-plane boxes from
    `radii`/`weights` or `sigma`, K; the depth boxes from `radii_z`/`weights_z`,
    `sigma_z` (with K) or, if neither is given, the in-plane ones."""
    torch = _torch()
    D, H, W, C = _volume_geom(x)
    in_dt = T.dtype_code(x.dtype)
    if radii is None:
        radii, weights = gauss_fit_boxes(sigma, K)
    if radii_z is None and sigma_z is not None:
        radii_z, weights_z = gauss_fit_boxes(sigma_z, K)
    if out is None:
        od = out_dtype if out_dtype is not None else (torch.float32 if in_dt in (T.GF_U8, T.GF_U16)
                                                      else x.dtype)
        out = torch.empty(x.shape, dtype=od, device=x.device)
    gauss_filter_volume(handle, x.data_ptr(), _volume_pitch(x), out.data_ptr(), _volume_pitch(out), D, H, W, C,
                        in_dt, T.dtype_code(out.dtype), radii, weights, boundary, radii_z, weights_z,
                        _stream_handle(stream))
    return out


def _attach_plan(d, plan):
    if plan is not None:
        d.plan = ctypes.pointer(plan)
        d._keep_plan = plan
    return d


def image_desc(x, out, sigma=None, K=4, boundary=T.GF_REPLICATE, radii=None, weights=None, plan=None):
    """gf_image_desc for CUDA tensors x -> out (explicit boxes if radii/weights
    given; `plan` a gf_plan or None for the default)."""
    H, W, C = _geom(x)
    d = gf_image_desc(x.data_ptr(), _pitch(x), out.data_ptr(), _pitch(out), H, W, C, T.dtype_code(x.dtype),
                      T.dtype_code(out.dtype), float(sigma or 0.0), int(K if radii is None else len(radii)),
                      int(boundary), None, None, None)
    if radii is not None:
        r = (ctypes.c_int32 * len(radii))(*[int(v) for v in radii])
        w = (ctypes.c_double * len(weights))(*[float(v) for v in weights])
        d.radii = ctypes.cast(r, _i32p)
        d.weights = ctypes.cast(w, _dblp)
        d._keep = (r, w)
    return _attach_plan(d, plan)


def request_desc(x, out_dtype, sigma=None, K=4, boundary=T.GF_REPLICATE, plan=None):
    """gf_image_desc for a server request: input tensor x, output dtype only
    (the server provides the output buffer)."""
    H, W, C = _geom(x)
    d = gf_image_desc(x.data_ptr(), _pitch(x), None, 0, H, W, C, T.dtype_code(x.dtype),
                      T.dtype_code(out_dtype), float(sigma or 0.0), int(K), int(boundary), None, None, None)
    return _attach_plan(d, plan)


class _DeviceView:
    def __init__(self, ptr, shape, typestr, strides=None):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": strides}


def completion_tensor(comp, H, W, C, out_dtype):
    """Zero-copy torch view (H, W[, C]) of a completed request's output buffer."""
    torch = _torch()
    code = T.dtype_code(out_dtype)
    esz = T.DTYPE_BYTES[code]
    typestr = {T.GF_F32: "<f4", T.GF_F16: "<f2", T.GF_BF16: "<u2"}[code]
    shape = (H, W, C) if C > 1 else (H, W)
    strides = (comp.out_pitch, C * esz, esz) if C > 1 else (comp.out_pitch, esz)
    t = torch.as_tensor(_DeviceView(comp.d_out, shape, typestr, strides), device="cuda")
    return t.view(torch.bfloat16) if code == T.GF_BF16 else t


def filter_batch_tensors(handle, xs, outs, sigmas, Ks, boundary=T.GF_REPLICATE, stream=None, plans=None):
    """Filters CUDA tensors xs[i] -> outs[i] with one gauss_filter_batch call."""
    plans = plans if plans is not None else [None] * len(xs)
    descs = [image_desc(x, o, s, k, boundary, plan=p) for x, o, s, k, p in zip(xs, outs, sigmas, Ks, plans)]
    gauss_filter_batch(handle, descs, _stream_handle(stream))
    return outs


def row_box_sums_tensor(x, radii, boundary=T.GF_REPLICATE, stream=None):
    """K int32 planes of exact row box sums of a uint8 / uint16 CUDA tensor."""
    torch = _torch()
    H, W, C = _geom(x)
    K = len(radii)
    out = torch.empty((K,) + tuple(x.shape), dtype=torch.int32, device=x.device)
    plane = out[0].numel()
    gauss_row_box_sums(x.data_ptr(), _pitch(x), out.data_ptr(), W * C * 4, plane, H, W, C,
                       T.dtype_code(x.dtype), radii, boundary, _stream_handle(stream))
    return out
