"""Helpers for the GPU parity tests: device images with optional row padding,
the exact values the oracle must see for each input dtype, and the error
metrics the tolerances are stated in."""
import numpy as np

DT_TORCH = None


def torch_dtype(name):
    import torch
    return {"u8": torch.uint8, "u16": torch.uint16, "f32": torch.float32, "bf16": torch.bfloat16,
            "f16": torch.float16}[name]


def to_device(arr, name, pad_elems=0):
    """CUDA tensor of dtype `name` holding `arr` (float arrays are rounded to the
    dtype); rows padded by `pad_elems` elements when nonzero (pitched layout)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(arr))
    if name in ("bf16", "f16"):
        t = t.to(torch_dtype(name))
    elif name == "u16":
        t = torch.from_numpy(np.ascontiguousarray(arr).astype(np.int32)).to(torch.uint16)
    t = t.cuda()
    if pad_elems:
        shape = tuple(t.shape)
        row = int(np.prod(shape[1:]))
        buf = torch.zeros((shape[0], row + pad_elems), dtype=t.dtype, device=t.device)
        buf[:, :row] = t.reshape(shape[0], row)
        strides = (row + pad_elems,) + tuple(t.stride()[1:])
        t = buf.as_strided(shape, strides)
    return t


def oracle_input(arr, name):
    """float64 values the device actually holds for `arr` stored as `name`."""
    import torch
    if name in ("bf16", "f16"):
        return torch.from_numpy(np.ascontiguousarray(arr)).to(torch_dtype(name)).double().numpy()
    return np.asarray(arr, dtype=np.float64)


def to_host(t):
    import torch
    return t.to(torch.float64).cpu().numpy() if t.dtype != torch.int32 else t.cpu().numpy()


def rel_err(got, ref, floor_frac=1e-3):
    """max |got - ref| / max(|ref|, floor_frac * mean |ref|): the error of each
    pixel relative to its own magnitude, with the denominator floored at
    1e-3 of the image's mean magnitude (the parity bar of the measurement
    contract), so that exactly-zero outputs do not divide by zero while
    outputs far below the mean are still held to their own scale."""
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    floor = max(floor_frac * float(np.mean(np.abs(ref))), 1e-30)
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def rms_rel(got, ref):
    ref = np.asarray(ref, np.float64)
    scale = max(float(np.sqrt(np.mean(ref * ref))), 1e-30)
    return float(np.sqrt(np.mean((np.asarray(got, np.float64) - ref) ** 2)) / scale)


# Tolerances (derivation in the design notes): FP32 output within 1e-5 relative;
# half-precision storage adds its own rounding (2^-9 bf16, 2^-12 f16) to that.
TOL = {"f32": 1e-5, "bf16": 2.0 ** -8, "f16": 2.0 ** -10}
