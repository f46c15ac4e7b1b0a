"""Codes of include/gaussbox.h mirrored for Python (no library needed)."""
GF_OK, GF_EINVAL, GF_ENOMEM, GF_ECUDA, GF_ETIMEOUT, GF_EUNSUPPORTED, GF_EADMIT, GF_EBUSY, GF_ELIMIT = range(9)
GF_NOALLOC_MAX_IMAGES = 64
GF_NOALLOC_SCRATCH_BYTES = 64 * 1024
GF_U8, GF_U16, GF_F32, GF_BF16, GF_F16 = range(5)
GF_REPLICATE, GF_ZERO, GF_REFLECT = range(3)
GF_ERR_QF, GF_ERR_L2 = range(2)
GF_KMAX = 5
GF_PATH_AUTO, GF_PATH_FUSED, GF_PATH_TWO_PASS, GF_PATH_HBM, GF_PATH_WALK = range(5)
GF_ACCUM_COMPENSATED, GF_ACCUM_OFFSET, GF_ACCUM_PLAIN = range(3)

BOUNDARY_CODE = {"replicate": GF_REPLICATE, "zero": GF_ZERO, "reflect": GF_REFLECT}
DTYPE_NAME = {GF_U8: "u8", GF_U16: "u16", GF_F32: "f32", GF_BF16: "bf16", GF_F16: "f16"}
DTYPE_BYTES = {GF_U8: 1, GF_U16: 2, GF_F32: 4, GF_BF16: 2, GF_F16: 2}


def dtype_code(torch_dtype):
    import torch  # noqa: PLC0415
    table = {torch.uint8: GF_U8, torch.uint16: GF_U16, torch.float32: GF_F32,
             torch.bfloat16: GF_BF16, torch.float16: GF_F16}
    if torch_dtype not in table:
        raise ValueError("unsupported dtype %s" % (torch_dtype,))
    return table[torch_dtype]
