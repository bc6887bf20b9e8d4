"""Helpers shared by the GPU tests: seeded inputs in the storage dtype, pinned
host tensors, and the rounding of coefficients to the compute type."""
import numpy as np

from paper_2309_08864_gb300 import inputs, so2dr

TORCH_DTYPES = None


def torch_dtype(dtype):
    import torch
    return {so2dr.F64: torch.float64, so2dr.F32: torch.float32, so2dr.BF16: torch.bfloat16,
            so2dr.F16: torch.float16}[dtype]


def pinned_from_storage(st, dtype):
    """Pinned torch tensor holding the storage array `st` (numpy)."""
    import torch
    if dtype == so2dr.BF16:
        t = torch.from_numpy(st.view(np.int16)).view(torch.bfloat16)
    else:
        t = torch.from_numpy(st)
    return t.pin_memory()


def storage_of(t, dtype):
    """numpy float64 copy of a host tensor of the storage dtype."""
    import torch
    if dtype == so2dr.BF16:
        return inputs.bf16_bits_to_f64(t.view(torch.int16).numpy().view(np.uint16))
    return t.numpy().astype(np.float64)


def compute_coeffs(c, dtype):
    """The weights the kernels use: rounded once to the compute type."""
    c = np.asarray(c, dtype=np.float64)
    return c if dtype == so2dr.F64 else c.astype(np.float32).astype(np.float64)


def rel_linf(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def rel_l2(x, ref):
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))
