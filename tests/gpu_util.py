"""Helpers for the GPU parity tests: device transfer of seeded inputs and
tolerance arithmetic.  No method arithmetic lives here."""
import numpy as np
import pytest

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_04650_gb300 import build
    build.build()
    return torch


def to_dev(x: np.ndarray, storage: str):
    """Storage-form numpy array (see synth.as_storage) -> CUDA tensor."""
    import torch
    if storage == "bf16":
        t = torch.from_numpy(x.view(np.int16).copy()).view(torch.bfloat16)
    else:
        t = torch.from_numpy(np.ascontiguousarray(x))
    return t.cuda()


def to_np(t) -> np.ndarray:
    return t.detach().double().cpu().numpy()


def wdt(storage: str):
    import torch
    return torch.float64 if storage == "f64" else torch.float32


def unit(storage: str) -> float:
    return U64 if storage == "f64" else U32


def rel(a, b) -> float:
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def product_bound(storage, s):
    """Relative bound (times |A| |B|) of a length-s product with A stored
    as `storage`: FP64 -> (s + 2) u; FP32 and BF16 run on the tensor cores
    with FP32 accumulation (2u per add) plus the operand-split residual:
    the thin operand as bf16 hi + lo leaves at most 2^-18 of it (BF16 A:
    2^-17 covers it); FP32 A split the same way in the fused pass leaves
    another 2^-18 and the dropped A_lo B_lo term a third (3xTF32, the
    product kernel for wider panels, leaves less: 2^-19); 2^-16 covers
    both."""
    u = unit(storage)
    if storage == "bf16":
        return (s + 2) * 2 * u + 2.0 ** -17
    if storage == "f32":
        return (s + 2) * 2 * u + 2.0 ** -16
    return (s + 2) * u
