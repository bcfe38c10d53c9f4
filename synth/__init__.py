"""Seeded synthetic inputs for compressed NMF / SNMF.

This module is shared by the FP64 oracle (``oracle/``) and by the GPU path
(tests, bench, smoke).  It holds only the input recipe -- random draws with
NumPy's PCG64 and the products that *define* a synthetic matrix -- and none of
the method's arithmetic (no compression, no factorization, no column
selection).  Every input is produced in FP64, row-major, and then cast by the
caller (``as_storage``) to the storage type the GPU reads.

Recipes (the paper's synthetic generator, Sec. V-A, with the shapes of its
workloads):

* ``lowrank``:   A = X0 . Y0 + |N(0, sigma^2)|, X0 (m x r), Y0 (r x n) i.i.d.
                 Uniform[0, 1).  Draw order: X0, then Y0, then the noise.
* ``separable``: A = X0 . [I_r | H] . Pi + |N(0, sigma^2)|; X0 Uniform[0,1);
                 columns of H Dirichlet(1) (i.i.d. Exp(1) normalised to sum
                 1); Pi a seeded permutation with A[:, perm[j]] = M[:, j], so
                 the planted anchor columns are perm[0:r].  Draw order: X0, H,
                 perm, noise.  (Sec. I, r-separable matrices; Sec. V-B.)
* ``init_factors``: U0 (m x r) then V0 (r x n), i.i.d. Uniform[0, 1).
* ``gaussian``:  explicit Gaussian test matrices (Omega n x d, then Psi m x d)
                 when a test wants to pass them in instead of using the
                 counter-based generator.

Large matrices are generated in row blocks; PCG64 draws are consumed in
order, so blocking does not change the values.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "CONFIGS", "lowrank", "separable", "init_factors", "gaussian",
    "as_storage", "bf16_round", "widen", "lowrank_torch", "init_torch",
    "separable_torch",
]

# Workload shapes: a small FP64 case, the large FP32 case, the wide separable
# case and the mixed-precision case; seeds data 1000+i, sketch 2000+i,
# init 3000+i.
CONFIGS = {
    0: dict(kind="lowrank", m=500, n=400, r=10, d=20, q=4, iters=100,
            sigma=0.01, dtype="f64"),
    1: dict(kind="lowrank", m=20000, n=10000, r=20, d=30, q=4, iters=500,
            sigma=0.01, dtype="f32"),
    2: dict(kind="separable", m=10000, n=100000, r=50, d=60, q=2,
            sigma=1e-3, dtype="f32"),
    3: dict(kind="lowrank", m=50000, n=50000, r=64, d=80, q=4, iters=200,
            sigma=0.01, dtype="bf16"),
}


def data_seed(cfg: int) -> int:
    return 1000 + cfg


def sketch_seed(cfg: int) -> int:
    return 2000 + cfg


def init_seed(cfg: int) -> int:
    return 3000 + cfg


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _noise_rows(g, rows, n, sigma, out, out_dtype, block):
    """Add |N(0, sigma^2)| to ``out`` in row blocks (draw order = row-major)."""
    for i0 in range(0, rows, block):
        i1 = min(rows, i0 + block)
        nz = np.abs(g.standard_normal((i1 - i0, n))) * sigma
        out[i0:i1] = (out[i0:i1].astype(np.float64) + nz).astype(out_dtype)


def lowrank(m: int, n: int, r: int, sigma: float, seed: int,
            dtype=np.float64, block: int = 2048, with_factors: bool = False):
    """A = X0 Y0 + |N(0, sigma^2)| (noiseless when sigma == 0).

    ``dtype`` is the dtype of the returned A (values are formed in FP64 and
    rounded once).  Returns A, or (A, X0, Y0) with ``with_factors``.
    """
    g = _rng(seed)
    X0 = g.random((m, r))
    Y0 = g.random((r, n))
    A = np.empty((m, n), dtype=dtype)
    for i0 in range(0, m, block):
        i1 = min(m, i0 + block)
        blk = X0[i0:i1] @ Y0
        if sigma > 0:
            blk = blk + np.abs(g.standard_normal((i1 - i0, n))) * sigma
        A[i0:i1] = blk.astype(dtype)
    if with_factors:
        return A, X0, Y0
    return A


def separable(m: int, n: int, r: int, sigma: float, seed: int,
              dtype=np.float64, block: int = 1024):
    """Near-separable A = X0 [I_r | H] Pi + |N(0, sigma^2)|.

    Returns (A, anchors) where ``anchors`` (int64, length r) are the planted
    extreme-column indices in the order of the identity block.
    """
    g = _rng(seed)
    X0 = g.random((m, r))
    E = g.standard_exponential((r, n - r))
    H = E / E.sum(axis=0, keepdims=True)
    perm = g.permutation(n)
    # M = X0 [I | H]; A[:, perm[j]] = M[:, j]
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    A = np.empty((m, n), dtype=dtype)
    W = np.concatenate([np.eye(r), H], axis=1)[:, inv]  # r x n, permuted
    for i0 in range(0, m, block):
        i1 = min(m, i0 + block)
        blk = X0[i0:i1] @ W
        if sigma > 0:
            blk = blk + np.abs(g.standard_normal((i1 - i0, n))) * sigma
        A[i0:i1] = blk.astype(dtype)
    return A, perm[:r].astype(np.int64)


def init_factors(m: int, n: int, r: int, seed: int):
    """U0 (m x r) then V0 (r x n), i.i.d. Uniform[0, 1), FP64."""
    g = _rng(seed)
    U0 = g.random((m, r))
    V0 = g.random((r, n))
    return U0, V0


def gaussian(n: int, m: int, d: int, seed: int):
    """Explicit Gaussian test matrices: Omega (n x d) then Psi (m x d)."""
    g = _rng(seed)
    return g.standard_normal((n, d)), g.standard_normal((m, d))


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even); returned as uint16 bits."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) >> 16
    return u.astype(np.uint16)


def widen(x: np.ndarray, storage: str) -> np.ndarray:
    """FP64 copy of the values a GPU kernel reads from ``x`` (storage form)."""
    if storage == "bf16":
        u = x.astype(np.uint32) << 16
        return u.view(np.float32).astype(np.float64)
    return np.asarray(x, dtype=np.float64)


def as_storage(A64: np.ndarray, storage: str) -> np.ndarray:
    """Cast an FP64 matrix to its storage form: f64, f32 or bf16 (uint16 bits)."""
    if storage == "f64":
        return np.ascontiguousarray(A64, dtype=np.float64)
    if storage == "f32":
        return np.ascontiguousarray(A64, dtype=np.float32)
    if storage == "bf16":
        return bf16_round(A64)
    raise ValueError(storage)


def lowrank_torch(m: int, n: int, r: int, sigma: float, seed: int,
                  device="cuda"):
    """The low-rank recipe drawn with PyTorch's generator on `device`
    (X0, then Y0, then the noise; FP32), for workloads too large to draw on
    the host.  The same (shape, seed, device type) gives the same matrix;
    copy it to the host to feed the oracle."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    X0 = torch.rand(m, r, generator=g, device=device)
    Y0 = torch.rand(r, n, generator=g, device=device)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        A = X0 @ Y0
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    if sigma > 0:
        A += torch.randn(m, n, generator=g, device=device).abs_() * sigma
    return A


def init_torch(m: int, n: int, r: int, seed: int, device="cuda"):
    """U0 (m x r) then V0^T (n x r), i.i.d. Uniform[0, 1), FP32, drawn with
    PyTorch's generator on `device`."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    U0 = torch.rand(m, r, generator=g, device=device)
    V0 = torch.rand(r, n, generator=g, device=device)
    return U0, V0.t().contiguous()


def separable_torch(m: int, n: int, r: int, sigma: float, seed: int,
                    device="cuda"):
    """The separable recipe drawn with PyTorch's generator on `device`
    (X0, then the Exp(1) draws of H, then the permutation, then the noise;
    FP32): A = X0 [I_r | H] Pi + |N(0, sigma^2)| with A[:, perm[j]] equal to
    column j of X0 [I_r | H].  Returns (A, anchors = perm[:r]) on `device`."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    X0 = torch.rand(m, r, generator=g, device=device)
    E = torch.empty(r, n - r, device=device).exponential_(1.0, generator=g)
    H = E / E.sum(dim=0, keepdim=True)
    perm = torch.randperm(n, generator=g, device=device)
    W = torch.cat([torch.eye(r, device=device), H], dim=1)
    Wp = torch.empty_like(W)
    Wp[:, perm] = W
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        A = X0 @ Wp
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    if sigma > 0:
        A += torch.randn(m, n, generator=g, device=device).abs_() * sigma
    return A, perm[:r].clone()
