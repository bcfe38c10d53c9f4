"""Relative reconstruction error and the compressed objective.  FP64 oracle.

TEST INFRASTRUCTURE -- only tests, the smoke check and the benchmark's
CPU-baseline leg call this.

The paper reports the relative reconstruction error ||A - U V||_F / ||A||_F
(Sec. V) and minimises ||Atilde - Xt Yt||_F (compressed problem, Sec. III).
Both are formed explicitly here.
"""
from __future__ import annotations

import numpy as np


def residual_sq(A, U, V):
    """(||A - U V||_F^2, ||A||_F^2) with A - U V formed explicitly."""
    A = np.asarray(A, dtype=np.float64)
    E = A - U @ V
    return float(np.sum(E * E)), float(np.sum(A * A))


def rel_residual(A, U, V) -> float:
    e2, a2 = residual_sq(A, U, V)
    return float(np.sqrt(e2 / a2))


def compressed_objective(Atilde, Xt, Yt) -> float:
    return float(np.linalg.norm(Atilde - Xt @ Yt))


def svd_floor(A, r: int) -> float:
    """Eckart-Young: the smallest ||A - Z||_F / ||A||_F over rank-r Z."""
    s = np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)
    return float(np.sqrt(np.sum(s[r:] ** 2) / np.sum(s ** 2)))
