"""Compressed alternating NMF (Alg. 2, Sec. III) with its two inner solvers.

TEST INFRASTRUCTURE -- only tests, the smoke check and the benchmark's
CPU-baseline leg call this.  FP64 NumPy / SciPy.

Alg. 2 works on A-check = A R^T (m x d) and A-hat = L^T A (d x n) with the
compression matrices of Alg. 1.  One iteration, in the printed order:
    Y-check = Y R^T                                  (r x d)
    X <- X' >= 0 with ||A-check - X' Y-check||_F <= ||A-check - X Y-check||_F
    X-hat = L^T X                                    (d x r)
    Y <- Y' >= 0 with ||A-hat - X-hat Y'||_F <= ||A-hat - X-hat Y||_F
The paper allows any multiplicative update or any nonnegative least-squares
method for the two steps and uses, in its experiments, an active-set NNLS
(Kim & Park 2008) and the multiplicative updates of Ding, Li & Jordan
(2010, Eq. 8).  Both are here:

``als``  -- each step solved exactly: every row of X (resp. column of Y) is
           an NNLS problem with the shared matrix Y-check^T (resp. X-hat);
           SciPy's Lawson-Hanson active-set NNLS per row / column (a library
           routine used as one step).  Exact block minimisation, so each
           step can only lower its objective.

``mu``   -- the semi-NMF multiplicative update of Ding et al.: the
           compressed matrices have entries of both signs, so with
           P = A-check Y-check^T, Q = Y-check Y-check^T and the positive /
           negative parts B+ = (|B| + B) / 2, B- = (|B| - B) / 2,
               X <- X * sqrt((P+ + X Q-) / (P- + X Q+))
           entrywise, and the same for Y^T from A-hat^T and X-hat.  Ding et
           al. prove the objective does not increase.  An entry that is
           zero stays zero; a zero denominator is floored at 1e-300 (a
           reading: the paper and Ding et al. leave it open).
"""
from __future__ import annotations

import numpy as np


def _nnls_rows(M: np.ndarray, Bt: np.ndarray) -> np.ndarray:
    """argmin_{x >= 0} ||M[i] - x Bt|| for every row i (Bt: r x d)."""
    from scipy.optimize import nnls
    B = Bt.T                              # d x r
    out = np.empty((M.shape[0], Bt.shape[0]))
    for i in range(M.shape[0]):
        out[i], _ = nnls(B, M[i])
    return out


def _pos(B):
    return (np.abs(B) + B) / 2.0


def _neg(B):
    return (np.abs(B) - B) / 2.0


def _mu_step(X: np.ndarray, M: np.ndarray, F: np.ndarray) -> np.ndarray:
    """One semi-NMF multiplicative update of X >= 0 for min ||M - X F||
    (F: r x d, any signs) -- Ding, Li & Jordan 2010, Eq. 8 (transposed)."""
    P = M @ F.T
    Q = F @ F.T
    num = _pos(P) + X @ _neg(Q)
    den = _neg(P) + X @ _pos(Q)
    return X * np.sqrt(num / np.maximum(den, 1e-300))


def iterate(Acheck, Ahat, L, Rt, X0, Y0, iters: int, solver: str = "als",
            history=None):
    """Alg. 2 for `iters` iterations from (X0, Y0); solver "als" or "mu".
    With `history` (a list), appends per iteration the two compressed
    objectives before and after each step:
    (||Ac - X Yc||, ||Ac - X' Yc||, ||Ah - Xh Y||, ||Ah - Xh Y'||)."""
    X = np.array(X0, dtype=np.float64, copy=True)
    Y = np.array(Y0, dtype=np.float64, copy=True)
    for _ in range(iters):
        Yc = Y @ Rt                                   # r x d
        before_x = np.linalg.norm(Acheck - X @ Yc)
        if solver == "als":
            X = _nnls_rows(Acheck, Yc)
        else:
            X = _mu_step(X, Acheck, Yc)
        after_x = np.linalg.norm(Acheck - X @ Yc)
        Xh = L.T @ X                                  # d x r
        before_y = np.linalg.norm(Ahat - Xh @ Y)
        if solver == "als":
            Y = _nnls_rows(Ahat.T, Xh.T).T
        else:
            Y = _mu_step(Y.T, Ahat.T, Xh.T).T
        after_y = np.linalg.norm(Ahat - Xh @ Y)
        if history is not None:
            history.append((before_x, after_x, before_y, after_y))
    return X, Y
