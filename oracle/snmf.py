"""Compressed separable NMF (Alg. 3): column selection with SPA (steps 1-2)
and the right factor (step 3).

TEST INFRASTRUCTURE -- only tests, the smoke check and the benchmark's
CPU-baseline leg call this.  FP64 NumPy.

Alg. 3 computes Q with Alg. 1, forms the small matrix Rhat = Q^T A
(d x n; the paper calls it R, which clashes with the NMF compression R) and
finds r extreme columns of Rhat.  The paper uses the successive projection
algorithm (SPA; Araujo et al. 2001, Gillis & Vavasis 2014) but does not
spell it out; this is its standard greedy form:
    repeat r times:
        j* = argmax_j ||Rhat[:, j]||_2^2     (ties -> lowest index)
        u  = Rhat[:, j*] / ||Rhat[:, j*]||
        Rhat <- (I - u u^T) Rhat
The column norms are recomputed from the explicitly projected matrix at
every step.

Step 3 solves, for every column i, the nonnegative least-squares problem
    Y[:, i] = argmin_{h >= 0} ||Rhat[:, i] - Rhat[:, K] h||_2
(h has r entries, one per selected column; the printed h in R^{r + r_ov}
reads as a slip, since Rhat[:, K] has r columns).  ``right_factor`` calls
SciPy's Lawson-Hanson NNLS per column, a library routine used as one step;
when Rhat[:, K] has full column rank the minimiser is unique.  K is returned in selection order, together with the per-step
margin mu_k = (N1 - N2) / N1 over the two largest squared norms, which
tells a test whether the selection is decided with room to spare.
"""
from __future__ import annotations

import numpy as np

from .compress import snmf_basis


def spa(Rhat: np.ndarray, r: int):
    """SPA on the columns of Rhat (d x n).  Returns (K int64[r], margins)."""
    W = np.array(Rhat, dtype=np.float64, copy=True)
    K = np.empty(r, dtype=np.int64)
    margins = np.empty(r)
    for k in range(r):
        nrm = np.einsum("ij,ij->j", W, W)
        j = int(np.argmax(nrm))                  # first maximum = lowest index
        top = nrm[j]
        rest = np.delete(nrm, j)
        second = rest.max() if rest.size else 0.0
        margins[k] = (top - second) / top if top > 0 else 0.0
        K[k] = j
        u = W[:, j] / np.sqrt(top)
        W = W - np.outer(u, u @ W)
    return K, margins


def snmf_select(A: np.ndarray, Omega: np.ndarray, r: int, q: int):
    """Alg. 3 steps 1-2: Q = Alg.1(A); K = SPA(Q^T A).

    Returns (K, margins, Q, Rhat).
    """
    Q, Rhat = snmf_basis(A, Omega, q)
    K, margins = spa(Rhat, r)
    return K, margins, Q, Rhat


def right_factor(Rhat: np.ndarray, K) -> np.ndarray:
    """Alg. 3 step 3: Y (r x n), column i the NNLS fit of Rhat[:, i] by the
    selected columns Rhat[:, K] (FP64, SciPy's Lawson-Hanson per column)."""
    from scipy.optimize import nnls
    R = np.asarray(Rhat, dtype=np.float64)
    B = R[:, np.asarray(K, dtype=np.int64)]
    n = R.shape[1]
    Y = np.empty((B.shape[1], n))
    for i in range(n):
        Y[:, i], _ = nnls(B, R[:, i])
    return Y
