"""Structured random compression (Alg. 1), one- and two-sided. FP64 oracle.

TEST INFRASTRUCTURE -- only tests, the smoke check and the benchmark's
CPU-baseline leg call this.  Plain NumPy/LAPACK in FP64; no blocking or
fusion beyond what the algorithm states.

Alg. 1 (Sec. II) forms B = (A A^T)^w A Omega with a Gaussian Omega of
r + r_ov columns and returns an orthonormal basis Q of B from a QR
decomposition.  This oracle follows the subspace-iteration reading: the same
2w + 1 products, with the running panel re-orthonormalised (Householder QR)
after every product.  In exact arithmetic the span is unchanged; the literal
form is ``compress_literal`` and a pin checks the two agree on
well-conditioned inputs.

Sec. III applies Alg. 1 to A and to A^T to get L (m x d, orthonormal
columns) and R (d x n, orthonormal rows); the library stores R^T (n x d).
Sec. III defines A-check = A R^T and App. B (Alg. 4, setup) the compressed
matrix A-tilde = L^T A R^T.

Gaussian compression (Sec. II, the note on data-agnostic compression) is
the baseline the paper compares against: Q = s^-1/2 Omega with a Gaussian
Omega of s columns and no power iteration or orthonormalisation.
``compress_gaussian`` applies it on both sides with s = d: L = d^-1/2 Psi,
R^T = d^-1/2 Omega, then A-check and A-tilde as above.
"""
from __future__ import annotations

import numpy as np


def orth(Y: np.ndarray) -> np.ndarray:
    """Thin Q of a Householder QR of Y, column signs chosen so diag(R) > 0.

    For Y of full column rank this Q is unique, so any correct QR algorithm
    (the GPU uses CholeskyQR2) must return the same matrix up to rounding.
    """
    Q, R = np.linalg.qr(Y, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def compress_literal(A: np.ndarray, Omega: np.ndarray, w: int) -> np.ndarray:
    """Alg. 1 as printed: Q = orth((A A^T)^w A Omega), single QR at the end."""
    B = A @ Omega
    for _ in range(w):
        B = A @ (A.T @ B)
    return orth(B)


def sketch_left(A: np.ndarray, Omega: np.ndarray, q: int) -> np.ndarray:
    """Alg. 1 on A with re-orthonormalisation after every product.

    Q0 = orth(A Omega); then q times: Z = orth(A^T Q); Q = orth(A Z).
    Returns Q (m x d) with orthonormal columns (2q + 1 products with A).
    """
    Q = orth(A @ Omega)
    for _ in range(q):
        Z = orth(A.T @ Q)
        Q = orth(A @ Z)
    return Q


def compress(A: np.ndarray, Omega: np.ndarray, Psi: np.ndarray, q: int):
    """Two-sided compression (Sec. III): L = Alg.1(A), R^T = Alg.1(A^T).

    Omega (n x d) seeds the left chain, Psi (m x d) the right chain.
    Returns (L m x d, Rt n x d, Acheck = A R^T m x d, Atilde = L^T A R^T).
    """
    A = np.asarray(A, dtype=np.float64)
    L = sketch_left(A, Omega, q)          # Alg. 1 applied to A
    Rt = sketch_left(A.T, Psi, q)         # Alg. 1 applied to A^T
    Acheck = A @ Rt
    Atilde = L.T @ Acheck
    return L, Rt, Acheck, Atilde


def snmf_basis(A: np.ndarray, Omega: np.ndarray, q: int):
    """Alg. 3 step 1 and the compressed matrix of step 2.

    Q = Alg.1(A) (m x d); Rhat = Q^T A (d x n).  Returns (Q, Rhat).
    """
    A = np.asarray(A, dtype=np.float64)
    Q = sketch_left(A, Omega, q)
    return Q, Q.T @ A


def compress_gaussian(A: np.ndarray, Omega: np.ndarray, Psi: np.ndarray):
    """Two-sided Gaussian compression (Sec. II note): L = d^-1/2 Psi (m x d),
    R^T = d^-1/2 Omega (n x d).  Returns (L, Rt, Acheck, Atilde)."""
    A = np.asarray(A, dtype=np.float64)
    d = Omega.shape[1]
    c = 1.0 / np.sqrt(d)
    L = np.asarray(Psi, dtype=np.float64) * c
    Rt = np.asarray(Omega, dtype=np.float64) * c
    Acheck = A @ Rt
    return L, Rt, Acheck, L.T @ Acheck
