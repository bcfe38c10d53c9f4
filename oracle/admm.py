"""Compressed ADMM NMF (Alg. 4, App. B) and its uncompressed special case.

TEST INFRASTRUCTURE -- only tests, the smoke check and the benchmark's
CPU-baseline leg call this.  FP64 NumPy, updates in the order Alg. 4 prints
them.

Problem (Sec. III, double-sided compressed problem):
    min ||Atilde - Xt Yt||_F^2  s.t.  U = L Xt, V = Yt R, U >= 0, V >= 0
with Atilde = L^T A R^T, Xt (d x r), Yt (r x d).  One ADMM sweep (Alg. 4):
    Xt <- (Atilde Yt^T + lam L^T U - L^T Lam) (Yt Yt^T + lam I)^-1
    Yt <- (Xt^T Xt + phi I)^-1 (Xt^T Atilde + phi V R^T - Phi R^T)
    U  <- P+(L Xt + Lam / lam)
    V  <- P+(Yt R + Phi / phi)
    Lam <- Lam + xi lam (L Xt - U)
    Phi <- Phi + xi phi (Yt R - V)
with P+ the entrywise max(., 0).  U and V use the *old* multipliers; the
multiplier updates use the new U, V.  Setup: Yt = V R^T, Lam = 0, Phi = 0.
The r x r inverses are applied by Cholesky solves (both matrices are SPD
because lam, phi > 0).

The uncompressed ADMM NMF of Xu et al. (Sec. III, problem "nmfEquiv") is
the same iteration with L = I_m and R = I_n; ``admm_plain`` writes it out
without the identity products (a pin checks it equals ``admm`` with
identities).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


@dataclass
class AdmmState:
    """The resumable state Z of App. B: (Xt, Yt, U, V, Lam, Phi) and k."""
    Xt: np.ndarray
    Yt: np.ndarray
    U: np.ndarray
    V: np.ndarray
    Lam: np.ndarray
    Phi: np.ndarray
    k: int = 0
    history: list = field(default_factory=list)


def _spd_solve(G: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve G X = B for SPD G (Cholesky)."""
    c = sla.cho_factor(G, lower=True)
    return sla.cho_solve(c, B)


def admm_init(Rt: np.ndarray, U0: np.ndarray, V0: np.ndarray) -> AdmmState:
    """Alg. 4 setup: Yt = V R^T, Lam = 0, Phi = 0 (Xt is computed first)."""
    m, r = U0.shape
    n = V0.shape[1]
    Yt = V0 @ Rt
    return AdmmState(Xt=np.zeros((Rt.shape[1], r)), Yt=Yt, U=U0.copy(),
                     V=V0.copy(), Lam=np.zeros((m, r)),
                     Phi=np.zeros((r, n)), k=0)


def admm_step(st: AdmmState, L, Rt, Atilde, lam, phi, xi) -> AdmmState:
    """One sweep of Alg. 4 in the printed order; returns the new state."""
    r = st.U.shape[1]
    I = np.eye(r)
    R = Rt.T
    Yt, U, V, Lam, Phi = st.Yt, st.U, st.V, st.Lam, st.Phi
    MX = Atilde @ Yt.T + lam * (L.T @ U) - L.T @ Lam            # d x r
    Xt = _spd_solve(Yt @ Yt.T + lam * I, MX.T).T                # right solve
    MY = Xt.T @ Atilde + phi * (V @ Rt) - Phi @ Rt              # r x d
    Yt = _spd_solve(Xt.T @ Xt + phi * I, MY)
    T = L @ Xt                                                  # m x r
    S = Yt @ R                                                  # r x n
    Un = np.maximum(T + Lam / lam, 0.0)
    Vn = np.maximum(S + Phi / phi, 0.0)
    Lam = Lam + xi * lam * (T - Un)
    Phi = Phi + xi * phi * (S - Vn)
    return AdmmState(Xt=Xt, Yt=Yt, U=Un, V=Vn, Lam=Lam, Phi=Phi, k=st.k + 1,
                     history=st.history)


def admm(L, Rt, Atilde, U0, V0, lam=1.0, phi=1.0, xi=1.0, iters=100,
         state: AdmmState | None = None, A=None, every: int = 0):
    """Run ``iters`` sweeps of Alg. 4 (from U0, V0, or resuming ``state``).

    With ``A`` and ``every`` > 0 the relative residual ||A - UV||/||A|| is
    appended to ``state.history`` as (k, rho) every ``every`` sweeps.
    """
    st = state if state is not None else admm_init(Rt, U0, V0)
    normA = np.linalg.norm(A) if A is not None else None
    for _ in range(iters):
        st = admm_step(st, L, Rt, Atilde, lam, phi, xi)
        if A is not None and every and st.k % every == 0:
            st.history.append(
                (st.k, np.linalg.norm(A - st.U @ st.V) / normA))
    return st


def admm_plain(A, U0, V0, lam=1.0, phi=1.0, xi=1.0, iters=100,
               state: AdmmState | None = None, every: int = 0):
    """Uncompressed ADMM NMF: Alg. 4 with L = I_m, R = I_n (Atilde = A).

    Xt is then X (m x r) and Yt is Y (r x n).  Same update order.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    r = U0.shape[1]
    I = np.eye(r)
    if state is None:
        st = AdmmState(Xt=np.zeros((m, r)), Yt=V0.copy(), U=U0.copy(),
                       V=V0.copy(), Lam=np.zeros((m, r)),
                       Phi=np.zeros((r, n)), k=0)
    else:
        st = state
    normA = np.linalg.norm(A)
    for _ in range(iters):
        Y, U, V, Lam, Phi = st.Yt, st.U, st.V, st.Lam, st.Phi
        MX = A @ Y.T + lam * U - Lam
        X = _spd_solve(Y @ Y.T + lam * I, MX.T).T
        MY = X.T @ A + phi * V - Phi
        Y = _spd_solve(X.T @ X + phi * I, MY)
        Un = np.maximum(X + Lam / lam, 0.0)
        Vn = np.maximum(Y + Phi / phi, 0.0)
        Lam = Lam + xi * lam * (X - Un)
        Phi = Phi + xi * phi * (Y - Vn)
        st = AdmmState(Xt=X, Yt=Y, U=Un, V=Vn, Lam=Lam, Phi=Phi,
                       k=st.k + 1, history=st.history)
        if every and st.k % every == 0:
            st.history.append(
                (st.k, np.linalg.norm(A - st.U @ st.V) / normA))
    return st


def kkt_residuals(L, Rt, Atilde, st: AdmmState):
    """Relative residuals of the KKT system of App. B at the state ``st``.

    Read with consistent dimensions (the printed (a) adds Lam, m x r, to a
    d x r term):
      (a) (Xt Yt - Atilde) Yt^T + L^T Lam = 0
      (b) Xt^T (Xt Yt - Atilde) + Phi R^T = 0
      (c) L Xt - U = 0          (d) Yt R - V = 0
      (e) Lam <= 0 <= U, Lam o U = 0   (f) Phi <= 0 <= V, Phi o V = 0
    Returns a dict of Frobenius norms, each relative to a natural scale.
    """
    R = Rt.T
    E = st.Xt @ st.Yt - Atilde
    sa = np.linalg.norm(Atilde)
    out = {
        "a": np.linalg.norm(E @ st.Yt.T + L.T @ st.Lam)
             / max(sa * np.linalg.norm(st.Yt), 1e-300),
        "b": np.linalg.norm(st.Xt.T @ E + st.Phi @ Rt)
             / max(sa * np.linalg.norm(st.Xt), 1e-300),
        "c": np.linalg.norm(L @ st.Xt - st.U) / max(np.linalg.norm(st.U), 1e-300),
        "d": np.linalg.norm(st.Yt @ R - st.V) / max(np.linalg.norm(st.V), 1e-300),
        "e": np.linalg.norm(st.Lam * st.U) / max(
            np.linalg.norm(st.Lam) * np.linalg.norm(st.U), 1e-300),
        "f": np.linalg.norm(st.Phi * st.V) / max(
            np.linalg.norm(st.Phi) * np.linalg.norm(st.V), 1e-300),
    }
    return out
