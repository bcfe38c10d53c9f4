"""Pins for the oracle's compressed ADMM NMF (Alg. 4, App. B).

P4 exact recovery (fixed point and convergence); P5 KKT sign and
complementarity conditions, and stationarity residuals shrinking; P6 the
uncompressed ADMM is Alg. 4 with L = I, R = I; P7 invariance of the U, V
trajectory under a change of orthonormal basis of L and R; P12 the
Eckart-Young floor; a planted sign error is caught by the fixed-point pin.
"""
import numpy as np
import pytest

import synth
from oracle import admm, compress, philox, residual


def _problem(m=60, n=50, r=4, d=None, sigma=0.0, seed=7, q=2):
    d = d or r
    A = synth.lowrank(m, n, r, sigma, seed)
    Om, Ps = philox.test_matrices(seed + 100, m, n, d)
    L, Rt, _, At = compress.compress(A, Om, Ps, q)
    U0, V0 = synth.init_factors(m, n, r, seed + 200)
    return A, L, Rt, At, U0, V0


def test_p4_planted_fixed_point():
    m, n, r = 60, 50, 4
    A, X0, Y0 = synth.lowrank(m, n, r, 0.0, 7, with_factors=True)
    Om, Ps = philox.test_matrices(107, m, n, r)
    L, Rt, _, At = compress.compress(A, Om, Ps, 2)
    st = admm.AdmmState(Xt=L.T @ X0, Yt=Y0 @ Rt, U=X0.copy(), V=Y0.copy(),
                        Lam=np.zeros((m, r)), Phi=np.zeros((r, n)))
    for lam in (1.0, 7.5):
        nxt = admm.admm_step(st, L, Rt, At, lam, lam, 1.0)
        assert np.abs(nxt.U - X0).max() < 1e-12 * np.abs(X0).max()
        assert np.abs(nxt.V - Y0).max() < 1e-12 * np.abs(Y0).max()
        assert np.abs(nxt.Lam).max() < 1e-10 and np.abs(nxt.Phi).max() < 1e-10


def test_p4_planted_mistake_is_caught(monkeypatch):
    """Alg. 4 with the sign of L^T Lam flipped drifts off the fixed point."""
    m, n, r = 60, 50, 4
    A, X0, Y0 = synth.lowrank(m, n, r, 0.0, 7, with_factors=True)
    Om, Ps = philox.test_matrices(107, m, n, r)
    L, Rt, _, At = compress.compress(A, Om, Ps, 2)
    lam = 5.0
    st = admm.AdmmState(Xt=L.T @ X0, Yt=Y0 @ Rt, U=X0.copy(), V=Y0.copy(),
                        Lam=-0.1 * np.ones((m, r)), Phi=np.zeros((r, n)))
    good = admm.admm_step(st, L, Rt, At, lam, lam, 1.0)
    orig = admm._spd_solve
    calls = {"n": 0}

    def bad_solve(G, B):
        calls["n"] += 1
        if calls["n"] == 1:       # X-tilde update: use +L^T Lam instead of -
            B = B + 2 * (L.T @ st.Lam).T
        return orig(G, B)
    monkeypatch.setattr(admm, "_spd_solve", bad_solve)
    bad = admm.admm_step(st, L, Rt, At, lam, lam, 1.0)
    assert np.abs(bad.U - good.U).max() > 1e-3


def test_p4_exact_recovery_from_random_init():
    A, L, Rt, At, U0, V0 = _problem()
    lam = np.linalg.norm(At) / 4
    st = admm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=2000)
    assert residual.rel_residual(A, st.U, st.V) < 1e-10


def test_p5_kkt_signs_hold_every_sweep():
    # with xi = 1: U > 0 => Lam = 0 (to rounding); U = 0 => Lam <= 0
    A, L, Rt, At, U0, V0 = _problem(m=80, n=70, r=5, d=10, sigma=0.05)
    lam = np.linalg.norm(At) / 5
    st = admm.admm_init(Rt, U0, V0)
    for _ in range(30):
        st = admm.admm_step(st, L, Rt, At, lam, lam, 1.0)
        assert st.U.min() >= 0 and st.V.min() >= 0
        scale = lam * np.abs(st.U).max()
        assert np.all(st.Lam[st.U == 0] <= 1e-12 * scale)
        assert np.all(np.abs(st.Lam[st.U > 0]) <= 1e-12 * scale)
        sp = lam * np.abs(st.V).max()
        assert np.all(st.Phi[st.V == 0] <= 1e-12 * sp)
        assert np.all(np.abs(st.Phi[st.V > 0]) <= 1e-12 * sp)


def test_p5_kkt_residuals_shrink():
    A, L, Rt, At, U0, V0 = _problem(m=80, n=70, r=5, d=10, sigma=0.05)
    lam = np.linalg.norm(At) / 5
    st = admm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=20)
    k20 = admm.kkt_residuals(L, Rt, At, st)
    st = admm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=1500, state=st)
    k = admm.kkt_residuals(L, Rt, At, st)
    for key in "abcd":
        assert k[key] < 1e-2 * k20[key] or k[key] < 1e-9, (key, k20[key], k[key])
    assert k["e"] < 1e-12 and k["f"] < 1e-12


def test_p6_plain_is_identity_compression():
    m, n, r = 30, 25, 3
    A = synth.lowrank(m, n, r, 0.02, 5)
    U0, V0 = synth.init_factors(m, n, r, 6)
    a = admm.admm(np.eye(m), np.eye(n), A, U0, V0, lam=3.0, phi=2.0, iters=15)
    b = admm.admm_plain(A, U0, V0, lam=3.0, phi=2.0, iters=15)
    assert np.array_equal(a.U, b.U) and np.array_equal(a.V, b.V)
    assert np.array_equal(a.Lam, b.Lam) and np.array_equal(a.Phi, b.Phi)


def test_p7_basis_invariance():
    A, L, Rt, At, U0, V0 = _problem(m=70, n=60, r=4, d=9, sigma=0.02)
    g = np.random.default_rng(0)
    O1, _ = np.linalg.qr(g.standard_normal((9, 9)))
    O2, _ = np.linalg.qr(g.standard_normal((9, 9)))
    L2, Rt2 = L @ O1, Rt @ O2
    At2 = L2.T @ A @ Rt2
    lam = np.linalg.norm(At) / 4
    a = admm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=20)
    b = admm.admm(L2, Rt2, At2, U0, V0, lam=lam, phi=lam, iters=20)
    assert np.abs(a.U - b.U).max() <= 1e-12 * np.abs(a.U).max() * 100
    assert np.abs(a.V - b.V).max() <= 1e-12 * np.abs(a.V).max() * 100


def test_p12_floor_and_trend():
    A, L, Rt, At, U0, V0 = _problem(m=100, n=80, r=5, d=15, sigma=0.01, q=4)
    lam = np.linalg.norm(At) / 5
    st = admm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=400, A=A,
                   every=50)
    floor = residual.svd_floor(A, 5)
    rho = [h[1] for h in st.history]
    assert min(rho) >= floor * (1 - 1e-12)
    assert rho[-1] < rho[0]
    assert rho[-1] <= floor + 1e-3
    # compressed result is as accurate as the uncompressed ADMM (Sec. V claim)
    p = admm.admm_plain(A, U0, V0, lam=lam, phi=lam, iters=400)
    assert rho[-1] <= residual.rel_residual(A, p.U, p.V) * 1.05 + 1e-4


def test_resume_equals_uninterrupted():
    A, L, Rt, At, U0, V0 = _problem(m=50, n=40, r=3, d=8, sigma=0.02)
    a = admm.admm(L, Rt, At, U0, V0, lam=4.0, phi=4.0, iters=30)
    b = admm.admm(L, Rt, At, U0, V0, lam=4.0, phi=4.0, iters=12)
    b = admm.admm(L, Rt, At, U0, V0, lam=4.0, phi=4.0, iters=18, state=b)
    assert np.array_equal(a.U, b.U) and np.array_equal(a.V, b.V)
