"""Pins for the oracle's compressed alternating NMF (Alg. 2).

Every step must satisfy the inequality Alg. 2 prints (the step does not
raise its compressed objective), for both inner solvers; the exact (ALS)
step must satisfy the NNLS optimality conditions row by row; without
compression (L = I, R = I) the iteration is plain alternating NMF, whose
residual then decreases monotonically; and the multiplicative update leaves
zero entries at zero.
"""
import numpy as np

import synth
from oracle import alternating as alt
from oracle import compress, philox


def _case(m=60, n=50, r=4, d=8, seed=3):
    A = synth.lowrank(m, n, r, 0.05, seed)
    Om, Ps = philox.test_matrices(seed + 1, m, n, d)
    L, Rt, Acheck, _ = compress.compress(A, Om, Ps, 2)
    Ahat = L.T @ A
    X0, Y0 = synth.init_factors(m, n, r, seed + 2)
    return A, L, Rt, Acheck, Ahat, X0, Y0


def test_steps_do_not_raise_their_objective():
    A, L, Rt, Ac, Ah, X0, Y0 = _case()
    for solver in ("als", "mu"):
        hist = []
        alt.iterate(Ac, Ah, L, Rt, X0, Y0, 15, solver, hist)
        for bx, ax, by, ay in hist:
            assert ax <= bx * (1 + 1e-12) + 1e-12
            assert ay <= by * (1 + 1e-12) + 1e-12


def test_als_step_is_the_nnls_minimiser():
    A, L, Rt, Ac, Ah, X0, Y0 = _case(seed=9)
    X, Y = alt.iterate(Ac, Ah, L, Rt, X0, Y0, 1, "als")
    Yc = Y0 @ Rt
    G = Yc @ Yc.T
    for i in range(X.shape[0]):          # KKT of min ||Ac[i] - x Yc||, x >= 0
        g = X[i] @ G - Ac[i] @ Yc.T
        scale = np.abs(Ac[i] @ Yc.T).max() + 1e-300
        assert X[i].min() >= 0
        assert np.all(np.where(X[i] > 0, np.abs(g), np.maximum(-g, 0)) <= 1e-9 * scale)


def test_uncompressed_als_is_monotone():
    m, n, r = 40, 30, 3
    A = synth.lowrank(m, n, r, 0.02, 5)
    X0, Y0 = synth.init_factors(m, n, r, 6)
    hist = []
    X, Y = alt.iterate(A, A, np.eye(m), np.eye(n), X0, Y0, 10, "als", hist)
    res = [h[3] for h in hist]       # ||A - X Y|| after each full iteration
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res, res[1:]))
    assert res[-1] <= 0.1 * np.linalg.norm(A)


def test_mu_keeps_zeros():
    A, L, Rt, Ac, Ah, X0, Y0 = _case(seed=4)
    X0 = X0.copy()
    X0[3, 1] = 0.0
    X, _ = alt.iterate(Ac, Ah, L, Rt, X0, Y0, 3, "mu")
    assert X[3, 1] == 0.0
    assert X.min() >= 0
