"""Pins for the oracle's compressed SNMF column selection (Alg. 3 + SPA).

P8 SPA returns the planted anchors of a noiseless separable matrix; P9
SPA(Q^T A) = SPA(A) when range(Q) contains range(A) (orthogonal invariance,
Sec. IV); a hand-worked 3 x 5 example; ties go to the lowest index.
"""
import numpy as np

import synth
from oracle import philox, snmf, compress


def test_spa_hand_example():
    # columns: e1 scaled 3, e2 scaled 2, e3, and two interior points.
    # norms^2: 9, 4, 1, 1.5, 2.54 -> col 0 (margin (9-4)/9); after
    # projecting e1 out: 0, 4, 1, 0.5, 0.29 -> col 1 (margin 3/4); then
    # 0, 0, 1, 0.25, 0.04 -> col 2 (margin 3/4).
    R = np.array([[3.0, 0.0, 0.0, 1.0, 1.5],
                  [0.0, 2.0, 0.0, 0.5, 0.5],
                  [0.0, 0.0, 1.0, 0.5, 0.2]])
    K, margins = snmf.spa(R, 3)
    assert list(K) == [0, 1, 2]
    assert np.allclose(margins, [5 / 9, 3 / 4, 3 / 4], rtol=1e-14)


def test_spa_ties_lowest_index():
    R = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 0.0]])
    K, _ = snmf.spa(R, 2)
    assert list(K) == [0, 1]


def test_p8_planted_anchors_noiseless():
    for seed in range(3):
        A, anchors = synth.separable(80, 300, 6, 0.0, seed)
        K, margins = snmf.spa(A, 6)
        assert sorted(K) == sorted(anchors)


def test_p8_p9_compressed_equals_uncompressed():
    m, n, r, d = 100, 400, 8, 18
    A, anchors = synth.separable(m, n, r, 0.0, 3)
    Om = philox.gaussian_matrix(9, 0, n, d)
    K, margins, Q, Rhat = snmf.snmf_select(A, Om, r, 1)
    K_full, _ = snmf.spa(A, r)
    assert list(K) == list(K_full)            # same order
    assert sorted(K) == sorted(anchors)
    assert np.linalg.norm(Q.T @ Q - np.eye(d)) < 1e-12


def test_p9_orthogonal_invariance():
    g = np.random.default_rng(1)
    A = np.abs(g.standard_normal((12, 40)))
    Q, _ = np.linalg.qr(g.standard_normal((12, 12)))
    K1, _ = snmf.spa(A, 6)
    K2, _ = snmf.spa(Q.T @ A, 6)
    assert list(K1) == list(K2)


def test_noisy_separable_with_margin():
    A, anchors = synth.separable(200, 2000, 10, 1e-3, 5)
    Om = philox.gaussian_matrix(6, 0, 2000, 20)
    K, margins, Q, Rhat = snmf.snmf_select(A, Om, 10, 2)
    assert sorted(K) == sorted(anchors)
    assert margins.min() > 1e-4


# ---- Alg. 3 step 3: the right factor (per-column NNLS)

def _kkt(B, b, h):
    """Largest violation of the NNLS optimality conditions at h: h >= 0,
    gradient g = B^T (B h - b) >= 0 where h = 0 and = 0 where h > 0."""
    g = B.T @ (B @ h - b)
    scale = np.linalg.norm(B.T @ b) + 1e-300
    viol = np.where(h > 0, np.abs(g), np.maximum(-g, 0.0))
    return max(viol.max() / scale, max(-h.min(), 0.0))


def test_right_factor_kkt_random():
    g = np.random.default_rng(7)
    for d, n, r in [(12, 40, 4), (30, 25, 9), (5, 8, 1)]:
        R = g.standard_normal((d, n))
        K = g.choice(n, r, replace=False)
        Y = snmf.right_factor(R, K)
        assert Y.shape == (r, n)
        for i in range(n):
            assert _kkt(R[:, K], R[:, i], Y[:, i]) <= 1e-10


def test_right_factor_exact_on_separable():
    # noiseless separable Rhat = W [I | H] Pi with H >= 0: the selected
    # columns reproduce every column with the planted weights
    g = np.random.default_rng(3)
    d, r, n = 10, 4, 30
    Wb = g.random((d, r))
    H = g.random((r, n - r))
    M = np.concatenate([np.eye(r), H], axis=1)
    perm = g.permutation(n)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    R = Wb @ M[:, inv]
    K = perm[:r]
    Y = snmf.right_factor(R, K)
    assert np.abs(Y - M[:, inv]).max() <= 1e-10
    # a selected column is its own unit vector
    for j, k in enumerate(K):
        assert np.abs(Y[:, k] - np.eye(r)[:, j]).max() <= 1e-12


def test_right_factor_brute_force_tiny():
    # enumerate every passive set of a 3-column problem: the minimiser is
    # the feasible unconstrained fit on some passive set with the smallest
    # residual
    import itertools
    g = np.random.default_rng(11)
    d, r = 6, 3
    for _ in range(20):
        B = g.standard_normal((d, r))
        b = g.standard_normal(d)
        best, hbest = np.inf, None
        for mask in itertools.product([0, 1], repeat=r):
            P = [j for j in range(r) if mask[j]]
            h = np.zeros(r)
            if P:
                sol, *_ = np.linalg.lstsq(B[:, P], b, rcond=None)
                if sol.min() < 0:
                    continue
                h[P] = sol
            res = np.linalg.norm(B @ h - b)
            if res < best - 1e-14:
                best, hbest = res, h
        R = np.concatenate([B, b[:, None]], axis=1)
        Y = snmf.right_factor(R, np.arange(r))
        assert np.abs(Y[:, r] - hbest).max() <= 1e-10
