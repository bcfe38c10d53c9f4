"""Pins of oracle/residual.py against what mathematics fixes, independent of
the functions' own formulas:

* residual_sq / rel_residual and compressed_objective on hand-worked
  2 x 2 examples;
* compressed_objective equals the uncompressed residual when the
  compression is exact (A = L Atilde R with orthonormal L columns and R
  rows; Frobenius norms are invariant under orthonormal maps, Sec. III);
* svd_floor on matrices with prescribed singular values (random
  orthogonal factors): the closed form (sum_{j>r} s_j^2 / sum s_j^2)^1/2,
  zero for an exact rank-r matrix, one for r = 0, attained by the rank-r
  truncation, and never beaten by random rank-r candidates (Eckart-Young).
"""
import math

import numpy as np

from oracle import residual


def _orth(g, rows, cols):
    q, _ = np.linalg.qr(g.standard_normal((rows, cols)))
    return q


def test_residual_hand_worked():
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    U = np.array([[1.0], [1.0]])
    V = np.array([[1.0, 1.0]])
    # A - U V = [[0, 1], [2, 3]]: 0 + 1 + 4 + 9 = 14; ||A||^2 = 30
    e2, a2 = residual.residual_sq(A, U, V)
    assert e2 == 14.0 and a2 == 30.0
    assert abs(residual.rel_residual(A, U, V) - math.sqrt(14.0 / 30.0)) < 1e-15


def test_compressed_objective_hand_worked():
    At = np.array([[1.0, 2.0], [3.0, 4.0]])
    Xt = np.array([[1.0], [1.0]])
    Yt = np.array([[1.0, 1.0]])
    assert abs(residual.compressed_objective(At, Xt, Yt) - math.sqrt(14.0)) < 1e-15
    # the factor order matters: Yt Xt (1 x 1) is not a 2 x 2 product
    Xt2 = np.array([[2.0], [0.0]])
    Yt2 = np.array([[0.5, 1.0]])
    # At - Xt2 Yt2 = [[0, 0], [3, 4]] -> 5
    assert abs(residual.compressed_objective(At, Xt2, Yt2) - 5.0) < 1e-15


def test_compressed_objective_equals_residual_under_exact_compression():
    g = np.random.default_rng(3)
    m, n, d, r = 60, 45, 7, 3
    L = _orth(g, m, d)                  # m x d, orthonormal columns
    R = _orth(g, n, d).T                # d x n, orthonormal rows
    M = g.standard_normal((d, d))
    A = L @ M @ R                       # exact rank d: L L^T A = A R^T R = A
    At = L.T @ A @ R.T                  # = M
    Xt = g.standard_normal((d, r))
    Yt = g.standard_normal((r, d))
    e2, _ = residual.residual_sq(A, L @ Xt, Yt @ R)
    obj = residual.compressed_objective(At, Xt, Yt)
    assert abs(obj - math.sqrt(e2)) <= 1e-12 * math.sqrt(e2)


def _with_singular_values(g, m, n, s):
    k = len(s)
    return (_orth(g, m, k) * np.asarray(s)) @ _orth(g, n, k).T


def test_svd_floor_closed_form():
    g = np.random.default_rng(5)
    s = np.array([9.0, 5.0, 3.0, 2.0, 1.0, 0.5, 0.25])
    A = _with_singular_values(g, 40, 30, s)
    for r in range(0, len(s) + 1):
        want = math.sqrt(float(np.sum(s[r:] ** 2) / np.sum(s ** 2)))
        assert abs(residual.svd_floor(A, r) - want) <= 1e-13


def test_svd_floor_exact_rank_and_attainment():
    g = np.random.default_rng(6)
    A = g.random((50, 4)) @ g.random((4, 35))         # rank 4
    assert residual.svd_floor(A, 4) <= 1e-14
    B = A + 0.01 * g.standard_normal(A.shape)
    r = 3
    f = residual.svd_floor(B, r)
    # the rank-r truncation attains the floor ...
    U, s, Vt = np.linalg.svd(B, full_matrices=False)
    Ur, Vr = U[:, :r] * s[:r], Vt[:r]
    assert abs(residual.rel_residual(B, Ur, Vr) - f) <= 1e-12
    # ... and no other rank-r product goes below it
    for t in range(200):
        X = g.standard_normal((50, r))
        Y = np.linalg.lstsq(X, B, rcond=None)[0]   # best Y for this X
        assert residual.rel_residual(B, X, Y) >= f * (1 - 1e-12)
