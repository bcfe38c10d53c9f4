"""Pins for the oracle's structured random compression (Alg. 1, Sec. III).

P1 orthonormality; P2 Eckart-Young lower bound; P3 Theorem 1 expectation
bound (w = 0) and agreement of the re-orthonormalised power scheme with the
literal B = (A A^T)^w A Omega; P4 exact range capture for rank-r A with
d = r; orth() against the uniqueness of the thin QR factor.  Gaussian
compression (the paper's baseline): norm preservation on average and the
operand order of A-tilde on a one-entry A.
"""
import numpy as np
import pytest

import synth
from oracle import compress, philox


def _spectrum_matrix(m, n, sig, seed):
    g = np.random.default_rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((m, len(sig))))
    V, _ = np.linalg.qr(g.standard_normal((n, len(sig))))
    return (U * sig) @ V.T


def test_orth_unique_thin_q():
    g = np.random.default_rng(1)
    Y = g.standard_normal((40, 6))
    Q = compress.orth(Y)
    assert np.linalg.norm(Q.T @ Q - np.eye(6)) < 1e-13
    R = Q.T @ Y
    # R upper triangular with positive diagonal and Q R = Y
    assert np.allclose(np.tril(R, -1), 0, atol=1e-12)
    assert np.all(np.diag(R) > 0)
    assert np.linalg.norm(Q @ R - Y) < 1e-12 * np.linalg.norm(Y)
    # Gram-Schmidt written out gives the same Q (uniqueness)
    G = np.zeros_like(Y)
    for j in range(6):
        v = Y[:, j].copy()
        for _ in range(2):
            v -= G[:, :j] @ (G[:, :j].T @ v)
        G[:, j] = v / np.linalg.norm(v)
    assert np.abs(G - Q).max() < 1e-12


@pytest.mark.parametrize("q", [0, 1, 4])
def test_p1_orthonormal(q):
    A = synth.lowrank(80, 60, 5, 0.01, 3)
    Om, Ps = philox.test_matrices(5, 80, 60, 12)
    L, Rt, Ac, At = compress.compress(A, Om, Ps, q)
    assert L.shape == (80, 12) and Rt.shape == (60, 12)
    assert np.linalg.norm(L.T @ L - np.eye(12)) <= 1e-12
    assert np.linalg.norm(Rt.T @ Rt - np.eye(12)) <= 1e-12
    assert np.allclose(Ac, A @ Rt) and np.allclose(At, L.T @ A @ Rt)


def test_p2_eckart_young_lower_bound():
    for seed in range(5):
        A = synth.lowrank(70, 50, 4, 0.05, 10 + seed)
        Om, Ps = philox.test_matrices(seed, 70, 50, 8)
        L, Rt, _, _ = compress.compress(A, Om, Ps, 1)
        s = np.linalg.svd(A, compute_uv=False)
        lb = np.sqrt(np.sum(s[8:] ** 2))
        assert np.linalg.norm(A - L @ (L.T @ A)) >= lb * (1 - 1e-12)
        assert np.linalg.norm(A - (A @ Rt) @ Rt.T) >= lb * (1 - 1e-12)


def test_p3_theorem1_expectation_bound():
    # w = 0, r = 5, r_ov = 5: E||A - PA||_F <= (1 + r/(r_ov-1))^1/2 tail_r
    sig = np.concatenate([np.ones(5) * 10, 0.8 ** np.arange(1, 36)])
    A = _spectrum_matrix(120, 90, sig, 0)
    r, rov = 5, 5
    errs = []
    for seed in range(30):
        Om = philox.gaussian_matrix(seed, 0, 90, r + rov)
        Q = compress.sketch_left(A, Om, 0)
        errs.append(np.linalg.norm(A - Q @ (Q.T @ A)))
    tail = np.sqrt(np.sum(sig[r:] ** 2))
    bound = np.sqrt(1 + r / (rov - 1)) * tail
    assert np.mean(errs) <= bound
    # and never below the optimum with r + r_ov columns
    assert min(errs) >= np.sqrt(np.sum(sig[r + rov:] ** 2)) * (1 - 1e-12)


@pytest.mark.parametrize("w", [0, 1, 2])
def test_p3_reorth_equals_literal_power_scheme(w):
    sig = np.geomspace(10.0, 1.0, 8)           # kappa 10 on the sketched span
    sig = np.concatenate([sig, 0.01 * np.ones(12)])
    A = _spectrum_matrix(60, 50, sig, 4)
    Om = philox.gaussian_matrix(7, 0, 50, 8)
    Q1 = compress.sketch_left(A, Om, w)
    Q2 = compress.compress_literal(A, Om, w)
    assert np.linalg.norm(Q1 @ Q1.T - Q2 @ Q2.T) < 1e-10


def test_p4_exact_range_capture():
    m, n, r = 60, 50, 4
    A = synth.lowrank(m, n, r, 0.0, 7)
    Om, Ps = philox.test_matrices(11, m, n, r)
    L, Rt, _, _ = compress.compress(A, Om, Ps, 2)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(L @ (L.T @ A) - A) <= 1e-12 * nA
    assert np.linalg.norm(A @ Rt @ Rt.T - A) <= 1e-12 * nA


def test_power_iterations_drive_error_to_optimum():
    # Theorem 3: the bound's extra factor -> 1 as w grows (spectral norm).
    sig = np.concatenate([np.ones(5) * 10, np.linspace(1.0, 0.5, 40)])
    A = _spectrum_matrix(150, 100, sig, 2)
    Om = philox.gaussian_matrix(3, 0, 100, 8)
    e = [np.linalg.norm(A - (Q := compress.sketch_left(A, Om, w)) @ (Q.T @ A), 2)
         for w in (0, 2, 6)]
    assert e[2] <= e[1] * 1.0001 and e[1] <= e[0] * 1.0001
    assert e[2] <= sig[5] * 1.05


# ---- Gaussian compression baseline (Sec. II note)

def test_gaussian_compression_preserves_norms_on_average():
    # E ||L^T x||^2 = ||x||^2 for L = d^-1/2 (i.i.d. N(0, 1)) (m x d): the
    # scaling that makes the Gaussian projection norm-preserving.  Over 400
    # draws the mean ratio is within 4 standard errors of 1 (one draw has
    # variance 2 / d).
    from oracle import philox
    m, n, d = 60, 7, 8
    x = np.random.default_rng(1).standard_normal(m)
    ratios = []
    for seed in range(400):
        Om, Ps = philox.test_matrices(seed, m, n, d)
        L, _, _, _ = compress.compress_gaussian(np.zeros((m, n)), Om, Ps)
        ratios.append(np.sum((L.T @ x) ** 2) / np.sum(x ** 2))
    se = np.sqrt(2.0 / d) / np.sqrt(len(ratios))
    assert abs(np.mean(ratios) - 1.0) <= 4 * se


def test_gaussian_compression_operand_order():
    # A = e_i e_j^T picks row i of L and row j of R^T: A-tilde = L[i]^T Rt[j]
    from oracle import philox
    m, n, d = 9, 6, 3
    Om, Ps = philox.test_matrices(5, m, n, d)
    A = np.zeros((m, n))
    A[4, 2] = 1.0
    L, Rt, Ach, At = compress.compress_gaussian(A, Om, Ps)
    assert np.allclose(At, np.outer(L[4], Rt[2]), rtol=0, atol=1e-15)
    assert np.allclose(Ach[4], Rt[2], rtol=0, atol=1e-15)
