"""GPU parity of compressed alternating NMF (Alg. 2) against the oracle:
exact NNLS steps (SciPy Lawson-Hanson per row / column in the oracle) and
the multiplicative updates (Ding et al. Eq. 8, semi-NMF form).

Both sides start from the same Y0 and run the same iterations on the same
inputs (the oracle's L, R^T in the working precision, A in its storage
form); each step's minimiser is unique (full-rank NNLS matrices), so the
iterates agree up to the stopping tolerance and the working precision,
carried through the iterations: FP64 1e-7, FP32 1e-3 of max|X|, max|Y|.
"""
import numpy as np
import pytest

import synth
from oracle import alternating as oalt
from oracle import compress as ocomp
from oracle import philox as ophil

from gpu_util import need_gpu, to_np, to_dev, wdt

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,r,d,iters", [("f64", 4, 10, 3),
                                               ("f32", 4, 10, 3),
                                               ("f64", 8, 16, 20),
                                               ("f32", 8, 16, 20)])
def test_als_matches_oracle(storage, r, d, iters):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n = 300, 220
    As = synth.as_storage(synth.lowrank(m, n, r, 0.02, 21), storage)
    A = synth.widen(As, storage)
    Om, Ps = ophil.test_matrices(22, m, n, d)
    L, Rt, _, _ = ocomp.compress(A, Om, Ps, 2)
    _, Y0 = synth.init_factors(m, n, r, 23)
    if storage == "f32":
        L, Rt, Y0 = (x.astype(np.float32).astype(np.float64) for x in (L, Rt, Y0))
    w = wdt(storage)
    dev = lambda x: torch.tensor(x, dtype=w).cuda()
    tol = 1e-12 if storage == "f64" else 1e-6
    X, Y, unconv, st = cn.cnmf_factor_als(to_dev(As, storage), dev(L), dev(Rt),
                                          dev(Y0), iters, max_sweeps=20000,
                                          tol=tol)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Ac = A @ Rt
    Ah = L.T @ A
    Xo, Yo = oalt.iterate(Ac, Ah, L, Rt, np.zeros((m, r)), Y0, iters, "als")
    Xg, Yg = to_np(X), to_np(Y)
    ex = np.abs(Xg - Xo).max() / np.abs(Xo).max()
    ey = np.abs(Yg - Yo).max() / np.abs(Yo).max()
    print(f"{storage}: X rel err {ex:.2e}, Y rel err {ey:.2e}, unconverged "
          f"{int(unconv.item())}")
    bar = 1e-7 if storage == "f64" else 1e-3
    assert ex <= bar and ey <= bar
    assert Xg.min() >= 0 and Yg.min() >= 0
    # every NNLS column met the stopping rule inside the sweep cap
    assert int(unconv.item()) == 0


@pytest.mark.parametrize("storage,r,d,iters,bar", [("f64", 4, 10, 5, 1e-10),
                                                   ("f32", 4, 10, 5, 1e-5),
                                                   ("f64", 12, 22, 50, 1e-9),
                                                   ("f32", 12, 22, 50, 1e-5),
                                                   ("bf16", 12, 22, 20, 1e-5)])
def test_mu_matches_oracle(storage, r, d, iters, bar):
    """The multiplicative update is a smooth map of (X, Y), so FP32 / BF16
    storage follows the FP64 oracle closely: relative Frobenius error of
    X and Y after `iters` iterations from the same start (X0, Y0) on the
    oracle's L, R^T in the working precision."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n = 400, 330
    As = synth.as_storage(synth.lowrank(m, n, r, 0.02, 31), storage)
    A = synth.widen(As, storage)
    Om, Ps = ophil.test_matrices(32, m, n, d)
    L, Rt, _, _ = ocomp.compress(A, Om, Ps, 2)
    X0, Y0 = synth.init_factors(m, n, r, 33)
    if storage != "f64":
        L, Rt, X0, Y0 = (x.astype(np.float32).astype(np.float64)
                         for x in (L, Rt, X0, Y0))
    w = wdt(storage)
    dev = lambda x: torch.tensor(x, dtype=w).cuda()
    X, Y, st = cn.cnmf_factor_mu(to_dev(As, storage), dev(L), dev(Rt), dev(X0),
                                 dev(Y0), iters)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Xo, Yo = oalt.iterate(A @ Rt, L.T @ A, L, Rt, X0, Y0, iters, "mu")
    Xg, Yg = to_np(X), to_np(Y)
    ex = np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo)
    ey = np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo)
    print(f"mu {storage} r={r}: X {ex:.2e}, Y {ey:.2e}")
    assert ex <= bar and ey <= bar
    assert Xg.min() >= 0 and Yg.min() >= 0
    # zeros stay zeros (the update is multiplicative)
    X0z = X0.copy()
    X0z[::7, 0] = 0.0
    Xz, _, _ = cn.cnmf_factor_mu(to_dev(As, storage), dev(L), dev(Rt),
                                 dev(X0z), dev(Y0), 3)
    assert np.all(to_np(Xz)[::7, 0] == 0.0)
