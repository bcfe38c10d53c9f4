"""GPU parity of Alg. 3 step 3 (the right factor: per-column NNLS on the
compressed matrix) against the oracle (SciPy's Lawson-Hanson per column).

Both sides solve the same problem: the oracle reads the FP64 widening of
the Rhat_t the GPU reads.  With Rhat[:, K] of full column rank the NNLS
minimiser is unique, so the GPU's coordinate-descent result must approach
it.  A perturbation of G or b of relative size eps moves the minimiser by
about kappa(G) eps, so the bar is 100 kappa(G) u of max|Y| in the working
precision (at least 1e-9 for FP64, 1e-5 for FP32), with the stopping
tolerance well below it.
"""
import numpy as np
import pytest

import synth
from oracle import snmf as osnmf

from gpu_util import need_gpu, to_np

pytestmark = pytest.mark.gpu


def _bar(Rw, K, fp64):
    B = Rw[:, K]
    kappa = np.linalg.cond(B.T @ B)
    u = 2.0 ** -53 if fp64 else 2.0 ** -24
    return max(100 * kappa * u, 1e-9 if fp64 else 1e-5), kappa


def _run(torch, Rt, K, dtype, tol, sweeps=2000):
    import paper_1505_04650_gb300 as cn
    Rd = torch.tensor(Rt, dtype=dtype).cuda()
    Kd = torch.tensor(np.asarray(K, dtype=np.int64)).cuda()
    Y, unconv, st = cn.snmf_right_factor(Rd, Kd, max_sweeps=sweeps, tol=tol)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return to_np(Y), int(unconv.item()), to_np(Rd)


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
@pytest.mark.parametrize("d,n,r", [(20, 1000, 6), (12, 129, 1), (40, 300, 17),
                                   (96, 257, 64), (30, 1, 5)])
def test_right_factor_random_matches_oracle(dtype_name, d, n, r):
    torch = need_gpu()
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    g = np.random.default_rng(d * 1000 + n + r)
    Rt = g.standard_normal((max(n, r), d))
    n = Rt.shape[0]
    K = g.choice(n, r, replace=False)
    tol = 1e-12 if dtype_name == "f64" else 1e-6
    Y, unconv, Rw = _run(torch, Rt, K, dtype, tol, sweeps=20000)
    Yo = osnmf.right_factor(Rw.T, K)
    scale = max(np.abs(Yo).max(), 1e-300)
    err = np.abs(Y - Yo).max() / scale
    bar, kappa = _bar(Rw.T, K, dtype_name == "f64")
    print(f"{dtype_name} d={d} n={n} r={r}: max rel err {err:.2e} "
          f"(bar {bar:.1e}, kappa(G) {kappa:.1e}), unconverged {unconv}")
    assert err <= bar
    assert unconv == 0
    assert Y.min() >= 0.0


def test_right_factor_after_snmf_select():
    """The pipeline: anchors and Rhat^T from snmf_select on a near-separable
    matrix, then the right factor; the anchors' own columns come back as
    unit vectors and the fit matches the oracle on the same Rhat."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, r, d = 400, 3000, 5, 12
    A, planted = synth.separable(m, n, r, 0.001, 31, dtype=np.float32)
    Ad = torch.tensor(A).cuda()
    anchors, Rt, st = cn.snmf_select(Ad, r, d, 2, seed=9, return_rhat=True)
    Y, unconv, st2 = cn.snmf_right_factor(Rt, anchors, max_sweeps=5000, tol=1e-7)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(st2.item()) == 0
    K = anchors.cpu().numpy()
    assert sorted(K) == sorted(planted)
    Yg = to_np(Y)
    Rw = to_np(Rt).T
    Yo = osnmf.right_factor(Rw, K)
    err = np.abs(Yg - Yo).max() / np.abs(Yo).max()
    bar, kappa = _bar(Rw, K, False)
    print(f"pipeline max rel err {err:.2e} (bar {bar:.1e}, kappa(G) "
          f"{kappa:.1e}), unconverged {int(unconv.item())}")
    assert err <= bar
    for j, k in enumerate(K):
        e = np.zeros(r)
        e[j] = 1.0
        assert np.abs(Yg[:, k] - e).max() <= bar


def test_right_factor_degenerate_columns():
    """A zero column fits with h = 0; a column equal to an anchor with that
    anchor's unit vector; an anchor index outside [0, n) is reported."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    g = np.random.default_rng(5)
    n, d, r = 200, 10, 4
    Rt = g.standard_normal((n, d))
    K = np.array([3, 50, 77, 120])
    Rt[10] = 0.0
    Rt[11] = Rt[50]
    Y, unconv, _ = _run(torch, Rt, K, torch.float64, 1e-12)
    assert np.abs(Y[:, 10]).max() == 0.0
    assert np.abs(Y[:, 11] - np.eye(r)[:, 1]).max() <= 1e-9
    Rd = torch.tensor(Rt).cuda()
    bad = torch.tensor(np.array([3, 50, 77, n], dtype=np.int64)).cuda()
    Yb, _, st = cn.snmf_right_factor(Rd, bad)
    torch.cuda.synchronize()
    assert int(st.item()) == 1   # CNMF_E_INVALID_ARG
