"""Edge and degenerate cases of the whole path, through the C ABI, against
the FP64 oracle or against what the mathematics fixes.

* sketch size at its limits: d = r, d = min(m, n) (R^T spans all of R^n),
  d = 128 (the largest panel);
* shapes: fewer rows than one 128-row tile, row pitches that are not
  16-byte multiples (the CUDA-core products), one power iteration or none;
* the rank r at its limits for the factorization (r = 1, r = d, and the
  largest working sets of the generic kernel: FP32 d = 128 with r = 32,
  d = 80 with r = 64; FP64 d = 64 with r = 32), sizes beyond them refused
  on the host; for SNMF r = d with q = 0, and r = 1;
* degenerate input: an all-zero A (the first Cholesky breaks down and the
  device status says so), a rank-deficient A with d above its rank (the
  shifted CholeskyQR keeps the basis orthonormal).
"""
import numpy as np
import pytest

import synth
from oracle import admm as oadmm
from oracle import compress as ocomp
from oracle import philox as ophil
from oracle import snmf as osnmf

from gpu_util import need_gpu, rel, to_dev, to_np, wdt

pytestmark = pytest.mark.gpu


def _planted(m, n, d, seed, extra=5):
    g = np.random.default_rng(seed)
    k = min(d + extra, m, n)
    U, _ = np.linalg.qr(g.standard_normal((m, k)))
    V, _ = np.linalg.qr(g.standard_normal((n, k)))
    s = np.concatenate([np.geomspace(100.0, 10.0, min(d, k)),
                        np.full(k - min(d, k), 0.01)])
    return (U * s) @ V.T


@pytest.mark.parametrize("storage,m,n,d,q", [
    ("f32", 33, 77, 5, 0),       # one partial row tile, pitch 77 (CUDA cores)
    ("f32", 200, 40, 40, 1),     # d = n: R^T spans R^n
    ("bf16", 300, 1024, 128, 1), # the largest panel
    ("f64", 129, 130, 128, 2),
])
def test_compress_limits(storage, m, n, d, q):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    As = synth.as_storage(_planted(m, n, d, m + n), storage)
    A = synth.widen(As, storage)
    Ld, Rtd, Atd, st = cn.cnmf_compress(to_dev(As, storage), min(d, 4), d, q,
                                        seed=91)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    L, Rt = to_np(Ld), to_np(Rtd)
    tol = 1e-10 if storage == "f64" else 1e-5
    assert np.linalg.norm(L.T @ L - np.eye(d)) <= tol * d
    assert np.linalg.norm(Rt.T @ Rt - np.eye(d)) <= tol * d
    if d == n:
        assert np.linalg.norm(Rt @ Rt.T - np.eye(n)) <= tol * n
    Om, Ps = ophil.test_matrices(91, m, n, d)
    L0, Rt0, _, _ = ocomp.compress(A, Om, Ps, q)
    # the span of L is well determined where the planted spectrum has its
    # gap (d below the rank) or is all of the range
    assert rel(L @ L.T, L0 @ L0.T) <= (1e-9 if storage == "f64" else 1e-4)


def test_compress_zero_matrix_reports_cholesky_breakdown():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    A = torch.zeros(300, 200, dtype=torch.float32, device="cuda")
    from paper_1505_04650_gb300 import _lib
    _, _, _, st = cn.cnmf_compress(A, 5, 10, 1, seed=3)
    torch.cuda.synchronize()
    assert int(st.item()) == _lib.CNMF_E_CHOLESKY


def test_compress_rank_deficient_stays_orthonormal():
    """Exact rank 3 with d = 12: the Gram of the first panel is singular in
    exact arithmetic; the shifted first sweep keeps the basis defined and
    the range of A is captured exactly."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    A64 = synth.lowrank(400, 300, 3, 0.0, 5)
    A32 = A64.astype(np.float32)
    Ld, Rtd, _, st = cn.cnmf_compress(to_dev(A32, "f32"), 3, 12, 1, seed=8)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    L = to_np(Ld)
    A = A32.astype(np.float64)
    assert np.linalg.norm(L.T @ L - np.eye(12)) <= 1e-4
    assert np.linalg.norm(A - L @ (L.T @ A)) <= 1e-5 * np.linalg.norm(A)


@pytest.mark.parametrize("storage,r,d", [("f32", 1, 2), ("f32", 8, 8),
                                         ("f32", 32, 128), ("f32", 64, 80),
                                         ("f64", 32, 64)])
def test_factor_rank_limits(storage, r, d):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n = 600, 500
    A = synth.lowrank(m, n, r, 0.01, 40 + r)
    if storage == "f32":
        A = A.astype(np.float32).astype(np.float64)
    Om, Ps = ophil.test_matrices(41, m, n, d)
    L, Rt, _, At = ocomp.compress(A, Om, Ps, 1)
    U0, V0 = synth.init_factors(m, n, r, 42)
    if storage == "f32":
        L, Rt, At, U0, V0 = (x.astype(np.float32).astype(np.float64)
                             for x in (L, Rt, At, U0, V0))
    lam = np.linalg.norm(At) / r
    w = wdt(storage)
    dev = lambda x: torch.tensor(x, dtype=w).cuda()
    Ud, Vtd, state, st = cn.cnmf_factor(dev(L), dev(Rt), dev(At), dev(U0),
                                        dev(V0.T.copy()), lam, lam, 20)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = oadmm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=20)
    tol = 1e-10 if storage == "f64" else 1e-4
    assert rel(to_np(Ud), ref.U) <= tol
    assert rel(to_np(Vtd).T, ref.V) <= tol
    assert float(Ud.min()) >= 0.0 and float(Vtd.min()) >= 0.0


def test_factor_beyond_working_set_is_refused():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    from paper_1505_04650_gb300 import CnmfError
    m, n, r, d = 300, 280, 64, 128
    dev = lambda *s: torch.rand(*s, device="cuda")
    with pytest.raises(CnmfError):
        cn.cnmf_factor(dev(m, d), dev(n, d), dev(d, d), dev(m, r), dev(n, r),
                       1.0, 1.0, 2)


@pytest.mark.parametrize("r,q", [(10, 0), (1, 1)])
def test_snmf_limits(r, q):
    """r = d (no oversampling) and q = 0, or a single anchor, on noiseless
    separable matrices: the planted anchors, bit-exact (Alg. 3, SPA).  With
    r = 1 the Dirichlet columns are all 1, so every column is the anchor:
    all norms tie and the lowest index wins."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n = 150, 900
    A64, planted = synth.separable(m, n, r, 0.0, 77 + r)
    A32 = A64.astype(np.float32)
    anchors, st = cn.snmf_select(to_dev(A32, "f32"), r, r, q, seed=5)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    want = [0] if r == 1 else sorted(planted.tolist())
    assert sorted(anchors.cpu().tolist()) == want
    K, _, _, _ = osnmf.snmf_select(A32.astype(np.float64),
                                   ophil.gaussian_matrix(5, 0, n, r), r, q)
    assert sorted(K) == want
