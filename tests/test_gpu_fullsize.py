"""Full-size workloads, checked where the oracle cannot run end to end:
through properties that hold at any size and through outputs the oracle can
compute one by one (sampled rows and columns of the products).

* compressed NMF at the bench's size (20000 x 10000, r = 20, d = 30, q = 4,
  500 sweeps, FP32, the launch configuration bench.py times): orthonormal
  L and R, nonnegative factors, and the final relative residual against
  the closed-form rank-r noise floor of the synthetic recipe;
* compressed SNMF on the wide separable workload (10000 x 100000, r = 50,
  d = 60, q = 2): the planted anchor set, bit-exact (Alg. 3; SPA recovers
  the extreme columns of a separable matrix, Sec. I / Sec. IV);
* the sketch products at the mixed-precision size (50000 x 50000, d = 80)
  for BF16 and FP32 storage: sampled rows of A X and columns of A^T Y
  against FP64 within the product bound;
* the mixed-precision error statement: projector and objective of the
  BF16 / FP32 paths against the FP64 oracle at a size it can run;
* parity with the FP64 oracle at the bench's size itself: the oracle's
  compression of the same FP32 matrix (same Omega, Psi), the rank-r signal
  projector (1e-5), the signal singular values of A-tilde, and 20 ADMM
  sweeps from the oracle's L, R^T, A-tilde (factors 1e-4).
"""
import math

import numpy as np
import pytest

import synth
from oracle import admm as oadmm
from oracle import compress as ocomp
from oracle import philox as ophil
from oracle import residual as ores

from gpu_util import need_gpu, product_bound, rel, to_dev, to_np, wdt

pytestmark = pytest.mark.gpu


def _noise_floor(r, sigma):
    """Relative rank-r floor of A = X0 Y0 + |N(0, sigma^2)|, X0, Y0 ~ U[0,1):
    the residual is the centred noise, std sigma sqrt(1 - 2/pi), against
    E[a^2] = r^2/16 + r (1/9 - 1/16) per entry."""
    return sigma * math.sqrt(1 - 2 / math.pi) / math.sqrt(r * r / 16 + r * (1 / 9 - 1 / 16))


def test_cnmf_fullsize_bench_workload():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, r, d, q, iters = 20000, 10000, 20, 30, 4, 500
    A = synth.lowrank_torch(m, n, r, 0.01, 1001)
    U0, Vt0 = synth.init_torch(m, n, r, 3001)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    L, Rt, At, _ = cn.cnmf_compress(A, r, d, q, 2001, status=st)
    lam = cn.default_penalty(At, r)
    U, Vt, state, _ = cn.cnmf_factor(L, Rt, At, U0.clone(), Vt0.clone(), lam,
                                     lam, iters, status=st)
    res = cn.cnmf_residual(A, U, Vt)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Ln, Rn = to_np(L), to_np(Rt)
    assert np.abs(Ln.T @ Ln - np.eye(d)).max() <= 1e-5
    assert np.abs(Rn.T @ Rn - np.eye(d)).max() <= 1e-5
    assert float(U.min()) >= 0.0 and float(Vt.min()) >= 0.0
    assert int(state.k.item()) == iters
    rho = math.sqrt(float(res[0]) / float(res[1]))
    # the same residual in FP64 on the host
    Ah = A.double().cpu().numpy()
    rho_h = ores.rel_residual(Ah, to_np(U), to_np(Vt).T)
    assert abs(rho - rho_h) <= 1e-6 * rho_h
    floor = _noise_floor(r, 0.01)
    print(f"rho {rho:.4e}  noise floor {floor:.4e}")
    assert 0.99 * floor <= rho <= floor + 1e-3


def test_snmf_fullsize_wide_planted_anchors():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, r, d, q = 10000, 100000, 50, 60, 2
    A, planted = synth.separable_torch(m, n, r, 1e-3, 1002)
    anchors, st = cn.snmf_select(A, r, d, q, seed=2002)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert sorted(anchors.cpu().tolist()) == sorted(planted.cpu().tolist())


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_products_fullsize_sampled(storage):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m = n = 50000
    k = 80
    A = synth.lowrank_torch(m, n, 64, 0.01, 1003)
    if storage == "bf16":
        A = A.to(torch.bfloat16)
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    X = torch.randn(n, k, generator=g, device="cuda")
    Y = torch.randn(m, k, generator=g, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Zm, Zn = cn.cnmf_sketch_pass(A, X, Y, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    rows = np.random.default_rng(7).choice(m, 16, replace=False)
    cols = np.random.default_rng(8).choice(n, 16, replace=False)
    Xh, Yh = to_np(X), to_np(Y)
    Ar = to_np(A[torch.as_tensor(rows, device="cuda")])            # 16 x n
    Ac = to_np(A[:, torch.as_tensor(cols, device="cuda")]).T        # 16 x m
    zm = to_np(Zm[torch.as_tensor(rows, device="cuda")])
    zn = to_np(Zn[torch.as_tensor(cols, device="cuda")])
    assert np.all(np.abs(zm - Ar @ Xh) <= product_bound(storage, n) * (np.abs(Ar) @ np.abs(Xh)))
    assert np.all(np.abs(zn - Ac @ Yh) <= product_bound(storage, m) * (np.abs(Ac) @ np.abs(Yh)))


def _signal_projector(L, A, r):
    U, _, _ = np.linalg.svd(L @ (L.T @ A), full_matrices=False)
    return U[:, :r] @ U[:, :r].T


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("q", [3, 4])
def test_mixed_precision_errors_vs_oracle(storage, q):
    """The mixed-precision sketch (BF16 storage / FP32 on 3xTF32 tensor
    cores, FP64-accurate CholeskyQR2) against the FP64 oracle run on the
    values the GPU reads: rank-r signal projector and the objective after
    100 sweeps.  BF16 is also compared with the FP64 matrix it was rounded
    from (the accuracy cost of the storage, not a parity figure)."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m = n = 3000
    r, d, iters = 64, 80, 100
    A64 = synth.lowrank(m, n, r, 0.01, 1003)
    As = synth.as_storage(A64, storage)
    Aw = synth.widen(As, storage)
    Om, Ps = ophil.test_matrices(2003, m, n, d)
    L0, Rt0, _, At0 = ocomp.compress(Aw, Om, Ps, q)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    L, Rt, At, _ = cn.cnmf_compress(to_dev(As, storage), r, d, q, 2003, status=st)
    U0, V0 = synth.init_factors(m, n, r, 3003)
    lam = float(np.linalg.norm(At0)) / r
    U, Vt, _, _ = cn.cnmf_factor(L, Rt, At, torch.tensor(U0, dtype=torch.float32).cuda(),
                                 torch.tensor(V0.T.copy(), dtype=torch.float32).cuda(),
                                 lam, lam, iters, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ep = rel(_signal_projector(to_np(L), Aw, r), _signal_projector(L0, Aw, r))
    ref = oadmm.admm(L0, Rt0, At0, U0, V0, lam=lam, phi=lam, iters=iters)
    rg = ores.rel_residual(Aw, to_np(U), to_np(Vt).T)
    ro = ores.rel_residual(Aw, ref.U, ref.V)
    eo = abs(rg - ro) / ro
    msg = f"{storage} q={q}: projector {ep:.2e}  objective {eo:.2e} (rho {rg:.4e} vs {ro:.4e})"
    if storage == "bf16":
        msg += f"  vs FP64 A: rho {ores.rel_residual(A64, to_np(U), to_np(Vt).T):.4e}"
    print(msg)
    assert ep <= 1e-5
    assert eo <= 1e-3


def _signal_basis(L, A, r):
    """Top-r left singular vectors of L L^T A, as L W_r from the SVD of the
    d x n matrix L^T A (the m x m projector itself is not formed)."""
    W, _, _ = np.linalg.svd(L.T @ A, full_matrices=False)
    return L @ W[:, :r]


def _projector_distance(U1, U2):
    """||U1 U1^T - U2 U2^T||_F / ||U2 U2^T||_F for orthonormal U1, U2 of
    rank r: sqrt(2) ||U1 - U2 (U2^T U1)||_F / sqrt(r), free of the
    cancellation in 2 r - 2 ||U2^T U1||_F^2."""
    r = U2.shape[1]
    return float(np.sqrt(2.0) * np.linalg.norm(U1 - U2 @ (U2.T @ U1)) / np.sqrt(r))


def test_cnmf_bench_size_matches_oracle():
    """m = 20000, n = 10000, r = 20, d = 30, q = 4, FP32: the workload the
    bench times, compared with the FP64 oracle on the values the GPU
    reads."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, r, d, q = 20000, 10000, 20, 30, 4
    A = synth.lowrank(m, n, r, 0.01, 1001, dtype=np.float32)
    Aw = A.astype(np.float64)
    Om, Ps = ophil.test_matrices(2001, m, n, d)
    L0, Rt0, _, At0 = ocomp.compress(Aw, Om, Ps, q)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Ad = torch.from_numpy(A).cuda()
    L, Rt, At, _ = cn.cnmf_compress(Ad, r, d, q, 2001, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Lg, Rg, Ag = to_np(L), to_np(Rt), to_np(At)
    # signal projectors of both sides
    ep_l = _projector_distance(_signal_basis(Lg, Aw, r), _signal_basis(L0, Aw, r))
    ep_r = _projector_distance(_signal_basis(Rg, Aw.T, r), _signal_basis(Rt0, Aw.T, r))
    # A-tilde: its signal singular values are basis-free
    sg = np.linalg.svd(Ag, compute_uv=False)
    so = np.linalg.svd(At0, compute_uv=False)
    es = float(np.abs(sg[:r] - so[:r]).max() / so[0])
    print(f"signal projector L {ep_l:.2e}, R {ep_r:.2e}; A-tilde singular values {es:.2e}")
    assert ep_l <= 1e-5 and ep_r <= 1e-5
    assert es <= 1e-5
    # 20 sweeps from the oracle's compression (rounded to the FP32 inputs)
    f32 = lambda x: x.astype(np.float32).astype(np.float64)
    Lf, Rtf, Atf = f32(L0), f32(Rt0), f32(At0)
    U0, V0 = synth.init_factors(m, n, r, 3001)
    U0, V0 = f32(U0), f32(V0)
    lam = float(np.linalg.norm(Atf)) / r
    dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")
    U, Vt, _, _ = cn.cnmf_factor(dev(Lf), dev(Rtf), dev(Atf), dev(U0),
                                 dev(V0.T.copy()), lam, lam, 20, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = oadmm.admm(Lf, Rtf, Atf, U0, V0, lam=lam, phi=lam, iters=20)
    eu = rel(to_np(U), ref.U)
    ev = rel(to_np(Vt).T, ref.V)
    print(f"20 sweeps: U {eu:.2e}, V {ev:.2e}")
    assert eu <= 1e-4 and ev <= 1e-4


def test_noiseless_bench_size_rank_deficient():
    """The bench shape without noise (A = X0 Y0 exactly: rank r = 20 below
    the sketch size d = 30, FP32): the compression must still return
    orthonormal L and R^T (the null directions are an arbitrary orthonormal
    completion) that capture A, A = L A-tilde R to FP32 rounding, and the
    compressed ADMM must reach rho <= 1e-3 as the FP64 oracle does on the
    same A (5.5e-4 after 200 sweeps at lambda = ||A-tilde|| / r).  The
    shifted first CholeskyQR sweep of each pass and the final unshifted
    one both meet a numerically rank-deficient panel here."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, r, d, q = 20000, 10000, 20, 30, 4
    A = torch.from_numpy(synth.lowrank(m, n, r, 0.0, 1001,
                                       dtype=np.float32)).cuda()
    L, Rt, At, st = cn.cnmf_compress(A, r, d, q, 2001)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    I = torch.eye(d, dtype=torch.float64, device="cuda")
    for P in (L, Rt):
        P = P.double()
        assert float(torch.linalg.norm(P.t() @ P - I)) <= 1e-4
    Ad = A.double()
    cap = torch.linalg.norm(Ad - (L.double() @ At.double()) @ Rt.double().t())
    assert float(cap / torch.linalg.norm(Ad)) <= 1e-5
    U0, V0 = synth.init_factors(m, n, r, 3001)
    U = torch.tensor(U0, dtype=torch.float32, device="cuda")
    Vt = torch.tensor(V0.T.copy(), dtype=torch.float32, device="cuda")
    lam = float(torch.linalg.norm(At.double())) / r
    cn.cnmf_factor(L, Rt, At, U, Vt, lam, lam, 400, status=st)
    e2, a2 = cn.cnmf_residual(A, U, Vt).cpu().tolist()
    cn.raise_on_status(st, "noiseless factor")
    assert math.sqrt(e2 / a2) <= 1e-3
