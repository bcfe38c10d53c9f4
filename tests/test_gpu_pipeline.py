"""GPU parity of the three entry points against the FP64 oracle.

cnmf_compress (Alg. 1 on A and A^T + A-tilde), cnmf_factor (Alg. 4),
cnmf_factor_plain (Alg. 4 with L = I, R = I) and snmf_select (Alg. 3 steps
1-2).  Both sides get the same inputs: the GPU reads the storage-form A, the
oracle its FP64 widening; test matrices come from the same Philox stream;
factor tests feed both sides the oracle's (L, Rt, Atilde) in the working
precision.  Acceptance (the tolerances the readings of the paper fix):
projector 1e-5 (FP32, planted well-conditioned input and the rank-r signal
projector) / 1e-10 (FP64); U, V after 20 sweeps 1e-4 (FP32) / 1e-10
(FP64); final objective 1e-3; SNMF anchors bit-exact as a set.
"""
import numpy as np
import pytest

import synth
from oracle import admm as oadmm
from oracle import compress as ocomp
from oracle import philox as ophil
from oracle import residual as ores
from oracle import snmf as osnmf

from gpu_util import need_gpu, rel, to_dev, to_np, wdt

pytestmark = pytest.mark.gpu


def _planted_spectrum(m, n, d, seed):
    """sigma_1 / sigma_d = 10, gap sigma_d / sigma_{d+1} = 1e3, A >= 0 not
    required for the compression."""
    g = np.random.default_rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((m, d + 5)))
    V, _ = np.linalg.qr(g.standard_normal((n, d + 5)))
    s = np.concatenate([np.geomspace(100.0, 10.0, d), np.full(5, 0.01)])
    return (U * s) @ V.T


def _signal_projector(L, A, r):
    Ub, _, _ = np.linalg.svd(L @ (L.T @ A), full_matrices=False)
    return Ub[:, :r] @ Ub[:, :r].T


@pytest.mark.parametrize("m,n,r,d,q,sigma", [(500, 400, 10, 20, 4, 0.01),
                                             (97, 131, 3, 9, 1, 0.05),
                                             (60, 50, 4, 4, 0, 0.0)])
def test_compress_fp64_matches_oracle(m, n, r, d, q, sigma):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    A = synth.lowrank(m, n, r, sigma, 1000 + m)
    Ld, Rtd, Atd, st = cn.cnmf_compress(to_dev(A, "f64"), r, d, q, seed=2000)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Om, Ps = ophil.test_matrices(2000, m, n, d)
    L0, Rt0, _, At0 = ocomp.compress(A, Om, Ps, q)
    L, Rt, At = to_np(Ld), to_np(Rtd), to_np(Atd)
    assert rel(L @ L.T, L0 @ L0.T) <= 1e-10
    assert rel(Rt @ Rt.T, Rt0 @ Rt0.T) <= 1e-10
    if sigma > 0:   # full rank sketches: Q unique -> elementwise
        assert np.abs(L - L0).max() <= 1e-9
        assert np.abs(Rt - Rt0).max() <= 1e-9
        assert rel(At, At0) <= 1e-9


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_compress_fp32_planted_projector(storage):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, d = 700, 520, 12
    As = synth.as_storage(_planted_spectrum(m, n, d, 5), storage)
    A = synth.widen(As, storage)
    Ld, Rtd, Atd, st = cn.cnmf_compress(to_dev(As, storage), d, d, 2, seed=77)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Om, Ps = ophil.test_matrices(77, m, n, d)
    L0, Rt0, _, At0 = ocomp.compress(A, Om, Ps, 2)
    L, Rt = to_np(Ld), to_np(Rtd)
    assert rel(L @ L.T, L0 @ L0.T) <= 1e-5
    assert rel(Rt @ Rt.T, Rt0 @ Rt0.T) <= 1e-5
    assert np.linalg.norm(L.T @ L - np.eye(d)) <= 1e-5


def test_compress_fp32_noisy_signal_projector():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, r, d = 2000, 1500, 10, 20
    A32 = synth.as_storage(synth.lowrank(m, n, r, 0.01, 1001), "f32")
    A = A32.astype(np.float64)
    Ld, Rtd, Atd, st = cn.cnmf_compress(to_dev(A32, "f32"), r, d, 4, seed=2001)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Om, Ps = ophil.test_matrices(2001, m, n, d)
    L0, Rt0, _, At0 = ocomp.compress(A, Om, Ps, 4)
    L, Rt = to_np(Ld), to_np(Rtd)
    assert rel(_signal_projector(L, A, r), _signal_projector(L0, A, r)) <= 1e-5
    assert rel(_signal_projector(Rt, A.T, r),
               _signal_projector(Rt0, A.T, r)) <= 1e-5
    full = rel(L @ L.T, L0 @ L0.T)
    print(f"full projector FP32 vs FP64 oracle (noise directions): {full:.2e}")
    # compression quality equals the oracle's
    e_gpu = np.linalg.norm(A - L @ (L.T @ A))
    e_ora = np.linalg.norm(A - L0 @ (L0.T @ A))
    assert abs(e_gpu - e_ora) <= 1e-4 * e_ora


def _factor_case(m, n, r, d, q, sigma, seed, storage):
    A = synth.lowrank(m, n, r, sigma, seed)
    if storage == "f32":
        A = A.astype(np.float32).astype(np.float64)
    Om, Ps = ophil.test_matrices(seed + 1, m, n, d)
    L, Rt, _, At = ocomp.compress(A, Om, Ps, q)
    U0, V0 = synth.init_factors(m, n, r, seed + 2)
    if storage == "f32":
        L, Rt, At, U0, V0 = (x.astype(np.float32).astype(np.float64)
                             for x in (L, Rt, At, U0, V0))
    return A, L, Rt, At, U0, V0


def _check_kept_inverse(state, phi, storage):
    """The state's kept Zy is -(Xt^T Xt + phi I)^-1 of the final Xt (the
    inverse the last Y update used), whichever way the kernel formed it."""
    sec = state._sections()
    Xt = to_np(sec["Xt"])
    Zy = to_np(sec["Z"][1])
    r = Xt.shape[1]
    ref = -np.linalg.inv(Xt.T @ Xt + phi * np.eye(r))
    tol = 1e-10 if storage == "f64" else 1e-4
    assert rel(Zy, ref) <= tol


@pytest.mark.parametrize("storage,iters", [("f64", 300), ("f32", 300)])
def test_factor_long_run_matches_oracle(storage, iters):
    """Hundreds of sweeps: after the first few the solves' inverses are
    refined from the previous sweep's, so this exercises that path."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    A, L, Rt, At, U0, V0 = _factor_case(500, 400, 10, 20, 4, 0.01, 1000,
                                        storage)
    lam = np.linalg.norm(At) / 10
    w = wdt(storage)
    dev = lambda x: torch.tensor(x, dtype=w).cuda()
    Ud, Vtd = dev(U0), dev(V0.T.copy())
    Ud, Vtd, state, st = cn.cnmf_factor(dev(L), dev(Rt), dev(At), Ud, Vtd,
                                        lam, lam, iters)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = oadmm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=iters)
    eu, ev = rel(to_np(Ud), ref.U), rel(to_np(Vtd).T, ref.V)
    print(f"{iters} sweeps: U rel err {eu:.2e}  V rel err {ev:.2e}")
    tol = 1e-9 if storage == "f64" else 1e-3
    assert eu <= tol and ev <= tol
    _check_kept_inverse(state, lam, storage)
    rg = ores.rel_residual(A, to_np(Ud), to_np(Vtd).T)
    ro = ores.rel_residual(A, ref.U, ref.V)
    assert abs(rg - ro) <= 1e-3 * ro


@pytest.mark.parametrize("storage,m,n,r,d", [("f64", 500, 400, 10, 20),
                                             ("f32", 500, 400, 10, 20),
                                             ("f32", 3000, 2000, 20, 30),
                                             ("f32", 77, 1031, 5, 15)])
def test_factor_20_sweeps_matches_oracle(storage, m, n, r, d):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    A, L, Rt, At, U0, V0 = _factor_case(m, n, r, d, 4, 0.01, 1000, storage)
    lam = np.linalg.norm(At) / r
    w = wdt(storage)
    dev = lambda x: torch.tensor(x, dtype=w).cuda()
    Ud, Vtd = dev(U0), dev(V0.T.copy())
    Ud, Vtd, state, st = cn.cnmf_factor(dev(L), dev(Rt), dev(At), Ud, Vtd,
                                        lam, lam, 20)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = oadmm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=20)
    tol = 1e-10 if storage == "f64" else 1e-4
    eu, ev = rel(to_np(Ud), ref.U), rel(to_np(Vtd).T, ref.V)
    print(f"U rel err {eu:.2e}  V rel err {ev:.2e}")
    assert eu <= tol and ev <= tol
    assert int(state.k.item()) == 20
    _check_kept_inverse(state, lam, storage)
    # final objective within 1e-3
    rg = ores.rel_residual(A, to_np(Ud), to_np(Vtd).T)
    ro = ores.rel_residual(A, ref.U, ref.V)
    assert abs(rg - ro) <= 1e-3 * ro


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_factor_resume_bitwise(storage):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    A, L, Rt, At, U0, V0 = _factor_case(300, 260, 6, 12, 2, 0.02, 7, storage)
    lam = np.linalg.norm(At) / 6
    w = wdt(storage)
    dev = lambda x: torch.tensor(x, dtype=w).cuda()
    Ld, Rtd, Atd = dev(L), dev(Rt), dev(At)
    Ua, Va = dev(U0), dev(V0.T.copy())
    cn.cnmf_factor(Ld, Rtd, Atd, Ua, Va, lam, lam, 30)
    Ub, Vb = dev(U0), dev(V0.T.copy())
    _, _, state, _ = cn.cnmf_factor(Ld, Rtd, Atd, Ub, Vb, lam, lam, 11)
    cn.cnmf_factor(Ld, Rtd, Atd, Ub, Vb, lam, lam, 19, state=state)
    torch.cuda.synchronize()
    assert torch.equal(Ua, Ub) and torch.equal(Va, Vb)
    assert int(state.k.item()) == 30


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_plain_admm_matches_oracle(storage):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, r = 400, 333, 8
    As = synth.as_storage(synth.lowrank(m, n, r, 0.01, 21), storage)
    A = synth.widen(As, storage)
    U0, V0 = synth.init_factors(m, n, r, 22)
    w = wdt(storage)
    if storage != "f64":
        U0 = U0.astype(np.float32).astype(np.float64)
        V0 = V0.astype(np.float32).astype(np.float64)
    lam = np.linalg.norm(A) / r
    Ud = torch.tensor(U0, dtype=w).cuda()
    Vtd = torch.tensor(V0.T.copy(), dtype=w).cuda()
    Ud, Vtd, state, st = cn.cnmf_factor_plain(to_dev(As, storage), Ud, Vtd,
                                              lam, lam, 20)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = oadmm.admm_plain(A, U0, V0, lam=lam, phi=lam, iters=20)
    tol = 1e-10 if storage == "f64" else 1e-4
    eu, ev = rel(to_np(Ud), ref.U), rel(to_np(Vtd).T, ref.V)
    print(f"plain U rel err {eu:.2e}  V rel err {ev:.2e}")
    assert eu <= tol and ev <= tol
    assert int(state.k.item()) == 20


@pytest.mark.parametrize("storage,m,n,r,d,q", [("f64", 200, 1500, 10, 20, 2),
                                               ("f32", 300, 2000, 10, 20, 2),
                                               ("bf16", 256, 3001, 12, 24, 1),
                                               ("f32", 1000, 10000, 50, 60, 2)])
def test_snmf_anchors_match_oracle(storage, m, n, r, d, q):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    A64, planted = synth.separable(m, n, r, 1e-3, 3000 + n)
    As = synth.as_storage(A64, storage)
    A = synth.widen(As, storage)
    anchors, rh, st = cn.snmf_select(to_dev(As, storage), r, d, q, seed=4000,
                                     return_rhat=True)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Om = ophil.gaussian_matrix(4000, 0, n, d)
    K, margins, Q, Rhat = osnmf.snmf_select(A, Om, r, q)
    got = anchors.cpu().numpy()
    # the planted anchor set, bit-exact, on both sides
    assert sorted(K) == sorted(planted)
    assert sorted(got) == sorted(planted)
    # where every SPA step is decided with margin >= 1e-4 the selection
    # order is unique too
    if margins.min() >= 1e-4:
        assert list(got) == list(K)
    print(f"min SPA margin {margins.min():.2e}")
    # Rhat^T is basis-dependent only through Q, which is unique
    assert rel(to_np(rh), Rhat.T) <= (1e-10 if storage == "f64" else 1e-4)


@pytest.mark.parametrize("limit", [7, "half"])
def test_cta_limit_two_streams_match_oracle(limit):
    """cnmf_set_thread_cta_limit: a compression on one stream beside the
    ADMM sweeps of another problem on a second stream, each grid capped,
    both still match the oracle (compression: signal projector 1e-5;
    ADMM: U, V after 20 sweeps 1e-4)."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    cap = nsm // 2 if limit == "half" else limit
    m, n, r, d = 2000, 1500, 10, 20
    A32 = synth.as_storage(synth.lowrank(m, n, r, 0.01, 1001), "f32")
    A = A32.astype(np.float64)
    Af, L, Rt, At, U0, V0 = _factor_case(3000, 2000, 20, 30, 4, 0.01, 1000, "f32")
    lam = np.linalg.norm(At) / 20
    dev = lambda x: torch.tensor(x, dtype=torch.float32).cuda()
    Ad = to_dev(A32, "f32")
    Ld_in, Rtd_in, Atd_in = dev(L), dev(Rt), dev(At)
    Ud, Vtd = dev(U0), dev(V0.T.copy())
    sA, sB = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    try:
        cn.set_thread_cta_limit(cap)
        with torch.cuda.stream(sA):
            Ud, Vtd, state, stf = cn.cnmf_factor(Ld_in, Rtd_in, Atd_in, Ud, Vtd,
                                                 lam, lam, 20)
        with torch.cuda.stream(sB):
            Ld, Rtd, Atd, stc = cn.cnmf_compress(Ad, r, d, 4, seed=2001)
        torch.cuda.synchronize()
    finally:
        cn.set_thread_cta_limit(0)
    assert int(stf.item()) == 0 and int(stc.item()) == 0
    Om, Ps = ophil.test_matrices(2001, m, n, d)
    L0, Rt0, _, _ = ocomp.compress(A, Om, Ps, 4)
    assert rel(_signal_projector(to_np(Ld), A, r), _signal_projector(L0, A, r)) <= 1e-5
    assert rel(_signal_projector(to_np(Rtd), A.T, r),
               _signal_projector(Rt0, A.T, r)) <= 1e-5
    ref = oadmm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=20)
    eu, ev = rel(to_np(Ud), ref.U), rel(to_np(Vtd).T, ref.V)
    assert eu <= 1e-4 and ev <= 1e-4


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_compress_gaussian_matches_oracle(storage):
    """The Gaussian-compression baseline: L, R^T are the scaled Philox test
    matrices (elementwise, the Gaussian's own rounding plus one product),
    A-tilde = L^T A R^T within a componentwise bound on |L|^T |A| |R^T|
    (FP64: 1e-12; FP32 / BF16 storage with FP32 work: 1e-4)."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, d = 300, 257, 12
    As = synth.as_storage(synth.lowrank(m, n, 5, 0.01, 77), storage)
    Aw = synth.widen(As, storage)
    Ld, Rtd, Atd, st = cn.cnmf_compress_gaussian(to_dev(As, storage), d, seed=123)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Om, Ps = ophil.test_matrices(123, m, n, d)
    L0, Rt0, _, At0 = ocomp.compress_gaussian(Aw, Om, Ps)
    L, Rt, At = to_np(Ld), to_np(Rtd), to_np(Atd)
    u = 2.0 ** -53 if storage == "f64" else 2.0 ** -24
    assert np.abs(L - L0).max() <= 8 * u * np.abs(L0).max()
    assert np.abs(Rt - Rt0).max() <= 8 * u * np.abs(Rt0).max()
    bound = np.abs(L0).T @ np.abs(Aw) @ np.abs(Rt0)
    tol = 1e-12 if storage == "f64" else 1e-4
    assert np.all(np.abs(At - At0) <= tol * bound)
