"""GPU tests of the batched compressed ADMM (cnmf_factor_batched).

A problem's result must not depend on the batch it runs in (bitwise), nor on
how its sweeps are split over launches (bitwise); it must match the oracle's
Alg. 4 (1e-4 after 20 sweeps, as the single-problem kernel) for every
cluster size.
"""
import numpy as np
import pytest

import synth
from oracle import admm as oadmm
from oracle import compress as ocomp
from oracle import philox as ophil

from gpu_util import need_gpu, rel, to_np

pytestmark = pytest.mark.gpu

SHAPES = [(500, 400, 10, 20), (1201, 333, 5, 15), (257, 3001, 32, 42),
          (2000, 1500, 20, 30)]


def _case(m, n, r, d, seed):
    A = synth.lowrank(m, n, r, 0.01, seed).astype(np.float32).astype(np.float64)
    Om, Ps = ophil.test_matrices(seed + 1, m, n, d)
    L, Rt, _, At = ocomp.compress(A, Om, Ps, 2)
    U0, V0 = synth.init_factors(m, n, r, seed + 2)
    f32 = lambda x: x.astype(np.float32).astype(np.float64)
    return A, f32(L), f32(Rt), f32(At), f32(U0), f32(V0)


def _problem(torch, cn, case):
    A, L, Rt, At, U0, V0 = case
    r = U0.shape[1]
    lam = float(np.linalg.norm(At)) / r
    dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")
    return cn.BatchProblem(dev(L), dev(Rt), dev(At), dev(U0), dev(V0.T.copy()),
                           lam, lam)


@pytest.mark.parametrize("cs", [1, 2, 4, 8])
def test_batched_matches_oracle(cs):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    cases = [_case(*s, seed=100 + i) for i, s in enumerate(SHAPES)]
    probs = [_problem(torch, cn, c) for c in cases]
    _, st = cn.cnmf_factor_batched(probs, 7, cluster_size=cs)
    _, st = cn.cnmf_factor_batched(probs, 13, cluster_size=cs, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    for pb, (A, L, Rt, At, U0, V0) in zip(probs, cases):
        lam = pb.lam
        ref = oadmm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=20)
        eu, ev = rel(to_np(pb.U), ref.U), rel(to_np(pb.Vt).T, ref.V)
        assert eu <= 1e-4 and ev <= 1e-4, (pb.m, pb.n, pb.r, eu, ev)
        assert int(pb.state.k.item()) == 20


def test_batched_alone_equals_in_mix_and_split_equals_whole():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    cases = [_case(*s, seed=200 + i) for i, s in enumerate(SHAPES)]
    mix = [_problem(torch, cn, c) for c in cases]
    alone = _problem(torch, cn, cases[2])
    whole = _problem(torch, cn, cases[2])
    # mix: problem 2 among others (and an empty slot), sweeps split 5 + 15
    cn.cnmf_factor_batched(mix[:2] + [None] + mix[2:], 5, cluster_size=2)
    cn.cnmf_factor_batched(mix[:2] + [None] + mix[2:], 15, cluster_size=2)
    cn.cnmf_factor_batched([alone], 5, cluster_size=2)
    cn.cnmf_factor_batched([alone], 15, cluster_size=2)
    cn.cnmf_factor_batched([whole], 20, cluster_size=2)
    torch.cuda.synchronize()
    assert torch.equal(mix[2].U, alone.U) and torch.equal(mix[2].Vt, alone.Vt)
    assert torch.equal(whole.U, alone.U) and torch.equal(whole.Vt, alone.Vt)
    assert torch.equal(whole.state.buf, alone.state.buf)


def test_batched_close_to_cooperative_kernel():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    case = _case(3000, 2000, 20, 30, seed=7)
    pb = _problem(torch, cn, case)
    cn.cnmf_factor_batched([pb], 50, cluster_size=4)
    A, L, Rt, At, U0, V0 = case
    dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")
    U, Vt = dev(U0), dev(V0.T.copy())
    cn.cnmf_factor(dev(L), dev(Rt), dev(At), U, Vt, pb.lam, pb.lam, 50)
    torch.cuda.synchronize()
    assert rel(to_np(pb.U), to_np(U)) <= 1e-4
    assert rel(to_np(pb.Vt), to_np(Vt)) <= 1e-4


def test_batched_default_penalty_formed_on_device():
    """lambda <= 0 in a batch item selects lambda = phi = ||Atilde||_F / r,
    formed by the kernel: the same trajectory as passing that value."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    cases = [_case(*s, seed=300 + i) for i, s in enumerate(SHAPES)]
    explicit = [_problem(torch, cn, c) for c in cases]
    auto = [_problem(torch, cn, c) for c in cases]
    for pb in auto:
        pb.lam = pb.phi = 0.0
    _, st = cn.cnmf_factor_batched(explicit, 30, cluster_size=2)
    _, st = cn.cnmf_factor_batched(auto, 30, cluster_size=2, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    for pe, pa in zip(explicit, auto):
        assert rel(to_np(pa.U), to_np(pe.U)) <= 1e-5
        assert rel(to_np(pa.Vt), to_np(pe.Vt)) <= 1e-5
