"""GPU tests of the serving loop (continuous batching) and the autotuner.

A request's factors are the same served alone and in a mix (bitwise, by
the batched kernel's independence), with a fixed sweep count and with the
accuracy-target stopping rule (the stopping decision depends only on the
request's own arithmetic); served results reach the oracle's final
objective after the same number of sweeps (1e-3 relative); with the
stopping rule every request ends at a check, at or below its target or at
the sweep cap; latency statistics are consistent.
"""
import copy

import numpy as np
import pytest

from oracle import admm as oadmm
from oracle import compress as ocomp
from oracle import philox as ophil
from oracle import residual as ores

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _workload(n=10):
    from paper_1505_04650_gb300 import serve
    return serve.make_workload(n, rate=0.0, seed=3, m_range=(200, 1200),
                               r_range=(5, 24), iters=60)


def test_autotuner_picks_a_cluster_size(tmp_path):
    need_gpu()
    from paper_1505_04650_gb300.autotune import Autotuner
    path = str(tmp_path / "tune.json")
    t = Autotuner(path, sweeps=5, problems=16, reps=1)
    cs = t.cluster_size(900, 700, 12, 22)
    assert cs in (1, 2, 4, 8)
    t2 = Autotuner(path)
    assert t2.cluster_size(900, 700, 12, 22) == cs   # from the cache


@pytest.mark.parametrize("to_target", [False, True])
def test_serving_alone_equals_mix(to_target):
    torch = need_gpu()
    from paper_1505_04650_gb300 import serve
    from paper_1505_04650_gb300.autotune import Autotuner
    tuner = Autotuner(None, sweeps=5, problems=8, reps=1)
    reqs = _workload(10)
    probe = 4
    reqs[probe].keep = True
    kw = dict(max_slots=64, sweeps_per_round=10, tuner=tuner,
              stop_at_target=to_target, check_every=20, max_sweeps=2000)
    srv = serve.Server(**kw)
    srv.prepare(reqs)
    stats = srv.run(reqs, realtime=False)
    assert stats["requests"] == 10
    assert stats["p50_ms"] <= stats["p99_ms"]
    alone = copy.copy(_workload(10)[probe])
    alone.keep = True
    srv2 = serve.Server(**kw)
    srv2.run([alone], realtime=False)
    torch.cuda.synchronize()
    assert alone.done_sweeps == reqs[probe].done_sweeps
    assert torch.equal(alone.U, reqs[probe].U)
    assert torch.equal(alone.Vt, reqs[probe].Vt)
    assert alone.rho == reqs[probe].rho


def test_served_objective_matches_oracle():
    """Fixed sweep count: the served objective is the oracle's after the
    same sweeps from the same start (1e-3 relative)."""
    torch = need_gpu()
    import synth
    from paper_1505_04650_gb300 import serve
    from paper_1505_04650_gb300.autotune import Autotuner
    tuner = Autotuner(None, sweeps=5, problems=8, reps=1)
    reqs = _workload(4)
    srv = serve.Server(max_slots=16, sweeps_per_round=10, tuner=tuner)
    srv.run(reqs, realtime=False)
    for rq in reqs[:3]:
        A = synth.lowrank_torch(rq.m, rq.n, rq.r, rq.sigma, rq.seed).double().cpu().numpy()
        U0, Vt0 = synth.init_torch(rq.m, rq.n, rq.r, rq.seed + 1)
        U0 = U0.double().cpu().numpy()
        V0 = Vt0.double().cpu().numpy().T
        Om, Ps = ophil.test_matrices(rq.seed + 2, rq.m, rq.n, rq.d)
        L, Rt, _, At = ocomp.compress(A, Om, Ps, rq.q)
        lam = srv.penalty_scale * float(np.linalg.norm(At)) / rq.r
        st = oadmm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam,
                        iters=rq.done_sweeps)
        rho = ores.rel_residual(A, st.U, st.V)
        assert abs(rq.rho - rho) <= 1e-3 * rho, (rq.rid, rq.rho, rho)


def test_served_to_target():
    """Accuracy-target stopping: every request leaves at a residual check,
    at or below its target or at the sweep cap; the reported residual is
    the FP64 residual of the returned factors (1e-5 relative), and the
    target is the rank-r floor of the request's sketch plus 1e-3, which
    the oracle's own compression of the same A reproduces (1e-3 relative
    on the floor).  After hundreds of sweeps FP32 and FP64 ADMM
    trajectories of this non-convex problem drift apart, so the factors
    themselves are compared with the oracle in the fixed-count test."""
    torch = need_gpu()
    import synth
    from paper_1505_04650_gb300 import serve
    from paper_1505_04650_gb300.autotune import Autotuner
    tuner = Autotuner(None, sweeps=5, problems=8, reps=1)
    reqs = _workload(4)
    for rq in reqs:
        rq.keep = True
    srv = serve.Server(max_slots=16, sweeps_per_round=10, tuner=tuner,
                       stop_at_target=True, check_every=20, max_sweeps=2000)
    stats = srv.run(reqs, realtime=False)
    assert stats["frac_at_target"] > 0
    for rq in reqs:
        assert rq.done_sweeps % 20 == 0
        assert rq.rho <= rq.tau or rq.done_sweeps >= 2000
        A = synth.lowrank_torch(rq.m, rq.n, rq.r, rq.sigma, rq.seed).double().cpu().numpy()
        rho = ores.rel_residual(A, rq.U.double().cpu().numpy(),
                                rq.Vt.double().cpu().numpy().T)
        assert abs(rq.rho - rho) <= 1e-5 * rho, (rq.rid, rq.rho, rho)
        Om, Ps = ophil.test_matrices(rq.seed + 2, rq.m, rq.n, rq.d)
        L, Rt, _, At = ocomp.compress(A, Om, Ps, rq.q)
        Us, s, Vh = np.linalg.svd(At)
        floor = ores.rel_residual(A, L @ (Us[:, :rq.r] * s[:rq.r]),
                                  (Rt @ Vh[:rq.r].T).T)
        assert abs(rq.floor - floor) <= 1e-3 * floor, (rq.rid, rq.floor, floor)
