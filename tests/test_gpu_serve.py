"""GPU tests of the serving loop (continuous batching) and the autotuner.

A request's factors are the same served alone and in a mix (bitwise, by
the batched kernel's independence); served results reach the oracle's
final objective (1e-3 relative); latency statistics are consistent.
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


def test_serving_alone_equals_mix():
    torch = need_gpu()
    from paper_1505_04650_gb300 import serve
    from paper_1505_04650_gb300.autotune import Autotuner
    tuner = Autotuner(None, sweeps=5, problems=8, reps=1)
    reqs = _workload(10)
    probe = 4
    reqs[probe].keep = True
    srv = serve.Server(max_slots=64, sweeps_per_round=10, tuner=tuner)
    srv.prepare(reqs)
    stats = srv.run(reqs, realtime=False)
    assert stats["requests"] == 10
    assert stats["p50_ms"] <= stats["p99_ms"]
    alone = copy.copy(_workload(10)[probe])
    alone.keep = True
    srv2 = serve.Server(max_slots=64, sweeps_per_round=10, tuner=tuner)
    srv2.run([alone], realtime=False)
    torch.cuda.synchronize()
    assert torch.equal(alone.U, reqs[probe].U)
    assert torch.equal(alone.Vt, reqs[probe].Vt)
    assert alone.rho == reqs[probe].rho


def test_served_objective_matches_oracle():
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
        lam = float(np.linalg.norm(At)) / rq.r
        st = oadmm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, iters=rq.iters)
        rho = ores.rel_residual(A, st.U, st.V)
        assert abs(rq.rho - rho) <= 1e-3 * rho, (rq.rid, rq.rho, rho)
