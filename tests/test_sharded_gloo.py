"""The row-sharded design of one large factorization, checked on two CPU
ranks (gloo, world size 2) against the one-rank FP64 oracle.

No GPU path is built for it (every call here uses one GPU); this test
checks that the design's exchange steps reproduce the single-rank method
exactly, so that it can be built on them:

* compression (Alg. 1 on A and A^T, Sec. III): rank i holds the row block
  A_i and the rows Psi_i; A X needs no exchange, A^T Y = sum_i A_i^T Y_i is
  one all-reduce of n x d, and the Gram of a row-sharded panel (the one
  central reduction of CholeskyQR, the role TSQR plays in App. A) is one
  all-reduce of d x d; A-tilde = sum_i L_i^T (A_i R^T) one more d x d;
* SNMF (Alg. 3 steps 1-2): R-hat = sum_i Q_i^T A_i, reduce-scattered into
  column shards; each SPA step a MAXLOC over the ranks (largest squared
  norm, lowest global index on ties) and a broadcast of the chosen column;
* ADMM (Alg. 4): L, U, Lambda row-sharded, V, Phi replicated; the only
  exchange per sweep is the all-reduce of L^T (lambda U - Lambda), d x r.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

M_SPLIT = (350, 250)      # uneven row blocks


def _chol_qr(Y_local, allreduce):
    """CholeskyQR2 of a row-distributed panel: the Gram is the sum of the
    blocks' Grams; Q_i = Y_i R^-1, twice (FP64)."""
    Q = Y_local
    for _ in range(2):
        G = allreduce(Q.T @ Q)
        R = np.linalg.cholesky(G).T              # upper, positive diagonal
        Q = np.linalg.solve(R.T, Q.T).T          # Q R^-1
    return Q


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      WORLD_SIZE=str(world), RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def allreduce(x):
        t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
        dist.all_reduce(t)
        return t.numpy()

    def allgather_rows(x):
        # gloo gathers equal shapes: pad every block to the longest
        mx = max(M_SPLIT)
        mine = np.zeros((mx,) + x.shape[1:])
        mine[:x.shape[0]] = x
        parts = [torch.zeros((mx,) + x.shape[1:], dtype=torch.float64)
                 for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(mine))
        return np.concatenate([parts[j].numpy()[:M_SPLIT[j]]
                               for j in range(world)])

    import synth
    from oracle import philox
    res = {}
    r0 = sum(M_SPLIT[:rank])
    rows = slice(r0, r0 + M_SPLIT[rank])

    # ---- two-sided compression
    m, n, r, d, q = sum(M_SPLIT), 400, 5, 12, 2
    A = synth.lowrank(m, n, r, 0.01, 71)
    Om, Ps = philox.test_matrices(72, m, n, d)
    Ai, Psi_i = A[rows], Ps[rows]
    rep = lambda Y: _chol_qr(Y, lambda G: G)    # replicated n x d panel
    Li = _chol_qr(Ai @ Om, allreduce)
    S = rep(allreduce(Ai.T @ Psi_i))
    for _ in range(q):
        Z = rep(allreduce(Ai.T @ Li))
        Pi = _chol_qr(Ai @ S, allreduce)
        Li = _chol_qr(Ai @ Z, allreduce)
        S = rep(allreduce(Ai.T @ Pi))
    Rt = S
    Atilde = allreduce(Li.T @ (Ai @ Rt))
    res["L"] = allgather_rows(Li)
    res["Rt"], res["Atilde"] = Rt, Atilde

    # ---- ADMM, 20 sweeps from (U0, V0), lambda = phi = ||Atilde|| / r
    U0, V0 = synth.init_factors(m, n, r, 73)
    lam = phi = float(np.linalg.norm(Atilde)) / r
    I = np.eye(r)
    Ui, Lami = U0[rows].copy(), np.zeros((M_SPLIT[rank], r))
    V, Phi = V0.copy(), np.zeros((r, n))
    Yt = V @ Rt
    for _ in range(20):
        SX = allreduce(Li.T @ (lam * Ui - Lami))                   # d x r
        MX = Atilde @ Yt.T + SX
        Xt = np.linalg.solve(Yt @ Yt.T + lam * I, MX.T).T
        MY = Xt.T @ Atilde + phi * (V @ Rt) - Phi @ Rt
        Yt = np.linalg.solve(Xt.T @ Xt + phi * I, MY)
        T = Li @ Xt
        Sv = Yt @ Rt.T
        Un = np.maximum(T + Lami / lam, 0.0)
        Vn = np.maximum(Sv + Phi / phi, 0.0)
        Lami = Lami + lam * (T - Un)
        Phi = Phi + phi * (Sv - Vn)
        Ui, V = Un, Vn
    res["U"], res["V"] = allgather_rows(Ui), V

    # ---- SNMF column selection on a separable matrix
    ms, ns, rs, ds, qs = m, 800, 6, 10, 1
    As, _ = synth.separable(ms, ns, rs, 1e-3, 74)
    Oms = philox.gaussian_matrix(75, 0, ns, ds)
    Asi = As[rows]
    Qi = _chol_qr(Asi @ Oms, allreduce)
    for _ in range(qs):
        Z = rep(allreduce(Asi.T @ Qi))
        Qi = _chol_qr(Asi @ Z, allreduce)
    Rhat = allreduce(Qi.T @ Asi)                 # then keep own column shard
    c0, c1 = rank * ns // world, (rank + 1) * ns // world
    W = Rhat[:, c0:c1].copy()
    K = []
    for _ in range(rs):
        nrm = np.einsum("ij,ij->j", W, W)
        jl = int(np.argmax(nrm))                 # lowest local index
        cand = torch.tensor([nrm[jl], float(c0 + jl)], dtype=torch.float64)
        allc = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(allc, cand)
        best = max(allc, key=lambda t: (t[0].item(), -t[1].item()))
        j = int(best[1].item())
        col = torch.from_numpy(np.ascontiguousarray(
            W[:, j - c0] if c0 <= j < c1 else np.zeros(ds)))
        dist.all_reduce(col)                     # the owner's column
        u = col.numpy() / np.sqrt(best[0].item())
        W = W - np.outer(u, u @ W)
        K.append(j)
    res["K"] = np.array(K)

    out.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_row_sharded_design_matches_one_rank_oracle():
    import synth
    from oracle import admm as oadmm
    from oracle import compress as ocomp
    from oracle import philox
    from oracle import snmf as osnmf
    mp = torch.multiprocessing.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = mp.Queue()
    procs = [mp.Process(target=_rank, args=(k, 2, port, out)) for k in range(2)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0

    m, n, r, d, q = sum(M_SPLIT), 400, 5, 12, 2
    A = synth.lowrank(m, n, r, 0.01, 71)
    Om, Ps = philox.test_matrices(72, m, n, d)
    L, Rt, _, At = ocomp.compress(A, Om, Ps, q)
    U0, V0 = synth.init_factors(m, n, r, 73)
    lam = float(np.linalg.norm(At)) / r
    st = oadmm.admm(L, Rt, At, U0, V0, lam=lam, phi=lam, xi=1.0, iters=20)
    As, _ = synth.separable(m, 800, 6, 1e-3, 74)
    K, _, _, _ = osnmf.snmf_select(As, philox.gaussian_matrix(75, 0, 800, 10),
                                   6, 1)
    for rank in (0, 1):
        g = got[rank]
        assert np.abs(g["L"] - L).max() <= 1e-9
        assert np.abs(g["Rt"] - Rt).max() <= 1e-9
        assert np.abs(g["Atilde"] - At).max() <= 1e-9 * np.abs(At).max()
        assert np.abs(g["U"] - st.U).max() <= 1e-8 * max(1.0, np.abs(st.U).max())
        assert np.abs(g["V"] - st.V).max() <= 1e-8 * max(1.0, np.abs(st.V).max())
        assert list(g["K"]) == [int(k) for k in K]
