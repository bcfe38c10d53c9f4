"""Serving loop for compressed-NMF requests with continuous batching.

Requests (each one factorization: its own A of shape m x n, rank r, sketch
size d, q power iterations, a number of ADMM sweeps) arrive over time.  The
server

* admits waiting requests in arrival order while the device-memory budget
  (bytes of A, the compression panels, factors, state and scratch) and the
  slot count allow;
* draws each admitted request's synthetic A and compresses it
  (cnmf_compress) on one of a few side streams, from a pool of host threads
  (the host-side launch work of a compression runs while the main loop
  waits for a round), so compression of new requests overlaps the sweeps of
  running ones;
* runs the compressed ADMM sweeps of all compressed requests in rounds:
  one batched launch per cluster size (cnmf_factor_batched, replayed from a
  captured CUDA graph) advances every running request by `sweeps_per_round`
  sweeps; requests join at the next round after their compression and leave
  when they are done (iteration-level continuous batching);
* "done" is either a fixed sweep count (`iters`) or, with
  `stop_at_target`, the accuracy target: the relative residual
  rho = ||A - U V||_F / ||A||_F at or below tau = rho* + 1e-3, where rho*
  is the residual of the rank-r truncation of the request's compressed
  matrix lifted back to m x n (formed when the request joins).  rho is
  computed every `check_every` sweeps between rounds, for all requests due
  in one launch (cnmf_residual_batched) read back with one copy; a
  request that reaches `max_sweeps` first leaves too and is counted as not
  at target;
* captures each batch group's CUDA graph with the admission threads held
  back (a shared/exclusive gate), so no other thread's CUDA call lands
  inside a capture;
* on completion keeps the relative residual and frees the request's
  memory.

Each request's arithmetic is independent of the others (batched kernel
property), so its result is the same whether it is served alone or in a
mix.  Latency = completion time - arrival time (host clock).
"""
from __future__ import annotations

import collections
import concurrent.futures
import ctypes as C
import math
import contextlib
import queue
import threading
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import (BatchProblem, _lib, cnmf_compress, cnmf_residual,
               cnmf_residual_batched, lib, residual_item_bytes,
               raise_on_status)
from .autotune import Autotuner


@dataclass
class Request:
    rid: int
    t_arrive: float
    m: int
    n: int
    r: int
    d: int
    q: int = 4
    iters: int = 200
    sigma: float = 0.01
    seed: int = 0
    # filled by the server
    t_admit: float = math.nan
    t_compressed: float = math.nan
    t_done: float = math.nan
    cluster_size: int = 1
    rho: float = math.nan
    floor: float = math.nan
    tau: float = math.nan        # accuracy target (stop_at_target)
    At_host: torch.Tensor | None = None    # A-tilde copied to pinned memory
    floor_res: torch.Tensor | None = None  # residual of the truncation
    nbytes: int = 0
    done_sweeps: int = 0
    problem: BatchProblem | None = None
    A: torch.Tensor | None = None
    event: torch.cuda.Event | None = None
    stream_idx: int = 0
    keep: bool = False          # keep U, Vt after completion
    fut: concurrent.futures.Future | None = None
    U: torch.Tensor | None = None
    Vt: torch.Tensor | None = None
    res_item: bytes = b""       # cnmf_residual_item record of the checks


def make_workload(nreq: int, rate: float, seed: int = 0, m_range=(200, 4000),
                  r_range=(5, 32), q: int = 4, iters: int = 200,
                  sigma: float = 0.01) -> list[Request]:
    """Poisson arrivals at `rate` requests/s (rate <= 0: all at t = 0);
    m, n ~ U[m_range], r ~ U{r_range}, d = r + 10."""
    g = np.random.Generator(np.random.PCG64(seed))
    gaps = g.exponential(1.0 / rate, nreq) if rate > 0 else np.zeros(nreq)
    t = np.cumsum(gaps) - (gaps[0] if rate > 0 else 0.0)
    reqs = []
    for i in range(nreq):
        m = int(g.integers(m_range[0], m_range[1] + 1))
        n = int(g.integers(m_range[0], m_range[1] + 1))
        r = int(g.integers(r_range[0], r_range[1] + 1))
        reqs.append(Request(i, float(t[i]), m, n, r, r + 10, q, iters, sigma,
                            seed=10_000 * (seed + 1) + i))
    return reqs


def truncation_factors(L: torch.Tensor, Rt: torch.Tensor, Atilde: torch.Tensor,
                       r: int):
    """(F, G) with F G^T = L Atilde_r R, Atilde_r the rank-r SVD truncation
    of the compressed matrix: m x r and n x r FP32 factors.  The residual
    ||A - F G^T|| is the best rank-r fit the sketch can express -- computed
    as a residual, not as ||A||^2 - sum sigma_i^2, which cancels
    catastrophically when the floor is small.  Atilde may be a host copy."""
    U, s, Vh = torch.linalg.svd(Atilde.double().cpu())
    Us = (U[:, :r] * s[:r]).to(L.device)
    V = Vh[:r].T.contiguous().to(L.device)
    F = (L.double() @ Us).float()
    G = (Rt.double() @ V).float()
    return F, G


def request_bytes(rq: Request) -> int:
    e = 4
    m, n, r, d = rq.m, rq.n, rq.r, rq.d
    b = m * n * e                                  # A
    b += (m + n) * d * e + d * d * e               # L, Rt, Atilde
    b += (m + n) * r * e * 2                       # U, Vt, Lam, Phit
    b += 2 * r * d * e * 2 + 256 * 4               # state tail, scratch
    return b


class _CaptureGate:
    """Admission threads issue CUDA work together (shared); a CUDA-graph
    capture on the serving thread runs alone (exclusive), so no other
    thread's call (an allocation, a synchronising query, the autotuner's
    timing) lands inside a capture and invalidates it.  A waiting capture
    holds back new admissions; admissions never wait on the serving
    thread, so the capture always gets its turn."""

    def __init__(self):
        self._c = threading.Condition()
        self._shared = 0
        self._excl = False
        self._waiting = 0

    @contextlib.contextmanager
    def shared(self):
        with self._c:
            while self._excl or self._waiting:
                self._c.wait()
            self._shared += 1
        try:
            yield
        finally:
            with self._c:
                self._shared -= 1
                self._c.notify_all()

    @contextlib.contextmanager
    def exclusive(self):
        with self._c:
            self._waiting += 1
            while self._excl or self._shared:
                self._c.wait()
            self._waiting -= 1
            self._excl = True
        try:
            yield
        finally:
            with self._c:
                self._excl = False
                self._c.notify_all()


class Server:
    def __init__(self, hbm_budget: float = 40e9, max_slots: int = 512,
                 sweeps_per_round: int = 20, compress_streams: int = 4,
                 tuner: Autotuner | None = None, use_graphs: bool = True,
                 stop_at_target: bool = False, check_every: int = 20,
                 max_sweeps: int = 3000, penalty_scale: float = 0.3,
                 device="cuda"):
        self.dev = torch.device(device)
        self.stop_at_target = stop_at_target
        # residual checks fall on round boundaries
        self.check_every = max(sweeps_per_round,
                               check_every // sweeps_per_round * sweeps_per_round)
        self.max_sweeps = max_sweeps
        # lambda = phi = penalty_scale ||Atilde||_F / r, formed by the
        # batched kernel from each request's A-tilde.  Alg. 4 leaves the
        # penalties open; on this request mix 0.3 reached the accuracy
        # target in every sampled request (1.0 stalled above it in several)
        self.penalty_scale = penalty_scale
        self.budget = int(hbm_budget)
        self.max_slots = max_slots
        self.S = sweeps_per_round
        self.tuner = tuner or Autotuner()
        self.use_graphs = use_graphs
        self.main = torch.cuda.current_stream(self.dev)
        self.side = [torch.cuda.Stream(self.dev) for _ in range(compress_streams)]
        self.status = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self.comp_ws = [None] * compress_streams
        # admission threads, one side stream (and workspace) each at a time
        self.pool = concurrent.futures.ThreadPoolExecutor(compress_streams)
        self.free = queue.Queue()
        for i in range(compress_streams):
            self.free.put(i)
        # the synthetic A is drawn with FP32 products; with several admission
        # threads that setting must not be toggled per call
        torch.backends.cuda.matmul.allow_tf32 = False
        self.groups: dict[int, dict] = {}
        self.lib = lib()
        self.gate = _CaptureGate()

    # ---- batched launches (one per cluster size), optionally graphed ----
    def _group(self, key) -> dict:
        if key not in self.groups:
            nbytes = C.sizeof(_lib.BatchItem) * self.max_slots
            self.groups[key] = {
                "items": torch.zeros(nbytes, dtype=torch.uint8, device=self.dev),
                "host": torch.zeros(nbytes, dtype=torch.uint8).pin_memory(),
                "graph": None,
            }
        return self.groups[key]

    def _launch(self, key, g: dict):
        cs, dm = key
        rc = self.lib.cnmf_factor_batched(
            C.c_void_p(g["items"].data_ptr()), self.max_slots, self.S, cs, 32,
            dm, C.c_void_p(self.status.data_ptr()),
            C.c_void_p(torch.cuda.current_stream(self.dev).cuda_stream))
        if rc != 0:
            raise RuntimeError(f"cnmf_factor_batched: status {rc}: "
                               f"{self.lib.cnmf_last_error().decode()}")

    def _round(self, key, reqs: list[Request]):
        g = self._group(key)
        # the device item array changes only when the group's members or a
        # member's FRESH flag change; then it is rebuilt from each problem's
        # cached host image (empty slots zero) and copied, once the previous
        # copy out of the pinned staging buffer has finished
        sig = [(id(rq), rq.problem.fresh) for rq in reqs]
        if g.get("sig") != sig:
            blob = b"".join(rq.problem.item_bytes() for rq in reqs)
            if g.get("copy_ev") is not None:
                g["copy_ev"].synchronize()
            host = g["host"].numpy()
            host[:len(blob)] = np.frombuffer(blob, dtype=np.uint8)
            host[len(blob):] = 0
            g["items"].copy_(g["host"], non_blocking=True)
            g["copy_ev"] = torch.cuda.Event()
            g["copy_ev"].record(torch.cuda.current_stream(self.dev))
            g["sig"] = sig
        if not self.use_graphs:
            self._launch(key, g)
        else:
            if g["graph"] is None:
                # no admission thread issues CUDA work during the capture
                with self.gate.exclusive():
                    # warm the kernel variant outside capture, on empty slots
                    scratch = torch.zeros_like(g["items"])
                    save = g["items"]
                    g["items"] = scratch
                    self._launch(key, g)
                    g["items"] = save
                    torch.cuda.synchronize(self.dev)
                    graph = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(graph,
                                          stream=torch.cuda.Stream(self.dev),
                                          capture_error_mode="thread_local"):
                        self._launch(key, g)
                g["graph"] = graph
                # the captured launch reads the item array when replayed
                g["items"].copy_(g["host"], non_blocking=True)
            g["graph"].replay()
        for rq in reqs:
            rq.problem.fresh = False
            rq.done_sweeps += self.S

    def _res_buf(self, n: int) -> torch.Tensor:
        """Device FP64 pairs for `n` residual checks, grown as needed."""
        if getattr(self, "_res", None) is None or self._res.shape[0] < n:
            self._res = torch.empty(max(n, 64), 2, dtype=torch.float64,
                                    device=self.dev)
        return self._res

    def _check_batch(self, due: list[Request], res_all: torch.Tensor):
        """The residuals of every request due for a check in one launch
        (cnmf_residual_batched) on the main stream, into res_all[:len(due)].
        The item records are staged in pinned memory (the previous check
        round ended with a synchronisation, so the staging buffer is free)
        and copied with the launch."""
        blob = b"".join(rq.res_item for rq in due)
        nb = len(blob)
        if getattr(self, "_ri_host", None) is None or \
                self._ri_host.numel() < nb:
            cap = max(nb, 64 * C.sizeof(_lib.ResidualItem)) * 2
            self._ri_host = torch.empty(cap, dtype=torch.uint8).pin_memory()
            self._ri_dev = torch.empty(cap, dtype=torch.uint8,
                                       device=self.dev)
        self._ri_host.numpy()[:nb] = np.frombuffer(blob, dtype=np.uint8)
        self._ri_dev[:nb].copy_(self._ri_host[:nb], non_blocking=True)
        ctas = 8
        wsb = self.lib.cnmf_residual_batched_workspace(len(due), ctas)
        if getattr(self, "_rbws", None) is None or self._rbws.numel() < wsb:
            self._rbws = torch.empty(2 * wsb, dtype=torch.uint8,
                                     device=self.dev)
        cnmf_residual_batched(self._ri_dev, len(due), torch.float32,
                              max(rq.r for rq in due), ctas,
                              out=res_all[:len(due)], ws=self._rbws,
                              status=self.status)

    def prepare(self, requests: list[Request]):
        """Tune every size bucket the requests touch before serving."""
        for rq in requests:
            self.tuner.cluster_size(rq.m, rq.n, rq.r, rq.d)

    # ---- request lifecycle ----
    def _admit(self, rq: Request):
        """Runs on an admission thread: draw A and the initial factors and
        compress, all on a free side stream, outside any graph capture of
        the serving thread (the gate's shared side)."""
        import synth
        slot = self.free.get()
        try:
            with self.gate.shared():
                rq.stream_idx = slot
                s = self.side[slot]
                with torch.cuda.stream(s):
                    rq.A = synth.lowrank_torch(rq.m, rq.n, rq.r, rq.sigma,
                                               rq.seed, device=self.dev)
                    U0, Vt0 = synth.init_torch(rq.m, rq.n, rq.r, rq.seed + 1,
                                               device=self.dev)
                    nb = self.lib.cnmf_compress_workspace(rq.m, rq.n, rq.d, 1)
                    ws = self.comp_ws[slot]
                    if ws is None or ws.numel() < nb:
                        ws = torch.empty(int(nb * 1.25) + 256,
                                         dtype=torch.uint8, device=self.dev)
                        self.comp_ws[slot] = ws
                    L, Rt, At, _ = cnmf_compress(rq.A, rq.r, rq.d, rq.q,
                                                 rq.seed + 2,
                                                 status=self.status, ws=ws)
                    rq.problem = BatchProblem(L, Rt, At, U0, Vt0, 1.0, 1.0)
                    if self.stop_at_target:
                        # A-tilde to the host for the target (asynchronous)
                        rq.At_host = torch.empty(At.shape, dtype=At.dtype,
                                                 pin_memory=True)
                        rq.At_host.copy_(At, non_blocking=True)
                    rq.event = torch.cuda.Event()
                    rq.event.record(s)
        finally:
            self.free.put(slot)
        # the autotuner may time kernels on the device for a new size bucket
        with self.gate.shared():
            rq.cluster_size = self.tuner.cluster_size(rq.m, rq.n, rq.r, rq.d)

    def _ready(self, rq: Request, now: float):
        # penalty: lambda = phi = penalty_scale ||Atilde||_F / r, formed by
        # the batched kernel itself (a negative lambda is that scale), so
        # nothing waits for the device here
        pb = rq.problem
        pb.lam = pb.phi = -self.penalty_scale
        for t in (pb.L, pb.Rt, pb.Atilde, pb.U, pb.Vt, pb.state.buf,
                  pb.scratch, rq.A):
            t.record_stream(self.main)
        rq.t_compressed = now
        # the record of this request's residual checks (its buffers stay in
        # place until it is done)
        rq.res_item = residual_item_bytes(rq.A, pb.U, pb.Vt)
        if self.stop_at_target:
            # the target's reference point, the residual of the rank-r
            # truncation of A-tilde (host SVD of the d x d copy), queued on
            # the main stream and read after the next round
            rq.floor_res = cnmf_residual(
                rq.A, *truncation_factors(pb.L, pb.Rt, rq.At_host, rq.r))

    def _finish(self, rq: Request, res: torch.Tensor,
                res_floor: torch.Tensor | None):
        e2, a2 = float(res[0]), float(res[1])
        rq.rho = math.sqrt(e2 / a2)
        if res_floor is not None:
            rq.floor = math.sqrt(float(res_floor[0]) / a2)
        if rq.keep:
            rq.U = rq.problem.U.clone()
            rq.Vt = rq.problem.Vt.clone()
        rq.problem = None
        rq.A = None

    def run(self, requests: list[Request], realtime: bool = True) -> dict:
        pending = collections.deque(sorted(requests, key=lambda q: q.t_arrive))
        waiting: collections.deque = collections.deque()
        compressing: list[Request] = []
        running: list[Request] = []
        done: list[Request] = []
        in_use = 0
        rounds = 0
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0
        total = len(requests)
        while len(done) < total:
            now = clock()
            while pending and (pending[0].t_arrive <= now or not realtime):
                waiting.append(pending.popleft())
            # admission by memory budget and slots
            while waiting:
                rq = waiting[0]
                need = request_bytes(rq)
                slots = len(compressing) + len(running)
                if slots >= self.max_slots or (in_use + need > self.budget
                                               and slots > 0):
                    break
                waiting.popleft()
                rq.nbytes = need
                in_use += need
                rq.t_admit = clock()
                rq.fut = self.pool.submit(self._admit, rq)
                compressing.append(rq)
            # compressed requests join the batch at this round
            still = []
            for rq in compressing:
                if rq.fut.done() and rq.fut.result() is None and \
                        rq.event.query():
                    self._ready(rq, clock())
                    running.append(rq)
                else:
                    still.append(rq)
            compressing = still
            if running:
                groups: dict = collections.defaultdict(list)
                for rq in running:
                    groups[(rq.cluster_size, 32 if rq.d <= 32 else 64)].append(rq)
                for key, reqs in groups.items():
                    for i in range(0, len(reqs), self.max_slots):
                        self._round(key, reqs[i:i + self.max_slots])
                rounds += 1
                if self.stop_at_target:
                    # residual of the requests due for a check, all into
                    # one device buffer and read back with one copy; a
                    # round with nothing due (and no target pending) goes
                    # on without waiting for the device
                    due = [rq for rq in running
                           if rq.done_sweeps % self.check_every == 0
                           or rq.done_sweeps >= self.max_sweeps]
                    newf = [rq for rq in running if rq.floor_res is not None]
                    if not due and not newf:
                        continue
                    res_all = self._res_buf(len(due))
                    if due:
                        self._check_batch(due, res_all)
                    self.main.synchronize()   # this round's checks
                    now = clock()
                    for rq in newf:
                        e2, a2 = rq.floor_res.cpu().tolist()
                        rq.floor = math.sqrt(e2 / a2)
                        rq.tau = rq.floor + 1e-3
                        rq.floor_res = None
                    vals = res_all[:len(due)].cpu()
                    finished = []
                    for rq, res in zip(due, vals):
                        e2, a2 = res.tolist()
                        if math.sqrt(e2 / a2) <= rq.tau or \
                                rq.done_sweeps >= self.max_sweeps:
                            rq.t_done = now
                            self._finish(rq, res, None)
                            finished.append(rq)
                    gone = set(id(rq) for rq in finished)
                    running = [rq for rq in running if id(rq) not in gone]
                    for rq in finished:
                        in_use -= rq.nbytes
                        done.append(rq)
                    continue
                finished = [rq for rq in running if rq.done_sweeps >= rq.iters]
                running = [rq for rq in running if rq.done_sweeps < rq.iters]
                outs = []
                for rq in finished:
                    outs.append(cnmf_residual(rq.A, rq.problem.U, rq.problem.Vt))
                self.main.synchronize()   # this round only; compressions go on
                now = clock()
                for rq in finished:
                    rq.t_done = now
                # the residual target's reference point (rank-r truncation
                # of the compressed matrix, lifted back): reporting only,
                # after the requests are done
                floors = [cnmf_residual(rq.A, *truncation_factors(
                    rq.problem.L, rq.problem.Rt, rq.problem.Atilde, rq.r))
                    for rq in finished]
                for rq, res, resf in zip(finished, outs, floors):
                    self._finish(rq, res.cpu(), resf.cpu())
                    in_use -= rq.nbytes
                    done.append(rq)
            elif compressing:
                compressing[0].fut.result()
                compressing[0].event.synchronize()
            elif pending and realtime:
                time.sleep(max(0.0, min(0.001, pending[0].t_arrive - clock())))
        raise_on_status(self.status, "serving")
        wall = clock()
        lat = np.array([rq.t_done - rq.t_arrive for rq in done]) * 1e3
        ok = np.array([rq.rho <= rq.floor + 1e-3 for rq in done])
        sweeps = np.array([rq.done_sweeps for rq in done])
        out = {
            "requests": total, "wall_s": wall,
            "factorizations_per_s": total / wall,
            "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()),
            "frac_at_target": float(ok.mean()),
            "sweeps_mean": float(sweeps.mean()),
            "sweeps_p99": float(np.percentile(sweeps, 99)),
            "stop": ("rho <= rho* + 1e-3, checked every "
                     f"{self.check_every} sweeps, cap {self.max_sweeps}"
                     if self.stop_at_target else "fixed sweep count"),
            "penalty": f"lambda = phi = {self.penalty_scale} ||Atilde||_F / r",
            "rounds": rounds, "sweeps_per_round": self.S,
            "cluster_sizes": {str(c): int(sum(rq.cluster_size == c for rq in done))
                              for c in (1, 2, 4, 8)},
        }
        if ok.any():
            out["p50_at_target_ms"] = float(np.percentile(lat[ok], 50))
            out["p99_at_target_ms"] = float(np.percentile(lat[ok], 99))
        return out
