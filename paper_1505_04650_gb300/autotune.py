"""Autotuner for the batched compressed ADMM kernel.

The tunable is the kernel's tile shape over one problem: how many CTAs (a
thread-block cluster of 1, 2, 4 or 8) share a problem's rows.  Small
problems are fastest on one CTA (no cluster barrier, no distributed
shared-memory reduction); larger ones need more SMs per problem.  For a
size bucket the tuner builds a batch of synthetic problems of that bucket,
times `cnmf_factor_batched` for every candidate cluster size with CUDA
events, and keeps the fastest in a JSON cache keyed by the bucket.

    tuner = Autotuner(cache_path)
    cs = tuner.cluster_size(m, n, r, d)       # tunes the bucket on first use
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import BatchProblem, cnmf_factor_batched, cnmf_compress

CANDIDATES = (1, 2, 4, 8)


def bucket(m: int, n: int, r: int, d: int) -> str:
    """Size bucket: rows rounded up to 1024, r to 16, d to 32."""
    up = lambda x, q: ((x + q - 1) // q) * q
    return f"m{up(m, 1024)}_n{up(n, 1024)}_r{up(r, 16)}_d{up(d, 32)}"


class Autotuner:
    def __init__(self, cache_path: str | None = None, sweeps: int = 10,
                 problems: int = 152, reps: int = 3):
        self.cache_path = cache_path
        self.sweeps, self.problems, self.reps = sweeps, problems, reps
        self.table: dict[str, dict] = {}
        self._lock = threading.Lock()
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.table = json.load(f)

    def cluster_size(self, m: int, n: int, r: int, d: int) -> int:
        key = bucket(m, n, r, d)
        with self._lock:
            if key not in self.table:
                self.table[key] = self.tune(m, n, r, d)
                self._save()
            return int(self.table[key]["cluster_size"])

    def _save(self):
        if self.cache_path:
            os.makedirs(os.path.dirname(os.path.abspath(self.cache_path)),
                        exist_ok=True)
            with open(self.cache_path, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)

    def tune(self, m: int, n: int, r: int, d: int) -> dict:
        """Time every candidate on `problems` copies of one synthetic
        problem of the bucket's upper size; returns the table entry."""
        up = lambda x, q: ((x + q - 1) // q) * q
        mm, nn = up(m, 1024), up(n, 1024)
        dev = torch.device("cuda")
        g = torch.Generator(device=dev)
        g.manual_seed(17)
        A = torch.rand(mm, r, device=dev, generator=g) @ \
            torch.rand(r, nn, device=dev, generator=g)
        A += 0.01 * torch.rand(mm, nn, device=dev, generator=g)
        L, Rt, At, st = cnmf_compress(A, r, d, 1, seed=17)
        lam = float(torch.linalg.norm(At.double())) / r
        del A
        probs = []
        for _ in range(self.problems):   # distinct buffers, as in serving
            U = torch.rand(mm, r, device=dev, generator=g)
            Vt = torch.rand(nn, r, device=dev, generator=g)
            probs.append(BatchProblem(L.clone(), Rt.clone(), At.clone(), U, Vt,
                                      lam, lam))
        times = {}
        items = None
        for cs in CANDIDATES:
            for pb in probs:
                pb.fresh = True
            items, st = cnmf_factor_batched(probs, 1, cs, items_dev=items,
                                            status=st)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            best = float("inf")
            for _ in range(self.reps):
                torch.cuda.synchronize()
                ev[0].record()
                items, st = cnmf_factor_batched(probs, self.sweeps, cs,
                                                items_dev=items, status=st)
                ev[1].record()
                torch.cuda.synchronize()
                best = min(best, ev[0].elapsed_time(ev[1]))
            times[cs] = best * 1e3 / (self.sweeps * self.problems)
        cs_best = min(times, key=times.get)
        return {"cluster_size": cs_best,
                "us_per_problem_sweep": {str(k): v for k, v in times.items()},
                "shape": [mm, nn, r, d]}
