"""Benchmark: compressed NMF on one GB300 (and N-GPU replicas).

Workload (one "step"): the large compressed-NMF configuration -- A = X0 Y0 +
|N(0, 0.01^2)|, m = 20000, n = 10000, r = 20, FP32 storage; two-sided
compression with d = 30, q = 4 (Alg. 1 on A and A^T, 2q + 2 = 10 reads of
A), then 500 compressed ADMM sweeps (Alg. 4).  Inputs are synthetic and
seeded, resident in HBM when the timed region starts; A (800 MB) is larger
than L2, so no flush is needed between steps.

The JSON line reports factorizations/s (value), the end-to-end figure
through the public API with host buffers (e2e), time to the residual
target against the uncompressed ADMM on the same GPU, the sketch kernel's
roofline, the FP64 oracle timed on the host cores (cpu_baseline), sampled
SM clocks, and the number of library kernel launches.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

CFG = dict(m=20000, n=10000, r=20, d=30, q=4, iters=500, sigma=0.01)
WORKLOAD = "cnmf_m20000_n10000_r20_d30_q4_admm500_fp32"
METRIC = ("cNMF time-to-rel-residual 1e-3 vs plain NMF; sketch HBM GB/s vs "
          "peak; served p99")
SEEDS = dict(data=1001, sketch=2001, init=3001)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm=d.get("hbm_gbs", 6800.0), src="measured",
                    sm_max_mhz=d.get("sm_max_mhz", 2070.0))
    return dict(hbm=6800.0, src="fallback", sm_max_mhz=2070.0)


def _inputs():
    A = synth.lowrank(CFG["m"], CFG["n"], CFG["r"], CFG["sigma"], SEEDS["data"],
                      dtype=np.float32)
    U0, V0 = synth.init_factors(CFG["m"], CFG["n"], CFG["r"], SEEDS["init"])
    return A, U0.astype(np.float32), np.ascontiguousarray(V0.T).astype(np.float32)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,"
         "clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)   # sampling is running when the timed region starts
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 8:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(f[1]) for f in rows if f[1].replace(".", "").isdigit()]
        mx = [float(f[2]) for f in rows if f[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({names[i] for f in rows for i in range(4)
                          if f[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_oracle_sample(iters_sample=40):
    """The FP64 oracle on the full workload: compression + `iters_sample`
    ADMM sweeps, timed, and scaled to one factorization (compression + 500
    sweeps).  Returns (factorizations/s, seconds, description)."""
    from oracle import admm, compress, philox
    A, U0, Vt0 = _inputs()
    A64 = A.astype(np.float64)
    m, n, r, d, q = CFG["m"], CFG["n"], CFG["r"], CFG["d"], CFG["q"]
    Om, Ps = philox.test_matrices(SEEDS["sketch"], m, n, d)
    t0 = time.perf_counter()
    L, Rt, _, At = compress.compress(A64, Om, Ps, q)
    t1 = time.perf_counter()
    lam = float(np.linalg.norm(At)) / r
    admm.admm(L, Rt, At, U0.astype(np.float64), Vt0.T.astype(np.float64),
              lam=lam, phi=lam, iters=iters_sample)
    t2 = time.perf_counter()
    per_fact = (t1 - t0) + (t2 - t1) * CFG["iters"] / iters_sample
    desc = (f"full workload compression ({t1 - t0:.2f} s) + {iters_sample} of "
            f"{CFG['iters']} ADMM sweeps ({t2 - t1:.2f} s), scaled to one "
            f"factorization")
    return 1.0 / per_fact, (t2 - t0), desc


def cpu_oracle_one_core(iters_sample=10):
    """cpu_oracle_sample in a child process whose BLAS runs one thread
    (the oracle on one host core); (factorizations/s, description)."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1",
               MKL_NUM_THREADS="1", GOTO_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__),
                        "--cpu-sample-only", str(iters_sample)],
                       env=env, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        return None, "failed: " + r.stderr.strip().splitlines()[-1][:200]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["value"], d["sample"]


def cpu_oracle_snmf_wide():
    """The FP64 oracle's compressed SNMF (Alg. 3 steps 1-2: one-sided sketch
    with q = 2, R-hat = Q^T A, SPA) on the wide separable workload
    (10000 x 100000, r = 50, d = 60), end to end on the host cores; the
    matrix is drawn beforehand (not timed).  Returns (seconds, anchors
    recovered)."""
    from oracle import philox, snmf
    m, n, r, d, q = 10000, 100000, 50, 60, 2
    A, planted = synth.separable(m, n, r, 1e-3, 1002)
    Om = philox.gaussian_matrix(2002, 0, n, d)
    t0 = time.perf_counter()
    K, _, _, _ = snmf.snmf_select(A, Om, r, q)
    secs = time.perf_counter() - t0
    return secs, sorted(int(k) for k in K) == sorted(int(k) for k in planted)


def admm_latency_model(breakdown: dict, pipelined_ms: float,
                       iters: int) -> dict:
    """The ADMM sweep against its latency model: the lead V-side CTA's
    critical path, phase by phase (staging of the reduced shares, the X
    Grams, the X solve, the Y Grams, the Y solve, publishing Yt, its row
    sweep, the reduction of its shares), measured with %globaltimer on all
    SMs, beside the measured time of a sweep alone and in the pipelined
    steps."""
    ph = breakdown.get("factor_phase_us_per_sweep", {})
    path = ["s_stage", "s_grams_x", "s_solve_x", "s_grams_y", "s_solve_y",
            "s_publish", "w_vrows", "w_vred"]
    comp = {k: ph[k] for k in path if k in ph}
    model = sum(comp.values())
    alone = breakdown.get("factor_us_per_sweep")
    return {"unit": "us per sweep",
            "lead_cta_path": comp, "model_us": model,
            "measured_us_all_sms": alone,
            "measured_us_pipelined": 1e3 * pipelined_ms / iters,
            "unexplained_us_all_sms": (alone - model) if alone else None,
            "note": "the remainder is waiting for the other side's shares"}


def bench_config(world: int) -> dict:
    """The workload both arms measure (the same dict in both JSON lines;
    run-specific settings such as the penalty go under "run")."""
    return {"workload": WORKLOAD, "m": CFG["m"], "n": CFG["n"], "r": CFG["r"],
            "d": CFG["d"], "q": CFG["q"], "admm_iters": CFG["iters"],
            "l2": "inputs larger than L2 (A = 800 MB)",
            "parallelism": f"replicas{world}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; a timed step is one sample
    t0 = time.perf_counter()
    vals = []
    desc = ""
    for _ in range(args.steps):
        v, _, desc = cpu_oracle_sample(iters_sample=20)
        vals.append(v)
    dt = time.perf_counter() - t0
    value = float(np.mean(vals))
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "factorizations/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": bench_config(int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": "factorizations/s",
                         "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "factorizations/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": dt,
    }
    print(json.dumps(line), flush=True)
    return 0


def launches_per_step(q):
    """Library kernel launches of one step (compress + one factor launch),
    for FP32 A with d <= 32 (the fused pass): two Gaussian panels; per pass
    the panel pack, the fused two-sided kernel and the partial-slot sum;
    between passes one CholeskyQR sweep of both panels (gram, finish,
    apply), CholeskyQR2 (gram, finish, apply, finish, apply) after the last
    pass; A-check (pack, fused one-sided, sum) and the cross product
    (gram, finish)."""
    passes = 2 * q + 1
    compress = 2 + passes * 3 + (passes - 1) * 3 + 5 + 3 + 2
    return compress + 1


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum)
# from one ncu capture of the kernel as it stands, with the SHA-256 of the
# sources it was compiled from; None once those sources change.
TRAFFIC = {
    # profiles/k_admm_fast_m20000_n10000_r20_d30.md: 8.573 MB read +
    # 0.034 MB written by the 500-sweep launch (104 CTAs, as in the
    # pipelined steps)
    "k_admm_fast": {"bytes_per_unit": 8.606976e6 / 500, "sha": "4f3983b76c9d29d1"},
    # profiles/k_tc_prod_f32_m20000_n10000_d30.md: A X 805.23 + 2.25 MB,
    # A^T Y 868.03 + 4.13 MB; one unit = one pass (both products)
    "k_tc_prod": {"bytes_per_unit": 1679.634432e6, "sha": "d74ba8dadf2e3d3d"},
    # profiles/k_fused_pass_f32_m20000_n10000_d30.md: 812.32 MB read +
    # 6.51 MB written by one two-sided pass (152 CTAs)
    "k_fused_pass": {"bytes_per_unit": 818.831104e6, "sha": "1c8dd4068a2d9931"},
}


def _src_sha(kernel):
    import hashlib
    files = {"k_admm_fast": ["admm_fast.cuh", "admm_impl.cuh", "common.cuh"],
             "k_tc_prod": ["tc.cu", "common.cuh"],
             "k_fused_pass": ["fused.cu", "tc_ptx.cuh", "common.cuh"]}[kernel]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1505_04650_gb300", "csrc", f),
                  "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel, units):
    t = TRAFFIC.get(kernel)
    if not t or t["sha"] != _src_sha(kernel):
        return None
    return t["bytes_per_unit"] * units


# ADMM launches in flight at once in the pipelined steps, and the SMs of
# each (the compression stream gets the rest); see admm_split
ADMM_STREAMS = 1


def admm_split(nsm: int, nfs: int, admm_ctas: int = 0):
    """(SMs per ADMM stream, SMs of the compression stream) for `nfs` ADMM
    launches in flight beside one compression stream.  Measured on the
    bench workload (factorizations/s): one ADMM stream on 76 / 92 / 104 /
    116 SMs gives 111 / 115 / 122 / 113 -- past ~100 SMs the ADMM gains
    nothing and the compression beside it loses; two streams of 48 / 54 /
    60 SMs give 92 / 99 / 98 and three of 36 / 40 give 99 / 94, because
    below ~70 CTAs the rows no longer stay in shared memory and a sweep
    takes ~40 us.  Default: one stream on 104 of 152 SMs."""
    if admm_ctas > 0:
        cap = admm_ctas
    elif nfs == 1:
        cap = nsm * 104 // 152
    else:
        cap = (nsm - nsm // 3) // nfs
    cap_c = nsm - nfs * cap
    if cap < 1 or cap_c < 8:
        raise ValueError(f"{nfs} ADMM streams of {cap} SMs leave {cap_c} "
                         f"of {nsm} SMs for the compression")
    return cap, cap_c


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttt", action="store_true",
                    help="skip the time-to-target measurement")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the served-stream measurement")
    ap.add_argument("--serving-requests", type=int, default=4096)
    ap.add_argument("--admm-ctas", type=int, default=0,
                    help="SMs for each ADMM stream of the pipelined steps "
                         "(the compression stream gets the rest; 0: the "
                         "default split)")
    ap.add_argument("--admm-streams", type=int, default=ADMM_STREAMS,
                    help="ADMM launches in flight at once in the pipelined "
                         "steps (one stream each)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the wide-SNMF and mixed-precision lines")
    ap.add_argument("--cpu-sample-only", type=int, default=0,
                    help=argparse.SUPPRESS)
    args = ap.parse_args(argv)
    if args.cpu_sample_only:
        v, secs, desc = cpu_oracle_sample(iters_sample=args.cpu_sample_only)
        print(json.dumps({"value": v, "seconds": secs, "sample": desc}))
        return 0
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1505_04650_gb300 as cn
    from paper_1505_04650_gb300 import build as cbuild

    from paper_1505_04650_gb300 import replicas
    world, rank, local = replicas.world()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        cbuild.build()
    if world > 1:
        dist.barrier()

    m, n, r, d, q, iters = (CFG[k] for k in ("m", "n", "r", "d", "q", "iters"))
    A_h, U0_h, Vt0_h = _inputs()
    A = torch.from_numpy(A_h).to(dev)
    U0 = torch.from_numpy(U0_h).to(dev)
    Vt0 = torch.from_numpy(Vt0_h).to(dev)
    stream = torch.cuda.current_stream(dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    lib = cn.lib()
    ws_c = torch.empty(lib.cnmf_compress_workspace(m, n, d, 1), dtype=torch.uint8,
                       device=dev)
    ws_f = torch.empty(lib.cnmf_factor_workspace(m, n, r, d, 1), dtype=torch.uint8,
                       device=dev)
    U = U0.clone()
    Vt = Vt0.clone()

    # penalty: lambda = phi = ||Atilde||_F / r, fixed once from a first
    # compression (host-side scalar, outside the timed region)
    L, Rt, At, _ = cn.cnmf_compress(A, r, d, q, SEEDS["sketch"], status=st,
                                    ws=ws_c)
    lam = cn.default_penalty(At, r)

    # ---- the timed steps.  One step = one factorization (compression + 500
    # ADMM sweeps).  Consecutive steps are independent problems, so they are
    # pipelined on two streams: the compression of step k + 1 runs beside
    # the ADMM sweeps of step k, each call's grids capped at its share of
    # the SMs (cnmf_set_thread_cta_limit; --admm-ctas, --admm-streams;
    # default: the ADMM on 104 of 152 SMs, see admm_split).  The ADMM is
    # latency-bound (every CTA repeats the small algebra), so fewer SMs slow
    # it far less than they speed up the compression running beside it.
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    nfs = max(1, args.admm_streams)
    cap, cap_c = admm_split(nsm, nfs, args.admm_ctas)
    sF = stream                          # ADMM sweeps
    sC = torch.cuda.Stream(dev)          # compressions
    sFs = [sF] + [torch.cuda.Stream(dev) for _ in range(nfs - 1)]
    Us = [U0.clone() for _ in range(nfs)]
    Vts = [Vt0.clone() for _ in range(nfs)]
    ws_fs = [ws_f] + [torch.empty_like(ws_f) for _ in range(nfs - 1)]
    U, Vt = Us[0], Vts[0]

    def pipe_step(i, fa=None):
        j = i % nfs
        sf = sFs[j]
        cn.set_thread_cta_limit(cap_c)
        with torch.cuda.stream(sC):
            L, Rt, At, _ = cn.cnmf_compress(A, r, d, q, SEEDS["sketch"],
                                            status=st, ws=ws_c)
            ev = torch.cuda.Event()
            ev.record(sC)
        sf.wait_event(ev)
        for t in (L, Rt, At):
            t.record_stream(sf)
        with torch.cuda.stream(sf):
            Us[j].copy_(U0)
            Vts[j].copy_(Vt0)
            cn.set_thread_cta_limit(cap)
            if fa is not None:
                fa[0].record(sf)
            cn.cnmf_factor(L, Rt, At, Us[j], Vts[j], lam, lam, iters,
                           status=st, ws=ws_fs[j])
            if fa is not None:
                fa[1].record(sf)

    def join_all():
        for o in sFs[1:]:
            sF.wait_stream(o)
        sF.wait_stream(sC)

    for i in range(max(args.warmup, 3)):
        pipe_step(i)
    torch.cuda.synchronize()
    cn.raise_on_status(st, "bench warm-up")

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fas = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with Clocks(local) as clk:
        ev0.record(sC)
        for o in sFs:
            o.wait_event(ev0)
        for k in range(args.steps):
            pipe_step(k, fas[k])
        join_all()
        ev1.record(sF)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = replicas.slowest_ms(ev0.elapsed_time(ev1) / args.steps, dev)
    cn.raise_on_status(st, "bench timed region")
    value = replicas.job_rate(1, ms, world)
    # the dominant kernel's launches inside the timed region (CUDA events on
    # the stream it runs on)
    admm_ms_live = sum(f0.elapsed_time(f1) for f0, f1 in fas) / args.steps
    cn.set_thread_cta_limit(0)

    # the same steps one after the other on one stream, every SM per call
    def seq_step():
        L, Rt, At, _ = cn.cnmf_compress(A, r, d, q, SEEDS["sketch"], status=st,
                                        ws=ws_c)
        U.copy_(U0)
        Vt.copy_(Vt0)
        cn.cnmf_factor(L, Rt, At, U, Vt, lam, lam, iters, status=st, ws=ws_f)
    for _ in range(2):
        seq_step()
    torch.cuda.synchronize()
    es0, es1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    es0.record(stream)
    nseq = max(3, min(args.steps, 10))
    for _ in range(nseq):
        seq_step()
    es1.record(stream)
    torch.cuda.synchronize()
    seq_ms = es0.elapsed_time(es1) / nseq
    cn.raise_on_status(st, "bench sequential steps")

    # ---- phase breakdown (CUDA events, same stream)
    eb = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    eb[0].record(stream)
    L, Rt, At, _ = cn.cnmf_compress(A, r, d, q, SEEDS["sketch"], status=st,
                                    ws=ws_c)
    eb[1].record(stream)
    U.copy_(U0)
    Vt.copy_(Vt0)
    cn.cnmf_factor(L, Rt, At, U, Vt, lam, lam, iters, status=st, ws=ws_f)
    eb[2].record(stream)
    torch.cuda.synchronize()
    breakdown = {"compress_ms": eb[0].elapsed_time(eb[1]),
                 "factor_ms": eb[1].elapsed_time(eb[2]),
                 "factor_us_per_sweep": 1e3 * eb[1].elapsed_time(eb[2]) / iters}
    ph = torch.zeros(20, dtype=torch.float64, device=dev)
    U.copy_(U0)
    Vt.copy_(Vt0)
    cn.cnmf_factor(L, Rt, At, U, Vt, lam, lam, iters, status=st, ws=ws_f,
                   phase_ns=ph)
    torch.cuda.synchronize()
    # slots 3, 4 and 18, 19 (the generic kernel's second and third barrier
    # phases) stay zero on the register-tiled kernel, whose sweep loop has
    # no grid barrier: its slot 2 is the reduction with its waits for the
    # other CTAs' shares
    names = ["small_algebra", "row_sweep", "reduce_incl_waits", None, None,
             "s_stage", "s_grams_x", "s_solve_x", "s_grams_y", "s_solve_y",
             "s_publish", "w_urows", "w_ured", "w_vrows", "w_vred",
             "u_small_algebra", "u_row_sweep", "u_reduce_incl_waits", None,
             None]
    breakdown["factor_phase_us_per_sweep"] = {
        k: float(v) / 1e3 / iters for k, v in zip(names, ph.cpu().tolist())
        if k is not None}

    # ---- one power pass of the two-sided sketch (A X and A^T Y from one
    # read of A), timed through the public call: panel pack + fused kernel
    # + partial-slot sum.  Algorithmic bytes: one read of A, the two panels
    # read and the two products written.
    X = torch.randn(n, d, device=dev)
    Y = torch.randn(m, d, device=dev)
    for _ in range(3):
        cn.cnmf_sketch_pass(A, X, Y)
    reps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        cn.cnmf_sketch_pass(A, X, Y)
    e1.record(stream)
    torch.cuda.synchronize()
    pass_ms = e0.elapsed_time(e1) / reps          # A X and A^T Y
    bytes_pass = 4.0 * m * n + 2 * 4.0 * (m + n) * d
    peaks = _peaks()
    sketch_gbs = bytes_pass / (pass_ms * 1e-3) / 1e9
    # the whole compression: (2q + 2) reads of A (2q + 1 fused passes and
    # A-check) over the compression's CUDA-event time
    comp_bytes = (2 * q + 2) * 4.0 * m * n
    comp_gbs = comp_bytes / (breakdown["compress_ms"] * 1e-3) / 1e9

    # ---- dominant kernel of the step: the compressed ADMM launch
    # (k_admm_fast, all 500 sweeps in one cooperative launch), timed by the
    # events around each cnmf_factor inside the timed region (half of the
    # SMs, beside the next step's compression).  Algorithmic bytes per
    # sweep: L, R^T (d each) and U, Lam, V^T, Phi^T (r each, read and
    # written) per row: 4 (m + n)(d + 4 r).
    admm_bytes = 4.0 * (m + n) * (d + 4 * r) * iters
    admm_gbs = admm_bytes / (admm_ms_live * 1e-3) / 1e9
    traffic = _traffic("k_admm_fast", iters)
    breakdown["sequential_ms_per_step"] = seq_ms
    breakdown["pipelined_admm_ms"] = admm_ms_live

    out = {
        "metric": METRIC, "value": value, "unit": "factorizations/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(world),
        "run": {"lambda": lam,
                "pipelining": f"compressions on one stream ({cap_c} SMs) "
                              f"beside the ADMM sweeps of the previous "
                              f"{nfs} step(s), each ADMM launch on its own "
                              f"stream ({cap} of {nsm} SMs each)"},
        "roofline": {"bound": "hbm", "achieved": admm_gbs,
                     "peak": peaks["hbm"], "unit": "GB/s",
                     "frac": admm_gbs / peaks["hbm"], "traffic": traffic,
                     "kernel": f"k_admm_fast ({iters} sweeps, one launch, "
                               f"{cap} CTAs, beside a compression and "
                               f"{nfs - 1} other ADMM launch(es))",
                     "algorithmic_bytes": admm_bytes,
                     "peak_source": peaks["src"] + " (copy bandwidth)",
                     "note": "latency-bound: the small algebra (two r x r "
                             "solves per sweep) and the waits for the "
                             "slowest CTA's shares; the working set stays "
                             "in shared memory and L2, so the HBM fraction "
                             "is a note and `latency` is the figure of "
                             "merit",
                     "latency": admm_latency_model(breakdown, admm_ms_live,
                                                   iters)},
        "roofline_sketch": {"bound": "hbm", "achieved": sketch_gbs,
                            "peak": peaks["hbm"], "unit": "GB/s",
                            "frac": sketch_gbs / peaks["hbm"],
                            "traffic": _traffic("k_fused_pass", 1),
                            "traffic_note": "the fused kernel's DRAM bytes "
                                            "per pass (ncu); the pack and "
                                            "the partial-slot sum read "
                                            "L2-resident data",
                            "kernel": "cnmf_sketch_pass: k_fu_pack + "
                                      "k_fused_pass (one read of A, tcgen05 "
                                      "bf16 hi+lo split) + k_fu_reduce",
                            "algorithmic_bytes": bytes_pass,
                            "algorithmic_bytes_note": "one read of A (4 m n) "
                                                      "+ panels read and "
                                                      "products written "
                                                      "(8 (m + n) d)",
                            "ms_per_pass": pass_ms,
                            "compression": {
                                "reads_of_A": 2 * q + 2,
                                "algorithmic_bytes": comp_bytes,
                                "ms": breakdown["compress_ms"],
                                "achieved": comp_gbs,
                                "frac": comp_gbs / peaks["hbm"],
                                "note": "whole cnmf_compress incl. "
                                        "CholeskyQR sweeps and A-tilde"}},
        "clocks": clk.summary(),
        "breakdown": breakdown,
        "gpu_launches": launches_per_step(q) * args.steps,
        "gpu_launches_note": "library kernels per step: 2 Gaussian panels, "
                             "per pass (pack, fused pass, partial sum) + "
                             "one CholeskyQR sweep (gram, finish, apply), "
                             "CholeskyQR2 after the last pass (5), A-check "
                             "(3), cross product (2), one ADMM launch",
    }

    # ---- end to end through the public API with host buffers: every step
    # copies its A, U0, V0^T from pinned host memory and reads U, V^T back,
    # pipelined like the timed steps (compressions on one stream, ADMM
    # sweeps on the ADMM streams, each capped at its share of the SMs).  The
    # copy of the
    # next step's A (a copy stream, into the other of two device buffers)
    # starts as soon as the previous step's compression is done with that
    # buffer.  The step's own U0, V0^T are queued before it: behind the
    # 800 MB copy they would wait for its whole transfer.
    A_pin = torch.from_numpy(A_h).pin_memory()
    U_pin = torch.from_numpy(U0_h).pin_memory()
    Vt_pin = torch.from_numpy(Vt0_h).pin_memory()
    U_outs = [torch.empty_like(U_pin).pin_memory() for _ in range(nfs)]
    Vt_outs = [torch.empty_like(Vt_pin).pin_memory() for _ in range(nfs)]
    U_out, Vt_out = U_outs[0], Vt_outs[0]
    A_dev = [A, torch.empty_like(A)]
    cstream = torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]     # A of step k landed
    ev_done = [torch.cuda.Event() for _ in range(2)]   # compression k done

    def h2d(k, after):
        with torch.cuda.stream(cstream):
            if after is not None:
                cstream.wait_event(after)
            A_dev[k % 2].copy_(A_pin, non_blocking=True)
            ev_in[k % 2].record(cstream)

    def e2e_step(k):
        b = k % 2
        j = k % nfs
        sf = sFs[j]
        with torch.cuda.stream(sf):
            Us[j].copy_(U_pin, non_blocking=True)
            Vts[j].copy_(Vt_pin, non_blocking=True)
        cn.set_thread_cta_limit(cap_c)
        with torch.cuda.stream(sC):
            sC.wait_event(ev_in[b])
            L, Rt, At, _ = cn.cnmf_compress(A_dev[b], r, d, q, SEEDS["sketch"],
                                            status=st, ws=ws_c)
            ev_done[b].record(sC)
        h2d(k + 1, ev_done[1 - b])      # buffer of step k - 1, now free
        sf.wait_event(ev_done[b])
        for t in (L, Rt, At):
            t.record_stream(sf)
        with torch.cuda.stream(sf):
            cn.set_thread_cta_limit(cap)
            cn.cnmf_factor(L, Rt, At, Us[j], Vts[j], lam, lam, iters,
                           status=st, ws=ws_fs[j])
            U_outs[j].copy_(Us[j], non_blocking=True)
            Vt_outs[j].copy_(Vts[j], non_blocking=True)

    h2d(0, None)
    e2e_step(0)
    torch.cuda.synchronize()
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ee0.record(sF)
    for o in sFs[1:] + [sC, cstream]:
        o.wait_event(ee0)
    for k in range(1, args.steps + 1):
        e2e_step(k)
    join_all()
    sF.wait_stream(cstream)            # the last copy ends inside the region
    ee1.record(sF)
    torch.cuda.synchronize()
    cn.set_thread_cta_limit(0)
    cn.raise_on_status(st, "bench e2e")
    e2e_ms = replicas.slowest_ms(ee0.elapsed_time(ee1) / args.steps, dev)
    out["e2e"] = {"value": replicas.job_rate(1, e2e_ms, world),
                  "unit": "factorizations/s",
                  "h2d_bytes_per_step": int(A_pin.numel() * 4 + U_pin.numel() * 4
                                            + Vt_pin.numel() * 4),
                  "d2h_bytes_per_step": int(U_out.numel() * 4 + Vt_out.numel() * 4),
                  "ms_per_step": e2e_ms,
                  "overlap": "the next step's H2D copy of A (copy stream, "
                             "second device buffer) and the next "
                             "compression run beside this step's ADMM "
                             "sweeps"}

    # ---- out-of-core compression: the same A from page-locked host memory,
    # streamed through the GPU in row blocks once per pass; against the
    # host-to-device copy rate of the same buffer
    out["out_of_core"] = out_of_core_bench(cn, A_pin, dev, stream,
                                           block_rows=2048)

    # ---- time to the residual target vs plain ADMM (same GPU)
    if not args.no_ttt:
        out["time_to_target"] = time_to_target(cn, A, U0, Vt0, ws_c, ws_f,
                                               st, stream)
        # the noiseless companion: A = X0 Y0 exactly, tau = 1e-3 literally
        A0 = torch.from_numpy(synth.lowrank(m, n, r, 0.0, SEEDS["data"],
                                            dtype=np.float32)).to(dev)
        out["time_to_target_noiseless"] = time_to_target(
            cn, A0, U0, Vt0, ws_c, ws_f, st, stream, noiseless=True,
            alg2=False)
        del A0

    if not args.no_serving:
        out["serving"] = serving_bench(args.serving_requests)
    if not args.no_extra:
        out["snmf_wide"] = snmf_bench(cn, dev)
        out["mixed_precision"] = mixed_bench(cn, dev)
        out["mixed_precision"]["errors"] = mixed_error_bench(cn, dev)
        out["small_fp64"] = small_fp64_bench(cn, dev)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, secs, desc = cpu_oracle_sample()
        v1, desc1 = cpu_oracle_one_core()
        out["cpu_baseline"] = {"value": v, "unit": "factorizations/s",
                               "cores": os.cpu_count(), "kind": "oracle",
                               "sample": desc, "seconds": secs,
                               "one_core": {"value": v1, "cores": 1,
                                            "sample": desc1}}
        if not args.no_extra:
            s_w, ok_w = cpu_oracle_snmf_wide()
            out["cpu_baseline"]["snmf_wide"] = {
                "seconds": s_w, "anchors_planted": ok_w,
                "cores": os.cpu_count(),
                "sample": "oracle snmf_select on the full 10000 x 100000 "
                          "FP64 matrix (q = 2, d = 60), one run"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _time(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def snmf_bench(cn, dev):
    """Compressed SNMF on the wide separable workload (10000 x 100000,
    r = 50, d = 60, q = 2, FP32): time of snmf_select (one-sided sketch,
    R-hat = Q^T A, SPA) and whether the planted anchors came back."""
    import torch
    m, n, r, d, q = 10000, 100000, 50, 60, 2
    A, planted = synth.separable_torch(m, n, r, 1e-3, 1002, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(cn.lib().snmf_select_workspace(m, n, d, 1),
                     dtype=torch.uint8, device=dev)
    res = {}
    ms = _time(lambda: res.update(a=cn.snmf_select(A, r, d, q, 2002, status=st,
                                                   ws=ws)[0]),
               5, torch.cuda.current_stream(dev))
    cn.raise_on_status(st, "snmf bench")
    ok = sorted(res["a"].cpu().tolist()) == sorted(planted.cpu().tolist())
    passes = 2 * q + 2          # 2q + 1 sketch products + R-hat
    out = {"workload": "separable 10000 x 100000, r=50, d=60, q=2, fp32",
           "ms": ms, "anchors_planted": ok,
           "sketch_gbs": passes * 4.0 * m * n / (ms * 1e-3) / 1e9}
    # Alg. 3 step 3: the right factor Y (r x n) by per-column NNLS on the
    # compressed Rhat, and the relative residual ||A - A[:, K] Y|| / ||A||
    anchors, Rt, _ = cn.snmf_select(A, r, d, q, 2002, status=st, ws=ws,
                                    return_rhat=True)
    wsr = torch.empty(cn.lib().snmf_right_factor_workspace(n, d, r, 1),
                      dtype=torch.uint8, device=dev)
    rf = {}
    ms_rf = _time(lambda: rf.update(y=cn.snmf_right_factor(
        Rt, anchors, max_sweeps=1000, tol=1e-6, status=st, ws=wsr)),
                  5, torch.cuda.current_stream(dev))
    cn.raise_on_status(st, "snmf right factor")
    Y, unconv, _ = rf["y"]
    Xk = A[:, anchors]
    res2 = torch.zeros(2, dtype=torch.float64, device=dev)
    cn.cnmf_residual(A, Xk.contiguous(), Y.t().contiguous(), out=res2)
    e2, a2 = res2.cpu().tolist()
    out["right_factor"] = {"ms": ms_rf, "unconverged_columns": int(unconv.item()),
                           "rel_residual": (e2 / a2) ** 0.5,
                           "solver": "projected coordinate descent on the "
                                     "shared r x r Gram, tol 1e-6"}
    return out


def mixed_bench(cn, dev):
    """Compression of the 50000 x 50000, r = 64 matrix (d = 80, q = 4) with
    BF16 and FP32 storage: time and algorithmic bytes of A per second
    ((2q + 2) reads of A), beside the bytes actually moved."""
    import torch
    m = n = 50000
    r, d, q = 64, 80, 4
    out = {"workload": "lowrank 50000 x 50000, r=64, d=80, q=4 (and the "
                       "same matrices with r=20, d=30: the fused pass)"}
    for name, dt in (("bf16", torch.bfloat16), ("fp32", torch.float32)):
        A = synth.lowrank_torch(m, n, r, 0.01, 1003, device=dev).to(dt)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        for rr, dd, key in ((r, d, name), (20, 30, name + "_d30")):
            ws = torch.empty(cn.lib().cnmf_compress_workspace(
                m, n, dd, 2 if name == "bf16" else 1), dtype=torch.uint8,
                device=dev)
            ms = _time(lambda: cn.cnmf_compress(A, rr, dd, q, 2003, status=st,
                                                ws=ws),
                       3, torch.cuda.current_stream(dev))
            cn.raise_on_status(st, "mixed bench")
            # algorithmic bytes: (2q + 2) reads of A (2q + 1 two-sided
            # passes and A-check, one read each).  d <= 32 runs the fused
            # pass and moves exactly that; wider panels read A once per
            # product (2 (2q + 1) + 1 reads moved)
            alg_reads = 2 * q + 2
            reads = alg_reads if dd <= 32 else 2 * (2 * q + 1) + 1
            gbs = alg_reads * A.element_size() * m * n / (ms * 1e-3) / 1e9
            out[key] = {"d": dd, "compress_ms": ms,
                        "algorithmic_reads_of_A": alg_reads,
                        "reads_of_A_moved": reads,
                        "gbs": gbs, "frac": gbs / _peaks()["hbm"],
                        "moved_gbs": gbs * reads / alg_reads}
            del ws
        del A
        torch.cuda.empty_cache()
    return out


def mixed_error_bench(cn, dev):
    """Accuracy cost of the mixed-precision sketch, per storage type: the
    compression of a 3000 x 3000, r = 64 matrix (d = 80, q = 4) against the
    library's FP64 compression of the same stored values (that path matches
    the FP64 oracle to 1e-9 in the GPU tests), and 200 FP32 ADMM sweeps from
    the same start on each.  Reported: the rank-r signal projector distance
    and the relative difference of the final residual rho."""
    import torch
    m = n = 3000
    r, d, q, it = 64, 80, 4, 200
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    A32 = synth.lowrank_torch(m, n, r, 0.01, 1003, device=dev)
    U0, Vt0 = synth.init_torch(m, n, r, 3003, device=dev)

    def basis(L, A):
        W, _, _ = np.linalg.svd(L.T @ A, full_matrices=False)
        return L @ W[:, :r]

    def resid(A, U, Vt):
        e2, a2 = cn.cnmf_residual(A, U, Vt).cpu().tolist()
        return float(np.sqrt(e2 / a2))

    out = {"workload": "lowrank 3000 x 3000, r=64, d=80, q=4, 200 ADMM sweeps",
           "reference": "the library's FP64 path on the same stored values"}
    for name, dt in (("bf16", torch.bfloat16), ("fp32", torch.float32)):
        As = A32.to(dt)
        A64 = As.double()
        res = {}
        for key, Ain in (("ref", A64), ("low", As)):
            L, Rt, At, _ = cn.cnmf_compress(Ain, r, d, q, 2003, status=st)
            # the same FP32 sweeps on both compressions, so the difference
            # is the sketch's (the FP64 factor kernel stops at r d below
            # this size)
            L, Rt, At = L.float(), Rt.float(), At.float()
            lam = cn.default_penalty(At, r)
            U, Vt = U0.clone(), Vt0.clone()
            cn.cnmf_factor(L, Rt, At, U, Vt, lam, lam, it, status=st)
            res[key] = (L.double().cpu().numpy(), resid(As, U, Vt))
        cn.raise_on_status(st, "mixed error bench")
        Ah = A64.cpu().numpy()
        B1, B0 = basis(res["low"][0], Ah), basis(res["ref"][0], Ah)
        ep = float(np.sqrt(2.0) * np.linalg.norm(B1 - B0 @ (B0.T @ B1)) /
                   np.sqrt(r))
        out[name] = {"signal_projector": ep,
                     "rho": res["low"][1], "rho_fp64_path": res["ref"][1],
                     "rho_rel_diff": abs(res["low"][1] - res["ref"][1]) /
                                     res["ref"][1]}
    return out


def serving_bench(nreq: int):
    """Served stream of compressed-NMF requests: m, n ~ U[200, 4000],
    r ~ U{5..32}, d = r + 10, q = 4, FP32, 40 GB budget.  Every request runs
    until its relative residual is within 1e-3 of the rank-r floor
    (checked every 20 sweeps, cap 3000).  Saturation throughput from a
    closed run (all requests at t = 0), then a Poisson stream at 0.8 x
    saturation; p50 / p99 latency of the latter, at that accuracy."""
    import tempfile
    from paper_1505_04650_gb300 import serve
    from paper_1505_04650_gb300.autotune import Autotuner
    tuner = Autotuner(os.path.join(tempfile.gettempdir(), "cnmf_autotune.json"),
                      sweeps=10, problems=64, reps=2)
    reqs = serve.make_workload(nreq, rate=0.0, seed=4)
    kw = dict(hbm_budget=40e9, tuner=tuner, stop_at_target=True,
              check_every=20, max_sweeps=3000)
    srv = serve.Server(**kw)
    t0 = time.perf_counter()
    srv.prepare(reqs)
    tune_s = time.perf_counter() - t0
    sat = srv.run(reqs, realtime=False)
    rate = 0.8 * sat["factorizations_per_s"]
    reqs = serve.make_workload(nreq, rate=rate, seed=4)
    srv = serve.Server(**kw)
    st = srv.run(reqs, realtime=True)
    return {"workload": f"{nreq} requests, m,n~U[200,4000], r~U{{5..32}}, "
                        "d=r+10, q=4, fp32, 40 GB budget, each to its "
                        "accuracy target",
            "saturation_factorizations_per_s": sat["factorizations_per_s"],
            "rate_per_s": rate, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "factorizations_per_s": st["factorizations_per_s"],
            "p50_at_target_ms": st.get("p50_at_target_ms"),
            "p99_at_target_ms": st.get("p99_at_target_ms"),
            "frac_at_target": st["frac_at_target"],
            "sweeps_mean": st["sweeps_mean"], "sweeps_p99": st["sweeps_p99"],
            "target": "rho <= rank-r floor + 1e-3 (floor from Atilde)",
            "stop": st["stop"], "penalty": st["penalty"],
            "cluster_sizes": st["cluster_sizes"], "autotune_s": tune_s}


def _first_at(step, check, every, cap):
    """Advance `step(k)` by `every` until `check()` <= 0 or `cap`; returns
    (k*, last value) with k* None when the cap came first."""
    val = None
    for k in range(every, cap + 1, every):
        step(every)
        val = check()
        if val <= 0:
            return k, val
    return None, val


def _replay(fn, stream, reps=4):
    """Median CUDA-event time (s) of `fn()` over reps - 1 timed runs."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ts = []
    for rep in range(reps):
        torch.cuda.synchronize()
        ev[0].record(stream)
        fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        if rep:
            ts.append(ev[0].elapsed_time(ev[1]))
    return float(np.median(ts)) / 1e3


def time_to_target(cn, A, U0, Vt0, ws_c, ws_f, st, stream, noiseless=False,
                   alg2=True):
    """Time to the residual target tau: the first sweep (iteration) count
    k* with rho = ||A - U V|| / ||A|| <= tau, found by checking rho every
    few sweeps, then a timed replay of compression + k* sweeps.  tau =
    rho* + 1e-3 with rho* the residual of the rank-r SVD truncation of
    A-tilde lifted back to m x n (an upper estimate of the rank-r floor);
    tau = 1e-3 literally for the noiseless companion (floor 0).

    The penalties are not given by the paper (Alg. 4); each ADMM -- the
    compressed one and the plain, uncompressed one on the same GPU -- runs
    at its best of lambda = phi = c ||M||_F / r, c in {0.03, 0.1, 0.3, 1, 3}, M =
    A-tilde or A.  Alg. 2 (exact NNLS steps and multiplicative updates)
    needs no penalty."""
    import torch
    m, n, r, d, q = CFG["m"], CFG["n"], CFG["r"], CFG["d"], CFG["q"]
    from paper_1505_04650_gb300.serve import truncation_factors
    sk = SEEDS["sketch"]
    L, Rt, At, _ = cn.cnmf_compress(A, r, d, q, sk, status=st, ws=ws_c)
    res = cn.cnmf_residual(A, *truncation_factors(L, Rt, At, r))
    a2 = float(res[1].item())
    floor = 0.0 if noiseless else float(np.sqrt(float(res[0].item()) / a2))
    tau = floor + 1e-3

    def rho_of(U, Vt):
        e2, b2 = cn.cnmf_residual(A, U, Vt).cpu().tolist()
        return float(np.sqrt(e2 / b2))

    scales = (0.03, 0.1, 0.3, 1.0, 3.0)
    out = {"tau": tau, "floor_est": floor,
           "penalty_sweep": "lambda = phi = c ||M||_F / r, c in "
                            f"{list(scales)}, best per method"}
    # ---- compressed ADMM (Alg. 4)
    nA = float(torch.linalg.norm(At.double()).item())
    comp = {"sweep": {}}
    for c in scales:
        lam = c * nA / r
        U, Vt = U0.clone(), Vt0.clone()
        box = {"state": None}

        def step(k, lam=lam, U=U, Vt=Vt, box=box):
            _, _, box["state"], _ = cn.cnmf_factor(L, Rt, At, U, Vt, lam, lam,
                                                   k, state=box["state"],
                                                   status=st, ws=ws_f)
        k, rho = _first_at(step, lambda: rho_of(U, Vt) - tau, 10, 1500)
        comp["sweep"][str(c)] = k
        if k is not None and ("k" not in comp or k < comp["k"]):
            comp.update(k=k, c=c, lam=lam)
    if "k" in comp:
        U, Vt = U0.clone(), Vt0.clone()

        def run_c():
            U.copy_(U0); Vt.copy_(Vt0)
            Lx, Rx, Ax, _ = cn.cnmf_compress(A, r, d, q, sk, status=st, ws=ws_c)
            cn.cnmf_factor(Lx, Rx, Ax, U, Vt, comp["lam"], comp["lam"],
                           comp["k"], status=st, ws=ws_f)
        comp["seconds"] = _replay(run_c, stream)
        comp["rho"] = rho_of(U, Vt)
    out["compressed_admm"] = comp
    # ---- plain (uncompressed) ADMM on the same GPU
    ws_p = torch.empty(cn.lib().cnmf_plain_workspace(m, n, r, 1),
                       dtype=torch.uint8, device=A.device)
    plain = {"sweep": {}, "cap": 3000}
    for c in scales:
        lam = c * float(np.sqrt(a2)) / r
        U, Vt = U0.clone(), Vt0.clone()
        box = {"state": None}

        def step(k, lam=lam, U=U, Vt=Vt, box=box):
            _, _, box["state"], _ = cn.cnmf_factor_plain(
                A, U, Vt, lam, lam, k, state=box["state"], status=st, ws=ws_p)
        k, rho = _first_at(step, lambda: rho_of(U, Vt) - tau, 10,
                           plain["cap"])
        plain["sweep"][str(c)] = k
        if k is not None and ("k" not in plain or k < plain["k"]):
            plain.update(k=k, c=c, lam=lam)
    if "k" in plain:
        U, Vt = U0.clone(), Vt0.clone()

        def run_p():
            U.copy_(U0); Vt.copy_(Vt0)
            cn.cnmf_factor_plain(A, U, Vt, plain["lam"], plain["lam"],
                                 plain["k"], status=st, ws=ws_p)
        plain["seconds"] = _replay(run_p, stream, reps=3)
        plain["rho"] = rho_of(U, Vt)
    out["plain_admm"] = plain
    if comp.get("seconds") and plain.get("seconds"):
        out["speedup_vs_plain"] = plain["seconds"] / comp["seconds"]
    if not alg2:
        cn.raise_on_status(st, "time to target")
        return out
    # ---- compressed alternating NMF (Alg. 2): exact NNLS steps and
    # multiplicative updates, from (0, V0) and (U0, V0)
    Y0 = Vt0.t().contiguous()
    for name, every, cap in (("alg2_nnls", 2, 100), ("alg2_mu", 20, 2000)):
        box = {"X": U0.clone(), "Y": Y0.clone()}

        def step(k, name=name, box=box):
            if name == "alg2_nnls":
                box["X"], box["Y"], _, _ = cn.cnmf_factor_als(
                    A, L, Rt, box["Y"], k, status=st)
            else:
                box["X"], box["Y"], _ = cn.cnmf_factor_mu(
                    A, L, Rt, box["X"], box["Y"], k, status=st)

        def chk(box=box):
            return rho_of(box["X"], box["Y"].t().contiguous()) - tau
        k, rho = _first_at(step, chk, every, cap)
        ent = {"k": k, "cap": cap, "rho_last": rho + tau}
        if k is not None:
            def run_a(name=name, k=k):
                Lx, Rx, _, _ = cn.cnmf_compress(A, r, d, q, sk, status=st,
                                                ws=ws_c)
                if name == "alg2_nnls":
                    cn.cnmf_factor_als(A, Lx, Rx, Y0, k, status=st)
                else:
                    cn.cnmf_factor_mu(A, Lx, Rx, U0, Y0, k, status=st)
            ent["seconds"] = _replay(run_a, stream, reps=3)
        out[name] = ent
    cn.raise_on_status(st, "time to target")
    return out


def out_of_core_bench(cn, A_pin, dev, stream, block_rows=2048):
    """cnmf_compress_host on the benchmark workload with A (800 MB FP32)
    in page-locked host memory: time, host bytes read per second over the
    (2q + 2) passes, and the plain host-to-device copy rate of A."""
    import torch
    m, n, r, d, q = CFG["m"], CFG["n"], CFG["r"], CFG["d"], CFG["q"]
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(cn.lib().cnmf_compress_host_workspace(m, n, d, 1,
                                                           block_rows),
                     dtype=torch.uint8, device=dev)
    ms = _time(lambda: cn.cnmf_compress_host(A_pin, r, d, q, SEEDS["sketch"],
                                             block_rows, device=dev,
                                             status=st, ws=ws),
               3, stream)
    cn.raise_on_status(st, "out-of-core compression")
    buf = torch.empty(m, n, dtype=torch.float32, device=dev)
    copy_ms = _time(lambda: buf.copy_(A_pin, non_blocking=True), 3, stream)
    nbytes = 4.0 * m * n
    reads = 2 * q + 2
    h2d = nbytes / (copy_ms * 1e-3) / 1e9
    gbs = reads * nbytes / (ms * 1e-3) / 1e9
    return {"workload": WORKLOAD + ", A in page-locked host memory",
            "block_rows": block_rows, "reads_of_A": reads, "ms": ms,
            "host_read_gbs": gbs, "h2d_copy_gbs": h2d,
            "frac_of_h2d": gbs / h2d,
            "device_bytes": int(ws.numel()),
            "note": "two block buffers: the copy of block k + 1 (the "
                    "library's copy stream) overlaps the products of block "
                    "k (the caller's stream)"}


def small_fp64_bench(cn, dev):
    """The small FP64 workload (m = 500, n = 400, r = 10, d = 20, q = 4,
    100 ADMM sweeps): GPU time of compression + sweeps and the residual."""
    import torch
    m, n, r, d, q, it = 500, 400, 10, 20, 4, 100
    A = torch.from_numpy(synth.lowrank(m, n, r, 0.01, 1000)).to(dev)
    U0, V0 = synth.init_factors(m, n, r, 3000)
    U0 = torch.from_numpy(U0).to(dev)
    Vt0 = torch.from_numpy(np.ascontiguousarray(V0.T)).to(dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    box = {}

    def run():
        L, Rt, At, _ = cn.cnmf_compress(A, r, d, q, 2000, status=st)
        lam = cn.default_penalty(At, r)
        U, Vt = U0.clone(), Vt0.clone()
        cn.cnmf_factor(L, Rt, At, U, Vt, lam, lam, it, status=st)
        box.update(U=U, Vt=Vt)
    ms = _time(run, 5, torch.cuda.current_stream(dev))
    cn.raise_on_status(st, "small fp64")
    e2, a2 = cn.cnmf_residual(A, box["U"], box["Vt"]).cpu().tolist()
    return {"workload": "lowrank 500 x 400, r=10, d=20, q=4, 100 sweeps, fp64",
            "ms": ms, "rho": float(np.sqrt(e2 / a2)),
            "note": "launch- and latency-bound (1.6 MB A); the penalty "
                    "lambda = ||Atilde||_F / r is read back to the host "
                    "inside the timed region"}


if __name__ == "__main__":
    sys.exit(main())
