"""Programmatic dependent launch changes scheduling only, never results.

The pass chain (panel pack, fused pass, partial-slot sum, CholeskyQR
kernels) is launched with programmatic stream serialisation; every kernel
waits for the kernels before it before it touches their outputs.  If a
wait were missing, a kernel could read a panel that is still being
written.  Here the same compressions run in one child process
(programmatic launch on) and in another with CNMF_NO_PDL set (plain stream
order), and L, R^T and A-tilde must agree bit for bit: FP32 and BF16 A
through the fused pass, FP64 A through the CUDA-core products, a ragged
shape, and the out-of-core path with its copy stream.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [("f32", 3000, 2000, 10, 30, 2), ("bf16", 2100, 3300, 8, 16, 1),
         ("f64", 700, 500, 5, 12, 2), ("f32", 1000, 777, 6, 20, 3)]

_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import synth
import paper_1505_04650_gb300 as cn
out = {}
for i, (dt, m, n, r, d, q) in enumerate(eval(sys.argv[2])):
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[dt]
    A = torch.from_numpy(synth.lowrank(m, n, r, 0.01, 40 + i)).to(tdt)
    L, Rt, At, st = cn.cnmf_compress(A.cuda(), r, d, q, 50 + i)
    cn.raise_on_status(st, "compress")
    out[f"c{i}"] = [x.double().cpu().numpy() for x in (L, Rt, At)]
    if dt != "f64":
        L, Rt, At, st = cn.cnmf_compress_host(A.pin_memory(), r, d, q, 50 + i,
                                             block_rows=m // 3 + 1)
        cn.raise_on_status(st, "compress_host")
        out[f"h{i}"] = [x.double().cpu().numpy() for x in (L, Rt, At)]
np.savez(sys.argv[3], **{k + "_" + str(j): v[j] for k, v in out.items()
                         for j in range(3)})
"""


def _run(tmp_path, env_extra, tag):
    env = dict(os.environ)
    env.update(env_extra)
    path = str(tmp_path / f"{tag}.npz")
    res = subprocess.run([sys.executable, "-c", _CHILD, ROOT, repr(CASES),
                          path], env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    return np.load(path)


def test_pdl_results_bitwise_equal_plain_order(tmp_path):
    need_gpu()
    env = {k: v for k, v in os.environ.items() if k == "CNMF_NO_PDL"}
    assert not env, "run without CNMF_NO_PDL in the environment"
    on = _run(tmp_path, {}, "pdl")
    off = _run(tmp_path, {"CNMF_NO_PDL": "1"}, "plain")
    assert sorted(on.files) == sorted(off.files)
    for k in on.files:
        a, b = on[k], off[k]
        assert a.shape == b.shape, k
        assert np.array_equal(a, b), (k, float(np.abs(a - b).max()))
