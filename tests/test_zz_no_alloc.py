"""cnmf_residual_noalloc against cnmf_residual, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device
memory (a plugin whose host application owns all device allocations, code
running while another allocator has reserved the device, a latency-critical
loop that must not reach cudaMalloc).  Its scratch is a static device array
inside the library, shared by every call, so two calls in a row must both
agree with the workspace-taking entry point, and the second call must leave
the device's allocated and free memory unchanged.  This file is collected
last.
"""
import ctypes as C

import numpy as np
import pytest

import synth

from gpu_util import need_gpu, to_dev, wdt

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,m,n,r", [("f32", 2000, 1500, 20),
                                           ("bf16", 513, 300, 7),
                                           ("f64", 300, 257, 5)])
def test_residual_noalloc_matches_workspace_entry_point(storage, m, n, r):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    from paper_1505_04650_gb300 import _lib
    lib = _lib.load()
    As = synth.as_storage(synth.lowrank(m, n, r, 0.05, 31), storage)
    Ad = to_dev(As, storage)
    U0, V0 = synth.init_factors(m, n, r, 32)
    w = wdt(storage)
    U = torch.tensor(U0, dtype=w).cuda()
    Vt = torch.tensor(V0.T.copy(), dtype=w).cuda()
    ref = cn.cnmf_residual(Ad, U, Vt).cpu().numpy()
    dt = {"f64": _lib.CNMF_F64, "f32": _lib.CNMF_F32, "bf16": _lib.CNMF_BF16}
    wt = _lib.CNMF_F64 if storage == "f64" else _lib.CNMF_F32
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    tol = 1e-12 if storage == "f64" else 2e-5
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    host = torch.empty(2, dtype=torch.float64, pin_memory=True)
    mem = []
    for call in range(2):
        out.fill_(-1.0)
        rc = lib.cnmf_residual_noalloc(
            C.c_void_p(Ad.data_ptr()), dt[storage], m, n, Ad.stride(0),
            C.c_void_p(U.data_ptr()), C.c_void_p(Vt.data_ptr()), wt, r,
            C.c_void_p(out.data_ptr()), s)
        assert rc == 0, lib.cnmf_last_error().decode()
        host.copy_(out)
        torch.cuda.synchronize()
        # what the process holds on the device after the call: PyTorch's
        # allocations and the driver's free-memory count
        mem.append((torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]))
        got = host.numpy()
        assert abs(got[1] - ref[1]) <= tol * ref[1], call
        assert abs(got[0] - ref[0]) <= tol * ref[1], call
    # the second call allocated nothing, through PyTorch or the driver
    assert mem[1] == mem[0], mem


def test_residual_noalloc_rejects_bad_arguments():
    torch = need_gpu()
    from paper_1505_04650_gb300 import _lib
    lib = _lib.load()
    x = torch.zeros(16, device="cuda")
    p = C.c_void_p(x.data_ptr())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # FP64 A with FP32 factors, and r out of range
    assert lib.cnmf_residual_noalloc(p, _lib.CNMF_F64, 2, 2, 2, p, p,
                                     _lib.CNMF_F32, 1, p, s) == 1
    assert lib.cnmf_residual_noalloc(p, _lib.CNMF_F32, 2, 2, 2, p, p,
                                     _lib.CNMF_F32, 200, p, s) == 1
