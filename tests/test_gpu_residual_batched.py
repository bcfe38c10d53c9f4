"""cnmf_residual_batched (many problems' ||A - U V||^2, ||A||^2 in one
launch) through the C ABI, against the one-problem cnmf_residual (itself
checked against the oracle) and the oracle's residual_sq.

Items of mixed sizes in one launch: fewer rows than one 64-row tile,
ragged columns, a row pitch above n, r from 1 to 32; FP32 and FP64; one
CTA per item and many.  An item whose r exceeds max_r gets NaN pairs and
the status word says CNMF_E_INVALID_ARG, while the others are unaffected.
"""
import numpy as np
import pytest

from oracle import residual as ores

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

SHAPES = [(30, 50, 1), (64, 64, 4), (200, 333, 7), (1000, 129, 20),
          (77, 2000, 32), (513, 700, 12)]


def _items(torch, cn, dt, pad):
    g = torch.Generator(device="cuda").manual_seed(3)
    probs = []
    for (m, n, r) in SHAPES:
        lda = n + (5 if pad else 0)
        buf = torch.rand(m, lda, generator=g, device="cuda", dtype=dt)
        A = buf[:, :n]
        U = torch.rand(m, r, generator=g, device="cuda", dtype=dt)
        Vt = torch.rand(n, r, generator=g, device="cuda", dtype=dt)
        probs.append((A, U, Vt))
    blob = b"".join(cn.residual_item_bytes(*p) for p in probs)
    items = torch.frombuffer(bytearray(blob), dtype=torch.uint8).cuda()
    return probs, items


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("ctas", [1, 8, 64])
def test_batched_matches_single_and_oracle(dtype, ctas):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    dt = torch.float32 if dtype == "f32" else torch.float64
    probs, items = _items(torch, cn, dt, pad=(ctas == 8))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = cn.cnmf_residual_batched(items, len(probs), dt, 32, ctas,
                                   status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    got = out.cpu().numpy()
    for k, (A, U, Vt) in enumerate(probs):
        one = cn.cnmf_residual(A, U, Vt).cpu().numpy()
        # the same sums split over other CTAs: FP64 rounding only
        assert np.allclose(got[k], one, rtol=1e-12, atol=0), (k, got[k], one)
        e2, a2 = ores.residual_sq(A.double().cpu().numpy(),
                                  U.double().cpu().numpy(),
                                  Vt.double().cpu().numpy().T)
        tol = 1e-5 if dtype == "f32" else 1e-12
        assert abs(got[k][0] - e2) <= tol * max(e2, 1e-30) + 1e-7 * a2
        assert abs(got[k][1] - a2) <= tol * a2


def test_bad_item_flags_and_others_unaffected():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    probs, items = _items(torch, cn, torch.float32, pad=False)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    # max_r = 12: the items with r = 20 and r = 32 are out of the launch
    out = cn.cnmf_residual_batched(items, len(probs), torch.float32, 12, 4,
                                   status=st).cpu().numpy()
    assert int(st.item()) == cn._lib.CNMF_E_INVALID_ARG
    for k, (A, U, Vt) in enumerate(probs):
        if SHAPES[k][2] > 12:
            assert np.isnan(out[k]).all()
        else:
            one = cn.cnmf_residual(A, U, Vt).cpu().numpy()
            assert np.allclose(out[k], one, rtol=1e-12, atol=0)


def test_host_errors():
    torch = need_gpu()
    import ctypes as C
    import paper_1505_04650_gb300 as cn
    L = cn.lib()
    ws = torch.empty(4096, dtype=torch.uint8, device="cuda")
    o = torch.empty(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(ws.data_ptr())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    f = L.cnmf_residual_batched
    assert f(None, 2, 1, 1, 8, 4, C.c_void_p(o.data_ptr()), p, 4096, None, s) == 1
    assert f(p, 0, 1, 1, 8, 4, C.c_void_p(o.data_ptr()), p, 4096, None, s) == 1
    assert f(p, 2, 1, 1, 200, 4, C.c_void_p(o.data_ptr()), p, 4096, None, s) == 1
    assert f(p, 2, 0, 1, 8, 4, C.c_void_p(o.data_ptr()), p, 4096, None, s) == 1
    assert f(p, 2, 1, 1, 8, 4, C.c_void_p(o.data_ptr()), p, 16, None, s) == 2
