"""The negative-entry flag (cnmf_check_nonnegative) through the C ABI.

NMF and SNMF are posed for A >= 0 (Sec. II; Sec. IV); a negative entry is
reported as the flag bit CNMF_STATUS_NEGATIVE_A of the device status word,
not as an error.  What the flag must say is fixed by the definition "some
entry compares below zero", checked here on planted cases:

* a nonnegative A (uniform, with exact zeros and -0.0 entries, and NaN)
  leaves the status word at zero;
* one negative entry planted at the first, the last and an interior
  position, in every storage type, with row lengths that are and are not
  whole 16-byte chunks and row pitches that are and are not 16-byte
  multiples (the vector and the scalar loads), sets the flag;
* negative values in the padding between n and lda are not part of A and
  leave the flag clear;
* the flag and an error code live side by side: a later error is still
  recorded (first error wins among errors) and the flag stays set.
"""
import ctypes as C

import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

DTYPES = ["f64", "f32", "bf16"]


def _tdt(torch, name):
    return {"f64": torch.float64, "f32": torch.float32,
            "bf16": torch.bfloat16}[name]


def _padded(torch, m, n, lda, dtype, seed, pad_value=-1.0):
    g = torch.Generator(device="cuda").manual_seed(seed)
    buf = torch.rand(m, lda, generator=g, device="cuda", dtype=torch.float32)
    buf[:, n:] = pad_value
    return buf.to(dtype)[:, :n]


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("m,n,lda", [(1, 1, 1), (37, 8, 8), (300, 1000, 1000),
                                     (300, 1003, 1003), (129, 77, 80),
                                     (257, 500, 516), (64, 4096, 4096)])
def test_flag_matches_definition(dt, m, n, lda):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    dtype = _tdt(torch, dt)
    A = _padded(torch, m, n, lda, dtype, 7 + m + n)
    assert A.stride(0) == lda
    # zeros, -0.0 and a NaN are not negative
    A[0, 0] = 0.0
    A[m - 1, n - 1] = -0.0
    if m * n > 2:
        A[m // 2, n // 2] = float("nan")
    st = cn.cnmf_check_nonnegative(A)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    for (i, j) in {(0, 0), (m - 1, n - 1), (m // 2, (3 * n) // 4)}:
        B = A.clone() if lda == n else _padded(torch, m, n, lda, dtype, 1)
        if lda != n:
            B[0, 0] = 0.0
        old = float(B[i, j])
        B[i, j] = -2.0 ** -10
        st = cn.cnmf_check_nonnegative(B)
        assert cn.has_negative_entries(st), (i, j)
        assert int(st.item()) == cn._lib.CNMF_STATUS_NEGATIVE_A
        B[i, j] = old


def test_padding_is_not_read():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    for dt in DTYPES:
        A = _padded(torch, 200, 301, 320, _tdt(torch, dt), 3, pad_value=-5.0)
        st = cn.cnmf_check_nonnegative(A)
        assert int(st.item()) == 0, dt


def test_flag_beside_error_code():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    L = cn.lib()
    A = torch.rand(100, 50, device="cuda")
    A[3, 4] = -1.0
    st = cn.cnmf_check_nonnegative(A)
    # a later device-detected error is still recorded, the flag stays: the
    # bounded grid barrier's self-test with one CTA that never arrives
    ws = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    code = L.cnmf_barrier_selftest(4, 2, 1, 200, C.c_void_p(ws.data_ptr()),
                                   ws.numel(), C.c_void_p(st.data_ptr()),
                                   C.c_void_p(out.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream()
                                              .cuda_stream))
    assert code == 0
    torch.cuda.synchronize()
    v = int(st.item())
    assert v & cn._lib.CNMF_STATUS_NEGATIVE_A
    assert v & cn._lib.CNMF_STATUS_CODE_MASK == cn._lib.CNMF_E_TIMEOUT
    with pytest.raises(cn.CnmfError):
        cn.raise_on_status(st, "selftest")
    # a flag alone is not an error
    st2 = cn.cnmf_check_nonnegative(A)
    cn.raise_on_status(st2, "flag only")


def test_host_errors():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    L = cn.lib()
    A = torch.rand(10, 10, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = C.c_void_p(A.data_ptr())
    ps = C.c_void_p(st.data_ptr())
    assert L.cnmf_check_nonnegative(p, 1, 10, 10, 10, None, s) == 1
    assert L.cnmf_check_nonnegative(None, 1, 10, 10, 10, ps, s) == 1
    assert L.cnmf_check_nonnegative(p, 1, 10, 10, 9, ps, s) == 1
    assert L.cnmf_check_nonnegative(p, 7, 10, 10, 10, ps, s) == 1
    assert L.cnmf_check_nonnegative(p, 1, 0, 10, 10, ps, s) == 1
