"""Host-side checks of the C ABI (no GPU needed).

The library must load, export every entry point that include/cnmf.h
declares, and reject invalid arguments on the host with
CNMF_E_INVALID_ARG before anything is enqueued.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "cnmf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(
        r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?((?:cnmf|snmf)_[a-z0-9_]+)\s*\(",
        txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1505_04650_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("cnmf_compress", "cnmf_factor", "snmf_select",
                 "cnmf_residual", "cnmf_status_string", "cnmf_factor_plain"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1505_04650_gb300 import _lib
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, name


def test_status_strings(lib):
    for code in range(7):
        s = lib.cnmf_status_string(code).decode()
        assert s.startswith("CNMF_")
    assert lib.cnmf_status_string(99).decode() == "CNMF_E_UNKNOWN"
    assert lib.cnmf_abi_version() == 1


def test_invalid_arguments_rejected_on_host(lib):
    from paper_1505_04650_gb300._lib import AdmmParams
    E = 1  # CNMF_E_INVALID_ARG
    nul = None
    # NULL A / bad sizes / d > min(m, n) / r > d / q < 0 / lda < n
    assert lib.cnmf_compress(nul, 1, 10, 10, 10, 2, 4, 1, 0, nul, nul, 1, 1, 1,
                             1, 1 << 20, nul, nul) == E
    fake = C.c_void_p(16)
    assert lib.cnmf_compress(fake, 1, 10, 10, 9, 2, 4, 1, 0, nul, nul, fake,
                             fake, fake, fake, 1 << 20, nul, nul) == E
    assert lib.cnmf_compress(fake, 1, 10, 3, 3, 2, 4, 1, 0, nul, nul, fake,
                             fake, fake, fake, 1 << 20, nul, nul) == E
    assert lib.cnmf_compress(fake, 1, 10, 10, 10, 5, 4, 1, 0, nul, nul, fake,
                             fake, fake, fake, 1 << 20, nul, nul) == E
    assert lib.cnmf_compress(fake, 1, 10, 10, 10, 2, 4, -1, 0, nul, nul, fake,
                             fake, fake, fake, 1 << 20, nul, nul) == E
    assert lib.cnmf_compress(fake, 7, 10, 10, 10, 2, 4, 1, 0, nul, nul, fake,
                             fake, fake, fake, 1 << 20, nul, nul) == E
    p = AdmmParams(0.0, 1.0, 1.0, 10, 0, None, 0, 0)      # lambda must be > 0
    assert lib.cnmf_factor(fake, fake, fake, 1, 10, 10, 2, 4, C.byref(p), fake,
                           fake, fake, 0, fake, 1 << 20, nul, nul) == E
    p = AdmmParams(1.0, 1.0, 1.0, 10, 0, None, 0, 0)
    assert lib.cnmf_factor(fake, fake, fake, 1, 10, 10, 5, 4, C.byref(p), fake,
                           fake, fake, 0, fake, 1 << 20, nul, nul) == E
    assert lib.snmf_select(fake, 1, 10, 10, 10, 3, 2, 1, 0, nul, fake, nul,
                           fake, 1 << 20, nul, nul) == E
    assert lib.cnmf_residual(fake, 0, 10, 10, 10, fake, fake, 1, 2, fake,
                             fake, 1 << 20, nul) == E   # f64 A with f32 U
    assert lib.cnmf_gaussian(0, 0, -1, 3, 1, fake, nul) == E
    assert lib.cnmf_sketch_pass(fake, 1, 10, 10, 10, 0, fake, nul, fake, nul,
                                fake, 1 << 20, nul, nul) == E


def test_workspace_queries(lib):
    assert lib.cnmf_compress_workspace(100, 80, 10, 1) > 0
    assert lib.cnmf_compress_workspace(100, 80, 200, 1) == 0
    assert lib.cnmf_factor_state_bytes(100, 80, 5, 10, 1) == \
        ((100 * 5 + 80 * 5 + 2 * 5 * 10) * 4 + 7) // 8 * 8 + 8 + \
        (2 * 5 * 5 * 4 + 7) // 8 * 8
    assert lib.snmf_select_workspace(100, 80, 10, 2) > 0
    assert lib.cnmf_plain_state_bytes(100, 80, 5, 0) == \
        (2 * 100 * 5 + 2 * 80 * 5) * 8 + 8


def test_thread_cta_limit_rejects_negative(lib):
    assert lib.cnmf_set_thread_cta_limit(-1) == 1   # CNMF_E_INVALID_ARG
    assert lib.cnmf_set_thread_cta_limit(0) == 0


def test_right_factor_invalid_arguments(lib):
    E = 1
    fake = C.c_void_p(16)
    ok = dict(n=100, d=10, ld=10, r=4, sweeps=10, tol=1e-6, ldy=100)
    def call(**kw):
        a = dict(ok, **kw)
        return lib.snmf_right_factor(fake, 1, a["n"], a["d"], a["ld"], fake,
                                     a["r"], a["sweeps"], a["tol"], fake,
                                     a["ldy"], None, fake, 1 << 30, None, None)
    assert call(r=11) == E           # r > d
    assert call(r=65, d=70, ld=70) == E
    assert call(sweeps=0) == E
    assert call(tol=-1.0) == E
    assert call(ld=9) == E
    assert call(ldy=99) == E
    assert call(d=129, ld=129) == E
    assert lib.snmf_right_factor(None, 1, 100, 10, 10, fake, 4, 10, 1e-6, fake,
                                 100, None, fake, 1 << 30, None, None) == E
    assert lib.snmf_right_factor_workspace(100, 10, 11, 1) == 0


def test_als_and_gaussian_compression_invalid_arguments(lib):
    E = 1
    f = C.c_void_p(16)
    # cnmf_factor_als(A, a_type, m, n, lda, L, Rt, r, d, iters, sweeps, tol,
    #                 X, Y, unconverged, ws, ws_bytes, status, stream)
    def als(**kw):
        a = dict(m=100, n=80, lda=80, r=4, d=10, iters=2, sweeps=10, tol=1e-6)
        a.update(kw)
        return lib.cnmf_factor_als(f, 1, a["m"], a["n"], a["lda"], f, f, a["r"],
                                   a["d"], a["iters"], a["sweeps"], a["tol"], f,
                                   f, None, f, 1 << 30, None, None)
    assert als(r=11) == E            # r > d
    assert als(d=81, r=4) == E       # d > n
    assert als(lda=79) == E
    assert als(iters=-1) == E
    assert als(sweeps=0) == E
    assert als(tol=-1.0) == E
    assert lib.cnmf_factor_als_workspace(100, 80, 11, 10, 1) == 0
    # cnmf_factor_mu(A, a_type, m, n, lda, L, Rt, r, d, iters, X, Y, ws,
    #                ws_bytes, status, stream)
    def mu(**kw):
        a = dict(m=100, n=80, lda=80, r=4, d=10, iters=2)
        a.update(kw)
        return lib.cnmf_factor_mu(f, 1, a["m"], a["n"], a["lda"], f, f, a["r"],
                                  a["d"], a["iters"], f, f, f, 1 << 30, None,
                                  None)
    assert mu(r=11) == E
    assert mu(d=81, r=4) == E
    assert mu(lda=79) == E
    assert mu(iters=-1) == E
    assert mu(r=65, d=70) == E
    assert lib.cnmf_factor_mu_workspace(100, 80, 11, 10, 1) == 0
    # cnmf_compress_host(A, a_type, m, n, lda, r, d, q, seed, Omega, Psi, L,
    #                    Rt, Atilde, block_rows, ws, ws_bytes, status, stream)
    def ch(**kw):
        a = dict(m=100, n=80, lda=80, r=4, d=10, q=2, blk=16)
        a.update(kw)
        return lib.cnmf_compress_host(f, 1, a["m"], a["n"], a["lda"], a["r"],
                                      a["d"], a["q"], 1, None, None, f, f, f,
                                      a["blk"], f, 1 << 30, None, None)
    assert ch(blk=0) == E
    assert ch(lda=79) == E
    assert ch(d=81) == E
    assert ch(r=11) == E
    assert ch(q=-1) == E
    assert lib.cnmf_compress_host_workspace(100, 80, 10, 1, 0) == 0
    assert lib.cnmf_compress_host_workspace(100, 80, 10, 1, 16) > 0
    assert lib.cnmf_compress_host(f, 1, 100, 80, 80, 4, 10, 2, 1, None, None,
                                  f, f, f, 16, f, 16, None, None) == 2
    assert lib.cnmf_factor_mu_workspace(100, 80, 4, 10, 1) == \
        lib.cnmf_factor_als_workspace(100, 80, 4, 10, 1)
    # cnmf_compress_gaussian(A, a_type, m, n, lda, d, seed, L, Rt, Atilde,
    #                        ws, ws_bytes, status, stream)
    assert lib.cnmf_compress_gaussian(f, 1, 100, 80, 80, 0, 1, f, f, f, f,
                                      1 << 30, None, None) == E
    assert lib.cnmf_compress_gaussian(f, 1, 100, 80, 80, 81, 1, f, f, f, f,
                                      1 << 30, None, None) == E
    assert lib.cnmf_compress_gaussian(None, 1, 100, 80, 80, 8, 1, f, f, f, f,
                                      1 << 30, None, None) == E
    assert lib.cnmf_compress_gaussian(f, 1, 100, 80, 80, 8, 1, f, f, f, f,
                                      16, None, None) == 2   # CNMF_E_WORKSPACE


def test_check_nonnegative_invalid_arguments(lib):
    """The negative-entry check rejects NULL pointers, unknown types, empty
    shapes and a pitch below n on the host (no GPU work)."""
    c = C.c_void_p
    a, st = c(0x1000), c(0x2000)
    f = lib.cnmf_check_nonnegative
    assert f(c(0), 1, 10, 10, 10, st, None) == 1
    assert f(a, 1, 10, 10, 10, c(0), None) == 1
    assert f(a, 9, 10, 10, 10, st, None) == 1
    assert f(a, 1, 0, 10, 10, st, None) == 1
    assert f(a, 1, 10, 0, 10, st, None) == 1
    assert f(a, 1, 10, 10, 9, st, None) == 1


def test_status_flag_bits_are_not_error_codes():
    """The flag bit lies above the error-code mask, and every error code
    fits inside it."""
    from paper_1505_04650_gb300 import _lib as L
    assert L.CNMF_STATUS_NEGATIVE_A & L.CNMF_STATUS_CODE_MASK == 0
    for code in (L.CNMF_E_INVALID_ARG, L.CNMF_E_WORKSPACE, L.CNMF_E_CUDA,
                 L.CNMF_E_CHOLESKY, L.CNMF_E_NONFINITE, L.CNMF_E_TIMEOUT):
        assert code & ~L.CNMF_STATUS_CODE_MASK == 0
    h = open(os.path.join(ROOT, "include", "cnmf.h")).read()
    assert "#define CNMF_STATUS_NEGATIVE_A 0x40000000" in h
    assert "#define CNMF_STATUS_CODE_MASK 0x0000FFFF" in h
