"""GB300-native compressed NMF / SNMF (Tepper & Sapiro, arXiv 1505.04650).

Thin PyTorch-facing binding over the C ABI of ``libcnmf.so`` (see
include/cnmf.h).  Each function only marshals arguments: it checks dtypes,
shapes and devices, allocates outputs and the workspace with PyTorch on the
tensors' CUDA device, and calls the entry point of the same name on the
current CUDA stream.  Every step of the method runs in the library's CUDA
kernels; if the library is missing the import of a function raises.

Storage dtypes: float64 (FP64 path), float32, bfloat16 (A only; arithmetic
in FP32).  Tall panels are row-major with the long dimension first
(L m x d, Rt = R^T n x d, Vt = V^T n x r).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import AdmmParams

__all__ = [
    "CnmfError", "lib", "cnmf_gaussian", "cnmf_philox_words",
    "cnmf_sketch_pass", "cnmf_orth", "cnmf_compress", "cnmf_factor",
    "cnmf_factor_plain", "snmf_select", "cnmf_residual", "FactorState",
    "sketch_size", "default_penalty", "BatchProblem", "cnmf_factor_batched",
    "set_thread_cta_limit", "snmf_right_factor", "cnmf_compress_gaussian",
    "cnmf_factor_als", "cnmf_factor_mu", "cnmf_compress_host",
]


class CnmfError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        msg = lib().cnmf_status_string(self.code).decode()
        if self.code == _lib.CNMF_E_CUDA:
            msg += " -- " + lib().cnmf_last_error().decode()
        super().__init__(f"{where}: {msg}")


def lib():
    return _lib.load()


_DT = {torch.float64: _lib.CNMF_F64, torch.float32: _lib.CNMF_F32,
       torch.bfloat16: _lib.CNMF_BF16}


def _wdtype(a_dtype: torch.dtype) -> torch.dtype:
    return torch.float64 if a_dtype == torch.float64 else torch.float32


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(dev):
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _check(code: int, where: str):
    if code != _lib.CNMF_OK:
        raise CnmfError(code, where)


def _mat(A: torch.Tensor, name: str = "A"):
    if A.dim() != 2 or A.dtype not in _DT or not A.is_cuda:
        raise ValueError(f"{name} must be a 2-D CUDA float64/float32/bfloat16 tensor")
    if A.stride(1) != 1 or A.stride(0) < A.shape[1]:
        raise ValueError(f"{name} must be row-major with unit column stride")
    return A.shape[0], A.shape[1], A.stride(0)


def _dense(t: torch.Tensor, shape, dtype, name):
    if tuple(t.shape) != tuple(shape) or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name}: expected contiguous {dtype} {tuple(shape)}, "
                         f"got {t.dtype} {tuple(t.shape)}")
    return t


def _ws(nbytes: int, dev) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)


def _status(dev):
    return torch.zeros(1, dtype=torch.int32, device=dev)


def raise_on_status(status: torch.Tensor, where: str):
    """Synchronising check of a device status word (first error wins; the
    flag bits, which are not errors, are ignored)."""
    code = int(status.item()) & _lib.CNMF_STATUS_CODE_MASK
    if code != _lib.CNMF_OK:
        raise CnmfError(code, where)


def has_negative_entries(status: torch.Tensor) -> bool:
    """Synchronising read of the flag that cnmf_check_nonnegative sets."""
    return bool(int(status.item()) & _lib.CNMF_STATUS_NEGATIVE_A)


def cnmf_check_nonnegative(A: torch.Tensor,
                           status: torch.Tensor | None = None):
    """ORs the negative-entry flag into the status word if A holds an entry
    below zero (NMF assumes A >= 0, Sec. II); returns the status word."""
    m, n, lda = _mat(A)
    st = status if status is not None else _status(A.device)
    _check(lib().cnmf_check_nonnegative(_ptr(A), _DT[A.dtype], m, n, lda,
                                        _ptr(st), _stream(A.device)),
           "cnmf_check_nonnegative")
    return st


def sketch_size(r: int, r_ov: int, n: int) -> int:
    """The paper's rule d = min(max(20, r + r_ov), n) (Sec. V)."""
    return min(max(20, r + r_ov), n)


def default_penalty(Atilde: torch.Tensor, r: int) -> float:
    """lambda = phi = ||Atilde||_F / r (the balanced reading of Alg. 4's
    unspecified penalties; a host-side scalar from the compressed matrix)."""
    return float(torch.linalg.norm(Atilde.double())) / r


def set_thread_cta_limit(ctas: int):
    """Cap the per-SM grids of this host thread's later calls at `ctas` CTAs
    (0: the whole device), so two calls on two streams can share the SMs."""
    _check(lib().cnmf_set_thread_cta_limit(int(ctas)), "cnmf_set_thread_cta_limit")


# --------------------------------------------------------------------------
def cnmf_gaussian(seed: int, stream_id: int, rows: int, cols: int,
                  dtype=torch.float32, device="cuda") -> torch.Tensor:
    out = torch.empty(rows, cols, dtype=dtype, device=device)
    _check(lib().cnmf_gaussian(seed, stream_id, rows, cols, _DT[dtype],
                               _ptr(out), _stream(out.device)), "cnmf_gaussian")
    return out


def cnmf_philox_words(seed: int, stream_id: int, first_block: int,
                      nblocks: int, device="cuda") -> torch.Tensor:
    """Raw Philox4x32-10 output words, nblocks x 4 (int32 bit patterns)."""
    out = torch.empty(nblocks, 4, dtype=torch.int32, device=device)
    _check(lib().cnmf_philox_words(seed, stream_id, first_block, nblocks,
                                   _ptr(out), _stream(out.device)),
           "cnmf_philox_words")
    return out


def cnmf_sketch_pass(A: torch.Tensor, X: torch.Tensor | None = None,
                     Y: torch.Tensor | None = None,
                     status: torch.Tensor | None = None):
    """(A X, A^T Y) with one read of A per product; either may be None."""
    m, n, lda = _mat(A)
    w = _wdtype(A.dtype)
    k = (X if X is not None else Y).shape[1]
    if X is not None:
        _dense(X, (n, k), w, "X")
    if Y is not None:
        _dense(Y, (m, k), w, "Y")
    Zm = torch.empty(m, k, dtype=w, device=A.device) if X is not None else None
    Zn = torch.empty(n, k, dtype=w, device=A.device) if Y is not None else None
    L = lib()
    nb = L.cnmf_sketch_workspace(m, n, k, _DT[A.dtype])
    ws = _ws(nb, A.device)
    _check(L.cnmf_sketch_pass(_ptr(A), _DT[A.dtype], m, n, lda, k, _ptr(X),
                              _ptr(Y), _ptr(Zm), _ptr(Zn), _ptr(ws), nb,
                              _ptr(status), _stream(A.device)),
           "cnmf_sketch_pass")
    return Zm, Zn


def cnmf_orth(Y: torch.Tensor, status: torch.Tensor | None = None):
    """In-place orthonormal basis of a tall panel (CholeskyQR2)."""
    rows, k = Y.shape
    if Y.dtype not in (torch.float64, torch.float32) or not Y.is_contiguous():
        raise ValueError("Y must be contiguous float64/float32")
    st = status if status is not None else _status(Y.device)
    L = lib()
    nb = L.cnmf_orth_workspace(rows, k, _DT[Y.dtype])
    ws = _ws(nb, Y.device)
    _check(L.cnmf_orth(_ptr(Y), _DT[Y.dtype], rows, k, _ptr(ws), nb, _ptr(st),
                       _stream(Y.device)), "cnmf_orth")
    return Y, st


def cnmf_compress(A: torch.Tensor, r: int, d: int, q: int, seed: int,
                  Omega: torch.Tensor | None = None,
                  Psi: torch.Tensor | None = None,
                  status: torch.Tensor | None = None, ws=None):
    """Two-sided compression -> (L m x d, Rt n x d, Atilde d x d, status)."""
    m, n, lda = _mat(A)
    w = _wdtype(A.dtype)
    if Omega is not None:
        _dense(Omega, (n, d), w, "Omega")
    if Psi is not None:
        _dense(Psi, (m, d), w, "Psi")
    dev = A.device
    Lm = torch.empty(m, d, dtype=w, device=dev)
    Rt = torch.empty(n, d, dtype=w, device=dev)
    At = torch.empty(d, d, dtype=w, device=dev)
    st = status if status is not None else _status(dev)
    L = lib()
    nb = L.cnmf_compress_workspace(m, n, d, _DT[A.dtype])
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    _check(L.cnmf_compress(_ptr(A), _DT[A.dtype], m, n, lda, r, d, q, seed,
                           _ptr(Omega), _ptr(Psi), _ptr(Lm), _ptr(Rt),
                           _ptr(At), _ptr(ws), ws.numel(), _ptr(st),
                           _stream(dev)), "cnmf_compress")
    return Lm, Rt, At, st


def cnmf_compress_host(A: torch.Tensor, r: int, d: int, q: int, seed: int,
                       block_rows: int, device="cuda",
                       Omega: torch.Tensor | None = None,
                       Psi: torch.Tensor | None = None,
                       status: torch.Tensor | None = None, ws=None):
    """Two-sided compression of an A that stays outside device memory (a
    CPU tensor, ideally pinned; a CUDA tensor is accepted too), streamed
    through the GPU in blocks of `block_rows` rows -> (L, Rt, Atilde,
    status) on `device`."""
    if A.dim() != 2 or A.dtype not in _DT or A.stride(1) != 1 or \
            A.stride(0) < A.shape[1]:
        raise ValueError("A must be a 2-D row-major float64/float32/bfloat16 "
                         "tensor with unit column stride")
    m, n, lda = A.shape[0], A.shape[1], A.stride(0)
    dev = torch.device(device)
    w = _wdtype(A.dtype)
    if Omega is not None:
        _dense(Omega, (n, d), w, "Omega")
    if Psi is not None:
        _dense(Psi, (m, d), w, "Psi")
    Lm = torch.empty(m, d, dtype=w, device=dev)
    Rt = torch.empty(n, d, dtype=w, device=dev)
    At = torch.empty(d, d, dtype=w, device=dev)
    st = status if status is not None else _status(dev)
    L = lib()
    nb = L.cnmf_compress_host_workspace(m, n, d, _DT[A.dtype], block_rows)
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    _check(L.cnmf_compress_host(_ptr(A), _DT[A.dtype], m, n, lda, r, d, q,
                                seed, _ptr(Omega), _ptr(Psi), _ptr(Lm),
                                _ptr(Rt), _ptr(At), block_rows, _ptr(ws),
                                ws.numel(), _ptr(st), _stream(dev)),
           "cnmf_compress_host")
    return Lm, Rt, At, st


def cnmf_compress_gaussian(A: torch.Tensor, d: int, seed: int,
                           status: torch.Tensor | None = None, ws=None):
    """Gaussian-compression baseline -> (L m x d, Rt n x d, Atilde, status):
    L = d^-1/2 Psi, R^T = d^-1/2 Omega (no power iteration or QR)."""
    m, n, lda = _mat(A)
    w = _wdtype(A.dtype)
    dev = A.device
    Lm = torch.empty(m, d, dtype=w, device=dev)
    Rt = torch.empty(n, d, dtype=w, device=dev)
    At = torch.empty(d, d, dtype=w, device=dev)
    st = status if status is not None else _status(dev)
    L = lib()
    nb = L.cnmf_compress_workspace(m, n, d, _DT[A.dtype])
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    _check(L.cnmf_compress_gaussian(_ptr(A), _DT[A.dtype], m, n, lda, d, seed,
                                    _ptr(Lm), _ptr(Rt), _ptr(At), _ptr(ws),
                                    ws.numel(), _ptr(st), _stream(dev)),
           "cnmf_compress_gaussian")
    return Lm, Rt, At, st


@dataclass
class FactorState:
    """Resumable ADMM state (device buffer in the ABI's layout)."""
    buf: torch.Tensor
    m: int
    n: int
    r: int
    d: int          # 0 for the plain (uncompressed) baseline
    dtype: torch.dtype

    def _sections(self):
        e = 8 if self.dtype == torch.float64 else 4
        m, n, r, d = self.m, self.n, self.r, self.d
        if self.d:
            sizes = [("Lam", (m, r)), ("Phit", (n, r)), ("Yt", (r, d)),
                     ("Xt", (d, r))]
        else:
            sizes = [("Lam", (m, r)), ("Phit", (n, r)), ("Yt", (n, r)),
                     ("X", (m, r))]
        out, off = {}, 0
        for name, shp in sizes:
            cnt = shp[0] * shp[1]
            out[name] = self.buf[off:off + cnt * e].view(self.dtype).view(*shp)
            off += cnt * e
        if self.d:
            # int64 k at the next 8-byte boundary, then the two kept r x r
            # inverses of the ADMM solves
            off = (off + 7) // 8 * 8
            out["k"] = self.buf[off:off + 8].view(torch.int64)
            out["Z"] = self.buf[off + 8:off + 8 + 2 * r * r * e] \
                .view(self.dtype).view(2, r, r)
        else:
            out["k"] = self.buf[self.buf.numel() - 8:].view(torch.int64)
        return out

    def __getattr__(self, name):
        if name in ("Lam", "Phit", "Yt", "Xt", "X", "k"):
            return self._sections()[name]
        raise AttributeError(name)


def cnmf_factor(L: torch.Tensor, Rt: torch.Tensor, Atilde: torch.Tensor,
                U: torch.Tensor, Vt: torch.Tensor, lam: float, phi: float,
                iters: int, xi: float = 1.0, state: FactorState | None = None,
                status: torch.Tensor | None = None,
                barrier_timeout_ms: int = 0, ws=None,
                phase_ns: torch.Tensor | None = None):
    """`iters` sweeps of compressed ADMM (Alg. 4); U (m x r), Vt (n x r)
    are updated in place.  Returns (U, Vt, state, status).  `phase_ns`
    (optional float64[5] on the device) accumulates per-phase times."""
    m, d = L.shape
    n = Rt.shape[0]
    r = U.shape[1]
    w = L.dtype
    for t, shp, nm in ((L, (m, d), "L"), (Rt, (n, d), "Rt"),
                       (Atilde, (d, d), "Atilde"), (U, (m, r), "U"),
                       (Vt, (n, r), "Vt")):
        _dense(t, shp, w, nm)
    dev = L.device
    lb = lib()
    resume = 1
    if state is None:
        nbs = lb.cnmf_factor_state_bytes(m, n, r, d, _DT[w])
        state = FactorState(torch.zeros(nbs, dtype=torch.uint8, device=dev),
                            m, n, r, d, w)
        resume = 0
    st = status if status is not None else _status(dev)
    nb = lb.cnmf_factor_workspace(m, n, r, d, _DT[w])
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    p = AdmmParams(lam, phi, xi, iters, barrier_timeout_ms,
                   None if phase_ns is None else phase_ns.data_ptr(),
                   0 if phase_ns is None else phase_ns.numel(), 0)
    _check(lb.cnmf_factor(_ptr(L), _ptr(Rt), _ptr(Atilde), _DT[w], m, n, r, d,
                          C.byref(p), _ptr(U), _ptr(Vt), _ptr(state.buf),
                          resume, _ptr(ws), ws.numel(), _ptr(st),
                          _stream(dev)), "cnmf_factor")
    return U, Vt, state, st


def cnmf_factor_plain(A: torch.Tensor, U: torch.Tensor, Vt: torch.Tensor,
                      lam: float, phi: float, iters: int, xi: float = 1.0,
                      state: FactorState | None = None,
                      status: torch.Tensor | None = None, ws=None):
    """Uncompressed ADMM NMF baseline (Alg. 4 with L = I, R = I)."""
    m, n, lda = _mat(A)
    w = _wdtype(A.dtype)
    r = U.shape[1]
    _dense(U, (m, r), w, "U")
    _dense(Vt, (n, r), w, "Vt")
    dev = A.device
    lb = lib()
    resume = 1
    if state is None:
        nbs = lb.cnmf_plain_state_bytes(m, n, r, _DT[A.dtype])
        state = FactorState(torch.zeros(nbs, dtype=torch.uint8, device=dev),
                            m, n, r, 0, w)
        resume = 0
    st = status if status is not None else _status(dev)
    nb = lb.cnmf_plain_workspace(m, n, r, _DT[A.dtype])
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    p = AdmmParams(lam, phi, xi, iters, 0, None, 0, 0)
    _check(lb.cnmf_factor_plain(_ptr(A), _DT[A.dtype], m, n, lda, r,
                                C.byref(p), _ptr(U), _ptr(Vt),
                                _ptr(state.buf), resume, _ptr(ws), ws.numel(),
                                _ptr(st), _stream(dev)), "cnmf_factor_plain")
    return U, Vt, state, st


def snmf_select(A: torch.Tensor, r: int, d: int, q: int, seed: int,
                Omega: torch.Tensor | None = None, return_rhat: bool = False,
                status: torch.Tensor | None = None, ws=None):
    """Alg. 3 steps 1-2 -> anchors (int64[r], selection order) [, Rhat_t]."""
    m, n, lda = _mat(A)
    w = _wdtype(A.dtype)
    dev = A.device
    if Omega is not None:
        _dense(Omega, (n, d), w, "Omega")
    anchors = torch.empty(r, dtype=torch.int64, device=dev)
    rh = torch.empty(n, d, dtype=w, device=dev) if return_rhat else None
    st = status if status is not None else _status(dev)
    lb = lib()
    nb = lb.snmf_select_workspace(m, n, d, _DT[A.dtype])
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    _check(lb.snmf_select(_ptr(A), _DT[A.dtype], m, n, lda, r, d, q, seed,
                          _ptr(Omega), _ptr(anchors), _ptr(rh), _ptr(ws),
                          ws.numel(), _ptr(st), _stream(dev)), "snmf_select")
    return (anchors, rh, st) if return_rhat else (anchors, st)


def snmf_right_factor(Rhat_t: torch.Tensor, anchors: torch.Tensor,
                      max_sweeps: int = 1000, tol: float = 1e-6,
                      status: torch.Tensor | None = None, ws=None):
    """Alg. 3 step 3 -> (Y r x n, unconverged int32[1], status): the
    nonnegative least-squares fit of every column of Rhat by the columns
    `anchors` (Rhat_t n x d as snmf_select returns it)."""
    n, d = Rhat_t.shape
    w = Rhat_t.dtype
    if w not in (torch.float32, torch.float64):
        raise ValueError(f"Rhat_t: expected float32 or float64, got {w}")
    _dense(Rhat_t, (n, d), w, "Rhat_t")
    if anchors.dtype != torch.int64 or not anchors.is_contiguous() \
            or anchors.device != Rhat_t.device or anchors.dim() != 1:
        raise ValueError("anchors: expected a contiguous int64 vector on "
                         "Rhat_t's device")
    r = anchors.numel()
    dev = Rhat_t.device
    Y = torch.empty(r, n, dtype=w, device=dev)
    unconv = torch.zeros(1, dtype=torch.int32, device=dev)
    st = status if status is not None else _status(dev)
    lb = lib()
    nb = lb.snmf_right_factor_workspace(n, d, r, _DT[w])
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    _check(lb.snmf_right_factor(_ptr(Rhat_t), _DT[w], n, d, d, _ptr(anchors),
                                r, max_sweeps, tol, _ptr(Y), n, _ptr(unconv),
                                _ptr(ws), ws.numel(), _ptr(st), _stream(dev)),
           "snmf_right_factor")
    return Y, unconv, st


def cnmf_factor_als(A: torch.Tensor, L: torch.Tensor, Rt: torch.Tensor,
                    Y0: torch.Tensor, iters: int, max_sweeps: int = 1000,
                    tol: float = 1e-6, status: torch.Tensor | None = None,
                    ws=None):
    """Alg. 2 with exact NNLS steps -> (X m x r, Y r x n, unconverged,
    status); Y0 (r x n) is the start (copied, not modified)."""
    m, n, lda = _mat(A)
    w = _wdtype(A.dtype)
    d = L.shape[1]
    r = Y0.shape[0]
    _dense(L, (m, d), w, "L")
    _dense(Rt, (n, d), w, "Rt")
    _dense(Y0, (r, n), w, "Y0")
    dev = A.device
    X = torch.empty(m, r, dtype=w, device=dev)
    Y = Y0.clone()
    unconv = torch.zeros(1, dtype=torch.int32, device=dev)
    st = status if status is not None else _status(dev)
    lb = lib()
    nb = lb.cnmf_factor_als_workspace(m, n, r, d, _DT[A.dtype])
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    _check(lb.cnmf_factor_als(_ptr(A), _DT[A.dtype], m, n, lda, _ptr(L),
                              _ptr(Rt), r, d, iters, max_sweeps, tol, _ptr(X),
                              _ptr(Y), _ptr(unconv), _ptr(ws), ws.numel(),
                              _ptr(st), _stream(dev)), "cnmf_factor_als")
    return X, Y, unconv, st


def cnmf_factor_mu(A: torch.Tensor, L: torch.Tensor, Rt: torch.Tensor,
                   X0: torch.Tensor, Y0: torch.Tensor, iters: int,
                   status: torch.Tensor | None = None, ws=None):
    """Alg. 2 with multiplicative-update steps -> (X m x r, Y r x n,
    status); X0 (m x r) and Y0 (r x n) are the start (copied)."""
    m, n, lda = _mat(A)
    w = _wdtype(A.dtype)
    d = L.shape[1]
    r = Y0.shape[0]
    _dense(L, (m, d), w, "L")
    _dense(Rt, (n, d), w, "Rt")
    _dense(X0, (m, r), w, "X0")
    _dense(Y0, (r, n), w, "Y0")
    dev = A.device
    X = X0.clone()
    Y = Y0.clone()
    st = status if status is not None else _status(dev)
    lb = lib()
    nb = lb.cnmf_factor_mu_workspace(m, n, r, d, _DT[A.dtype])
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    _check(lb.cnmf_factor_mu(_ptr(A), _DT[A.dtype], m, n, lda, _ptr(L),
                             _ptr(Rt), r, d, iters, _ptr(X), _ptr(Y),
                             _ptr(ws), ws.numel(), _ptr(st), _stream(dev)),
           "cnmf_factor_mu")
    return X, Y, st


def cnmf_residual(A: torch.Tensor, U: torch.Tensor, Vt: torch.Tensor,
                  out: torch.Tensor | None = None, ws=None) -> torch.Tensor:
    """Device FP64 pair (||A - U V||^2, ||A||^2)."""
    m, n, lda = _mat(A)
    w = _wdtype(A.dtype)
    r = U.shape[1]
    _dense(U, (m, r), w, "U")
    _dense(Vt, (n, r), w, "Vt")
    dev = A.device
    out = out if out is not None else torch.empty(2, dtype=torch.float64,
                                                  device=dev)
    lb = lib()
    nb = lb.cnmf_residual_workspace(m, n, r, _DT[A.dtype])
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    _check(lb.cnmf_residual(_ptr(A), _DT[A.dtype], m, n, lda, _ptr(U),
                            _ptr(Vt), _DT[w], r, _ptr(out), _ptr(ws),
                            ws.numel(), _stream(dev)), "cnmf_residual")
    return out


def residual_item_bytes(A: torch.Tensor, U: torch.Tensor,
                        Vt: torch.Tensor) -> bytes:
    """Host image of one cnmf_residual_item (for cnmf_residual_batched)."""
    m, n, lda = _mat(A)
    r = U.shape[1]
    w = _wdtype(A.dtype)
    _dense(U, (m, r), w, "U")
    _dense(Vt, (n, r), w, "Vt")
    return bytes(_lib.ResidualItem(A.data_ptr(), U.data_ptr(), Vt.data_ptr(),
                                   m, n, lda, r, 0))


def cnmf_residual_batched(items_dev: torch.Tensor, nitems: int,
                          a_dtype: torch.dtype, max_r: int,
                          ctas_per_item: int = 8,
                          out: torch.Tensor | None = None, ws=None,
                          status: torch.Tensor | None = None) -> torch.Tensor:
    """(nitems, 2) device FP64 pairs (||A - U V||^2, ||A||^2), one launch for
    all items; items_dev holds nitems cnmf_residual_item records (device
    memory, e.g. copied from residual_item_bytes images)."""
    dev = items_dev.device
    lb = lib()
    if out is None:
        out = torch.empty(nitems, 2, dtype=torch.float64, device=dev)
    nb = lb.cnmf_residual_batched_workspace(nitems, ctas_per_item)
    if ws is None or ws.numel() < nb:
        ws = _ws(nb, dev)
    _check(lb.cnmf_residual_batched(_ptr(items_dev), nitems, _DT[a_dtype],
                                    _DT[_wdtype(a_dtype)], max_r,
                                    ctas_per_item, _ptr(out), _ptr(ws),
                                    ws.numel(), _ptr(status), _stream(dev)),
           "cnmf_residual_batched")
    return out


# --------------------------------------------------------------------------
class BatchProblem:
    """Device buffers of one problem for cnmf_factor_batched (FP32).

    Holds L, Rt, Atilde (from cnmf_compress), U, Vt (in/out), the resumable
    state and the scratch the batched kernel keeps between launches."""

    def __init__(self, L, Rt, Atilde, U, Vt, lam, phi, xi=1.0):
        m, d = L.shape
        n = Rt.shape[0]
        r = U.shape[1]
        for t, shp, nm in ((L, (m, d), "L"), (Rt, (n, d), "Rt"),
                           (Atilde, (d, d), "Atilde"), (U, (m, r), "U"),
                           (Vt, (n, r), "Vt")):
            _dense(t, shp, torch.float32, nm)
        lb = lib()
        self.L, self.Rt, self.Atilde, self.U, self.Vt = L, Rt, Atilde, U, Vt
        self.m, self.n, self.r, self.d = m, n, r, d
        self.lam, self.phi, self.xi = float(lam), float(phi), float(xi)
        nbs = lb.cnmf_factor_state_bytes(m, n, r, d, _lib.CNMF_F32)
        self.state = FactorState(torch.zeros(nbs, dtype=torch.uint8,
                                             device=L.device), m, n, r, d,
                                 torch.float32)
        self.scratch = torch.zeros(lb.cnmf_batch_scratch_bytes(r, d),
                                   dtype=torch.uint8, device=L.device)
        self.fresh = True

    def item(self) -> "_lib.BatchItem":
        p = lambda t: t.data_ptr()
        return _lib.BatchItem(p(self.L), p(self.Rt), p(self.Atilde), p(self.U),
                              p(self.Vt), p(self.state.buf), p(self.scratch),
                              self.m, self.n, self.r, self.d, self.lam,
                              self.phi, self.xi,
                              _lib.CNMF_BATCH_FRESH if self.fresh else 0, 0)

    def item_bytes(self) -> bytes:
        """Host image of item(), kept until the penalties or the FRESH flag
        change (building the ctypes record costs more than a round's GPU
        work when many problems are in flight)."""
        key = (self.fresh, self.lam, self.phi, self.xi)
        if getattr(self, "_item_key", None) != key:
            self._item_bytes = bytes(self.item())
            self._item_key = key
        return self._item_bytes


def pack_items(problems) -> bytes:
    """Host image of a cnmf_batch_item array (None -> empty slot)."""
    arr = (_lib.BatchItem * max(1, len(problems)))()
    for i, pb in enumerate(problems):
        if pb is not None:
            arr[i] = pb.item()
    return bytes(arr)


def cnmf_factor_batched(problems, sweeps: int, cluster_size: int = 1,
                        items_dev: torch.Tensor | None = None,
                        status: torch.Tensor | None = None,
                        max_r: int | None = None, max_d: int | None = None):
    """`sweeps` compressed ADMM sweeps for every problem in one launch.

    `problems` is a list of BatchProblem (or None for an empty slot).  The
    item array is copied to `items_dev` (a device uint8 tensor, allocated if
    None) before the launch; after it every problem's fresh flag is
    cleared.  Returns (items_dev, status)."""
    live = [p for p in problems if p is not None]
    if not live:
        return items_dev, status
    dev = live[0].L.device
    img = pack_items(problems)
    if items_dev is None or items_dev.numel() < len(img):
        items_dev = torch.empty(len(img), dtype=torch.uint8, device=dev)
    host = torch.frombuffer(bytearray(img), dtype=torch.uint8)
    items_dev[:len(img)].copy_(host, non_blocking=False)
    st = status if status is not None else _status(dev)
    mr = max_r or max(p.r for p in live)
    md = max_d or max(p.d for p in live)
    _check(lib().cnmf_factor_batched(_ptr(items_dev), len(problems), sweeps,
                                     cluster_size, mr, md, _ptr(st),
                                     _stream(dev)), "cnmf_factor_batched")
    for p in live:
        p.fresh = False
    return items_dev, st
