"""ctypes declarations of the C ABI in include/cnmf.h (argument marshalling only).

The library is the in-tree ``libcnmf.so`` built by ``build.py`` for sm_103a.
Loading fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcnmf.so")

c_void_p, c_size_t, c_int32, c_int64, c_uint32, c_uint64, c_double = (
    C.c_void_p, C.c_size_t, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64,
    C.c_double)

# status codes and storage types (cnmf.h)
CNMF_OK, CNMF_E_INVALID_ARG, CNMF_E_WORKSPACE, CNMF_E_CUDA = 0, 1, 2, 3
CNMF_E_CHOLESKY, CNMF_E_NONFINITE, CNMF_E_TIMEOUT = 4, 5, 6
# bits of the device status word: error code low, flags (not errors) high
CNMF_STATUS_CODE_MASK = 0x0000FFFF
CNMF_STATUS_NEGATIVE_A = 0x40000000
CNMF_F64, CNMF_F32, CNMF_BF16 = 0, 1, 2


class AdmmParams(C.Structure):
    _fields_ = [("lambda_", c_double), ("phi", c_double), ("xi", c_double),
                ("iters", c_int32), ("barrier_timeout_ms", c_int32),
                ("phase_ns", c_void_p), ("phase_ns_len", c_int32),
                ("reserved", c_int32)]


CNMF_BATCH_FRESH = 1


class BatchItem(C.Structure):
    """cnmf_batch_item (include/cnmf.h)."""
    _fields_ = [("L", c_void_p), ("Rt", c_void_p), ("Atilde", c_void_p),
                ("U", c_void_p), ("Vt", c_void_p), ("state", c_void_p),
                ("scratch", c_void_p), ("m", c_int64), ("n", c_int64),
                ("r", c_int32), ("d", c_int32), ("lambda_", c_double),
                ("phi", c_double), ("xi", c_double), ("flags", c_int32),
                ("reserved", c_int32)]


class ResidualItem(C.Structure):
    """cnmf_residual_item (include/cnmf.h)."""
    _fields_ = [("A", c_void_p), ("U", c_void_p), ("Vt", c_void_p),
                ("m", c_int64), ("n", c_int64), ("lda", c_int64),
                ("r", c_int32), ("reserved", c_int32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "cnmf_status_string": (C.c_char_p, [c_int32]),
    "cnmf_abi_version": (c_int32, []),
    "cnmf_last_error": (C.c_char_p, []),
    "cnmf_gaussian": (c_int32, [c_uint64, c_uint32, c_int64, c_int64, c_int32,
                                c_void_p, c_void_p]),
    "cnmf_philox_words": (c_int32, [c_uint64, c_uint32, c_int64, c_int64,
                                    c_void_p, c_void_p]),
    "cnmf_sketch_workspace": (c_size_t, [c_int64, c_int64, c_int32, c_int32]),
    "cnmf_sketch_pass": (c_int32, [c_void_p, c_int32, c_int64, c_int64,
                                   c_int64, c_int32, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_size_t,
                                   c_void_p, c_void_p]),
    "cnmf_orth_workspace": (c_size_t, [c_int64, c_int32, c_int32]),
    "cnmf_orth": (c_int32, [c_void_p, c_int32, c_int64, c_int32, c_void_p,
                            c_size_t, c_void_p, c_void_p]),
    "cnmf_compress_workspace": (c_size_t, [c_int64, c_int64, c_int32,
                                           c_int32]),
    "cnmf_compress": (c_int32, [c_void_p, c_int32, c_int64, c_int64, c_int64,
                                c_int32, c_int32, c_int32, c_uint64, c_void_p,
                                c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_size_t, c_void_p, c_void_p]),
    "cnmf_compress_host_workspace": (c_size_t, [c_int64, c_int64, c_int32,
                                                c_int32, c_int64]),
    "cnmf_compress_host": (c_int32, [c_void_p, c_int32, c_int64, c_int64,
                                     c_int64, c_int32, c_int32, c_int32,
                                     c_uint64, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_int64, c_void_p,
                                     c_size_t, c_void_p, c_void_p]),
    "cnmf_factor_workspace": (c_size_t, [c_int64, c_int64, c_int32, c_int32,
                                         c_int32]),
    "cnmf_factor_state_bytes": (c_size_t, [c_int64, c_int64, c_int32, c_int32,
                                           c_int32]),
    "cnmf_factor": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int64,
                              c_int64, c_int32, c_int32, C.POINTER(AdmmParams),
                              c_void_p, c_void_p, c_void_p, c_int32, c_void_p,
                              c_size_t, c_void_p, c_void_p]),
    "cnmf_plain_workspace": (c_size_t, [c_int64, c_int64, c_int32, c_int32]),
    "cnmf_plain_state_bytes": (c_size_t, [c_int64, c_int64, c_int32,
                                          c_int32]),
    "cnmf_factor_plain": (c_int32, [c_void_p, c_int32, c_int64, c_int64,
                                    c_int64, c_int32, C.POINTER(AdmmParams),
                                    c_void_p, c_void_p, c_void_p, c_int32,
                                    c_void_p, c_size_t, c_void_p, c_void_p]),
    "snmf_select_workspace": (c_size_t, [c_int64, c_int64, c_int32, c_int32]),
    "snmf_select": (c_int32, [c_void_p, c_int32, c_int64, c_int64, c_int64,
                              c_int32, c_int32, c_int32, c_uint64, c_void_p,
                              c_void_p, c_void_p, c_void_p, c_size_t,
                              c_void_p, c_void_p]),
    "cnmf_compress_gaussian": (c_int32, [c_void_p, c_int32, c_int64, c_int64,
                                         c_int64, c_int32, c_uint64, c_void_p,
                                         c_void_p, c_void_p, c_void_p,
                                         c_size_t, c_void_p, c_void_p]),
    "cnmf_factor_als_workspace": (c_size_t, [c_int64, c_int64, c_int32,
                                             c_int32, c_int32]),
    "cnmf_factor_als": (c_int32, [c_void_p, c_int32, c_int64, c_int64, c_int64,
                                  c_void_p, c_void_p, c_int32, c_int32,
                                  c_int32, c_int32, c_double, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_size_t,
                                  c_void_p, c_void_p]),
    "cnmf_factor_mu_workspace": (c_size_t, [c_int64, c_int64, c_int32,
                                            c_int32, c_int32]),
    "cnmf_factor_mu": (c_int32, [c_void_p, c_int32, c_int64, c_int64, c_int64,
                                 c_void_p, c_void_p, c_int32, c_int32, c_int32,
                                 c_void_p, c_void_p, c_void_p, c_size_t,
                                 c_void_p, c_void_p]),
    "snmf_right_factor_workspace": (c_size_t, [c_int64, c_int32, c_int32,
                                               c_int32]),
    "snmf_right_factor": (c_int32, [c_void_p, c_int32, c_int64, c_int32,
                                    c_int64, c_void_p, c_int32, c_int32,
                                    c_double, c_void_p, c_int64, c_void_p,
                                    c_void_p, c_size_t, c_void_p, c_void_p]),
    "cnmf_residual_workspace": (c_size_t, [c_int64, c_int64, c_int32,
                                           c_int32]),
    "cnmf_residual": (c_int32, [c_void_p, c_int32, c_int64, c_int64, c_int64,
                                c_void_p, c_void_p, c_int32, c_int32,
                                c_void_p, c_void_p, c_size_t, c_void_p]),
    "cnmf_residual_batched_workspace": (c_size_t, [c_int32, c_int32]),
    "cnmf_residual_batched": (c_int32, [c_void_p, c_int32, c_int32, c_int32,
                                        c_int32, c_int32, c_void_p, c_void_p,
                                        c_size_t, c_void_p, c_void_p]),
    "cnmf_check_nonnegative": (c_int32, [c_void_p, c_int32, c_int64,
                                         c_int64, c_int64, c_void_p,
                                         c_void_p]),
    "cnmf_residual_noalloc": (c_int32, [c_void_p, c_int32, c_int64, c_int64,
                                        c_int64, c_void_p, c_void_p, c_int32,
                                        c_int32, c_void_p, c_void_p]),
    "cnmf_batch_scratch_bytes": (c_size_t, [c_int32, c_int32]),
    "cnmf_factor_batched": (c_int32, [c_void_p, c_int32, c_int32, c_int32,
                                      c_int32, c_int32, c_void_p, c_void_p]),
    "cnmf_barrier_selftest": (c_int32, [c_int32, c_int32, c_int32, c_int32,
                                        c_void_p, c_size_t, c_void_p,
                                        c_void_p, c_void_p]),
    "cnmf_tagwait_selftest": (c_int32, [c_int32, c_int32, c_int32, c_int32,
                                        c_void_p, c_size_t, c_void_p,
                                        c_void_p, c_void_p]),
    "cnmf_set_thread_cta_limit": (c_int32, [c_int32]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libcnmf.so and declare every entry point (raises if missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with "
            "`python -m paper_1505_04650_gb300.build` (needs nvcc); "
            "there is no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
