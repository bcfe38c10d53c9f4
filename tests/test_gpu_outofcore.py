"""GPU parity of out-of-core compression (cnmf_compress_host): A stays in
host memory (or, to exercise the block path on in-HBM data, device memory)
and is streamed through the GPU in row blocks once per pass.

* FP64 A: L and R^T elementwise against cnmf_compress on the same A and
  against the FP64 oracle (the unique thin Q of full-rank sketches), 1e-9;
* FP32 / BF16 A: the rank-r signal projectors of L and R^T against
  cnmf_compress's and against the oracle's, 1e-5 (summation order is all
  that differs from the in-HBM path); on a planted well-conditioned input
  the full projector L L^T against the oracle's, 1e-5;
* ragged blocks (block sizes that do not divide m), one-row blocks, and a
  block larger than A.
"""
import numpy as np
import pytest

import synth
from oracle import compress as ocomp
from oracle import philox as ophil

from gpu_util import need_gpu, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def _basis(L, A, r):
    W, _, _ = np.linalg.svd(L.T @ A, full_matrices=False)
    return L @ W[:, :r]


def _pdist(U1, U2):
    r = U2.shape[1]
    return float(np.sqrt(2.0) * np.linalg.norm(U1 - U2 @ (U2.T @ U1)) / np.sqrt(r))


def _host(As, storage, pinned=True):
    import torch
    t = to_dev(As, storage).cpu()
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("block_rows", [123, 500, 37])
def test_host_fp64_matches_device_and_oracle(block_rows):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, r, d, q = 500, 400, 10, 20, 4
    A = synth.lowrank(m, n, r, 0.01, 1000 + block_rows)
    Ah = _host(A, "f64")
    L, Rt, At, st = cn.cnmf_compress_host(Ah, r, d, q, 2000, block_rows)
    Ld, Rtd, Atd, _ = cn.cnmf_compress(to_dev(A, "f64"), r, d, q, 2000)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Om, Ps = ophil.test_matrices(2000, m, n, d)
    L0, Rt0, _, At0 = ocomp.compress(A, Om, Ps, q)
    for got in (to_np(L), ):
        assert np.abs(got - to_np(Ld)).max() <= 1e-9
        assert np.abs(got - L0).max() <= 1e-9
    assert np.abs(to_np(Rt) - to_np(Rtd)).max() <= 1e-9
    assert np.abs(to_np(Rt) - Rt0).max() <= 1e-9
    assert np.abs(to_np(At) - At0).max() <= 1e-9 * np.abs(At0).max()


@pytest.mark.parametrize("storage,block_rows,pinned", [("f32", 777, True),
                                                        ("f32", 3000, False),
                                                        ("bf16", 1024, True),
                                                        ("f32", 5000, True)])
def test_host_fp32_bf16_signal_projector(storage, block_rows, pinned):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, r, d, q = 3000, 2000, 20, 30, 3
    As = synth.as_storage(synth.lowrank(m, n, r, 0.01, 77), storage)
    Aw = synth.widen(As, storage)
    L, Rt, At, st = cn.cnmf_compress_host(_host(As, storage, pinned), r, d, q,
                                          2077, block_rows)
    Ld, Rtd, _, _ = cn.cnmf_compress(to_dev(As, storage), r, d, q, 2077)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Om, Ps = ophil.test_matrices(2077, m, n, d)
    L0, Rt0, _, _ = ocomp.compress(Aw, Om, Ps, q)
    Lg, Rg = to_np(L), to_np(Rt)
    bl, br = _basis(Lg, Aw, r), _basis(Rg, Aw.T, r)
    e_dev = max(_pdist(bl, _basis(to_np(Ld), Aw, r)),
                _pdist(br, _basis(to_np(Rtd), Aw.T, r)))
    e_or = max(_pdist(bl, _basis(L0, Aw, r)), _pdist(br, _basis(Rt0, Aw.T, r)))
    print(f"{storage} blocks of {block_rows}: vs device {e_dev:.2e}, vs oracle {e_or:.2e}")
    assert e_dev <= 1e-5 and e_or <= 1e-5
    assert np.abs(Lg.T @ Lg - np.eye(d)).max() <= 1e-5


def test_block_path_on_device_memory_planted_projector():
    """A in device memory forced through the block path (a device pointer
    is accepted): the full projector on a planted well-conditioned input
    (sigma_1 / sigma_d = 10, gap 1e3) against the oracle, 1e-5."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, d, q = 1500, 1100, 24, 2
    g = np.random.default_rng(5)
    U, _ = np.linalg.qr(g.standard_normal((m, d + 5)))
    V, _ = np.linalg.qr(g.standard_normal((n, d + 5)))
    s = np.concatenate([np.geomspace(100.0, 10.0, d), np.full(5, 0.01)])
    A = ((U * s) @ V.T).astype(np.float32)
    Aw = A.astype(np.float64)
    L, Rt, _, st = cn.cnmf_compress_host(to_dev(A, "f32"), d, d, q, 31, 400)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Om, Ps = ophil.test_matrices(31, m, n, d)
    L0, Rt0, _, _ = ocomp.compress(Aw, Om, Ps, q)
    assert rel(to_np(L) @ to_np(L).T, L0 @ L0.T) <= 1e-5
    assert rel(to_np(Rt) @ to_np(Rt).T, Rt0 @ Rt0.T) <= 1e-5


def test_host_one_row_blocks():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, r, d, q = 37, 64, 3, 8, 1
    A = synth.lowrank(m, n, r, 0.05, 9).astype(np.float32)
    L, Rt, _, st = cn.cnmf_compress_host(_host(A, "f32"), r, d, q, 5, 1)
    Ld, Rtd, _, _ = cn.cnmf_compress(to_dev(A, "f32"), r, d, q, 5)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Aw = A.astype(np.float64)
    assert _pdist(_basis(to_np(L), Aw, r), _basis(to_np(Ld), Aw, r)) <= 1e-5
