"""GPU parity of the fused two-sided sketch pass (one read of A gives both
A X and A^T Y; Alg. 1 power scheme on A and A^T, Sec. III).

Both products are compared entry by entry with the exact product of the
values the GPU reads (FP64 matmul of the widened A and the FP32 panels),
within the rounding bound of a length-s dot product with FP32 accumulation
plus the operand-split residual (see gpu_util.product_bound: bf16 hi + lo
of the FP32 panels, and of FP32 A, which the converter warps split in
shared memory).  The shapes
exercise the tile walk of the fused kernel: ragged 128-tiles on both sides,
more tile columns than one group of A^T Y accumulators holds, rows and
column runs split between CTAs, and CTA caps from 1 CTA upwards (long ranges
that span many row blocks and groups).
"""
import numpy as np
import pytest

import synth

from gpu_util import need_gpu, product_bound, to_dev, to_np

pytestmark = pytest.mark.gpu

SHAPES = [  # m, n, k   (n % 8 == 0: rows 16-byte aligned for BF16 and FP32)
    (1, 8, 1), (130, 136, 5), (128, 128, 16), (300, 2056, 30),
    (2000, 3000, 32), (5003, 264, 20), (129, 4104, 16), (777, 1536, 31),
    (4096, 4096, 30)]


def _case(m, n, k, storage, seed):
    A64 = synth.lowrank(m, n, min(5, m, n), 0.01, seed)
    As = synth.as_storage(A64, storage)
    Aw = synth.widen(As, storage)
    g = np.random.default_rng(seed + 1)
    X = g.standard_normal((n, k)).astype(np.float32).astype(np.float64)
    Y = g.standard_normal((m, k)).astype(np.float32).astype(np.float64)
    return As, Aw, X, Y


def _check(Aw, X, Y, Zm, Zn, storage):
    m, n = Aw.shape
    bm = product_bound(storage, n) * (np.abs(Aw) @ np.abs(X))
    bn = product_bound(storage, m) * (np.abs(Aw).T @ np.abs(Y))
    em = np.abs(to_np(Zm) - Aw @ X)
    en = np.abs(to_np(Zn) - Aw.T @ Y)
    assert np.all(em <= bm + 1e-300), float((em / (bm + 1e-300)).max())
    assert np.all(en <= bn + 1e-300), float((en / (bn + 1e-300)).max())


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_fused_pass_matches_exact_products(storage, m, n, k):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    As, Aw, X, Y = _case(m, n, k, storage, 100 + m + n + k)
    Ad = to_dev(As, storage)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Zm, Zn = cn.cnmf_sketch_pass(Ad, torch.tensor(X, dtype=torch.float32).cuda(),
                                 torch.tensor(Y, dtype=torch.float32).cuda(),
                                 status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    _check(Aw, X, Y, Zm, Zn, storage)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("side", ["x", "y"])
@pytest.mark.parametrize("m,n,k", [(300, 2056, 30), (5003, 264, 20),
                                   (2000, 3000, 32), (129, 4104, 16)])
def test_fused_one_sided_matches_exact_product(storage, side, m, n, k):
    """A X alone (A-check = A R^T) and A^T Y alone: one group spans every
    column when A^T Y is left out; A^T Y alone keeps more accumulators."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    As, Aw, X, Y = _case(m, n, k, storage, 300 + m + k)
    Ad = to_dev(As, storage)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Xd = torch.tensor(X, dtype=torch.float32).cuda() if side == "x" else None
    Yd = torch.tensor(Y, dtype=torch.float32).cuda() if side == "y" else None
    Zm, Zn = cn.cnmf_sketch_pass(Ad, Xd, Yd, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    if side == "x":
        assert Zn is None
        b = product_bound(storage, n) * (np.abs(Aw) @ np.abs(X))
        e = np.abs(to_np(Zm) - Aw @ X)
    else:
        assert Zm is None
        b = product_bound(storage, m) * (np.abs(Aw).T @ np.abs(Y))
        e = np.abs(to_np(Zn) - Aw.T @ Y)
    assert np.all(e <= b + 1e-300), float((e / (b + 1e-300)).max())


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("ctas", [1, 3, 7, 40])
def test_fused_pass_under_cta_caps(storage, ctas):
    """Few CTAs: each range spans many rows, groups and row blocks."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, k = 1100, 2600, 30
    As, Aw, X, Y = _case(m, n, k, storage, 7 + ctas)
    Ad = to_dev(As, storage)
    Xd = torch.tensor(X, dtype=torch.float32).cuda()
    Yd = torch.tensor(Y, dtype=torch.float32).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    cn.set_thread_cta_limit(ctas)
    try:
        Zm, Zn = cn.cnmf_sketch_pass(Ad, Xd, Yd, status=st)
        torch.cuda.synchronize()
    finally:
        cn.set_thread_cta_limit(0)
    assert int(st.item()) == 0
    _check(Aw, X, Y, Zm, Zn, storage)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_fused_pass_is_deterministic(storage):
    """Partials are summed in a fixed order: repeated calls agree bitwise."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, k = 3000, 2000, 30
    As, Aw, X, Y = _case(m, n, k, storage, 55)
    Ad = to_dev(As, storage)
    Xd = torch.tensor(X, dtype=torch.float32).cuda()
    Yd = torch.tensor(Y, dtype=torch.float32).cuda()
    Zm0, Zn0 = cn.cnmf_sketch_pass(Ad, Xd, Yd)
    for _ in range(3):
        Zm, Zn = cn.cnmf_sketch_pass(Ad, Xd, Yd)
        torch.cuda.synchronize()
        assert torch.equal(Zm, Zm0) and torch.equal(Zn, Zn0)
    _check(Aw, X, Y, Zm0, Zn0, storage)


def test_fused_pass_pitched_fp32():
    """A with a row pitch larger than n (lda = n + 8)."""
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, k = 700, 1000, 24
    big = synth.as_storage(synth.lowrank(m, n + 8, 4, 0.01, 9), "f32")
    Ad = to_dev(big, "f32")[:, :n]
    Aw = big[:, :n].astype(np.float64)
    g = np.random.default_rng(2)
    X = g.standard_normal((n, k)).astype(np.float32).astype(np.float64)
    Y = g.standard_normal((m, k)).astype(np.float32).astype(np.float64)
    Zm, Zn = cn.cnmf_sketch_pass(Ad, torch.tensor(X, dtype=torch.float32).cuda(),
                                 torch.tensor(Y, dtype=torch.float32).cuda())
    torch.cuda.synchronize()
    _check(Aw, X, Y, Zm, Zn, "f32")
