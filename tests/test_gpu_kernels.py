"""GPU parity of the building blocks against the FP64 oracle / definitions.

Every call goes through the C ABI (ctypes binding).  Tolerances:
* integer work (Philox words, anchors): bit-exact;
* products with A: the componentwise rounding bound of a length-s dot
  product, |Z - Z_exact| <= (s + 2) u (|A| |X|), u = 2^-53 (FP64); FP32 and
  BF16 A run on the tensor cores with FP32 accumulation (2u per add, u =
  2^-24) plus the operand-split residual (bf16 hi + lo of X: 2^-17; 3xTF32:
  2^-19) -- holds at any size;
* orthonormal bases: unique thin Q (positive diag R) elementwise, with a
  tolerance scaled by u and the panel's condition number.
"""
import numpy as np
import pytest

import synth
from oracle import compress as ocomp
from oracle import philox as ophil
from oracle import residual as ores

from gpu_util import need_gpu, product_bound, rel, to_dev, to_np, unit, wdt

pytestmark = pytest.mark.gpu


def test_philox_words_bitwise():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    for seed, stream, first, nb in [(0, 0, 0, 1000), (2003, 1, 77, 513),
                                    ((1 << 40) + 5, 0, (1 << 33) - 3, 64)]:
        g = cn.cnmf_philox_words(seed, stream, first, nb)
        got = g.cpu().numpy().view(np.uint32)
        ref = ophil.raw_words(seed, stream, nb, first_block=first)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_gaussian_matches_oracle(dtype):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    for rows, cols in [(1, 1), (7, 5), (1001, 30)]:
        z = to_np(cn.cnmf_gaussian(2001, 1, rows, cols, dtype=wdt(dtype)))
        ref = ophil.gaussian_matrix(2001, 1, rows, cols)
        if dtype == "f64":
            assert np.abs(z - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
        else:
            assert np.abs(z - ref).max() <= 2 * 2.0 ** -24 * np.abs(ref).max()


CASES = [  # m, n, k  (n % 4 == 0: FP32 rows 16-byte aligned, tensor cores)
    (1, 1, 1), (37, 53, 5), (300, 257, 30), (129, 4100, 16), (5000, 33, 20),
    (640, 700, 60), (200, 300, 80), (150, 170, 128), (1000, 1028, 30),
    (257, 516, 128), (4100, 260, 48), (3, 8, 2)]


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n,k", CASES)
def test_sketch_pass_products(storage, m, n, k):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    A64 = synth.lowrank(m, n, min(5, m, n), 0.01, 11)
    As = synth.as_storage(A64, storage)
    Aw = synth.widen(As, storage)
    g = np.random.default_rng(3)
    X = g.standard_normal((n, k))
    Y = g.standard_normal((m, k))
    if storage != "f64":
        X = X.astype(np.float32).astype(np.float64)
        Y = Y.astype(np.float32).astype(np.float64)
    Ad = to_dev(As, storage)
    Xd = torch.tensor(X, dtype=wdt(storage)).cuda()
    Yd = torch.tensor(Y, dtype=wdt(storage)).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Zm, Zn = cn.cnmf_sketch_pass(Ad, Xd, Yd, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref_m = Aw @ X
    bnd_m = product_bound(storage, n) * (np.abs(Aw) @ np.abs(X))
    ref_n = Aw.T @ Y
    bnd_n = product_bound(storage, m) * (np.abs(Aw).T @ np.abs(Y))
    assert np.all(np.abs(to_np(Zm) - ref_m) <= bnd_m + 1e-300)
    assert np.all(np.abs(to_np(Zn) - ref_n) <= bnd_n + 1e-300)


def test_sketch_pass_pitched_and_one_sided():
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    m, n, k = 333, 211, 12
    big = synth.as_storage(synth.lowrank(m, n + 9, 4, 0.01, 5), "f32")
    Ad = to_dev(big, "f32")[:, :n]               # lda = n + 9 > n
    A = big[:, :n].astype(np.float64)
    X = np.random.default_rng(1).standard_normal((n, k)).astype(np.float32)
    Zm, Zn = cn.cnmf_sketch_pass(Ad, torch.tensor(X).cuda(), None)
    assert Zn is None
    bnd = product_bound("f32", n) * (np.abs(A) @ np.abs(X.astype(np.float64)))
    assert np.all(np.abs(to_np(Zm) - A @ X) <= bnd)


def _planted(rows, k, kappa, seed):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((rows, k)))
    V, _ = np.linalg.qr(g.standard_normal((k, k)))
    s = np.geomspace(1.0, 1.0 / kappa, k)
    return (Q * s) @ V.T


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("rows,k,kappa", [(50, 1, 1.0), (97, 7, 10.0),
                                          (3000, 30, 1e3), (20000, 30, 1e4),
                                          (1000, 80, 1e2), (700, 128, 10.0),
                                          (400, 45, 1e2), (2000, 60, 1e3),
                                          (500, 90, 10.0)])
def test_orth_unique_q(storage, rows, k, kappa):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    Y = _planted(rows, k, kappa, rows + k)
    if storage == "f32":
        Y = Y.astype(np.float32).astype(np.float64)
    Yd = torch.tensor(Y, dtype=wdt(storage)).cuda()
    Qd, st = cn.cnmf_orth(Yd)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Q = to_np(Qd)
    Qo = ocomp.orth(Y)
    u = unit(storage)
    assert np.linalg.norm(Q.T @ Q - np.eye(k)) <= 50 * k * u
    assert np.abs(Q - Qo).max() <= 50 * k * u * kappa


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n,r", [(1, 1, 1), (70, 90, 3), (513, 300, 20),
                                   (64, 4097, 7)])
def test_residual(storage, m, n, r):
    torch = need_gpu()
    import paper_1505_04650_gb300 as cn
    As = synth.as_storage(synth.lowrank(m, n, r, 0.05, 2), storage)
    Aw = synth.widen(As, storage)
    U0, V0 = synth.init_factors(m, n, r, 4)
    w = wdt(storage)
    Ud = torch.tensor(U0, dtype=w).cuda()
    Vtd = torch.tensor(V0.T.copy(), dtype=w).cuda()
    U = to_np(Ud)
    V = to_np(Vtd).T
    out = cn.cnmf_residual(to_dev(As, storage), Ud, Vtd).cpu().numpy()
    e2, a2 = ores.residual_sq(Aw, U, V)
    tol = 1e-12 if storage == "f64" else 2e-5
    assert abs(out[1] - a2) <= tol * a2
    assert abs(out[0] - e2) <= tol * a2 * 50


def test_barrier_timeout_returns_status():
    torch = need_gpu()
    import ctypes as C
    from paper_1505_04650_gb300 import _lib
    lib = _lib.load()
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rounds = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    ctas = min(16, nsm)
    # every CTA arrives: 50 barriers pass, status OK
    assert lib.cnmf_barrier_selftest(ctas, 50, -1, 1000, C.c_void_p(ws.data_ptr()),
                                     256, C.c_void_p(st.data_ptr()),
                                     C.c_void_p(rounds.data_ptr()), s) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(rounds.item()) == 50
    # CTA 3 never arrives: the others give up after ~100 ms with TIMEOUT
    import time
    t0 = time.time()
    assert lib.cnmf_barrier_selftest(ctas, 5, 3, 100, C.c_void_p(ws.data_ptr()),
                                     256, C.c_void_p(st.data_ptr()),
                                     C.c_void_p(rounds.data_ptr()), s) == 0
    torch.cuda.synchronize()
    assert time.time() - t0 < 5.0
    assert int(st.item()) == 6  # CNMF_E_TIMEOUT
    assert int(rounds.item()) == 0
    # the context is still usable
    x = torch.ones(10, device="cuda").sum()
    assert float(x) == 10.0


def test_tagwait_timeout_returns_status():
    torch = need_gpu()
    import ctypes as C
    from paper_1505_04650_gb300 import _lib
    lib = _lib.load()
    ws = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rounds = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    ctas = min(16, nsm)
    # every CTA publishes: 200 rounds through two buffers, status OK
    assert lib.cnmf_tagwait_selftest(ctas, 200, -1, 1000, C.c_void_p(ws.data_ptr()),
                                     4096, C.c_void_p(st.data_ptr()),
                                     C.c_void_p(rounds.data_ptr()), s) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(rounds.item()) == 200
    # CTA 3 never publishes: its neighbours give up after ~100 ms with
    # TIMEOUT, the abort flag releases everyone else
    import time
    st.zero_()
    t0 = time.time()
    assert lib.cnmf_tagwait_selftest(ctas, 20, 3, 100, C.c_void_p(ws.data_ptr()),
                                     4096, C.c_void_p(st.data_ptr()),
                                     C.c_void_p(rounds.data_ptr()), s) == 0
    torch.cuda.synchronize()
    assert time.time() - t0 < 5.0
    assert int(st.item()) == 6  # CNMF_E_TIMEOUT
    assert int(rounds.item()) < 20
    x = torch.ones(10, device="cuda").sum()
    assert float(x) == 10.0
