"""Host logic of the serving loop and the autotuner, without a GPU: the
request stream (workload 4: Poisson arrivals, m, n ~ U[200, 4000],
r ~ U{5..32}, d = r + 10), the per-request device-memory estimate used by
admission, and the autotuner's size buckets."""
import numpy as np

from paper_1505_04650_gb300 import serve
from paper_1505_04650_gb300.autotune import bucket


def test_workload_shape_and_reproducibility():
    a = serve.make_workload(2000, 500.0, seed=3)
    b = serve.make_workload(2000, 500.0, seed=3)
    assert [(x.m, x.n, x.r, x.t_arrive) for x in a] == \
           [(x.m, x.n, x.r, x.t_arrive) for x in b]
    m = np.array([x.m for x in a]); n = np.array([x.n for x in a])
    r = np.array([x.r for x in a]); d = np.array([x.d for x in a])
    assert m.min() >= 200 and m.max() <= 4000 and n.min() >= 200 and n.max() <= 4000
    assert r.min() >= 5 and r.max() <= 32 and np.all(d == r + 10)
    t = np.array([x.t_arrive for x in a])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    # Poisson process: mean gap 1 / rate within 5 standard errors
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 500.0) <= 5 * (1 / 500.0) / np.sqrt(len(gaps))
    # distinct seeds per request, all requests at t = 0 without a rate
    assert len({x.seed for x in a}) == len(a)
    z = serve.make_workload(10, 0.0)
    assert all(x.t_arrive == 0.0 for x in z)


def test_request_bytes_counts_every_resident_buffer():
    rq = serve.Request(0, 0.0, m=1000, n=800, r=10, d=20)
    e = 4
    expect = (1000 * 800 + (1000 + 800) * 20 + 20 * 20
              + 2 * (1000 + 800) * 10 + 2 * 2 * 10 * 20) * e + 1024
    assert serve.request_bytes(rq) == expect
    big = serve.Request(1, 0.0, m=2000, n=800, r=10, d=20)
    assert serve.request_bytes(big) > serve.request_bytes(rq)


def test_autotune_buckets():
    assert bucket(1, 1, 1, 1) == "m1024_n1024_r16_d32"
    assert bucket(1024, 1025, 16, 33) == "m1024_n2048_r16_d64"
    assert bucket(3000, 200, 20, 30) == bucket(2100, 1, 17, 31)



def test_capture_gate_excludes_admissions():
    """The serving thread's graph capture (exclusive) never overlaps an
    admission thread's CUDA work (shared); a waiting capture holds back new
    admissions, and several admissions run together."""
    import threading
    import time
    from paper_1505_04650_gb300.serve import _CaptureGate
    gate = _CaptureGate()
    log, lock = [], threading.Lock()
    inside = {"shared": 0, "excl": 0, "max_shared": 0, "overlap": False}

    def admit(k):
        with gate.shared():
            with lock:
                inside["shared"] += 1
                inside["max_shared"] = max(inside["max_shared"],
                                           inside["shared"])
                inside["overlap"] |= inside["excl"] > 0
            time.sleep(0.05)
            with lock:
                inside["shared"] -= 1
                log.append(("a", k))

    def capture():
        with gate.exclusive():
            with lock:
                inside["excl"] += 1
                inside["overlap"] |= inside["shared"] > 0
            time.sleep(0.05)
            with lock:
                inside["excl"] -= 1
                log.append(("c", 0))

    ts = [threading.Thread(target=admit, args=(k,)) for k in range(3)]
    for t in ts:
        t.start()
    time.sleep(0.01)
    tc = threading.Thread(target=capture)
    tc.start()
    time.sleep(0.01)
    late = threading.Thread(target=admit, args=(9,))   # arrives while the
    late.start()                                       # capture waits
    for t in ts + [tc, late]:
        t.join(timeout=10)
    assert not inside["overlap"]
    assert inside["max_shared"] >= 2
    # the capture ran before the late admission
    assert log.index(("c", 0)) < log.index(("a", 9))
