"""Serving scheduler host logic on the CPU: the device calls are replaced
by fakes, so this checks admission, eviction, batching and completion
without a GPU."""
import sys
import types

import numpy as np
import pytest

from paper_2510_08230_gb300 import workloads as W


class _FakeTensor:
    def __init__(self, a):
        self.a = np.asarray(a)

    def to(self, *a, **k):
        return self

    def cpu(self):
        return self

    def numpy(self):
        return self.a


class _FakeTorch(types.ModuleType):
    float64 = "f64"

    def __init__(self):
        super().__init__("torch")
        cuda = types.SimpleNamespace()
        cuda.set_device = lambda d: None

        class Stream:
            def __init__(self, device=None, priority=0):
                self.priority = priority

            @staticmethod
            def priority_range():
                return 0, -1

        class stream:
            def __init__(self, s):
                pass

            def __enter__(self):
                return self

            def __exit__(self, *a):
                return False

        cuda.Stream, cuda.stream = Stream, stream
        self.cuda = cuda

    @staticmethod
    def device(s):
        return s

    @staticmethod
    def from_numpy(a):
        return _FakeTensor(a)

    @staticmethod
    def zeros(n, dtype=None, device=None):
        return _FakeTensor(np.zeros(n))


@pytest.fixture()
def fake_server(monkeypatch):
    import paper_2510_08230_gb300.serve as sv

    class FakeMat:
        made = []

        def __init__(self, m):
            self.m, self.handle, self.closed = m, 1, False
            FakeMat.made.append(self)

        def close(self):
            self.closed = True

        def solve(self, b, x, stream, **kw):
            return {"return": 0, "status": 0, "iters": 1}

    monkeypatch.setattr(sv, "Matrix", types.SimpleNamespace(from_csr=lambda m, dt: FakeMat(m)))
    monkeypatch.setattr(sv, "gk_solve_batched",
                        lambda hs, bs, xs, o, s, tols=None: (0, [{"status": 0} for _ in hs]))
    monkeypatch.setitem(sys.modules, "torch", _FakeTorch())
    return sv, FakeMat


def _reqs(sv, pool, params):
    return [sv.SolveRequest(i, mi, pool[mi], np.ones(pool[mi].n), tol, prec)
            for i, (mi, prec, tol, seed) in enumerate(params)]


def test_admission_respects_budget_and_everything_completes(fake_server):
    sv, FakeMat = fake_server
    pool = W.serving_pool(10, seed=77, n_lo=500, n_hi=60000, max_nnz=2_000_000)
    reqs = _reqs(sv, pool, W.serving_requests(pool, 60, seed=9))
    budget = 1.5 * max(sv.matrix_bytes(r.m, True) + sv.request_bytes(r, 16384) for r in reqs)
    srv = sv.SolveServer(budget_bytes=budget, workers=4)
    peak = [0.0]
    orig = srv._admit

    def watched():
        orig()
        peak[0] = max(peak[0], srv.used)

    srv._admit = watched
    for r in reqs:
        srv.submit(r)
    assert all(r.event.wait(30) for r in reqs)
    srv.close()
    assert srv.error is None
    assert peak[0] <= budget
    assert all(r.info["status"] == 0 for r in reqs)
    assert any(m.closed for m in FakeMat.made)  # the tight budget forced evictions


def test_small_systems_are_batched_while_workers_are_busy(fake_server):
    sv, _ = fake_server
    pool = [W.laplacian_2d(20), W.laplacian_2d(30), W.laplacian_3d(12)]
    params = [(i % 3, "f64", 1e-10, i) for i in range(24)]
    reqs = _reqs(sv, pool, params)
    srv = sv.SolveServer(budget_bytes=1e9, workers=1)
    with srv.cv:  # hold the dispatcher while the burst arrives
        for r in reqs:
            r.t_submit = 0.0
            srv.queue.append(r)
    assert all(r.event.wait(30) for r in reqs)
    srv.close()
    assert all(r.batched for r in reqs)
    assert max(r.info["batch"] for r in reqs) >= 2  # launched together


def test_refined_and_large_requests_run_alone(fake_server):
    sv, _ = fake_server
    big = W.laplacian_2d(200)  # 40000 rows > small_n
    reqs = [sv.SolveRequest(0, 0, big, np.ones(big.n), 1e-8, "f64"),
            sv.SolveRequest(1, 1, W.laplacian_2d(10), np.ones(100), 1e-8, "ir32")]
    srv = sv.SolveServer(budget_bytes=1e9, workers=2)
    for r in reqs:
        srv.submit(r)
    assert all(r.event.wait(30) for r in reqs)
    srv.close()
    assert not reqs[0].batched and not reqs[1].batched


def test_ilu_and_block_jacobi_requests_run_alone_and_count_their_factors(fake_server):
    """The batched engine runs no ILU(0) or block-Jacobi: small requests with
    them go to gk_solve alone, and an ILU(0) request charges the factors to
    the cached matrix once."""
    sv, _ = fake_server
    m = W.laplacian_2d(12)
    reqs = [sv.SolveRequest(0, 0, m, np.ones(m.n), 1e-8, "f64", precond="ilu"),
            sv.SolveRequest(1, 1, m, np.ones(m.n), 1e-8, "f64", precond="block_jacobi"),
            sv.SolveRequest(2, 2, m, np.ones(m.n), 1e-8, "f64", precond="jacobi"),
            sv.SolveRequest(3, 0, m, np.ones(m.n), 1e-8, "f64", precond="ilu")]
    srv = sv.SolveServer(budget_bytes=1e9, workers=2)
    for r in reqs:
        srv.submit(r)
    assert all(r.event.wait(30) for r in reqs)
    cached = dict(srv.cache)
    srv.close()
    assert not reqs[0].batched and not reqs[1].batched and not reqs[3].batched
    assert reqs[2].batched
    want = sv.matrix_bytes(m, False) + sv.ilu_bytes(m, False)
    assert cached[0][1] == want and cached[0][4]  # charged once for both ILU requests
    assert cached[2][1] == sv.matrix_bytes(m, False) and not cached[2][4]


def test_long_solves_use_their_own_lane_and_short_ones_pass_them(fake_server):
    """Solves expected to run long go to the long lane (at most long_workers
    at a time); short solves submitted behind them are served by the short
    lane while the long ones still run; observed solve times replace the
    size-based estimate."""
    import threading
    sv, FakeMat = fake_server
    gate = threading.Event()
    running_long = []
    peak_long = [0]

    def solve(self, b, x, stream, **kw):
        if self.m.n > 100000:
            running_long.append(1)
            peak_long[0] = max(peak_long[0], len(running_long))
            gate.wait(10)
            running_long.pop()
        return {"return": 0, "status": 0, "iters": 1}

    FakeMat.solve = solve
    big = W.laplacian_2d(800)      # expected above long_s
    mid = W.laplacian_2d(150)      # 22500 rows: not batched, expected short
    srv = sv.SolveServer(budget_bytes=1e12, workers=4, long_workers=2, long_s=0.02)
    assert srv.expected_seconds(sv.SolveRequest(0, 0, big, np.ones(big.n))) > 0.02
    assert srv.expected_seconds(sv.SolveRequest(0, 1, mid, np.ones(mid.n))) < 0.02
    longs = [srv.submit(sv.SolveRequest(i, 0, big, np.ones(big.n))) for i in range(4)]
    shorts = [srv.submit(sv.SolveRequest(10 + i, 1, mid, np.ones(mid.n))) for i in range(6)]
    assert all(r.event.wait(10) for r in shorts)  # done while the long ones are held
    assert not any(r.event.is_set() for r in longs)
    assert peak_long[0] <= 2
    gate.set()
    assert all(r.event.wait(30) for r in longs)
    assert srv.cost[(1, "f64")] < 0.02  # learned from the served solves
    srv.close()
    assert srv.error is None
