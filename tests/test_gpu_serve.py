"""Serving loop: continuous batching under a memory budget; each result is
the same alone and in the mix (the scheduler only changes when and with
whom a system runs, never its arithmetic), and meets its tolerance."""
import numpy as np
import pytest

import oracle
from paper_2510_08230_gb300 import workloads as W
from gpu_util import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.fixture(scope="module")
def pool():
    return W.serving_pool(10, seed=77, n_lo=500, n_hi=60000, max_nnz=2_000_000)


def _requests(pool, params):
    from paper_2510_08230_gb300.serve import SolveRequest
    reqs = []
    for rid, (mi, prec, tol, seed) in enumerate(params):
        m = pool[mi]
        b = W.uniform_vector(m.n, seed)
        reqs.append(SolveRequest(rid, mi, m, b, tol=tol, precision=prec))
    return reqs


def test_alone_equals_mix_and_meets_tolerance(pool):
    from paper_2510_08230_gb300.serve import SolveServer
    params = W.serving_requests(pool, 36, seed=5)
    srv = SolveServer(budget_bytes=4e9, workers=3)
    mix = _requests(pool, params)
    for r in mix:
        srv.submit(r)
    for r in mix:
        assert r.event.wait(300)
    alone = _requests(pool, params)
    for r in alone:
        srv.submit(r)
        assert r.event.wait(300)
    srv.close()
    assert any(r.info["batch"] > 1 for r in mix), "no request was batched with another"
    for a, b in zip(mix, alone):
        assert a.info["status"] == 0 and b.info["status"] == 0, (a.info, b.info)
        assert np.array_equal(a.x, b.x), (a.rid, a.info, b.info)
        assert oracle.true_rel_residual(a.m, a.b, a.x) <= a.tol * 1.0000001


def test_budget_is_respected(pool):
    from paper_2510_08230_gb300.serve import SolveServer, matrix_bytes, request_bytes
    params = W.serving_requests(pool, 20, seed=9)
    reqs = _requests(pool, params)
    biggest = max(matrix_bytes(r.m, True) + request_bytes(r, 16384) for r in reqs)
    srv = SolveServer(budget_bytes=biggest * 1.5, workers=4)
    peak = [0.0]
    orig = srv._admit

    def watched():
        orig()
        peak[0] = max(peak[0], srv.used)
    srv._admit = watched
    for r in reqs:
        srv.submit(r)
    for r in reqs:
        assert r.event.wait(300)
    srv.close()
    assert peak[0] <= biggest * 1.5
    bad = [(r.rid, r.m.n, r.method, r.precision, r.precond, r.tol, r.info)
           for r in reqs if r.info["status"] != 0]
    assert not bad, bad
