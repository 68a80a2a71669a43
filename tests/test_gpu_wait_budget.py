"""Bounded device-side waits with a caller's budget (gk_solve_opts.
wait_budget_ns and the wait_budget_ns argument of gk_precond_apply /
gk_triangular_solve), exercised on correct kernels.

A banded matrix makes every substitution chunk depend on the one before
it, so the ILU(0) and triangular-solve kernels poll for values other warps
are still producing.  A budget of a few hundred nanoseconds is shorter than
one hand-off, so the waits give up: the call must return GK_ERR_TIMEOUT
promptly, gk_matrix_describe must report the error, and the next call with
the default budget must succeed with the exact result (the kernels leave
nothing behind).  No wait here is on a value that never comes, and every
kernel finishes: a wait that gives up sets an error word, later waits of
the launch give up at once, and the launch runs to its end.
"""
import time

import numpy as np
import pytest

import oracle
import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W
from gpu_util import ensure_built, torch_dev

pytestmark = pytest.mark.gpu

SHORT_NS = 300


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.fixture(scope="module")
def banded():
    m = W.banded_spd(32768, 16, 7)
    return m, gk.Matrix.from_csr(m, "f64")


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch_dev())


def test_ilu_apply_times_out_then_recovers(banded):
    import torch
    m, A = banded
    r = W.uniform_vector(m.n, 3)
    rt, zt = _dev(r), _dev(np.zeros(m.n))
    A.precond_apply(rt, zt, "ilu")  # builds the factors; default budget
    torch.cuda.synchronize()
    want = oracle.ilu0_apply(m, oracle.ilu0(m), r)
    assert np.array_equal(zt.cpu().numpy(), want)
    t0 = time.perf_counter()
    st = gk.gk_precond_apply(A.handle, "ilu", 0, rt, zt, SHORT_NS)
    el = time.perf_counter() - t0
    assert st == gk.GK_ERR_TIMEOUT
    assert el < 1.0, el  # far below the 2 s default: the waits gave up
    assert A.describe()["device_error"] & 2
    zt.zero_()
    A.precond_apply(rt, zt, "ilu")
    torch.cuda.synchronize()
    assert np.array_equal(zt.cpu().numpy(), want)
    assert A.describe()["device_error"] == 0


def test_triangular_solve_times_out_then_recovers(banded):
    import torch
    m, A = banded
    b = W.uniform_vector(m.n, 4)
    bt, xt = _dev(b), _dev(np.zeros(m.n))
    for upper in (False, True):
        A.triangular_solve(bt, xt, upper=upper)
        torch.cuda.synchronize()
        want = oracle.trsv(m, b, upper=upper)
        assert np.array_equal(xt.cpu().numpy(), want)
        st = gk.lib().gk_triangular_solve(A.handle, int(upper), 0, bt.data_ptr(), xt.data_ptr(),
                                          SHORT_NS, gk._stream(None))
        assert st == gk.GK_ERR_TIMEOUT
        assert A.describe()["device_error"] & 4
        A.triangular_solve(bt, xt, upper=upper)
        torch.cuda.synchronize()
        assert np.array_equal(xt.cpu().numpy(), want)


@pytest.mark.parametrize("method", ["cg", "gmres"])
@pytest.mark.parametrize("mixed", [0, 1])
def test_ilu_solve_times_out_then_recovers(banded, method, mixed):
    """A solve whose ILU(0) substitutions run past the budget stops with
    GK_ERR_TIMEOUT (also inside refinement, where the inner solve's error
    must not be applied as a correction); the same solve with the default
    budget then converges."""
    m, A = banded
    b = W.uniform_vector(m.n, 5)
    bt = _dev(b)
    xt = _dev(np.zeros(m.n))
    t0 = time.perf_counter()
    info = A.solve(bt, xt, method=method, precond="ilu", tol=1e-10, max_iters=2000,
                   mixed=mixed, wait_budget_ns=SHORT_NS)
    el = time.perf_counter() - t0
    assert info["return"] == gk.GK_ERR_TIMEOUT, info
    assert el < 20.0, el
    xt.zero_()
    info = A.solve(bt, xt, method=method, precond="ilu", tol=1e-10, max_iters=2000,
                   mixed=mixed)
    assert info["return"] == gk.GK_OK, info
    assert oracle.true_rel_residual(m, b, xt.cpu().numpy()) <= 1e-10


def test_window_mode_times_out_then_recovers(monkeypatch):
    """The window mode's substitutions wait only for their own bulk copies
    of the rows' records: with a budget shorter than one copy (the first
    level's is waited for right after it is issued) the apply returns
    GK_ERR_TIMEOUT, the blocks still wait for their copies in flight before
    they exit, and the next apply with the default budget is exact."""
    import torch
    monkeypatch.setenv("GK_ILU_CHUNK", "win")
    m = W.laplacian_3d(24)
    A = gk.Matrix.from_csr(m, "f64")
    r = W.uniform_vector(m.n, 8)
    rt, zt = _dev(r), _dev(np.zeros(m.n))
    want = oracle.ilu0_apply(m, oracle.ilu0(m), r)
    A.precond_apply(rt, zt, "ilu")
    torch.cuda.synchronize()
    assert np.array_equal(zt.cpu().numpy(), want)
    st = gk.gk_precond_apply(A.handle, "ilu", 0, rt, zt, 1)
    assert st == gk.GK_ERR_TIMEOUT
    zt.zero_()
    A.precond_apply(rt, zt, "ilu")
    torch.cuda.synchronize()
    assert np.array_equal(zt.cpu().numpy(), want)
    b = W.uniform_vector(m.n, 9)
    bt, xt = _dev(b), _dev(np.zeros(m.n))
    info = A.solve(bt, xt, method="cg", precond="ilu", tol=1e-10, max_iters=500, wait_budget_ns=1)
    assert info["return"] == gk.GK_ERR_TIMEOUT, info
    xt.zero_()
    info = A.solve(bt, xt, method="cg", precond="ilu", tol=1e-10, max_iters=500)
    assert info["return"] == gk.GK_OK, info
    assert oracle.true_rel_residual(m, b, xt.cpu().numpy()) <= 1e-10
    A.close()


def test_negative_budget_is_invalid(banded):
    m, A = banded
    rt, zt = _dev(np.ones(m.n)), _dev(np.zeros(m.n))
    assert gk.gk_precond_apply(A.handle, "ilu", 0, rt, zt, -1) == gk.GK_ERR_INVALID
    assert gk.lib().gk_triangular_solve(A.handle, 0, 0, rt.data_ptr(), zt.data_ptr(), -5,
                                        gk._stream(None)) == gk.GK_ERR_INVALID
    info = A.solve(rt, zt, method="cg", tol=1e-8, wait_budget_ns=-1)
    assert info["return"] == gk.GK_ERR_INVALID


def test_budget_does_not_change_results(banded):
    """A generous explicit budget gives the same bits as the default."""
    import torch
    m, A = banded
    b = W.uniform_vector(m.n, 6)
    bt = _dev(b)
    outs = []
    for budget in (0, 5_000_000_000):
        xt = _dev(np.zeros(m.n))
        info = A.solve(bt, xt, method="cg", precond="ilu", tol=1e-10, max_iters=2000,
                       wait_budget_ns=budget)
        assert info["return"] == gk.GK_OK, info
        torch.cuda.synchronize()
        outs.append(xt.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
