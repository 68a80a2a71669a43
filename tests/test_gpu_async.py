"""gk_solve_async: the whole Krylov loop enqueued on a stream (one CUDA
graph with a conditional loop node), the outcome written to device memory.
It must give the bits of the synchronous multi-kernel solve, meet the
oracle's true residual, and let one host thread enqueue many solves before
waiting once."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W
from gpu_util import ensure_built, torch_dev

pytestmark = pytest.mark.gpu

INFO_BYTES = ctypes.sizeof(gk.gk_solve_info)


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _info_buf():
    import torch
    return torch.zeros(INFO_BYTES, dtype=torch.uint8, device=torch_dev())


def _read(buf):
    return gk.solve_info_from_bytes(buf.cpu().numpy())


CASES = {
    "lap2d_48": lambda: W.laplacian_2d(48),
    "diff3d_20": lambda: W.diffusion_3d(20),
    "convdiff_40": lambda: W.convection_diffusion_2d(40, 1.0),
    "banded_3000": lambda: W.banded_spd(3000, 12, 5),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("method,precond", [("cg", "jacobi"), ("cg", None), ("cg", "ilu"),
                                            ("bicgstab", "jacobi"), ("gmres", "jacobi"),
                                            ("gmres", "ilu"), ("cgs", "jacobi"),
                                            ("cg", "block_jacobi")])
def test_async_equals_sync_and_meets_tol(name, method, precond):
    import torch
    m = CASES[name]()
    if method == "cg" and name == "convdiff_40":
        pytest.skip("CG needs a symmetric matrix")
    dev = torch_dev()
    b = W.uniform_vector(m.n, 7)
    bt = torch.from_numpy(b).to(dev)
    A = gk.Matrix.from_csr(m)
    kw = dict(method=method, precond=precond, tol=1e-10, max_iters=5000, engine=1,
              block_size=4 if precond == "block_jacobi" else 0)
    xs = torch.zeros_like(bt)
    sync = A.solve(bt, xs, **kw)
    assert sync["return"] == gk.GK_OK, sync
    xa = torch.zeros_like(bt)
    info = _info_buf()
    st = gk.gk_solve_async(A.handle, bt, xa, gk.make_opts(**kw), info)
    assert st == gk.GK_OK
    torch.cuda.synchronize()
    ia = _read(info)
    assert ia["status"] == gk.GK_OK, ia
    assert np.array_equal(xa.cpu().numpy(), xs.cpu().numpy())
    assert ia["iters"] == sync["iters"] and ia["restarts"] == sync["restarts"]
    assert ia["rel_res_true"] == sync["rel_res_true"]
    assert oracle.true_rel_residual(m, b, xa.cpu().numpy()) <= 1e-10
    A.close()


def test_many_async_solves_one_wait():
    """One host thread enqueues solves on several matrices (two per matrix,
    different right-hand sides and initial guesses) on one stream and waits
    once; every outcome matches the synchronous solve of the same system."""
    import torch
    dev = torch_dev()
    mats = [W.laplacian_2d(30), W.laplacian_3d(14), W.banded_spd(2000, 9, 2)]
    As = [gk.Matrix.from_csr(m) for m in mats]
    jobs = []
    for k, (m, A) in enumerate(zip(mats, As)):
        for j in range(2):
            b = torch.from_numpy(W.uniform_vector(m.n, 10 * k + j)).to(dev)
            x0 = torch.from_numpy(0.01 * W.uniform_vector(m.n, 99 + j)).to(dev)
            x = x0.clone()
            info = _info_buf()
            st = gk.gk_solve_async(A.handle, b, x, gk.make_opts(method="cg", precond="jacobi",
                                                                tol=1e-9, max_iters=4000), info)
            assert st == gk.GK_OK
            jobs.append((m, A, b, x0, x, info))
    torch.cuda.synchronize()
    for m, A, b, x0, x, info in jobs:
        ia = _read(info)
        assert ia["status"] == gk.GK_OK
        xs = x0.clone()
        ref = A.solve(b, xs, method="cg", precond="jacobi", tol=1e-9, max_iters=4000, engine=1)
        assert np.array_equal(x.cpu().numpy(), xs.cpu().numpy())
        assert ia["iters"] == ref["iters"]
    for A in As:
        A.close()


def test_async_not_converged_and_errors():
    import torch
    dev = torch_dev()
    m = W.laplacian_2d(40)
    A = gk.Matrix.from_csr(m)
    bt = torch.from_numpy(W.uniform_vector(m.n, 1)).to(dev)
    x = torch.zeros_like(bt)
    info = _info_buf()
    assert gk.gk_solve_async(A.handle, bt, x, gk.make_opts(method="cg", tol=1e-12, max_iters=5),
                             info) == gk.GK_OK
    torch.cuda.synchronize()
    ia = _read(info)
    assert ia["status"] == gk.GK_NOT_CONVERGED and ia["iters"] <= 5 + 32
    # b = 0: x = 0 after 0 iterations
    x.fill_(1.0)
    assert gk.gk_solve_async(A.handle, torch.zeros_like(bt), x, gk.make_opts(method="cg"),
                             info) == gk.GK_OK
    torch.cuda.synchronize()
    ia = _read(info)
    assert ia["status"] == gk.GK_OK and ia["iters"] == 0 and not x.any()
    # refinement runs its outer loop on the host: not offered asynchronously
    assert gk.gk_solve_async(A.handle, bt, x, gk.make_opts(method="cg", mixed=1),
                             info) == gk.GK_ERR_UNSUPPORTED
    assert gk.gk_solve_async(A.handle, bt, x, gk.make_opts(method="cg"),
                             None) == gk.GK_ERR_INVALID
    A.close()


def test_unrolled_profiling_graph_gives_the_same_solve(monkeypatch):
    """GK_SOLVE_UNROLLED=k builds the solve graph without its loop node (the
    body repeated k times, so that a profiler can see every kernel): for a
    solve that needs exactly those passes it gives the bits of the looped
    graph."""
    import torch
    dev = torch_dev()
    m = W.laplacian_2d(48)  # 2304 rows: passes of 32 iterations
    b = torch.from_numpy(W.uniform_vector(m.n, 4)).to(dev)
    out = []
    for unrolled in (None, "2"):
        if unrolled:
            monkeypatch.setenv("GK_SOLVE_UNROLLED", unrolled)
        else:
            monkeypatch.delenv("GK_SOLVE_UNROLLED", raising=False)
        A = gk.Matrix.from_csr(m)  # a fresh handle: the graph is built for this solve
        x = torch.zeros_like(b)
        info = A.solve(b, x, method="cg", precond="jacobi", tol=1e-14, max_iters=64, engine=1)
        out.append((x.cpu().numpy(), info))
        A.close()
    (x0, i0), (x1, i1) = out
    assert i0["return"] == i1["return"] == gk.GK_NOT_CONVERGED and i0["iters"] == i1["iters"] == 64
    assert np.array_equal(x0, x1)


@pytest.mark.parametrize("method,precond", [("cg", "jacobi"), ("bicgstab", "jacobi"),
                                            ("gmres", "jacobi"), ("cgs", None), ("cg", "ilu")])
def test_host_driven_loop_equals_device_loop(monkeypatch, method, precond):
    """GK_SOLVE_LOOP=host runs the same passes from the host (one graph per
    pass, two in flight): the same bits, iterations and outcome as the
    loop inside one graph, including a solve that converges mid-pass and
    FP32 refinement (whose inner solves run the loop too)."""
    import torch
    m = W.diffusion_3d(20)
    b = torch.from_numpy(W.uniform_vector(m.n, 8)).to(torch_dev())
    out = {}
    for mode in ("device", "host"):
        monkeypatch.setenv("GK_SOLVE_LOOP", mode)
        A = gk.Matrix.from_csr(m)
        for mixed in (0, 1):
            x = torch.zeros_like(b)
            info = A.solve(b, x, method=method, precond=precond, tol=1e-10, max_iters=5000,
                           engine=1, mixed=mixed)
            out[mode, mixed] = (x.cpu().numpy(), info)
        A.close()
    for mixed in (0, 1):
        (xd, idv), (xh, ih) = out["device", mixed], out["host", mixed]
        assert idv["return"] == ih["return"] == gk.GK_OK, (idv, ih)
        assert np.array_equal(xd, xh), mixed
        assert (idv["iters"], idv["restarts"], idv["outer_iters"]) == \
            (ih["iters"], ih["restarts"], ih["outer_iters"])
