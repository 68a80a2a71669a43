"""Single-block engine: many independent systems in one launch
(gk_solve_batched) and small single systems (engine 2), against the
oracle.  A system's result must not depend on the rest of the batch."""
import numpy as np
import pytest

import oracle
import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W
from gpu_util import ensure_built, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _batch(mats, rhs, dtype, method, precond, tol, max_iters=20000):
    import torch
    dev = torch_dev()
    vt = torch.float64 if dtype == "f64" else torch.float32
    As = [gk.Matrix.from_csr(m, dtype) for m in mats]
    bs = [torch.from_numpy(b).to(dev, vt) for b in rhs]
    xs = [torch.zeros(m.n, dtype=vt, device=dev) for m in mats]
    opts = gk.make_opts(method=method, precond=precond, tol=tol, max_iters=max_iters)
    st, infos = gk.gk_solve_batched([A.handle for A in As], bs, xs, opts)
    torch.cuda.synchronize()
    out = [x.cpu().numpy().astype(np.float64) for x in xs]
    for A in As:
        A.close()
    return st, infos, out


@pytest.fixture(scope="module")
def systems():
    mats, rhs = W.batched_rectangles(96, seed=W.SEED_BASE + 4)
    return mats, rhs


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
@pytest.mark.parametrize("precond", [None, "jacobi"])
def test_batched_fp64_matches_oracle(systems, method, precond):
    mats, rhs = systems
    st, infos, xs = _batch(mats, rhs, "f64", method, precond, 1e-10)
    assert st == gk.GK_OK
    for m, b, x, info in zip(mats, rhs, xs, infos):
        assert info["status"] == gk.GK_OK, info
        rel = oracle.true_rel_residual(m, b, x)
        assert rel <= 1e-10, (rel, info)
        assert abs(info["rel_res_true"] - rel) <= 1e-3 * rel + 1e-16
        if method == "cg":
            _, io = oracle.solve(m, b, method=oracle.CG, precond=1 if precond else 0, tol=1e-10,
                                 max_iters=20000)
            assert abs(info["iters"] - io["iters"]) <= max(3, 0.1 * io["iters"]), (info, io)


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
def test_batched_fp32(systems, method):
    mats, rhs = systems
    st, infos, xs = _batch(mats[:32], rhs[:32], "f32", method, "jacobi", 1e-5)
    for m, b, x, info in zip(mats, rhs, xs, infos):
        assert info["status"] == gk.GK_OK, info
        assert oracle.true_rel_residual(m, b, x) <= 3e-5


def test_alone_equals_in_batch(systems):
    """Bit-identical results for a system solved alone or inside a batch."""
    mats, rhs = systems
    st, infos, xs = _batch(mats[:40], rhs[:40], "f64", "cg", "jacobi", 1e-10)
    for i in (0, 7, 39):
        st1, inf1, x1 = _batch([mats[i]], [rhs[i]], "f64", "cg", "jacobi", 1e-10)
        assert np.array_equal(x1[0], xs[i]) and inf1[0]["iters"] == infos[i]["iters"]


def test_batched_edge_cases():
    good = W.shifted_rectangle(5, 7, 0.3)
    zero_diag = W.CSR(3, 3, np.array([0, 1, 2, 3]), np.array([0, 1, 0]), np.array([1.0, 2.0, 3.0]))
    one = W.CSR(1, 1, np.array([0, 1]), np.array([0]), np.array([4.0]))
    mats = [good, zero_diag, one, good]
    rhs = [W.uniform_vector(good.n, 1), np.ones(3), np.array([2.0]), np.zeros(good.n)]
    st, infos, xs = _batch(mats, rhs, "f64", "cg", "jacobi", 1e-10)
    assert infos[0]["status"] == gk.GK_OK
    assert infos[1]["status"] == gk.GK_ERR_ZERO_DIAG
    assert infos[2]["status"] == gk.GK_OK and xs[2][0] == 0.5
    assert infos[3]["status"] == gk.GK_OK and infos[3]["iters"] == 0 and np.all(xs[3] == 0)


def test_batched_rejects_gmres_and_bad_input(systems):
    import torch
    mats, rhs = systems
    A = gk.Matrix.from_csr(mats[0])
    b = torch.from_numpy(rhs[0]).cuda()
    x = torch.zeros_like(b)
    st, _ = gk.gk_solve_batched([A.handle], [b], [x], gk.make_opts(method="gmres"))
    assert st == gk.GK_ERR_UNSUPPORTED
    E = A.convert("ell")
    st, _ = gk.gk_solve_batched([E.handle], [b], [x], gk.make_opts(method="cg"))
    assert st == gk.GK_ERR_INVALID


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
@pytest.mark.parametrize("precond", [None, "jacobi"])
def test_single_block_engine(method, precond):
    import torch
    m = W.laplacian_2d(64)
    b = W.uniform_vector(m.n, W.SEED_BASE + 1)
    A = gk.Matrix.from_csr(m)
    bt = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bt)
    info = A.solve(bt, x, method=method, precond=precond, tol=1e-10, max_iters=5000, engine=2)
    assert info["return"] == gk.GK_OK, info
    assert oracle.true_rel_residual(m, b, x.cpu().numpy()) <= 1e-10


def _with_env(env, fn):
    import os
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return fn()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_batched_layouts_give_identical_results(systems, method, dtype):
    """Every SpMV layout the autotuner can pick (CSR, ELL where it pads
    little, SELL-P with 8 to 64 rows per slice) and every block size sums a
    row in CSR order and reduces over fixed virtual lanes: the solutions are
    bit-identical, and infos report the layout each system ran on."""
    mats, rhs = systems
    mats = mats[:24] + [W.banded_spd(700, 40, 5)]  # rows of up to 81 entries
    rhs = rhs[:24] + [W.uniform_vector(700, 3)]
    tol = 1e-10 if dtype == "f64" else 1e-5
    ref = None
    for layout, S in (("csr", 0), ("ell", 0), ("sellp8", 8), ("sellp16", 16), ("sellp32", 32),
                      ("sellp64", 64)):
        for nt in ("128", "512"):
            st, infos, xs = _with_env({"GK_BATCH_LAYOUT": layout, "GK_BATCH_THREADS": nt},
                                      lambda: _batch(mats, rhs, dtype, method, "jacobi", tol))
            assert st == gk.GK_OK
            for m, info in zip(mats, infos):
                assert info["status"] == gk.GK_OK, info
                assert info["block_threads"] == int(nt)
                want = {"csr": gk.GK_CSR, "ell": gk.GK_ELL}.get(layout, gk.GK_SELLP)
                if layout == "ell" and m.row_lengths().max() * m.n > m.nnz + m.nnz // 5:
                    want = gk.GK_CSR  # ELL would pad too much: the system keeps CSR
                assert info["spmv_format"] == want and info["slice_size"] == S, (layout, info)
            if ref is None:
                ref = xs
                for m, b, x, info in zip(mats, rhs, xs, infos):
                    if dtype == "f64":
                        assert oracle.true_rel_residual(m, b, x) <= 1e-10
                    else:  # the residual of the stored (rounded) matrix
                        assert info["rel_res_true"] <= 1e-5
            else:
                for x0, x1 in zip(ref, xs):
                    assert np.array_equal(x0, x1), (layout, nt)


def test_autotuner_reports_its_choice(systems):
    """A tuned batch reports the chosen layout and block size, and its
    results equal those of any forced configuration."""
    mats, rhs = systems
    st, infos, xs = _batch(mats, rhs, "f64", "cg", "jacobi", 1e-10)  # 96 >= 64: tuned
    assert st == gk.GK_OK
    assert all(i["block_threads"] in (128, 256, 512) for i in infos)
    assert all(i["spmv_format"] in (gk.GK_CSR, gk.GK_ELL, gk.GK_SELLP) for i in infos)
    st2, infos2, xs2 = _with_env({"GK_BATCH_LAYOUT": "csr", "GK_BATCH_THREADS": "256"},
                                 lambda: _batch(mats, rhs, "f64", "cg", "jacobi", 1e-10))
    for a, b in zip(xs, xs2):
        assert np.array_equal(a, b)
