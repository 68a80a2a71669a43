"""gk_spmv_csr_f64_noalloc: the SpMV entry point for callers that cannot
allocate device memory (their memory belongs to a framework pool, or they
run where an allocation is not allowed).  Its output must match the
allocating gk_apply on the same matrix, call after call, although every
call shares one fixed scratch array.  This file is collected last."""
import numpy as np
import pytest

import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W
from gpu_util import TOL, assert_rows_close, ensure_built, oracle_apply

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _device_csr(m):
    import torch
    dev = torch.device("cuda:0")
    return (torch.from_numpy(m.row_ptr.astype(np.int32)).to(dev),
            torch.from_numpy(m.col_idx.astype(np.int32)).to(dev),
            torch.from_numpy(m.values.astype(np.float64)).to(dev))


@pytest.mark.parametrize("name", ["powerlaw_60k", "lap3d_30", "rand_ragged"])
def test_noalloc_matches_apply_on_two_calls(name):
    import torch
    m = {"powerlaw_60k": lambda: W.power_law(60000, max_len=4096, seed=13),
         "lap3d_30": lambda: W.laplacian_3d(30),
         "rand_ragged": lambda: W.random_csr(777, 500, 0.05, 4, empty_rows=40, full_rows=2)}[name]()
    rp, ci, va = _device_csr(m)
    A = gk.Matrix.from_csr(m, "f64")
    rng = np.random.default_rng(3)
    calls = [(1.0, 0.0), (-2.0, 0.5)]
    for alpha, beta in calls:  # two calls in a row share the scratch array
        x = rng.uniform(-1, 1, m.ncols)
        y0 = rng.uniform(-1, 1, m.n)
        xt = torch.from_numpy(x).cuda()
        want = torch.from_numpy(y0).cuda()
        got = torch.from_numpy(y0).cuda()
        A.apply_adv(alpha, xt, beta, want)
        st = gk.gk_spmv_csr_f64_noalloc(m.n, m.ncols, m.nnz, rp, ci, va, alpha, xt, beta, got)
        assert st == gk.GK_OK
        torch.cuda.synchronize()
        ref, scale = oracle_apply(m, x, alpha, beta, y0, "f64")
        assert_rows_close(got.cpu().numpy(), want.cpu().numpy(), scale, TOL["f64"],
                          f"noalloc vs gk_apply {name} a={alpha} b={beta}")
        assert_rows_close(got.cpu().numpy(), ref, scale, TOL["f64"], f"noalloc vs oracle {name}")
    A.close()


def test_noalloc_allocates_nothing_after_setup():
    import torch
    m = W.power_law(30000, max_len=2000, seed=5)
    rp, ci, va = _device_csr(m)
    xt = torch.from_numpy(W.uniform_vector(m.n, 1)).cuda()
    y = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    assert gk.gk_spmv_csr_f64_noalloc(m.n, m.ncols, m.nnz, rp, ci, va, 1.0, xt, 0.0, y) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert gk.gk_spmv_csr_f64_noalloc(m.n, m.ncols, m.nnz, rp, ci, va, 1.0, xt, 0.0, y) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # a call captured in global mode: any allocation (or other call that may
    # synchronise the device) inside it would fail the capture
    g = torch.cuda.CUDAGraph()
    y2 = torch.full_like(y, float("nan"))
    with torch.cuda.graph(g, capture_error_mode="global"):
        st = gk.gk_spmv_csr_f64_noalloc(m.n, m.ncols, m.nnz, rp, ci, va, 1.0, xt, 0.0, y2)
    assert st == 0
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y2, y)


def test_noalloc_rejects_sizes_over_the_limit():
    # checked on the host before any pointer is touched
    n = 1 << 20
    st = gk.gk_spmv_csr_f64_noalloc(n, n, 134217728 - n + 1, None, None, None,
                                    1.0, None, 0.0, None)
    assert st == gk.GK_ERR_INVALID
    assert gk.gk_spmv_csr_f64_noalloc(-1, 1, 0, None, None, None, 1.0, None, 0.0, None) == \
        gk.GK_ERR_INVALID


def test_noalloc_near_limit_256cubed():
    """The 3D 7-point Laplacian 256^3: n + nnz = 133,824,512, just under the
    134,217,728 limit (65,346 of the 65,536 merge blocks the scratch holds).
    With x_i = i mod 7 every product and partial sum is an exact integer, so
    the output must equal A x exactly, for two calls in a row."""
    import oracle
    import torch
    m = W.laplacian_3d(256)
    assert m.n + m.nnz <= 134217728
    rp, ci, va = _device_csr(m)
    x = (np.arange(m.n) % 7).astype(np.float64)
    exact, _ = oracle.spmv_omp(m, x)  # plain sums of exact integers: exact
    xt = torch.from_numpy(x).cuda()
    y = torch.full((m.n,), float("nan"), dtype=torch.float64, device="cuda")
    assert gk.gk_spmv_csr_f64_noalloc(m.n, m.ncols, m.nnz, rp, ci, va, 1.0, xt, 0.0, y) == 0
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), exact)
    y0 = (np.arange(m.n) % 5).astype(np.float64)
    y = torch.from_numpy(y0).cuda()
    assert gk.gk_spmv_csr_f64_noalloc(m.n, m.ncols, m.nnz, rp, ci, va, -2.0, xt, 0.5, y) == 0
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), -2.0 * exact + 0.5 * y0)
