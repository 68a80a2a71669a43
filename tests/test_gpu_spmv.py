"""GPU SpMV parity against the CPU oracle, through the C ABI: every format,
kernel variant and value type, alpha/beta forms, edge cases, and sampled
rows of the full-size 256^3 stencil and 2^22-row power-law matrices."""
import os

import numpy as np
import pytest

import oracle
import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W
from gpu_util import (TOL, assert_rows_close, ensure_built, oracle_apply, sub_rows, torch_dev,
                      vec_dtype)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _make(m, fmt, dtype, kernel=None, S=0, f=0):
    """Device matrix in the requested format (CSR kernel forced by kind)."""
    old = os.environ.get("GK_CSR_KERNEL")
    if kernel is not None:
        os.environ["GK_CSR_KERNEL"] = str(kernel)
    try:
        A = gk.Matrix.from_csr(m, dtype)
    finally:
        if kernel is not None:
            if old is None:
                del os.environ["GK_CSR_KERNEL"]
            else:
                os.environ["GK_CSR_KERNEL"] = old
    if fmt == "csr":
        return A
    B = A.convert(fmt, None, S, f)
    A.close()
    return B


def _run(A, x, alpha, beta, y0, dtype):
    import torch
    dev = torch_dev()
    xt = torch.from_numpy(np.asarray(x)).to(dev, vec_dtype(dtype))
    yt = (torch.from_numpy(np.asarray(y0)).to(dev, vec_dtype(dtype)) if y0 is not None
          else torch.full((A.n,), float("nan"), dtype=vec_dtype(dtype), device=dev))
    if alpha == 1.0 and beta == 0.0:
        A.apply(xt, yt)
    else:
        A.apply_adv(alpha, xt, beta, yt)
    torch.cuda.synchronize()
    return yt.cpu().numpy()


MATS = {
    "rand_33x40": lambda: W.random_csr(33, 40, 0.2, 3, empty_rows=5, full_rows=1),
    "rand_1x1": lambda: W.random_csr(1, 1, 1.0, 1),
    "rand_300x7": lambda: W.random_csr(300, 7, 0.4, 5, empty_rows=30),
    "lap2d_64": lambda: W.laplacian_2d(64),
    "lap3d_40": lambda: W.laplacian_3d(40),
    "powerlaw_20k": lambda: W.power_law(20000, max_len=4096, seed=11),
    "banded_5000": lambda: W.banded_spd(5000, 37, 3),
    "empty_rows_only": lambda: W.CSR(50, 50, np.zeros(51, np.int32), np.zeros(0, np.int32),
                                     np.zeros(0)),
}
VARIANTS = [("csr", 1, 0, 0), ("csr", 2, 0, 0), ("csr", 0, 0, 0), ("csr", 3, 0, 0),
            ("ell", None, 0, 0),
            ("sellp", None, 32, 1), ("sellp", None, 8, 4), ("sellp", None, 64, 2),
            ("coo", None, 0, 0)]


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("fmt,kernel,S,f", VARIANTS)
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
def test_spmv_matches_oracle(name, fmt, kernel, S, f, dtype):
    m = MATS[name]()
    if fmt == "ell" and m.nnz and m.row_lengths().max() * m.n > 50_000_000:
        pytest.skip("ELL padding too large")
    A = _make(m, fmt, dtype, kernel, S, f)
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, m.ncols)
    y0 = rng.uniform(-1, 1, m.n)
    for alpha, beta, use_y0 in ((1.0, 0.0, False), (2.5, 0.0, False), (-0.5, 2.0, True)):
        y = _run(A, x, alpha, beta, y0 if use_y0 else None, dtype)
        ref, scale = oracle_apply(m, x, alpha, beta, y0 if use_y0 else None, dtype)
        assert_rows_close(y, ref, scale, TOL[dtype], f"{name} {fmt}/{kernel} {dtype} a={alpha} b={beta}")
    A.close()


@pytest.mark.parametrize("rpl,stages", [(1, 1), (1, 2), (2, 2), (4, 1), (4, 3)])
@pytest.mark.parametrize("name", ["lap3d_40", "rand_300x7", "banded_5000", "empty_rows_only"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_warptile_shapes(rpl, stages, name, dtype):
    """The warp-tile CSR kernel for every tile height (32, 64, 128 rows)
    and ring depth it can be configured with."""
    env = {"GK_WT_RPL": str(rpl), "GK_WT_STAGES": str(stages)}
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        m = MATS[name]()
        A = _make(m, "csr", dtype, 3)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    if A.desc["spmv_kernel"] != 6:
        pytest.skip("tile does not fit shared memory; another CSR kernel is used")
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, m.ncols)
    y0 = rng.uniform(-1, 1, m.n)
    for alpha, beta, use_y0 in ((1.0, 0.0, False), (-0.5, 2.0, True)):
        y = _run(A, x, alpha, beta, y0 if use_y0 else None, dtype)
        ref, scale = oracle_apply(m, x, alpha, beta, y0 if use_y0 else None, dtype)
        assert_rows_close(y, ref, scale, TOL[dtype], f"{name} warptile rpl={rpl} nst={stages}")
    A.close()


@pytest.mark.parametrize("fmt,kernel,S,f", VARIANTS)
def test_integer_exact_stencil(fmt, kernel, S, f):
    """5-point Laplacian times ones (and times i mod 7) is exact in FP64:
    the GPU must match bit for bit."""
    N = 64
    m = W.laplacian_2d(N)
    A = _make(m, fmt, "f64", kernel, S, f)
    y = _run(A, np.ones(m.n), 1.0, 0.0, None, "f64")
    cnt = np.zeros((N, N), dtype=np.int64)
    cnt[:, 1:] += 1; cnt[:, :-1] += 1; cnt[1:, :] += 1; cnt[:-1, :] += 1
    assert np.array_equal(y, (4 - cnt.reshape(-1)).astype(np.float64))
    x = (np.arange(m.n) % 7).astype(np.float64)
    y = _run(A, x, 1.0, 0.0, None, "f64")
    assert np.array_equal(y, oracle.spmv(m, x))
    A.close()


def test_beta_zero_ignores_nan_in_output():
    m = W.laplacian_2d(20)
    A = _make(m, "csr", "f64")
    y = _run(A, np.ones(m.n), 3.0, 0.0, None, "f64")  # output prefilled with NaN
    assert np.all(np.isfinite(y))


def test_host_pointer_apply_matches_device():
    m = W.power_law(5000, max_len=1000, seed=2)
    A = _make(m, "csr", "f64")
    x = W.uniform_vector(m.n, 4)
    yh = np.zeros(m.n)
    A.apply(x, yh)  # numpy host buffers: staged, blocking
    yd = _run(A, x, 1.0, 0.0, None, "f64")
    assert np.array_equal(yh, yd)
    y0 = W.uniform_vector(m.n, 5)
    yh = y0.copy()
    A.apply_adv(2.0, x, -1.0, yh)
    ref, scale = oracle_apply(m, x, 2.0, -1.0, y0, "f64")
    assert_rows_close(yh, ref, scale, 1e-13, "host apply_adv")


@pytest.mark.parametrize("fmt,kernel", [("csr", 0), ("csr", 1), ("csr", 2), ("coo", None)])
def test_spmv_deterministic(fmt, kernel):
    m = W.power_law(50000, max_len=4096, seed=9)
    A = _make(m, fmt, "f64", kernel)
    x = W.uniform_vector(m.n, 1)
    y1 = _run(A, x, 1.0, 0.0, None, "f64")
    y2 = _run(A, x, 1.0, 0.0, None, "f64")
    assert np.array_equal(y1, y2)


@pytest.fixture(scope="module")
def lap256():
    return W.laplacian_3d(256)


@pytest.fixture(scope="module")
def powerlaw4m():
    return W.power_law(1 << 22, seed=W.SEED_BASE + 2)


def _sampled_check(m, A, dtype, seed):
    x = W.uniform_vector(m.ncols, seed)
    y = _run(A, x, 1.0, 0.0, None, dtype)
    rng = np.random.default_rng(seed)
    rows = np.unique(np.concatenate([rng.integers(0, m.n, 20000), [0, m.n - 1],
                                     np.argsort(m.row_lengths())[-50:]]))
    sub = sub_rows(m, rows)
    ref, scale = oracle_apply(sub, x, 1.0, 0.0, None, dtype)
    assert_rows_close(y[rows], ref, scale, TOL[dtype], f"{m.name} {dtype} sampled")
    assert np.all(np.isfinite(y))


@pytest.mark.parametrize("fmt", ["csr", "ell", "sellp", "coo"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_stencil_sampled(lap256, fmt, dtype):
    A = _make(lap256, fmt, dtype)
    _sampled_check(lap256, A, dtype, 21)
    A.close()


@pytest.mark.parametrize("fmt", ["csr", "sellp", "coo"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_full_size_powerlaw_sampled(powerlaw4m, fmt, dtype):
    A = _make(powerlaw4m, fmt, dtype)
    _sampled_check(powerlaw4m, A, dtype, 22)
    A.close()


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_coo_layout_and_oracle_coo_spmv(name, dtype):
    """The COO handle holds the row of every entry in CSR order (bit-exact
    against the expanded row pointer), and its apply matches the oracle's
    COO SpMV (triplets visited in storage order)."""
    from gpu_util import rounded_values, rounded_vector
    m = MATS[name]()
    A = _make(m, "coo", dtype)
    assert A.desc["format"] == gk.GK_COO and A.desc["spmv_kernel"] == 5
    e = A.export()
    rows = np.repeat(np.arange(m.n, dtype=np.int32), np.diff(m.row_ptr))
    assert np.array_equal(e["row"], rows) and np.array_equal(e["col_idx"], m.col_idx)
    vals = rounded_values(m, dtype)
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, m.ncols)
    y0 = rng.uniform(-1, 1, m.n)
    xv, y0v = rounded_vector(x, dtype), rounded_vector(y0, dtype)
    for alpha, beta in ((1.0, 0.0), (-1.5, 0.5)):
        y = _run(A, x, alpha, beta, y0 if beta else None, dtype)
        ref = oracle.spmv_coo(m.n, m.ncols, rows, m.col_idx, vals, xv, alpha, beta,
                              y=y0v if beta else None)
        scale = abs(alpha) * oracle.spmv_coo(m.n, m.ncols, rows, m.col_idx, np.abs(vals),
                                             np.abs(xv)) + abs(beta) * np.abs(y0v)
        assert_rows_close(y, ref, scale, TOL[dtype], f"coo {name} {dtype} a={alpha} b={beta}")
    # round trip: COO -> CSR gives the original arrays
    B = A.convert("csr")
    eb = B.export()
    assert np.array_equal(eb["row_ptr"], m.row_ptr) and np.array_equal(eb["col_idx"], m.col_idx)
    B.close()
    A.close()


@pytest.mark.parametrize("fmt", ["csr", "ell", "sellp", "coo"])
def test_f16_values_round_once_to_nearest_even(fmt):
    """FP64 values converted on the device to IEEE half are the correctly
    rounded halves (numpy's float64 -> float16), bit for bit, in every
    layout; the padding of ELL / SELL-P stays +0.0."""
    m = W.power_law(3000, max_len=300, seed=4)
    A = _make(m, fmt, "f16")
    e = A.export()
    want = np.asarray(m.values, np.float64).astype(np.float16)
    got = e["values"]
    if fmt in ("csr", "coo"):
        assert np.array_equal(got.view(np.uint16), want.view(np.uint16))
    else:
        assert np.array_equal(np.sort(got[e["col"] >= 0].view(np.uint16)),
                              np.sort(want.view(np.uint16)))
        assert np.all(got[e["col"] < 0].view(np.uint16) == 0)
    A.close()
