"""Pins for the CPU oracle: each test checks the oracle against something
other than itself (a dense matvec or LAPACK solve from numpy, a closed
form, an invariant, brute force, or a hand-written layout).  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2510_08230_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr(n, ncols, rp, ci, va):
    return W.CSR(n, ncols, np.asarray(rp), np.asarray(ci), np.asarray(va, dtype=np.float64))


# ----------------------------------------------------------------- SpMV

@pytest.mark.parametrize("seed,n,ncols,dens,empty,full", [
    (1, 1, 1, 1.0, 0, 0), (2, 7, 5, 0.4, 2, 1), (3, 33, 40, 0.2, 5, 1),
    (4, 64, 64, 0.1, 10, 2), (5, 37, 3, 0.5, 0, 0), (6, 50, 1, 0.5, 3, 0)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.5, 2.0), (2.5, -1.0)])
def test_spmv_matches_dense_matvec(seed, n, ncols, dens, empty, full, alpha, beta):
    m = W.random_csr(n, ncols, dens, seed, empty_rows=empty, full_rows=full)
    rng = np.random.default_rng(seed + 100)
    x = rng.standard_normal(ncols)
    y0 = rng.standard_normal(n)
    ref = alpha * (m.to_dense() @ x) + beta * y0
    for comp in (True, False):
        y = oracle.spmv(m, x, alpha, beta, y0, compensated=comp)
        scale = abs(alpha) * (np.abs(m.to_dense()) @ np.abs(x)) + abs(beta) * np.abs(y0)
        assert np.all(np.abs(y - ref) <= 1e-14 * scale + 1e-300)


@pytest.mark.parametrize("make", [lambda: W.random_csr(301, 97, 0.1, 12, empty_rows=20, full_rows=2),
                                  lambda: W.power_law(20000, max_len=2000, seed=3),
                                  lambda: W.laplacian_3d(23)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.5, 2.0), (2.5, -1.0)])
def test_spmv_omp_is_the_plain_row_sum(make, alpha, beta):
    """The row-parallel timing-mode SpMV (the CPU baseline) gives, for any
    thread count, the bits of the sequential plain-sum SpMV: every row is
    one thread's left-to-right sum.  It also matches the dense matvec, does
    not read y when beta = 0, and reports the threads it used."""
    m = make()
    rng = np.random.default_rng(8)
    x = rng.standard_normal(m.ncols)
    y0 = rng.standard_normal(m.n)
    seq = oracle.spmv(m, x, alpha, beta, y0, compensated=False)
    import os as _os
    cores = len(_os.sched_getaffinity(0))
    for threads in sorted({1, 2, cores}):
        y = np.full(m.n, np.nan) if beta == 0.0 else y0.copy()
        out, used = oracle.spmv_omp(m, x, threads, alpha, beta, y)
        assert used == threads
        assert np.array_equal(out.view(np.uint64), seq.view(np.uint64)), threads
    if m.n <= 400:
        ref = alpha * (m.to_dense() @ x) + beta * y0
        scale = abs(alpha) * (np.abs(m.to_dense()) @ np.abs(x)) + abs(beta) * np.abs(y0)
        assert np.all(np.abs(seq - ref) <= 1e-14 * scale + 1e-300)
    else:
        # integer-valued matrix and vector: every product and sum is exact
        mi = W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx, np.rint(4 * m.values))
        xi = np.arange(m.ncols, dtype=np.float64) % 7 - 3
        yi, _ = oracle.spmv_omp(mi, xi, cores)
        rows = np.repeat(np.arange(m.n), m.row_lengths())
        exact = np.zeros(m.n, dtype=np.int64)
        np.add.at(exact, rows, mi.values.astype(np.int64) * xi.astype(np.int64)[m.col_idx])
        assert np.array_equal(yi, exact.astype(np.float64))


def test_spmv_beta_zero_does_not_read_y():
    m = W.laplacian_2d(4)
    y = np.full(m.n, np.nan)
    out = oracle.spmv(m, np.ones(m.n), 1.0, 0.0, y)
    assert np.all(np.isfinite(out))


def _interior_neighbours_2d(N):
    cnt = np.zeros((N, N), dtype=np.int64)  # [y, x]
    cnt[:, 1:] += 1
    cnt[:, :-1] += 1
    cnt[1:, :] += 1
    cnt[:-1, :] += 1
    return cnt.reshape(-1)


def test_spmv_integer_exact_5pt_ones():
    """A*1 for the 5-point Dirichlet Laplacian is 4 - (number of grid
    neighbours), exactly."""
    N = 64
    m = W.laplacian_2d(N)
    y = oracle.spmv(m, np.ones(m.n))
    expect = 4 - _interior_neighbours_2d(N)
    assert np.array_equal(y, expect.astype(np.float64))


def test_spmv_integer_exact_mod7():
    """Integer matrix times integer vector is exact in FP64: compare with an
    int64 brute-force product."""
    m = W.laplacian_3d(9, 7, 5)
    x = (np.arange(m.n) % 7).astype(np.int64)
    rows = np.repeat(np.arange(m.n), m.row_lengths())
    ref = np.zeros(m.n, dtype=np.int64)
    np.add.at(ref, rows, m.values.astype(np.int64) * x[m.col_idx])
    y = oracle.spmv(m, x.astype(np.float64), compensated=False)
    assert np.array_equal(y, ref.astype(np.float64))


def test_spmv_compensated_sum():
    """Neumaier compensation recovers the exact row sum where the plain sum
    cancels: 1e16 + 1 - 1e16 = 1."""
    m = _csr(1, 3, [0, 3], [0, 1, 2], [1e16, 1.0, -1e16])
    x = np.ones(3)
    assert oracle.spmv(m, x, compensated=True)[0] == 1.0
    assert oracle.spmv(m, x, compensated=False)[0] == 0.0


@pytest.mark.parametrize("dims", [(50,), (17, 13), (9, 8, 7)])
def test_laplacian_closed_form_eigenpairs(dims):
    """Dirichlet Laplacian eigenpairs: lambda = sum_d 4 sin^2(k_d pi / (2 (N_d + 1))),
    v = prod_d sin(i_d k_d pi / (N_d + 1))."""
    m = {1: W.laplacian_1d, 2: W.laplacian_2d, 3: W.laplacian_3d}[len(dims)](*dims)
    rng = np.random.default_rng(7)
    grids = np.meshgrid(*[np.arange(1, N + 1) for N in dims], indexing="ij")
    for _ in range(4):
        ks = [int(rng.integers(1, N + 1)) for N in dims]
        lam = sum(4.0 * math.sin(k * math.pi / (2 * (N + 1))) ** 2 for k, N in zip(ks, dims))
        v = np.ones_like(grids[0], dtype=np.float64)
        for g, k, N in zip(grids, ks, dims):
            v = v * np.sin(g * k * math.pi / (N + 1))
        # workloads index x fastest: flatten with axis 0 fastest
        v = v.transpose(tuple(reversed(range(len(dims))))).reshape(-1)
        Av = oracle.spmv(m, v)
        assert np.linalg.norm(Av - lam * v) <= 1e-13 * np.linalg.norm(v) * max(1.0, lam)


# ------------------------------------------------------------ COO -> CSR

def _brute_coo_to_csr(n, row, col, val):
    """Dictionary of (row, col) -> list of values in input order."""
    d = {}
    for r, c, v in zip(row.tolist(), col.tolist(), val.tolist()):
        d.setdefault((r, c), []).append(v)
    keys = sorted(d)
    rp = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for (r, c) in keys:
        rp[r + 1] += 1
        cols.append(c)
        s = 0.0
        first = True
        for v in d[(r, c)]:
            s = v if first else s + v
            first = False
        vals.append(s)
    return np.cumsum(rp), np.array(cols, dtype=np.int64), np.array(vals)


@pytest.mark.parametrize("seed,n,ncols,nnz", [(1, 10, 10, 40), (2, 100, 7, 500),
                                              (3, 1, 1, 5), (4, 300, 300, 50)])
def test_coo_to_csr_brute_force(seed, n, ncols, nnz):
    r, c, v = W.random_coo(n, ncols, nnz, seed)
    rp, ci, va = oracle.coo_to_csr(n, ncols, r, c, v)
    brp, bci, bva = _brute_coo_to_csr(n, r, c, v)
    assert np.array_equal(rp, brp) and np.array_equal(ci, bci)
    assert np.array_equal(va, bva)


def test_coo_duplicates_summed_in_input_order():
    row = np.array([0, 0, 0, 1, 1, 1], dtype=np.int32)
    col = np.array([1, 1, 1, 0, 0, 0], dtype=np.int32)
    # row 0: ((1e16 + 1) - 1e16) = 0 ; row 1: ((1e16 - 1e16) + 1) = 1
    val = np.array([1e16, 1.0, -1e16, 1e16, -1e16, 1.0])
    rp, ci, va = oracle.coo_to_csr(2, 2, row, col, val)
    assert rp.tolist() == [0, 1, 2] and ci.tolist() == [1, 0]
    assert va.tolist() == [0.0, 1.0]


def test_coo_duplicates_summed_in_float32_for_fp32():
    row = np.zeros(3, dtype=np.int32)
    col = np.zeros(3, dtype=np.int32)
    val = np.array([1.0, 2.0 ** -24, 2.0 ** -24])
    _, _, v32 = oracle.coo_to_csr(1, 1, row, col, val, sum_f32=True)
    _, _, v64 = oracle.coo_to_csr(1, 1, row, col, val, sum_f32=False)
    assert v32[0] == 1.0  # each float32 add rounds back to 1 (ties to even)
    assert v64[0] == 1.0 + 2.0 ** -23


def test_coo_keeps_explicit_zeros_and_empty_rows():
    row = np.array([2, 0], dtype=np.int32)
    col = np.array([1, 0], dtype=np.int32)
    val = np.array([0.0, 5.0])
    rp, ci, va = oracle.coo_to_csr(4, 2, row, col, val)
    assert rp.tolist() == [0, 1, 1, 2, 2]
    assert ci.tolist() == [0, 1] and va.tolist() == [5.0, 0.0]


def test_coo_permutation_gives_same_csr():
    m = W.power_law(2000, seed=3)
    rows = np.repeat(np.arange(m.n), m.row_lengths()).astype(np.int32)
    perm = np.random.default_rng(1).permutation(m.nnz)
    rp, ci, va = oracle.coo_to_csr(m.n, m.ncols, rows[perm], m.col_idx[perm], m.values[perm])
    assert np.array_equal(rp, m.row_ptr) and np.array_equal(ci, m.col_idx)
    assert np.array_equal(va, m.values)


def test_coo_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.coo_to_csr(2, 2, np.array([0, 2]), np.array([0, 0]), np.ones(2))


# --------------------------------------------------------- ELL / SELL-P

def _golden_layout():
    with open(os.path.join(GOLDEN, "layout_5x4.json")) as f:
        g = json.load(f)
    m = _csr(g["n"], g["ncols"], g["row_ptr"], g["col_idx"], g["values"])
    return g, m


def test_ell_golden_layout():
    g, m = _golden_layout()
    K, stride, ec, ev = oracle.csr_to_ell(m)
    assert K == g["ell"]["K"] and stride == g["ell"]["stride"]
    ec, ev = ec.reshape(K, stride), ev.reshape(K, stride)
    assert ec[:, :m.n].tolist() == g["ell"]["col_first_n_per_k"]
    assert ev[:, :m.n].tolist() == g["ell"]["val_first_n_per_k"]
    assert np.all(ec[:, m.n:] == -1) and np.all(ev[:, m.n:] == 0.0)
    assert not np.any(np.signbit(ev[ec < 0]))  # padding is +0.0


def test_sellp_golden_layout():
    g, m = _golden_layout()
    sl, ss, sc, sv = oracle.csr_to_sellp(m, S=2, f=2)
    gs = g["sellp_S2_f2"]
    assert sl.tolist() == gs["slice_lengths"] and ss.tolist() == gs["slice_sets"]
    assert sc.tolist() == gs["col"] and sv.tolist() == gs["val"]


@pytest.mark.parametrize("S,f", [(32, 1), (8, 2), (16, 4), (64, 1), (1, 1)])
def test_round_trips(S, f):
    for m in (W.random_csr(70, 90, 0.1, 11, empty_rows=9, full_rows=1),
              W.power_law(3000, seed=5), W.laplacian_2d(9, 5)):
        sl, ss, sc, sv = oracle.csr_to_sellp(m, S, f)
        assert np.all(sl % f == 0)
        rp, ci, va = oracle.sellp_to_csr(m.n, S, sl, ss, sc, sv)
        assert np.array_equal(rp, m.row_ptr) and np.array_equal(ci, m.col_idx)
        assert np.array_equal(va, m.values)
        K, st, ec, ev = oracle.csr_to_ell(m)
        assert K == int(m.row_lengths().max())
        rp, ci, va = oracle.ell_to_csr(m.n, K, st, ec, ev)
        assert np.array_equal(rp, m.row_ptr) and np.array_equal(ci, m.col_idx)
        assert np.array_equal(va, m.values)


# --------------------------------------------------------------- Jacobi

def test_jacobi_values_and_errors():
    m = W.diffusion_3d(6)
    d = oracle.jacobi(m)
    assert np.allclose(d * np.diag(m.to_dense()), 1.0, rtol=0, atol=1e-15)
    bad = _csr(2, 2, [0, 1, 2], [0, 1], [1.0, 0.0])
    with pytest.raises(ZeroDivisionError):
        oracle.jacobi(bad)
    missing = _csr(2, 2, [0, 1, 2], [0, 0], [1.0, 3.0])
    with pytest.raises(ZeroDivisionError):
        oracle.jacobi(missing)


# --------------------------------------------------------------- solvers

def _spd_dense_csr(n, cond, seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    a = (q * ev) @ q.T
    a = 0.5 * (a + a.T)
    rp = np.arange(0, n * n + 1, n)
    ci = np.tile(np.arange(n), n)
    return _csr(n, n, rp, ci, a.reshape(-1)), a


def _dense_csr(a):
    n = a.shape[0]
    rp = np.arange(0, n * n + 1, n)
    ci = np.tile(np.arange(n), n)
    return _csr(n, n, rp, ci, a.reshape(-1))


@pytest.mark.parametrize("precond", [0, 1])
def test_cg_matches_lapack(precond):
    m = W.shifted_rectangle(11, 13, 0.3)
    b = W.uniform_vector(m.n, 1)
    x, info = oracle.solve(m, b, method=oracle.CG, precond=precond, tol=1e-12)
    xs = np.linalg.solve(m.to_dense(), b)
    assert info["status"] == oracle.OK
    kappa = np.linalg.cond(m.to_dense())
    assert np.linalg.norm(x - xs) <= kappa * 1e-12 * np.linalg.norm(xs) * 2
    assert oracle.true_rel_residual(m, b, x) <= 1e-12


@pytest.mark.parametrize("n,seed", [(5, 1), (12, 2), (16, 3)])
def test_cg_exact_termination(n, seed):
    """CG on an n x n SPD system terminates in n steps in exact arithmetic;
    with kappa = 10 rounding costs at most two more."""
    m, a = _spd_dense_csr(n, 10.0, seed)
    b = np.random.default_rng(seed).standard_normal(n)
    x, info = oracle.solve(m, b, method=oracle.CG, tol=1e-12, max_iters=n + 2)
    assert info["status"] == oracle.OK and info["iters"] <= n + 2


def test_cg_eigenvector_rhs_one_iteration():
    N = 20
    m = W.laplacian_1d(N)
    i = np.arange(1, N + 1)
    b = np.sin(i * 3 * math.pi / (N + 1))
    x, info = oracle.solve(m, b, method=oracle.CG, tol=1e-12)
    assert info["status"] == oracle.OK and info["iters"] == 1


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_cg_k_distinct_eigenvalues(k):
    n = 40
    vals = np.repeat(np.arange(1.0, k + 1.0), n // k + 1)[:n] * 1.7
    m = _csr(n, n, np.arange(n + 1), np.arange(n), vals)
    b = np.random.default_rng(k).standard_normal(n)
    x, info = oracle.solve(m, b, method=oracle.CG, tol=1e-12)
    assert info["status"] == oracle.OK and info["iters"] <= k + 1


def test_jacobi_cg_diagonal_one_iteration():
    n = 30
    vals = np.linspace(0.5, 50.0, n)
    m = _csr(n, n, np.arange(n + 1), np.arange(n), vals)
    b = np.random.default_rng(2).standard_normal(n)
    x, info = oracle.solve(m, b, method=oracle.CG, precond=1, tol=1e-13)
    assert info["status"] == oracle.OK and info["iters"] == 1
    assert np.allclose(x, b / vals, rtol=1e-15, atol=0)


def test_cg_breakdown_on_negative_definite():
    n = 5
    m = _csr(n, n, np.arange(n + 1), np.arange(n), -np.ones(n))
    _, info = oracle.solve(m, np.ones(n), method=oracle.CG)
    assert info["status"] == oracle.BREAKDOWN


@pytest.mark.parametrize("method", [oracle.CG, oracle.BICGSTAB, oracle.GMRES, oracle.CGS])
def test_zero_rhs_returns_zero(method):
    m = W.laplacian_2d(5)
    x, info = oracle.solve(m, np.zeros(m.n), x0=np.ones(m.n), method=method)
    assert info["status"] == oracle.OK and info["iters"] == 0 and np.all(x == 0)


def test_cg_config1_iteration_bound_and_residuals():
    """64x64 5-point Laplacian: kappa from the closed-form extreme
    eigenvalues gives the CG A-norm bound 2((sqrt k - 1)/(sqrt k + 1))^it."""
    N = 64
    m = W.laplacian_2d(N)
    b = W.uniform_vector(m.n, W.SEED_BASE + 1)
    x, info, hist = oracle.solve(m, b, method=oracle.CG, tol=1e-10, max_iters=2000,
                                 history=True)
    lmin = 8 * math.sin(math.pi / (2 * (N + 1))) ** 2
    lmax = 8 * math.sin(N * math.pi / (2 * (N + 1))) ** 2
    kappa = lmax / lmin
    q = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    bound = math.ceil(math.log(1e-10 / 2) / math.log(q))
    assert info["status"] == oracle.OK
    assert info["iters"] <= bound + 80
    assert info["rel_res_true"] <= 1e-10
    # recurrence residual tracks the recomputed true residual
    assert abs(info["rel_res_true"] - info["rel_res_rec"]) <= 1e-12


def test_residual_replacement_restart_reaches_tol():
    """A tolerance near the rounding floor: the recurrence residual keeps
    falling while the true one stalls; the replacement restart must still
    return only with the true residual passing, or report non-convergence."""
    m = W.diffusion_3d(8, sigma=2.0, seed=9)
    b = W.uniform_vector(m.n, 9)
    x, info = oracle.solve(m, b, method=oracle.CG, tol=1e-15, max_iters=3000)
    if info["status"] == oracle.OK:
        assert oracle.true_rel_residual(m, b, x) <= 1e-15 * 1.0001
    else:
        assert info["status"] == oracle.NOT_CONVERGED


def _convdiff_1d(n, peclet):
    """Upwind-free central 1D convection-diffusion: nonsymmetric tridiagonal."""
    lo, di, up = -1.0 - peclet, 2.0, -1.0 + peclet
    rp = [0]
    ci, va = [], []
    for i in range(n):
        if i > 0:
            ci.append(i - 1); va.append(lo)
        ci.append(i); va.append(di)
        if i < n - 1:
            ci.append(i + 1); va.append(up)
        rp.append(len(ci))
    return _csr(n, n, rp, ci, va)


@pytest.mark.parametrize("precond", [0, 1])
def test_bicgstab_matches_lapack(precond):
    m = _convdiff_1d(60, 0.4)
    b = np.random.default_rng(4).standard_normal(m.n)
    x, info = oracle.solve(m, b, method=oracle.BICGSTAB, precond=precond, tol=1e-12,
                           max_iters=500)
    xs = np.linalg.solve(m.to_dense(), b)
    assert info["status"] == oracle.OK
    kappa = np.linalg.cond(m.to_dense())
    assert np.linalg.norm(x - xs) <= 2 * kappa * 1e-12 * np.linalg.norm(xs)
    assert oracle.true_rel_residual(m, b, x) <= 1e-12


@pytest.mark.parametrize("n,seed", [(10, 1), (25, 2), (30, 3)])
def test_full_gmres_terminates_in_n_steps(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + n * 0.3 * np.eye(n)
    m = _dense_csr(a)
    b = rng.standard_normal(n)
    x, info, hist = oracle.solve(m, b, method=oracle.GMRES, krylov_dim=n, tol=1e-11,
                                 max_iters=n, history=True)
    assert info["status"] == oracle.OK and info["iters"] <= n
    h = hist[1:info["iters"] + 1]
    assert np.all(np.diff(h) <= 1e-15 * np.abs(h[:-1]) + 1e-300)  # non-increasing
    xs = np.linalg.solve(a, b)
    assert np.linalg.norm(x - xs) <= np.linalg.cond(a) * 1e-10 * np.linalg.norm(xs)


@pytest.mark.parametrize("precond", [0, 1])
def test_restarted_gmres_matches_lapack(precond):
    m = _convdiff_1d(80, 0.3)
    b = np.random.default_rng(8).standard_normal(m.n)
    x, info = oracle.solve(m, b, method=oracle.GMRES, precond=precond, krylov_dim=10,
                           tol=1e-11, max_iters=5000)
    assert info["status"] == oracle.OK and info["restarts"] >= 1
    xs = np.linalg.solve(m.to_dense(), b)
    assert np.linalg.norm(x - xs) <= 2 * np.linalg.cond(m.to_dense()) * 1e-11 * np.linalg.norm(xs)
    assert oracle.true_rel_residual(m, b, x) <= 1e-11


def test_gmres_givens_estimate_equals_true_residual_in_cycle():
    """Inside a cycle, |g_{k+1}| equals ||b - A x_k|| in exact arithmetic;
    with full GMRES on a well-conditioned system they agree to rounding."""
    n = 20
    rng = np.random.default_rng(5)
    a = rng.standard_normal((n, n)) + 2 * math.sqrt(n) * np.eye(n)
    m = _dense_csr(a)
    b = rng.standard_normal(n)
    for steps in (3, 7, 12):
        x, info = oracle.solve(m, b, method=oracle.GMRES, krylov_dim=n, tol=1e-30,
                               max_iters=steps)
        assert info["iters"] == steps
        true = np.linalg.norm(b - a @ x) / np.linalg.norm(b)
        assert abs(info["rel_res_rec"] - true) <= 1e-12


def test_solvers_jacobi_on_diffusion_reach_tol():
    m = W.diffusion_3d(10)
    b = W.uniform_vector(m.n, 3)
    for method in (oracle.CG, oracle.BICGSTAB, oracle.GMRES, oracle.CGS):
        x, info = oracle.solve(m, b, method=method, precond=1, tol=1e-10, max_iters=5000)
        assert info["status"] == oracle.OK, (method, info)
        assert oracle.true_rel_residual(m, b, x) <= 1e-10


# ---------------------------------------------------------------- CGS pins


@pytest.mark.parametrize("precond", [0, 1])
def test_cgs_matches_lapack(precond):
    """CGS on the nonsymmetric 1D convection-diffusion system reaches the
    dense LU solution within kappa * tol."""
    m = _convdiff_1d(60, 0.4)
    b = np.random.default_rng(6).standard_normal(m.n)
    x, info = oracle.solve(m, b, method=oracle.CGS, precond=precond, tol=1e-12, max_iters=500)
    xs = np.linalg.solve(m.to_dense(), b)
    assert info["status"] == oracle.OK
    kappa = np.linalg.cond(m.to_dense())
    assert np.linalg.norm(x - xs) <= 2 * kappa * 1e-12 * np.linalg.norm(xs)
    assert oracle.true_rel_residual(m, b, x) <= 1e-12


@pytest.mark.parametrize("n,seed", [(8, 1), (12, 2)])
def test_cgs_finite_termination(n, seed):
    """CGS squares the BiCG residual polynomial; BiCG ends in at most n steps
    in exact arithmetic, so a well-conditioned nonsymmetric n x n system
    reaches 1e-11 in n (+2 for rounding) iterations."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) * 0.2 + 3.0 * np.eye(n)
    m = _dense_csr(a)
    b = rng.standard_normal(n)
    x, info = oracle.solve(m, b, method=oracle.CGS, tol=1e-11, max_iters=n + 2)
    assert info["status"] == oracle.OK and info["iters"] <= n + 2
    xs = np.linalg.solve(a, b)
    assert np.linalg.norm(x - xs) <= np.linalg.cond(a) * 1e-10 * np.linalg.norm(xs)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_cgs_residual_is_squared_cg_polynomial(k):
    """For SPD A with shadow residual r_0, BiCG is CG, and the CGS residual
    after k steps is P_k(A)^2 r_0 where P_k(A) r_0 is the CG residual.  On a
    diagonal A the polynomial is read per eigenvalue: P_k(l_i) = r^CG_i / r0_i,
    and r^CGS_i must equal P_k(l_i)^2 r0_i (a wrong alpha or beta breaks it)."""
    n = 8
    lam = np.linspace(1.0, 3.0, n)
    m = _csr(n, n, np.arange(n + 1), np.arange(n), lam)
    b = np.random.default_rng(10 + k).uniform(0.5, 1.5, n)
    x_cg, i_cg = oracle.solve(m, b, method=oracle.CG, tol=1e-30, max_iters=k)
    x_cgs, i_cgs = oracle.solve(m, b, method=oracle.CGS, tol=1e-30, max_iters=k)
    assert i_cg["iters"] == k and i_cgs["iters"] == k
    pk = (b - lam * x_cg) / b
    r_cgs = b - lam * x_cgs
    assert np.allclose(r_cgs, pk * pk * b, rtol=1e-9, atol=1e-12 * np.linalg.norm(b))


def test_jacobi_cgs_diagonal_one_iteration():
    n = 30
    d = np.linspace(1.0, 50.0, n)
    m = _csr(n, n, np.arange(n + 1), np.arange(n), d)
    b = np.random.default_rng(3).standard_normal(n)
    x, info = oracle.solve(m, b, method=oracle.CGS, precond=1, tol=1e-12)
    assert info["status"] == oracle.OK and info["iters"] == 1
    assert np.allclose(x, b / d, rtol=1e-15, atol=0)


# ---------------------------------------------------------------- COO SpMV pins


@pytest.mark.parametrize("seed,n,ncols,nnz", [(1, 1, 1, 1), (2, 17, 9, 40), (3, 64, 70, 300),
                                               (4, 50, 50, 0)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.5, 2.0)])
def test_coo_spmv_matches_dense_matvec(seed, n, ncols, nnz, alpha, beta):
    """Unsorted triplets with duplicates and empty rows: the COO SpMV equals
    alpha * D x + beta * y for the densified D (duplicates add)."""
    rng = np.random.default_rng(seed)
    row = rng.integers(0, n, nnz)
    col = rng.integers(0, ncols, nnz)
    val = rng.standard_normal(nnz)
    d = np.zeros((n, ncols))
    np.add.at(d, (row, col), val)
    x = rng.standard_normal(ncols)
    y = rng.standard_normal(n)
    got = oracle.spmv_coo(n, ncols, row, col, val, x, alpha, beta, y=y)
    ref = alpha * (d @ x) + beta * y
    scale = np.abs(alpha) * (np.abs(d) @ np.abs(x)) + np.abs(beta) * np.abs(y)
    assert np.all(np.abs(got - ref) <= 1e-14 * scale + 1e-300)


def test_coo_spmv_integer_exact_and_rejects_out_of_range():
    m = W.laplacian_2d(12)
    row = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    x = (np.arange(m.n) % 7).astype(np.float64)
    got = oracle.spmv_coo(m.n, m.n, row, m.col_idx, m.values, x, compensated=False)
    ref = m.to_dense() @ x  # integers: exact in either order
    assert np.array_equal(got, ref)
    with pytest.raises(ValueError):
        oracle.spmv_coo(3, 3, [0, 3], [0, 0], [1.0, 1.0], np.ones(3))


# ---------------------------------------------------------------- block-Jacobi pins


@pytest.mark.parametrize("n,bs", [(40, 4), (37, 8), (5, 8), (64, 1)])
def test_block_jacobi_blocks_are_numpy_inverses(n, bs):
    """Each stored block is the inverse (numpy LAPACK) of A's dense diagonal
    block over bs rows, the short last block included."""
    m = W.banded_spd(n, 5, 7)
    binv = oracle.block_jacobi(m, bs)
    d = m.to_dense()
    for kb in range(binv.shape[0]):
        r0 = kb * bs
        k = min(bs, n - r0)
        want = np.linalg.inv(d[r0:r0 + k, r0:r0 + k])
        assert np.allclose(binv[kb, :k, :k], want, rtol=1e-12, atol=1e-14)
        assert np.all(binv[kb, k:, :] == 0) and np.all(binv[kb, :, k:] == 0)
    r = np.random.default_rng(n).standard_normal(n)
    z = oracle.block_jacobi_apply(n, bs, binv, r)
    zz = np.concatenate([binv[kb, :min(bs, n - kb * bs), :min(bs, n - kb * bs)] @
                         r[kb * bs:kb * bs + min(bs, n - kb * bs)] for kb in range(binv.shape[0])])
    assert np.allclose(z, zz, rtol=1e-14, atol=1e-15)


def test_block_jacobi_pivots_and_rejects_singular_blocks():
    # a block with a zero diagonal needs a row exchange: [[0, 2], [3, 0]]
    m = _csr(2, 2, [0, 1, 2], [1, 0], [2.0, 3.0])
    binv = oracle.block_jacobi(m, 2)
    assert np.allclose(binv[0], np.linalg.inv(np.array([[0.0, 2.0], [3.0, 0.0]])), rtol=0, atol=1e-15)
    with pytest.raises(ZeroDivisionError):  # the same matrix has zero diagonals for Jacobi
        oracle.jacobi(m)
    sing = _csr(2, 2, [0, 2, 4], [0, 1, 0, 1], [1.0, 2.0, 2.0, 4.0])
    with pytest.raises(ZeroDivisionError):
        oracle.block_jacobi(sing, 2)
    x, info = oracle.solve(sing, np.ones(2), precond=2, block_size=2)
    assert info["status"] == oracle.ERR_ZERO_DIAG


def test_block_size_one_is_jacobi():
    m = W.diffusion_3d(6)
    b = W.uniform_vector(m.n, 2)
    assert np.array_equal(oracle.block_jacobi(m, 1).reshape(-1), oracle.jacobi(m))
    for method in (oracle.CG, oracle.GMRES):
        x1, i1 = oracle.solve(m, b, method=method, precond=1, tol=1e-10, max_iters=2000)
        x2, i2 = oracle.solve(m, b, method=method, precond=2, block_size=1, tol=1e-10,
                              max_iters=2000)
        assert np.array_equal(x1, x2) and i1["iters"] == i2["iters"]


def test_block_jacobi_exact_on_block_diagonal_matrix():
    """When A is block diagonal with blocks of bs rows, block-Jacobi is A^-1:
    preconditioned CG, BiCGSTAB, CGS and GMRES converge in one step."""
    rng = np.random.default_rng(9)
    bs, nb = 4, 6
    d = np.zeros((bs * nb, bs * nb))
    for k in range(nb):
        q = rng.standard_normal((bs, bs))
        d[k * bs:(k + 1) * bs, k * bs:(k + 1) * bs] = q @ q.T + bs * np.eye(bs)
    m = _dense_csr(d)
    b = rng.standard_normal(bs * nb)
    for method in (oracle.CG, oracle.BICGSTAB, oracle.CGS, oracle.GMRES):
        x, info = oracle.solve(m, b, method=method, precond=2, block_size=bs, tol=1e-12)
        assert info["status"] == oracle.OK and info["iters"] == 1, (method, info)
        assert np.allclose(x, np.linalg.solve(d, b), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("method", [oracle.CG, oracle.BICGSTAB, oracle.CGS, oracle.GMRES])
def test_block_jacobi_solvers_reach_tol(method):
    m = W.diffusion_3d(10)
    b = W.uniform_vector(m.n, 3)
    x, info = oracle.solve(m, b, method=method, precond=2, block_size=8, tol=1e-10, max_iters=5000)
    assert info["status"] == oracle.OK, info
    assert oracle.true_rel_residual(m, b, x) <= 1e-10


# ----------------------------------------------------------------- ILU(0)

def _split_lu(m, lu):
    """Dense unit-lower L and upper U from factors stored in m's pattern."""
    n = m.n
    L = np.eye(n)
    U = np.zeros((n, n))
    rows = np.repeat(np.arange(n), m.row_lengths())
    for r, c, v in zip(rows, m.col_idx, lu):
        if c < r:
            L[r, c] = v
        else:
            U[r, c] = v
    return L, U


def _pattern(m):
    rows = np.repeat(np.arange(m.n), m.row_lengths())
    P = np.zeros((m.n, m.ncols), dtype=bool)
    P[rows, m.col_idx] = True
    return P


def test_ilu0_1d_laplacian_closed_form():
    # tridiag(-1, 2, -1): no fill, so ILU(0) is the exact LU with
    # u_ii = (i + 2) / (i + 1), l_i,i-1 = -i / (i + 1), u_i,i+1 = -1
    n = 40
    m = W.laplacian_1d(n)
    L, U = _split_lu(m, oracle.ilu0(m))
    i = np.arange(n)
    assert np.allclose(np.diag(U), (i + 2) / (i + 1), rtol=1e-15, atol=0)
    assert np.allclose(np.diag(L, -1), -i[1:] / (i[1:] + 1), rtol=1e-15, atol=0)
    assert np.all(np.diag(U, 1) == -1.0)


def test_ilu0_tridiagonal_nonsymmetric_is_exact_solve():
    rng = np.random.default_rng(7)
    n = 30
    lo, up = rng.uniform(-1, 0, n - 1), rng.uniform(-2, 1, n - 1)
    d = 4.0 + rng.uniform(0, 1, n)
    D = np.diag(d) + np.diag(lo, -1) + np.diag(up, 1)
    rp, ci, va = [0], [], []
    for r in range(n):
        for c in range(max(r - 1, 0), min(r + 2, n)):
            ci.append(c)
            va.append(D[r, c])
        rp.append(len(ci))
    m = _csr(n, n, rp, ci, va)
    lu = oracle.ilu0(m)
    L, U = _split_lu(m, lu)
    assert np.allclose(L @ U, D, rtol=0, atol=1e-14)
    r = rng.uniform(-1, 1, n)
    assert np.allclose(oracle.ilu0_apply(m, lu, r), np.linalg.solve(D, r), rtol=1e-12, atol=1e-13)


def test_ilu0_full_pattern_matches_lapack_lu():
    # every entry stored: ILU(0) drops nothing and is Doolittle LU; columns
    # dominated by the diagonal, so LAPACK's partial pivoting swaps no rows
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(11)
    n = 12
    D = rng.uniform(-1, 1, (n, n))
    D[np.arange(n), np.arange(n)] = np.abs(D).sum(axis=0) + 1.0
    rp = np.arange(0, n * n + 1, n)
    ci = np.tile(np.arange(n), n)
    m = _csr(n, n, rp, ci, D.reshape(-1))
    L, U = _split_lu(m, oracle.ilu0(m))
    P, Ls, Us = scipy_linalg.lu(D)
    assert np.array_equal(P, np.eye(n))
    assert np.allclose(L, Ls, rtol=0, atol=1e-14)
    assert np.allclose(U, Us, rtol=1e-14, atol=1e-13)


@pytest.mark.parametrize("dims", [(7, 6), (5, 4, 3)])
def test_ilu0_stencil_recurrence(dims):
    # 5-/7-point Laplacian, natural order, every side >= 3: no two lower
    # neighbours of a row share a stored entry, so ILU(0) reduces to
    # l_ik = -1 / u_kk, u_ij = -1 above the diagonal and
    # u_ii = a_ii - sum over lower neighbours k of 1 / u_kk
    m = W.laplacian_2d(*dims) if len(dims) == 2 else W.laplacian_3d(*dims)
    lu = oracle.ilu0(m)
    u = np.zeros(m.n)
    for i in range(m.n):
        row = slice(m.row_ptr[i], m.row_ptr[i + 1])
        cols, f = m.col_idx[row], lu[row]
        lower = cols < i
        assert np.allclose(f[lower], -1.0 / u[cols[lower]], rtol=1e-15, atol=0)
        assert np.all(f[cols > i] == -1.0)
        expect = 2.0 * len(dims) - np.sum(1.0 / u[cols[lower]])
        u[i] = f[cols == i][0]
        assert u[i] == pytest.approx(expect, rel=1e-15)


@pytest.mark.parametrize("make", [lambda: W.laplacian_2d(8, 7),
                                  lambda: W.convection_diffusion_2d(9, 2.0),
                                  lambda: W.diffusion_3d(5)])
def test_ilu0_reproduces_a_on_its_pattern(make):
    # the defining property: (L U)_ij = a_ij for every stored (i, j); fill
    # outside the pattern is dropped, so L U differs from A somewhere else
    m = make()
    L, U = _split_lu(m, oracle.ilu0(m))
    A = m.to_dense()
    P = _pattern(m)
    LU = L @ U
    assert np.allclose(LU[P], A[P], rtol=0, atol=1e-13 * np.abs(A).max())
    assert np.abs(LU[~P]).max() > 1e-3


def test_ilu0_apply_is_the_two_triangular_solves():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    m = W.convection_diffusion_2d(11, 1.5)
    lu = oracle.ilu0(m)
    L, U = _split_lu(m, lu)
    r = W.uniform_vector(m.n, 5)
    y = scipy_linalg.solve_triangular(L, r, lower=True, unit_diagonal=True)
    z = scipy_linalg.solve_triangular(U, y, lower=False)
    got = oracle.ilu0_apply(m, lu, r)
    assert np.allclose(got, z, rtol=1e-13, atol=1e-14)
    assert np.allclose(L @ (U @ got), r, rtol=0, atol=1e-12)


def _ilu0_textbook(m):
    """ILU(0) in the IKJ order with plain arithmetic: l_ik = a_ik / u_kk
    (a division) and a_ij = a_ij - l_ik * u_kj (a rounded product, then a
    rounded difference), pattern entries only."""
    lu = m.values.astype(np.float64).copy()
    pos = [dict(zip(m.col_idx[m.row_ptr[i]:m.row_ptr[i + 1]].tolist(),
                    range(m.row_ptr[i], m.row_ptr[i + 1]))) for i in range(m.n)]
    for i in range(m.n):
        for k in sorted(c for c in pos[i] if c < i):
            lik = lu[pos[i][k]] / lu[pos[k][k]]
            lu[pos[i][k]] = lik
            for j, pkj in pos[k].items():
                if j > k and j in pos[i]:
                    lu[pos[i][j]] = lu[pos[i][j]] - lik * lu[pkj]
    return lu


def _ilu0_apply_textbook(m, lu, r):
    """Forward then backward substitution, dividing by u_ii."""
    y = np.zeros(m.n)
    for i in range(m.n):
        a, b = m.row_ptr[i], m.row_ptr[i + 1]
        s = r[i]
        for k in range(a, b):
            if m.col_idx[k] < i:
                s = s - lu[k] * y[m.col_idx[k]]
        y[i] = s
    z = np.zeros(m.n)
    for i in reversed(range(m.n)):
        a, b = m.row_ptr[i], m.row_ptr[i + 1]
        s, d = y[i], None
        for k in range(a, b):
            c = m.col_idx[k]
            if c > i:
                s = s - lu[k] * z[c]
            elif c == i:
                d = lu[k]
        z[i] = s / d
    return z


@pytest.mark.parametrize("make", [lambda: W.diffusion_3d(6),
                                  lambda: W.convection_diffusion_2d(12, 2.0),
                                  lambda: W.banded_spd(150, 6, 4),
                                  lambda: W.power_law(300, max_len=40, seed=5)])
def test_ilu0_fused_rounding_is_within_rounding_of_textbook(make):
    """The oracle's ILU(0) takes each update as one fused multiply-add and
    scales by a reciprocal pivot; the textbook form divides and rounds the
    product separately.  Both are the same algorithm: factors and the
    application agree to a few units of rounding (relative to the row's
    magnitude), so the rounding reading cannot hide a wrong index, sign or
    dropped term."""
    m = make()
    if m.name.startswith("powerlaw"):
        # a diagonally dominant nonsymmetric matrix on the power-law pattern
        # plus the diagonal
        d = m.to_dense()
        d[np.arange(m.n), np.arange(m.n)] = np.abs(d).sum(axis=1) + 1.0
        rows, cols = np.nonzero(d)
        rp = np.zeros(m.n + 1, np.int64)
        np.add.at(rp, rows + 1, 1)
        m = W.CSR(m.n, m.n, np.cumsum(rp), cols, d[rows, cols])
    lu = oracle.ilu0(m)
    ref = _ilu0_textbook(m)
    rows = np.repeat(np.arange(m.n), m.row_lengths())
    rowmax = np.zeros(m.n)
    np.maximum.at(rowmax, rows, np.abs(ref))
    assert np.all(np.abs(lu - ref) <= 1e-13 * rowmax[rows])
    r = W.uniform_vector(m.n, 6)
    z = oracle.ilu0_apply(m, lu, r)
    zt = _ilu0_apply_textbook(m, ref, r)
    assert np.allclose(z, zt, rtol=1e-12, atol=1e-13 * np.abs(zt).max())


def test_ilu0_errors():
    # missing diagonal
    with pytest.raises(ZeroDivisionError):
        oracle.ilu0(_csr(2, 2, [0, 1, 2], [1, 0], [1.0, 1.0]))
    # the elimination creates a zero pivot: [[1, 1], [1, 1]]
    with pytest.raises(ZeroDivisionError):
        oracle.ilu0(_csr(2, 2, [0, 2, 4], [0, 1, 0, 1], [1.0, 1.0, 1.0, 1.0]))
    # columns not ascending within a row
    with pytest.raises(ValueError):
        oracle.ilu0(_csr(2, 2, [0, 2, 3], [1, 0, 1], [1.0, 2.0, 3.0]))
    # duplicates are rejected too
    with pytest.raises(ValueError):
        oracle.ilu0(_csr(1, 1, [0, 2], [0, 0], [1.0, 2.0]))


def test_ilu_cg_beats_jacobi_cg_on_laplacian():
    m = W.laplacian_2d(32)
    b = W.uniform_vector(m.n, 2)
    x1, i1 = oracle.solve(m, b, method=oracle.CG, precond=1, tol=1e-10)
    x3, i3 = oracle.solve(m, b, method=oracle.CG, precond=3, tol=1e-10)
    assert i1["status"] == oracle.OK and i3["status"] == oracle.OK
    assert oracle.true_rel_residual(m, b, x3) <= 1e-10
    assert i3["iters"] < 0.7 * i1["iters"], (i1["iters"], i3["iters"])


@pytest.mark.parametrize("method", [oracle.BICGSTAB, oracle.CGS, oracle.GMRES])
def test_ilu_solvers_on_convection_diffusion(method):
    m = W.convection_diffusion_2d(24, 3.0)
    b = W.uniform_vector(m.n, 4)
    x0, i0 = oracle.solve(m, b, method=method, precond=1, tol=1e-10, max_iters=4000)
    x, info = oracle.solve(m, b, method=method, precond=3, tol=1e-10, max_iters=4000)
    assert info["status"] == oracle.OK, info
    assert oracle.true_rel_residual(m, b, x) <= 1e-10
    assert info["iters"] < i0["iters"], (i0["iters"], info["iters"])


# ----------------------------------------------------------------- triangular solves

@pytest.mark.parametrize("upper", [False, True])
@pytest.mark.parametrize("unit", [False, True])
def test_trsv_matches_lapack_triangular_solve(upper, unit):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    m = W.convection_diffusion_2d(13, 2.0)
    D = m.to_dense()
    T = np.triu(D) if upper else np.tril(D)
    if unit:
        np.fill_diagonal(T, 1.0)
    b = W.uniform_vector(m.n, 31)
    want = scipy_linalg.solve_triangular(T, b, lower=not upper, unit_diagonal=unit)
    got = oracle.trsv(m, b, upper=upper, unit=unit)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-14)
    # residual relative to |T| |x| + |b| (a unit triangle with -3 below the
    # diagonal grows x like 3^n)
    assert np.all(np.abs(T @ got - b) <= 1e-13 * (np.abs(T) @ np.abs(got) + np.abs(b)))


def test_trsv_closed_form_bidiagonal():
    # lower bidiagonal with 1 on the diagonal and -1 below: x_i = b_0 + ... + b_i
    n = 50
    rows, cols, vals = [], [], []
    for i in range(n):
        if i > 0:
            rows.append(i); cols.append(i - 1); vals.append(-1.0)
        rows.append(i); cols.append(i); vals.append(1.0)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    m = _csr(n, n, rp, cols, vals)
    b = np.arange(1.0, n + 1)
    assert np.array_equal(oracle.trsv(m, b), np.cumsum(b))
    # the same matrix's upper triangle is the identity
    assert np.array_equal(oracle.trsv(m, b, upper=True), b)


def test_trsv_on_ilu_factors_is_ilu_apply():
    # L y = r with unit diagonal, then U z = y: the two substitutions of ILU(0)
    m = W.laplacian_2d(9, 7)
    lu = oracle.ilu0(m)
    F = W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx, lu)
    r = W.uniform_vector(m.n, 4)
    z = oracle.trsv(F, oracle.trsv(F, r, upper=False, unit=True), upper=True)
    assert np.array_equal(z, oracle.ilu0_apply(m, lu, r))


def test_trsv_errors():
    with pytest.raises(ValueError):  # missing diagonal
        oracle.trsv(_csr(2, 2, [0, 1, 2], [1, 0], [1.0, 1.0]), np.ones(2))
    with pytest.raises(ZeroDivisionError):
        oracle.trsv(_csr(2, 2, [0, 1, 2], [0, 1], [0.0, 1.0]), np.ones(2))
    # a zero diagonal is fine with a unit diagonal
    x = oracle.trsv(_csr(2, 2, [0, 1, 3], [0, 0, 1], [0.0, 2.0, 0.0]), np.ones(2), unit=True)
    assert np.array_equal(x, [1.0, -1.0])
