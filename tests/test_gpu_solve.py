"""GPU Krylov solvers against the CPU oracle, through the C ABI.

Solver parity (several iterates are correct, rounding differs): (i) the
true relative residual ||b - A x|| / ||b||, recomputed by the oracle's FP64
SpMV from the GPU's x, is <= tol; (ii) the iteration count is within
max(3, 10 %) of the oracle's for CG and within max(one restart cycle,
10 %) for GMRES.  ||x - x_oracle|| / ||x_oracle|| is reported, not gated."""
import numpy as np
import pytest

import oracle
import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W
from gpu_util import ensure_built, torch_dev

pytestmark = pytest.mark.gpu

METHOD = {"cg": oracle.CG, "bicgstab": oracle.BICGSTAB, "gmres": oracle.GMRES, "cgs": oracle.CGS}


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _convdiff_1d(n, peclet):
    lo, di, up = -1.0 - peclet, 2.0, -1.0 + peclet
    rp, ci, va = [0], [], []
    for i in range(n):
        if i > 0:
            ci.append(i - 1); va.append(lo)
        ci.append(i); va.append(di)
        if i < n - 1:
            ci.append(i + 1); va.append(up)
        rp.append(len(ci))
    return W.CSR(n, n, np.array(rp), np.array(ci), np.array(va))


def _gpu_solve(m, b, method, precond, tol, max_iters=5000, fmt="csr", dtype="f64", x0=None,
               engine=0, **kw):
    import torch
    dev = torch_dev()
    A = gk.Matrix.from_csr(m, dtype if dtype != "mixed" else "f64")
    if fmt != "csr":
        B = A.convert(fmt)
        A.close()
        A = B
    vt = torch.float64 if dtype in ("f64", "mixed") else torch.float32
    bt = torch.from_numpy(np.asarray(b)).to(dev, vt)
    xt = torch.zeros(m.n, dtype=vt, device=dev) if x0 is None else \
        torch.from_numpy(np.asarray(x0)).to(dev, vt)
    info = A.solve(bt, xt, method=method, precond=precond, tol=tol, max_iters=max_iters,
                   engine=engine, **kw)
    torch.cuda.synchronize()
    x = xt.cpu().numpy().astype(np.float64)
    A.close()
    return x, info


def _check(m, b, method, precond, tol, fmt="csr", krylov_dim=30, iters_gate=True, **kw):
    x, info = _gpu_solve(m, b, method, 1 if precond else 0, tol, fmt=fmt,
                         krylov_dim=krylov_dim, **kw)
    assert info["return"] == gk.GK_OK, info
    rel = oracle.true_rel_residual(m, b, x)
    assert rel <= tol, (rel, info)
    xo, io = oracle.solve(m, b, method=METHOD[method], precond=1 if precond else 0, tol=tol,
                          max_iters=5000, krylov_dim=krylov_dim)
    assert io["status"] == oracle.OK
    if iters_gate:
        if method == "gmres":
            # one restart cycle, or 10 % when rounding differences between
            # CGS2 (GPU) and MGS (oracle) compound over many cycles
            assert abs(info["iters"] - io["iters"]) <= max(krylov_dim, 0.1 * io["iters"]), (info, io)
        else:
            assert abs(info["iters"] - io["iters"]) <= max(3, 0.1 * io["iters"]), (info, io)
    assert abs(info["rel_res_true"] - rel) <= 1e-3 * max(rel, 1e-16) + 1e-15
    return x, info, xo, io


CASES = {
    "lap2d_64": lambda: (W.laplacian_2d(64), W.uniform_vector(4096, W.SEED_BASE + 1)),
    "diff3d_12": lambda: (W.diffusion_3d(12, seed=4), W.uniform_vector(12 ** 3, 5)),
    "convdiff_300": lambda: (_convdiff_1d(300, 0.3), W.uniform_vector(300, 6)),
    "banded_2000": lambda: (W.banded_spd(2000, 9, 2), W.uniform_vector(2000, 7)),
}


@pytest.mark.parametrize("case", ["lap2d_64", "diff3d_12", "banded_2000"])
@pytest.mark.parametrize("precond", [False, True])
@pytest.mark.parametrize("engine", [1, 2, 3])
def test_cg(case, precond, engine):
    """CG on the multi-kernel (1), single-block (2) and cluster (3) engines."""
    m, b = CASES[case]()
    _check(m, b, "cg", precond, 1e-10, engine=engine)


@pytest.mark.parametrize("n_side", [1, 3, 17, 128])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cluster_engine_sizes(n_side, dtype):
    """Cluster engine from one row up to its 16384-row limit (row slices
    of 1..1024 rows per block)."""
    m = W.shifted_rectangle(n_side, n_side, 0.05)
    b = W.uniform_vector(m.n, 11)
    tol = 1e-10 if dtype == "f64" else 1e-5
    x, info = _gpu_solve(m, b, "cg", 1, tol, dtype=dtype, engine=3)
    assert info["return"] == gk.GK_OK, info
    assert oracle.true_rel_residual(m, b, x) <= (tol if dtype == "f64" else 3e-5)


def test_cluster_engine_rejects_too_large():
    m = W.laplacian_2d(129)  # 16641 rows > 16384
    b = W.uniform_vector(m.n, 1)
    _, info = _gpu_solve(m, b, "cg", 0, 1e-8, engine=3)
    assert info["return"] == gk.GK_ERR_UNSUPPORTED
    x, info = _gpu_solve(m, b, "cg", 0, 1e-8, engine=0)  # automatic: multi-kernel
    assert info["return"] == gk.GK_OK


@pytest.mark.parametrize("case", ["lap2d_64", "diff3d_12", "convdiff_300"])
@pytest.mark.parametrize("precond", [False, True])
def test_bicgstab(case, precond):
    m, b = CASES[case]()
    # BiCGSTAB's iteration count is sensitive to rounding: gate the residual only
    _check(m, b, "bicgstab", precond, 1e-10, iters_gate=False)


@pytest.mark.parametrize("case", ["lap2d_64", "diff3d_12", "convdiff_300", "banded_2000"])
@pytest.mark.parametrize("precond", [False, True])
def test_cgs(case, precond):
    """CGS squares the BiCG residual polynomial, so rounding differences grow
    faster than in CG: the residual is gated, the iteration count only
    loosely (within 1.5x + 10 of the oracle's)."""
    m, b = CASES[case]()
    x, info, xo, io = _check(m, b, "cgs", precond, 1e-10, iters_gate=False)
    assert info["iters"] <= 1.5 * io["iters"] + 10, (info, io)


def test_cgs_rejected_by_single_block_and_batched_engines():
    m, b = CASES["lap2d_64"]()
    _, info = _gpu_solve(m, b, "cgs", 0, 1e-10, engine=2)
    assert info["return"] == gk.GK_ERR_UNSUPPORTED
    import torch
    dev = torch_dev()
    A = gk.Matrix.from_csr(m)
    bt = torch.from_numpy(b).to(dev)
    xt = torch.zeros_like(bt)
    st, _ = gk.gk_solve_batched([A.handle], [bt], [xt], gk.make_opts(method="cgs", tol=1e-10))
    assert st == gk.GK_ERR_UNSUPPORTED
    A.close()


@pytest.mark.parametrize("case", ["lap2d_64", "diff3d_12", "convdiff_300"])
@pytest.mark.parametrize("precond", [False, True])
def test_gmres(case, precond):
    m, b = CASES[case]()
    _check(m, b, "gmres", precond, 1e-10)


@pytest.mark.parametrize("fmt", ["ell", "sellp"])
@pytest.mark.parametrize("method", ["cg", "bicgstab", "gmres", "cgs"])
def test_solvers_on_padded_formats(fmt, method):
    m, b = CASES["diff3d_12"]()
    _check(m, b, method, True, 1e-10, fmt=fmt, iters_gate=(method not in ("bicgstab", "cgs")))


def test_small_gmres_restart_length():
    m, b = CASES["convdiff_300"]()
    x, info, _, io = _check(m, b, "gmres", False, 1e-10, krylov_dim=8)
    assert info["restarts"] >= 1


def test_dense_solution_matches_lapack():
    m = W.shifted_rectangle(9, 11, 0.5)
    b = W.uniform_vector(m.n, 3)
    xs = np.linalg.solve(m.to_dense(), b)
    kappa = np.linalg.cond(m.to_dense())
    for method in ("cg", "bicgstab", "gmres"):
        x, info = _gpu_solve(m, b, method, 0, 1e-12)
        assert info["return"] == gk.GK_OK
        assert np.linalg.norm(x - xs) <= 2 * kappa * 1e-12 * np.linalg.norm(xs)


@pytest.mark.parametrize("method", ["cg", "bicgstab", "gmres", "cgs"])
def test_zero_rhs(method):
    m = W.laplacian_2d(10)
    x, info = _gpu_solve(m, np.zeros(m.n), method, 0, 1e-10, x0=np.ones(m.n))
    assert info["return"] == gk.GK_OK and info["iters"] == 0 and np.all(x == 0)


def test_zero_diagonal_rejected():
    m = W.CSR(3, 3, np.array([0, 1, 2, 3]), np.array([0, 1, 0]), np.array([1.0, 2.0, 3.0]))
    _, info = _gpu_solve(m, np.ones(3), "cg", 1, 1e-10)
    assert info["return"] == gk.GK_ERR_ZERO_DIAG


def test_cg_breakdown_on_indefinite():
    n = 6
    m = W.CSR(n, n, np.arange(n + 1), np.arange(n), -np.ones(n))
    _, info = _gpu_solve(m, np.ones(n), "cg", 0, 1e-10)
    assert info["return"] == gk.GK_BREAKDOWN


@pytest.mark.parametrize("method", ["cg", "bicgstab", "gmres", "cgs"])
def test_iteration_cap(method):
    m, b = CASES["lap2d_64"]()
    x, info = _gpu_solve(m, b, method, 0, 1e-12, max_iters=7)
    assert info["return"] == gk.GK_NOT_CONVERGED and info["iters"] == 7
    rel = oracle.true_rel_residual(m, b, x)
    assert abs(rel - info["rel_res_true"]) <= 1e-6 * rel
    # x holds the last iterate: same residual as the oracle after 7 steps
    xo, io = oracle.solve(m, b, method=METHOD[method], tol=1e-12, max_iters=7)
    assert abs(io["rel_res_true"] - rel) <= 1e-6 * rel


def test_nonzero_initial_guess():
    m, b = CASES["diff3d_12"]()
    x0 = W.uniform_vector(m.n, 99)
    x, info = _gpu_solve(m, b, "cg", 1, 1e-10, x0=x0)
    assert info["return"] == gk.GK_OK and oracle.true_rel_residual(m, b, x) <= 1e-10


def test_solve_deterministic():
    m, b = CASES["diff3d_12"]()
    x1, i1 = _gpu_solve(m, b, "cg", 1, 1e-10)
    x2, i2 = _gpu_solve(m, b, "cg", 1, 1e-10)
    assert np.array_equal(x1, x2) and i1["iters"] == i2["iters"]


@pytest.mark.parametrize("method", ["cg", "bicgstab", "gmres", "cgs"])
def test_fp32_solve(method):
    m, b = CASES["diff3d_12"]()
    x, info = _gpu_solve(m, b, method, 1, 1e-5, dtype="f32")
    assert info["return"] == gk.GK_OK
    assert oracle.true_rel_residual(m, b, x) <= 2e-5  # FP32-rounded A differs from A


@pytest.mark.parametrize("mixed", [1, 2, 3])
@pytest.mark.parametrize("method", ["cg", "gmres", "cgs"])
def test_mixed_precision_refinement(mixed, method):
    """FP32 (or BF16-stored) inner solves inside FP64 refinement reach the
    FP64 tolerance, and x agrees with the plain FP64 solve within kappa*tol."""
    m, b = CASES["diff3d_12"]()
    x, info = _gpu_solve(m, b, method, 1, 1e-10, dtype="mixed", mixed=mixed)
    assert info["return"] == gk.GK_OK, info
    assert info["outer_iters"] >= 1
    assert oracle.true_rel_residual(m, b, x) <= 1e-10
    xo, _ = oracle.solve(m, b, method=METHOD[method], precond=1, tol=1e-12, max_iters=5000)
    kappa = np.linalg.cond(m.to_dense())
    assert np.linalg.norm(x - xo) <= kappa * 2e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("mixed", [1, 2])
def test_refinement_recovers_from_a_wandering_inner_solve(mixed):
    """On the 2D 5-point Laplacian 1024^2 (condition number ~4e5) FP32
    BiCGSTAB inner solves wander and hand back corrections that raise the
    residual; refinement undoes such a correction and finishes in FP64, so
    the solve still reaches the FP64 tolerance (FP64 BiCGSTAB converges)."""
    m = W.laplacian_2d(1024)
    b = W.uniform_vector(m.n, W.SEED_BASE + 3)
    x, info = _gpu_solve(m, b, "bicgstab", 1, 1e-10, max_iters=40000, dtype="mixed", mixed=mixed)
    assert info["return"] == gk.GK_OK, info
    assert info["restarts"] >= 1  # the FP64 finish counts as one
    assert oracle.true_rel_residual(m, b, x) <= 1e-10


def test_refinement_hands_a_stagnating_solve_to_fp64():
    """Block-Jacobi(8) GMRES(30) on the 2D Laplacian 512^2: FP32 inner GMRES
    solves stop early and the refinement gains ~15 % per outer step; after
    three such steps the solve finishes in FP64 (which converges) instead of
    running into the outer cap."""
    m = W.laplacian_2d(512)
    b = W.uniform_vector(m.n, W.SEED_BASE + 3)
    x, info = _gpu_solve(m, b, "gmres", 2, 1e-10, max_iters=20000, dtype="mixed", mixed=1,
                         block_size=8)
    assert info["return"] == gk.GK_OK, info
    assert info["outer_iters"] < 50
    assert oracle.true_rel_residual(m, b, x) <= 1e-10


def test_refinement_default_inner_tolerance_by_method_and_storage():
    """The default inner reduction: 1e-5 for FP32 CG, 1e-2 for GMRES and for
    BF16-stored values (fewer inner iterations, more outer steps); every
    variant reaches the FP64 tolerance."""
    m, b = CASES["diff3d_12"]()
    for method, mixed in (("cg", 1), ("gmres", 1), ("cg", 2)):
        x, info = _gpu_solve(m, b, method, 1, 1e-10, dtype="mixed", mixed=mixed)
        assert info["return"] == gk.GK_OK, (method, mixed, info)
        assert oracle.true_rel_residual(m, b, x) <= 1e-10
        x5, info5 = _gpu_solve(m, b, method, 1, 1e-10, dtype="mixed", mixed=mixed, inner_tol=1e-5)
        x2, info2 = _gpu_solve(m, b, method, 1, 1e-10, dtype="mixed", mixed=mixed, inner_tol=1e-2)
        want = info2 if (mixed == 2 or method == "gmres") else info5
        assert (info["iters"], info["outer_iters"]) == (want["iters"], want["outer_iters"])
        assert np.array_equal(x, x2 if want is info2 else x5)


def test_config3_full_size_jacobi_cg_and_refinement():
    """128^3 log-normal diffusion: Jacobi-CG in FP64 and FP32-refined CG both
    reach a true residual of 1e-10 (oracle SpMV on the GPU's x)."""
    m = W.diffusion_3d(128)
    b = W.uniform_vector(m.n, W.SEED_BASE + 3)
    x, info = _gpu_solve(m, b, "cg", 1, 1e-10, max_iters=20000)
    assert info["return"] == gk.GK_OK
    assert oracle.true_rel_residual(m, b, x) <= 1e-10
    x2, info2 = _gpu_solve(m, b, "cg", 1, 1e-10, max_iters=20000, dtype="mixed", mixed=1)
    assert info2["return"] == gk.GK_OK
    assert oracle.true_rel_residual(m, b, x2) <= 1e-10


def _with_long_row(m, row, width):
    """m plus `width` symmetric entries 1e-3 between `row` and a contiguous
    block of columns far from the band: ELL padding explodes, SELL-P pads
    mostly the one slice holding `row` (the matrix stays SPD: the added
    entries keep it diagonally dominant)."""
    d = m.to_dense()
    cols = np.arange(m.n // 2, m.n // 2 + width)
    assert not np.any(d[row, cols])
    d[row, cols] = d[cols, row] = 1e-3
    return _dense_to_csr(d)


def _dense_to_csr(d):
    rp, ci, va = [0], [], []
    for i in range(d.shape[0]):
        nz = np.flatnonzero(d[i])
        ci.extend(nz.tolist()); va.extend(d[i, nz].tolist())
        rp.append(len(ci))
    return W.CSR(d.shape[0], d.shape[1], np.array(rp), np.array(ci), np.array(va))


def _solve_format(m, **kw):
    import torch
    dev = torch_dev()
    A = gk.Matrix.from_csr(m, "f64")
    assert A.describe()["solve_format"] == -1
    b = torch.from_numpy(W.uniform_vector(m.n, 11)).to(dev)
    x = torch.zeros(m.n, dtype=torch.float64, device=dev)
    info = A.solve(b, x, method="cg", precond=1, tol=1e-10, max_iters=5000, engine=1, **kw)
    fmt = A.describe()["solve_format"]
    A.close()
    return fmt, x.cpu().numpy(), info


def test_solve_format_selection(monkeypatch):
    """Solves on a CSR handle whose plan is the warp-tile kernel (short rows
    of near-uniform length) and which holds at least 2^24 entries run on the
    CSR itself; other CSR handles use ELL when its padding is <= 20 %, else
    SELL-P(32) when its padding is <= 20 %, else the CSR kernels.  The choice
    reads only the pattern, so a matrix always solves the same way
    (bit-reproducible); every choice meets the tolerance.  (The row sums of
    the layouts agree, but the fused dot products add per-thread partials in
    a layout-specific order, so the iterates of different layouts differ in
    rounding.)"""
    import torch
    monkeypatch.delenv("GK_SOLVE_FORMAT", raising=False)
    big = W.laplacian_3d(140)  # 19.1M entries, warp-tile plan
    assert big.nnz >= 1 << 24
    Ab = gk.Matrix.from_csr(big, "f64")
    bb = torch.ones(big.n, dtype=torch.float64, device=torch_dev())
    xb = torch.zeros_like(bb)
    Ab.solve(bb, xb, method="cg", precond="jacobi", tol=1e-10, max_iters=2, engine=1)
    assert Ab.describe()["solve_format"] == gk.GK_CSR
    Ab.close()
    del big, bb, xb
    m, b = CASES["lap2d_64"]()
    fmt, x, info = _solve_format(m)  # warp-tile plan, but small: the ELL copy
    assert fmt == gk.GK_ELL and info["return"] == gk.GK_OK
    assert oracle.true_rel_residual(m, W.uniform_vector(m.n, 11), x) <= 1e-10
    fmt_again, x_again, _ = _solve_format(m)
    assert fmt_again == fmt and np.array_equal(x, x_again)
    xe, ie = _gpu_solve(m, W.uniform_vector(m.n, 11), "cg", 1, 1e-10, fmt="ell", engine=1)
    assert abs(info["iters"] - ie["iters"]) <= max(3, 0.1 * ie["iters"])
    # rows too long for the warp tiles' shared-memory budget (33 entries in
    # FP64): ELL
    mw = W.banded_spd(2000, 16, 3)
    fmtw, xw, infow = _solve_format(mw)
    assert fmtw == gk.GK_ELL and infow["return"] == gk.GK_OK

    m2 = _with_long_row(W.banded_spd(2000, 4, 3), 700, 64)
    fmt2, x2, info2 = _solve_format(m2)
    assert fmt2 == gk.GK_SELLP and info2["return"] == gk.GK_OK
    assert oracle.true_rel_residual(m2, W.uniform_vector(m2.n, 11), x2) <= 1e-10 * 1.01

    m3 = W.power_law(8192)
    A3 = gk.Matrix.from_csr(m3, "f64")
    import torch
    dev = torch_dev()
    b3 = torch.ones(m3.n, dtype=torch.float64, device=dev)
    x3 = torch.zeros_like(b3)
    A3.solve(b3, x3, method="gmres", precond=0, tol=1e-10, max_iters=3, engine=1)
    assert A3.describe()["solve_format"] == gk.GK_CSR  # Zipf rows: padding too large
    A3.close()

    monkeypatch.setenv("GK_SOLVE_FORMAT", "csr")
    fmt4, x4, info4 = _solve_format(m)
    assert fmt4 == gk.GK_CSR and info4["return"] == gk.GK_OK
    assert oracle.true_rel_residual(m, W.uniform_vector(m.n, 11), x4) <= 1e-10
    monkeypatch.setenv("GK_SOLVE_FORMAT", "timed")
    fmt5, x5, info5 = _solve_format(m)
    # the fastest admissible layout (all three are within the padding bound here)
    assert fmt5 in (gk.GK_CSR, gk.GK_ELL, gk.GK_SELLP) and info5["return"] == gk.GK_OK
    assert oracle.true_rel_residual(m, W.uniform_vector(m.n, 11), x5) <= 1e-10


@pytest.mark.parametrize("method", ["cg", "bicgstab", "gmres", "cgs"])
def test_f16_stored_solve(method):
    """A solve on FP16-stored values (FP32 vectors) reaches its tolerance on
    the FP16-rounded system (residual recomputed by the oracle with the
    rounded values); the single-block and cluster engines refuse FP16."""
    m, b = CASES["diff3d_12"]()
    x, info = _gpu_solve(m, b, method, 1, 1e-5, dtype="f16")
    assert info["return"] == gk.GK_OK, info
    m16 = W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx,
                np.asarray(m.values, np.float64).astype(np.float16).astype(np.float64))
    assert oracle.true_rel_residual(m16, b, x) <= 2e-5
    if method == "cg":
        _, i2 = _gpu_solve(m, b, method, 1, 1e-5, dtype="f16", engine=2)
        assert i2["return"] == gk.GK_ERR_UNSUPPORTED


# ---------------------------------------------------------------- block-Jacobi


def _block_diag_csr(bs, nb, seed):
    rng = np.random.default_rng(seed)
    d = np.zeros((bs * nb, bs * nb))
    for k in range(nb):
        q = rng.standard_normal((bs, bs))
        d[k * bs:(k + 1) * bs, k * bs:(k + 1) * bs] = q @ q.T + bs * np.eye(bs)
    n = bs * nb
    return W.CSR(n, n, np.arange(0, n * n + 1, n), np.tile(np.arange(n), n), d.reshape(-1)), d


@pytest.mark.parametrize("method", ["cg", "bicgstab", "cgs", "gmres"])
@pytest.mark.parametrize("case,bs", [("diff3d_12", 8), ("convdiff_300", 5), ("banded_2000", 32)])
def test_block_jacobi_solvers(method, case, bs):
    """Block-Jacobi (diagonal blocks of bs rows) against the oracle: the true
    residual meets tol and the iteration count is close to the oracle's."""
    m, b = CASES[case]()
    if method == "cg" and case == "convdiff_300":
        pytest.skip("CG needs an SPD matrix")
    x, info = _gpu_solve(m, b, method, "block_jacobi", 1e-10, block_size=bs, engine=0)
    assert info["return"] == gk.GK_OK, info
    assert oracle.true_rel_residual(m, b, x) <= 1e-10
    xo, io = oracle.solve(m, b, method=METHOD[method], precond=2, block_size=bs, tol=1e-10,
                          max_iters=5000)
    assert io["status"] == oracle.OK
    assert info["iters"] <= max(io["iters"] + 30, 1.5 * io["iters"]), (info, io)


def test_block_jacobi_exact_on_block_diagonal_and_size_one_is_jacobi():
    m, d = _block_diag_csr(4, 50, 3)
    b = np.random.default_rng(4).standard_normal(m.n)
    for method in ("cg", "bicgstab", "cgs", "gmres"):
        x, info = _gpu_solve(m, b, method, "block_jacobi", 1e-12, block_size=4)
        assert info["return"] == gk.GK_OK and info["iters"] == 1, (method, info)
        assert np.allclose(x, np.linalg.solve(d, b), rtol=1e-11, atol=1e-12)
    mc, bc = CASES["diff3d_12"]()
    _, i1 = _gpu_solve(mc, bc, "cg", 1, 1e-10, engine=1)
    _, i2 = _gpu_solve(mc, bc, "cg", "block_jacobi", 1e-10, block_size=1)
    assert abs(i1["iters"] - i2["iters"]) <= 1, (i1, i2)


def test_block_jacobi_padded_formats_refinement_and_errors():
    m, b = CASES["diff3d_12"]()
    for fmt in ("ell", "sellp"):
        x, info = _gpu_solve(m, b, "cg", "block_jacobi", 1e-10, block_size=6, fmt=fmt)
        assert info["return"] == gk.GK_OK and oracle.true_rel_residual(m, b, x) <= 1e-10
    x, info = _gpu_solve(m, b, "cg", "block_jacobi", 1e-10, block_size=12, dtype="mixed", mixed=1)
    assert info["return"] == gk.GK_OK and oracle.true_rel_residual(m, b, x) <= 1e-10
    for engine in (2, 3):
        _, info = _gpu_solve(m, b, "cg", "block_jacobi", 1e-10, block_size=4, engine=engine)
        assert info["return"] == gk.GK_ERR_UNSUPPORTED
    _, info = _gpu_solve(m, b, "cg", "block_jacobi", 1e-10, block_size=33)
    assert info["return"] == gk.GK_ERR_INVALID
    sing = W.CSR(2, 2, np.array([0, 2, 4]), np.array([0, 1, 0, 1]), np.array([1.0, 2.0, 2.0, 4.0]))
    _, info = _gpu_solve(sing, np.ones(2), "gmres", "block_jacobi", 1e-10, block_size=2)
    assert info["return"] == gk.GK_ERR_ZERO_DIAG
    # a zero diagonal inside a non-singular block is fine for block-Jacobi
    piv = W.CSR(2, 2, np.array([0, 1, 2]), np.array([1, 0]), np.array([2.0, 3.0]))
    x, info = _gpu_solve(piv, np.array([4.0, 9.0]), "gmres", "block_jacobi", 1e-12, block_size=2)
    assert info["return"] == gk.GK_OK and np.allclose(x, [3.0, 2.0])


def test_full_size_gmres_bicgstab_128cubed():
    """GMRES(30) and BiCGSTAB with Jacobi on the full 128^3 diffusion system
    (2,097,152 rows).  Oracle runs of the whole solves are too slow for a
    test, so parity is checked where it is cheap and exact in intent: after
    one full GMRES cycle (30 Arnoldi steps) both minimise the residual over
    the same Krylov space (the GPU with classical Gram-Schmidt applied twice,
    the oracle with modified Gram-Schmidt), so their true residuals agree to
    rounding; after 5 BiCGSTAB iterations the iterates agree to rounding.
    The full solves to 1e-10 must meet the tolerance by the oracle's own
    true residual."""
    import torch
    m = W.diffusion_3d(128)
    b = W.uniform_vector(m.n, W.SEED_BASE + 3)
    dev = torch_dev()
    A = gk.Matrix.from_csr(m)
    bt = torch.from_numpy(b).to(dev)
    x = torch.zeros_like(bt)
    A.solve(bt, x, method="gmres", precond="jacobi", tol=1e-30, max_iters=30, krylov_dim=30)
    xo, io = oracle.solve(m, b, method=oracle.GMRES, precond=1, tol=1e-30, max_iters=30,
                          krylov_dim=30)
    r_gpu = oracle.true_rel_residual(m, b, x.cpu().numpy())
    assert abs(r_gpu - io["rel_res_true"]) <= 1e-8 * io["rel_res_true"], (r_gpu, io)
    x.zero_()
    A.solve(bt, x, method="bicgstab", precond="jacobi", tol=1e-30, max_iters=5)
    xo, io = oracle.solve(m, b, method=oracle.BICGSTAB, precond=1, tol=1e-30, max_iters=5)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)
    for method in ("gmres", "bicgstab"):
        x.zero_()
        info = A.solve(bt, x, method=method, precond="jacobi", tol=1e-10, max_iters=20000)
        assert info["return"] == gk.GK_OK, (method, info)
        assert oracle.true_rel_residual(m, b, x.cpu().numpy()) <= 1e-10, method
    A.close()
