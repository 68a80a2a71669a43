"""ILU(0) on the GPU against the oracle: the factors bit for bit (FP64, and
FP32 / BF16 / FP16 values factored in double and rounded once), the
substitutions z = U^-1 L^-1 r bit for bit in FP64 and within a rounding
bound in FP32, every format, repeated applies, errors, and ILU-
preconditioned CG / BiCGSTAB / CGS / GMRES / refinement."""
import numpy as np
import pytest

import oracle
import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W
from gpu_util import ensure_built, rounded_values, torch_dev

pytestmark = pytest.mark.gpu

METHOD = {"cg": oracle.CG, "bicgstab": oracle.BICGSTAB, "gmres": oracle.GMRES, "cgs": oracle.CGS}


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _dd_random(n, dens, seed):
    """Nonsymmetric, diagonally dominant random sparse matrix (diagonal
    stored), sorted columns."""
    rng = np.random.default_rng(seed)
    m = W.random_csr(n, n, dens, seed)
    d = m.to_dense()
    d[np.arange(n), np.arange(n)] = np.abs(d).sum(axis=1) + 1.0
    rp, ci, va = [0], [], []
    for i in range(n):
        cols = np.nonzero(d[i])[0]
        ci.extend(cols.tolist())
        va.extend(d[i, cols].tolist())
        rp.append(len(ci))
    return W.CSR(n, n, np.array(rp), np.array(ci), np.array(va) * rng.uniform(0.5, 2.0))


CASES = {
    # ragged last chunk (1073 = 33 * 32 + 17 rows)
    "lap2d_37x29": lambda: W.laplacian_2d(37, 29),
    "convdiff_45": lambda: W.convection_diffusion_2d(45, 2.0),
    "diff3d_12": lambda: W.diffusion_3d(12, seed=4),
    "banded_3000": lambda: W.banded_spd(3000, 7, 3),
    "random_700": lambda: _dd_random(700, 0.01, 5),
    "one_row": lambda: W.CSR(1, 1, np.array([0, 1]), np.array([0]), np.array([3.0])),
    "lap1d_33": lambda: W.laplacian_1d(33),
}


def _lu_oracle(m, dtype):
    """The oracle's factors of the values the GPU stores, in the vector type."""
    mr = W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx, rounded_values(m, dtype))
    lu = oracle.ilu0(mr)
    return mr, (lu if dtype == "f64" else lu.astype(np.float32))


def _matrix(m, dtype):
    if dtype in ("f64", "f32"):
        return gk.Matrix.from_csr(m, dtype)
    A = gk.Matrix.from_csr(m, "f64")
    B = A.convert("csr", dtype)
    A.close()
    return B


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f16"])
def test_factors_bit_exact(case, dtype):
    m = CASES[case]()
    A = _matrix(m, dtype)
    got = A.ilu_factors()
    A.close()
    _, want = _lu_oracle(m, dtype)
    assert got.dtype == want.dtype
    assert np.array_equal(got.view(np.uint64 if dtype == "f64" else np.uint32),
                          want.view(np.uint64 if dtype == "f64" else np.uint32)), \
        np.max(np.abs(got - want))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_apply_matches_substitution(case, dtype):
    """FP64: bit for bit the oracle's forward / backward substitution
    (same order of subtractions, separate roundings).  FP32 (substitution
    in float): within 1e-4 relative, plus 1e-7 of the largest entry, of the
    FP64 substitution of the same float factors (the triangular factors of
    these diagonally dominant matrices are well conditioned)."""
    import torch
    dev = torch_dev()
    m = CASES[case]()
    mr, lu = _lu_oracle(m, dtype)
    A = gk.Matrix.from_csr(m, dtype)
    vt = torch.float64 if dtype == "f64" else torch.float32
    rng = np.random.default_rng(9)
    for rep in range(3):  # repeated applies reuse the synchronisation words
        r = rng.uniform(-1, 1, m.n)
        if dtype == "f32":
            r = r.astype(np.float32).astype(np.float64)
        rt = torch.from_numpy(r).to(dev, vt)
        zt = torch.full((m.n,), float("nan"), dtype=vt, device=dev)
        A.precond_apply(rt, zt, "ilu")
        torch.cuda.synchronize()
        z = zt.cpu().numpy()
        want = oracle.ilu0_apply(mr, lu.astype(np.float64), r)
        if dtype == "f64":
            assert np.array_equal(z.view(np.uint64), want.view(np.uint64)), \
                (rep, np.max(np.abs(z - want)))
        else:
            err = np.abs(z.astype(np.float64) - want)
            bound = 1e-4 * np.abs(want) + 1e-7 * np.max(np.abs(want))
            assert np.all(err <= bound), (rep, np.max(err / np.maximum(bound, 1e-300)))
    A.close()


@pytest.mark.parametrize("fmt", ["ell", "sellp", "coo"])
def test_formats_give_the_same_factors(fmt):
    import torch
    dev = torch_dev()
    m = W.convection_diffusion_2d(40, 1.0)
    A = gk.Matrix.from_csr(m, "f64")
    B = A.convert(fmt)
    want = A.ilu_factors()
    assert np.array_equal(B.ilu_factors(), want)
    r = torch.from_numpy(W.uniform_vector(m.n, 3)).to(dev)
    z1 = torch.empty_like(r)
    z2 = torch.empty_like(r)
    A.precond_apply(r, z1, "ilu")
    B.precond_apply(r, z2, "ilu")
    torch.cuda.synchronize()
    assert torch.equal(z1, z2)
    A.close()
    B.close()


def test_other_preconditioners_as_operators():
    import torch
    dev = torch_dev()
    m = W.diffusion_3d(8, seed=2)
    A = gk.Matrix.from_csr(m, "f64")
    r = W.uniform_vector(m.n, 4)
    rt = torch.from_numpy(r).to(dev)
    zt = torch.empty_like(rt)
    A.precond_apply(rt, zt, "none")
    torch.cuda.synchronize()
    assert np.array_equal(zt.cpu().numpy(), r)
    A.precond_apply(rt, zt, "jacobi")
    torch.cuda.synchronize()
    assert np.allclose(zt.cpu().numpy(), oracle.jacobi(m) * r, rtol=1e-15, atol=0)
    A.precond_apply(rt, zt, "block_jacobi", block_size=8)
    torch.cuda.synchronize()
    want = oracle.block_jacobi_apply(m.n, 8, oracle.block_jacobi(m, 8), r)
    assert np.allclose(zt.cpu().numpy(), want, rtol=1e-12, atol=1e-14)
    A.close()


def test_errors():
    import torch
    dev = torch_dev()
    # missing diagonal
    A = gk.Matrix.from_csr(W.CSR(2, 2, np.array([0, 1, 2]), np.array([1, 0]),
                                 np.array([1.0, 1.0])), "f64")
    r = torch.ones(2, dtype=torch.float64, device=dev)
    z = torch.empty_like(r)
    with pytest.raises(gk.GkError) as e:
        A.precond_apply(r, z, "ilu")
    assert e.value.status == gk.GK_ERR_ZERO_DIAG
    A.close()
    # zero pivot made by the elimination
    A = gk.Matrix.from_csr(W.CSR(2, 2, np.array([0, 2, 4]), np.array([0, 1, 0, 1]),
                                 np.ones(4)), "f64")
    with pytest.raises(gk.GkError) as e:
        A.precond_apply(r, z, "ilu")
    assert e.value.status == gk.GK_ERR_ZERO_DIAG
    # the failure is kept: the next call fails the same way
    with pytest.raises(gk.GkError):
        A.ilu_factors()
    A.close()
    # unsorted columns
    A = gk.Matrix.from_csr(W.CSR(2, 2, np.array([0, 2, 3]), np.array([1, 0, 1]),
                                 np.array([1.0, 2.0, 3.0])), "f64")
    with pytest.raises(gk.GkError) as e:
        A.precond_apply(r, z, "ilu")
    assert e.value.status == gk.GK_ERR_INVALID
    A.close()
    # not square
    A = gk.Matrix.from_csr(W.random_csr(4, 5, 0.5, 1), "f64")
    with pytest.raises(gk.GkError) as e:
        A.precond_apply(torch.ones(5, dtype=torch.float64, device=dev), z, "ilu")
    assert e.value.status == gk.GK_ERR_INVALID
    A.close()
    # empty matrix
    A = gk.Matrix.from_csr(W.CSR(0, 0, np.array([0]), np.array([], np.int32), np.array([])), "f64")
    e0 = torch.empty(0, dtype=torch.float64, device=dev)
    A.precond_apply(e0, e0.clone(), "ilu")
    A.close()


def _gpu_solve(m, b, method, tol, dtype="f64", fmt="csr", **kw):
    import torch
    dev = torch_dev()
    A = gk.Matrix.from_csr(m, "f64" if dtype == "mixed" else dtype)
    if fmt != "csr":
        B = A.convert(fmt)
        A.close()
        A = B
    vt = torch.float32 if dtype == "f32" else torch.float64
    bt = torch.from_numpy(np.asarray(b)).to(dev, vt)
    xt = torch.zeros(m.n, dtype=vt, device=dev)
    info = A.solve(bt, xt, method=method, precond="ilu", tol=tol, max_iters=5000, **kw)
    torch.cuda.synchronize()
    x = xt.cpu().numpy().astype(np.float64)
    A.close()
    return x, info


SOLVE_CASES = {
    "lap2d_64": lambda: (W.laplacian_2d(64), W.uniform_vector(4096, W.SEED_BASE + 1)),
    "diff3d_16": lambda: (W.diffusion_3d(16, seed=4), W.uniform_vector(16 ** 3, 5)),
    "convdiff_60": lambda: (W.convection_diffusion_2d(60, 3.0), W.uniform_vector(3600, 6)),
    "banded_3000": lambda: (W.banded_spd(3000, 9, 2), W.uniform_vector(3000, 7)),
}


@pytest.mark.parametrize("method", ["cg", "bicgstab", "cgs", "gmres"])
@pytest.mark.parametrize("case", list(SOLVE_CASES))
def test_ilu_solvers_match_oracle(method, case):
    m, b = SOLVE_CASES[case]()
    if method == "cg" and case == "convdiff_60":
        pytest.skip("CG needs an SPD matrix")
    x, info = _gpu_solve(m, b, method, 1e-10)
    assert info["return"] == gk.GK_OK, info
    rel = oracle.true_rel_residual(m, b, x)
    assert rel <= 1e-10, (rel, info)
    xo, io = oracle.solve(m, b, method=METHOD[method], precond=3, tol=1e-10, max_iters=5000)
    assert io["status"] == oracle.OK
    slack = 30 if method == "gmres" else 3
    assert abs(info["iters"] - io["iters"]) <= max(slack, 0.1 * io["iters"]), (info, io)
    # ILU(0) needs fewer iterations than Jacobi
    _, ij = oracle.solve(m, b, method=METHOD[method], precond=1, tol=1e-10, max_iters=5000)
    assert info["iters"] < ij["iters"], (info, ij)


def test_ilu_padded_formats_f32_refinement_and_engines():
    m, b = SOLVE_CASES["diff3d_16"]()
    for fmt in ("ell", "sellp"):
        x, info = _gpu_solve(m, b, "cg", 1e-10, fmt=fmt)
        assert info["return"] == gk.GK_OK and oracle.true_rel_residual(m, b, x) <= 1e-10
    x, info = _gpu_solve(m, b, "bicgstab", 1e-5, dtype="f32")
    assert info["return"] == gk.GK_OK and oracle.true_rel_residual(m, b, x) <= 1e-5
    for mixed in (1, 2, 3):
        x, info = _gpu_solve(m, b, "gmres", 1e-10, dtype="mixed", mixed=mixed)
        assert info["return"] == gk.GK_OK, (mixed, info)
        assert oracle.true_rel_residual(m, b, x) <= 1e-10
    for engine in (2, 3):
        _, info = _gpu_solve(m, b, "cg", 1e-10, engine=engine)
        assert info["return"] == gk.GK_ERR_UNSUPPORTED


def test_full_size_diffusion_128_factors_and_apply_bit_exact():
    """The 128^3 diffusion matrix of the solver benchmark (2,097,152 rows):
    factors and one substitution pair bit for bit against the oracle."""
    import torch
    dev = torch_dev()
    m = W.diffusion_3d(128)
    A = gk.Matrix.from_csr(m, "f64")
    lu = oracle.ilu0(m)
    got = A.ilu_factors()
    assert np.array_equal(got.view(np.uint64), lu.view(np.uint64))
    r = W.uniform_vector(m.n, 11)
    rt = torch.from_numpy(r).to(dev)
    zt = torch.empty_like(rt)
    A.precond_apply(rt, zt, "ilu")
    torch.cuda.synchronize()
    want = oracle.ilu0_apply(m, lu, r)
    assert np.array_equal(zt.cpu().numpy().view(np.uint64), want.view(np.uint64))
    A.close()


def test_input_holding_the_unsolved_marker_is_a_plain_nan():
    """The substitutions mark unsolved slots with one signalling-NaN bit
    pattern; an input entry with exactly that pattern must come out as an
    ordinary NaN (propagating to the rows that depend on it), not stall."""
    import torch
    dev = torch_dev()
    m = W.laplacian_2d(40, 9)
    A = gk.Matrix.from_csr(m, "f64")
    r = W.uniform_vector(m.n, 12)
    r.view(np.uint64)[[0, 77]] = np.uint64(0x7FF0DEADBEEF1B1B)
    rt = torch.from_numpy(r).to(dev)
    zt = torch.empty_like(rt)
    A.precond_apply(rt, zt, "ilu")
    torch.cuda.synchronize()
    z = zt.cpu().numpy()
    assert np.isnan(z).any()
    assert not np.any(z.view(np.uint64) == np.uint64(0x7FF0DEADBEEF1B1B))
    # a clean input afterwards is exact again
    r2 = W.uniform_vector(m.n, 13)
    rt2 = torch.from_numpy(r2).to(dev)
    A.precond_apply(rt2, zt, "ilu")
    torch.cuda.synchronize()
    want = oracle.ilu0_apply(m, oracle.ilu0(m), r2)
    assert np.array_equal(zt.cpu().numpy().view(np.uint64), want.view(np.uint64))
    A.close()


def _power_law_with_diagonal(n, seed):
    """Zipf(1.8) power-law rows (uniform random columns, up to 4096 long)
    with a dominant diagonal merged into each row, columns ascending."""
    m = W.power_law(n, seed=seed)
    rows = np.repeat(np.arange(n), m.row_lengths())
    keep = m.col_idx != rows
    r, c, v = rows[keep], m.col_idx[keep], m.values[keep]
    absum = np.bincount(r, weights=np.abs(v), minlength=n)
    r = np.concatenate([r, np.arange(n)])
    c = np.concatenate([c, np.arange(n)])
    v = np.concatenate([v, absum + 1.0])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rp[1:])
    return W.CSR(n, n, rp, c, v)


def test_power_law_hub_rows_bit_exact():
    """Irregular dependencies: hub rows thousands of entries long, random
    columns (shallow, wide dependency levels)."""
    import torch
    dev = torch_dev()
    m = _power_law_with_diagonal(1 << 15, W.SEED_BASE + 7)
    assert m.row_lengths().max() >= 1000
    A = gk.Matrix.from_csr(m, "f64")
    lu = oracle.ilu0(m)
    assert np.array_equal(A.ilu_factors().view(np.uint64), lu.view(np.uint64))
    r = W.uniform_vector(m.n, 21)
    rt = torch.from_numpy(r).to(dev)
    zt = torch.empty_like(rt)
    A.precond_apply(rt, zt, "ilu")
    torch.cuda.synchronize()
    want = oracle.ilu0_apply(m, lu, r)
    assert np.array_equal(zt.cpu().numpy().view(np.uint64), want.view(np.uint64))
    xt = torch.zeros_like(rt)
    info = A.solve(rt, xt, method="bicgstab", precond="ilu", tol=1e-10, max_iters=500)
    assert info["return"] == gk.GK_OK, info
    assert oracle.true_rel_residual(m, r, xt.cpu().numpy()) <= 1e-10
    A.close()


@pytest.mark.parametrize("low", ["bf16", "f16"])
def test_low_precision_storage_equals_fp32_of_the_rounded_values(low):
    """A BF16- or FP16-stored handle factors its stored values in double and
    rounds the factors to float, exactly as an FP32 handle holding the same
    (exactly representable) values: factors and applications bit-identical."""
    import torch
    dev = torch_dev()
    m = W.convection_diffusion_2d(50, 1.5)
    L = _matrix(m, low)
    F = gk.Matrix.from_csr(W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx,
                                 rounded_values(m, low).astype(np.float32)), "f32")
    assert np.array_equal(L.ilu_factors().view(np.uint32), F.ilu_factors().view(np.uint32))
    r = torch.from_numpy(W.uniform_vector(m.n, 8)).to(dev, torch.float32)
    z1 = torch.empty_like(r)
    z2 = torch.empty_like(r)
    L.precond_apply(r, z1, "ilu")
    F.precond_apply(r, z2, "ilu")
    torch.cuda.synchronize()
    assert torch.equal(z1, z2)
    L.close()
    F.close()


@pytest.mark.parametrize("chunk", ["1", "8", "32", "lvl", "win"])
@pytest.mark.parametrize("case", ["lap2d_37x29", "convdiff_45", "diff3d_12", "random_700",
                                  "lap1d_33", "one_row", "power_law"])
def test_every_substitution_shape_bit_exact(monkeypatch, chunk, case):
    """Each shape the setup can time for the substitutions (single rows,
    32 of one dependency level to a warp; 8- or 32-row chunks, one to a
    warp; "lvl": one thread-block cluster, level by level with a cluster
    barrier between levels; "win": the same with the recent levels' values
    in distributed shared memory, where the matrix qualifies -- the others
    fall back to the timed shapes) gives the oracle's substitution bit for bit,
    repeated applies included: the shape changes only who computes a row,
    never its order of subtractions."""
    import torch
    monkeypatch.setenv("GK_ILU_CHUNK", chunk)
    dev = torch_dev()
    m = (_power_law_with_diagonal(1 << 12, W.SEED_BASE + 8) if case == "power_law"
         else CASES[case]())
    A = gk.Matrix.from_csr(m, "f64")
    lu = oracle.ilu0(m)
    rng = np.random.default_rng(31)
    for rep in range(2):
        r = rng.uniform(-1, 1, m.n)
        rt = torch.from_numpy(r).to(dev)
        zt = torch.full_like(rt, float("nan"))
        A.precond_apply(rt, zt, "ilu")
        torch.cuda.synchronize()
        want = oracle.ilu0_apply(m, lu, r)
        assert np.array_equal(zt.cpu().numpy().view(np.uint64), want.view(np.uint64)), rep
    A.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", ["lap2d_37x29", "diff3d_12", "lap1d_33", "one_row"])
def test_shapes_agree_bit_for_bit_with_signalling_nan_inputs(monkeypatch, dtype, case):
    """Every substitution shape gives the same bits as the 32-row chunks, in
    FP32 as in FP64, for an input holding signalling NaNs: each shape
    multiplies its inputs by 1 before the first subtraction (the window mode
    in its level-order gather), so a NaN comes out the same in every row
    that depends on it, and the other rows are untouched."""
    import torch
    dev = torch_dev()
    m = CASES[case]()
    vt = torch.float64 if dtype == "f64" else torch.float32
    ut = np.uint64 if dtype == "f64" else np.uint32
    snan = ut(0x7FF0000000000005) if dtype == "f64" else ut(0x7F800005)
    r = W.uniform_vector(m.n, 17).astype(np.float64 if dtype == "f64" else np.float32)
    bad = sorted({m.n // 2, m.n - 1})
    r.view(ut)[bad] = snan
    outs = {}
    for chunk in ["32", "8", "1", "lvl", "win"]:
        monkeypatch.setenv("GK_ILU_CHUNK", chunk)
        A = gk.Matrix.from_csr(m, dtype)
        rt = torch.from_numpy(r).to(dev)
        zt = torch.zeros(m.n, dtype=vt, device=dev)
        A.precond_apply(rt, zt, "ilu")
        torch.cuda.synchronize()
        outs[chunk] = zt.cpu().numpy().view(ut).copy()
        A.close()
    z = outs["32"].view(r.dtype)
    assert np.isnan(z[bad]).all()
    assert not np.any(outs["32"] == snan)
    for chunk, o in outs.items():
        assert np.array_equal(o, outs["32"]), chunk


def test_window_mode_on_a_stencil_bit_exact(monkeypatch):
    """The 3D diffusion stencil qualifies for the shared-memory window mode
    (3 terms a row per triangle, dependencies one level back); forced, it
    must give the oracle's ILU(0) application and ILU-preconditioned GMRES
    must converge as with the other shapes."""
    import torch
    monkeypatch.setenv("GK_ILU_CHUNK", "win")
    m = W.diffusion_3d(40, seed=6)  # 64,000 rows, 118 levels per triangle
    A = gk.Matrix.from_csr(m, "f64")
    lu = oracle.ilu0(m)
    r = W.uniform_vector(m.n, 23)
    rt = torch.from_numpy(r).to(torch_dev())
    zt = torch.full_like(rt, float("nan"))
    for _ in range(2):
        A.precond_apply(rt, zt, "ilu")
        torch.cuda.synchronize()
        want = oracle.ilu0_apply(m, lu, r)
        assert np.array_equal(zt.cpu().numpy().view(np.uint64), want.view(np.uint64))
    xt = torch.zeros_like(rt)
    info = A.solve(rt, xt, method="gmres", precond="ilu", tol=1e-10, max_iters=2000)
    assert info["return"] == gk.GK_OK, info
    assert oracle.true_rel_residual(m, r, xt.cpu().numpy()) <= 1e-10
    A.close()
