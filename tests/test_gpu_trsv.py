"""Sparse triangular solves with a matrix's own triangles
(gk_triangular_solve) against the oracle: bit for bit in FP64 (same order
of fused updates, reciprocal diagonal), within a rounding bound in FP32,
unit diagonals, every storage format, repeated solves and errors."""
import numpy as np
import pytest

import oracle
import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W
from gpu_util import ensure_built, rounded_values, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


CASES = {
    "lap2d_37x29": lambda: W.laplacian_2d(37, 29),
    "convdiff_45": lambda: W.convection_diffusion_2d(45, 2.0),
    "diff3d_12": lambda: W.diffusion_3d(12, seed=4),
    "banded_3000": lambda: W.banded_spd(3000, 7, 3),
    "one_row": lambda: W.CSR(1, 1, np.array([0, 1]), np.array([0]), np.array([3.0])),
}


def _solve(A, b, upper, unit, dtype):
    import torch
    dev = torch_dev()
    vt = torch.float64 if dtype == "f64" else torch.float32
    bt = torch.from_numpy(np.asarray(b)).to(dev, vt)
    xt = torch.full_like(bt, float("nan"))
    A.triangular_solve(bt, xt, upper=upper, unit_diagonal=unit)
    torch.cuda.synchronize()
    return xt.cpu().numpy()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("upper", [False, True])
@pytest.mark.parametrize("unit", [False, True])
@pytest.mark.parametrize("mode", ["tuned", "lvl", "win"])
def test_fp64_bit_exact(monkeypatch, case, upper, unit, mode):
    """mode "lvl": the level-synchronous cluster substitution forced; "win":
    its shared-memory window variant, where the matrix qualifies."""
    if mode in ("lvl", "win"):
        monkeypatch.setenv("GK_ILU_CHUNK", mode)
    else:
        monkeypatch.delenv("GK_ILU_CHUNK", raising=False)
    m = CASES[case]()
    A = gk.Matrix.from_csr(m, "f64")
    rng = np.random.default_rng(5)
    for rep in range(2):  # the analysis is reused by the second solve
        b = rng.uniform(-1, 1, m.n)
        x = _solve(A, b, upper, unit, "f64")
        want = oracle.trsv(m, b, upper=upper, unit=unit)
        assert np.array_equal(x.view(np.uint64), want.view(np.uint64)), \
            (rep, np.max(np.abs(x - want)))
    A.close()


@pytest.mark.parametrize("upper", [False, True])
def test_fp32_within_rounding(upper):
    m = W.convection_diffusion_2d(60, 1.0)
    A = gk.Matrix.from_csr(m, "f32")
    mr = W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx, rounded_values(m, "f32"))
    b = W.uniform_vector(m.n, 6).astype(np.float32).astype(np.float64)
    x = _solve(A, b, upper, False, "f32").astype(np.float64)
    want = oracle.trsv(mr, b, upper=upper)
    assert np.all(np.abs(x - want) <= 1e-4 * np.abs(want) + 1e-7 * np.abs(want).max())
    A.close()


@pytest.mark.parametrize("fmt", ["ell", "sellp", "coo"])
def test_formats(fmt):
    m = W.laplacian_2d(33, 17)
    A = gk.Matrix.from_csr(m, "f64")
    B = A.convert(fmt)
    b = W.uniform_vector(m.n, 7)
    for upper in (False, True):
        assert np.array_equal(_solve(A, b, upper, False, "f64"), _solve(B, b, upper, False, "f64"))
    A.close()
    B.close()


def test_triangles_of_the_ilu_factors_give_the_ilu_application():
    import torch
    dev = torch_dev()
    m = W.convection_diffusion_2d(40, 1.5)
    A = gk.Matrix.from_csr(m, "f64")
    lu = A.ilu_factors()
    F = gk.Matrix.from_csr(W.CSR(m.n, m.ncols, m.row_ptr, m.col_idx, lu), "f64")
    r = W.uniform_vector(m.n, 9)
    y = _solve(F, r, False, True, "f64")
    z = _solve(F, y, True, False, "f64")
    rt = torch.from_numpy(r).to(dev)
    zt = torch.empty_like(rt)
    A.precond_apply(rt, zt, "ilu")
    torch.cuda.synchronize()
    assert np.array_equal(z.view(np.uint64), zt.cpu().numpy().view(np.uint64))
    A.close()
    F.close()


def test_errors():
    import torch
    dev = torch_dev()
    b = torch.ones(2, dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    # missing diagonal
    A = gk.Matrix.from_csr(W.CSR(2, 2, np.array([0, 1, 2]), np.array([1, 0]),
                                 np.array([1.0, 1.0])), "f64")
    with pytest.raises(gk.GkError) as e:
        A.triangular_solve(b, x)
    assert e.value.status == gk.GK_ERR_INVALID
    A.close()
    # zero diagonal: an error unless the diagonal is taken as 1
    A = gk.Matrix.from_csr(W.CSR(2, 2, np.array([0, 1, 3]), np.array([0, 0, 1]),
                                 np.array([0.0, 2.0, 0.0])), "f64")
    with pytest.raises(gk.GkError) as e:
        A.triangular_solve(b, x)
    assert e.value.status == gk.GK_ERR_ZERO_DIAG
    A.triangular_solve(b, x, unit_diagonal=True)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), [1.0, -1.0])
    # b and x the same vector
    with pytest.raises(gk.GkError) as e:
        A.triangular_solve(b, b, unit_diagonal=True)
    assert e.value.status == gk.GK_ERR_INVALID
    A.close()
    # unsorted columns
    A = gk.Matrix.from_csr(W.CSR(2, 2, np.array([0, 2, 3]), np.array([1, 0, 1]),
                                 np.array([1.0, 2.0, 3.0])), "f64")
    with pytest.raises(gk.GkError) as e:
        A.triangular_solve(b, x)
    assert e.value.status == gk.GK_ERR_INVALID
    A.close()
