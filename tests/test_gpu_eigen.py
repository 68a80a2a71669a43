"""Rayleigh-Ritz composed from the library's SpMV (paper_2510_08230_gb300.eigen)
against closed-form Laplacian spectra and LAPACK's dense symmetric
eigenvalues."""
import math

import numpy as np
import pytest

import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import eigen
from paper_2510_08230_gb300 import workloads as W
from gpu_util import ensure_built, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _lap2d_eigs(nx, ny):
    p = np.arange(1, nx + 1)[:, None]
    q = np.arange(1, ny + 1)[None, :]
    return (4 - 2 * np.cos(p * np.pi / (nx + 1)) - 2 * np.cos(q * np.pi / (ny + 1))).reshape(-1)


def _lap2d_vec(nx, ny, p, q):
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]  # row index = y * nx + x (x fastest)
    v = np.sin(p * np.pi * (x + 1) / (nx + 1)) * np.sin(q * np.pi * (y + 1) / (ny + 1))
    return v.reshape(-1) / np.linalg.norm(v)


def test_full_basis_gives_the_whole_closed_form_spectrum():
    import torch
    dev = torch_dev()
    m = W.laplacian_2d(8)
    A = gk.Matrix.from_csr(m, "f64")
    V = torch.eye(m.n, dtype=torch.float64, device=dev)
    theta, X, AX = eigen.rayleigh_ritz(A, V)
    got = np.sort(theta.cpu().numpy())
    assert np.allclose(got, np.sort(_lap2d_eigs(8, 8)), rtol=0, atol=1e-12)
    res = torch.linalg.vector_norm(AX - theta[:, None] * X, dim=1).max().item()
    assert res <= 1e-12
    A.close()


def test_invariant_subspace_gives_its_eigenvalues():
    import torch
    dev = torch_dev()
    nx, ny = 30, 20
    m = W.laplacian_2d(nx, ny)
    A = gk.Matrix.from_csr(m, "f64")
    pairs = [(1, 1), (2, 3), (7, 5), (30, 20), (12, 1)]
    V = np.stack([_lap2d_vec(nx, ny, p, q) for p, q in pairs])
    want = np.sort([4 - 2 * math.cos(p * math.pi / (nx + 1)) - 2 * math.cos(q * math.pi / (ny + 1))
                    for p, q in pairs])
    Vt = eigen.orthonormalize(torch.from_numpy(V).to(dev))
    theta, _, _ = eigen.rayleigh_ritz(A, Vt)
    assert np.allclose(theta.cpu().numpy(), want, rtol=0, atol=1e-12)
    A.close()


def test_ritz_values_lie_inside_the_spectrum():
    import torch
    dev = torch_dev()
    nx, ny = 25, 19
    m = W.laplacian_2d(nx, ny)
    A = gk.Matrix.from_csr(m, "f64")
    lam = _lap2d_eigs(nx, ny)
    g = torch.Generator().manual_seed(3)
    V = eigen.orthonormalize(torch.randn(12, m.n, generator=g, dtype=torch.float64).to(dev))
    theta, _, _ = eigen.rayleigh_ritz(A, V)
    t = theta.cpu().numpy()
    assert t.min() >= lam.min() - 1e-12 and t.max() <= lam.max() + 1e-12
    A.close()


def _separated_tridiagonal(n):
    d = np.arange(1, n + 1, dtype=np.float64)
    d[-5:] = [480.0, 550.0, 650.0, 800.0, 1000.0]
    rp, ci, va = [0], [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                ci.append(j)
                va.append(d[i] if j == i else 0.5)
        rp.append(len(ci))
    return W.CSR(n, n, np.array(rp), np.array(ci), np.array(va))


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_subspace_iteration_matches_lapack(dtype, tol):
    m = _separated_tridiagonal(600)
    A = gk.Matrix.from_csr(m, dtype)
    out = eigen.subspace_iteration(A, k=6, nev=3, iters=2000, tol=tol, seed=1)
    want = np.sort(np.linalg.eigvalsh(m.to_dense()))[::-1][:3]
    got = out["theta"].cpu().numpy().astype(np.float64)
    assert out["iters"] < 2000, out["iters"]
    assert np.all(out["resid"].cpu().numpy() <= tol * np.abs(got) * 1.0001)
    assert np.allclose(got, want, rtol=10 * tol, atol=0), (got, want)
    A.close()
