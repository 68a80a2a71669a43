"""Rayleigh-Ritz on top of the library's SpMV.

The paper implements the Rayleigh-Ritz method on the Python side as a proof
that new algorithms compose from the operators the binding exposes, SpMV
first among them (Section 3.4).  This module does the same with this
library: every product with A is a ``gk_apply`` of the matrix handle (the
library's SpMV kernels on the device).  The small dense steps - the k x k
projection, its symmetric eigen-decomposition and the orthonormalisation
of an n x k block - are plain PyTorch library calls on the same device.

Blocks are (k, n) tensors: k vectors of length n, each row contiguous, so
that each row is passed to ``gk_apply`` as it is.
"""
from __future__ import annotations


def apply_block(A, V, stream=None):
    """W[j] = A V[j] for every row of the (k, n) block V (one gk_apply per
    vector)."""
    import torch
    W = torch.empty_like(V)
    for j in range(V.shape[0]):
        A.apply(V[j], W[j], stream)
    return W


def orthonormalize(V):
    """Rows of V made orthonormal (a reduced QR of V^T); same span."""
    import torch
    q, _ = torch.linalg.qr(V.T, mode="reduced")
    return q.T.contiguous()


def rayleigh_ritz(A, V, stream=None, W=None):
    """Ritz pairs of the symmetric matrix A on span(V).

    V: (k, n) device block with orthonormal rows.  Forms H = V A V^T (k x k,
    symmetrised), solves H s = theta s, and returns (theta ascending,
    X = S^T V the Ritz vectors as rows, AX = S^T (A V) their images).  W,
    when given, is A V already computed."""
    import torch
    if W is None:
        W = apply_block(A, V, stream)
    H = V @ W.T
    H = 0.5 * (H + H.T)
    theta, S = torch.linalg.eigh(H)
    return theta, S.T @ V, S.T @ W


def subspace_iteration(A, k, nev=None, iters=200, tol=1e-8, seed=0, dtype=None, device=None):
    """The nev (default k) eigenpairs of largest magnitude of a symmetric A:
    block power iteration on a k-dimensional subspace with a Rayleigh-Ritz
    step every iteration, stopping when every wanted Ritz pair has
    ||A x - theta x|| <= tol * |theta|.

    Returns a dict: theta (nev values, largest first), X (nev Ritz vectors
    as rows), resid (their residual norms), iters."""
    import torch
    nev = k if nev is None else nev
    n = A.n
    if dtype is None:
        dtype = torch.float64 if A.desc["dtype"] == 0 else torch.float32
    device = device or torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device="cpu").manual_seed(seed)
    V = orthonormalize(torch.randn(k, n, generator=g, dtype=dtype).to(device))
    theta = X = res = None
    it = 0
    for it in range(1, iters + 1):
        W = apply_block(A, V)
        theta, X, AX = rayleigh_ritz(A, V, W=W)
        order = torch.argsort(theta.abs(), descending=True)
        theta, X, AX = theta[order], X[order], AX[order]
        res = torch.linalg.vector_norm(AX - theta[:, None] * X, dim=1)
        if bool(torch.all(res[:nev] <= tol * theta[:nev].abs())):
            break
        V = orthonormalize(AX)
    return {"theta": theta[:nev], "X": X[:nev], "resid": res[:nev], "iters": it}
