"""Host threads on different handles at once: every first solve captures
its CUDA graph while other threads capture theirs, upload and destroy
matrices.  Each result must equal the same solve run alone (a handle's
arithmetic does not depend on what other threads do)."""
import threading

import numpy as np
import pytest

import paper_2510_08230_gb300 as gk
from paper_2510_08230_gb300 import workloads as W
from gpu_util import ensure_built, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


# (matrix, solve options): n > 16,384 keeps the plain solves on the
# graph-captured multi-kernel engine; mixed=1 adds FP32 inner-solve graphs
CASES = [(lambda: W.laplacian_2d(140), dict(method="cg", precond="jacobi", tol=1e-9)),
         (lambda: W.laplacian_2d(150), dict(method="cg", precond="jacobi", tol=1e-9, mixed=1)),
         (lambda: W.laplacian_3d(30), dict(method="bicgstab", precond="jacobi", tol=1e-9)),
         (lambda: W.diffusion_3d(28, seed=3), dict(method="gmres", precond="jacobi", tol=1e-8)),
         (lambda: W.laplacian_3d(32), dict(method="cg", precond=None, tol=1e-9, mixed=1)),
         (lambda: W.banded_spd(40000, 6, 4), dict(method="cgs", precond="jacobi", tol=1e-9))]


def _solve(m, kw, stream, out, idx, start):
    import torch
    dev = torch_dev()
    with torch.cuda.stream(stream):
        A = gk.Matrix.from_csr(m)
        b = torch.from_numpy(W.uniform_vector(m.n, 40 + idx)).to(dev)
        x = torch.zeros_like(b)
        if start is not None:
            start.wait()
        info = A.solve(b, x, stream, max_iters=20000, **kw)
        stream.synchronize()
        out[idx] = (info, x.cpu().numpy())
        A.close()


def test_concurrent_first_solves_equal_sequential():
    import torch
    mats = [c() for c, _ in CASES]
    seq = {}
    for i, (m, (_, kw)) in enumerate(zip(mats, CASES)):
        _solve(m, kw, torch.cuda.Stream(), seq, i, None)
    for rep in range(3):
        par = {}
        start = threading.Barrier(len(CASES) + 1)
        stop = threading.Event()

        def churn():  # uploads and destroys matrices meanwhile
            start.wait()
            k = 0
            while not stop.is_set():
                M = gk.Matrix.from_csr(W.laplacian_2d(64 + k % 7))
                M.close()
                k += 1

        ths = [threading.Thread(target=_solve, args=(m, kw, torch.cuda.Stream(), par, i, start))
               for i, (m, (_, kw)) in enumerate(zip(mats, CASES))]
        ch = threading.Thread(target=churn)
        for t in ths + [ch]:
            t.start()
        for t in ths:
            t.join(300)
        stop.set()
        ch.join(60)
        for i in range(len(CASES)):
            info, x = par[i]
            assert info["return"] == gk.GK_OK, (rep, i, info)
            assert info["iters"] == seq[i][0]["iters"], (rep, i)
            assert np.array_equal(x, seq[i][1]), (rep, i)
