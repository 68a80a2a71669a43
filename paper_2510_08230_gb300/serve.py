"""Continuous-batching solve server on one GPU.

Requests (a CSR matrix by key, a right-hand side, a tolerance and a
precision) arrive at any time.  The server:

* keeps uploaded matrices resident on the device in an LRU cache keyed by
  the request's matrix key (a matrix, its solver workspace and its
  low-precision copy stay on the device while cached);
* admits a request when its device bytes (matrix if not cached, Krylov
  workspace, b and x) fit the budget next to everything admitted or
  cached; unused cached matrices are evicted to make room;
* runs admitted work on a pool of worker threads, each owning a CUDA
  stream, so solves overlap on the device;
* batches continuously: small FP64 systems (n <= small_n) that arrive while
  the workers are busy wait in a pending list and are all launched together
  in one gk_solve_batched call as soon as a worker frees up; larger systems
  and FP32-refined solves run gk_solve one per worker.

Latency is measured from submit() to the solution being back on the host.
All compute runs in libgk.so; this module only schedules.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

from . import GK_OK, Matrix, gk_solve_batched, make_opts

__all__ = ["SolveRequest", "SolveServer", "request_bytes"]


class SolveRequest:
    """One solve: A (workloads.CSR, shared by key) x = b."""

    __slots__ = ("rid", "key", "m", "b", "tol", "precision", "method", "precond", "max_iters",
                 "t_submit", "t_start", "t_done", "x", "info", "need", "batched", "event")

    def __init__(self, rid, key, m, b, tol=1e-10, precision="f64", method="cg",
                 precond="jacobi", max_iters=20000):
        self.rid, self.key, self.m, self.b = rid, key, m, np.asarray(b, dtype=np.float64)
        self.tol, self.precision, self.method = tol, precision, method
        self.precond, self.max_iters = precond, max_iters
        self.t_submit = self.t_start = self.t_done = None
        self.x = self.info = None
        self.need = 0
        self.batched = False
        self.event = threading.Event()


def matrix_bytes(m, refined):
    """Device bytes that stay with a cached matrix: FP64 CSR arrays, the
    padded copy the solvers may keep for their SpMV (ELL or SELL-P, at most
    1.2 x nnz entries), the solver workspace its handle keeps (up to 10 FP64
    vectors), and, once a refined solve used it, the FP32 copy with its own
    padded copy and FP32 workspace."""
    b = 4 * (m.n + 1) + 12 * m.nnz + int(1.2 * 12 * m.nnz) + 10 * 8 * m.n
    if refined:
        b += 4 * (m.n + 1) + 8 * m.nnz + int(1.2 * 8 * m.nnz) + 10 * 4 * m.n
    return b


def ilu_bytes(m, refined):
    """Device bytes an ILU(0) solve adds to a cached matrix: the factors'
    pattern, values, diagonal data and claim orders (per value type: twice
    once a refined solve factors the FP32 copy too) and two more solver
    vectors."""
    b = 4 * (m.n + 1) + 12 * m.nnz + 20 * m.n
    return b * (2 if refined else 1) + 2 * 8 * m.n


# preconditioners the batched engine runs (others go to gk_solve alone)
BATCHED_PRECONDS = (None, False, True, 0, 1, "none", "jacobi")


def request_bytes(req, small_n):
    """Device bytes held only while a request runs: b and x, plus the
    batched engine's per-system workspace (4 FP64 vectors)."""
    n = req.m.n
    if n <= small_n and req.precision == "f64":
        return 16 * n + 4 * 8 * n
    return 16 * n


class SolveServer:
    def __init__(self, budget_bytes=40e9, workers=6, small_n=16384, batch_max=1024, device=0):
        import torch
        self.torch = torch
        self.dev = torch.device(f"cuda:{device}")
        self.budget = float(budget_bytes)
        self.small_n = small_n
        self.batch_max = batch_max
        self.cv = threading.Condition()
        self.queue = collections.deque()      # submitted, not admitted
        self.pending_small = []               # admitted, waiting for a batch launch
        self.pending_single = collections.deque()
        self.cache = collections.OrderedDict()  # key -> [Matrix, bytes, users, refined]
        self.used = 0.0                       # admitted request bytes + cached matrix bytes
        self.idle = workers
        self.jobs = collections.deque()
        self.running = True
        self.completed = []
        self.error = None
        self.threads = [threading.Thread(target=self._worker, daemon=True) for _ in range(workers)]
        self.disp = threading.Thread(target=self._dispatch, daemon=True)
        for t in self.threads:
            t.start()
        self.disp.start()

    # ---------------------------------------------------------------- API
    def submit(self, req):
        req.t_submit = time.perf_counter()
        with self.cv:
            self.queue.append(req)
            self.cv.notify_all()
        return req

    def close(self):
        with self.cv:
            self.running = False
            self.cv.notify_all()
        for t in self.threads + [self.disp]:
            t.join(timeout=30)
        for entry in self.cache.values():
            if entry[0] is not None:
                entry[0].close()
        self.cache.clear()

    # ----------------------------------------------------------- scheduler
    def _evict(self, need, keep=None):
        """Evict unused cached matrices (LRU first, never `keep`) until
        `need` fits."""
        for key in list(self.cache.keys()):
            if self.used + need <= self.budget:
                return
            if key == keep:
                continue
            mat, nb, users = self.cache[key][:3]
            if users == 0:
                self.used -= nb
                del self.cache[key]
                if mat is not None:
                    mat.close()

    def _admit(self):
        while self.queue:
            req = self.queue[0]
            refined = req.precision == "ir32"
            ilu = req.precond == "ilu"
            need = request_bytes(req, self.small_n)
            entry = self.cache.get(req.key)
            if entry is None:
                mb = matrix_bytes(req.m, refined) + (ilu_bytes(req.m, refined) if ilu else 0)
            else:
                mb = 0
                if refined and not entry[3]:  # a cached matrix gains its FP32 copy
                    mb += matrix_bytes(req.m, True) - matrix_bytes(req.m, False)
                if ilu and not entry[4]:  # ... or its ILU(0) factors
                    mb += ilu_bytes(req.m, refined or entry[3])
            if self.used + need + mb > self.budget:
                self._evict(need + mb, keep=req.key)
                if self.used + need + mb > self.budget:
                    return  # head of line waits for memory
            self.queue.popleft()
            req.need = need
            self.used += need + mb
            if entry is None:
                self.cache[req.key] = [None, mb, 1, refined, ilu]
            else:
                entry[2] += 1
                self.cache.move_to_end(req.key)
                entry[1] += mb
                entry[3] = entry[3] or refined
                entry[4] = entry[4] or ilu
            small = req.m.n <= self.small_n and req.precision == "f64" and \
                req.method in ("cg", "bicgstab") and req.precond in BATCHED_PRECONDS
            req.batched = small
            (self.pending_small if small else self.pending_single).append(req)

    def _dispatch(self):
        try:
            self._dispatch_loop()
        except Exception as e:  # fail everything still waiting, loudly
            with self.cv:
                self.error = e
                waiting = list(self.queue) + self.pending_small + list(self.pending_single)
                for r in waiting:
                    r.info = {"status": -3, "error": repr(e)}
                    r.event.set()
            raise

    def _dispatch_loop(self):
        with self.cv:
            while self.running:
                self._admit()
                while self.idle > 0 and (self.pending_small or self.pending_single):
                    # serve the older head first; small heads take every pending
                    # small system of the same kind with them
                    if self.pending_small and (not self.pending_single or
                                               self.pending_small[0].t_submit <=
                                               self.pending_single[0].t_submit):
                        # group by method/precond so one launch serves them all
                        head = self.pending_small[0]
                        grp = [r for r in self.pending_small
                               if r.method == head.method and r.precond == head.precond]
                        grp = grp[:self.batch_max]
                        ids = {id(r) for r in grp}
                        self.pending_small = [r for r in self.pending_small if id(r) not in ids]
                        self.jobs.append(("batch", grp))
                    else:
                        self.jobs.append(("single", [self.pending_single.popleft()]))
                    self.idle -= 1
                    self.cv.notify_all()
                self.cv.wait(timeout=0.05)

    # -------------------------------------------------------------- workers
    def _matrix(self, req):
        """Device matrix for the request (uploaded once, then cached)."""
        with self.cv:
            entry = self.cache[req.key]
            mat = entry[0]
        if mat is None:
            mat = Matrix.from_csr(req.m, "f64")
            with self.cv:
                if self.cache[req.key][0] is None:
                    self.cache[req.key][0] = mat
                else:
                    mat.close()
                    mat = self.cache[req.key][0]
        return mat

    def _finish(self, reqs):
        now = time.perf_counter()
        with self.cv:
            for r in reqs:
                r.t_done = now
                self.used -= r.need
                entry = self.cache.get(r.key)
                if entry is not None:
                    entry[2] -= 1
                self.completed.append(r)
                r.event.set()
            self.idle += 1
            self.cv.notify_all()

    def _worker(self):
        torch = self.torch
        torch.cuda.set_device(self.dev)
        stream = torch.cuda.Stream(device=self.dev)
        while True:
            with self.cv:
                while self.running and not self.jobs:
                    self.cv.wait(timeout=0.1)
                if not self.running and not self.jobs:
                    return
                kind, reqs = self.jobs.popleft()
            try:
                with torch.cuda.stream(stream):
                    t0 = time.perf_counter()
                    for r in reqs:
                        r.t_start = t0
                    if kind == "batch":
                        self._run_batch(reqs, stream)
                    else:
                        self._run_single(reqs[0], stream)
            except Exception as e:  # surface as a failed request
                for r in reqs:
                    r.info = {"status": -3, "error": repr(e)}
            self._finish(reqs)

    def _run_batch(self, reqs, stream):
        torch = self.torch
        mats = [self._matrix(r) for r in reqs]
        bs = [torch.from_numpy(r.b).to(self.dev, non_blocking=True) for r in reqs]
        xs = [torch.zeros(r.m.n, dtype=torch.float64, device=self.dev) for r in reqs]
        head = reqs[0]
        opts = make_opts(method=head.method, precond=head.precond, tol=head.tol,
                         max_iters=max(r.max_iters for r in reqs))
        st, infos = gk_solve_batched([m.handle for m in mats], bs, xs, opts, stream,
                                     tols=[r.tol for r in reqs])
        out = [x.cpu().numpy() for x in xs]
        for r, x, info in zip(reqs, out, infos):
            r.x = x
            r.info = dict(info, batch=len(reqs), launch_status=st)

    def _run_single(self, req, stream):
        torch = self.torch
        mat = self._matrix(req)
        b = torch.from_numpy(req.b).to(self.dev, non_blocking=True)
        x = torch.zeros(req.m.n, dtype=torch.float64, device=self.dev)
        info = mat.solve(b, x, stream, method=req.method, precond=req.precond, tol=req.tol,
                         max_iters=req.max_iters, mixed=1 if req.precision == "ir32" else 0)
        req.x = x.cpu().numpy()
        req.info = dict(info, batch=1)

    # -------------------------------------------------------------- metrics
    @staticmethod
    def summarize(reqs, t0, t1):
        lat = np.array([r.t_done - r.t_submit for r in reqs if r.t_done is not None])
        wait = np.array([r.t_start - r.t_submit for r in reqs if r.t_start is not None])
        ok = sum(1 for r in reqs if r.info and r.info.get("status") == GK_OK)
        return {"requests": len(reqs), "ok": ok,
                "solves_per_s": round(len(lat) / max(t1 - t0, 1e-9), 2),
                "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 2) if lat.size else None,
                "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 2) if lat.size else None,
                "mean_wait_ms": round(float(wait.mean()) * 1e3, 2) if wait.size else None,
                "batched_fraction": round(sum(r.batched for r in reqs) / max(len(reqs), 1), 3)}
