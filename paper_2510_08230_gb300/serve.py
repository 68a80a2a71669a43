"""Continuous-batching solve server on one GPU.

Requests (a CSR matrix by key, a right-hand side, a tolerance and a
precision) arrive at any time.  The server:

* keeps uploaded matrices resident on the device in an LRU cache keyed by
  the request's matrix key (a matrix, its solver workspace and its
  low-precision copy stay on the device while cached);
* admits a request when its device bytes (matrix if not cached, Krylov
  workspace, b and x) fit the budget next to everything admitted or
  cached; unused cached matrices are evicted to make room;
* runs admitted work on a pool of worker threads in arrival order (or,
  with order="sjf", the job with the smallest expected solve time first,
  aged by its waiting time); the expected time is learned per matrix key
  and precision from the solves already served, else estimated from the
  matrix size.  Optionally (long_workers > 0) solves expected to run long
  get a lane of their own, so that they never occupy every worker;
* batches continuously: small FP64 systems (n <= small_n) that arrive while
  the workers are busy wait in a pending list and are all launched together
  in one gk_solve_batched call as soon as a worker frees up; other solves
  run gk_solve one per worker.  Measured on GB300 (the 24-matrix mix): two
  lanes of 2 + 4 workers lowered the saturation throughput and raised p99
  at 0.8x load, because the long solves queued behind each other, so one
  pool is the default.  Batches on the highest-priority CUDA stream
  (batch_priority="high") starved the large solves (the slowest request's
  service time 3.2 s against 0.55 s, 73 against 92 solves/s at
  saturation), so every launch uses the same priority by default.

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


def estimate_seconds(m, precision):
    """Prior for a matrix never solved before: CG iterations grow like the
    grid's side for these stencils and bands, so nnz * sqrt(n) measures the
    work (calibrated on GB300: ~60 ms for the 2D Laplacian 969^2 in FP64);
    refinement about 1.5x faster."""
    t = 1.5e-11 * m.nnz * np.sqrt(max(m.n, 1))
    return t / 1.5 if precision == "ir32" else t


class SolveServer:
    def __init__(self, budget_bytes=40e9, workers=6, small_n=16384, batch_max=1024, device=0,
                 long_workers=0, long_s=0.02, aging=1.0, order="fifo", long_priority="low",
                 batch_priority="low"):
        import torch
        self.torch = torch
        self.dev = torch.device(f"cuda:{device}")
        self.budget = float(budget_bytes)
        self.small_n = small_n
        self.batch_max = batch_max
        self.long_s = long_s          # expected seconds above which a solve is long
        self.aging = aging            # seconds of priority gained per second waited
        self.order = order            # "fifo" or "sjf" (smallest expected time, aged)
        self.long_priority = long_priority  # stream priority of the long lane: "low" or "high"
        self.batch_priority = batch_priority  # stream priority of batched launches: "high" or "low"
        self.cv = threading.Condition()
        self.queue = collections.deque()      # submitted, not admitted
        self.pending_small = []               # admitted, waiting for a batch launch
        self.pending_single = []              # admitted short solves
        self.pending_long = []                # admitted long solves
        self.cache = collections.OrderedDict()  # key -> [Matrix, bytes, users, refined]
        self.used = 0.0                       # admitted request bytes + cached matrix bytes
        self.cost = {}                        # (key, precision) -> observed solve seconds (EWMA)
        long_workers = max(0, min(long_workers, workers - 1))  # 0: one lane for everything
        self.n_long = long_workers
        self.idle = {"short": workers - long_workers, "long": long_workers}
        self.jobs = {"short": collections.deque(), "long": collections.deque()}
        self.running = True
        self.completed = []
        self.error = None
        lanes = ["long"] * long_workers + ["short"] * (workers - long_workers)
        self.threads = [threading.Thread(target=self._worker, args=(lane,), daemon=True)
                        for lane in lanes]
        self.disp = threading.Thread(target=self._dispatch, daemon=True)
        for t in self.threads:
            t.start()
        self.disp.start()

    def expected_seconds(self, req):
        c = self.cost.get((req.key, req.precision))
        return c if c is not None else estimate_seconds(req.m, req.precision)

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
            if small:
                self.pending_small.append(req)
            elif self.n_long and self.expected_seconds(req) > self.long_s:
                self.pending_long.append(req)
            else:
                self.pending_single.append(req)

    def _dispatch(self):
        try:
            self._dispatch_loop()
        except Exception as e:  # fail everything still waiting, loudly
            with self.cv:
                self.error = e
                waiting = list(self.queue) + self.pending_small + self.pending_single + \
                    self.pending_long
                for r in waiting:
                    r.info = {"status": -3, "error": repr(e)}
                    r.event.set()
            raise

    def _prio(self, req, now):
        """Dispatch key (smaller first): arrival time, or for "sjf" the
        expected seconds minus aging x seconds waited (no starvation)."""
        if self.order == "fifo":
            return req.t_submit
        return self.expected_seconds(req) - self.aging * (now - req.t_submit)

    def _take(self, pending, now):
        k = min(range(len(pending)), key=lambda i: self._prio(pending[i], now))
        return pending.pop(k)

    def _dispatch_loop(self):
        with self.cv:
            while self.running:
                self._admit()
                now = time.perf_counter()
                while self.idle["long"] > 0 and self.pending_long:
                    self.jobs["long"].append(("single", [self._take(self.pending_long, now)]))
                    self.idle["long"] -= 1
                    self.cv.notify_all()
                while self.idle["short"] > 0 and (self.pending_small or self.pending_single):
                    # a batch of every pending small system (expected to take about as
                    # long as its slowest member) or the best short solve
                    bt = -1.0
                    if self.pending_small:
                        head = min(self.pending_small, key=lambda r: r.t_submit)
                        bt = head.t_submit if self.order == "fifo" else \
                            max(self.expected_seconds(r) for r in self.pending_small) - \
                            self.aging * (now - head.t_submit)
                    st = min((self._prio(r, now) for r in self.pending_single), default=None)
                    if self.pending_small and (st is None or bt <= st):
                        # group by method/precond so one launch serves them all
                        grp = [r for r in self.pending_small
                               if r.method == head.method and r.precond == head.precond]
                        grp = grp[:self.batch_max]
                        ids = {id(r) for r in grp}
                        self.pending_small = [r for r in self.pending_small if id(r) not in ids]
                        self.jobs["short"].append(("batch", grp))
                    else:
                        self.jobs["short"].append(("single",
                                                   [self._take(self.pending_single, now)]))
                    self.idle["short"] -= 1
                    self.cv.notify_all()
                # a long-lane worker with nothing long to do helps with short work
                while self.idle["long"] > 0 and not self.pending_long and self.pending_single \
                        and self.idle["short"] == 0:
                    self.jobs["long"].append(("single", [self._take(self.pending_single, now)]))
                    self.idle["long"] -= 1
                    self.cv.notify_all()
                self.cv.wait(timeout=0.005)

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

    def _finish(self, reqs, lane, t_run):
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
            if len(reqs) == 1 and reqs[0].info and reqs[0].info.get("status") == GK_OK:
                k = (reqs[0].key, reqs[0].precision)
                old = self.cost.get(k)
                self.cost[k] = t_run if old is None else 0.5 * (old + t_run)
            self.idle[lane] += 1
            self.cv.notify_all()

    def _worker(self, lane):
        torch = self.torch
        torch.cuda.set_device(self.dev)
        # batch_priority="high": batched small systems on the highest-priority
        # stream, their blocks scheduled ahead of a large solve's
        lo, hi = torch.cuda.Stream.priority_range()
        stream_hi = torch.cuda.Stream(device=self.dev, priority=hi)
        stream_lo = torch.cuda.Stream(device=self.dev, priority=lo)
        if lane == "long" and self.long_priority == "high":
            stream_lo = stream_hi  # long solves ahead of everything else
        if self.batch_priority != "high":
            stream_hi = stream_lo  # batches at the priority of single solves
        while True:
            with self.cv:
                while self.running and not self.jobs[lane]:
                    self.cv.wait(timeout=0.1)
                if not self.running and not self.jobs[lane]:
                    return
                kind, reqs = self.jobs[lane].popleft()
            t0 = time.perf_counter()
            stream = stream_hi if kind == "batch" else stream_lo
            try:
                with torch.cuda.stream(stream):
                    for r in reqs:
                        r.t_start = t0
                    if kind == "batch":
                        self._run_batch(reqs, stream)
                    else:
                        self._run_single(reqs[0], stream)
            except Exception as e:  # surface as a failed request
                for r in reqs:
                    r.info = {"status": -3, "error": repr(e)}
            self._finish(reqs, lane, time.perf_counter() - t0)

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
        serv = np.array([r.t_done - r.t_start for r in reqs
                         if r.t_start is not None and r.t_done is not None])
        ok = sum(1 for r in reqs if r.info and r.info.get("status") == GK_OK)

        def pct(a, q):
            return round(float(np.percentile(a, q)) * 1e3, 2) if a.size else None

        return {"requests": len(reqs), "ok": ok,
                "solves_per_s": round(len(lat) / max(t1 - t0, 1e-9), 2),
                "p50_ms": pct(lat, 50), "p90_ms": pct(lat, 90), "p99_ms": pct(lat, 99),
                "p99_over_p50": (round(float(np.percentile(lat, 99) / np.percentile(lat, 50)), 2)
                                 if lat.size else None),
                "mean_wait_ms": round(float(wait.mean()) * 1e3, 2) if wait.size else None,
                "p99_wait_ms": pct(wait, 99), "service_p50_ms": pct(serv, 50),
                "service_p99_ms": pct(serv, 99),
                "batched_fraction": round(sum(r.batched for r in reqs) / max(len(reqs), 1), 3)}
