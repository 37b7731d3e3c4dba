"""Continuous-batching solve server on resident factors (one GPU).

The factors of each frequency stay resident (one factored handle per frequency).  Requests
(a frequency and a set of point sources) are cut into column work items of at most
``max_cols`` right-hand sides and queued per frequency.  Worker threads -- each with its own
handle and CUDA stream; the first worker of a frequency is the factor owner, further workers are
``hz_create_shared`` handles on the same factors -- take work items in arrival order as soon as
they are free, so requests that arrive while other batches are on the GPU join the next batch
of a free worker, and batches of different frequencies (and of the same frequency, when several
workers are admitted) run on the device at the same time.  A new worker is admitted only while
the free device memory, less the estimated workspace of admitted workers that have not yet
allocated theirs (workspaces are allocated on a worker's first batch), covers its own estimated
workspace for a full batch (admission by free HBM).  A batch that still runs out of device
memory is put back at the head of its queue; an extra worker that hit it is retired (its
workspace freed), and a work item is retried at most twice before its request fails.

All arithmetic runs in the CUDA library; this module only places sources, moves columns in and
out of batches and keeps time.
"""
from __future__ import annotations

import collections
import threading
import time
from typing import List, Optional, Sequence

import numpy as np

from . import hz


class Request:
    """One request: frequency index, point sources (R, 3) as (z, y, x), arrival time."""

    def __init__(self, rid: int, omega_idx: int, sources: np.ndarray, t_arrival: float = 0.0):
        self.rid = rid
        self.omega_idx = omega_idx
        self.sources = np.asarray(sources, dtype=np.int64).reshape(-1, 3)
        self.t_arrival = t_arrival
        self.t_done: Optional[float] = None
        self.result = None          # full solution (R, nz, ny, nx) or receiver samples (R, nrec)
        self.status = 0             # 0 delivered; -1 failed (a work item raised or did not converge)
        self._left = 0

    @property
    def R(self) -> int:
        return int(self.sources.shape[0])

    @property
    def latency(self) -> Optional[float]:
        return None if self.t_done is None else self.t_done - self.t_arrival


class Server:
    def __init__(self, m: np.ndarray, omegas: Sequence[float], npml: int, C: float, n_layers: int,
                 npml_local: int = -1, precision: str = "mixed", max_cols: int = 64, max_workers: int = 2,
                 opts: Optional[hz.SolveOpts] = None, receivers: Optional[np.ndarray] = None,
                 mem_reserve_bytes: float = 4e9, log=None):
        import torch
        self.torch = torch
        self.shape = tuple(m.shape)
        self.max_cols = int(max_cols)
        self.max_workers = int(max_workers)
        self.opts = opts if opts is not None else hz.default_opts(precision)
        self.receivers = None if receivers is None else np.asarray(receivers, dtype=np.int64)
        self.mem_reserve = float(mem_reserve_bytes)
        self.log = log          # None or a callable taking one line of progress text
        self.primaries: List[hz.Solver] = []
        for om in omegas:
            s = hz.Solver(m, om, npml, C, n_layers, precision=precision, npml_local=npml_local,
                          stream=torch.cuda.Stream())
            s.factor()
            self.primaries.append(s)
        self.queues = [collections.deque() for _ in omegas]
        self.cv = threading.Condition()
        self.workers: List[List[hz.Solver]] = [[] for _ in omegas]
        self.threads: List[threading.Thread] = []
        self.running = False
        self.errors: List[str] = []
        self.batches = 0
        self.max_requests_per_batch = 0
        self.admission_log: List[str] = []
        self.pending: dict = {}       # id(solver) -> estimated workspace not yet allocated
        self.retries: dict = {}       # (rid, first column) -> out-of-memory retries so far

    # ------------------------------------------------------------------ admission
    def worker_bytes(self, cols: int) -> float:
        """Estimated device memory of one worker solving a batch of ``cols`` columns: layer slot
        vectors (accumulator + solution, up to 4 stacked source blocks), the GMRES basis and
        scratch trace vectors, and the volume buffers (rhs, u, residual, correction)."""
        nz, ny, nx = self.shape
        s = self.primaries[0]
        L, K = s.n_layers, s.K
        esz = 16 if s.precision == "fp64" else 8
        lay = 0
        for ell in range(L):
            lo, hi, zlo, zhi = s.layer_info(ell)
            lay += (zhi - zlo + 1) * ny * nx
        slots = 2.0 * lay * 4 * cols * esz
        ntr = 4 * K * nx * ny
        m = max(1, min(self.opts.restart, self.opts.max_iter))
        gm = (m + 8) * cols * ntr * 16.0
        vol = 6.0 * cols * nx * ny * nz * 16.0
        return slots + gm + vol

    def _admit_worker(self, w: int) -> bool:
        if len(self.workers[w]) >= self.max_workers:
            return False
        need = self.worker_bytes(self.max_cols)
        if self.workers[w]:
            free, _ = self.torch.cuda.mem_get_info()
            pending = sum(self.pending.values())
            if free - self.mem_reserve - pending < need:
                self.admission_log.append(f"omega {w}: extra worker refused ({free/1e9:.1f} GB free, "
                                          f"{pending/1e9:.1f} GB promised, {need/1e9:.1f} GB needed)")
                return False
            solver = hz.Solver.shared(self.primaries[w])
        else:
            solver = self.primaries[w]
        self.pending[id(solver)] = need
        self.workers[w].append(solver)
        if self.log:
            self.log(f"omega {w}: worker {len(self.workers[w])} admitted")
        self._start(w, solver)
        self.admission_log.append(f"omega {w}: worker {len(self.workers[w])} admitted")
        return True

    def _start(self, w: int, solver: hz.Solver):
        th = threading.Thread(target=self._work, args=(w, solver), daemon=True)
        self.threads.append(th)
        th.start()

    # ------------------------------------------------------------------ queue
    def submit(self, req: Request):
        req._left = req.R
        with self.cv:
            for c0 in range(0, req.R, self.max_cols):
                self.queues[req.omega_idx].append((req, c0, min(req.R, c0 + self.max_cols)))
            backlog = sum(b - a for _, a, b in self.queues[req.omega_idx])
            self.cv.notify_all()
        # admit another worker for this frequency when its backlog exceeds one batch
        if backlog > self.max_cols and self.running:
            with self.cv:
                self._admit_worker(req.omega_idx)

    def _take(self, w: int):
        items, cols = [], 0
        q = self.queues[w]
        while q and cols + (q[0][2] - q[0][1]) <= self.max_cols:
            it = q.popleft()
            items.append(it)
            cols += it[2] - it[1]
        return items, cols

    def _work(self, w: int, solver: hz.Solver):
        torch = self.torch
        nz, ny, nx = self.shape
        while True:
            with self.cv:
                while self.running and not self.queues[w]:
                    self.cv.wait(0.05)
                if not self.running and not self.queues[w]:
                    return
                items, cols = self._take(w)
            if not items:
                continue
            try:
                with torch.cuda.stream(solver.stream):
                    # every batch is solved max_cols wide (unused columns are zero and converge at
                    # once): one batch signature per handle, so the substitution autotuner and the
                    # CUDA-graph capture of the matrix-vector product run once, not once per width
                    rhs = torch.zeros((self.max_cols, nz, ny, nx), dtype=torch.complex128, device="cuda")
                    c = 0
                    for req, a, b in items:
                        src = torch.from_numpy(req.sources[a:b]).to("cuda")
                        k = torch.arange(c, c + (b - a), device="cuda")
                        rhs[k, src[:, 0], src[:, 1], src[:, 2]] = 1.0
                        c += b - a
                solver.stream.synchronize()
                # a batch that does not converge raises (HZ_ERR_NO_CONVERGENCE): its requests fail
                # instead of receiving unconverged columns
                u, info, st = solver.solve(rhs, self.opts)
                with torch.cuda.stream(solver.stream):
                    c = 0
                    outs = []
                    for req, a, b in items:
                        part = u[c:c + (b - a)]
                        if self.receivers is not None:
                            flat = part.reshape(b - a, -1)
                            part = flat[:, torch.from_numpy(self.receivers).to("cuda")]
                        outs.append(part.clone())
                        c += b - a
                solver.stream.synchronize()
                self._deliver(items, outs, time.perf_counter())
                if self.log:
                    self.log(f"omega {w}: batch of {cols} columns ({len(items)} items) done, "
                             f"iterations {info[0].iters}, refinements {info[0].refinements}")
            except Exception as e:  # a failed batch marks its requests; the server keeps going
                if self._failed_batch(w, solver, items, e):
                    solver.close()
                    return
                continue
            with self.cv:
                self.pending.pop(id(solver), None)

    def _deliver(self, items, outs, now: float):
        """Bookkeeping of a solved batch: copy each work item's columns into its request.  A request
        that already has a failed work item keeps its failure status (-1); it completes when its
        last work item has been accounted for, failed or delivered."""
        with self.cv:
            self.batches += 1
            self.max_requests_per_batch = max(self.max_requests_per_batch, len({id(r) for r, _, _ in items}))
            for (req, a, b), part in zip(items, outs):
                if req.status == 0:
                    if req.result is None:
                        shp = (req.R,) + tuple(part.shape[1:])
                        req.result = self.torch.empty(shp, dtype=part.dtype, device=part.device)
                    req.result[a:b] = part
                req._left -= (b - a)
                if req._left == 0:
                    req.t_done = now
            self.cv.notify_all()

    def _failed_batch(self, w: int, solver, items, e: Exception) -> bool:
        """Bookkeeping of a batch that raised: an out-of-memory batch goes back to the head of its
        queue (each work item at most twice) and an extra worker that hit it is retired; any other
        failure, or a third out-of-memory failure, marks the requests failed.  Returns whether the
        calling worker must retire (its handle is then closed by the caller)."""
        torch = self.torch
        # device memory ran out: an allocation failed, or a solve workspace did not fit (admission)
        oom = (isinstance(e, hz.HzError) and e.status in (hz.HZ_ERR_OOM, hz.HZ_ERR_ADMISSION)) or \
            isinstance(e, getattr(getattr(torch, "cuda", None), "OutOfMemoryError", ()))
        retire = False
        with self.cv:
            self.pending.pop(id(solver), None)
            if oom:
                retry, failed = [], []
                for it in items:
                    key = (it[0].rid, it[1])
                    self.retries[key] = self.retries.get(key, 0) + 1
                    (retry if self.retries[key] <= 2 else failed).append(it)
                for it in reversed(retry):       # back at the head, in their order
                    self.queues[w].appendleft(it)
                items = failed
                retire = solver is not self.primaries[w]
                if retire:
                    self.workers[w].remove(solver)
                    self.admission_log.append(f"omega {w}: worker retired after running out of memory")
            if items:
                self.errors.append(repr(e))
            if self.log:
                self.log(f"omega {w}: batch failed ({'out of memory' if oom else repr(e)})")
            for req, a, b in items:
                req.status = -1
                req.result = None           # a failed request delivers no partial result
                req._left -= (b - a)
                if req._left == 0:
                    req.t_done = time.perf_counter()
            self.cv.notify_all()
        if oom and not retire:
            time.sleep(0.2)   # let retiring workers free their memory before the retry
        return retire

    # ------------------------------------------------------------------ driver
    def serve(self, requests: Sequence[Request], realtime: bool = True, timeout: float = 3600.0):
        """Feed ``requests`` at their arrival offsets (seconds from now) and wait for all of them.
        Returns the wall time from the first arrival to the last completion."""
        self.running = True
        with self.cv:
            for w in range(len(self.primaries)):
                if self.workers[w]:          # handles admitted by an earlier serve(): run them again
                    for solver in self.workers[w]:
                        self._start(w, solver)
                else:
                    self._admit_worker(w)
        t0 = time.perf_counter()
        order = sorted(requests, key=lambda r: r.t_arrival)
        offsets = [r.t_arrival for r in order]
        for r, off in zip(order, offsets):
            if realtime:
                dt = t0 + off - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            r.t_arrival = time.perf_counter()
            self.submit(r)
        deadline = time.perf_counter() + timeout
        with self.cv:
            while any(r.t_done is None for r in order) and time.perf_counter() < deadline:
                self.cv.wait(0.05)
        self.running = False
        with self.cv:
            self.cv.notify_all()
        for th in self.threads:
            th.join(timeout=60)
        self.threads = []
        done = [r.t_done for r in order if r.t_done is not None]
        return (max(done) - min(r.t_arrival for r in order)) if done else float("nan")

    def close(self):
        for ws in self.workers:
            for s in ws[1:]:
                s.close()
        for s in self.primaries:
            s.close()


def latency_stats(requests: Sequence[Request]):
    lat = np.array([r.latency for r in requests if r.latency is not None])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "n": int(lat.size)}
