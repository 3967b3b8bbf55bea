"""Served solve stream with continuous batching.

Requests (a mesh, order p, form, precision) arrive over time.  The scheduler keeps
every admitted request resident on the device (its mesh, D factors and CG state, in a
library op on a stream of its own), admits waiting requests in arrival order whenever
the HBM budget allows, and on every tick advances each active request by a bounded
number of CG iterations (fepa_solver_advance), so requests that arrive while others
are running join at the next tick and their work overlaps on the device.  Finished
requests leave at tick boundaries and release their memory.  With solver="auto",
diffusion requests of at least pmg_min_dofs DOFs are solved by CG preconditioned with
the p-multigrid V-cycle (Sec. 2.1; FP64 V-cycle for FP64 requests, FP32 V-cycle inside
the FP64 CG for mixed ones) instead of Jacobi-PCG, advanced by the resumable
fepa_mg_solver_* calls; the others keep Jacobi (mass matrices are well conditioned, and
below the threshold the V-cycle's set-up and launches cost more than they save).

The scheduler is plain host logic; all device work goes through the C ABI of
libfepa.so (GpuExecutor).  A FakeExecutor with the same interface drives the host
logic in CPU tests.
"""
from __future__ import annotations

import dataclasses
import math
import time
from collections import deque
from typing import Callable, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    form: str                 # "mass" | "diffusion"
    p: int
    n: tuple                  # elements per direction
    mesh_seed: int
    precision: str = "fp64"   # "fp64" | "mixed"
    arrival: float = 0.0      # seconds after the start of the run
    rtol: float = 1e-10
    solver: str = "jacobi"    # "jacobi" | "pmg" (set by the server's solver policy)

    @property
    def ndofs(self) -> int:
        nx, ny, nz = self.n
        return (self.p * nx + 1) * (self.p * ny + 1) * (self.p * nz + 1)

    @property
    def nelems(self) -> int:
        nx, ny, nz = self.n
        return nx * ny * nz


def _torch_block(nbytes: int) -> int:
    """Device memory torch's caching allocator may take for one tensor: a 2 MB segment below
    1 MB, a 20 MB segment below 10 MB, else the size rounded up to 2 MB."""
    mb = 1 << 20
    if nbytes <= mb:
        return 2 * mb
    if nbytes <= 10 * mb:
        return 20 * mb
    return (nbytes + 2 * mb - 1) // (2 * mb) * (2 * mb)


def device_bytes(req: Request) -> int:
    """Upper estimate of the device memory a resident request holds: vertices, element
    map, FP64 D and its (hi, lo) float copy for the double-float action, FP32 D (mixed),
    the CG work vectors; the right-hand side and solution as torch allocates them; and a
    fixed 16 MB for the small arrays, graphs and allocation granularity of an op (measured:
    within it for every request of the served mix once the library is loaded)."""
    n, q, E, N = req.p + 1, req.p + 2, req.nelems, req.ndofs
    ncomp = 6 if req.form == "diffusion" else 1
    nv = (req.n[0] + 1) * (req.n[1] + 1) * (req.n[2] + 1)
    by = 24 * nv + 4 * n ** 3 * E + 2 * 8 * ncomp * q ** 3 * E
    by += 8 * N * 6                                   # r, d, h, 1/diag, copies
    if req.precision == "mixed":
        by += 4 * ncomp * (((q ** 3) + 3) & ~3) * E   # padded FP32 D
        by += 4 * N * 6 + 8 * N                       # FP32 loop vectors, FP64 residual
    levels = 0
    if req.solver == "pmg":
        # coarser levels (orders p/2, p/4, ..., 1): each at most the fine level's D (FP64, its
        # (hi, lo) and FP32 copies) and map scaled by its point and node counts, plus the V-cycle
        # and outer PCG vectors of every level and a fixed 16 MB per level op
        pc, frac = req.p, 0.0
        while pc > 1:
            pc = max(1, pc // 2)
            frac += ((pc + 2) / q) ** 3 + ((pc + 1) / n) ** 3
            levels += 1
        by += int(frac * (20 * ncomp * q ** 3 * E + 4 * n ** 3 * E)) + 8 * N * 20
    return int(by * 1.1) + 2 * _torch_block(8 * N) + (16 << 20) * (1 + levels)


def estimated_work(req: Request) -> float:
    """Rough GPU cost of a request for scheduling (not a measurement): DOFs times the Jacobi-PCG
    iteration count, which grows like p times the elements per side, with an FP32 iteration of
    the mixed solve counted at a quarter of an FP64 one (the FP32 action moves half the bytes and
    avoids the FP64-accurate arithmetic)."""
    if req.solver == "pmg":
        return req.ndofs * 120.0   # ~15 iterations of a V-cycle costing ~8 operator actions
    its = 4.4 * req.p * max(req.n)
    return req.ndofs * its * (0.25 if req.precision == "mixed" else 1.0)


@dataclasses.dataclass
class Outcome:
    rid: int
    arrival: float
    admitted: float
    finished: float
    status: int
    iterations: int
    outer_iterations: int
    rel_residual: float
    ndofs: int
    result: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Server:
    """Continuous-batching scheduler over an executor (GpuExecutor or FakeExecutor)."""

    def __init__(self, executor, hbm_budget: float = 150e9, tick_iters: int = 32, max_active: int = 256,
                 keep_results: bool = False, clock: Callable[[], float] = time.perf_counter, policy: str = "fifo",
                 tick_seconds: Optional[float] = None, solver: str = "jacobi", pmg_min_dofs: int = 50000):
        """policy: "fifo" admits waiting requests in arrival order; "sjf" admits the waiting request
        with the least estimated work first (shorter waits for short requests when slots or memory
        are scarce; a request that can never fit is rejected either way).  tick_seconds: if set, a
        request advances by enough iterations per tick for about this much estimated GPU time (at
        least tick_iters, at most 4096); else by tick_iters.  solver: "jacobi" solves every request
        by Jacobi-PCG (or its refined mixed form); "auto" gives diffusion requests of at least
        pmg_min_dofs DOFs the p-multigrid preconditioner."""
        if solver not in ("jacobi", "auto"):
            raise ValueError("solver must be 'jacobi' or 'auto'")
        self.solver = solver
        self.pmg_min_dofs = int(pmg_min_dofs)
        self.tick_seconds = tick_seconds
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be 'fifo' or 'sjf'")
        self.policy = policy
        self.ex = executor
        self.budget = float(hbm_budget)
        self.tick_iters = int(tick_iters)
        self.max_active = int(max_active)
        self.keep_results = keep_results
        self.clock = clock
        self.in_use = 0
        self.peak_in_use = 0
        self.pending: deque = deque()
        self.active: dict = {}       # rid -> (request, handle, bytes, admitted)
        self.done: list = []
        self.rejected: list = []
        self.ticks = 0
        self.max_concurrent = 0
        self.inflight: dict = {}     # rid -> an advance of the request may still be running
        self.pmg_count = 0

    def _admit(self, now: float):
        if self.policy == "sjf" and len(self.pending) > 1:
            self.pending = deque(sorted(self.pending, key=lambda r: (estimated_work(r), r.arrival, r.rid)))
        while self.pending and len(self.active) < self.max_active:
            req = self.pending[0]
            need = device_bytes(req)
            if need > self.budget:             # can never fit: reject rather than block the queue
                self.pending.popleft()
                self.rejected.append(req.rid)
                continue
            if self.in_use + need > self.budget:
                break                          # wait for memory to free up (queue order kept)
            self.pending.popleft()
            handle = self.ex.start(req)
            self.pmg_count += req.solver == "pmg"
            self.in_use += need
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            self.active[req.rid] = (req, handle, need, now)
        self.max_concurrent = max(self.max_concurrent, len(self.active))

    def choose_solver(self, req: Request):
        """The solver policy, applied when a request arrives."""
        if self.solver == "auto" and req.form == "diffusion" and req.ndofs >= self.pmg_min_dofs:
            req.solver = "pmg"

    def tick_size(self, req: Request) -> int:
        """Iterations per advance: tick_iters, or with tick_seconds enough for about that much GPU
        time (estimated from the DOFs), so the host's per-tick round trip stays small next to it.
        A multigrid-preconditioned request advances by 1 to 4 of its (much costlier) iterations."""
        if req.solver == "pmg":
            if self.tick_seconds is None:
                return 1
            return int(min(4, max(1, self.tick_seconds / max(req.ndofs / 1.2e8, 1e-12))))
        if self.tick_seconds is None:
            return self.tick_iters
        per_it = req.ndofs / (25e9 if req.precision == "mixed" else 6e9)
        return int(min(4096, max(self.tick_iters, self.tick_seconds / max(per_it, 1e-12))))

    def _tick(self):
        advanced = 0
        for rid, (req, h, need, adm) in self.active.items():
            if not self.inflight.get(rid):   # one advance in flight per request: no queue flooding
                self.ex.advance(h, self.tick_size(req))
                self.inflight[rid] = True
                advanced += 1
        self.ticks += 1
        finished = []
        for rid, (req, h, need, adm) in self.active.items():
            st = self.ex.poll(h)
            if st is not None:
                self.inflight[rid] = False
            if st is not None and st["done"]:
                finished.append(rid)
                res = self.ex.result(h) if self.keep_results else None
                self.done.append(Outcome(rid, req.arrival, adm, self.clock() - self.t0, st["status"],
                                         st["iterations"], st["outer_iterations"], st["rel_residual"],
                                         req.ndofs, res))
        for rid in finished:
            req, h, need, adm = self.active.pop(rid)
            self.inflight.pop(rid, None)
            self.ex.release(h)
            self.in_use -= need
        if not advanced and not finished:
            time.sleep(50e-6)   # everything is busy on the device: let other threads run

    def run(self, requests):
        """Serve `requests` (arrival times relative to the start); returns the outcomes."""
        arrivals = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        self.t0 = self.clock()
        while arrivals or self.pending or self.active:
            now = self.clock() - self.t0
            while arrivals and arrivals[0].arrival <= now:
                req = arrivals.popleft()
                self.choose_solver(req)
                self.pending.append(req)
            self._admit(now)
            if self.active:
                self._tick()
            elif arrivals and not self.pending:
                wait = arrivals[0].arrival - (self.clock() - self.t0)
                if wait > 0:
                    time.sleep(min(wait, 0.01))
        self.makespan = self.clock() - self.t0
        return sorted(self.done, key=lambda o: o.rid)

    def report(self):
        lat = np.array([o.latency for o in self.done]) if self.done else np.zeros(1)
        work = sum(o.ndofs * o.iterations for o in self.done)
        mem = getattr(self.ex, "measured", [])
        return {"completed": len(self.done), "rejected": len(self.rejected), "makespan_s": self.makespan,
                "policy": self.policy, "solver": self.solver, "pmg_requests": self.pmg_count,
                "device_bytes_check": {"requests": len(mem),
                                       "max_measured_over_estimate": max((m / e for m, e in mem), default=None)},
                "solves_per_s": len(self.done) / self.makespan if self.makespan > 0 else 0.0,
                "gdofs_per_cg_iter": work / self.makespan / 1e9 if self.makespan > 0 else 0.0,
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "max_concurrent": self.max_concurrent, "peak_device_bytes": self.peak_in_use, "ticks": self.ticks}


def poisson_arrivals(requests, rate: float, seed: int = 0):
    """Assign Poisson arrival times (rate requests/s) in request order."""
    rng = np.random.default_rng(seed)
    t = 0.0
    for r in requests:
        t += rng.exponential(1.0 / rate)
        r.arrival = t
    return requests


# ----------------------------------------------------------------------------- executors

class GpuExecutor:
    """Runs each request as a resident library op on its own CUDA stream.  With priorities, a
    request whose estimated work is below short_work runs on a high-priority stream, so the GPU
    dispatches its small kernels ahead of the long requests' (shorter latency for short requests;
    the long ones take the rest of the machine).  With async_start, a request's op is built (mesh,
    D, diagonal, solver state: 1-40 ms each on the host, up to ~0.5 s for a new size class) by a
    worker thread while the scheduler keeps advancing the requests already running; until it is
    ready the request takes no steps and polls as busy.  Without it, each start also measures the
    device memory the request took (free memory before and after) against device_bytes."""

    def __init__(self, vertices_fn, inner_rtol: float = 1e-4, priorities: bool = True, short_work: float = 5e9,
                 async_start: bool = False, workers: int = 1):
        import torch
        self.torch = torch
        self.vertices_fn = vertices_fn      # (n, seed) -> vertex array
        self.inner_rtol = inner_rtol
        self.priorities = priorities
        self.short_work = short_work
        self.measured = []                  # (device bytes taken, device_bytes estimate) per request
        self.device = torch.cuda.current_device()
        self.pool = None
        if async_start:
            from concurrent.futures import ThreadPoolExecutor
            self.pool = ThreadPoolExecutor(max_workers=workers)

    def start(self, req: Request):
        if self.pool is None:
            return self._create(req)
        return {"future": self.pool.submit(self._create, req)}

    def _ready(self, h):
        f = h.get("future")
        if f is None:
            return True
        if not f.done():
            return False
        h.update(f.result())    # (re-raises a failed creation)
        del h["future"]
        return True

    def _create(self, req: Request):
        from .fepa import Multigrid, Operator
        torch = self.torch
        if self.pool is not None:
            torch.cuda.set_device(self.device)   # (the current device is per thread)
        high = self.priorities and estimated_work(req) < self.short_work
        stream = torch.cuda.Stream(priority=-1 if high else 0)
        free0 = torch.cuda.mem_get_info()[0]   # (allocations are synchronous: no device sync needed)
        with torch.cuda.stream(stream):
            op = Operator(*req.n, self.vertices_fn(req.n, req.mesh_seed), req.p, form=req.form)
            if req.form == "diffusion":
                op.set_essential(op.boundary_dofs())
                b = op.rhs_sine(3 * math.pi ** 2)
            else:
                b = op.rhs_sine(1.0)
            x = torch.zeros(op.N, dtype=torch.float64, device="cuda")
            mg = None
            if req.solver == "pmg":
                mg = Multigrid(op, smooth_degree=2, coarse_degree=24,
                               precision="fp32" if req.precision == "mixed" else "fp64")
                mg.solver_start(b, x, rtol=req.rtol)
            else:
                op.solver_start(b, x, kind="refined" if req.precision == "mixed" else "cg", rtol=req.rtol,
                                inner_rtol=self.inner_rtol)
        if self.pool is None:   # (other threads' allocations would blur the difference)
            self.measured.append((max(0, free0 - torch.cuda.mem_get_info()[0]), device_bytes(req)))
        return {"op": op, "mg": mg, "stream": stream, "b": b, "x": x}

    def advance(self, h, iters: int):
        if not self._ready(h):
            return
        with self.torch.cuda.stream(h["stream"]):
            (h["mg"] or h["op"]).solver_advance(iters)

    def poll(self, h):
        if not self._ready(h):
            return None
        with self.torch.cuda.stream(h["stream"]):
            return (h["mg"] or h["op"]).solver_poll(blocking=False)

    def result(self, h):
        with self.torch.cuda.stream(h["stream"]):
            return h["x"].cpu().numpy()

    def release(self, h):
        if "future" in h:
            h.update(h.pop("future").result())
        h["stream"].synchronize()
        if h["mg"] is not None:
            h["mg"].close()
        h["op"].close()
        h.clear()


class FakeExecutor:
    """Host-only stand-in: a request needs `iters_fn(req)` iterations; every advance
    performs up to the given number.  Used to test the scheduler without a GPU."""

    def __init__(self, iters_fn):
        self.iters_fn = iters_fn
        self.log = []

    def start(self, req):
        self.log.append(("start", req.rid))
        return {"req": req, "need": int(self.iters_fn(req)), "done": 0}

    def advance(self, h, iters):
        h["done"] = min(h["need"], h["done"] + iters)

    def poll(self, h):
        d = h["done"] >= h["need"]
        return {"done": d, "status": 0, "iterations": h["done"], "outer_iterations": 0, "rel_residual": 0.0}

    def result(self, h):
        return None

    def release(self, h):
        self.log.append(("release", h["req"].rid))
