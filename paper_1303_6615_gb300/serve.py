"""Continuous-batching server for parareal solves of the 1D rotating shallow-water system.

A request is one parareal problem (grid N, eps, nu, slices, horizon T, fine step
dt, quadrature points M, initial spectrum u0) solved until KMAX iterations or a
relative change <= TOL.  The server keeps every admitted problem's slice states
resident on the device and advances all of them together: each `step()` runs
one batched parareal level (arp_batch_iterate), so the fine sweeps and coarse
chains of all active problems share fused launches.  A request that runs alone
with nothing queued is finished in one arp_parareal_solve instead (its levels
overlapped where the library pipelines them), with the same result, when requests
arrive more slowly than that solve takes (mean inter-arrival gap, or the time since
the last arrival, above the remaining levels times the measured time per level of
such solves): under heavier load the one call would hold newcomers back, so the
request keeps advancing a level per step beside them.  Requests that arrive while
others are running are admitted at the next step, in arrival order, as slots
and device memory (arp_query_bytes) free up; finished problems leave the batch
and their slices are copied to the host.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import binding as b


@dataclass
class Request:
    n_grid: int
    eps: float
    nu: float
    slices: int
    t_end: float
    dt: float
    m_quad: int
    u0: np.ndarray                # (3, N/2+1) complex128
    k_max: int = 5
    tol: float = 0.0
    rid: int = -1
    arrival: float = 0.0          # server clock (seconds) when submitted
    # filled by the server
    admitted: float = float("nan")
    finished: float = float("nan")
    levels: int = -1
    change: float = float("nan")
    result: Optional[np.ndarray] = field(default=None, repr=False)   # (slices+1, 3, N/2+1)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def lone_solve_worthwhile(mean_gap: Optional[float], since_last: float, level_seconds: Optional[float],
                          remaining_levels: int) -> bool:
    """Whether a request running alone should finish in one call: with no arrival
    history or no measured level time, yes; else when the expected gap until the
    next arrival (the mean gap, or the time already passed since the last one if
    longer) exceeds the time the remaining levels take."""
    if mean_gap is None or level_seconds is None:
        return True
    return max(mean_gap, since_last) > remaining_levels * level_seconds


class Server:
    """Admits requests by device memory and slot count and advances all admitted
    ones by one parareal level per step."""

    def __init__(self, memory_budget: int = 16 << 30, max_active: int = 256, precision: int = b.ARP_FP32,
                 stream=None, lone_solve: bool = True):
        import torch
        self.torch = torch
        self.budget = memory_budget
        self.max_active = max_active
        self.precision = precision
        self.stream = stream
        self.pending: collections.deque[Request] = collections.deque()
        self.active: list[tuple[Request, b.Solver]] = []
        self.done: list[Request] = []
        self.in_use = 0
        self.batch = b.arp_batch_create(None, capacity=max_active)
        self.members: list[int] = []
        self.t0 = time.perf_counter()
        self.next_id = 0
        # a request running alone with nothing queued finishes in one arp_parareal_solve
        # (its levels pipelined where the library can), which gives the same slices,
        # levels and change as the batched levels -- while arrivals are sparse enough
        self.lone_solve = lone_solve
        self.mean_gap: Optional[float] = None       # running mean of inter-arrival gaps (s)
        self.last_arrival: Optional[float] = None
        self.level_seconds: Optional[float] = None  # running mean time per level of lone solves (s)

    def clock(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request) -> Request:
        req.rid = self.next_id
        self.next_id += 1
        req.arrival = self.clock()
        if self.last_arrival is not None:
            gap = req.arrival - self.last_arrival
            self.mean_gap = gap if self.mean_gap is None else 0.75 * self.mean_gap + 0.25 * gap
        self.last_arrival = req.arrival
        self.pending.append(req)
        return req

    def _bytes(self, r: Request) -> int:
        return b.arp_query_bytes(r.n_grid, r.slices, r.m_quad, self.precision)

    def _admit(self) -> None:
        while self.pending and len(self.active) < self.max_active:
            r = self.pending[0]
            need = self._bytes(r)
            if need > self.budget:
                raise ValueError(f"request {r.rid} needs {need} bytes, more than the whole budget")
            if self.in_use + need > self.budget:
                break
            self.pending.popleft()
            s = b.Solver(r.n_grid, r.eps, r.nu, r.slices, r.t_end / r.slices, r.dt, r.m_quad,
                         precision=self.precision)
            b.arp_set_initial(s.ctx, self.torch.from_numpy(np.ascontiguousarray(r.u0)).cuda(), self.stream)
            r.admitted = self.clock()
            self.active.append((r, s))
            self.in_use += need

    def _sync_members(self) -> None:
        ctxs = [s.ctx for _, s in self.active]
        if ctxs != self.members:
            b.arp_batch_reset(self.batch, ctxs)
            self.members = ctxs

    def step(self) -> int:
        """Admit what fits, run one batched level, retire finished requests.
        Returns the number of active requests after the step."""
        self._admit()
        if not self.active:
            return 0
        if self.lone_solve and len(self.active) == 1 and not self.pending and self._lone_ok():
            r, s = self.active[0]
            b.arp_set_option(s.ctx, b.ARP_OPT_KMAX, r.k_max)
            b.arp_set_option(s.ctx, b.ARP_OPT_TOL, r.tol)
            lv0 = b.arp_info(s.ctx)["level"]
            t = time.perf_counter()
            lv, ch = b.arp_parareal_solve(s.ctx, self.stream)
            if lv > lv0:  # the call returns after the last level's change is read back
                per = (time.perf_counter() - t) / (lv - lv0)
                self.level_seconds = per if self.level_seconds is None else 0.75 * self.level_seconds + 0.25 * per
            levels, changes = [lv], [ch]
        else:
            self._sync_members()
            levels, changes = b.arp_batch_iterate(self.batch, len(self.active), self.stream)
        still = []
        for (r, s), lv, ch in zip(self.active, levels, changes):
            r.levels, r.change = lv, ch
            if lv >= r.k_max or (lv >= 1 and ch <= r.tol):
                out = self.torch.empty((r.slices + 1, 3, r.n_grid // 2 + 1), dtype=self.torch.complex128)
                b.arp_get_slices(s.ctx, out, self.stream)
                r.result = out.numpy()
                r.finished = self.clock()
                self.in_use -= self._bytes(r)
                s.close()
                self.done.append(r)
            else:
                still.append((r, s))
        self.active = still
        return len(self.active)

    def _lone_ok(self) -> bool:
        r, s = self.active[0]
        since = self.clock() - self.last_arrival if self.last_arrival is not None else 0.0
        remaining = r.k_max - b.arp_info(s.ctx)["level"]
        return lone_solve_worthwhile(self.mean_gap, since, self.level_seconds, remaining)

    def close(self) -> None:
        for _, s in self.active:
            s.close()
        self.active = []
        if self.batch:
            b.arp_batch_destroy(self.batch)
            self.batch = 0


def replay(server: Server, trace: list[tuple[float, Request]]) -> list[Request]:
    """Submits each request of `trace` (arrival offset in seconds, request) when the
    server clock reaches its offset, stepping the server meanwhile; returns the
    finished requests in completion order."""
    trace = sorted(trace, key=lambda t: t[0])
    i = 0
    start = server.clock()
    while i < len(trace) or server.active or server.pending:
        now = server.clock() - start
        while i < len(trace) and trace[i][0] <= now:
            server.submit(trace[i][1])
            i += 1
        if server.active or server.pending:
            server.step()
        elif i < len(trace):
            time.sleep(min(0.001, max(0.0, trace[i][0] - now)))
    return list(server.done)


def solve_alone(req: Request, precision: int, stream=None) -> np.ndarray:
    """The same request on its own context (the reference for batch invariance,
    and the one-at-a-time path)."""
    import torch
    with b.Solver(req.n_grid, req.eps, req.nu, req.slices, req.t_end / req.slices, req.dt, req.m_quad,
                  precision=precision) as s:
        b.arp_set_initial(s.ctx, torch.from_numpy(np.ascontiguousarray(req.u0)).cuda(), stream)
        lv, ch = -1, float("inf")
        while not (lv >= req.k_max or (lv >= 1 and ch <= req.tol)):
            lv, ch = b.arp_parareal_iterate(s.ctx, stream)
        out = torch.empty((req.slices + 1, 3, req.n_grid // 2 + 1), dtype=torch.complex128)
        b.arp_get_slices(s.ctx, out, stream)
        return out.numpy()
