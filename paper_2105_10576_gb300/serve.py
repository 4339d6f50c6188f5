"""Serving loop for OSCAR simulations (continuous batching).

Requests arrive over time; each asks for a number of OSCAR steps (one drag step
and one relaxation per step) on its own grid and geometry. The server admits a
waiting request, first come first served, as soon as its device memory
(oscar_footprint, computed without allocating) fits the budget beside the
instances already resident, and keeps every admitted instance's fields and
multigrid hierarchy in device memory until its last step. Each instance runs on
its own stream: whenever its launched phase has finished (oscar_query) the server
collects it and launches the next one at once, so requests that arrive while
others are on the GPU join the work already in flight. A request's
time-to-solution runs from its arrival to the end of its last step. Each
instance's arithmetic and launch order are its own, so its results are those it
gives when run alone.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import oscar as ox


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    params: dict
    solid: np.ndarray
    alpha0: np.ndarray
    dt_vd: float
    dt_cr: float
    N: int                  # relaxation sub-steps allowed per step
    steps: int              # OSCAR steps requested


@dataclass
class Record:
    rid: int
    arrival: float
    admitted: float = -1.0
    done: float = -1.0
    n_fluid: int = 0
    cell_updates: int = 0
    device_bytes: int = 0
    status: int = 0         # 0, or the first non-zero status of a step (or -1 rejected: larger than the budget)
    k_f: List[int] = field(default_factory=list)
    alpha: Optional[np.ndarray] = None

    @property
    def time_to_solution(self) -> float:
        return self.done - self.arrival


class Server:
    def __init__(self, budget_bytes: int, max_active: int = 256,
                 clock: Callable[[], float] = time.perf_counter, idle_sleep: float = 50e-6):
        self.budget = int(budget_bytes)
        self.max_active = max_active
        self.clock = clock
        self.idle_sleep = idle_sleep

    def run(self, requests: List[Request], keep_alpha: bool = False) -> List[Record]:
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque = deque()
        active = []          # [request, sim, record, footprint, phase (0 drag, 1 relax), steps done]
        records = []
        used = 0
        self.max_concurrent = 0
        self.max_used = 0
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting and len(active) < self.max_active:
                r = waiting[0]
                fp = ox.oscar_footprint(r.params)
                rec = Record(r.rid, r.arrival)
                if fp > self.budget:              # can never fit: reject
                    waiting.popleft()
                    rec.status = -1
                    records.append(rec)
                    continue
                if used + fp > self.budget:
                    break                         # first come, first served
                waiting.popleft()
                sim = ox.Oscar(r.params, r.solid, r.alpha0)
                used += fp
                rec.admitted = self.clock() - t0
                rec.n_fluid = sim.stats()["n_fluid"]
                rec.device_bytes = fp
                sim.drag_step_async(r.dt_vd)
                active.append([r, sim, rec, fp, 0, 0])
            self.max_concurrent = max(self.max_concurrent, len(active))
            self.max_used = max(self.max_used, used)
            progressed = False
            still = []
            for a in active:
                r, sim, rec, fp, phase, done = a
                if not sim.query():
                    still.append(a)
                    continue
                progressed = True
                rc, kf, _ = sim.wait(strict=False)
                if rc and not rec.status:
                    rec.status = rc
                if phase == 0:
                    rec.cell_updates += rec.n_fluid
                    sim.relax_async(r.dt_cr, r.N)
                    a[4] = 1
                    still.append(a)
                    continue
                rec.cell_updates += rec.n_fluid * kf
                rec.k_f.append(kf)
                a[5] = done = done + 1
                if done < r.steps:
                    sim.drag_step_async(r.dt_vd)
                    a[4] = 0
                    still.append(a)
                    continue
                rec.done = self.clock() - t0
                if keep_alpha:
                    rec.alpha = sim.field(ox.FIELD_ALPHA)
                sim.close()
                used -= fp
                records.append(rec)
            active = still
            if not progressed and active:
                time.sleep(self.idle_sleep)
            elif not active and pending and not waiting:
                time.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
        return sorted(records, key=lambda x: x.rid)


def run_alone(r: Request) -> Record:
    """The same request on an idle GPU, synchronously (for comparison)."""
    sim = ox.Oscar(r.params, r.solid, r.alpha0)
    rec = Record(r.rid, 0.0, n_fluid=sim.stats()["n_fluid"])
    for _ in range(r.steps):
        rc = sim.drag_step(r.dt_vd, strict=False)
        rc2, kf, _ = sim.relax(r.dt_cr, r.N, strict=False)
        rec.status = rec.status or rc or rc2
        rec.k_f.append(kf)
        rec.cell_updates += rec.n_fluid * (1 + kf)
    rec.alpha = sim.field(ox.FIELD_ALPHA)
    sim.close()
    return rec
