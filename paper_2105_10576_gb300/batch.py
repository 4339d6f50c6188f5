"""Concurrent stepping of many independent OSCAR instances (the batched sweep).

Each instance owns its CUDA stream. A batched step launches every instance's
drag step (oscar_drag_step_async), collects them (oscar_wait), then launches
every relaxation and collects those, so that the launches of many small grids
overlap on the GPU instead of running one instance at a time. Every instance
keeps its own arithmetic and launch order, so its results are the ones it gives
when stepped alone.
"""
from __future__ import annotations

from typing import Sequence

from . import oscar as ox


class Batch:
    def __init__(self, sims: Sequence["ox.Oscar"]):
        self.sims = list(sims)

    def _collect(self, launched):
        out = []
        err = None
        for s in launched:
            try:
                out.append(s.wait(strict=False))
            except ox.OscarError as e:   # keep collecting the others
                err = err or e
                out.append((e.code, 0, 0.0))
        if err is not None:
            raise err
        return out

    def step(self, dt_vd: Sequence[float], dt_cr: Sequence[float], N: Sequence[int]) -> list:
        """One drag step and one relaxation (up to N sub-steps) of every
        instance; returns k_f per instance."""
        launched = []
        try:
            for s, dt in zip(self.sims, dt_vd):
                s.drag_step_async(dt)
                launched.append(s)
        finally:
            self._collect(launched)
        launched = []
        try:
            for s, dt, n in zip(self.sims, dt_cr, N):
                s.relax_async(dt, n)
                launched.append(s)
        finally:
            res = self._collect(launched)
        return [kf for _, kf, _ in res]

    def close(self):
        for s in self.sims:
            s.close()
