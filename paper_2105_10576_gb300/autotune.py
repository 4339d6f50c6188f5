"""Measuring autotuner of the pressure solver's schedule (oscar_schedule).

The multigrid schedule (smoothing sweeps per level group, which levels go to
the single coarse CTA, how often the coarsest level's inverse is refreshed)
and the block shape of the cell kernels change how fast the pressure solves
of an instance converge and run, not what they converge to. The best choice
depends on the grid: on a small 2D grid every launch is latency-bound and
fewer sweeps win, on a large 3D grid more sweeps pay for themselves through
fewer PCG iterations. This module picks a schedule per problem by timing it.

tune() does a coordinate descent over SPACE: starting from the default, each
knob in turn takes each of its values with the others fixed, and the fastest
(wall seconds per cell-update of a few OSCAR steps of a fresh instance of the
same problem, after one untimed step that builds the graphs) is kept. Results
are cached per (dimension, grid, precision), so a batch of instances of a few
grid sizes is tuned once per size. Tuning runs on scratch instances; the
caller's instances are not touched.
"""
from __future__ import annotations

import time

from . import oscar as ox

DEFAULT = dict(mg_nu=2, mg_nu_mid=2, mg_nu_cta=2, cta_cells=1024, coarse_refresh=8, block_x=0, cta_global=1)
SPACE = (("mg_nu", (1, 2, 3)), ("mg_nu_mid", (1, 2, 3)), ("mg_nu_cta", (1, 2, 3)),
         ("cta_cells", (256, 512, 1024)), ("cta_global", (1, 0)), ("block_x", (0, 128, 64, 32)))

_cache: dict = {}


def _key(params: dict):
    return (params["dim"], params["nx"], params["ny"], params["nz"] if params["dim"] == 3 else 1,
            params["precision"])


def probe(params, solid, alpha0, sched, dt_vd, dt_cr, n_sub, rounds=2, stream=0):
    """Wall seconds per cell-update of `rounds` OSCAR steps (one drag step and
    up to n_sub relaxation sub-steps each) of a fresh instance using `sched`,
    after one untimed step; inf when a step fails or the schedule is refused."""
    g = ox.Oscar(params, solid, alpha0, stream)
    try:
        try:
            g.set_schedule(sched)
        except ox.OscarError:
            return float("inf")
        g.drag_step(dt_vd)
        g.relax(dt_cr, n_sub)
        cu0 = g.stats()["cell_updates"]
        t0 = time.perf_counter()
        for _ in range(rounds):
            g.drag_step(dt_vd)
            g.relax(dt_cr, n_sub)
        cu = g.stats()["cell_updates"] - cu0
        return (time.perf_counter() - t0) / max(cu, 1)
    except ox.OscarError:
        return float("inf")
    finally:
        g.close()


def tune(params, solid, alpha0, dt_vd, dt_cr, n_sub=8, rounds=2, stream=0, use_cache=True, log=None):
    """The fastest schedule found by coordinate descent (see the module text).
    `log`, if a list, receives (schedule, seconds per cell-update) per trial."""
    key = _key(params)
    if use_cache and key in _cache:
        return dict(_cache[key])
    best = dict(DEFAULT)
    seen = {}

    def cost(s):
        k = tuple(sorted(s.items()))
        if k not in seen:
            seen[k] = probe(params, solid, alpha0, s, dt_vd, dt_cr, n_sub, rounds, stream)
            if log is not None:
                log.append((dict(s), seen[k]))
        return seen[k]

    best_cost = cost(best)
    for name, values in SPACE:
        for v in values:
            if v == best[name]:
                continue
            cand = dict(best, **{name: v})
            c = cost(cand)
            if c < best_cost:
                best, best_cost = cand, c
    _cache[key] = dict(best)
    return best
