#!/usr/bin/env python3
"""Write bubble_rounding_spread.json: how far the FP64 oracle's own 128x16
bubble-channel runs move when the initial phase field is perturbed at the
rounding level.

The oracle solves every pressure equation of this case exactly (banded
Cholesky). Each perturbed run multiplies alpha0 by (1 + s 2^-52) with s a
seeded pattern of -1/0/+1 per cell (one unit in the last place), then runs the
same OSCAR sequence (20 drag steps, each followed by up to 50 relaxation
sub-steps; Section 3) and the same 2000 standard steps (Section 2.2). The
largest max-norm relative difference to the unperturbed run, per field, is the
spread that rounding alone produces in this problem: at the 1000:1.2 density
ratio the parasitic-current dynamics amplify rounding differences over
thousands of pressure solves. No implementation whose arithmetic is rounded
differently (another summation order, another solver) can be expected to agree
with the oracle more closely than this.

Calls only the oracle and the seeded input generators.
  python tests/golden/make_bubble_rounding_spread.py [--runs K] [--jobs J]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

FIELDS = ["alpha", "p", "ux", "uy", "uvdx", "uvdy", "ucrx", "ucry", "p_vd", "p_cr",
          "phi_vd_x", "phi_vd_y", "phi_cr_x", "phi_cr_y"]


def _ids(oracle):
    return {"alpha": oracle.ALPHA, "p": oracle.P, "ux": oracle.UX, "uy": oracle.UY, "uvdx": oracle.UVDX,
            "uvdy": oracle.UVDY, "ucrx": oracle.UCRX, "ucry": oracle.UCRY, "p_vd": oracle.P_VD,
            "p_cr": oracle.P_CR, "phi_vd_x": oracle.PHI_VD, "phi_vd_y": oracle.PHI_VD + 1,
            "phi_cr_x": oracle.PHI_CR, "phi_cr_y": oracle.PHI_CR + 1}


def run_case(seed):
    """Fields after the OSCAR run and after the standard run; seed < 0 = unperturbed."""
    import oracle
    from paper_2105_10576_gb300 import inputs
    c = inputs.channel_bubble_2d(cg_rtol=1e-15, cg_maxit=400)
    a0 = c.alpha0.copy()
    if seed >= 0:
        s = np.random.default_rng(seed).integers(-1, 2, a0.shape)
        a0 = a0 * (1.0 + s * 2.0 ** -52)
    dt_cfl, dt_b, dt_vd, N = oracle.timesteps(c.params, c.meta["c_cfl"])
    ids = _ids(oracle)
    o = oracle.OracleState(c.params, c.solid, a0)
    for _ in range(c.meta["n_drag"]):
        o.drag_step(dt_vd)
        o.relax(dt_vd / N, N)
    oscar = {k: o.field(v) for k, v in ids.items()}
    s_ = oracle.OracleState(c.params, c.solid, a0)
    for _ in range(c.meta["n_standard"]):
        s_.standard_step(dt_vd / N)
    std = {k: s_.field(v) for k, v in ids.items()}
    return oscar, std


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=8)
    ap.add_argument("--jobs", type=int, default=min(8, os.cpu_count() or 1))
    args = ap.parse_args()
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.jobs) as pool:
        res = pool.map(run_case, [-1] + list(range(args.runs)))
    base = res[0]
    out = {"runs": args.runs, "perturbation": "alpha0 * (1 + s 2^-52), s in {-1,0,1} per cell, seeds 0..runs-1",
           "oscar": {}, "standard": {}}
    for which, idx in (("oscar", 0), ("standard", 1)):
        for f in FIELDS:
            y = base[idx][f]
            m = np.abs(y).max()
            worst = 0.0
            for r in res[1:]:
                d = np.abs(r[idx][f] - y).max()
                worst = max(worst, d / m if m > 0 else d)
            out[which][f] = worst
    path = os.path.join(HERE, "bubble_rounding_spread.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(json.dumps(out, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
