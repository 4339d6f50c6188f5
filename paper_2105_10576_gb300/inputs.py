"""Seeded synthetic inputs: grids, solid masks, initial phase fields, fluid sets.

This module is shared by the CUDA path, the oracle, the tests and the bench. It
holds geometry and problem-statement data only (the inputs of the paper's
problem statement, Section 3: grid with solid walls, an inlet with a constant
injected velocity, a free outlet, fluid properties, initial alpha). It holds
none of the method's arithmetic: no transport, curvature, pressure or
time-step control.

Array conventions (used everywhere in this project):
  * cell arrays have shape (nz, ny, nx) in 3D and (ny, nx) in 2D, C order, so
    the flat cell index is i + nx*(j + ny*k) (x fastest);
  * solid masks are uint8, 1 = solid, 0 = fluid;
  * alpha = 1 marks phase 1 (density rho1, viscosity mu1);
  * the inlet is the x-min boundary, the outlet the x-max boundary, every other
    domain boundary is a solid wall.

The injected velocity comes from the capillary number Ca = mu U / sigma
(Section 2.1), with mu the viscosity of water in every workload.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Convergence-test modes (mirrors include/oscar.h).
CONV_PRES_RESID = 0   # normalised initial residual of the 1st PISO pressure equation (Section 3.2)
CONV_DU_MAX = 1       # max |u_cr^{k+1} - u_cr^k| / U_inlet
CONV_AREA = 2         # relative change of sigma * area + kinetic energy per sub-step (Section 6 variant)

PREC_FP64 = 0
PREC_MIXED = 1


def default_params(**kw) -> dict:
    """Numerical parameters shared by every workload; keyword overrides win."""
    p = dict(
        dim=2, nx=8, ny=8, nz=1, hx=1e-6, hy=1e-6, hz=1e-6,
        rho1=1.0, rho2=1.0, mu1=1e-3, mu2=1e-3, sigma=0.0, theta_deg=90.0,
        U_inlet=0.0, alpha_inlet=0.0,
        n_piso=3, n_smooth=2, c_alpha=1.0,
        conv_mode=CONV_PRES_RESID, conv_tol=1e-4,
        cg_rtol=1e-13, cg_maxit=2000,
        precision=PREC_FP64,
    )
    p.update(kw)
    return p


@dataclasses.dataclass
class Case:
    """One simulation instance: parameters, solid mask, initial alpha, run meta."""
    name: str
    params: dict
    solid: np.ndarray
    alpha0: np.ndarray
    meta: dict

    @property
    def shape(self):
        return self.solid.shape

    @property
    def n_fluid(self) -> int:
        return int((self.solid == 0).sum())


def _cell_centres(n: int, h: float) -> np.ndarray:
    return (np.arange(n) + 0.5) * h


def keep_outlet_connected(solid: np.ndarray) -> np.ndarray:
    """Turn fluid regions with no face-connected path to the outlet into solid.

    A fluid pocket cut off from the outlet has no Dirichlet pressure face, so
    its pressure is defined only up to a constant; such pockets are removed
    from the geometry before any run.
    """
    from scipy import ndimage
    fluid = solid == 0
    structure = ndimage.generate_binary_structure(fluid.ndim, 1)
    labels, _ = ndimage.label(fluid, structure=structure)
    out_labels = np.unique(labels[..., -1])
    out_labels = out_labels[out_labels != 0]
    keep = np.isin(labels, out_labels)
    return np.where(keep, 0, 1).astype(np.uint8)


# ----------------------------------------------------------------------------
# 2D air bubble in a straight channel (128x16 over 800x100 um, Ca = 1e-3)
# ----------------------------------------------------------------------------
def channel_bubble_2d(nx: int = 128, ny: int = 16, Lx: float = 800e-6, Ly: float = 100e-6,
                      Ca: float = 1e-3, bubble_len: float = 300e-6,
                      bubble_x: Optional[float] = None, c_cfl: float = 0.29,
                      n_drag: int = 20, n_relax_max: int = 50, n_standard: int = 2000,
                      theta_deg: float = 180.0, **overrides) -> Case:
    """Air bubble (alpha = 1) centred in a water-filled channel.

    The bubble is a stadium: a rectangle of the channel's full width with
    semicircular caps of radius Ly/2, total length `bubble_len`; alpha0 is the
    area fraction of the cell inside the stadium, from 8x8 sub-samples (a
    sharp 0/1 cell-centre test starts the run with unbalanced capillary
    forces strong enough to make the explicit scheme diverge). Water wets the walls (contact angle 0 through
    water), i.e. 180 degrees measured through the air phase alpha = 1.
    Water is injected at the inlet (alpha_inlet = 0).
    """
    mu_w, sigma = 1e-3, 0.07
    hx, hy = Lx / nx, Ly / ny
    U = Ca * sigma / mu_w
    xc = Lx / 2 if bubble_x is None else bubble_x
    r = Ly / 2
    half_straight = bubble_len / 2 - r
    sub = 8
    off = (np.arange(sub) + 0.5) / sub
    alpha0 = np.zeros((ny, nx))
    for ox in off:
        for oy in off:
            x = (np.arange(nx) + ox)[None, :] * hx
            y = (np.arange(ny) + oy)[:, None] * hy
            dx = np.maximum(np.abs(x - xc) - half_straight, 0.0)
            alpha0 += dx * dx + (y - Ly / 2) ** 2 <= r * r
    alpha0 /= sub * sub
    solid = np.zeros((ny, nx), np.uint8)
    p = default_params(dim=2, nx=nx, ny=ny, nz=1, hx=hx, hy=hy, hz=hx,
                       rho1=1.2, rho2=1000.0, mu1=1.8e-5, mu2=1e-3, sigma=sigma,
                       theta_deg=theta_deg, U_inlet=U, alpha_inlet=0.0,
                       conv_mode=CONV_DU_MAX, conv_tol=1e-6)
    p.update(overrides)
    return Case("channel_bubble_2d", p, solid, alpha0,
                dict(c_cfl=c_cfl, n_drag=n_drag, n_relax_max=n_relax_max,
                     n_standard=n_standard, Ca=Ca))


# ----------------------------------------------------------------------------
# Benchmark case 1 of Section 5.1: air bubble in ethanol, 600x100 um channel
# ----------------------------------------------------------------------------
def bubble_film_2d(Ca: float = 1e-2, h: float = 1e-6, Lx: float = 600e-6, W: float = 100e-6,
                   bubble_len: float = 200e-6, bubble_x0: float = 20e-6, c_cfl: float = 0.01,
                   mu_liquid: float = 1.2e-3, rho_liquid: float = 789.0, **overrides) -> Case:
    """The paper's first benchmark (Section 5.1): a non-wetting air bubble
    (rho 1, mu 18 uPa s) in ethanol (rho 789, mu 1.2 mPa s), sigma 20 mN/m, in
    a straight 2D channel 600 um long and 100 um wide; the bubble starts as a
    full-width rectangle 200 um long whose left end is 20 um from the inlet.
    The liquid wets the walls (0 degrees through the liquid, i.e. 180 degrees
    through the air, alpha = 1), and ethanol is injected at U = Ca sigma / mu.
    The drag steps use dt_vd = 0.01 dt_CFL as in the paper. Uniform square
    cells of size h (1 um gives 600x100 cells)."""
    sigma = 0.02
    nx, ny = int(round(Lx / h)), int(round(W / h))
    U = Ca * sigma / mu_liquid
    x = _cell_centres(nx, h)
    frac = np.clip((np.minimum(x + h / 2, bubble_x0 + bubble_len) - np.maximum(x - h / 2, bubble_x0)) / h, 0.0, 1.0)
    alpha0 = np.broadcast_to(frac[None, :], (ny, nx)).copy()
    solid = np.zeros((ny, nx), np.uint8)
    p = default_params(dim=2, nx=nx, ny=ny, nz=1, hx=h, hy=h, hz=h,
                       rho1=1.0, rho2=rho_liquid, mu1=1.8e-5, mu2=mu_liquid, sigma=sigma,
                       theta_deg=180.0, U_inlet=U, alpha_inlet=0.0)
    p.update(overrides)
    return Case("bubble_film_2d", p, solid, alpha0,
                dict(c_cfl=c_cfl, Ca=Ca, W=W, bubble_len=bubble_len, t_end=bubble_len / U))


# ----------------------------------------------------------------------------
# 3D constricted square channel, CO2 slug (256x64x64 over 1600x100x100 um)
# ----------------------------------------------------------------------------
def constricted_channel_3d(nx: int = 256, ny: int = 64, nz: int = 64,
                           Lx: float = 1600e-6, W: float = 100e-6, Ca: float = 1e-4,
                           throat: float = 0.30, wavelength: float = 800e-6,
                           slug_frac: float = 0.40, c_cfl: float = 0.1,
                           theta_deg: float = 150.0, **overrides) -> Case:
    """Square channel whose cross-section narrows sinusoidally at mid-length.

    Half-width w(x) = (W/2) [1 - (1 - throat) (1 + cos(2 pi (x - x_c)/lambda))/2]
    for |x - x_c| < lambda/2, W/2 elsewhere; the square section shrinks
    uniformly in y and z, reaching `throat` of the width at x_c. CO2 (alpha = 1)
    fills x < slug_frac * Lx and is injected at the inlet. Water-wet walls at
    30 degrees through water are 150 degrees through CO2.
    """
    mu_w, sigma = 1e-3, 0.03
    hx, hy, hz = Lx / nx, W / ny, W / nz
    U = Ca * sigma / mu_w
    x = _cell_centres(nx, hx)[None, None, :]
    y = _cell_centres(ny, hy)[None, :, None]
    z = _cell_centres(nz, hz)[:, None, None]
    xc = Lx / 2
    s = np.abs(x - xc)
    bump = np.where(s < wavelength / 2, 0.5 * (1.0 + np.cos(2 * np.pi * (x - xc) / wavelength)), 0.0)
    half = (W / 2) * (1.0 - (1.0 - throat) * bump)
    solid = ((np.abs(y - W / 2) > half) | (np.abs(z - W / 2) > half)).astype(np.uint8)
    solid = np.broadcast_to(solid, (nz, ny, nx)).copy()
    solid = keep_outlet_connected(solid)
    xf = slug_frac * Lx
    frac_x = np.clip((xf - (x - hx / 2)) / hx, 0.0, 1.0)   # area fraction of the cell left of the front
    alpha0 = np.broadcast_to(frac_x, (nz, ny, nx)).copy()
    alpha0[solid == 1] = 0.0
    p = default_params(dim=3, nx=nx, ny=ny, nz=nz, hx=hx, hy=hy, hz=hz,
                       rho1=700.0, rho2=1000.0, mu1=5e-5, mu2=1e-3, sigma=sigma,
                       theta_deg=theta_deg, U_inlet=U, alpha_inlet=1.0,
                       precision=PREC_MIXED)
    p.update(overrides)
    return Case("constricted_channel_3d", p, solid, alpha0,
                dict(c_cfl=c_cfl, Ca=Ca, throat=throat))


# ----------------------------------------------------------------------------
# 2D oil-wet micromodel of random discs (2048x1024 over 4x2 mm)
# ----------------------------------------------------------------------------
def disc_mask(nx: int, ny: int, Lx: float, Ly: float, seed: int = 0,
              r_min: float = 40e-6, r_max: float = 120e-6, porosity: float = 0.5,
              min_gap: float = 15e-6, clear_x: float = 100e-6,
              max_tries: int = 200000) -> np.ndarray:
    """Non-overlapping random discs by seeded rejection sampling.

    A candidate disc (radius uniform in [r_min, r_max], centre uniform) is
    accepted when its gap to every accepted disc and to the y walls is at
    least `min_gap`, and it stays `clear_x` away from inlet and outlet.
    Sampling stops once the disc-area fraction reaches 1 - porosity or after
    `max_tries` candidates. Cells whose centre lies in a disc are solid.
    """
    rng = np.random.default_rng(seed)
    discs = []
    area_target = (1.0 - porosity) * Lx * Ly
    area = 0.0
    for _ in range(max_tries):
        r = rng.uniform(r_min, r_max)
        cx = rng.uniform(clear_x + r, Lx - clear_x - r)
        cy = rng.uniform(r + min_gap, Ly - r - min_gap)
        ok = True
        for (ox, oy, orr) in discs:
            if (cx - ox) ** 2 + (cy - oy) ** 2 < (r + orr + min_gap) ** 2:
                ok = False
                break
        if not ok:
            continue
        discs.append((cx, cy, r))
        area += math.pi * r * r
        if area >= area_target:
            break
    hx, hy = Lx / nx, Ly / ny
    x = _cell_centres(nx, hx)[None, :]
    y = _cell_centres(ny, hy)[:, None]
    solid = np.zeros((ny, nx), np.uint8)
    for (cx, cy, r) in discs:
        i0 = max(int((cx - r) / hx) - 1, 0)
        i1 = min(int((cx + r) / hx) + 2, nx)
        j0 = max(int((cy - r) / hy) - 1, 0)
        j1 = min(int((cy + r) / hy) + 2, ny)
        sub = (x[:, i0:i1] - cx) ** 2 + (y[j0:j1, :] - cy) ** 2 <= r * r
        solid[j0:j1, i0:i1] |= sub.astype(np.uint8)
    return solid


def micromodel_2d(nx: int = 2048, ny: int = 1024, Lx: float = 4e-3, Ly: float = 2e-3,
                  Ca: float = 1e-5, seed: int = 0, c_cfl: float = 0.1,
                  theta_deg: float = 150.0, **overrides) -> Case:
    """Oil-filled disc micromodel; water (alpha = 1, non-wetting) injected."""
    mu_w, sigma = 1e-3, 0.035
    U = Ca * sigma / mu_w
    scale = nx / 2048.0
    solid = disc_mask(nx, ny, Lx, Ly, seed=seed,
                      clear_x=100e-6, min_gap=max(15e-6, 2.5 * Lx / nx))
    solid = keep_outlet_connected(solid)
    alpha0 = np.zeros((ny, nx))
    p = default_params(dim=2, nx=nx, ny=ny, nz=1, hx=Lx / nx, hy=Ly / ny, hz=Lx / nx,
                       rho1=1000.0, rho2=850.0, mu1=1e-3, mu2=5e-3, sigma=sigma,
                       theta_deg=theta_deg, U_inlet=U, alpha_inlet=1.0,
                       precision=PREC_MIXED)
    p.update(overrides)
    return Case("micromodel_2d", p, solid, alpha0, dict(c_cfl=c_cfl, Ca=Ca, seed=seed, scale=scale))


# ----------------------------------------------------------------------------
# Batched sweep: 64 channel-bubble instances of uneven size
# ----------------------------------------------------------------------------
def batched_sweep(n_inst: int = 64, seed: int = 0,
                  grids=((128, 16), (256, 32), (512, 64), (1024, 128))) -> list:
    """Channel-bubble instances with grid, Ca and bubble length drawn per seed.

    Domain 800x100 um for every grid; Ca log-uniform in [1e-6, 1e-3]; bubble
    length uniform in [2, 5] channel widths; fluids as the 128x16 case.
    """
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(n_inst):
        nx, ny = grids[int(rng.integers(len(grids)))]
        Ca = 10.0 ** rng.uniform(-6, -3)
        L = rng.uniform(2.0, 5.0) * 100e-6
        L = min(L, 700e-6)
        cases.append(channel_bubble_2d(nx=nx, ny=ny, Ca=Ca, bubble_len=L))
    return cases


# ----------------------------------------------------------------------------
# Small cases for pins and parity
# ----------------------------------------------------------------------------
def static_drop(n: int = 32, R_cells: float = 8.0, dim: int = 2, h: float = 1e-6,
                sigma: float = 0.03, rho_in: float = 1000.0, rho_out: float = 1000.0,
                mu_in: float = 1e-3, mu_out: float = 1e-3, theta_deg: float = 90.0,
                profile: str = "fraction", width_cells: float = 1.0, **overrides) -> Case:
    """Disc (2D) or sphere (3D) of alpha = 1, radius R_cells*h, box centre.

    The domain is an n^dim box of walls with the usual inlet (no injection)
    and outlet. profile="fraction": alpha0 is a 4^dim sub-sampled volume
    fraction; profile="tanh": alpha0 = (1 - tanh((r - R)/(width_cells h)))/2,
    a smooth field whose discrete curvature converges under refinement.
    """
    nz = n if dim == 3 else 1
    shape = (nz, n, n) if dim == 3 else (n, n)
    sub = 4
    off = (np.arange(sub) + 0.5) / sub
    c = n * h / 2
    R = R_cells * h
    a = np.zeros(shape)
    idx = np.indices(shape)
    for ox in off:
        for oy in off:
            for oz in (off if dim == 3 else [0.5]):
                x = (idx[-1] + ox) * h
                y = (idx[-2] + oy) * h
                r2 = (x - c) ** 2 + (y - c) ** 2
                if dim == 3:
                    zz = (idx[0] + oz) * h
                    r2 = r2 + (zz - c) ** 2
                a += (r2 <= R * R)
    a /= sub ** dim
    if profile == "tanh":
        r2 = sum(((idx[-1 - d] + 0.5) * h - c) ** 2 for d in range(dim))
        a = 0.5 * (1.0 - np.tanh((np.sqrt(r2) - R) / (width_cells * h)))
    solid = np.zeros(shape, np.uint8)
    p = default_params(dim=dim, nx=n, ny=n, nz=nz, hx=h, hy=h, hz=h,
                       rho1=rho_in, rho2=rho_out, mu1=mu_in, mu2=mu_out, sigma=sigma,
                       theta_deg=theta_deg, U_inlet=0.0, alpha_inlet=0.0)
    p.update(overrides)
    return Case("static_drop", p, solid, a, dict(R=R))


def random_small_case(seed: int, nx: int, ny: int, nz: int = 1, dim: int = 2,
                      solid_frac: float = 0.15, sigma: float = 0.02, U: float = 0.01,
                      **overrides) -> Case:
    """Ragged small grid with random solid blocks and a smooth random blob of alpha.

    Used for element-by-element parity at sizes the oracle finishes in
    seconds. Fluid pockets cut off from the outlet are made solid.
    """
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx) if dim == 3 else (ny, nx)
    solid = (rng.random(shape) < solid_frac).astype(np.uint8)
    solid[..., 0] = 0
    solid[..., -1] = 0
    solid = keep_outlet_connected(solid)
    idx = np.indices(shape).astype(np.float64)
    cx, cy = nx * rng.uniform(0.35, 0.65), ny * rng.uniform(0.35, 0.65)
    r2 = (idx[-1] + 0.5 - cx) ** 2 + (idx[-2] + 0.5 - cy) ** 2
    if dim == 3:
        cz = nz * rng.uniform(0.35, 0.65)
        r2 = r2 + (idx[0] + 0.5 - cz) ** 2
    R = 0.3 * min(nx, ny, nz if dim == 3 else ny)
    alpha0 = np.clip(0.5 - (np.sqrt(r2) - R) / 2.0, 0.0, 1.0)
    alpha0[solid == 1] = 0.0
    h = 2e-6
    p = default_params(dim=dim, nx=nx, ny=ny, nz=nz, hx=h, hy=h * 0.75, hz=h,
                       rho1=1.2, rho2=1000.0, mu1=1.8e-5, mu2=1e-3, sigma=sigma,
                       theta_deg=135.0, U_inlet=U, alpha_inlet=0.0)
    p.update(overrides)
    return Case("random_small", p, solid, alpha0, dict(seed=seed))
