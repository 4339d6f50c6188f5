"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

FP64 path: every state field (alpha, u, p, fluxes) within 1e-10 relative
(max-norm) of the oracle. The interface normal n = g/(|g| + delta_N) and the
curvature kappa = -div n amplify rounding-level differences of alpha by up to
1/(h delta_N) = 1e8 where alpha is uniform (|g| << delta_N), so they are
compared where they are well conditioned and act: kappa on the interface band
0.01 < alpha < 0.99 (the CSF force sigma kappa grad alpha vanishes elsewhere).
Mixed path: alpha within 1e-5 absolute, bubble velocity within 0.5 %.
"""
import numpy as np
import pytest

import oracle
from paper_2105_10576_gb300 import inputs
from paper_2105_10576_gb300 import oscar as ox

pytestmark = pytest.mark.gpu

CELL_FIELDS = [("alpha", ox.FIELD_ALPHA, oracle.ALPHA), ("p", ox.FIELD_P, oracle.P),
               ("ux", ox.FIELD_U, oracle.UX), ("uy", ox.FIELD_U + 1, oracle.UY),
               ("uvdx", ox.FIELD_U_VD, oracle.UVDX), ("uvdy", ox.FIELD_U_VD + 1, oracle.UVDY),
               ("ucrx", ox.FIELD_U_CR, oracle.UCRX), ("ucry", ox.FIELD_U_CR + 1, oracle.UCRY),
               ("p_vd", ox.FIELD_P_VD, oracle.P_VD), ("p_cr", ox.FIELD_P_CR, oracle.P_CR),
               ("kappa", ox.FIELD_KAPPA, oracle.KAPPA)]
FACE_FIELDS = [("phi_vd_x", ox.FIELD_PHI_VD, oracle.PHI_VD), ("phi_vd_y", ox.FIELD_PHI_VD + 1, oracle.PHI_VD + 1),
               ("phi_cr_x", ox.FIELD_PHI_CR, oracle.PHI_CR), ("phi_cr_y", ox.FIELD_PHI_CR + 1, oracle.PHI_CR + 1)]
BAND = (0.01, 0.99)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def fields_for(dim):
    cf = list(CELL_FIELDS)
    ff = list(FACE_FIELDS)
    if dim == 3:
        cf += [("uz", ox.FIELD_U + 2, oracle.UZ), ("uvdz", ox.FIELD_U_VD + 2, oracle.UVDZ),
               ("ucrz", ox.FIELD_U_CR + 2, oracle.UCRZ)]
        ff += [("phi_vd_z", ox.FIELD_PHI_VD + 2, oracle.PHI_VD + 2),
               ("phi_cr_z", ox.FIELD_PHI_CR + 2, oracle.PHI_CR + 2)]
    return cf + ff


def rel_err(x, y):
    m = np.abs(y).max()
    d = np.abs(x - y).max()
    if m == 0.0:
        return d
    return d / m


def compare(g, o, dim, tol, skip=()):
    worst = {}
    a_or = o.field(oracle.ALPHA)
    band = (a_or > BAND[0]) & (a_or < BAND[1])
    for name, wg, wo in fields_for(dim):
        if name in skip:
            continue
        x, y = g.field(wg), o.field(wo)
        if name == "kappa":
            if not band.any():
                continue
            x, y = x[band], y[band]
        e = rel_err(x, y)
        worst[name] = e
    bad = {k: v for k, v in worst.items() if not v <= tol}
    assert not bad, f"fields over {tol}: {bad}"
    return worst


def run_oscar_pair(case, n_drag, n_sub, dt_vd, dt_cr, precision=inputs.PREC_FP64, N=None):
    p = dict(case.params, precision=precision)
    g = ox.Oscar(p, case.solid, case.alpha0)
    o = oracle.OracleState(p, case.solid, case.alpha0)
    kg, ko = [], []
    for _ in range(n_drag):
        g.drag_step(dt_vd)
        o.drag_step(dt_vd)
        _, k1, _ = g.relax(dt_cr, N or n_sub)
        _, k2, _ = o.relax(dt_cr, N or n_sub)
        kg.append(k1)
        ko.append(k2)
    return g, o, kg, ko


SMALL = [("2d_ragged", lambda: inputs.random_small_case(1, 37, 13)),
         ("2d_ragged_b", lambda: inputs.random_small_case(2, 23, 29, solid_frac=0.25)),
         ("3d_ragged", lambda: inputs.random_small_case(3, 19, 11, nz=9, dim=3))]


@pytest.mark.parametrize("name,make", SMALL)
def test_fp64_oscar_small_matches_oracle(name, make):
    c = make()
    c.params.update(conv_mode=inputs.CONV_PRES_RESID, conv_tol=0.0)   # forced k_f = N
    # the gaps between random solids carry up to ~8 U: c = 0.02 keeps the drag Courant number < 1
    dt_cfl, dt_b, dt_vd, N = oracle.timesteps(c.params, 0.02)
    g, o, kg, ko = run_oscar_pair(c, 2, 4, dt_vd, 0.9 * dt_b)
    assert kg == ko == [4, 4]
    compare(g, o, c.params["dim"], 1e-10)
    sg, so = g.stats(), o.stats()
    assert sg["phase_volume"] == pytest.approx(so["phase_volume"], rel=1e-12)


@pytest.mark.parametrize("name,make", SMALL)
def test_fp64_standard_small_matches_oracle(name, make):
    c = make()
    dt_cfl, dt_b, dt_vd, N = oracle.timesteps(c.params, 0.02)
    g = ox.Oscar(c.params, c.solid, c.alpha0)
    o = oracle.OracleState(c.params, c.solid, c.alpha0)
    for _ in range(5):
        g.standard_step(0.9 * dt_b)
        o.standard_step(0.9 * dt_b)
    compare(g, o, c.params["dim"], 1e-10, skip=("ucrx", "ucry", "ucrz", "phi_cr_x", "phi_cr_y", "phi_cr_z"))


def test_fp64_early_exit_residual_matches_oracle():
    """E_k (Section 3.2) per sub-step agrees, so both sides stop at the same k_f."""
    c = inputs.random_small_case(4, 31, 17, sigma=0.0005)
    c.params.update(conv_mode=inputs.CONV_PRES_RESID, conv_tol=5e-3)
    dt_cfl, dt_b, dt_vd, N = oracle.timesteps(c.params, 0.02)
    g = ox.Oscar(c.params, c.solid, c.alpha0)
    o = oracle.OracleState(c.params, c.solid, c.alpha0)
    g.drag_step(dt_vd)
    o.drag_step(dt_vd)
    _, kg, Eg = g.relax(dt_vd / 40, 40)
    _, ko, hist = o.relax(dt_vd / 40, 40)
    assert kg == ko
    assert Eg == pytest.approx(hist[-1], rel=1e-6)
    compare(g, o, 2, 1e-10)


def _spread_bounds(which):
    """Per-field parity bounds of the full bubble run: 1e-10 relative, or four
    times the oracle's own spread under one-ulp perturbations of alpha0 where
    that spread is larger (tests/golden/bubble_rounding_spread.json, written by
    tests/golden/make_bubble_rounding_spread.py from oracle runs only)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bubble_rounding_spread.json")
    spread = json.load(open(path))[which]
    return {k: max(1e-10, 4.0 * v) for k, v in spread.items()}


def _compare_bounded(g, o, bounds, skip=()):
    worst = {}
    for name, wg, wo in fields_for(2):
        if name in skip:
            continue
        x, y = g.field(wg), o.field(wo)
        if name == "kappa":
            a_or = o.field(oracle.ALPHA)
            band = (a_or > BAND[0]) & (a_or < BAND[1])
            x, y = x[band], y[band]
        worst[name] = (rel_err(x, y), bounds.get(name, 1e-10))
    bad = {k: v for k, v in worst.items() if not v[0] <= v[1]}
    assert not bad, f"fields over their bound (error, bound): {bad}"
    return worst


def test_fp64_bubble_channel_full_run_matches_oracle():
    """The 128x16 bubble channel: 20 drag steps, each followed by up to 50
    relaxation sub-steps (tolerance 1e-6 on max |du_cr|/U), and 2000 standard
    steps at the relaxation time-step, against the oracle with exact (banded
    Cholesky) pressure solves. alpha, p, p_vd, p_cr and kappa stay within
    1e-10 relative. The velocity and flux fields are held to four times the
    spread of the oracle's own runs when alpha0 is perturbed by one ulp (at
    most 7e-10 after the OSCAR run, 3.3e-9 after the standard run): at the
    1000:1.2 density ratio the parasitic-current dynamics amplify rounding
    differences over thousands of pressure solves, so no differently rounded
    implementation can agree more closely; where that spread is below 2.5e-11
    the bound stays 1e-10."""
    c = inputs.channel_bubble_2d(cg_rtol=1e-15, cg_maxit=400)   # oracle: exact banded solves
    dt_cfl, dt_b, dt_vd, N = oracle.timesteps(c.params, c.meta["c_cfl"], c.solid)
    assert N == 50
    g, o, kg, ko = run_oscar_pair(c, c.meta["n_drag"], N, dt_vd, dt_vd / N)
    assert kg == ko
    worst = _compare_bounded(g, o, _spread_bounds("oscar"))
    print("oscar (error, bound)", {k: f"{v[0]:.1e}/{v[1]:.1e}" for k, v in worst.items()})
    gs = ox.Oscar(c.params, c.solid, c.alpha0)
    os_ = oracle.OracleState(c.params, c.solid, c.alpha0)
    for _ in range(c.meta["n_standard"]):
        gs.standard_step(dt_vd / N)
        os_.standard_step(dt_vd / N)
    crf = ("ucrx", "ucry", "phi_cr_x", "phi_cr_y")
    worst = _compare_bounded(gs, os_, _spread_bounds("standard"), skip=crf)
    print("standard (error, bound)", {k: f"{v[0]:.1e}/{v[1]:.1e}" for k, v in worst.items()})


def _bubble_velocity(st, is_oracle):
    a = st.field(oracle.ALPHA if is_oracle else ox.FIELD_ALPHA)
    u = st.field(oracle.UX if is_oracle else ox.FIELD_U)
    return (a * u).sum() / a.sum()


@pytest.mark.parametrize("make", [lambda: inputs.channel_bubble_2d(),
                                  lambda: inputs.random_small_case(5, 20, 12, nz=10, dim=3)])
def test_mixed_precision_within_tolerance(make):
    c = make()
    c.params.update(conv_mode=inputs.CONV_PRES_RESID, conv_tol=0.0, cg_rtol=1e-8)   # the bench's tolerance
    dt_cfl, dt_b, dt_vd, N = oracle.timesteps(c.params, c.meta.get("c_cfl", 0.02))
    g, o, kg, ko = run_oscar_pair(c, 3, min(N, 10), dt_vd, dt_vd / N, precision=inputs.PREC_MIXED, N=min(N, 10))
    da = np.abs(g.field(ox.FIELD_ALPHA) - o.field(oracle.ALPHA)).max()
    assert da <= 1e-5
    vg, vo = _bubble_velocity(g, False), _bubble_velocity(o, True)
    assert vg == pytest.approx(vo, rel=5e-3)


def _batch_setup(case, n_sub):
    p = dict(case.params, precision=inputs.PREC_MIXED, cg_rtol=1e-8)
    dt_cfl, dt_b, dt_vd, N = ox.oscar_timesteps(p, case.meta["c_cfl"], case.solid)
    dt_cr = 0.99 * dt_b
    return p, n_sub * dt_cr, dt_cr


def test_batched_instances_match_alone():
    """Instances stepped concurrently (asynchronous launches on their own
    streams, collected with oscar_wait) give exactly the fields they give when
    stepped alone: every kernel reduces in a fixed order, and an instance's
    launches do not depend on the others."""
    from paper_2105_10576_gb300 import batch
    cases = inputs.batched_sweep(4, seed=3)
    n_sub = 5
    setups = [_batch_setup(c, n_sub) for c in cases]
    sims = [ox.Oscar(p, c.solid, c.alpha0) for c, (p, _, _) in zip(cases, setups)]
    b = batch.Batch(sims)
    for _ in range(2):
        kfs = b.step([s[1] for s in setups], [s[2] for s in setups], [n_sub] * len(sims))
    mixed = [(sm.field(ox.FIELD_ALPHA), sm.field(ox.FIELD_P), sm.field(ox.FIELD_U)) for sm in sims]
    with pytest.raises(ox.OscarError):     # one pending step per handle: only oscar_wait is accepted
        sims[0].drag_step_async(setups[0][1])
        sims[0].stats()
    sims[0].wait(strict=False)
    b.close()
    for q, (c, (p, dtv, dtc)) in enumerate(zip(cases, setups)):
        g = ox.Oscar(p, c.solid, c.alpha0)
        for _ in range(2):
            g.drag_step(dtv, strict=False)
            _, kf, _ = g.relax(dtc, n_sub, strict=False)
        assert kf == kfs[q]
        alone = (g.field(ox.FIELD_ALPHA), g.field(ox.FIELD_P), g.field(ox.FIELD_U))
        for x, y in zip(mixed[q], alone):
            assert np.array_equal(x, y)
        g.close()


def test_serving_results_match_alone():
    """Requests admitted while others run (all arrive at once; the memory
    budget holds only some of them, so the rest are admitted as the first ones
    finish) finish with exactly the fields they give when run alone, and the
    admission never exceeds the budget."""
    from paper_2105_10576_gb300 import serve
    cases = inputs.batched_sweep(5, seed=4, grids=((128, 16), (256, 32)))
    reqs = []
    for q, c in enumerate(cases):
        p, dtv, dtc = _batch_setup(c, 4)
        reqs.append(serve.Request(q, 0.0, p, c.solid, c.alpha0, dtv, dtc, 4, 2))
    fps = [ox.oscar_footprint(r.params) for r in reqs]
    g = ox.Oscar(reqs[0].params, reqs[0].solid, reqs[0].alpha0)
    assert fps[0] == g.stats()["device_bytes"]     # the footprint is what create allocates
    g.close()
    budget = max(fps) + min(fps)                      # not all of them fit at once
    assert sum(fps) > budget
    srv = serve.Server(budget)
    recs = srv.run(reqs, keep_alpha=True)
    assert srv.max_concurrent >= 2 and srv.max_used <= budget
    assert [r.rid for r in recs] == list(range(len(reqs)))
    for r, rec in zip(reqs, recs):
        alone = serve.run_alone(r)
        assert rec.status in (0, -3) and rec.k_f == alone.k_f
        assert rec.cell_updates == alone.cell_updates
        assert np.array_equal(rec.alpha, alone.alpha)
        assert rec.done >= rec.admitted >= rec.arrival


def test_instances_of_different_sizes_do_not_interfere():
    """Creating a small instance while a larger one is in use must not change
    the larger one's results (kernel attributes are process-wide)."""
    big = inputs.random_small_case(9, 64, 32, nz=32, dim=3)
    small = inputs.random_small_case(10, 12, 8)
    pb = dict(big.params, precision=inputs.PREC_MIXED, cg_rtol=1e-8)
    ps = dict(small.params, precision=inputs.PREC_MIXED, cg_rtol=1e-8)
    dt_b = ox.oscar_timesteps(pb, 0.02)[1]

    def steps(g):
        g.drag_step(3 * 0.99 * dt_b, strict=False)
        rc, kf, _ = g.relax(0.99 * dt_b, 3, strict=False)
        return rc, kf

    ref = ox.Oscar(pb, big.solid, big.alpha0)
    r_ref = steps(ref)
    a_ref = ref.field(ox.FIELD_P)
    ref.close()
    g = ox.Oscar(pb, big.solid, big.alpha0)
    g.drag_step(3 * 0.99 * dt_b, strict=False)      # graphs of the big instance exist
    h = ox.Oscar(ps, small.solid, small.alpha0)     # then a small one is created
    h.drag_step(3 * 0.99 * dt_b, strict=False)
    rc, kf, _ = g.relax(0.99 * dt_b, 3, strict=False)
    assert (rc, kf) == r_ref
    assert np.array_equal(g.field(ox.FIELD_P), a_ref)
    g.close()
    h.close()


def test_edge_cases():
    # all-solid grid is rejected; a single fluid column works
    c = inputs.random_small_case(6, 5, 4)
    with pytest.raises(ox.OscarError):
        ox.Oscar(c.params, np.ones_like(c.solid), c.alpha0)
    p = inputs.default_params(dim=2, nx=1, ny=1, hx=1e-6, hy=1e-6, U_inlet=1e-3, rho1=1.0, rho2=1.0, sigma=0.01)
    s = np.zeros((1, 1), np.uint8)
    a = np.full((1, 1), 0.3)
    g = ox.Oscar(p, s, a)
    o = oracle.OracleState(p, s, a)
    for _ in range(3):
        g.drag_step(1e-4)
        o.drag_step(1e-4)
        g.relax(1e-6, 2)
        o.relax(1e-6, 2)
    compare(g, o, 2, 1e-10)


@pytest.mark.parametrize("which", ["constriction_3d", "micromodel_2d"])
def test_full_size_invariants(which):
    """At the bench's full sizes (mixed precision): alpha stays in [0, 1], face
    fluxes are divergence-free to the solver tolerance, the phase volume
    changes only by what crosses inlet and outlet, and nothing is non-finite."""
    c = (inputs.constricted_channel_3d(cg_rtol=1e-8) if which == "constriction_3d"
         else inputs.micromodel_2d(cg_rtol=1e-8))
    p = c.params
    dt_cfl, dt_b, dt_vd, N = ox.oscar_timesteps(p, c.meta["c_cfl"], c.solid)
    g = ox.Oscar(p, c.solid, c.alpha0)
    v0 = g.stats()["phase_volume"]
    g.drag_step(dt_vd)
    g.relax(dt_vd / N, 3)
    a = g.field(ox.FIELD_ALPHA)
    assert np.isfinite(a).all()
    assert a.min() >= -1e-5 and a.max() <= 1 + 1e-5
    for base in (ox.FIELD_PHI_VD, ox.FIELD_PHI_CR):
        phi = [g.field(base + d) for d in range(p["dim"])]
        if p["dim"] == 2:
            div = (phi[0][:, 1:] - phi[0][:, :-1]) + (phi[1][1:, :] - phi[1][:-1, :])
        else:
            div = ((phi[0][:, :, 1:] - phi[0][:, :, :-1]) + (phi[1][:, 1:, :] - phi[1][:, :-1, :])
                   + (phi[2][1:, :, :] - phi[2][:-1, :, :]))
        scale = max(np.abs(x).max() for x in phi)
        assert np.abs(div[c.solid == 0]).max() <= 1e-5 * scale
    # volume balance: the drag step moves alpha_inlet * inflow * dt in
    phix = g.field(ox.FIELD_PHI_VD)
    v1 = g.stats()["phase_volume"]
    assert abs(v1 - v0) <= 2.0 * abs(phix[..., 0]).sum() * dt_vd + 1e-6 * v0


def test_bench_workload_long_run_stays_bounded():
    """The bench workload (3D constriction 256x64x64, mixed precision, the
    time steps of the bench) for 50 OSCAR steps, more than the bench runs
    (warm-up, timed and end-to-end steps): every drag step and relaxation
    returns 0 (solves converged, nothing non-finite), alpha stays in [0, 1],
    the drag Courant number stays below 1 and the phase volume grows by what
    the inlet injects (nothing of the injected phase reaches the outlet)."""
    c = inputs.constricted_channel_3d(cg_rtol=1e-8)
    p = c.params
    dt_cfl, dt_b, dt_vd, N = ox.oscar_timesteps(p, c.meta["c_cfl"], c.solid)
    g = ox.Oscar(p, c.solid, c.alpha0)
    v0 = g.stats()["phase_volume"]
    S = [p["hy"] * p["hz"], p["hx"] * p["hz"], p["hx"] * p["hy"]]
    h = [p["hx"], p["hy"], p["hz"]]
    inflow = 0.0
    for step in range(50):
        # the drag step transports alpha with the drag flux of the previous step (Eq. VOFd)
        inflow += g.field(ox.FIELD_PHI_VD)[..., 0].sum() * dt_vd
        assert g.drag_step(dt_vd) == 0
        rc, kf, _ = g.relax(dt_vd / N, N)
        assert rc == 0 and 1 <= kf <= N
        if step % 10 == 9:
            a = g.field(ox.FIELD_ALPHA)
            assert np.isfinite(a).all()
            assert a.min() >= -1e-5 and a.max() <= 1 + 1e-5
            co = max(np.abs(g.field(ox.FIELD_PHI_VD + d)).max() / S[d] * dt_vd / h[d] for d in range(3))
            assert co < 1.0, co
    v1 = g.stats()["phase_volume"]
    assert v1 - v0 == pytest.approx(p["alpha_inlet"] * inflow, rel=2e-3)
    g.close()


def _constriction_fields(c, prec, alpha0, n_steps):
    p = dict(c.params, precision=prec)
    dt_cfl, dt_b, dt_vd, N = ox.oscar_timesteps(p, c.meta["c_cfl"], c.solid)
    g = ox.Oscar(p, c.solid, alpha0)
    for _ in range(n_steps):
        assert g.drag_step(dt_vd) == 0
        assert g.relax(dt_vd / N, N)[0] == 0
    f = {"a": g.field(ox.FIELD_ALPHA), "p": g.field(ox.FIELD_P), "u": g.field(ox.FIELD_U)}
    g.close()
    return f


def test_mixed_precision_against_fp64_on_the_constriction():
    """Mixed precision against the FP64 GPU path on a reduced 3D constriction
    (128x32x32, the bench geometry's generator, 10 drag steps of 110 relaxation
    sub-steps). The integral results the method is used for agree within 0.5 %:
    the bubble velocity (alpha-weighted mean u_x) and the capillary pressure
    (mean p where alpha > 0.99 minus where alpha < 0.01); alpha agrees within
    1e-5 in L1 over the injected volume. Pointwise, alpha is held to four times
    the spread that a one-ulp FP32 perturbation of alpha0 produces in the mixed
    run itself (two seeds; at least 1e-5): the capillary dynamics amplify
    rounding differences (at 256x64x64 such a perturbation moves alpha by 0.1
    after 10 steps), so no FP32 path can agree pointwise more closely."""
    c = inputs.constricted_channel_3d(nx=128, ny=32, nz=32, cg_rtol=1e-8)
    fl = c.solid == 0
    n = 10
    ref = _constriction_fields(c, inputs.PREC_FP64, c.alpha0, n)
    mix = _constriction_fields(c, inputs.PREC_MIXED, c.alpha0, n)
    spread = 0.0
    for seed in (0, 1):
        s = np.random.default_rng(seed).integers(-1, 2, c.alpha0.shape)
        pert = _constriction_fields(c, inputs.PREC_MIXED, c.alpha0 * (1 + s * 2.0 ** -23), n)
        spread = max(spread, float(np.abs(pert["a"] - mix["a"])[fl].max()))

    def vb(f):
        return (f["a"][fl] * f["u"][fl]).sum() / f["a"][fl].sum()

    def pc(f):
        a, p = f["a"], f["p"]
        return p[(a > 0.99) & fl].mean() - p[(a < 0.01) & fl].mean()

    assert vb(mix) == pytest.approx(vb(ref), rel=5e-3)
    assert pc(mix) == pytest.approx(pc(ref), rel=5e-3)
    da = np.abs(mix["a"] - ref["a"])[fl]
    assert da.sum() / ref["a"][fl].sum() <= 1e-5
    assert da.max() <= max(1e-5, 4.0 * spread), (da.max(), spread)


def _benchmark1(Ca, prec):
    """Benchmark 1 of Section 5.1 at 1 um (600x100 cells): relax the initial
    rectangle towards capillary equilibrium, then inject ethanol up to
    t* = U t / L = 1 with dt_vd = 0.01 dt_CFL, dt_cr = dt_vd / N."""
    c = inputs.bubble_film_2d(Ca=Ca, cg_rtol=1e-10, precision=prec)
    p = c.params
    dt_cfl, dt_b, dt_vd, N = ox.oscar_timesteps(p, c.meta["c_cfl"], c.solid)
    g = ox.Oscar(p, c.solid, c.alpha0)
    assert g.relax(0.99 * dt_b, 3000)[0] == 0
    for _ in range(int(round(c.meta["t_end"] / dt_vd))):
        assert g.drag_step(dt_vd) == 0
        assert g.relax(dt_vd / N, N)[0] == 0
    a, ux = g.field(ox.FIELD_ALPHA), g.field(ox.FIELD_U)
    g.close()
    W, h = c.meta["W"], p["hx"]
    b = a.sum(axis=0) * h                 # bubble width per column
    cols = np.where(b > 0.5 * W)[0]
    L = cols[-1] - cols[0] + 1
    mid = np.arange(cols[0] + L // 3, cols[-1] - L // 3 + 1)
    film = (W - b[mid].mean()) / 2        # flat part of the film, both walls averaged
    return film, float((a * ux).sum() / a.sum()) / p["U_inlet"], W


def _aq(Ca, W):
    x = Ca ** (2.0 / 3.0)
    return (W / 2) * 1.34 * x / (1 + 3.35 * x)


def test_film_thickness_benchmark1():
    """The paper's benchmark 1 (Section 5.1; film-thickness figure): the liquid
    film left by an air bubble driven through a 100 um channel, against the
    Aussillous-Quere correlation h = r 1.34 Ca^(2/3) / (1 + 3.35 Ca^(2/3)),
    r = W/2 (2.69 um at Ca = 1e-2; the paper obtains 2.61 um with OSCAR).
    Checked: the film at Ca = 1e-2 within 25 % of the correlation (measured
    -20 % with two smoothing passes; the film is 2.7 cells thick and its value
    moves between 5.1 and 2.2 um with the number of smoothing passes, a
    quantity the paper does not state); the growth of the film from
    Ca = 1e-2 to 1e-1 within 20 % of the correlation's ratio (3.1); the bubble
    velocity equal to the mass-conservation value U W / (W - 2 h) within 2 %;
    and the mixed path within 0.5 % of the FP64 path in film thickness and
    bubble velocity at Ca = 1e-2."""
    h64, v64, W = _benchmark1(1e-2, inputs.PREC_FP64)
    h32, v32, _ = _benchmark1(1e-2, inputs.PREC_MIXED)
    h1, v1, _ = _benchmark1(1e-1, inputs.PREC_MIXED)
    print(f"film Ca=1e-2: FP64 {h64 * 1e6:.3f} um, mixed {h32 * 1e6:.3f} um, AQ {_aq(1e-2, W) * 1e6:.3f} um; "
          f"Ca=1e-1: {h1 * 1e6:.3f} um, AQ {_aq(1e-1, W) * 1e6:.3f} um")
    assert h64 == pytest.approx(_aq(1e-2, W), rel=0.25)
    assert h1 / h64 == pytest.approx(_aq(1e-1, W) / _aq(1e-2, W), rel=0.20)
    assert v64 == pytest.approx(W / (W - 2 * h64), rel=0.02)
    assert v1 == pytest.approx(W / (W - 2 * h1), rel=0.02)
    assert h32 == pytest.approx(h64, rel=5e-3)
    assert v32 == pytest.approx(v64, rel=5e-3)


def test_schedule_changes_speed_not_the_solution():
    """The solver schedule (sweeps per level group, coarse CTA levels, refresh
    of the coarsest inverse, block shape) changes how the pressure solves
    converge, not what they converge to: a 3D case stepped with two different
    schedules agrees within what the solver tolerance allows, a schedule out of
    range is refused and leaves the instance's schedule unchanged, and the
    autotuner returns a schedule from its search space."""
    from paper_2105_10576_gb300 import autotune
    c = inputs.random_small_case(11, 48, 24, nz=20, dim=3)
    c.params.update(conv_mode=inputs.CONV_PRES_RESID, conv_tol=0.0)
    p = dict(c.params, precision=inputs.PREC_FP64, cg_rtol=1e-13)
    dt_cfl, dt_b, dt_vd, N = ox.oscar_timesteps(p, 0.02)
    out = []
    for sched in (dict(autotune.DEFAULT), dict(mg_nu=1, mg_nu_mid=3, mg_nu_cta=1, cta_cells=256,
                                                coarse_refresh=1, block_x=32)):
        g = ox.Oscar(p, c.solid, c.alpha0)
        g.set_schedule(sched)
        sched = dict(autotune.DEFAULT, **sched)
        assert g.schedule() == sched
        g.drag_step(dt_vd)
        g.relax(dt_vd / N, 3)
        out.append((g.field(ox.FIELD_ALPHA), g.field(ox.FIELD_P), g.field(ox.FIELD_U)))
        with pytest.raises(ox.OscarError):
            g.set_schedule(dict(mg_nu=9))
        assert g.schedule() == sched
        g.close()
    for x, y in zip(out[0], out[1]):
        assert rel_err(x, y) <= 1e-9
    best = autotune.tune(dict(p, precision=inputs.PREC_MIXED, cg_rtol=1e-8), c.solid, c.alpha0, dt_vd, dt_vd / N,
                         n_sub=3, rounds=1, use_cache=False)
    for name, values in autotune.SPACE:
        assert best[name] in values


def test_coarse_cta_with_global_level_is_the_same_vcycle():
    """The level above the coarse CTA's levels worked by the CTA itself (x and
    b in shared memory, coefficients from global memory) performs the same
    operations as the per-level kernels: the fields after a drag step and
    relaxation sub-steps are bitwise equal with and without it (mixed path,
    3D grid; with the CTA holding the levels of at most 256 cells, the
    360-cell level above them qualifies)."""
    c = inputs.random_small_case(12, 48, 24, nz=20, dim=3)
    c.params.update(conv_mode=inputs.CONV_PRES_RESID, conv_tol=0.0)
    p = dict(c.params, precision=inputs.PREC_MIXED, cg_rtol=1e-8)
    dt_cfl, dt_b, dt_vd, N = ox.oscar_timesteps(p, 0.02)
    out = []
    for flag in (1, 0):
        g = ox.Oscar(p, c.solid, c.alpha0)
        g.set_schedule(dict(cta_global=flag, cta_cells=256))
        st = g.stats()
        assert (st["mg_cta_global_level"] == st["mg_first_cta_level"] - 1) if flag else st["mg_cta_global_level"] == -1
        g.drag_step(dt_vd)
        g.relax(dt_vd / N, 3)
        out.append([g.field(w) for w in (ox.FIELD_ALPHA, ox.FIELD_P, ox.FIELD_U, ox.FIELD_U + 2)])
        g.close()
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)


def test_profile_repeat_keeps_the_fields():
    """The in-graph timing mode (every plain finest-level half sweep issued
    twice) leaves the fields bitwise equal to normal steps, with the same PCG
    iterations and more kernel launches (mixed path, 3D)."""
    c = inputs.random_small_case(17, 40, 20, nz=16, dim=3)
    p = dict(c.params, precision=inputs.PREC_MIXED, cg_rtol=1e-8)
    dt_cfl, dt_b, dt_vd, N = ox.oscar_timesteps(p, 0.02)
    out, st = [], []
    for rep in (False, True):
        g = ox.Oscar(p, c.solid, c.alpha0)
        g.profile_repeat(rep)
        g.drag_step(dt_vd)
        g.relax(dt_vd / N, 3)
        out.append([g.field(w) for w in (ox.FIELD_ALPHA, ox.FIELD_P, ox.FIELD_U)])
        st.append(g.stats())
        g.close()
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)
    assert st[0]["cg_iters_total"] == st[1]["cg_iters_total"]
    assert st[1]["kernel_launches"] > st[0]["kernel_launches"]


def test_energy_exit_test_matches_oracle():
    """The energy exit test (relative change per sub-step of sigma A + kinetic
    energy of u_cr, the Section 6 variant): the GPU FP64 path and the oracle
    give the same test values and stop at the same k_f (a tolerance the first
    sub-step passes, and one no sub-step passes), and the fields agree to
    1e-10."""
    for tol, k_expect in ((1e-4, 1), (5e-5, 40)):
        c = inputs.random_small_case(13, 31, 17, sigma=0.002)
        c.params.update(conv_mode=inputs.CONV_AREA, conv_tol=tol)
        dt_cfl, dt_b, dt_vd, N = oracle.timesteps(c.params, 0.02)
        g = ox.Oscar(c.params, c.solid, c.alpha0)
        o = oracle.OracleState(c.params, c.solid, c.alpha0)
        g.drag_step(dt_vd)
        o.drag_step(dt_vd)
        _, kg, tg = g.relax(dt_vd / 40, 40)
        _, ko, hist = o.relax(dt_vd / 40, 40)
        assert kg == ko == k_expect
        assert tg == pytest.approx(hist[-1], rel=1e-6)
        compare(g, o, 2, 1e-10)
