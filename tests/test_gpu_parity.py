"""GPU parity: the sm_103a path through the C ABI against the FP64 CPU oracle on the
same seeded inputs.

Tolerances (the workload statement's): FP64 path relative L2 <= 1e-10 on
velocity after 100 steps; mixed-precision path <= 1e-4.  Costs and gradients of the
FP64 path are compared to the oracle's at the precision the two solvers converge to.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
import paper_2605_23812_gb300 as pkg
from paper_2605_23812_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def tight(nx, ny, **kw):
    # 1e-12 divergence: 100x below the 1e-10 target and above the rounding floor of the
    # singular Neumann solve (a constant residual component of ~1e-16 |b| per cell)
    base = dict(div_tol=1e-12, max_outer=4, max_inner=40, inner_rtol=1e-12, precision=pkg.FP64_BATCHED)
    base.update(kw)
    return pkg.default_config(nx, ny, **base)


def member_forcings(E, w, eps):
    f0 = E @ w
    return [f0] + [f0 + eps * E[:, i] for i in range(E.shape[1])]


def rel_l2(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b**2).sum()))


def vel_rel(gu, gv, ou, ov):
    num = ((gu - ou) ** 2).sum() + ((gv - ov) ** 2).sum()
    den = (ou**2).sum() + (ov**2).sum()
    return float(np.sqrt(num / den))


def oracle_trajectories(P, u0, v0, forcings, n_steps, workers=8):
    def one(f):
        fu, fv = oracle.control_to_faces(P, f)
        return oracle.trajectory(P, u0, v0, n_steps, fu, fv)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(one, forcings))


@pytest.mark.parametrize("precision", [pkg.FP64_BATCHED, pkg.FP64_PLAIN, pkg.MIXED])
def test_trajectory_parity_100_steps(precision):
    nx, ny, N, steps = 64, 32, 2, 100
    P = oracle.cavity_params(nx, ny, 1000.0)
    cfg = tight(nx, ny, Re=1000.0, n_steps=steps, n_window=10, n_members=N, precision=precision)
    if precision == pkg.MIXED:
        cfg.div_tol, cfg.inner_rtol, cfg.max_inner = 1e-12, 1e-5, 12
    E = oracle.ensemble_seeded(P, cfg.sigma, cfg.corr_len, N, cfg.seed)
    w = synth.weights(N)
    u0, v0 = synth.cavity_ic(nx, ny)
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(u0, v0)
    ens.set_ensemble(E)
    ens.forward_ensemble(w)
    ref = oracle_trajectories(P, u0, v0, member_forcings(E, w, cfg.eps), steps)
    F = oracle.fluid_mask(P).astype(bool)
    tol = 1e-4 if precision == pkg.MIXED else 1e-10
    members = [N] if precision == pkg.FP64_PLAIN else range(N + 1)
    for m in members:
        u, v, p = (t.cpu().numpy() for t in ens.get_state(m))
        ou, ov, op, _, _ = ref[m]
        err = vel_rel(u, v, ou, ov)
        assert err <= tol, (precision, m, err)
        pm, opm = p[F] - p[F].mean(), op[F] - op[F].mean()
        assert rel_l2(pm, opm) <= (1e-3 if precision == pkg.MIXED else 1e-8)
    d = ens.diagnostics()
    assert d["max_div"] <= cfg.div_tol
    assert (ens.member_status() == 0).all()
    ens.close()


# Tolerances of the cost / gradient parity.  FP64: the two solvers converge to 1e-12 divergence
# (GPU) and 1e-13 relative CG residual (oracle), so J agrees to ~1e-10 relative and the gradient,
# a difference quotient with eps = 1e-2, to ~1e-8 of its largest component; the bounds keep 10-100x
# of margin.  MIXED: the velocity tolerance of the mixed path is 1e-4 relative; J = 1/2||h||^2 is
# quadratic in the fluctuation, whose rounding errors are correlated across the window, so J is
# held to 1e-5 relative (measured: 7.7e-7 DOMAIN, 3.5e-6 SENSORS), and the gradient (member
# differences, where most of the mixed rounding cancels) to 1e-3 of its largest component.
TOL = {pkg.FP64_BATCHED: dict(J=1e-9, g=1e-6, series=1e-10), pkg.MIXED: dict(J=1e-5, g=1e-3, series=1e-6)}


@pytest.mark.parametrize("precision", [pkg.FP64_BATCHED, pkg.MIXED])
@pytest.mark.parametrize("mode", [pkg.COST_DOMAIN, pkg.COST_SENSORS])
def test_envar_costs_and_gradient_parity(mode, precision):
    nx, ny, N = 32, 16, 3
    P = oracle.cavity_params(nx, ny, 300.0)
    cfg = tight(nx, ny, Re=300.0, n_steps=120, n_window=60, n_members=N, cost_mode=mode, precision=precision)
    if precision == pkg.MIXED:
        cfg.div_tol, cfg.inner_rtol, cfg.max_inner, cfg.max_outer = 1e-12, 1e-5, 12, 6
    E = oracle.ensemble_seeded(P, cfg.sigma, cfg.corr_len, N, cfg.seed)
    w = synth.weights(N)
    u0, v0 = synth.cavity_ic(nx, ny)
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(u0, v0)
    ens.set_ensemble(E)
    ens.forward_ensemble(w)
    J, jp = ens.cost()
    g = ens.gradient()
    gs = ens.gradient_scalar()
    tol = TOL[precision]
    ref = oracle.envar_gradient(P, u0, v0, E, w, cfg.eps, cfg.n_steps, cfg.n_window, cost_mode=mode,
                                nthreads=4, want_series=True)
    np.testing.assert_allclose(J, ref["J"], rtol=tol["J"])
    assert jp == pytest.approx(ref["J_prior"], rel=1e-14)
    # scalar-anomaly form against the oracle's, the explicit contraction Y^T h_0 against the oracle's
    assert np.abs(gs - ref["g"]).max() <= tol["g"] * np.abs(ref["g"]).max(), (gs, ref["g"])
    if mode == pkg.COST_DOMAIN:
        gref, _ = oracle.envar_gradient_domain(P, u0, v0, E, w, cfg.eps, cfg.n_steps, cfg.n_window, nthreads=3)
    else:
        gref = oracle.sensor_gradient(ref["series"], w, cfg.eps)
    assert np.abs(g - gref).max() <= tol["g"] * np.abs(gref).max(), (g, gref)
    for m in range(N + 1):
        np.testing.assert_allclose(ens.get_series(m), ref["series"][m], rtol=0, atol=tol["series"])
    # df = E g / (N - 1)
    _, df = ens.gradient(want_df=True)
    np.testing.assert_allclose(df.cpu().numpy(), E @ g / (N - 1), rtol=1e-12, atol=1e-15)
    assert ens.excluded_members() == 0
    ens.close()


def test_plain_and_batched_agree():
    nx, ny, N = 32, 16, 3
    outs = []
    for prec in (pkg.FP64_PLAIN, pkg.FP64_BATCHED):
        cfg = tight(nx, ny, Re=300.0, n_steps=60, n_window=30, n_members=N, precision=prec)
        ens = pkg.Ensemble(cfg)
        ens.set_initial_state(*synth.cavity_ic(nx, ny))
        ens.forward_ensemble(synth.weights(N))
        outs.append((ens.cost()[0], ens.gradient()))
        ens.close()
    np.testing.assert_allclose(outs[0][0], outs[1][0], rtol=1e-13)
    np.testing.assert_allclose(outs[0][1], outs[1][1], rtol=1e-9, atol=1e-12 * np.abs(outs[1][1]).max())


@pytest.mark.parametrize("nx,ny,N", [(32, 16, 3), (128, 64, 8), (512, 256, 32)])
def test_ensemble_draw_matches_oracle(nx, ny, N):
    cfg = pkg.default_config(nx, ny, n_members=N, n_steps=2, n_window=1)
    ens = pkg.Ensemble(cfg)
    Eg = ens.get_ensemble().cpu().numpy()
    P = oracle.cavity_params(nx, ny, cfg.Re)
    Eo = oracle.ensemble_seeded(P, cfg.sigma, cfg.corr_len, N, cfg.seed)
    assert Eg.shape == Eo.shape
    assert np.abs(Eg - Eo).max() <= 1e-12 * np.abs(Eo).max()
    ens.close()


def test_step_applies_prior_preconditioned_update():
    """envar_step = forward ensemble + envar_gradient + the oracle's update of Sec. 3.3.1 (and the
    total cost of Eq. J_w), on the same w."""
    nx, ny, N = 32, 16, 4
    cfg = tight(nx, ny, Re=300.0, n_steps=40, n_window=20, n_members=N)
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(*synth.cavity_ic(nx, ny))
    w = synth.weights(N)
    ens.forward_ensemble(w)
    J, jp = ens.cost()
    g = ens.gradient()
    w1, J0 = ens.step(0.5, w)
    w_ref, J_ref = oracle.envar_step(w, g, 0.5, J[0])
    assert J0 == pytest.approx(J_ref, rel=1e-13)
    np.testing.assert_allclose(w1, w_ref, rtol=1e-13, atol=1e-16)
    ens.close()


def test_failed_member_is_excluded_from_the_gradient():
    """Host-side fault injection: one column of E scaled by 1e6 drives its member over the CFL
    limit (the kernels flag it; every loop stays bounded by its iteration cap).  That member's
    component of g keeps only the prior term, every other component is unchanged bit for bit, and
    the count is reported."""
    nx, ny, N, bad = 32, 16, 4, 2
    out = []
    for scale in (1.0, 1e6):
        cfg = tight(nx, ny, Re=300.0, n_steps=30, n_window=10, n_members=N, max_outer=3, max_inner=20)
        ens = pkg.Ensemble(cfg)
        ens.set_initial_state(*synth.cavity_ic(nx, ny))
        E = ens.get_ensemble().cpu().numpy()
        E[:, bad] *= scale
        ens.set_ensemble(E)
        w = synth.weights(N)
        w[bad] = 0.0   # the unperturbed forcing E w must not see the scaled column
        ens.forward_ensemble(w)
        st = ens.member_status()
        out.append((st, ens.gradient(), ens.excluded_members(), w))
        ens.close()
    (st0, g0, n0, _), (st1, g1, n1, w) = out
    assert (st0 == 0).all() and n0 == 0
    assert st1[bad + 1] & (pkg.ST_CFL | pkg.ST_NONFINITE) and n1 == 1
    assert all(st1[m] == 0 for m in range(N + 1) if m != bad + 1)
    assert g1[bad] == (N - 1) * w[bad]
    keep = [i for i in range(N) if i != bad]
    np.testing.assert_array_equal(g1[keep], g0[keep])


def test_unconverged_pressure_solve_is_reported():
    """max_outer = 1 with a divergence tolerance no solve can reach: every member carries the
    divergence bit, and with the unperturbed member failed there is no gradient."""
    nx, ny, N = 32, 16, 2
    cfg = tight(nx, ny, Re=300.0, n_steps=6, n_window=3, n_members=N, max_outer=1, max_inner=2, div_tol=1e-30)
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(*synth.cavity_ic(nx, ny))
    ens.forward_ensemble(synth.weights(N))
    st = ens.member_status()
    assert all(s & pkg.ST_DIVERGENCE for s in st), st
    with pytest.raises(pkg.EnvarError, match="ESTATE"):
        ens.gradient()
    with pytest.raises(pkg.EnvarError, match="ESTATE"):
        ens.step(0.5, synth.weights(N))
    ens.close()


def divergence_max(P, u, v):
    """max |D u| over the fluid cells, recomputed from an exported state."""
    F = oracle.fluid_mask(P).astype(bool)
    d = (u[:, 1:] - u[:, :-1]) / P.dx + (v[1:, :] - v[:-1, :]) / P.dy
    return float(np.abs(d[F]).max())


def test_bench_configuration_100_steps_parity():
    """The bench's launch configuration (512x256, Re 7500, N = 32, mixed precision, all 33 members in
    one launch, four member groups, solver parameters chosen by the autotuner exactly as the bench
    does) over 100 steps: members 0, 1, 16 and 32 against the oracle at the mixed tolerance 1e-4, and
    the divergence of every member's final state recomputed here from the exported fields."""
    nx, ny, N, steps = 512, 256, 32, 100
    cfg = pkg.default_config(nx, ny, Re=7500.0, n_steps=steps, n_window=50, n_members=N, precision=pkg.MIXED,
                             div_tol=1e-10)
    P = oracle.cavity_params(nx, ny, 7500.0)
    u0, v0 = synth.cavity_ic(nx, ny)
    w = synth.weights(N)
    sample = [0, 1, 16, N]
    Eo = oracle.ensemble_seeded(P, cfg.sigma, cfg.corr_len, N, cfg.seed)
    fs = member_forcings(Eo, w, cfg.eps)
    with cf.ThreadPoolExecutor(max_workers=1) as pool:
        # the oracle runs on the host cores while the GPU works
        fut = pool.submit(oracle_trajectories, P, u0, v0, [fs[m] for m in sample], steps, len(sample))
        ens = pkg.Ensemble(cfg)
        ens.set_initial_state(u0, v0)
        E = ens.get_ensemble().cpu().numpy()
        assert np.abs(E - Eo).max() <= 1e-12 * np.abs(Eo).max()
        chosen = ens.autotune(200)
        ens.forward_ensemble(w)
        assert (ens.member_status() == 0).all()
        assert ens.diagnostics()["max_div"] <= 1e-10
        states = {m: tuple(t.cpu().numpy() for t in ens.get_state(m)) for m in range(N + 1)}
        ens.close()
        ref = fut.result()
    for m in range(N + 1):
        assert divergence_max(P, states[m][0], states[m][1]) <= 1e-10, (m, chosen)
    for m, r in zip(sample, ref):
        u, v, _ = states[m]
        assert vel_rel(u, v, r[0], r[1]) <= 1e-4, (m, chosen)


@pytest.mark.parametrize("precision", [pkg.FP64_BATCHED, pkg.MIXED])
@pytest.mark.parametrize("nx,ny", [(64, 32), (512, 256)])
def test_multigrid_preconditioner_is_symmetric_positive(precision, nx, ny):
    """One V-cycle z = M r must be a fixed symmetric positive operator on mean-zero fluid fields
    (the tiled smoothers must reproduce a global red-black sweep exactly); CG relies on it."""
    cfg = pkg.default_config(nx, ny, n_members=1, n_steps=2, n_window=1, precision=precision)
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(*synth.cavity_ic(nx, ny))
    F = oracle.fluid_mask(oracle.cavity_params(nx, ny, 1000.0)).astype(bool)
    rng = np.random.default_rng(0)

    def field():
        r = np.where(F, rng.standard_normal(F.shape), 0.0)
        r[F] -= r[F].mean()
        return r

    r1, r2 = field(), field()
    z1 = ens.apply_preconditioner(r1).cpu().numpy()
    z2 = ens.apply_preconditioner(r2).cpu().numpy()
    tol = 1e-5 if precision == pkg.MIXED else 1e-12
    a, b = (z1 * r2).sum(), (r1 * z2).sum()
    assert abs(a - b) <= tol * np.sqrt((z1**2).sum() * (r2**2).sum()), (a, b)
    assert (z1 * r1).sum() > 0 and (z2 * r2).sum() > 0
    # linear: M (r1 + 2 r2) = z1 + 2 z2
    z3 = ens.apply_preconditioner(r1 + 2 * r2).cpu().numpy()
    assert np.abs(z3 - (z1 + 2 * z2)).max() <= 10 * tol * np.abs(z3).max()
    ens.close()


def test_forward_is_deterministic_at_bench_size():
    """All reductions are fixed-order and no kernel updates a field its neighbours read, so two
    identical forward runs must agree bit for bit (a race shows up here first)."""
    nx, ny, N = 512, 256, 32
    cfg = pkg.default_config(nx, ny, Re=7500.0, n_steps=20, n_window=10, n_members=N, precision=pkg.MIXED)
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(*synth.cavity_ic(nx, ny))
    w = synth.weights(N)
    outs = []
    for _ in range(2):
        ens.forward_ensemble(w)
        u, v, p = ens.get_state(N)
        outs.append((ens.cost()[0], u.cpu().numpy(), ens.diagnostics()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]
    assert outs[0][2]["max_div"] <= cfg.div_tol
    ens.close()


@pytest.mark.parametrize("precision", [pkg.FP64_BATCHED, pkg.MIXED])
def test_member_groups_give_identical_results(precision):
    """Concurrent member groups (parallel graph branches over member ranges) must not change any
    member's arithmetic: states, costs and the gradient agree bit for bit with one group."""
    nx, ny, N = 64, 32, 8
    out = []
    for groups in (1, 2, 3, 8):
        cfg = pkg.default_config(nx, ny, Re=1000.0, n_steps=24, n_window=8, n_members=N, precision=precision,
                                 member_groups=groups, steps_per_graph=10)
        ens = pkg.Ensemble(cfg)
        ens.set_initial_state(*synth.cavity_ic(nx, ny))
        w = synth.weights(N)
        ens.forward_ensemble(w)
        J, _ = ens.cost()
        g = ens.gradient()
        u, v, p = (t.cpu().numpy() for t in ens.get_state(N))
        out.append((J, g, u, v))
        ens.close()
    for J, g, u, v in out[1:]:
        assert np.array_equal(J, out[0][0]) and np.array_equal(g, out[0][1])
        assert np.array_equal(u, out[0][2]) and np.array_equal(v, out[0][3])


def test_autotune_keeps_the_divergence_target():
    """The autotuner only trades speed: the chosen parameters keep every member within div_tol,
    and the forward results stay within the mixed-precision tolerance of the untuned run."""
    nx, ny, N = 128, 64, 8
    cfgs = []
    outs = []
    for tune in (False, True):
        cfg = pkg.default_config(nx, ny, Re=1000.0, n_steps=60, n_window=20, n_members=N, precision=pkg.MIXED,
                                 div_tol=1e-10)
        ens = pkg.Ensemble(cfg)
        ens.set_initial_state(*synth.cavity_ic(nx, ny))
        if tune:
            chosen = ens.autotune(30)
            assert chosen["max_outer"] >= 1 and chosen["max_inner"] >= 1 and chosen["probe_ms_per_step"] > 0
            assert ens.config().max_inner == chosen["max_inner"]
        ens.forward_ensemble(synth.weights(N))
        assert ens.diagnostics()["max_div"] <= 1e-10
        assert (ens.member_status() == 0).all()
        u, v, _ = (t.cpu().numpy() for t in ens.get_state(N))
        outs.append((u, v))
        ens.close()
    assert vel_rel(outs[1][0], outs[1][1], outs[0][0], outs[0][1]) <= 1e-6


@pytest.mark.parametrize("precision", [pkg.FP64_BATCHED, pkg.MIXED])
def test_conditional_refinement_loop_is_exact_and_skips_work(precision):
    """The refinement loop as a conditional WHILE graph node runs only the refinements some member of
    the group needs; converged members never change, so the results equal the unrolled loop's bit for
    bit, with fewer kernel launches."""
    nx, ny, N = 64, 32, 8
    out = []
    for cond in (0, 1):
        cfg = pkg.default_config(nx, ny, Re=1000.0, n_steps=24, n_window=8, n_members=N, precision=precision,
                                 max_outer=8, conditional_refinement=cond, steps_per_graph=10)
        ens = pkg.Ensemble(cfg)
        ens.set_initial_state(*synth.cavity_ic(nx, ny))
        w = synth.weights(N)
        ens.forward_ensemble(w)   # captures the graphs
        n0 = pkg.capi.kernel_launches()
        ens.forward_ensemble(w)
        launches = pkg.capi.kernel_launches() - n0
        J, _ = ens.cost()
        u, v, p = (t.cpu().numpy() for t in ens.get_state(N))
        out.append((J, u, v, p, launches, ens.diagnostics()["max_div"]))
        assert (ens.member_status() == 0).all()
        ens.close()
    (J0, u0, v0, p0, l0, d0), (J1, u1, v1, p1, l1, d1) = out
    assert np.array_equal(J0, J1) and np.array_equal(u0, u1) and np.array_equal(v0, v1) and np.array_equal(p0, p1)
    assert d0 == d1
    assert l1 < 0.8 * l0, (l0, l1)


def test_extrapolated_initial_guess_changes_only_the_refinement_count():
    """MIXED: the pressure increment's initial guess 2 dp^n - dp^(n-1) against the last increment
    alone, at the bench grid, 33 member slots, over 1000 steps with the tuned solver.  Every solve
    ends at div_tol either way, so costs and gradients agree to the solver's accuracy (the
    trajectories differ by the divergence tolerance only).  In this forced, unsteady flow the
    extrapolated guess needs fewer refinements; in a near-steady one both guesses sit at the floor
    set by the FP32 rounding of the tendencies (fresh divergence every step), which no guess
    predicts."""
    nx, ny, N, n = 512, 256, 32, 1000
    out = []
    for ex in (0, 1):
        cfg = pkg.default_config(nx, ny, Re=7500.0, n_steps=n, n_window=n // 2, n_members=N, precision=pkg.MIXED,
                                 guess_extrapolation=ex, max_outer=10, max_inner=2, coarse_sweeps=1, inner_rtol=1e-3)
        cfg.nu_pre = cfg.nu_post = 3
        ens = pkg.Ensemble(cfg)
        ens.set_initial_state(*synth.cavity_ic(nx, ny))
        ens.forward_ensemble(synth.weights(N))
        J, _ = ens.cost()
        d = ens.diagnostics()
        out.append((J, ens.gradient(), d["outer_its"], d["max_div"]))
        assert (ens.member_status() == 0).all()
        ens.close()
    (J0, g0, o0, d0), (J1, g1, o1, d1) = out
    assert d0 <= 1e-10 and d1 <= 1e-10
    np.testing.assert_allclose(J1, J0, rtol=1e-6)
    assert np.linalg.norm(g1 - g0) <= 1e-5 * np.linalg.norm(g0)
    assert o1 < 0.9 * o0, (o0, o1)


def test_chaotic_configuration_statistics_mixed_against_fp64():
    """The chaotic-regime configuration (1024x512, Re 15000) shortened to 600 + 600 steps with N = 8:
    the mixed-precision batched path against the FP64 batched path (itself tied to the oracle at
    1e-10), at the statistics tolerances of that regime: the time-mean fluctuation energy of every
    member within 2 %, and the EnVar gradient with cosine >= 0.95."""
    nx, ny, N = 1024, 512, 8
    out = {}
    for prec in (pkg.FP64_BATCHED, pkg.MIXED):
        # the FP64 reference at its own rounding floor (a few FP64 solves at this size end just above
        # 1e-10 however many refinements they get); the mixed path at the 1e-10 target
        kw = dict(max_outer=12, max_inner=8, inner_rtol=1e-4, div_tol=1e-9) if prec == pkg.FP64_BATCHED else \
            dict(div_tol=1e-10)
        cfg = pkg.default_config(nx, ny, Re=15000.0, n_steps=1200, n_window=600, n_members=N, precision=prec, **kw)
        ens = pkg.Ensemble(cfg)
        ens.set_initial_state(*synth.cavity_ic(nx, ny))
        w = synth.weights(N)
        ens.forward_ensemble(w)
        J, _ = ens.cost()
        out[prec] = (J, ens.gradient(), ens.member_status())
        ens.close()
    J64, g64, s64 = out[pkg.FP64_BATCHED]
    Jmx, gmx, smx = out[pkg.MIXED]
    assert (smx == 0).all() and (s64 == 0).all()
    assert np.abs(Jmx / J64 - 1.0).max() <= 0.02, (Jmx, J64)
    cos = float(gmx @ g64 / (np.linalg.norm(gmx) * np.linalg.norm(g64)))
    assert cos >= 0.95, cos
