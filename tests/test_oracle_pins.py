"""Pins for the FP64 CPU oracle against facts fixed by the paper or by mathematics,
independent of the oracle's own code: closed forms, exact discrete fixed points,
invariants, library routines (numpy Philox, dense LU) and brute force.

Each pin is chosen so that a plausible mistake (a dropped term, a wrong sign, a
transposed index, a wrong boundary reflection) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2605_23812_gb300 import synth

TWO_PI = 2.0 * math.pi


def periodic_box(n, Re, dt, advection=1, origin=0.0):
    return oracle.make_params(nx=n, ny=n, x0=origin, x1=origin + TWO_PI, y0=origin, y1=origin + TWO_PI,
                              Re=Re, dt=dt, bc_x=1, bc_y=1, geometry=1, advection=advection)


def face_coords(P):
    dx, dy = P.dx, P.dy
    xu = P.x0 + np.arange(P.nx + 1) * dx           # u faces (x)
    yu = P.y0 + (np.arange(P.ny) + 0.5) * dy       # u faces (y)
    xv = P.x0 + (np.arange(P.nx) + 0.5) * dx       # v faces (x)
    yv = P.y0 + np.arange(P.ny + 1) * dy           # v faces (y)
    return xu, yu, xv, yv


# --------------------------------------------------------------------------
# random numbers: Philox4x64-10 against numpy's implementation (a library
# routine built from the same published definition), Box-Muller from its
# textbook formula applied to numpy's words.
# --------------------------------------------------------------------------
def test_philox_matches_numpy():
    M = 2**64 - 1
    for key in [(0, 0), (123, 456), (M, 7), (1000, 0)]:
        # counter pre-incremented by numpy: start at -1 so the first block is counter 0
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array([M, M, M, M], dtype=np.uint64))
        raw = bg.random_raw(20)
        for b in range(5):
            out = oracle.philox4x64_10([b, 0, 0, 0], key)
            assert (out == raw[4 * b:4 * b + 4]).all(), (key, b)


def test_normals_are_box_muller_of_philox_words():
    seed, stream = 1001, 0
    M = 2**64 - 1
    bg = np.random.Philox(key=np.array([seed, stream], dtype=np.uint64),
                          counter=np.array([M, M, M, M], dtype=np.uint64))
    w = bg.random_raw(64).reshape(16, 4)
    ref = []
    for blk in w:
        for a, b in ((blk[0], blk[1]), (blk[2], blk[3])):
            u1 = (float(int(a) >> 11) + 1.0) * 2.0**-53
            u2 = float(int(b) >> 11) * 2.0**-53
            r = math.sqrt(-2.0 * math.log(u1))
            ref += [r * math.cos(TWO_PI * u2), r * math.sin(TWO_PI * u2)]
    got = oracle.normals(seed, stream, 0, 64)
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-15)
    # an offset window is the same stream
    np.testing.assert_array_equal(oracle.normals(seed, stream, 13, 20), got[13:33])


def test_normals_distribution():
    scipy_stats = pytest.importorskip("scipy.stats")
    z = oracle.normals(99, 3, 0, 200000)
    assert abs(z.mean()) < 5.0 / math.sqrt(len(z))
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / len(z))
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-4


# --------------------------------------------------------------------------
# Poiseuille: the exact discrete steady state with walls on face lines is
# u_j = (f Re / 2) ((y_j - y_lo)(y_hi - y_j) + h^2/4)  (the h^2/4 term is what
# the mirror-ghost no-slip rule adds to the parabola; it solves the discrete
# equations exactly).  Pins diffusion, forcing, both wall reflections (domain
# edge and buried solid faces) and the projection being inert.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("geometry", [1, 2])
def test_poiseuille_horizontal_fixed_point(geometry):
    lo, hi = (0.0, 1.0) if geometry == 1 else (0.25, 0.75)
    P = oracle.make_params(nx=8, ny=32, x0=0.0, x1=0.5, y0=0.0, y1=1.0, Re=50.0, dt=2e-3,
                           bc_x=1, bc_y=2, geometry=geometry, ch_lo=lo, ch_hi=hi)
    fx, Re, dy = 0.3, P.Re, P.dy
    _, yu, _, _ = face_coords(P)
    prof = np.where((yu > lo) & (yu < hi), 0.5 * fx * Re * ((yu - lo) * (hi - yu) + 0.25 * dy * dy), 0.0)
    u = np.repeat(prof[:, None], P.nx + 1, axis=1)
    v = np.zeros((P.ny + 1, P.nx))
    s = oracle.Sim(P)
    s.set_state(u, v)
    s.set_forcing(np.full_like(u, fx), np.zeros_like(v))
    s.step(25)
    u1, v1, _ = s.state()
    assert np.abs(u1 - u).max() <= 1e-12 * np.abs(u).max()
    assert np.abs(v1).max() <= 1e-13
    # and the plain parabola (no h^2/4) is NOT a fixed point: the ghost rule matters
    prof2 = np.where((yu > lo) & (yu < hi), 0.5 * fx * Re * (yu - lo) * (hi - yu), 0.0)
    s.set_state(np.repeat(prof2[:, None], P.nx + 1, axis=1), v)
    s.step(25)
    assert np.abs(s.state()[0] - np.repeat(prof2[:, None], P.nx + 1, axis=1)).max() > 1e-6


def test_poiseuille_vertical_fixed_point():
    lo, hi = 0.25, 0.75
    P = oracle.make_params(nx=32, ny=8, x0=0.0, x1=1.0, y0=0.0, y1=0.5, Re=40.0, dt=2e-3,
                           bc_x=1, bc_y=1, geometry=3, ch_lo=lo, ch_hi=hi)
    fy, Re, dx = -0.2, P.Re, P.dx
    _, _, xv, _ = face_coords(P)
    prof = np.where((xv > lo) & (xv < hi), 0.5 * fy * Re * ((xv - lo) * (hi - xv) + 0.25 * dx * dx), 0.0)
    v = np.repeat(prof[None, :], P.ny + 1, axis=0)
    u = np.zeros((P.ny, P.nx + 1))
    s = oracle.Sim(P)
    s.set_state(u, v)
    s.set_forcing(np.zeros_like(u), np.full_like(v, fy))
    s.step(25)
    u1, v1, _ = s.state()
    assert np.abs(v1 - v).max() <= 1e-12 * np.abs(v).max()
    assert np.abs(u1).max() <= 1e-13


# --------------------------------------------------------------------------
# Free-slip top (Sec. 4.4 boundary conditions, the workload's reading: symmetry at the top,
# no slip at the bottom).  Half channel of height H, periodic in x, uniform fx: the continuous
# steady profile is u = (fx Re / 2) y (2H - y), maximal at the top.  On the MAC grid the mirror
# ghost of the bottom wall adds h^2/4 as for Poiseuille, and the even ghost of the top
# (u_ny = u_ny-1) is exactly the symmetry of y (2H - y) about y = H, so
# u_j = (fx Re / 2)(y_j (2H - y_j) + h^2/4) solves the discrete equations exactly.
# --------------------------------------------------------------------------
def _half_channel(P, fx):
    _, yu, _, _ = face_coords(P)
    H = P.y1 - P.y0
    y = yu - P.y0
    return 0.5 * fx * P.Re * (y * (2.0 * H - y) + 0.25 * P.dy * P.dy)


def _half_channel_drift(P, fx):
    prof = _half_channel(P, fx)
    u = np.repeat(prof[:, None], P.nx + 1, axis=1)
    v = np.zeros((P.ny + 1, P.nx))
    s = oracle.Sim(P)
    s.set_state(u, v)
    s.set_forcing(np.full_like(u, fx), np.zeros_like(v))
    s.step(25)
    u1, v1, _ = s.state()
    return np.abs(u1 - u).max() / np.abs(u).max(), np.abs(v1).max()


def _half_channel_params(bc_y):
    return oracle.make_params(nx=8, ny=24, x0=0.0, x1=0.5, y0=0.0, y1=0.75, Re=40.0, dt=2e-3,
                              bc_x=1, bc_y=bc_y, geometry=1)


def test_free_slip_top_half_channel_fixed_point():
    du, vmax = _half_channel_drift(_half_channel_params(0), 0.25)
    assert du <= 1e-12 and vmax <= 1e-13, (du, vmax)
    # a no-slip top (bc_y = 2) does not hold the half-channel profile
    du2, _ = _half_channel_drift(_half_channel_params(2), 0.25)
    assert du2 > 1e-4, du2


def test_free_slip_top_pin_fails_on_a_no_slip_top(tmp_path):
    """Plant the plausible mistake (an odd ghost, i.e. no slip, at the top) in a copy of the
    oracle: the fixed-point pin must catch it."""
    with oracle.planted_mistake("UG(s, i, ny) = UG(s, i, ny - 1);      /* top: free slip */",
                                "UG(s, i, ny) = -UG(s, i, ny - 1);", str(tmp_path)):
        du, _ = _half_channel_drift(_half_channel_params(0), 0.25)
    assert du > 1e-4, du


# --------------------------------------------------------------------------
# Slip segments of the lower wall (Sec. 4.4, the paper's boundary conditions): a channel buried in
# the mask with a slip lower wall and a no-slip upper wall is the free-slip half channel upside down,
# u_j = (fx Re / 2)(y'_j (2H - y'_j) + h^2/4) with y' measured down from the upper wall.
# --------------------------------------------------------------------------
def _slip_channel_drift(lip_slip):
    lo, hi = 0.25, 0.75
    P = oracle.make_params(nx=8, ny=32, x0=0.0, x1=0.5, y0=0.0, y1=1.0, Re=50.0, dt=2e-3, bc_x=1, bc_y=2,
                           geometry=2, ch_lo=lo, ch_hi=hi, lip_slip=lip_slip, slip_lo=1e9, slip_hi=2e9)
    fx, H = 0.3, hi - lo
    _, yu, _, _ = face_coords(P)
    yp = hi - yu
    prof = np.where((yu > lo) & (yu < hi), 0.5 * fx * P.Re * (yp * (2 * H - yp) + 0.25 * P.dy**2), 0.0)
    u = np.repeat(prof[:, None], P.nx + 1, axis=1)
    v = np.zeros((P.ny + 1, P.nx))
    s = oracle.Sim(P)
    s.set_state(u, v)
    s.set_forcing(np.full_like(u, fx), np.zeros_like(v))
    s.step(25)
    return np.abs(s.state()[0] - u).max() / np.abs(u).max()


def test_lower_wall_slip_segments_fixed_point():
    assert _slip_channel_drift(1) <= 1e-12
    assert _slip_channel_drift(0) > 1e-4      # the no-slip lower wall does not hold this profile


# --------------------------------------------------------------------------
# Convective outlet (the workload's outlet reading of Sec. 4.4: du/dt + Uc du/dx = 0 at the
# outflow face with Uc = 1, then a uniform flux shift).  A channel periodic in y carries a
# divergence-free disturbance u = 1 + e a(x) cos(ky), v = -e a'(x) sin(ky)/k on the uniform
# stream U = 1; linearised about U the inviscid equations are pure transport at speed 1 (the
# pressure disturbance vanishes), so the exact outflow profile is 1 + e a(x_out - t) cos(ky),
# averaged over the face.  The outlet values must converge to it as the grid is refined; a
# wrong sign, neighbour or speed in the upwind update does not converge.
# --------------------------------------------------------------------------
def _outlet_error(nx, T=0.8, eps=1e-3, sigma=0.15, xc=1.2):
    ny = nx // 2
    k = TWO_PI
    # y in [1, 2]: the inlet profile erf(y / 0.1) equals 1 to rounding there
    P = oracle.make_params(nx=nx, ny=ny, x0=0.0, x1=2.0, y0=1.0, y1=2.0, Re=1e6, dt=0.3 * 2.0 / nx,
                           bc_x=0, bc_y=1, geometry=1, advection=1)
    dx, dy = P.dx, P.dy
    bump = lambda x: np.exp(-((x - xc) / sigma) ** 2)
    X, Y = np.meshgrid(np.arange(nx + 1) * dx, P.y0 + np.arange(ny + 1) * dy)
    psi = Y + eps * bump(X) * np.sin(k * Y) / k          # streamfunction at cell corners
    u0 = (psi[1:, :] - psi[:-1, :]) / dy
    v0 = -(psi[:, 1:] - psi[:, :-1]) / dx
    s = oracle.Sim(P)
    s.set_state(u0, v0)
    yc = P.y0 + (np.arange(ny) + 0.5) * dy
    face_avg_cos = (np.sin(k * (yc + dy / 2)) - np.sin(k * (yc - dy / 2))) / (k * dy)
    err = 0.0
    for n in range(1, int(round(T / P.dt)) + 1):
        s.step(1)
        u = s.state()[0]
        exact = 1.0 + eps * bump(P.x1 - n * P.dt) * face_avg_cos
        err = max(err, np.abs(u[:, nx] - exact).max())
    return err / eps


def test_convective_outlet_converges_to_transport_solution():
    errs = [_outlet_error(n) for n in (32, 64)]
    assert errs[1] < 0.15, errs
    assert errs[0] / errs[1] > 2.0, errs


@pytest.mark.parametrize("old,new", [
    # sign of the upwind difference
    ("s->ub_next[j] = ub - s->P.dt * s->P.conv_speed * (ub - ui) / s->dx;",
     "s->ub_next[j] = ub + s->P.dt * s->P.conv_speed * (ub - ui) / s->dx;"),
    # wrong upwind neighbour (two faces in)
    ("double ub = s->u[IU(s, nx, j)], ui = s->u[IU(s, nx - 1, j)];",
     "double ub = s->u[IU(s, nx, j)], ui = s->u[IU(s, nx - 2, j)];"),
    # time step dropped from the update
    ("s->ub_next[j] = ub - s->P.dt * s->P.conv_speed * (ub - ui) / s->dx;",
     "s->ub_next[j] = ub - s->P.conv_speed * (ub - ui) * 0.5;"),
])
def test_convective_outlet_pin_fails_on_planted_mistakes(tmp_path, old, new):
    with oracle.planted_mistake(old, new, str(tmp_path)):
        errs = [_outlet_error(n) for n in (32, 64)]
    assert not (errs[1] < 0.15 and errs[0] / errs[1] > 2.0), errs


# --------------------------------------------------------------------------
# Taylor-Green, Stokes: on a square periodic MAC grid the sampled TG field is
# discretely divergence-free and an eigenvector of the discrete Laplacian with
# eigenvalue lam = -(4/dx^2) sin^2(dx/2) - (4/dy^2) sin^2(dy/2).  The explicit
# scheme then multiplies the amplitude by the Euler-then-AB2 recurrence exactly.
# --------------------------------------------------------------------------
def tg_fields(P):
    xu, yu, xv, yv = face_coords(P)
    u = np.sin(xu)[None, :] * np.cos(yu)[:, None]
    v = -np.cos(xv)[None, :] * np.sin(yv)[:, None]
    return u, v


def test_taylor_green_stokes_exact_recurrence():
    P = periodic_box(16, Re=10.0, dt=0.01, advection=0)
    u0, v0 = tg_fields(P)
    nu, dt = 1.0 / P.Re, P.dt
    lam = -(4 / P.dx**2) * math.sin(P.dx / 2) ** 2 - (4 / P.dy**2) * math.sin(P.dy / 2) ** 2
    a = [1.0, 1.0 + dt * nu * lam]
    for _ in range(40):
        a.append(a[-1] + dt * nu * lam * (1.5 * a[-1] - 0.5 * a[-2]))
    s = oracle.Sim(P)
    s.set_state(u0, v0)
    done = 0
    for n in (1, 2, 7, 41):
        s.step(n - done)
        done = n
        u, v, _ = s.state()
        np.testing.assert_allclose(u, a[n] * u0, rtol=0, atol=1e-13)
        np.testing.assert_allclose(v, a[n] * v0, rtol=0, atol=1e-13)


def test_taylor_green_second_order():
    """Full Navier-Stokes TG decay u = sin x cos y e^{-2t/Re}: second-order error."""
    errs = []
    for n in (16, 32, 64):
        dx = TWO_PI / n
        P = periodic_box(n, Re=100.0, dt=0.2 * dx)
        T = 0.8
        steps = int(round(T / P.dt))
        u0, v0 = tg_fields(P)
        u, v, _, md, _ = oracle.trajectory(P, u0, v0, steps)
        decay = math.exp(-2.0 * steps * P.dt / P.Re)
        errs.append(max(np.abs(u - decay * u0).max(), np.abs(v - decay * v0).max()))
        assert md < 1e-11
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(slopes) > 1.85, (errs, slopes)


def test_manufactured_solution_second_order():
    """Steady manufactured flow with a non-gradient advection term; f = (u.grad)u - lap(u)/Re.
    A dropped or mis-signed advection or diffusion piece leaves an O(T) error instead of O(h^2)."""
    sp = pytest.importorskip("sympy")
    X, Y = sp.symbols("x y")
    Re = 10.0
    psi = sp.sin(X) * sp.sin(Y) + sp.Rational(3, 10) * sp.sin(2 * X + Y)
    U, V = sp.diff(psi, Y), -sp.diff(psi, X)
    fx = U * sp.diff(U, X) + V * sp.diff(U, Y) - (sp.diff(U, X, 2) + sp.diff(U, Y, 2)) / Re
    fy = U * sp.diff(V, X) + V * sp.diff(V, Y) - (sp.diff(V, X, 2) + sp.diff(V, Y, 2)) / Re
    lam = {k: sp.lambdify((X, Y), e, "numpy") for k, e in dict(psi=psi, U=U, V=V, fx=fx, fy=fy).items()}
    errs, errs_noadv = [], []
    for n in (16, 32, 64):
        dx = TWO_PI / n
        P = periodic_box(n, Re=Re, dt=min(0.1 * dx * dx * Re, 0.1 * dx))
        xu, yu, xv, yv = face_coords(P)
        xc_, yc_ = np.meshgrid(P.x0 + np.arange(n + 1) * dx, P.y0 + np.arange(n + 1) * P.dy)
        ps = lam["psi"](xc_, yc_)                       # psi at cell corners [j][i]
        u0 = (ps[1:, :] - ps[:-1, :]) / P.dy            # (ny, nx+1)
        v0 = -(ps[:, 1:] - ps[:, :-1]) / dx             # (ny+1, nx)
        fu = lam["fx"](xu[None, :], yu[:, None]) * np.ones((n, n + 1))
        fv = lam["fy"](xv[None, :], yv[:, None]) * np.ones((n + 1, n))
        ue = lam["U"](xu[None, :], yu[:, None]) * np.ones((n, n + 1))
        ve = lam["V"](xv[None, :], yv[:, None]) * np.ones((n + 1, n))
        steps = int(round(0.3 / P.dt))
        u, v, _, _, _ = oracle.trajectory(P, u0, v0, steps, fu, fv)
        errs.append(max(np.abs(u - ue).max(), np.abs(v - ve).max()))
        # forcing without its advection part: the solution must drift O(1)
        fxd = sp.lambdify((X, Y), -(sp.diff(U, X, 2) + sp.diff(U, Y, 2)) / Re, "numpy")
        fyd = sp.lambdify((X, Y), -(sp.diff(V, X, 2) + sp.diff(V, Y, 2)) / Re, "numpy")
        u2, v2, _, _, _ = oracle.trajectory(P, u0, v0, steps, fxd(xu[None, :], yu[:, None]) * np.ones((n, n + 1)),
                                            fyd(xv[None, :], yv[:, None]) * np.ones((n + 1, n)))
        errs_noadv.append(max(np.abs(u2 - ue).max(), np.abs(v2 - ve).max()))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(slopes) > 1.85, (errs, slopes)
    assert min(errs_noadv) > 20 * errs[-1]


def test_inviscid_energy_conservation():
    """Central divergence-form advection conserves discrete kinetic energy for a
    divergence-free field; the only drift is the time integrator's, which falls
    at least 2^2 per halving of dt (a sign error in any advection term gives a
    drift that does not fall with dt)."""
    drifts = []
    n = 24
    for dt in (0.02, 0.01):
        P = periodic_box(n, Re=1e30, dt=dt)
        dx = P.dx
        xc_, yc_ = np.meshgrid(np.arange(n + 1) * dx, np.arange(n + 1) * dx)
        ps = np.zeros_like(xc_)
        r = np.random.default_rng(5)
        for kx in range(1, 4):
            for ky in range(1, 4):
                ps += r.normal() * np.sin(kx * xc_ + r.uniform(0, 6)) * np.sin(ky * yc_ + r.uniform(0, 6)) / (kx * kx + ky * ky)
        u0 = (ps[1:, :] - ps[:-1, :]) / dx
        v0 = -(ps[:, 1:] - ps[:, :-1]) / dx
        steps = int(round(0.6 / dt))
        u, v, _, _, _ = oracle.trajectory(P, u0, v0, steps)
        e0 = (u0[:, :-1] ** 2).sum() + (v0[:-1, :] ** 2).sum()
        e1 = (u[:, :-1] ** 2).sum() + (v[:-1, :] ** 2).sum()
        drifts.append(abs(e1 - e0) / e0)
    assert drifts[0] < 1e-3
    assert drifts[1] < drifts[0] / 3.5, drifts


# --------------------------------------------------------------------------
# Open cavity invariants: divergence below the solver tolerance, inflow flux
# equals outflow flux, walls and buried faces hold zero, inlet holds erf(y/0.1).
# --------------------------------------------------------------------------
def test_cavity_invariants():
    P = oracle.cavity_params(64, 32, 1000.0)
    u0, v0 = synth.cavity_ic(64, 32)
    s = oracle.Sim(P)
    s.set_state(u0, v0)
    s.step(15)
    u, v, _ = s.state()
    assert s.max_div() < 1e-11
    qin, qout = s.fluxes()
    assert abs(qin - qout) <= 1e-13 * abs(qin)
    uk, vk = s.face_kinds()
    assert np.all(u[(uk == oracle.FK_WALL) | (uk == oracle.FK_SOLID)] == 0.0)
    assert np.all(v[(vk == oracle.FK_WALL) | (vk == oracle.FK_SOLID)] == 0.0)
    yc = P.y0 + (np.arange(P.ny) + 0.5) * P.dy
    inl = uk[:, 0] == oracle.FK_INLET
    np.testing.assert_allclose(u[inl, 0], [math.erf(y / 0.1) for y in yc[inl]], rtol=1e-15)
    assert np.all(yc[inl] > 0) and np.all(~inl[yc < 0])
    F = oracle.fluid_mask(P)
    # open cavity geometry: everything above y=0 fluid; below, exactly the cells with 0 < xc < 1
    xc = P.x0 + (np.arange(P.nx) + 0.5) * P.dx
    assert F[yc > 0].all()
    assert (F[yc < 0] == ((xc > 0) & (xc < 1))[None, :]).all()


def test_projection_idempotent_and_symmetric():
    P = oracle.cavity_params(32, 16, 1000.0)
    s = oracle.Sim(P)
    uk, vk = s.face_kinds()
    rng = np.random.default_rng(3)

    def rand_field():
        u = np.where(uk == oracle.FK_UNKNOWN, rng.standard_normal(uk.shape), 0.0)
        v = np.where(vk == oracle.FK_UNKNOWN, rng.standard_normal(vk.shape), 0.0)
        return u, v

    a, b = rand_field(), rand_field()
    pa, pb = s.project(*a), s.project(*b)
    ppa = s.project(*pa)
    np.testing.assert_allclose(ppa[0], pa[0], atol=1e-11)
    np.testing.assert_allclose(ppa[1], pa[1], atol=1e-11)
    lhs = (pa[0] * b[0]).sum() + (pa[1] * b[1]).sum()
    rhs = (a[0] * pb[0]).sum() + (a[1] * pb[1]).sum()
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1.0)
    # projected field is discretely divergence-free
    div = (pa[0][:, 1:] - pa[0][:, :-1]) / P.dx + (pa[1][1:, :] - pa[1][:-1, :]) / P.dy
    F = oracle.fluid_mask(P).astype(bool)
    assert np.abs(div[F]).max() < 1e-10


# --------------------------------------------------------------------------
# Poisson: periodic eigenfunctions (closed form), dense least-squares solve
# (library) of the masked Neumann Laplacian assembled from the face rule.
# --------------------------------------------------------------------------
def test_negative_laplacian_periodic_eigen():
    P = oracle.make_params(nx=20, ny=12, x0=0.0, x1=TWO_PI, y0=0.0, y1=TWO_PI, bc_x=1, bc_y=1, geometry=1)
    s = oracle.Sim(P)
    xc = (np.arange(P.nx) + 0.5) * P.dx
    yc = (np.arange(P.ny) + 0.5) * P.dy
    for kx, ky in ((1, 0), (2, 3), (3, 1)):
        x = np.cos(kx * xc)[None, :] * np.cos(ky * yc)[:, None]
        lam = (4 / P.dx**2) * math.sin(kx * P.dx / 2) ** 2 + (4 / P.dy**2) * math.sin(ky * P.dy / 2) ** 2
        np.testing.assert_allclose(s.apply_negL(x), lam * x, atol=1e-10)


def test_poisson_solve_matches_dense_lstsq():
    P = oracle.cavity_params(24, 12, 1000.0)
    s = oracle.Sim(P)
    F = oracle.fluid_mask(P).astype(bool)
    uk, vk = s.face_kinds()
    ny, nx = F.shape
    idx = -np.ones((ny, nx), dtype=int)
    idx[F] = np.arange(F.sum())
    n = F.sum()
    A = np.zeros((n, n))
    for j in range(ny):
        for i in range(nx):
            if not F[j, i]:
                continue
            for (di, dj, open_, h) in ((1, 0, i + 1 < nx and uk[j, i + 1] == oracle.FK_UNKNOWN, P.dx),
                                       (-1, 0, i > 0 and uk[j, i] == oracle.FK_UNKNOWN, P.dx),
                                       (0, 1, j + 1 < ny and vk[j + 1, i] == oracle.FK_UNKNOWN, P.dy),
                                       (0, -1, j > 0 and vk[j, i] == oracle.FK_UNKNOWN, P.dy)):
                if open_:
                    A[idx[j, i], idx[j, i]] += 1 / h**2
                    A[idx[j, i], idx[j + dj, i + di]] -= 1 / h**2
    rng = np.random.default_rng(11)
    b = np.zeros((ny, nx))
    b[F] = rng.standard_normal(n)
    b[F] -= b[F].mean()
    x = s.poisson_solve(b)
    xd = np.linalg.lstsq(A, b[F], rcond=None)[0]
    xd -= xd.mean()
    np.testing.assert_allclose(x[F], xd, atol=1e-9 * np.abs(xd).max())
    assert np.all(x[~F] == 0.0)
    # and the oracle's operator is the assembled one
    np.testing.assert_allclose(s.apply_negL(x)[F], A @ x[F], atol=1e-9)


# --------------------------------------------------------------------------
# Ensemble (Sec. 3.3.2): the sampler's factors reproduce the paper's kernel
# exp(-d^2/a^2); E is sigma (Gx (x) Gy) Z restricted to the control cells; the
# sample covariance of many draws approaches B.
# --------------------------------------------------------------------------
def test_sampler_factor_reproduces_gaussian_kernel():
    for nx, ny in ((32, 16), (128, 64), (512, 256)):
        P = oracle.cavity_params(nx, ny, 1000.0)
        a = 0.05
        Gx, Gy = oracle.sampler_factors(P, a)
        ia, ib, ja, jb = oracle.control_rect(P)
        xc = P.x0 + (np.arange(ia, ib + 1) + 0.5) * P.dx
        yc = P.y0 + (np.arange(ja, jb + 1) + 0.5) * P.dy
        Kx = np.exp(-((xc[:, None] - xc[None, :]) ** 2) / a**2)
        Ky = np.exp(-((yc[:, None] - yc[None, :]) ** 2) / a**2)
        np.testing.assert_allclose(Gx @ Gx.T, Kx, atol=1e-13)
        np.testing.assert_allclose(Gy @ Gy.T, Ky, atol=1e-13)


def test_ensemble_is_kronecker_draw_on_control_cells():
    P = oracle.cavity_params(32, 16, 1000.0)
    sigma, a, N = 0.1, 0.05, 3
    nrx, nry, nxix, nxiy = oracle.sampler_dims(P, a)
    rng = np.random.default_rng(2)
    Z = rng.standard_normal((N, 2, nxiy, nxix))
    E = oracle.ensemble_from_noise(P, sigma, a, N, Z)
    Gx, Gy = oracle.sampler_factors(P, a)
    ci, cj = oracle.control_cells(P)
    ia, _, ja, _ = oracle.control_rect(P)
    ncc = len(ci)
    assert E.shape == (2 * ncc, N)
    for k in range(N):
        for c in range(2):
            field = sigma * np.einsum("yk,ckx,xj->cyj", Gy, Z[k, c][None], Gx.T)[0]   # [iy][ix]
            np.testing.assert_allclose(E[c * ncc:(c + 1) * ncc, k], field[cj - ja, ci - ia], atol=1e-14)
    Es = oracle.ensemble_seeded(P, sigma, a, N, 1000)
    Zs = oracle.normals(1000, 0, 0, N * 2 * nxiy * nxix).reshape(N, 2, nxiy, nxix)
    np.testing.assert_allclose(Es, oracle.ensemble_from_noise(P, sigma, a, N, Zs), atol=0)


def test_ensemble_sample_covariance_approaches_B():
    P = oracle.make_params(nx=40, ny=40, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x=1, bc_y=1, geometry=1)
    region = (0.3, 0.45, 0.4, 0.5)
    sigma, a, N = 0.1, 0.05, 4000
    E = oracle.ensemble_seeded(P, sigma, a, N, 77, region=region)
    ci, cj = oracle.control_cells(P, region)
    x = P.x0 + (ci + 0.5) * P.dx
    y = P.y0 + (cj + 0.5) * P.dy
    B = sigma**2 * np.exp(-((x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2) / a**2)
    ncc = len(ci)
    for c in range(2):
        S = E[c * ncc:(c + 1) * ncc] @ E[c * ncc:(c + 1) * ncc].T / N
        assert np.abs(S - B).max() < 5 * sigma**2 * math.sqrt(2.0 / N)
    # components are independent
    C = E[:ncc] @ E[ncc:].T / N
    assert np.abs(C).max() < 5 * sigma**2 * math.sqrt(2.0 / N)


def test_control_to_faces_is_cell_average():
    P = oracle.cavity_params(32, 16, 1000.0)
    ci, cj = oracle.control_cells(P)
    ncc = len(ci)
    s = oracle.Sim(P)
    uk, vk = s.face_kinds()
    q = ncc // 2
    f = np.zeros(2 * ncc)
    f[q] = 1.0
    f[ncc + q] = -2.0
    fu, fv = oracle.control_to_faces(P, f)
    i, j = ci[q], cj[q]
    expect_u = np.zeros_like(fu)
    for ii in (i, i + 1):
        if uk[j, ii] == oracle.FK_UNKNOWN:
            expect_u[j, ii] = 0.5
    expect_v = np.zeros_like(fv)
    for jj in (j, j + 1):
        if vk[jj, i] == oracle.FK_UNKNOWN:
            expect_v[jj, i] = -1.0
    np.testing.assert_array_equal(fu, expect_u)
    np.testing.assert_array_equal(fv, expect_v)
    # the control region is the fluid part of [-0.5,1]x[-0.2,0.3] (centres, inclusive)
    F = oracle.fluid_mask(P)
    xc = P.x0 + (np.arange(P.nx) + 0.5) * P.dx
    yc = P.y0 + (np.arange(P.ny) + 0.5) * P.dy
    inside = ((xc[None, :] >= -0.5) & (xc[None, :] <= 1.0) & (yc[:, None] >= -0.2) & (yc[:, None] <= 0.3)) & (F > 0)
    assert inside.sum() == ncc
    assert inside[cj, ci].all()


# --------------------------------------------------------------------------
# EnVar gradient (Eq. gradient_EnVar) against closed forms and brute force.
# --------------------------------------------------------------------------
def test_gradient_quadratic_closed_form():
    """J(w) = 1/2 w^T Q w + b^T w with E = I: forward differences of step eps give
    exactly Q w + b + eps/2 diag(Q); plus the prior gradient (N-1) w."""
    rng = np.random.default_rng(4)
    N = 6
    A = rng.standard_normal((N, N))
    Q = A @ A.T + N * np.eye(N)
    bvec = rng.standard_normal(N)
    w = rng.standard_normal(N)
    eps = 1e-3
    Jf = lambda x: 0.5 * x @ Q @ x + bvec @ x
    J = np.array([Jf(w)] + [Jf(w + eps * np.eye(N)[i]) for i in range(N)])
    g, jp = oracle.gradient_from_costs(J, w, eps)
    np.testing.assert_allclose(g, Q @ w + bvec + 0.5 * eps * np.diag(Q) + (N - 1) * w, rtol=1e-9)
    assert jp == pytest.approx(0.5 * (N - 1) * w @ w, rel=1e-15)


def test_envar_gradient_matches_central_differences():
    """Brute force: each g_i must agree with a central difference of the oracle's
    own observation cost along column i of E (forcings built here, not by the
    oracle's EnVar driver), to O(eps)."""
    P = oracle.cavity_params(32, 16, 300.0)
    N, eps, sigma, a = 3, 1e-2, 0.1, 0.05
    E = oracle.ensemble_seeded(P, sigma, a, N, 1000)
    u0, v0 = synth.cavity_ic(32, 16)
    w = np.array([0.3, -0.2, 0.1])
    n_steps, n_window = 120, 60
    for mode, key in ((oracle.COST_DOMAIN, "J_domain"), (oracle.COST_SENSORS, "J_sensor")):
        out = oracle.envar_gradient(P, u0, v0, E, w, eps, n_steps, n_window, cost_mode=mode, nthreads=4)

        def Jobs(f):
            fu, fv = oracle.control_to_faces(P, f)
            return oracle.member_run(P, u0, v0, n_steps, n_window, fu, fv)[key]

        f0 = E @ w
        assert out["J"][0] == pytest.approx(Jobs(f0), rel=1e-12)
        h = 1e-2
        gc = np.array([(Jobs(f0 + h * E[:, i]) - Jobs(f0 - h * E[:, i])) / (2 * h) for i in range(N)])
        gobs = out["g"] - (N - 1) * w
        assert np.abs(gobs - gc).max() <= 0.05 * np.abs(gc).max() + 1e-12, (mode, gobs, gc)
        # and its members are the N+1 forcings of Eq. (fdapprox)
        for i in range(N):
            assert out["J"][i + 1] == pytest.approx(Jobs(f0 + eps * E[:, i]), rel=1e-12)
        if mode == oracle.COST_SENSORS:
            # the explicit Y^T (Hq_0 - y) of Eq. (gradient_EnVar) on the sensor series
            ser = oracle.envar_gradient(P, u0, v0, E, w, eps, n_steps, n_window, cost_mode=mode, nthreads=4,
                                        want_series=True)["series"]
            gy = oracle.sensor_gradient(ser, w, eps) - (N - 1) * w
            assert np.abs(gy - gc).max() <= 0.05 * np.abs(gc).max() + 1e-12, (gy, gc)
            # forward differences of 1/2||h||^2 exceed Y^T h_0 by exactly eps/2 ||Y_i||^2 >= 0
            assert np.all(gobs - gy >= -1e-12 * np.abs(gy).max())


def test_domain_observation_vector_reproduces_the_domain_cost():
    """J_domain = 1/2 ||h|| ^2 for the observation vector h (Eq. kinenergy / n_w, R = I, y = 0),
    against the two-pass cost of orc_member_run; h is mean-free over the window in every cell."""
    P = oracle.cavity_params(32, 16, 300.0)
    u0, v0 = synth.cavity_ic(32, 16)
    h = oracle.domain_observation(P, u0, v0, 80, 30)
    J = oracle.member_run(P, u0, v0, 80, 30)["J_domain"]
    assert 0.5 * (h**2).sum() == pytest.approx(J, rel=1e-12)
    assert np.abs(h.sum(axis=0)).max() <= 1e-12 * np.abs(h).max()
    F = oracle.fluid_mask(P).astype(bool)
    assert np.all(h[:, ~F, :] == 0.0)


def _domain_case(advection):
    P = oracle.cavity_params(32, 16, 300.0, advection=advection)
    N, sigma, a = 3, 0.1, 0.05
    E = oracle.ensemble_seeded(P, sigma, a, N, 1000)
    u0, v0 = synth.cavity_ic(32, 16)
    w = np.array([0.3, -0.2, 0.1])
    return P, E, u0, v0, w, 100, 40


def test_domain_gradient_exact_for_linear_dynamics():
    """Stokes flow (no advection term): the velocity, hence h, is affine in the forcing, so Y of
    Eq. (fdapprox) is exact for any eps and Y^T h_0 equals the true gradient of J_obs = 1/2||h||^2.
    Central differences of a quadratic J are exact too, so all three agree to rounding, while the
    scalar form (J_i - J_0)/eps carries exactly the bias (eps/2)||Y_i||^2."""
    P, E, u0, v0, w, n_steps, n_window = _domain_case(0)
    N = E.shape[1]

    def Jobs(f):
        fu, fv = oracle.control_to_faces(P, f)
        return oracle.member_run(P, u0, v0, n_steps, n_window, fu, fv)["J_domain"]

    f0 = E @ w
    h = 0.05
    gc = np.array([(Jobs(f0 + h * E[:, i]) - Jobs(f0 - h * E[:, i])) / (2 * h) for i in range(N)])
    for eps in (1e-2, 1e-1):
        g, yy = oracle.envar_gradient_domain(P, u0, v0, E, w, eps, n_steps, n_window, nthreads=3)
        np.testing.assert_allclose(g - (N - 1) * w, gc, rtol=1e-7, atol=1e-9 * np.abs(gc).max())
        J = oracle.envar_gradient(P, u0, v0, E, w, eps, n_steps, n_window, nthreads=4)["J"]
        scalar = (J[1:] - J[0]) / eps
        np.testing.assert_allclose(scalar - (g - (N - 1) * w), 0.5 * eps * yy, rtol=1e-6)
        assert np.all(yy > 0)


def test_domain_gradient_identity_and_first_order_convergence():
    """Navier-Stokes: the identity (J_i - J_0)/eps = Y_i^T h_0 + (eps/2)||Y_i||^2 holds for the
    forward-difference Y (J from the independent two-pass cost), and Y^T h_0 converges to the
    central-difference gradient at first order in eps."""
    P, E, u0, v0, w, n_steps, n_window = _domain_case(1)
    N = E.shape[1]

    def Jobs(f):
        fu, fv = oracle.control_to_faces(P, f)
        return oracle.member_run(P, u0, v0, n_steps, n_window, fu, fv)["J_domain"]

    f0 = E @ w
    hc = 1e-3
    gc = np.array([(Jobs(f0 + hc * E[:, i]) - Jobs(f0 - hc * E[:, i])) / (2 * hc) for i in range(N)])
    errs = []
    for eps in (4e-2, 2e-2):
        g, yy = oracle.envar_gradient_domain(P, u0, v0, E, w, eps, n_steps, n_window, nthreads=3)
        J = oracle.envar_gradient(P, u0, v0, E, w, eps, n_steps, n_window, nthreads=4)["J"]
        gy = g - (N - 1) * w
        np.testing.assert_allclose((J[1:] - J[0]) / eps - gy, 0.5 * eps * yy, rtol=1e-6)
        errs.append(np.abs(gy - gc).max())
    assert errs[1] < 0.7 * errs[0], errs


def test_envar_step_update_and_total_cost():
    """Sec. 3.3.1 update with the prior-Hessian step: on the prior term alone (J_obs constant,
    g = (N-1) w) a unit step lands on its minimiser w = 0 and alpha = 1/2 halves w; the total cost
    is Eq. (J_w)."""
    rng = np.random.default_rng(11)
    N = 7
    w = rng.standard_normal(N)
    w1, J = oracle.envar_step(w, (N - 1) * w, 1.0, 0.25)
    np.testing.assert_array_equal(w1, np.zeros(N))
    assert J == pytest.approx(0.25 + 0.5 * (N - 1) * (w @ w), rel=1e-15)
    w2, _ = oracle.envar_step(w, (N - 1) * w, 0.5, 0.0)
    np.testing.assert_allclose(w2, 0.5 * w, rtol=1e-15)
    # a quadratic observation cost 1/2 c |w|^2 on top: the step moves along -g scaled by 1/(N-1)
    g = (N - 1 + 3.0) * w
    w3, _ = oracle.envar_step(w, g, 0.5, 0.0)
    np.testing.assert_allclose(w3, w * (1.0 - 0.5 * (N + 2) / (N - 1)), rtol=1e-14)


# --------------------------------------------------------------------------
# Eigenvector ensemble (Sec. 3.3.2, Eq. eigenvm1)
# --------------------------------------------------------------------------
def test_eigen_ensemble_separable_rectangle_reduces_to_1d_kernels():
    """A control region entirely in the open channel (no mask): B_s = sigma^2 K_x (x) K_y, so its
    eigenvalues are sigma^2 times products of the 1-D kernels' eigenvalues and its leading eigenvector
    is the Kronecker product of the 1-D leading eigenvectors (1-D kernels from the formula, 1-D
    eigenpairs from the library routine)."""
    P = oracle.cavity_params(64, 32, 1000.0)
    region = (-1.0, -0.4, 0.1, 0.5)
    sigma, a, N = 0.1, 0.1, 6
    E, lam = oracle.eigen_ensemble(P, sigma, a, N, region)
    ia, ib, ja, jb = oracle.control_rect(P, region)
    x = P.x0 + (np.arange(ia, ib + 1) + 0.5) * P.dx
    y = P.y0 + (np.arange(ja, jb + 1) + 0.5) * P.dy
    lx, Vx = np.linalg.eigh(np.exp(-(x[:, None] - x[None, :]) ** 2 / a**2))
    ly, Vy = np.linalg.eigh(np.exp(-(y[:, None] - y[None, :]) ** 2 / a**2))
    prods = np.sort(np.outer(ly, lx).ravel())[::-1] * sigma**2
    np.testing.assert_allclose(lam[::2], prods[:N // 2], rtol=1e-10)
    v1 = np.kron(Vy[:, -1], Vx[:, -1])            # row-major cells: y outer, x inner
    e1 = E[: len(v1), 0] / np.linalg.norm(E[: len(v1), 0])
    assert abs(abs(e1 @ v1) - 1.0) < 1e-10


def test_eigen_ensemble_invariants_on_the_cavity_region():
    """Eigen-equation residual against Eq. (covarianceB) evaluated here, orthogonality of the members,
    the scaling of Eq. (eigenvm1), and E E^T/(N-1) as the best rank-N approximation of B (its
    spectral-norm error is the next eigenvalue)."""
    P = oracle.cavity_params(64, 32, 1000.0)
    sigma, a, N = 0.1, 0.05, 8
    E, lam = oracle.eigen_ensemble(P, sigma, a, N)
    ci, cj = oracle.control_cells(P)
    xs, ys = P.x0 + (ci + 0.5) * P.dx, P.y0 + (cj + 0.5) * P.dy
    Bs = sigma**2 * np.exp(-((xs[:, None] - xs[None, :]) ** 2 + (ys[:, None] - ys[None, :]) ** 2) / a**2)
    n = len(ci)
    for k in range(N):
        comp = k % 2
        v = E[comp * n:(comp + 1) * n, k]
        assert np.all(E[(1 - comp) * n:(2 - comp) * n, k] == 0.0)
        assert np.linalg.norm(Bs @ v - lam[k] * v) <= 1e-10 * lam[0] * np.linalg.norm(v)
        assert np.linalg.norm(v) ** 2 == pytest.approx(lam[k] * (N - 1), rel=1e-12)
    G = E.T @ E
    assert np.abs(G - np.diag(np.diag(G))).max() <= 1e-12 * np.abs(G).max()
    assert np.all(np.diff(lam[::2]) <= 0)
    lam_all = np.sort(np.linalg.eigvalsh(Bs))[::-1]
    err = np.linalg.norm(Bs - E[:n, ::2] @ E[:n, ::2].T / (N - 1), 2)
    assert err == pytest.approx(lam_all[N // 2], rel=1e-8)


# --------------------------------------------------------------------------
# H^1 smoothing of the adjoint gradient (Sec. 4.2, Eq. lsob)
# --------------------------------------------------------------------------
def test_h1_smoothing_closed_forms():
    """On a control set that is a full rectangle, the no-flux Laplacian has the cosine eigenvectors
    cos(pi k (x - x_a)/L_x) cos(pi l (y - y_a)/L_y) sampled at the cell centres with eigenvalues
    -(4/dx^2) sin^2(pi k dx/(2 L_x)) - (4/dy^2) sin^2(pi l dy/(2 L_y)), so Eq. (lsob) scales such a
    mode by (1 + l^2)/(1 + l^2 |lambda|); a constant is scaled by 1 + l^2."""
    P = oracle.cavity_params(64, 32, 1000.0)
    region = (-1.0, -0.4, 0.1, 0.5)
    ci, cj = oracle.control_cells(P, region)
    ia, ib, ja, jb = oracle.control_rect(P, region)
    Lx, Ly = (ib - ia + 1) * P.dx, (jb - ja + 1) * P.dy
    xr, yr = (ci - ia + 0.5) * P.dx, (cj - ja + 0.5) * P.dy
    l = 0.02
    for k, m in ((0, 0), (1, 0), (2, 3)):
        mode = np.cos(np.pi * k * xr / Lx) * np.cos(np.pi * m * yr / Ly)
        lam = (4 / P.dx**2) * np.sin(np.pi * k * P.dx / (2 * Lx)) ** 2 + (4 / P.dy**2) * np.sin(np.pi * m * P.dy / (2 * Ly)) ** 2
        g = np.concatenate([mode, -2.0 * mode])
        gs = oracle.h1_smooth(P, g, l, region)
        np.testing.assert_allclose(gs, g * (1 + l * l) / (1 + l * l * lam), rtol=1e-10, atol=1e-12)


def test_h1_smoothing_operator_is_symmetric_and_smoothing():
    P = oracle.cavity_params(64, 32, 1000.0)
    n = len(oracle.control_cells(P)[0])
    rng = np.random.default_rng(8)
    a, b = rng.standard_normal(2 * n), rng.standard_normal(2 * n)
    Sa, Sb = oracle.h1_smooth(P, a, 0.02), oracle.h1_smooth(P, b, 0.02)
    assert abs(Sa @ b - a @ Sb) <= 1e-12 * np.linalg.norm(Sa) * np.linalg.norm(b)
    assert a @ Sa > 0
    # a rough field loses energy to the filter, a smooth one keeps it
    assert np.linalg.norm(Sa) < np.linalg.norm(a)


# --------------------------------------------------------------------------
# Reduced-space optimisers (Sec. 3.3.1, Eq. Hessian_EnVar, update_Newton, update_BFGS).
# --------------------------------------------------------------------------
def test_gauss_newton_is_exact_in_one_step_for_linear_dynamics():
    """Stokes flow and the sensor cost: h(w) is affine, so J(w) = 1/2||h0 + Y w||^2 + (N-1)/2 w^T w is
    quadratic with Hessian exactly Y^T Y + (N-1) I; one Gauss-Newton step lands on its minimiser, where
    the EnVar gradient (new forward runs at the new w) vanishes."""
    P = oracle.cavity_params(32, 16, 300.0, advection=0)
    N, sigma, a, eps = 3, 0.1, 0.05, 1e-2
    E = oracle.ensemble_seeded(P, sigma, a, N, 1000)
    u0, v0 = synth.cavity_ic(32, 16)
    n_steps, n_window = 80, 40
    w = np.array([0.3, -0.2, 0.1])
    out = oracle.envar_gradient(P, u0, v0, E, w, eps, n_steps, n_window, cost_mode=oracle.COST_SENSORS,
                                nthreads=4, want_series=True)
    Y, h0 = oracle.sensor_anomalies(out["series"], eps)
    w1, H, g = oracle.gauss_newton_step(Y, h0, w, 1.0)
    np.testing.assert_allclose(g, oracle.sensor_gradient(out["series"], w, eps), rtol=1e-12)
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-14 * np.abs(H).max())
    assert np.linalg.eigvalsh(H - (N - 1) * np.eye(N)).min() >= -1e-12 * np.abs(H).max()
    out1 = oracle.envar_gradient(P, u0, v0, E, w1, eps, n_steps, n_window, cost_mode=oracle.COST_SENSORS,
                                 nthreads=4, want_series=True)
    g1 = oracle.sensor_gradient(out1["series"], w1, eps)
    assert np.abs(g1).max() <= 1e-7 * np.abs(g).max(), (g1, g)
    # and the minimum is below the start (J = J_obs + J_prior of Eq. J_w)
    assert out1["J"][0] + out1["J_prior"] < out["J"][0] + out["J_prior"]


def test_gauss_newton_hessian_matches_dense_definition():
    rng = np.random.default_rng(21)
    N, nw = 5, 12
    series = rng.standard_normal((N + 1, nw, 8))
    eps = 0.1
    Y, h0 = oracle.sensor_anomalies(series, eps)
    h = series - series.mean(axis=1, keepdims=True)
    Yref = ((h[1:] - h[0]) / eps).reshape(N, -1)
    np.testing.assert_allclose(Y, Yref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(h0, h[0].reshape(-1), rtol=1e-13, atol=1e-14)
    w = rng.standard_normal(N)
    w1, H, g = oracle.gauss_newton_step(Y, h0, w, 0.5)
    Href = Yref @ Yref.T + (N - 1) * np.eye(N)
    np.testing.assert_allclose(H, Href, rtol=1e-12)
    np.testing.assert_allclose(w1, w - 0.5 * np.linalg.solve(Href, Yref @ h[0].reshape(-1) + (N - 1) * w),
                               rtol=1e-10)


def test_lbfgs_two_loop_equals_dense_bfgs_update():
    """The two-loop recursion reproduces the dense BFGS inverse update
    H+ = (I - rho s y^T) H (I - rho y s^T) + rho s s^T applied to gamma I, pair by pair."""
    rng = np.random.default_rng(5)
    N, m = 6, 4
    A = rng.standard_normal((N, N))
    A = A @ A.T + N * np.eye(N)
    S = rng.standard_normal((m, N))
    Yh = S @ A                       # curvature pairs of a convex quadratic: s^T y > 0
    g = rng.standard_normal(N)
    gamma = 0.37
    H = gamma * np.eye(N)
    for s, y in zip(S, Yh):
        rho = 1.0 / (y @ s)
        V = np.eye(N) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    np.testing.assert_allclose(oracle.lbfgs_direction(S, Yh, g, gamma), -H @ g, rtol=1e-11)
    # with no pairs the direction is steepest descent scaled by gamma
    np.testing.assert_allclose(oracle.lbfgs_direction(np.zeros((0, N)), np.zeros((0, N)), g, gamma), -gamma * g)


# --------------------------------------------------------------------------
# Costs (Sec. 4.1, Eq. specific_cost_function; Eq. kinenergy): closed forms.
# --------------------------------------------------------------------------
def test_costs_closed_form_on_stokes_decay():
    """With Stokes TG the window samples are a_t * (initial field), so both costs
    are known in closed form from the exact amplitude recurrence."""
    P = periodic_box(16, Re=5.0, dt=0.02, advection=0, origin=-math.pi)  # sensors (x, 0) interior
    u0, v0 = tg_fields(P)
    nu, dt = 1.0 / P.Re, P.dt
    lam = -(4 / P.dx**2) * math.sin(P.dx / 2) ** 2 - (4 / P.dy**2) * math.sin(P.dy / 2) ** 2
    a = [1.0, 1.0 + dt * nu * lam]
    n_steps, n_window = 30, 12
    for _ in range(n_steps):
        a.append(a[-1] + dt * nu * lam * (1.5 * a[-1] - 0.5 * a[-2]))
    at = np.array(a[n_steps - n_window + 1:n_steps + 1])
    var_sum = ((at - at.mean()) ** 2).sum()
    uc = 0.5 * (u0[:, :-1] + u0[:, 1:])
    vc = 0.5 * (v0[:-1, :] + v0[1:, :])
    Jd = P.dx * P.dy / (2 * n_window) * ((uc**2).sum() + (vc**2).sum()) * var_sum
    s = oracle.Sim(P)
    s.set_state(u0, v0)
    s0 = s.sensors()
    Js = 0.5 * (s0**2).sum() * var_sum
    out = oracle.member_run(P, u0, v0, n_steps, n_window, want_series=True)
    assert out["J_domain"] == pytest.approx(Jd, rel=1e-10)
    assert out["J_sensor"] == pytest.approx(Js, rel=1e-10)
    np.testing.assert_allclose(out["series"], at[:, None] * s0[None, :], atol=1e-14)


def test_sensors_exact_for_bilinear_field():
    P = oracle.cavity_params(64, 32, 1000.0)
    xu, yu, xv, yv = face_coords(P)
    u = 0.3 + 0.7 * xu[None, :] - 0.4 * yu[:, None]
    v = -0.2 + 0.5 * xv[None, :] + 0.9 * yv[:, None]
    s = oracle.Sim(P)
    s.set_state(u, v)
    got = s.sensors()
    for q in range(4):
        x = 0.2 * (q + 1)
        assert got[2 * q] == pytest.approx(0.3 + 0.7 * x, abs=1e-14)
        assert got[2 * q + 1] == pytest.approx(-0.2 + 0.5 * x, abs=1e-14)


# --------------------------------------------------------------------------
# Discrete adjoint (Sec. 3.2, Eq. adjoint_discrete / gradient_forcing): brute force.
# --------------------------------------------------------------------------
def test_adjoint_gradient_matches_central_differences():
    """The oracle's reverse sweep gives dJ/dF for the DOMAIN cost; directional derivatives along
    random face-forcing directions must equal central differences of the oracle's own cost."""
    P = oracle.cavity_params(32, 16, 300.0)
    u0, v0 = synth.cavity_ic(32, 16)
    rng = np.random.default_rng(0)
    s = oracle.Sim(P)
    uk, vk = s.face_kinds()
    fu = 0.05 * rng.standard_normal(uk.shape) * (uk == oracle.FK_UNKNOWN)
    fv = 0.05 * rng.standard_normal(vk.shape) * (vk == oracle.FK_UNKNOWN)
    n_steps, n_window = 60, 30
    J, gu, gv = oracle.adjoint_gradient(P, u0, v0, n_steps, n_window, fu, fv)
    # J is the same cost the forward two-pass evaluation reports
    assert J == pytest.approx(oracle.member_run(P, u0, v0, n_steps, n_window, fu, fv)["J_domain"], rel=1e-12)
    assert np.all(gu[uk != oracle.FK_UNKNOWN] == 0) and np.all(gv[vk != oracle.FK_UNKNOWN] == 0)
    h = 1e-4
    for _ in range(3):
        du = rng.standard_normal(uk.shape) * (uk == oracle.FK_UNKNOWN)
        dv = rng.standard_normal(vk.shape) * (vk == oracle.FK_UNKNOWN)
        Jp = oracle.adjoint_gradient(P, u0, v0, n_steps, n_window, fu + h * du, fv + h * dv)[0]
        Jm = oracle.adjoint_gradient(P, u0, v0, n_steps, n_window, fu - h * du, fv - h * dv)[0]
        fd = (Jp - Jm) / (2 * h)
        ad = (gu * du).sum() + (gv * dv).sum()
        assert abs(ad - fd) <= 1e-5 * abs(fd), (ad, fd)


def test_faces_to_control_is_transpose_of_control_to_faces():
    P = oracle.cavity_params(32, 16, 1000.0)
    rng = np.random.default_rng(1)
    n = len(oracle.control_cells(P)[0])
    f = rng.standard_normal(2 * n)
    s = oracle.Sim(P)
    uk, vk = s.face_kinds()
    gu = rng.standard_normal(uk.shape)
    gv = rng.standard_normal(vk.shape)
    fu, fv = oracle.control_to_faces(P, f)
    lhs = (fu * gu).sum() + (fv * gv).sum()
    rhs = f @ oracle.faces_to_control(P, gu, gv)
    assert lhs == pytest.approx(rhs, rel=1e-13)


# ----------------------------------------------------------------------------
# the paper's own flow configuration against its printed geometry (golden fixture)
# ----------------------------------------------------------------------------
def _table1():
    vals = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_table1_geometry.txt")
    for line in open(path):
        f = line.split("#")[0].split()
        if len(f) == 2:
            vals[f[0]] = float(f[1])
    return vals


def test_paper_workload_geometry_matches_table_1():
    """The paper workload (its Table 1, tests/golden/paper_table1_geometry.txt): the box
    [-L1, D + L2] x [-D, H], the no-slip part [-L1_slip, D + L2_slip] of the lower wall, and on that
    box the oracle's mask: every cell of the channel (y > 0) fluid, below it exactly the cavity
    0 < x < D, so the fluid area is (L1 + D + L2) H + D^2 on a grid whose faces meet the edges."""
    t = _table1()
    assert synth.PAPER_BOX == pytest.approx((-t["L1"], t["D"] + t["L2"], -t["D"], t["H"]), abs=1e-15)
    assert synth.PAPER_NOSLIP_SPAN == pytest.approx((-t["L1_slip"], t["D"] + t["L2_slip"]), abs=1e-15)
    nx, ny = 74, 30                        # dx = dy = 0.05
    P = oracle.cavity_params(nx, ny, 6250.0, box=synth.PAPER_BOX, inlet_delta=synth.PAPER_INLET_DELTA, lip_slip=1,
                             noslip_span=synth.PAPER_NOSLIP_SPAN)
    assert P.slip_lo == pytest.approx(-t["L1_slip"]) and P.slip_hi == pytest.approx(t["D"] + t["L2_slip"])
    F = oracle.fluid_mask(P).astype(bool)
    xc = P.x0 + (np.arange(nx) + 0.5) * P.dx
    yc = P.y0 + (np.arange(ny) + 0.5) * P.dy
    channel = yc > 0
    assert F[channel].all()
    cavity_cols = (xc > 0) & (xc < t["D"])
    assert np.array_equal(F[~channel], np.broadcast_to(cavity_cols, F[~channel].shape))
    area = F.sum() * P.dx * P.dy
    assert area == pytest.approx((t["L1"] + t["D"] + t["L2"]) * t["H"] + t["D"] ** 2, rel=1e-12)


# ----------------------------------------------------------------------------
# planted mistakes in the core arithmetic: each must make an independent pin fail
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("old,new,pin", [
    # sign of the advective cross term d(uv)/dy of the u equation
    ("A = (fe * fe - fw * fw) / dx + (un_c * vn_c - us_c * vs_c) / dy;",
     "A = (fe * fe - fw * fw) / dx - (un_c * vn_c - us_c * vs_c) / dy;",
     "test_manufactured_solution_second_order"),
    # the domain cost normalised by n_w + 1 window samples instead of n_w
    ("jd *= s->dx * s->dy / (2.0 * n_window);",
     "jd *= s->dx * s->dy / (2.0 * (n_window + 1));",
     "test_costs_closed_form_on_stokes_decay"),
    # the sensor cost without its factor 1/2
    ("        js *= 0.5;",
     "        js *= 1.0;",
     "test_costs_closed_form_on_stokes_decay"),
    # the prior term of Eq. (gradient_EnVar) with N instead of N - 1
    ("g[i] = (J[i + 1] - J[0]) / eps + (double)(N - 1) * w[i];",
     "g[i] = (J[i + 1] - J[0]) / eps + (double)N * w[i];",
     "test_gradient_quadratic_closed_form"),
    # the exact DOMAIN contraction against the perturbed observation instead of h_0
    ("            acc += yk * jb->h0[k];",
     "            acc += yk * hi[k];",
     "test_domain_gradient_exact_for_linear_dynamics"),
    # the Gauss-Newton Hessian with N I instead of (N - 1) I (Eq. Hessian_EnVar)
    ("            H[(size_t)i * N + j] = a + (i == j ? (double)(N - 1) : 0.0);",
     "            H[(size_t)i * N + j] = a + (i == j ? (double)N : 0.0);",
     "test_gauss_newton_is_exact_in_one_step_for_linear_dynamics"),
    # the L-BFGS second loop with the correction's sign flipped
    ("        for (int i = 0; i < N; ++i) q[i] += s[i] * (a[k] - b);",
     "        for (int i = 0; i < N; ++i) q[i] += s[i] * (b - a[k]);",
     "test_lbfgs_two_loop_equals_dense_bfgs_update"),
    # the sampler's convolution factor with the kernel's own width (not half of it)
    ("            G[(size_t)r * nxi + k] = c * exp(-2.0 * d * d / (a * a));",
     "            G[(size_t)r * nxi + k] = c * exp(-d * d / (a * a));",
     "test_sampler_factor_reproduces_gaussian_kernel"),
    # the adjoint of the advective cross term with its operands transposed
    ("                double bun = a * vn_c / dy, bvn = a * un_c / dy;",
     "                double bun = a * un_c / dy, bvn = a * vn_c / dy;",
     "test_adjoint_gradient_matches_central_differences"),
    # the pressure CG's residual update with the wrong sign
    ("        for (size_t k = 0; k < nc; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * q[k]; }",
     "        for (size_t k = 0; k < nc; ++k) { x[k] += alpha * p[k]; r[k] += alpha * q[k]; }",
     "test_poisson_solve_matches_dense_lstsq"),
    # the control forcing on u faces from one neighbouring cell instead of the two
    ("            fu[k] = 0.5 * (FX[(size_t)j * nx + il] + FX[(size_t)j * nx + ir]);",
     "            fu[k] = FX[(size_t)j * nx + ir];",
     "test_faces_to_control_is_transpose_of_control_to_faces"),
])
def test_core_pins_fail_on_planted_mistakes(tmp_path, old, new, pin):
    """Plant one plausible mistake in a copy of the oracle: the named pin, which does not restate
    the formula it checks, must fail on it."""
    if pin == "test_manufactured_solution_second_order":
        pytest.importorskip("sympy")
    with oracle.planted_mistake(old, new, str(tmp_path)):
        with pytest.raises(AssertionError):
            globals()[pin]()


class _planted_py:
    """Plant a mistake in one function of the oracle's Python layer: its source with one text
    replacement, compiled in a copy of the module's namespace, stands in for it inside the block."""

    def __init__(self, name, old, new):
        self.name, self.old, self.new = name, old, new

    def __enter__(self):
        import inspect
        import textwrap
        src = textwrap.dedent(inspect.getsource(getattr(oracle, self.name)))
        assert src.count(self.old) == 1, src.count(self.old)
        ns = dict(vars(oracle))
        exec(compile(src.replace(self.old, self.new), f"<planted {self.name}>", "exec"), ns)
        self.saved = getattr(oracle, self.name)
        setattr(oracle, self.name, ns[self.name])
        return self

    def __exit__(self, *exc):
        setattr(oracle, self.name, self.saved)
        return False


@pytest.mark.parametrize("name,old,new,pin", [
    # Eq. (lsob) without the (1 + l^2) normalisation of the right-hand side
    ("h1_smooth", "spla.spsolve(A, (1.0 + l_sob**2) * g[:n])", "spla.spsolve(A, g[:n])",
     "test_h1_smoothing_closed_forms"),
    # Eq. (eigenvm1) scaled by sqrt(N) instead of sqrt(N - 1)
    ("eigen_ensemble", "np.sqrt(max(lam[r], 0.0) * (N - 1)) * v", "np.sqrt(max(lam[r], 0.0) * N) * v",
     "test_eigen_ensemble_invariants_on_the_cavity_region"),
])
def test_python_layer_pins_fail_on_planted_mistakes(name, old, new, pin):
    with _planted_py(name, old, new):
        with pytest.raises(AssertionError):
            globals()[pin]()
