"""The paper's own flow configuration as far as this MAC solver can state it (Sec. 4.1, Sec. 4.4,
Table 1): channel height H = 0.5 above a cavity of depth 1, uniform inflow, free slip on the lower
wall outside the no-slip span [-0.4, 1.75], forcing in the y-momentum equation only, the sensor cost,
Re = 6250.  The GPU (FP64) against the oracle: trajectories, the ensemble, and the discrete adjoint
with the slip rule transposed.  (The outlet stays convective: a traction-free outlet would make the
pressure Dirichlet there, a non-singular Poisson problem the solver does not handle.)
"""
import numpy as np
import pytest

import oracle
import paper_2605_23812_gb300 as pkg
from paper_2605_23812_gb300 import synth

pytestmark = pytest.mark.gpu

BOX = synth.PAPER_BOX
DELTA = synth.PAPER_INLET_DELTA
SPAN = synth.PAPER_NOSLIP_SPAN


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def paper_cfg(nx, ny, **kw):
    base = dict(x0=BOX[0], x1=BOX[1], y0=BOX[2], y1=BOX[3], Re=6250.0, inlet_delta=DELTA, lip_slip=1,
                noslip_span=SPAN, forcing_y_only=1, cost_mode=pkg.COST_SENSORS, precision=pkg.FP64_BATCHED,
                div_tol=1e-12, max_outer=4, max_inner=40, inner_rtol=1e-12)
    base.update(kw)
    return pkg.default_config(nx, ny, **base)


def paper_params(nx, ny):
    return oracle.cavity_params(nx, ny, 6250.0, box=BOX, inlet_delta=DELTA, lip_slip=1, noslip_span=SPAN)


def test_paper_workload_trajectories_and_ensemble():
    nx, ny, N, steps = 64, 24, 4, 100
    cfg = paper_cfg(nx, ny, n_steps=steps, n_window=40, n_members=N)
    P = paper_params(nx, ny)
    u0, v0 = synth.cavity_ic(nx, ny, box=BOX, delta=DELTA)
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(u0, v0)
    E = ens.get_ensemble().cpu().numpy()
    Eo = oracle.ensemble_seeded(P, cfg.sigma, cfg.corr_len, N, cfg.seed)
    ncc = E.shape[0] // 2
    assert np.all(E[:ncc] == 0.0)                                   # y-momentum forcing only
    np.testing.assert_allclose(E[ncc:], Eo[ncc:], rtol=0, atol=1e-12 * np.abs(Eo).max())
    w = synth.weights(N)
    ens.forward_ensemble(w)
    Ez = Eo.copy()
    Ez[:ncc] = 0.0
    for m in (0, N):
        f = Ez @ w + (cfg.eps * Ez[:, m - 1] if m else 0.0)
        fu, fv = oracle.control_to_faces(P, f)
        ou, ov, _, _, _ = oracle.trajectory(P, u0, v0, steps, fu, fv)
        u, v, _ = (t.cpu().numpy() for t in ens.get_state(m))
        err = np.sqrt((((u - ou) ** 2).sum() + ((v - ov) ** 2).sum()) / ((ou**2).sum() + (ov**2).sum()))
        assert err <= 1e-10, (m, err)
    assert (ens.member_status() == 0).all()
    # the slip segments change the flow: the no-slip run differs
    ref_noslip = oracle.trajectory(oracle.cavity_params(nx, ny, 6250.0, box=BOX, inlet_delta=DELTA), u0, v0, steps)
    u, v, _ = (t.cpu().numpy() for t in ens.get_state(0))
    f0 = Ez @ w
    fu, fv = oracle.control_to_faces(P, f0)
    ou, ov, _, _, _ = oracle.trajectory(P, u0, v0, steps, fu, fv)
    assert np.abs(ref_noslip[0] - ou).max() > 1e-3
    ens.close()


def test_paper_workload_adjoint_transposes_the_slip_rule():
    nx, ny, n, nw = 32, 12, 40, 20
    cfg = paper_cfg(nx, ny, n_steps=n, n_window=nw, n_members=2, cost_mode=pkg.COST_DOMAIN)
    P = paper_params(nx, ny)
    u0, v0 = synth.cavity_ic(nx, ny, box=BOX, delta=DELTA)
    Eo = oracle.ensemble_seeded(P, cfg.sigma, cfg.corr_len, 2, cfg.seed)
    f = Eo @ np.array([0.8, -0.5])
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(u0, v0)
    J, g = ens.adjoint_gradient(f, 8)
    g = g.cpu().numpy()
    ens.close()
    fu, fv = oracle.control_to_faces(P, f)
    Jo, gu, gv = oracle.adjoint_gradient(P, u0, v0, n, nw, fu, fv)
    go = oracle.faces_to_control(P, gu, gv)
    assert abs(J - Jo) <= 1e-9 * abs(Jo)
    assert np.linalg.norm(g - go) <= 1e-8 * np.linalg.norm(go)


def test_paper_workload_gauss_newton_reduces_the_sensor_cost():
    nx, ny, N = 64, 24, 6
    cfg = paper_cfg(nx, ny, n_steps=120, n_window=60, n_members=N)
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(*synth.cavity_ic(nx, ny, box=BOX, delta=DELTA))
    ens.use_eigen_ensemble()
    w = np.zeros(N)
    Js = []
    for _ in range(2):
        w, J0 = ens.gn_step(1.0, w)
        Js.append(J0)
    ens.forward_ensemble(w)
    J, jp = ens.cost()
    assert J[0] + jp < Js[0]
    ens.close()
