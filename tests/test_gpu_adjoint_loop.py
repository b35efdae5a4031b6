"""The adjoint approach of Sec. 3.2 with the H^1 regularisation of Sec. 4.2 on the GPU, against the
oracle: the smoothing of Eq. (lsob) and two L-BFGS iterations in control space, which the oracle
replays with its own discrete adjoint, its sparse H^1 solve, its two-loop recursion and its own
Armijo cost evaluations (FP64; the two adjoints agree to 1e-8, so the iterates are compared at 1e-6).
"""
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


@pytest.mark.parametrize("nx,ny", [(128, 64), (512, 256)])
def test_h1_smoothing_matches_oracle(nx, ny):
    cfg = pkg.default_config(nx, ny, n_members=2, n_steps=2, n_window=1, precision=pkg.FP64_BATCHED)
    ens = pkg.Ensemble(cfg)
    rng = np.random.default_rng(3)
    g = rng.standard_normal(ens.n_ctrl)
    gs = ens.h1_smooth(g, 0.02).cpu().numpy()
    ens.close()
    ref = oracle.h1_smooth(oracle.cavity_params(nx, ny, cfg.Re), g, 0.02)
    np.testing.assert_allclose(gs, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_adjoint_lbfgs_iterations_match_oracle():
    import torch
    nx, ny, n, nw, l_sob, step0 = 32, 16, 60, 30, 0.02, 2e-2
    cfg = pkg.default_config(nx, ny, Re=300.0, n_steps=n, n_window=nw, n_members=1, precision=pkg.FP64_BATCHED,
                             div_tol=1e-12, max_outer=4, max_inner=40, inner_rtol=1e-12)
    u0, v0 = synth.cavity_ic(nx, ny)
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(u0, v0)
    f = torch.zeros(ens.n_ctrl, dtype=torch.float64, device="cuda")
    f_gpu, J_gpu = [], []
    for _ in range(2):
        J, a, ev = ens.adjoint_lbfgs_step(f, 16, l_sob, step0)
        f_gpu.append(f.cpu().numpy().copy())
        J_gpu.append(J)
    ens.close()

    P = oracle.cavity_params(nx, ny, 300.0)
    dA = P.dx * P.dy

    def J_and_grad(fc):
        fu, fv = oracle.control_to_faces(P, fc)
        J, gu, gv = oracle.adjoint_gradient(P, u0, v0, n, nw, fu, fv)
        return J, oracle.faces_to_control(P, gu, gv)

    def J_only(fc):
        fu, fv = oracle.control_to_faces(P, fc)
        return oracle.member_run(P, u0, v0, n, nw, fu, fv)["J_domain"]

    fk = np.zeros(f_gpu[0].size)
    S, Yh, prev = [], [], None
    for k in range(2):
        J, g = J_and_grad(fk)
        assert J == pytest.approx(J_gpu[k], rel=1e-10)
        gs = oracle.h1_smooth(P, g / dA, l_sob)
        if prev is not None:
            s, y = fk - prev[0], gs - prev[1]
            if s @ y > 1e-10 * np.linalg.norm(s) * np.linalg.norm(y):
                S.append(s)
                Yh.append(y)
        gamma = (S[-1] @ Yh[-1]) / (Yh[-1] @ Yh[-1]) if S else 1.0
        p = oracle.lbfgs_direction(np.array(S).reshape(-1, len(fk)), np.array(Yh).reshape(-1, len(fk)), gs, gamma)
        slope = g @ p
        assert slope < 0
        a = step0 / np.abs(p).max() if not S else 1.0
        for _ in range(12):
            Jt = J_only(fk + a * p)
            if Jt <= J + 1e-4 * a * slope:
                break
            a *= 0.5
        prev = (fk, gs)
        fk = fk + a * p
        np.testing.assert_allclose(f_gpu[k], fk, rtol=1e-6, atol=1e-9 * np.abs(fk).max())
    assert J_only(fk) < J_gpu[0]
