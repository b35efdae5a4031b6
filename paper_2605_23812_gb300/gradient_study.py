"""Gradient accuracy of the batched mixed-precision EnVar estimate against the FP64 discrete adjoint.

    python -m paper_2605_23812_gb300.gradient_study [--nx 512 --ny 256 --Re 7500 --spinup 20000
                                                     --horizon 10000 --members 16,32,64,128,256
                                                     --snapshots 64 --fd-directions 16 --fd-step 0.01]

The open cavity is first spun up from the seeded initial state (mixed precision, no forcing); the
spun-up state is the initial state of every run below.  The cost is the DOMAIN fluctuation energy
over the whole horizon (Sec. 4.1), the forcing is zero (w = 0, the first EnVar iteration).

  * reference: dJ/df by the discrete adjoint of the FP64 stepper (Sec. 3.2) with binomial
    checkpointing;
  * the adjoint itself against central differences of the FP64 forward model in --fd-directions
    smooth random control directions d_k (normalised prior draws; one one-member FP64 run per point
    +h d_k and -h d_k);
  * EnVar: for each ensemble size N, the mixed-precision batched gradient of Eq. (gradient_EnVar) at
    w = 0, g = Y^T h_0 with Y from Eq. (fdapprox) (the explicit contraction), and for comparison the
    scalar-anomaly form (J_i - J_0)/eps, both estimates of E^T dJ/df.

Printed (one JSON line each): the adjoint's FD check, then per N the cosine and relative L2 error
between g and E^T dJ/df (the ensemble-space comparison: EnVar only sees the span of E), for both
forms, the cosine between the f-space directions E g / (N - 1) and dJ/df, and the times.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=256)
    ap.add_argument("--Re", type=float, default=7500.0)
    ap.add_argument("--spinup", type=int, default=20000)
    ap.add_argument("--horizon", type=int, default=10000)
    ap.add_argument("--members", default="16,32,64,128,256")
    ap.add_argument("--fd-directions", type=int, default=16)
    ap.add_argument("--fd-step", type=float, default=1e-2)
    ap.add_argument("--snapshots", type=int, default=64)
    ap.add_argument("--eps", type=float, default=1e-2)
    ap.add_argument("--fd-batched", default="",
                    help="also run the FD points as the members of one FP64 batched ensemble with these solver "
                         "settings, 'max_outer,max_inner,inner_rtol' (e.g. 20,30,1e-6 or 10,2,1e-3)")
    args = ap.parse_args()
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_23812_gb300 as pkg
    from paper_2605_23812_gb300 import synth

    nx, ny, T = args.nx, args.ny, args.horizon
    stream = torch.cuda.Stream()
    # spin-up (one member, mixed precision, no forcing)
    spin = pkg.Ensemble(pkg.default_config(nx, ny, Re=args.Re, n_steps=args.spinup, n_window=1, n_members=1,
                                           precision=pkg.MIXED, div_tol=1e-10), stream=stream)
    spin.set_initial_state(*synth.cavity_ic(nx, ny))
    spin.forward_ensemble(np.zeros(1))
    u0, v0, _ = spin.get_state(0)
    spin.close()

    # reference gradient: FP64 discrete adjoint
    # FP64 reference: generous solver caps, and a divergence target of 1e-9: the rounding floor of
    # the FP64 residual at 512x256 lies between 1e-10 and 3e-10, so over a 10k-step horizon a step
    # may stop above a tighter target, which would flag the run without changing the gradient
    adj = pkg.Ensemble(pkg.default_config(nx, ny, Re=args.Re, n_steps=T, n_window=T, n_members=1,
                                          precision=pkg.FP64_BATCHED, div_tol=1e-9, max_outer=20, max_inner=30,
                                          inner_rtol=1e-6), stream=stream)
    adj.set_initial_state(u0, v0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J_adj, g_adj = adj.adjoint_gradient(np.zeros(adj.n_ctrl), args.snapshots)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    g_adj = g_adj.cpu().numpy()
    stats = adj.adjoint_stats()
    adj.close()
    print(json.dumps({"adjoint": {"J": J_adj, "seconds": t_adj, "stats": stats, "snapshots": args.snapshots}}),
          flush=True)

    if args.fd_directions > 0:
        # central differences of the FP64 forward model along smooth random unit directions d_k
        # (normalised prior draws: the library's sampler, another seed), one member run per point
        # (+h d_k and -h d_k) on a one-member FP64 handle.  White-noise directions force grid-scale
        # modes that the central advection scheme at cell Reynolds numbers near 50 does not damp.
        K, hstep = args.fd_directions, args.fd_step
        draw = pkg.Ensemble(pkg.default_config(nx, ny, Re=args.Re, n_steps=2, n_window=1, n_members=K,
                                               precision=pkg.MIXED, seed=2024), stream=stream)
        D = draw.get_ensemble().cpu().numpy()[:, :K]
        draw.close()
        D /= np.linalg.norm(D, axis=0)
        fd = pkg.Ensemble(pkg.default_config(nx, ny, Re=args.Re, n_steps=T, n_window=T, n_members=0,
                                             precision=pkg.FP64_PLAIN, div_tol=1e-9), stream=stream)
        fd.set_initial_state(u0, v0)
        with torch.cuda.stream(stream):
            fd_solver = fd.autotune(200)
        t0 = time.perf_counter()
        Jp, Jm = [], []
        for k in range(K):
            Jp.append(fd.forward_control(hstep * D[:, k]))
            Jm.append(fd.forward_control(-hstep * D[:, k]))
        torch.cuda.synchronize()
        t_fd = time.perf_counter() - t0
        cfd = (np.array(Jp) - np.array(Jm)) / (2 * hstep)
        adj_dir = D.T @ g_adj
        print(json.dumps({"adjoint_fd_check": {
            "directions": K, "h": hstep, "path": "FP64, one member per run", "solver": fd_solver,
            "max_rel_err": float(np.abs(adj_dir - cfd).max() / np.abs(cfd).max()),
            "cos": float(adj_dir @ cfd / (np.linalg.norm(adj_dir) * np.linalg.norm(cfd))),
            "adjoint_directional": [float(x) for x in adj_dir], "central_differences": [float(x) for x in cfd],
            "seconds": t_fd}}), flush=True)
        fd.close()
        for spec in [x for x in args.fd_batched.split(";") if x]:
            mo, mi, rt = spec.split(",")
            cfg = pkg.default_config(nx, ny, Re=args.Re, n_steps=T, n_window=T, n_members=2 * K,
                                     precision=pkg.FP64_BATCHED, div_tol=1e-9, eps=hstep, max_outer=int(mo),
                                     max_inner=int(mi), inner_rtol=float(rt))
            fb = pkg.Ensemble(cfg, stream=stream)
            fb.set_initial_state(u0, v0)
            fb.set_ensemble(np.concatenate([D, -D], axis=1))
            t0 = time.perf_counter()
            fb.forward_ensemble(np.zeros(2 * K))
            torch.cuda.synchronize()
            tb = time.perf_counter() - t0
            Jb, _ = fb.cost()
            cb = (Jb[1:K + 1] - Jb[K + 1:]) / (2 * hstep)
            print(json.dumps({"fd_batched": {
                "settings": spec, "seconds": tb, "status": [int(x) for x in fb.member_status()],
                "max_div": fb.diagnostics()["max_div"],
                "max_rel_dev_from_one_member_runs": float(np.abs(cb - cfd).max() / np.abs(cfd).max())}}), flush=True)
            fb.close()

    for N in [int(x) for x in args.members.split(",")]:
        cfg = pkg.default_config(nx, ny, Re=args.Re, n_steps=T, n_window=T, n_members=N, precision=pkg.MIXED,
                                 div_tol=1e-10, eps=args.eps)
        ens = pkg.Ensemble(cfg, stream=stream)
        ens.set_initial_state(u0, v0)
        with torch.cuda.stream(stream):
            solver = ens.autotune(200)
        E = ens.get_ensemble().cpu().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens.forward_ensemble(np.zeros(N))
        g = ens.gradient()
        torch.cuda.synchronize()
        t_env = time.perf_counter() - t0
        gs = ens.gradient_scalar()
        J, _ = ens.cost()
        proj = E.T @ g_adj

        def cos(a, b):
            return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))

        df = E @ g / max(N - 1, 1)
        print(json.dumps({"grid": [nx, ny], "Re": args.Re, "horizon": T, "spinup": args.spinup, "N": N,
                          "eps": args.eps, "cos_ensemble_space": cos(g, proj),
                          "rel_l2_ensemble_space": float(np.linalg.norm(g - proj) / np.linalg.norm(proj)),
                          "cos_ensemble_space_scalar_form": cos(gs, proj),
                          "rel_l2_ensemble_space_scalar_form": float(np.linalg.norm(gs - proj) / np.linalg.norm(proj)),
                          "cos_control_space": cos(df, g_adj), "J0_envar": float(J[0]), "J_adjoint_fp64": J_adj,
                          "envar_gradient_s": t_env, "solver": solver,
                          "status_nonzero": int((ens.member_status() != 0).sum())}),
              flush=True)
        ens.close()


if __name__ == "__main__":
    main()
