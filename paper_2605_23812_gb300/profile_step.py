"""Profiling driver: run time steps of the bench workload with the hot kernels in an NVTX range.

    python -m paper_2605_23812_gb300.profile_step [--steps 20] [--kernels 1,2]

Builds the library, autotunes the solver parameters as bench.py does (unless --no-autotune), runs
one forward evaluation of the 512x256 / Re 7500 / 33-member ensemble over --steps time steps to
warm up (graph capture), then a second one inside the NVTX range "timed" (for
ncu --nvtx --nvtx-include "timed/").  --kernels additionally launches the listed
hot kernels standalone (envar_time_kernel, one launch each) inside the range "kernels", for
targeted captures of a single launch.  --unrolled replaces the conditional refinement loop by the
unrolled one, whose kernel nodes a profiler can list one by one.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--members", type=int, default=32)
    ap.add_argument("--kernels", default="")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default solver parameters")
    ap.add_argument("--nu", type=int, default=0,
                    help="fix the smoothing sweep pairs (no autotuning: under a profiler the tuner's timings change)")
    ap.add_argument("--max-outer", type=int, default=0, help="with --nu: the refinement cap")
    ap.add_argument("--max-inner", type=int, default=0, help="with --nu: the inner-iteration cap")
    ap.add_argument("--coarse-sweeps", type=int, default=0, help="with --nu: coarse-level sweep pairs")
    ap.add_argument("--inner-rtol", type=float, default=0.0, help="with --nu: inner tolerance")
    ap.add_argument("--nu-coarse", type=int, default=0, help="with --nu: sweep pairs below the finest level")
    ap.add_argument("--unrolled", action="store_true",
                    help="capture the refinement loop unrolled instead of as a conditional graph node (ncu does "
                         "not profile the kernel nodes of graphs that hold conditional nodes); refinements past "
                         "convergence then launch and return at once")
    args = ap.parse_args()
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_23812_gb300 as pkg
    from paper_2605_23812_gb300 import synth
    cfg = pkg.default_config(512, 256, Re=7500.0, n_steps=args.steps, n_window=max(1, args.steps // 2),
                             n_members=args.members, precision=pkg.MIXED)
    if args.nu:
        cfg.nu_pre = cfg.nu_post = args.nu
        if args.max_outer:
            cfg.max_outer = args.max_outer
        if args.max_inner:
            cfg.max_inner = args.max_inner
        if args.coarse_sweeps:
            cfg.coarse_sweeps = args.coarse_sweeps
        if args.inner_rtol:
            cfg.inner_rtol = args.inner_rtol
        cfg.nu_coarse = args.nu_coarse
    if args.unrolled:
        cfg.conditional_refinement = 0
    ens = pkg.Ensemble(cfg, stream=torch.cuda.Stream())
    ens.set_initial_state(*synth.cavity_ic(512, 256))
    if not args.nu and not args.no_autotune:   # the solver parameters the bench uses
        with torch.cuda.stream(ens.stream):
            print("solver", ens.autotune(200))
    w = synth.weights(args.members)
    ens.forward_ensemble(w)
    torch.cuda.nvtx.range_push("timed")
    ens.forward_ensemble(w)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if args.kernels:
        torch.cuda.nvtx.range_push("kernels")
        for k in [int(x) for x in args.kernels.split(",")]:
            print(k, ens.time_kernel(k, 1))
        torch.cuda.nvtx.range_pop()
    print("diagnostics", ens.diagnostics())
    ens.close()


if __name__ == "__main__":
    main()
