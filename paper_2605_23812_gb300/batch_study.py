"""Throughput of the two large batched workloads, shortened: the uneven batch and the chaotic grid.

    python -m paper_2605_23812_gb300.batch_study [--scale 0.1] [--chaotic-steps 300]

Uneven batch: 96 member slots in three handles advancing together (one captured graph per chunk,
``envar_batch_*``): 32 slots at 256x128 / Re 4000 / 5000 steps, 48 at 512x256 / Re 7500 / 10 000
and 16 at 1024x512 / Re 15 000 / 20 000, every horizon multiplied by --scale; each handle's solver
parameters tuned by ``envar_autotune`` for its own grid.  Chaotic grid: 1024x512 / Re 15 000, 65
member slots (N = 64), mixed precision, tuned, --chaotic-steps steps.  Both in mixed precision from
the seeded initial state with the test weights; cost window the second half of each horizon.

One JSON line per workload: cell updates per second over the timed forward run (CUDA events on
the handles' stream, after one untimed forward run that captures the graphs), the chunking, the
solver choices and the largest divergence met.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=float, default=0.1)
    ap.add_argument("--chaotic-steps", type=int, default=300)
    args = ap.parse_args()
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_23812_gb300 as pkg
    from paper_2605_23812_gb300 import synth

    stream = torch.cuda.Stream()

    def handle(nx, ny, Re, steps, slots):
        cfg = pkg.default_config(nx, ny, Re=Re, n_steps=steps, n_window=steps // 2, n_members=slots - 1,
                                 precision=pkg.MIXED)
        ens = pkg.Ensemble(cfg, stream=stream)
        ens.set_initial_state(*synth.cavity_ic(nx, ny))
        with torch.cuda.stream(stream):
            solver = ens.autotune(200)
        return ens, solver

    def timed(fn):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    # uneven batch
    groups = [(256, 128, 4000.0, 5000, 32), (512, 256, 7500.0, 10000, 48), (1024, 512, 15000.0, 20000, 16)]
    hs, solvers, ws, work = [], [], [], 0.0
    for nx, ny, Re, steps, slots in groups:
        n = max(2, int(round(steps * args.scale)))
        e, sv = handle(nx, ny, Re, n, slots)
        hs.append(e)
        solvers.append(sv)
        ws.append(synth.weights(slots - 1, seed=len(hs)))
        work += float(nx) * ny * slots * n
    batch = pkg.Batch(hs, stream=stream)
    n_chunks, per = batch.info()
    t = timed(lambda: batch.forward(ws))
    print(json.dumps({"workload": "uneven batch (96 slots: 32 @ 256x128, 48 @ 512x256, 16 @ 1024x512)",
                      "horizon_scale": args.scale, "seconds": t, "cell_updates_per_s": work / t,
                      "chunks": n_chunks, "steps_per_chunk": [int(x) for x in per], "solvers": solvers,
                      "max_div": max(e.diagnostics()["max_div"] for e in hs),
                      "status_nonzero": int(sum((e.member_status() != 0).sum() for e in hs))}), flush=True)
    batch.close()
    for e in hs:
        e.close()

    # chaotic grid
    n = args.chaotic_steps
    e, sv = handle(1024, 512, 15000.0, n, 65)
    w = synth.weights(64)
    t = timed(lambda: e.forward_ensemble(w))
    print(json.dumps({"workload": "1024x512 Re 15000, 65 slots (N = 64)", "steps": n, "seconds": t,
                      "ms_per_step": 1e3 * t / n, "cell_updates_per_s": 1024.0 * 512 * 65 * n / t, "solver": sv,
                      "max_div": e.diagnostics()["max_div"],
                      "status_nonzero": int((e.member_status() != 0).sum())}), flush=True)
    e.close()


if __name__ == "__main__":
    main()
