"""Flow regime and time-mean statistics of the unperturbed run, mixed precision against FP64.

    python -m paper_2605_23812_gb300.regime_study [--nx 1024 --ny 512 --Re 15000 --warmup 20000
                                                   --window 20000] [--paper-workload]

Runs the unperturbed member (w = 0, no forcing) of a workload once in the batched mixed-precision
path and once in the FP64 path, from the same seeded initial state, and prints one JSON line per
path and one comparison line:

  * the time-mean fluctuation energy J = 1/(2 n_w) sum_t sum_cells |u - mean u|^2 dx dy over the
    window (the DOMAIN cost, Eq. kinenergy normalised by the window length);
  * the sensor series of Sec. 4.1 over the window: rms of the fluctuation of each channel, the
    dominant angular frequency of their summed power spectrum (Hann window) and its strongest
    local peaks (the paper reports, for its uncontrolled flow at Re 6250, a dominant oscillation at
    omega = 11.31 and a lower component at omega = 2.49, Sec. 4.3);
  * the relative difference of J between the two paths (the statistics tolerance of a chaotic
    regime is 2 %: there, trajectories separate and only such statistics are comparable).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def spectrum(series, dt, npeaks=4):
    import numpy as np
    s = np.asarray(series, dtype=np.float64)
    f = s - s.mean(axis=0)
    n = f.shape[0]
    spec = (np.abs(np.fft.rfft(f * np.hanning(n)[:, None], axis=0)) ** 2).sum(axis=1)
    spec[0] = 0.0
    k = int(np.argmax(spec))
    dw = 2.0 * np.pi / (n * dt)
    # local maxima of the summed power spectrum, strongest first, each refined by a parabola
    # through its bin and the two neighbours (in log power)
    peaks = []
    for b in range(1, len(spec) - 1):
        if spec[b] > spec[b - 1] and spec[b] >= spec[b + 1] and spec[b] > 0:
            a, c = np.log(max(spec[b - 1], 1e-300)), np.log(max(spec[b + 1], 1e-300))
            m = np.log(spec[b])
            den = a - 2.0 * m + c
            off = 0.5 * (a - c) / den if den < 0 else 0.0
            peaks.append((float(spec[b]), (b + off) * dw))
    peaks.sort(reverse=True)
    tot = float(spec.sum())
    return {"sensor_rms": [float(x) for x in np.sqrt((f ** 2).mean(axis=0))],
            "dominant_omega": k * dw, "omega_resolution": dw,
            "peak_power_fraction": float(spec[k] / tot) if tot > 0 else None,
            "peaks": [{"omega": w, "power_fraction": p / tot} for p, w in peaks[:npeaks]] if tot > 0 else []}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--Re", type=float, default=15000.0)
    ap.add_argument("--warmup", type=int, default=20000)
    ap.add_argument("--window", type=int, default=20000)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--paper-workload", action="store_true",
                    help="the paper's own configuration (Sec. 4.1): box [-1.2, 2.5] x [-1, 0.5] (channel height "
                         "0.5), uniform inflow, free-slip lower wall outside [-0.4, 1.75]")
    args = ap.parse_args()
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_23812_gb300 as pkg
    from paper_2605_23812_gb300 import synth

    nx, ny = args.nx, args.ny
    n = args.warmup + args.window
    geo, ic = {}, {}
    if args.paper_workload:
        box = synth.PAPER_BOX
        geo = dict(x0=box[0], x1=box[1], y0=box[2], y1=box[3], inlet_delta=synth.PAPER_INLET_DELTA, lip_slip=1,
                   noslip_span=synth.PAPER_NOSLIP_SPAN)
        ic = dict(box=box, delta=synth.PAPER_INLET_DELTA)
    res = {}
    paths = [("mixed", pkg.MIXED, dict(div_tol=1e-10))]
    if not args.skip_fp64:
        paths.append(("fp64", pkg.FP64_PLAIN, dict(div_tol=1e-9, max_outer=12, max_inner=8, inner_rtol=1e-4)))
    for name, prec, kw in paths:
        cfg = pkg.default_config(nx, ny, Re=args.Re, n_steps=n, n_window=args.window, n_members=0, precision=prec,
                                 **kw, **geo)
        stream = torch.cuda.Stream()
        ens = pkg.Ensemble(cfg, stream=stream)
        ens.set_initial_state(*synth.cavity_ic(nx, ny, **ic))
        if prec == pkg.MIXED:
            with torch.cuda.stream(stream):
                ens.autotune(200)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ens.forward_ensemble(np.zeros(0))
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        J, _ = ens.cost()
        line = {"path": name, "workload": "paper" if args.paper_workload else "cavity", "grid": [nx, ny],
                "Re": args.Re, "warmup": args.warmup, "window": args.window,
                "dt": ens.dt, "J_time_mean_energy": float(J[0]), "seconds": el,
                "status": int(ens.member_status()[0]), "max_div": ens.diagnostics()["max_div"]}
        line.update(spectrum(ens.get_series(0), ens.dt))
        print(json.dumps(line), flush=True)
        res[name] = line
        ens.close()
    if "fp64" in res:
        print(json.dumps({"compare": "mixed vs fp64",
                          "J_rel_diff": res["mixed"]["J_time_mean_energy"] / res["fp64"]["J_time_mean_energy"] - 1.0,
                          "omega_mixed": res["mixed"]["dominant_omega"], "omega_fp64": res["fp64"]["dominant_omega"]}),
              flush=True)


if __name__ == "__main__":
    main()
