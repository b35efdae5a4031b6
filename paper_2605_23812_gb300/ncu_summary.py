"""Summaries of ncu CSV logs (``ncu --csv --log-file``) as Markdown tables.

    python -m paper_2605_23812_gb300.ncu_summary launches <log.csv> [--real-us 6]
    python -m paper_2605_23812_gb300.ncu_summary metrics <log.csv>

``launches``: a launch list taken with ``--metrics gpu__time_duration.sum``: per kernel, its
launches, total time and share of the listed time, and the launches longer than --real-us
(microseconds).  With the refinement loop unrolled, refinements past a member group's convergence
still launch and return at once; the threshold separates those from launches that did work.

``metrics``: a capture of several metrics per launch: one row per launch with every metric.
"""
from __future__ import annotations

import argparse
import collections
import csv
import re

_SCALE_US = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3, "s": 1e6,
             "second": 1e6}


def _rows(path):
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    return list(csv.DictReader(lines))


def _short(name):
    name = re.sub(r"^void ", "", name)
    return re.sub(r"\(.*", "", name)


def _num(v):
    return float(v.replace(",", ""))


def launches(path, real_us):
    agg = collections.OrderedDict()
    total = 0.0
    n = 0
    for r in _rows(path):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        us = _num(r["Metric Value"]) * _SCALE_US[r["Metric Unit"]]
        a = agg.setdefault(_short(r["Kernel Name"]), [0, 0.0, 0, 0.0])
        a[0] += 1
        a[1] += us
        if us > real_us:
            a[2] += 1
            a[3] += us
        total += us
        n += 1
    print(f"{n} launches, {total / 1e3:.2f} ms listed (serialised, cold caches)\n")
    print(f"| kernel | launches | total ms | share | launches > {real_us:g} us | mean of those (us) |")
    print("|---|---|---|---|---|---|")
    for k, (cnt, t, nr, tr) in sorted(agg.items(), key=lambda x: -x[1][1]):
        mean = tr / nr if nr else 0.0
        print(f"| `{k}` | {cnt} | {t / 1e3:.2f} | {100 * t / total:.1f} % | {nr} | {mean:.1f} |")


def metrics(path):
    per = collections.OrderedDict()
    names = []
    for r in _rows(path):
        key = (r["ID"], _short(r["Kernel Name"]))
        m = r["Metric Name"]
        if m not in names:
            names.append(m)
        per.setdefault(key, {})[m] = (r["Metric Value"], r["Metric Unit"])
    for (lid, k), vals in per.items():
        print(f"### launch {lid}: `{k}`\n")
        print("| metric | value | unit |")
        print("|---|---|---|")
        for m in names:
            if m in vals:
                print(f"| {m} | {vals[m][0]} | {vals[m][1]} |")
        print()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["launches", "metrics"])
    ap.add_argument("csv")
    ap.add_argument("--real-us", type=float, default=6.0)
    a = ap.parse_args()
    if a.mode == "launches":
        launches(a.csv, a.real_us)
    else:
        metrics(a.csv)


if __name__ == "__main__":
    main()
