"""Host-side tools whose output the profiles quote: the regime study's spectrum and peak finder,
and the ncu CSV summariser (no GPU)."""
import io
import contextlib

import numpy as np
import pytest

from paper_2605_23812_gb300 import ncu_summary, regime_study


def test_spectrum_finds_the_two_frequencies_of_a_quasi_periodic_signal():
    """Two incommensurate sinusoids (the paper's omega = 11.31 and 2.49 at unequal amplitudes) plus
    noise on eight channels: the strongest peaks come back at both frequencies, refined well below
    the bin width, in the order of their power."""
    dt, n = 0.002, 40000
    t = np.arange(n) * dt
    rng = np.random.default_rng(5)
    chans = [np.sin(11.31 * t + k) + 0.4 * np.sin(2.49 * t + 2 * k) + 0.05 * rng.standard_normal(n) for k in range(8)]
    r = regime_study.spectrum(np.stack(chans, axis=1), dt)
    dw = 2 * np.pi / (n * dt)
    assert r["omega_resolution"] == pytest.approx(dw)
    w = [p["omega"] for p in r["peaks"]]
    assert abs(w[0] - 11.31) < 0.1 * dw and abs(w[1] - 2.49) < 0.1 * dw
    assert r["peaks"][0]["power_fraction"] > r["peaks"][1]["power_fraction"] > 0.05
    assert abs(r["dominant_omega"] - 11.31) <= dw


def test_spectrum_of_a_constant_signal_has_no_peaks():
    r = regime_study.spectrum(np.ones((1000, 8)), 0.01)
    assert r["peaks"] == [] and r["peak_power_fraction"] is None


CSV = '''==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","p","h","void k_a<float>(int)","1","13","(128, 1, 1)","(8, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ns","10,000"
"1","1","p","h","void k_b(int)","1","13","(128, 1, 1)","(8, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","2.5"
"2","1","p","h","void k_a<float>(int)","1","13","(128, 1, 1)","(8, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ns","30000"
'''


def test_launch_summary_aggregates_per_kernel(tmp_path):
    """Units (ns with a thousands separator, us), per-kernel totals and shares, and the split of
    launches above the threshold."""
    p = tmp_path / "l.csv"
    p.write_text(CSV)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        ncu_summary.launches(str(p), 6.0)
    text = out.getvalue()
    assert "3 launches, 0.04 ms listed" in text
    rows = [ln for ln in text.splitlines() if ln.startswith("| `")]
    assert rows[0].startswith("| `k_a<float>` | 2 | 0.04 | 94.1 % | 2 | 20.0 |")
    assert rows[1].startswith("| `k_b` | 1 | 0.00 | 5.9 % | 0 | 0.0 |")
