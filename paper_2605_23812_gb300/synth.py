"""Seeded synthetic inputs for the open-cavity ensemble workload.

This module holds input data only -- none of the method's arithmetic.  Both the
CUDA path (through the C-ABI) and the CPU oracle take these arrays as inputs.

* ``cavity_ic``: raw initial velocity fields on every face of the MAC grid: the
  inlet-like profile erf(y/delta) above the cavity lip (zero below), plus seeded
  Gaussian noise of the given amplitude.  Each solver applies its own boundary
  rules (walls, inlet, outlet) when it loads them.
* ``weights``: seeded ensemble weights w (the reduced control vector).
* ``PAPER_BOX``, ``PAPER_NOSLIP_SPAN``, ``PAPER_INLET_DELTA``: the paper's own flow configuration
  (its Table 1 geometry: the box [-L1, D + L2] x [-D, H], the no-slip part [-L1_slip, D + L2_slip]
  of the lower wall, and a uniform inflow written as an erf profile of negligible width).
"""
from __future__ import annotations

import math

import numpy as np

CAVITY_BOX = (-1.2, 2.5, -1.0, 1.0)
PAPER_BOX = (-1.2, 2.5, -1.0, 0.5)
PAPER_NOSLIP_SPAN = (-0.4, 1.75)
PAPER_INLET_DELTA = 1e-6          # erf(y / delta) = 1 on every fluid row: uniform inflow


def cavity_ic(nx: int, ny: int, box=CAVITY_BOX, seed: int = 1234, noise: float = 1e-3,
              delta: float = 0.1):
    """Return (u0, v0): u0 has shape (ny, nx+1), v0 has shape (ny+1, nx), float64."""
    x0, x1, y0, y1 = box
    dy = (y1 - y0) / ny
    yc = y0 + (np.arange(ny) + 0.5) * dy
    prof = np.array([math.erf(y / delta) if y > 0.0 else 0.0 for y in yc])
    rng = np.random.default_rng(seed)
    u0 = prof[:, None] + noise * rng.standard_normal((ny, nx + 1))
    v0 = noise * rng.standard_normal((ny + 1, nx))
    return np.ascontiguousarray(u0), np.ascontiguousarray(v0)


def weights(N: int, seed: int = 7, scale: float = 0.1) -> np.ndarray:
    """Seeded ensemble weights w in R^N."""
    return scale * np.random.default_rng(seed).standard_normal(N)
