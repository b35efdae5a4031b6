"""The allocation-free ensemble draw (envar_draw_ensemble_noalloc) against the handle path.

Callers that cannot let a library call cudaMalloc (a framework whose caching allocator owns the
device, a fixed memory budget) draw the ensemble straight into their own buffer; the draw uses a
fixed-size static device scratch array instead of allocating.  It must give the same E as
envar_init + envar_get_ensemble, on every call (the scratch keeps the previous call's contents).
This file is collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import paper_2605_23812_gb300 as pkg
from paper_2605_23812_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def draw_noalloc(cfg, n_ctrl):
    import torch
    out = torch.full((cfg.n_members, n_ctrl), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = capi.lib().envar_draw_ensemble_noalloc(ctypes.byref(cfg), ctypes.c_void_p(out.data_ptr()), n_ctrl, None)
    assert rc == 0, capi.lib().envar_last_error(None)
    return out.cpu().numpy().T     # n_ctrl x N


@pytest.mark.parametrize("nx,ny,N", [(128, 64, 8), (512, 256, 32)])
def test_noalloc_draw_equals_handle_draw_on_consecutive_calls(nx, ny, N):
    cfg = pkg.default_config(nx, ny, n_members=N, n_steps=2, n_window=1)
    ens = pkg.Ensemble(cfg)
    ref = ens.get_ensemble().cpu().numpy()
    n_ctrl = ens.n_ctrl
    ens.close()
    for _ in range(2):
        E = draw_noalloc(cfg, n_ctrl)
        assert np.isfinite(E).all()
        np.testing.assert_allclose(E, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_noalloc_rejects_oversized_configurations():
    import torch
    cfg = pkg.default_config(4096, 2048, n_members=2, n_steps=2, n_window=1)
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = capi.lib().envar_draw_ensemble_noalloc(ctypes.byref(cfg), ctypes.c_void_p(out.data_ptr()), 0, None)
    assert rc != 0
    msg = capi.lib().envar_last_error(None).decode()
    assert "envar_draw_ensemble_noalloc" in msg and "scratch" in msg
