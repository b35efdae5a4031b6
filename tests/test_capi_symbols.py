"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/envar.h declares (no compute calls: this runs without a GPU)."""
import ctypes

import pytest

from paper_2605_23812_gb300 import build as pkg_build
from paper_2605_23812_gb300 import capi


@pytest.fixture(scope="module")
def so():
    path = pkg_build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(so):
    names = capi.header_symbols()
    assert len(names) >= 18
    for n in names:
        assert hasattr(so, n), n


def test_config_struct_matches_header(so):
    # envar_default_config runs on the host only
    c = capi.default_config(128, 64)
    assert (c.nx, c.ny) == (128, 64)
    assert c.x0 == -1.2 and c.x1 == 2.5 and c.y0 == -1.0 and c.y1 == 1.0
    assert list(c.region) == [-0.5, 1.0, -0.2, 0.3]
    assert c.steps_per_graph == 10 and c.nu_pre == 2 and c.coarse_sweeps == 8
    assert ctypes.sizeof(capi.Config) == 8 * ((ctypes.sizeof(capi.Config) + 7) // 8)
    # the trailing fields, whose offsets depend on every field before them
    assert c.lip_slip == 0 and list(c.noslip_span) == [-0.4, 1.75] and c.forcing_y_only == 0
    assert c.conditional_refinement == 1 and c.guess_extrapolation == 1 and c.nu_coarse == 0


def test_config_struct_is_not_shorter_than_the_c_one(so):
    """envar_default_config clears and fills sizeof(envar_config) bytes: run it on a buffer with a
    sentinel region after the Python structure; a C structure with fields the binding lacks would
    write into the sentinel."""
    n = ctypes.sizeof(capi.Config)
    buf = (ctypes.c_ubyte * (n + 256))(*([0xA5] * (n + 256)))
    assert so.envar_default_config(ctypes.cast(buf, ctypes.c_void_p), 64, 32) == 0
    assert all(b == 0xA5 for b in bytes(buf)[n:])
    c = capi.Config.from_buffer_copy(bytes(buf)[:n])
    assert (c.nx, c.ny, c.nu_coarse, c.guess_extrapolation) == (64, 32, 0, 1)


def test_init_without_device_fails_cleanly(so):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    c = capi.default_config(32, 16)
    rc = capi.lib().envar_init(ctypes.byref(h), ctypes.byref(c), None)
    assert rc == -5 and not h.value
    assert b"device" in capi.lib().envar_last_error(None)
