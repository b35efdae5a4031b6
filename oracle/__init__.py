"""FP64 CPU oracle for the EnVar open-cavity hot path (arXiv 2605.23812).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product package ``paper_2605_23812_gb300`` never imports it, and the
two share no code: the oracle is a separate plain-C library (``ns2d_oracle.c``)
compiled with gcc, wrapped here with ctypes.

Every function cites the passage of the paper it follows; see ``ns2d_oracle.c``
for the discretisation readings.  Pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ns2d_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_ns2d.so")
_lock = threading.Lock()
_lib = None

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")

COST_DOMAIN, COST_SENSORS = 0, 1
#: control region of the synthetic open-cavity workload, [x0, x1, y0, y1]
CAVITY_REGION = (-0.5, 1.0, -0.2, 0.3)
#: box of the synthetic open-cavity workload
CAVITY_BOX = (-1.2, 2.5, -1.0, 1.0)


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", c_int), ("ny", c_int),
        ("x0", c_double), ("x1", c_double), ("y0", c_double), ("y1", c_double),
        ("Re", c_double), ("dt", c_double),
        ("bc_x", c_int), ("bc_y", c_int), ("geometry", c_int), ("advection", c_int),
        ("inlet_delta", c_double), ("conv_speed", c_double),
        ("cg_rtol", c_double), ("cg_maxit", c_int),
        ("ch_lo", c_double), ("ch_hi", c_double),
        ("lip_slip", c_int), ("slip_lo", c_double), ("slip_hi", c_double),
    ]

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + pthreads, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                   "-o", tmp, _SRC, "-lm", "-lpthread"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _configure(L):
    """Declare the argument and result types of every exported oracle function on a loaded library."""
    P = ctypes.POINTER(Params)
    sig = {
        "orc_version": (c_int, []),
        "orc_fluid_mask": (None, [P, _u8p]),
        "orc_create": (c_void_p, [P]),
        "orc_destroy": (None, [c_void_p]),
        "orc_set_state": (None, [c_void_p, _dp, _dp, c_void_p]),
        "orc_get_state": (None, [c_void_p, _dp, _dp, _dp]),
        "orc_set_face_forcing": (None, [c_void_p, _dp, _dp]),
        "orc_step": (c_int, [c_void_p, c_int]),
        "orc_max_div": (c_double, [c_void_p]),
        "orc_last_cg_relres": (c_double, [c_void_p]),
        "orc_last_cg_iters": (c_int, [c_void_p]),
        "orc_fluxes": (None, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
        "orc_face_kinds": (None, [c_void_p, _u8p, _u8p]),
        "orc_project": (None, [c_void_p, _dp, _dp]),
        "orc_apply_negL": (None, [c_void_p, _dp, _dp]),
        "orc_poisson_solve": (c_int, [c_void_p, _dp, _dp]),
        "orc_explicit_rhs": (None, [c_void_p, _dp, _dp]),
        "orc_control_rect": (c_int, [P, _dp, _i32p]),
        "orc_control_cells": (c_int, [P, _dp, c_void_p, c_void_p]),
        "orc_control_to_faces": (None, [P, _dp, _dp, _dp, _dp]),
        "orc_philox4x64_10": (None, [_u64p, _u64p, _u64p]),
        "orc_normals": (None, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, _dp]),
        "orc_sampler_dims": (c_int, [P, _dp, c_double, _i32p]),
        "orc_sampler_factors": (c_int, [P, _dp, c_double, _dp, _dp]),
        "orc_ensemble_from_noise": (c_int, [P, _dp, c_double, c_double, c_int, _dp, _dp]),
        "orc_ensemble_seeded": (c_int, [P, _dp, c_double, c_double, c_int, ctypes.c_uint64, _dp]),
        "orc_sensors": (None, [c_void_p, _dp]),
        "orc_member_run": (c_int, [P, _dp, _dp, _dp, _dp, c_int, c_int,
                                   ctypes.POINTER(c_double), ctypes.POINTER(c_double), c_void_p,
                                   c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double)]),
        "orc_trajectory": (c_int, [P, _dp, _dp, c_void_p, _dp, _dp, c_int, _dp, _dp, _dp,
                                   ctypes.POINTER(c_double), ctypes.POINTER(c_int)]),
        "orc_gradient_from_costs": (None, [c_int, _dp, _dp, c_double, _dp, ctypes.POINTER(c_double)]),
        "orc_sensor_gradient": (None, [c_int, c_int, _dp, c_double, _dp, _dp]),
        "orc_adjoint_gradient": (c_int, [P, _dp, _dp, _dp, _dp, c_int, c_int, ctypes.POINTER(c_double), _dp, _dp]),
        "orc_faces_to_control": (None, [P, _dp, _dp, _dp, _dp]),
        "orc_envar_gradient": (c_int, [P, _dp, _dp, _dp, c_int, c_int, _dp, _dp, c_double,
                                       c_int, c_int, c_int, c_int, _dp, _dp,
                                       ctypes.POINTER(c_double), c_void_p]),
        "orc_envar_step": (None, [c_int, _dp, _dp, c_double, c_double, _dp, ctypes.POINTER(c_double)]),
        "orc_sensor_anomalies": (None, [c_int, c_int, _dp, c_double, _dp, _dp]),
        "orc_gauss_newton_step": (c_int, [c_int, c_int, _dp, _dp, _dp, c_double, _dp, c_void_p, c_void_p]),
        "orc_lbfgs_direction": (None, [c_int, c_int, _dp, _dp, _dp, c_double, _dp]),
        "orc_domain_observation": (c_int, [P, _dp, _dp, _dp, _dp, c_int, c_int, _dp]),
        "orc_envar_gradient_domain": (c_int, [P, _dp, _dp, _dp, c_int, c_int, _dp, _dp, c_double, c_int,
                                              c_int, c_int, _dp, _dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    global _lib
    if _lib is not None:
        return _lib
    build()
    _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


class planted_mistake:
    """Context manager for pin tests that must FAIL on a wrong oracle: compiles a copy of the
    oracle source with one text replacement (the planted mistake) into ``workdir`` and routes
    every oracle call inside the ``with`` block through that copy.  The product never uses it."""

    def __init__(self, old: str, new: str, workdir: str):
        self.old, self.new, self.workdir = old, new, workdir

    def __enter__(self):
        global _lib
        src = open(_SRC).read()
        if src.count(self.old) != 1:
            raise ValueError(f"planted_mistake: the text to replace occurs {src.count(self.old)} times")
        tag = abs(hash((self.old, self.new))) % 10**8
        csrc = os.path.join(self.workdir, f"mutant_{tag}.c")
        so = os.path.join(self.workdir, f"libmutant_{tag}.so")
        with open(csrc, "w") as f:
            f.write(src.replace(self.old, self.new))
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-o", so, csrc,
                        "-lm", "-lpthread"], check=True)
        self._saved = lib()
        _lib = _configure(ctypes.CDLL(so))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


# ----------------------------------------------------------------------------
# parameter helpers
# ----------------------------------------------------------------------------
def cavity_params(nx: int, ny: int, Re: float, cfl: float = 0.3, box=CAVITY_BOX,
                  cg_rtol: float = 1e-13, cg_maxit: int = 100000, advection: int = 1, inlet_delta: float = 0.1,
                  lip_slip: int = 0, noslip_span=(-0.4, 1.75)) -> Params:
    """Open-cavity workload: box [-1.2,2.5]x[-1,1], cavity [0,1]x[-1,0] (Fig. 1 with
    the synthetic workload's channel height), inlet erf(y/inlet_delta), convective outlet,
    free-slip top, no-slip walls (or, with lip_slip, free slip on the lower wall outside
    noslip_span, Sec. 4.4); dt = cfl * min(dx, dy) with U = 1."""
    x0, x1, y0, y1 = box
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    return Params(nx=nx, ny=ny, x0=x0, x1=x1, y0=y0, y1=y1, Re=Re, dt=cfl * min(dx, dy),
                  bc_x=0, bc_y=0, geometry=0, advection=advection, inlet_delta=inlet_delta, conv_speed=1.0,
                  cg_rtol=cg_rtol, cg_maxit=cg_maxit, ch_lo=0.0, ch_hi=0.0, lip_slip=lip_slip,
                  slip_lo=noslip_span[0], slip_hi=noslip_span[1])


def make_params(**kw) -> Params:
    base = dict(nx=16, ny=16, x0=0.0, x1=1.0, y0=0.0, y1=1.0, Re=100.0, dt=1e-3, bc_x=1, bc_y=1,
                geometry=1, advection=1, inlet_delta=0.1, conv_speed=1.0, cg_rtol=1e-13,
                cg_maxit=100000, ch_lo=0.0, ch_hi=0.0, lip_slip=0, slip_lo=0.0, slip_hi=0.0)
    base.update(kw)
    return Params(**base)


def shapes(P: Params):
    return (P.ny, P.nx + 1), (P.ny + 1, P.nx), (P.ny, P.nx)


# ----------------------------------------------------------------------------
# simulation object
# ----------------------------------------------------------------------------
class Sim:
    """One FP64 simulation (Sec. 2, Eq. forced_NS on the MAC grid)."""

    def __init__(self, P: Params):
        self.P = P
        self._h = lib().orc_create(ctypes.byref(P))
        if not self._h:
            raise ValueError("oracle: bad parameters")
        self.su, self.sv, self.sp = shapes(P)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_state(self, u, v, p=None):
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.su)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(self.sv)
        if p is None:
            lib().orc_set_state(self._h, u, v, None)
        else:
            p = np.ascontiguousarray(p, dtype=np.float64).reshape(self.sp)
            lib().orc_set_state(self._h, u, v, p.ctypes.data_as(c_void_p))

    def state(self):
        u, v, p = np.zeros(self.su), np.zeros(self.sv), np.zeros(self.sp)
        lib().orc_get_state(self._h, u, v, p)
        return u, v, p

    def set_forcing(self, fu, fv):
        lib().orc_set_face_forcing(self._h, np.ascontiguousarray(fu, dtype=np.float64).reshape(self.su),
                                   np.ascontiguousarray(fv, dtype=np.float64).reshape(self.sv))

    def step(self, n: int = 1) -> int:
        return lib().orc_step(self._h, int(n))

    def max_div(self) -> float:
        return lib().orc_max_div(self._h)

    def last_cg(self):
        return lib().orc_last_cg_iters(self._h), lib().orc_last_cg_relres(self._h)

    def fluxes(self):
        a, b = c_double(), c_double()
        lib().orc_fluxes(self._h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def face_kinds(self):
        uk = np.zeros(self.su, dtype=np.uint8)
        vk = np.zeros(self.sv, dtype=np.uint8)
        lib().orc_face_kinds(self._h, uk, vk)
        return uk, vk

    def project(self, u, v):
        u = np.array(u, dtype=np.float64).reshape(self.su)
        v = np.array(v, dtype=np.float64).reshape(self.sv)
        lib().orc_project(self._h, u, v)
        return u, v

    def apply_negL(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.sp)
        y = np.zeros(self.sp)
        lib().orc_apply_negL(self._h, x, y)
        return y

    def poisson_solve(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(self.sp)
        x = np.zeros(self.sp)
        lib().orc_poisson_solve(self._h, b, x)
        return x

    def explicit_rhs(self):
        Ru, Rv = np.zeros(self.su), np.zeros(self.sv)
        lib().orc_explicit_rhs(self._h, Ru, Rv)
        return Ru, Rv

    def sensors(self):
        out = np.zeros(8)
        lib().orc_sensors(self._h, out)
        return out


FK_WALL, FK_UNKNOWN, FK_INLET, FK_OUTLET, FK_SOLID, FK_COPY = range(6)


def fluid_mask(P: Params) -> np.ndarray:
    F = np.zeros((P.ny, P.nx), dtype=np.uint8)
    lib().orc_fluid_mask(ctypes.byref(P), F)
    return F


# ----------------------------------------------------------------------------
# control, ensemble, random numbers
# ----------------------------------------------------------------------------
def control_rect(P: Params, region=CAVITY_REGION):
    r = np.zeros(4, dtype=np.int32)
    rc = lib().orc_control_rect(ctypes.byref(P), np.asarray(region, dtype=np.float64), r)
    if rc != 0:
        raise ValueError("empty control region")
    return tuple(int(x) for x in r)


def control_cells(P: Params, region=CAVITY_REGION):
    reg = np.asarray(region, dtype=np.float64)
    n = lib().orc_control_cells(ctypes.byref(P), reg, None, None)
    ci = np.zeros(n, dtype=np.int32)
    cj = np.zeros(n, dtype=np.int32)
    lib().orc_control_cells(ctypes.byref(P), reg, ci.ctypes.data_as(c_void_p), cj.ctypes.data_as(c_void_p))
    return ci, cj


def control_to_faces(P: Params, f, region=CAVITY_REGION):
    su, sv, _ = shapes(P)
    fu, fv = np.zeros(su), np.zeros(sv)
    lib().orc_control_to_faces(ctypes.byref(P), np.asarray(region, dtype=np.float64),
                               np.ascontiguousarray(f, dtype=np.float64), fu, fv)
    return fu, fv


def philox4x64_10(ctr, key):
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(np.asarray(ctr, dtype=np.uint64), np.asarray(key, dtype=np.uint64), out)
    return out


def normals(seed: int, stream: int, first: int, n: int) -> np.ndarray:
    out = np.zeros(n)
    lib().orc_normals(ctypes.c_uint64(seed), ctypes.c_uint64(stream), first, n, out)
    return out


def sampler_dims(P: Params, a: float, region=CAVITY_REGION):
    d = np.zeros(4, dtype=np.int32)
    if lib().orc_sampler_dims(ctypes.byref(P), np.asarray(region, dtype=np.float64), a, d) != 0:
        raise ValueError("empty control region")
    return tuple(int(x) for x in d)


def sampler_factors(P: Params, a: float, region=CAVITY_REGION):
    nrx, nry, nxix, nxiy = sampler_dims(P, a, region)
    Gx, Gy = np.zeros((nrx, nxix)), np.zeros((nry, nxiy))
    lib().orc_sampler_factors(ctypes.byref(P), np.asarray(region, dtype=np.float64), a, Gx, Gy)
    return Gx, Gy


def ensemble_from_noise(P: Params, sigma: float, a: float, N: int, Z, region=CAVITY_REGION):
    ncc = len(control_cells(P, region)[0])
    E = np.zeros((N, 2 * ncc))  # row k = column k of E (column-major n_ctrl x N)
    rc = lib().orc_ensemble_from_noise(ctypes.byref(P), np.asarray(region, dtype=np.float64), sigma, a, N,
                                       np.ascontiguousarray(Z, dtype=np.float64), E)
    if rc != 0:
        raise ValueError("ensemble generation failed")
    return E.T.copy()  # n_ctrl x N


def ensemble_seeded(P: Params, sigma: float, a: float, N: int, seed: int, region=CAVITY_REGION):
    ncc = len(control_cells(P, region)[0])
    E = np.zeros((N, 2 * ncc))
    rc = lib().orc_ensemble_seeded(ctypes.byref(P), np.asarray(region, dtype=np.float64), sigma, a, N,
                                   ctypes.c_uint64(seed), E)
    if rc != 0:
        raise ValueError("ensemble generation failed")
    return E.T.copy()


# ----------------------------------------------------------------------------
# runs
# ----------------------------------------------------------------------------
def trajectory(P: Params, u0, v0, n_steps: int, fu=None, fv=None, p0=None):
    su, sv, sp = shapes(P)
    fu = np.zeros(su) if fu is None else np.ascontiguousarray(fu, dtype=np.float64).reshape(su)
    fv = np.zeros(sv) if fv is None else np.ascontiguousarray(fv, dtype=np.float64).reshape(sv)
    u, v, p = np.zeros(su), np.zeros(sv), np.zeros(sp)
    md, it = c_double(), c_int()
    p0p = None
    if p0 is not None:
        p0 = np.ascontiguousarray(p0, dtype=np.float64).reshape(sp)
        p0p = p0.ctypes.data_as(c_void_p)
    rc = lib().orc_trajectory(ctypes.byref(P), np.ascontiguousarray(u0, dtype=np.float64).reshape(su),
                              np.ascontiguousarray(v0, dtype=np.float64).reshape(sv), p0p, fu, fv, int(n_steps),
                              u, v, p, ctypes.byref(md), ctypes.byref(it))
    if rc != 0:
        raise RuntimeError(f"oracle trajectory failed ({rc})")
    return u, v, p, md.value, it.value


def member_run(P: Params, u0, v0, n_steps: int, n_window: int, fu=None, fv=None, want_series=False,
               want_state=False):
    su, sv, sp = shapes(P)
    fu = np.zeros(su) if fu is None else np.ascontiguousarray(fu, dtype=np.float64).reshape(su)
    fv = np.zeros(sv) if fv is None else np.ascontiguousarray(fv, dtype=np.float64).reshape(sv)
    jd, js, md = c_double(), c_double(), c_double()
    ser = np.zeros((max(n_window, 1), 8)) if want_series else None
    ue, ve, pe = (np.zeros(su), np.zeros(sv), np.zeros(sp)) if want_state else (None, None, None)
    ptr = lambda a: None if a is None else a.ctypes.data_as(c_void_p)
    rc = lib().orc_member_run(ctypes.byref(P), np.ascontiguousarray(u0, dtype=np.float64).reshape(su),
                              np.ascontiguousarray(v0, dtype=np.float64).reshape(sv), fu, fv, int(n_steps),
                              int(n_window), ctypes.byref(jd), ctypes.byref(js), ptr(ser), ptr(ue), ptr(ve),
                              ptr(pe), ctypes.byref(md))
    if rc != 0:
        raise RuntimeError(f"oracle member run failed ({rc})")
    out = {"J_domain": jd.value, "J_sensor": js.value, "max_div": md.value}
    if want_series:
        out["series"] = ser[:n_window]
    if want_state:
        out["state"] = (ue, ve, pe)
    return out


def gradient_from_costs(J, w, eps: float):
    """Eq. (gradient_EnVar) from the N+1 observation costs (see ns2d_oracle.c)."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.zeros(len(w))
    jp = c_double()
    lib().orc_gradient_from_costs(len(w), J, w, eps, g, ctypes.byref(jp))
    return g, jp.value


def sensor_gradient(series, w, eps: float):
    """Eq. (gradient_EnVar) with Y from Eq. (fdapprox) on the sensor series [N+1][n_window][8]."""
    series = np.ascontiguousarray(series, dtype=np.float64)
    N = series.shape[0] - 1
    g = np.zeros(N)
    lib().orc_sensor_gradient(N, series.shape[1], series.reshape(-1), eps,
                              np.ascontiguousarray(w, dtype=np.float64), g)
    return g


def adjoint_gradient(P: Params, u0, v0, n_steps: int, n_window: int, fu=None, fv=None):
    """Discrete adjoint (Sec. 3.2, Eq. adjoint_discrete / gradient_forcing): DOMAIN cost J and dJ/dF on faces."""
    su, sv, _ = shapes(P)
    fu = np.zeros(su) if fu is None else np.ascontiguousarray(fu, dtype=np.float64).reshape(su)
    fv = np.zeros(sv) if fv is None else np.ascontiguousarray(fv, dtype=np.float64).reshape(sv)
    gu, gv, J = np.zeros(su), np.zeros(sv), c_double()
    rc = lib().orc_adjoint_gradient(ctypes.byref(P), np.ascontiguousarray(u0, dtype=np.float64).reshape(su),
                                    np.ascontiguousarray(v0, dtype=np.float64).reshape(sv), fu, fv, int(n_steps),
                                    int(n_window), ctypes.byref(J), gu, gv)
    if rc != 0:
        raise RuntimeError(f"oracle adjoint failed ({rc})")
    return J.value, gu, gv


def faces_to_control(P: Params, gu, gv, region=CAVITY_REGION):
    """Transpose of control_to_faces: control-space gradient from a face gradient."""
    n = len(control_cells(P, region)[0])
    g = np.zeros(2 * n)
    lib().orc_faces_to_control(ctypes.byref(P), np.asarray(region, dtype=np.float64),
                               np.ascontiguousarray(gu, dtype=np.float64), np.ascontiguousarray(gv, dtype=np.float64), g)
    return g


def envar_gradient(P: Params, u0, v0, E, w, eps: float, n_steps: int, n_window: int,
                   cost_mode: int = COST_DOMAIN, nthreads: int | None = None, region=CAVITY_REGION,
                   want_series=False):
    """Fig. (envar_loop): N+1 forward runs, costs and the EnVar gradient."""
    su, sv, _ = shapes(P)
    E = np.asarray(E, dtype=np.float64)
    n_ctrl, N = E.shape
    Ecm = np.ascontiguousarray(E.T)  # column-major storage
    J, g, jp = np.zeros(N + 1), np.zeros(N), c_double()
    ser = np.zeros((N + 1, max(n_window, 1), 8)) if want_series else None
    nthreads = nthreads or min(N + 1, os.cpu_count() or 1)
    rc = lib().orc_envar_gradient(ctypes.byref(P), np.asarray(region, dtype=np.float64),
                                  np.ascontiguousarray(u0, dtype=np.float64).reshape(su),
                                  np.ascontiguousarray(v0, dtype=np.float64).reshape(sv),
                                  n_ctrl, N, Ecm.reshape(-1), np.ascontiguousarray(w, dtype=np.float64), eps,
                                  int(n_steps), int(n_window), int(cost_mode), int(nthreads), J, g,
                                  ctypes.byref(jp), None if ser is None else ser.ctypes.data_as(c_void_p))
    if rc != 0:
        raise RuntimeError(f"oracle envar gradient failed ({rc})")
    out = {"J": J, "g": g, "J_prior": jp.value}
    if want_series:
        out["series"] = ser[:, :n_window]
    return out


def envar_step(w, g, alpha: float, J0_obs: float):
    """Weight update of Sec. 3.3.1, w - alpha g / (N-1), and the total cost J(w) of Eq. (J_w)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out, jt = np.zeros(len(w)), c_double()
    lib().orc_envar_step(len(w), w, g, float(alpha), float(J0_obs), out, ctypes.byref(jt))
    return out, jt.value


def domain_observation(P: Params, u0, v0, n_steps: int, n_window: int, fu=None, fv=None):
    """Observation vector h of the DOMAIN cost, [n_window][ny][nx][2], with J_domain = ||h||^2 / 2."""
    su, sv, _ = shapes(P)
    fu = np.zeros(su) if fu is None else np.ascontiguousarray(fu, dtype=np.float64).reshape(su)
    fv = np.zeros(sv) if fv is None else np.ascontiguousarray(fv, dtype=np.float64).reshape(sv)
    h = np.zeros((n_window, P.ny, P.nx, 2))
    rc = lib().orc_domain_observation(ctypes.byref(P), np.ascontiguousarray(u0, dtype=np.float64).reshape(su),
                                      np.ascontiguousarray(v0, dtype=np.float64).reshape(sv), fu, fv,
                                      int(n_steps), int(n_window), h)
    if rc != 0:
        raise RuntimeError(f"oracle domain observation failed ({rc})")
    return h


def envar_gradient_domain(P: Params, u0, v0, E, w, eps: float, n_steps: int, n_window: int,
                          nthreads: int | None = None, region=CAVITY_REGION):
    """Eq. (gradient_EnVar) with Y from Eq. (fdapprox) on the DOMAIN observation vector:
    g_i = Y_i^T h_0 + (N-1) w_i.  Returns (g, ||Y_i||^2)."""
    su, sv, _ = shapes(P)
    E = np.asarray(E, dtype=np.float64)
    n_ctrl, N = E.shape
    g, yy = np.zeros(N), np.zeros(N)
    nthreads = nthreads or min(N, os.cpu_count() or 1)
    rc = lib().orc_envar_gradient_domain(ctypes.byref(P), np.asarray(region, dtype=np.float64),
                                         np.ascontiguousarray(u0, dtype=np.float64).reshape(su),
                                         np.ascontiguousarray(v0, dtype=np.float64).reshape(sv), n_ctrl, N,
                                         np.ascontiguousarray(E.T).reshape(-1),
                                         np.ascontiguousarray(w, dtype=np.float64), float(eps), int(n_steps),
                                         int(n_window), int(nthreads), g, yy)
    if rc != 0:
        raise RuntimeError(f"oracle domain gradient failed ({rc})")
    return g, yy


def sensor_anomalies(series, eps: float):
    """Sensor-space Y of Eq. (fdapprox) and h_0: series [N+1][n_window][8] -> (Y [N][8 n_w], h0)."""
    series = np.ascontiguousarray(series, dtype=np.float64)
    N, nw = series.shape[0] - 1, series.shape[1]
    Y, h0 = np.zeros((N, 8 * nw)), np.zeros(8 * nw)
    lib().orc_sensor_anomalies(N, nw, series.reshape(-1), float(eps), Y, h0)
    return Y, h0


def gauss_newton_step(Y, h0, w, alpha: float = 1.0):
    """Sec. 3.3.1 Gauss-Newton: (w + alpha dw, H_GN, g) with H_GN = Y^T Y + (N-1) I,
    g = Y^T h0 + (N-1) w, dw = -H_GN^{-1} g."""
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    N, nobs = Y.shape
    w = np.ascontiguousarray(w, dtype=np.float64)
    out, H, g = np.zeros(N), np.zeros((N, N)), np.zeros(N)
    rc = lib().orc_gauss_newton_step(N, nobs, Y, np.ascontiguousarray(h0, dtype=np.float64), w, float(alpha), out,
                                     H.ctypes.data_as(c_void_p), g.ctypes.data_as(c_void_p))
    if rc != 0:
        raise ValueError("Gauss-Newton Hessian is not positive definite")
    return out, H, g


def lbfgs_direction(S, Yh, g, gamma: float):
    """L-BFGS direction -H g (two-loop recursion) from pairs S, Yh [m][N], oldest first."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    N = len(g)
    S = np.ascontiguousarray(np.reshape(S, (-1, N)), dtype=np.float64)
    Yh = np.ascontiguousarray(np.reshape(Yh, (-1, N)), dtype=np.float64)
    p = np.zeros(N)
    lib().orc_lbfgs_direction(N, S.shape[0], S.reshape(-1), Yh.reshape(-1), g, float(gamma), p)
    return p


# ----------------------------------------------------------------------------
# eigenvector ensemble (Sec. 3.3.2, Eq. eigenvm1)
# ----------------------------------------------------------------------------
def covariance_B(P: Params, sigma: float, a: float, region=CAVITY_REGION):
    """Dense prior covariance of one forcing component on the control cells, Eq. (covarianceB) with
    sigma_i = sigma, a_x = a_y = a and c_xy = infinity: B_ij = sigma^2 exp(-dx^2/a^2 - dy^2/a^2)."""
    ci, cj = control_cells(P, region)
    x = P.x0 + (ci + 0.5) * P.dx
    y = P.y0 + (cj + 0.5) * P.dy
    d2 = (x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2
    return sigma * sigma * np.exp(-d2 / (a * a))


def eigen_ensemble(P: Params, sigma: float, a: float, N: int, region=CAVITY_REGION, y_only: bool = False):
    """Sec. 3.3.2: B = U Sigma U^T with U^T M_f U = I and E = U_N Sigma_N^{1/2} sqrt(N - 1)
    (Eq. eigenvm1).  On this uniform grid M_f = dx dy I, which cancels: E = V_N Lambda_N^{1/2} sqrt(N-1)
    with (V, Lambda) the Euclidean eigenpairs of B.  The control vector holds two independent
    components with the same covariance, so B = diag(B_s, B_s): each eigenpair of B_s appears twice,
    and the columns of E take the eigenvectors of B_s in decreasing eigenvalue order, each first as an
    fx field and then as an fy field (with y_only, forcing in the y-momentum equation only, the fx
    variance is zero and every column is an fy field).  Each eigenvector's sign makes its
    largest-magnitude entry positive.  Returns (E [n_ctrl x N], the N eigenvalues of B used)."""
    Bs = covariance_B(P, sigma, a, region)
    lam, V = np.linalg.eigh(Bs)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    n = Bs.shape[0]
    E = np.zeros((2 * n, N))
    lams = np.zeros(N)
    for k in range(N):
        r = k if y_only else k // 2
        v = V[:, r].copy()
        j = int(np.argmax(np.abs(v)))
        if v[j] < 0:
            v = -v
        comp = 1 if y_only else k % 2
        E[comp * n:(comp + 1) * n, k] = np.sqrt(max(lam[r], 0.0) * (N - 1)) * v
        lams[k] = lam[r]
    return E, lams


# ----------------------------------------------------------------------------
# H^1 gradient smoothing of the adjoint approach (Sec. 4.2, Eq. lsob)
# ----------------------------------------------------------------------------
def control_laplacian(P: Params, region=CAVITY_REGION):
    """5-point Laplacian on the control cells with no flux through the boundary of the control set
    (a neighbour outside the set contributes nothing), as a scipy sparse matrix on one component."""
    import scipy.sparse as sp
    ci, cj = control_cells(P, region)
    n = len(ci)
    where = {(int(i), int(j)): q for q, (i, j) in enumerate(zip(ci, cj))}
    rows, cols, vals = [], [], []
    for q, (i, j) in enumerate(zip(ci, cj)):
        for di, dj, h2 in ((1, 0, P.dx**2), (-1, 0, P.dx**2), (0, 1, P.dy**2), (0, -1, P.dy**2)):
            r = where.get((int(i) + di, int(j) + dj))
            if r is None:
                continue
            rows += [q, q]
            cols += [r, q]
            vals += [1.0 / h2, -1.0 / h2]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def h1_smooth(P: Params, g, l_sob: float, region=CAVITY_REGION):
    """Eq. (lsob): (I - l^2 Lap) g_H1 = (1 + l^2) g for each forcing component, Lap the control-set
    Laplacian with no flux through its boundary.  g: [fx over control cells | fy over control cells]."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    L = control_laplacian(P, region)
    n = L.shape[0]
    A = (sp.identity(n, format="csc") - l_sob * l_sob * L).tocsc()
    g = np.asarray(g, dtype=np.float64)
    return np.concatenate([spla.spsolve(A, (1.0 + l_sob**2) * g[:n]), spla.spsolve(A, (1.0 + l_sob**2) * g[n:])])
