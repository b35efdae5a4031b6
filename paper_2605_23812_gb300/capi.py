"""ctypes binding of the C ABI in ``include/envar.h`` (argument marshalling only).

Every computation runs in ``libenvar_gb300.so`` (sm_103a kernels).  There is no
Python or CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libenvar_gb300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "envar.h")

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p

FP64_PLAIN, FP64_BATCHED, MIXED = 0, 1, 2
COST_DOMAIN, COST_SENSORS = 0, 1
ST_NONFINITE, ST_DIVERGENCE, ST_CFL, ST_ADJOINT = 1, 2, 4, 8
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ESTATE", -5: "EDEVICE"}


class Config(ctypes.Structure):
    """Mirror of ``envar_config``."""
    _fields_ = [
        ("nx", c_int), ("ny", c_int),
        ("x0", c_double), ("x1", c_double), ("y0", c_double), ("y1", c_double),
        ("Re", c_double), ("cfl", c_double), ("inlet_delta", c_double), ("conv_speed", c_double),
        ("n_steps", c_int), ("n_window", c_int), ("n_members", c_int),
        ("region", c_double * 4),
        ("sigma", c_double), ("corr_len", c_double), ("eps", c_double),
        ("seed", ctypes.c_ulonglong),
        ("precision", c_int), ("cost_mode", c_int),
        ("div_tol", c_double),
        ("max_outer", c_int), ("max_inner", c_int), ("inner_rtol", c_double),
        ("nu_pre", c_int), ("nu_post", c_int), ("coarse_sweeps", c_int), ("steps_per_graph", c_int),
        ("member_groups", c_int),
        ("lip_slip", c_int), ("noslip_span", c_double * 2), ("forcing_y_only", c_int),
        ("conditional_refinement", c_int), ("guess_extrapolation", c_int), ("nu_coarse", c_int),
    ]


def header_symbols() -> list[str]:
    """Entry points declared in include/envar.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(envar_\w+)\s*\(", txt, flags=re.M)))


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    H = c_void_p
    sig = {
        "envar_default_config": [ctypes.POINTER(Config), c_int, c_int],
        "envar_init": [ctypes.POINTER(c_void_p), ctypes.POINTER(Config), c_void_p],
        "envar_destroy": [H],
        "envar_sizes": [H, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                        ctypes.POINTER(c_double)],
        "envar_set_initial_state": [H, c_void_p, c_void_p],
        "envar_set_ensemble": [H, c_void_p, c_int, c_int],
        "envar_get_ensemble": [H, c_void_p],
        "envar_forward_ensemble": [H, c_void_p],
        "envar_cost": [H, c_void_p, c_void_p],
        "envar_gradient": [H, c_void_p, c_void_p],
        "envar_gradient_scalar": [H, c_void_p],
        "envar_excluded_members": [H, ctypes.POINTER(c_int)],
        "envar_gn_step": [H, c_double, c_void_p, c_void_p],
        "envar_eigen_ensemble": [H, c_void_p],
        "envar_batch_create": [ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_int, c_void_p],
        "envar_batch_destroy": [c_void_p],
        "envar_batch_forward": [c_void_p, ctypes.POINTER(c_void_p)],
        "envar_batch_info": [c_void_p, ctypes.POINTER(c_int), c_void_p],
        "envar_h1_smooth": [H, c_void_p, c_void_p, c_double],
        "envar_adjoint_lbfgs_step": [H, c_void_p, c_int, c_double, c_double, c_void_p, c_void_p, c_void_p],
        "envar_adjoint_lbfgs_reset": [H, c_int],
        "envar_gn_hessian": [H, c_void_p],
        "envar_lbfgs_step": [H, c_void_p, c_void_p, c_void_p, c_void_p],
        "envar_lbfgs_reset": [H, c_int],
        "envar_step": [H, c_double, c_void_p, c_void_p],
        "envar_step_device": [H, c_double, c_void_p, c_void_p],
        "envar_forward_control": [H, c_void_p, c_void_p],
        "envar_member_status": [H, c_void_p],
        "envar_get_state": [H, c_int, c_void_p, c_void_p, c_void_p],
        "envar_get_series": [H, c_int, c_void_p],
        "envar_diagnostics": [H, ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(ctypes.c_longlong)],
        "envar_reset_members": [H, c_void_p],
        "envar_advance": [H, c_int],
        "envar_kernel_launches": [H, ctypes.POINTER(ctypes.c_longlong)],
        "envar_time_kernel": [H, c_int, c_int, ctypes.POINTER(c_double)],
        "envar_apply_preconditioner": [H, c_void_p, c_void_p],
        "envar_adjoint_gradient": [H, c_void_p, c_void_p, c_int, c_void_p],
        "envar_autotune": [H, c_int, ctypes.POINTER(c_double), ctypes.POINTER(c_int)],
        "envar_get_config": [H, ctypes.POINTER(Config)],
        "envar_adjoint_stats": [H] + [ctypes.POINTER(ctypes.c_longlong)] * 4,
        "envar_revolve_plan": [ctypes.c_longlong, c_int] + [ctypes.POINTER(ctypes.c_longlong)] * 3,
        "envar_draw_ensemble_noalloc": [ctypes.POINTER(Config), c_void_p, c_int, c_void_p],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = c_int
    L.envar_last_error.argtypes = [H]
    L.envar_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def default_config(nx: int, ny: int, **kw) -> Config:
    c = Config()
    lib().envar_default_config(ctypes.byref(c), nx, ny)
    for k, v in kw.items():
        if k == "region":
            c.region = (c_double * 4)(*v)
        elif k == "noslip_span":
            c.noslip_span = (c_double * 2)(*v)
        else:
            setattr(c, k, v)
    return c


def _ptr(t):
    return c_void_p(0 if t is None else t.data_ptr())


def _np_ptr(a):
    return a.ctypes.data_as(c_void_p)


class EnvarError(RuntimeError):
    pass


class Ensemble:
    """One handle of the library: N+1 forced cavity simulations and their EnVar gradient."""

    def __init__(self, cfg: Config, stream=None):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = c_void_p()
        rc = lib().envar_init(ctypes.byref(h), ctypes.byref(cfg), c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise EnvarError(f"envar_init: {ERRORS.get(rc, rc)}: {lib().envar_last_error(None).decode()}")
        self._h = h
        n_ctrl, n_cc, nlev, dt = c_int(), c_int(), c_int(), c_double()
        self._check(lib().envar_sizes(h, ctypes.byref(n_ctrl), ctypes.byref(n_cc), ctypes.byref(nlev),
                                      ctypes.byref(dt)), "envar_sizes")
        self.n_ctrl, self.n_cc, self.n_levels, self.dt = n_ctrl.value, n_cc.value, nlev.value, dt.value
        self.N = cfg.n_members

    def _check(self, rc, what):
        if rc != 0:
            raise EnvarError(f"{what}: {ERRORS.get(rc, rc)}: {lib().envar_last_error(self._h).decode()}")

    def close(self):
        if getattr(self, "_h", None):
            lib().envar_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, shape=None):
        t = self.torch
        x = a if isinstance(a, t.Tensor) else t.as_tensor(np.asarray(a, dtype=np.float64))
        x = x.to(device="cuda", dtype=t.float64).contiguous()
        if shape is not None:
            x = x.reshape(shape)
        return x

    # ---- inputs
    def set_initial_state(self, u0, v0):
        u = self._dev(u0, (self.cfg.ny, self.cfg.nx + 1))
        v = self._dev(v0, (self.cfg.ny + 1, self.cfg.nx))
        self.torch.cuda.current_stream().synchronize()
        self._check(lib().envar_set_initial_state(self._h, _ptr(u), _ptr(v)), "envar_set_initial_state")

    def set_ensemble(self, E):
        """E: (n_ctrl, N) array or tensor."""
        Et = self._dev(E, (self.n_ctrl, self.N)).t().contiguous()   # column-major storage
        self.torch.cuda.current_stream().synchronize()
        self._check(lib().envar_set_ensemble(self._h, _ptr(Et), self.n_ctrl, self.N), "envar_set_ensemble")

    def use_eigen_ensemble(self):
        """Replace E by the eigenvector ensemble of Eq. (eigenvm1); returns the members' eigenvalues."""
        lam = np.zeros(self.N)
        self._check(lib().envar_eigen_ensemble(self._h, _np_ptr(lam)), "envar_eigen_ensemble")
        return lam

    def get_ensemble(self):
        out = self.torch.empty((self.N, self.n_ctrl), dtype=self.torch.float64, device="cuda")
        self._check(lib().envar_get_ensemble(self._h, _ptr(out)), "envar_get_ensemble")
        return out.t()

    # ---- EnVar calls
    def forward_ensemble(self, w):
        wt = self._dev(w, (self.N,))
        self.torch.cuda.current_stream().synchronize()
        self._check(lib().envar_forward_ensemble(self._h, _ptr(wt)), "envar_forward_ensemble")

    def cost(self):
        J = np.zeros(self.N + 1)
        jp = np.zeros(1)
        self._check(lib().envar_cost(self._h, _np_ptr(J), _np_ptr(jp)), "envar_cost")
        return J, float(jp[0])

    def gradient(self, want_df=False):
        g = np.zeros(self.N)
        df = self.torch.empty(self.n_ctrl, dtype=self.torch.float64, device="cuda") if want_df else None
        self._check(lib().envar_gradient(self._h, _np_ptr(g), _ptr(df)), "envar_gradient")
        return (g, df) if want_df else g

    def gradient_scalar(self):
        """Scalar-anomaly form (J_i - J_0)/eps + (N-1) w_i of the last forward run."""
        g = np.zeros(self.N)
        self._check(lib().envar_gradient_scalar(self._h, _np_ptr(g)), "envar_gradient_scalar")
        return g

    def excluded_members(self) -> int:
        n = c_int()
        self._check(lib().envar_excluded_members(self._h, ctypes.byref(n)), "envar_excluded_members")
        return n.value

    def step(self, alpha, w):
        w = np.ascontiguousarray(w, dtype=np.float64).copy()
        J0 = np.zeros(1)
        self._check(lib().envar_step(self._h, float(alpha), _np_ptr(w), _np_ptr(J0)), "envar_step")
        return w, float(J0[0])

    def gn_step(self, alpha, w):
        """Gauss-Newton EnVar iteration (SENSORS cost): returns (w_new, J(w))."""
        w = np.ascontiguousarray(w, dtype=np.float64).copy()
        J0 = np.zeros(1)
        self._check(lib().envar_gn_step(self._h, float(alpha), _np_ptr(w), _np_ptr(J0)), "envar_gn_step")
        return w, float(J0[0])

    def gn_hessian(self):
        H = np.zeros((self.N, self.N))
        self._check(lib().envar_gn_hessian(self._h, _np_ptr(H)), "envar_gn_hessian")
        return H

    def lbfgs_step(self, w):
        """L-BFGS EnVar iteration with Armijo backtracking: returns (w_new, J(w), step length, trials)."""
        w = np.ascontiguousarray(w, dtype=np.float64).copy()
        J0, a = np.zeros(1), np.zeros(1)
        n = c_int()
        self._check(lib().envar_lbfgs_step(self._h, _np_ptr(w), _np_ptr(J0), _np_ptr(a), ctypes.byref(n)),
                    "envar_lbfgs_step")
        return w, float(J0[0]), float(a[0]), n.value

    def lbfgs_reset(self, memory: int = 8):
        self._check(lib().envar_lbfgs_reset(self._h, int(memory)), "envar_lbfgs_reset")

    def step_device(self, alpha, w_dev, J0_dev=None):
        """envar_step on device-resident tensors (w_dev updated in place)."""
        self._check(lib().envar_step_device(self._h, float(alpha), _ptr(w_dev), _ptr(J0_dev)), "envar_step_device")

    def forward_control(self, f):
        ft = self._dev(f, (self.n_ctrl,))
        J = np.zeros(1)
        self.torch.cuda.current_stream().synchronize()
        self._check(lib().envar_forward_control(self._h, _ptr(ft), _np_ptr(J)), "envar_forward_control")
        return float(J[0])

    # ---- diagnostics
    def member_status(self):
        s = np.zeros(self.N + 1, dtype=np.int32)
        self._check(lib().envar_member_status(self._h, _np_ptr(s)), "envar_member_status")
        return s

    def get_state(self, member):
        t = self.torch
        u = t.empty((self.cfg.ny, self.cfg.nx + 1), dtype=t.float64, device="cuda")
        v = t.empty((self.cfg.ny + 1, self.cfg.nx), dtype=t.float64, device="cuda")
        p = t.empty((self.cfg.ny, self.cfg.nx), dtype=t.float64, device="cuda")
        self._check(lib().envar_get_state(self._h, int(member), _ptr(u), _ptr(v), _ptr(p)), "envar_get_state")
        return u, v, p

    def get_series(self, member):
        s = np.zeros((self.cfg.n_window, 8))
        self._check(lib().envar_get_series(self._h, int(member), _np_ptr(s)), "envar_get_series")
        return s

    def diagnostics(self):
        md, oi, ii = c_double(), ctypes.c_longlong(), ctypes.c_longlong()
        self._check(lib().envar_diagnostics(self._h, ctypes.byref(md), ctypes.byref(oi), ctypes.byref(ii)),
                    "envar_diagnostics")
        return {"max_div": md.value, "outer_its": oi.value, "inner_its": ii.value}

    def reset_members(self, w=None):
        wt = None if w is None else self._dev(w, (self.N,))
        self.torch.cuda.current_stream().synchronize()
        self._check(lib().envar_reset_members(self._h, _ptr(wt)), "envar_reset_members")

    def advance(self, n):
        self._check(lib().envar_advance(self._h, int(n)), "envar_advance")

    def apply_preconditioner(self, r):
        t = self.torch
        rr = self._dev(r, (self.cfg.ny, self.cfg.nx))
        z = t.empty_like(rr)
        t.cuda.current_stream().synchronize()
        self._check(lib().envar_apply_preconditioner(self._h, _ptr(rr), _ptr(z)), "envar_apply_preconditioner")
        return z

    def time_kernel(self, which: int, reps: int = 20) -> float:
        ms = c_double()
        self._check(lib().envar_time_kernel(self._h, int(which), int(reps), ctypes.byref(ms)), "envar_time_kernel")
        return ms.value

    # ---- solver tuning
    def autotune(self, probe_steps: int = 200):
        """Fastest pressure-solve parameters on this GPU (see envar_autotune); returns them."""
        ms = c_double()
        ch = (c_int * 4)()
        self.torch.cuda.current_stream().synchronize()
        self._check(lib().envar_autotune(self._h, int(probe_steps), ctypes.byref(ms), ch), "envar_autotune")
        c = self.config()
        return {"max_outer": ch[0], "max_inner": ch[1], "nu": ch[2], "coarse_sweeps": ch[3],
                "inner_rtol": c.inner_rtol, "nu_coarse": c.nu_coarse, "probe_ms_per_step": ms.value}

    def config(self) -> Config:
        c = Config()
        self._check(lib().envar_get_config(self._h, ctypes.byref(c)), "envar_get_config")
        return c

    # ---- discrete adjoint (FP64 handles)
    def adjoint_gradient(self, f, max_snapshots: int = 64):
        """(J, dJ/df) of one forward run with control forcing f, by the discrete adjoint."""
        ft = self._dev(f, (self.n_ctrl,))
        g = self.torch.empty_like(ft)
        J = np.zeros(1)
        self.torch.cuda.current_stream().synchronize()
        self._check(lib().envar_adjoint_gradient(self._h, _ptr(ft), _ptr(g), int(max_snapshots), _np_ptr(J)),
                    "envar_adjoint_gradient")
        return float(J[0]), g

    def h1_smooth(self, g, l_sob: float = 0.02):
        """Eq. (lsob) on a control-space vector (array or tensor); returns a device tensor."""
        gt = self._dev(g, (self.n_ctrl,))
        out = self.torch.empty_like(gt)
        self.torch.cuda.current_stream().synchronize()
        self._check(lib().envar_h1_smooth(self._h, _ptr(gt), _ptr(out), float(l_sob)), "envar_h1_smooth")
        return out

    def adjoint_lbfgs_step(self, f_dev, max_snapshots: int = 64, l_sob: float = 0.02, first_step: float = 1e-3):
        """One adjoint-approach iteration (updates the device tensor f_dev in place): (J(f), step, trials)."""
        J, a = np.zeros(1), np.zeros(1)
        n = c_int()
        self.torch.cuda.current_stream().synchronize()
        self._check(lib().envar_adjoint_lbfgs_step(self._h, _ptr(f_dev), int(max_snapshots), float(l_sob),
                                                   float(first_step), _np_ptr(J), _np_ptr(a), ctypes.byref(n)),
                    "envar_adjoint_lbfgs_step")
        return float(J[0]), float(a[0]), n.value

    def adjoint_lbfgs_reset(self, memory: int = 8):
        self._check(lib().envar_adjoint_lbfgs_reset(self._h, int(memory)), "envar_adjoint_lbfgs_reset")

    def adjoint_stats(self):
        v = [ctypes.c_longlong() for _ in range(4)]
        self._check(lib().envar_adjoint_stats(self._h, *[ctypes.byref(x) for x in v]), "envar_adjoint_stats")
        return dict(zip(("forward_steps", "reverse_steps", "stores", "restores"), (x.value for x in v)))


class Batch:
    """Uneven member groups (handles of different grids, Reynolds numbers and horizons) advancing
    together, one CUDA graph per chunk (envar_batch_* in include/envar.h)."""

    def __init__(self, ensembles, stream=None):
        import torch
        self.torch = torch
        self.ens = list(ensembles)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        hs = (c_void_p * len(self.ens))(*[e._h for e in self.ens])
        b = c_void_p()
        rc = lib().envar_batch_create(ctypes.byref(b), hs, len(self.ens), c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise EnvarError(f"envar_batch_create: {ERRORS.get(rc, rc)}: {lib().envar_last_error(None).decode()}")
        self._b = b

    def forward(self, ws):
        """ws: one weight vector per handle (arrays or device tensors)."""
        wt = [e._dev(w, (e.N,)) for e, w in zip(self.ens, ws)]
        ptrs = (c_void_p * len(wt))(*[c_void_p(t.data_ptr()) for t in wt])
        self.torch.cuda.synchronize()
        rc = lib().envar_batch_forward(self._b, ptrs)
        if rc != 0:
            raise EnvarError(f"envar_batch_forward: {ERRORS.get(rc, rc)}: {lib().envar_last_error(self.ens[0]._h).decode()}")

    def info(self):
        n = c_int()
        per = np.zeros(len(self.ens), dtype=np.int32)
        lib().envar_batch_info(self._b, ctypes.byref(n), _np_ptr(per))
        return n.value, per

    def close(self):
        if getattr(self, "_b", None):
            lib().envar_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def revolve_plan(n_steps: int, n_slots: int):
    """Dry run of the adjoint's checkpoint schedule (host only): recompute, stores, restores."""
    v = [ctypes.c_longlong() for _ in range(3)]
    rc = lib().envar_revolve_plan(int(n_steps), int(n_slots), *[ctypes.byref(x) for x in v])
    if rc != 0:
        raise EnvarError(f"envar_revolve_plan: {ERRORS.get(rc, rc)}")
    return dict(zip(("recompute", "stores", "restores"), (x.value for x in v)))


def _adjoint_cost_function():
    import torch

    class AdjointCost(torch.autograd.Function):
        """J(f) with backward by the discrete adjoint: forward runs envar_forward_control, backward
        envar_adjoint_gradient (which reruns the forward with checkpoints)."""

        @staticmethod
        def forward(ctx, f, ens, max_snapshots):
            ctx.ens, ctx.max_snapshots = ens, max_snapshots
            ctx.save_for_backward(f)
            J = ens.forward_control(f.detach())
            return torch.tensor(J, dtype=torch.float64, device=f.device)

        @staticmethod
        def backward(ctx, gJ):
            (f,) = ctx.saved_tensors
            _, g = ctx.ens.adjoint_gradient(f.detach(), ctx.max_snapshots)
            return gJ * g, None, None

    return AdjointCost


def adjoint_cost(f, ens: "Ensemble", max_snapshots: int = 64):
    """Differentiable DOMAIN cost of one forward run with control forcing f (float64, n_ctrl)."""
    return _adjoint_cost_function().apply(f, ens, max_snapshots)


def kernel_launches() -> int:
    n = ctypes.c_longlong()
    lib().envar_kernel_launches(None, ctypes.byref(n))
    return n.value


KERNELS = {0: "predict", 1: "mg_presmooth_restrict_l0", 2: "mg_prolong_postsmooth_dot_l0", 3: "cg_spmv",
           4: "cg_axpy", 5: "outer_residual_fp64", 6: "correct_welford", 7: "mg_coarse_block", 8: "poisson_rhs"}
