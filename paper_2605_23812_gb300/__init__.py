"""GB300 (sm_103a) ensemble-variational open-loop control of an open-cavity flow.

The hot path of arXiv 2605.23812 -- N+1 forced Navier-Stokes cavity runs, their
fluctuation-energy costs and the EnVar gradient -- runs in the CUDA kernels of
``libenvar_gb300.so`` behind the C ABI of ``include/envar.h``.  ``capi`` is the
thin ctypes binding (with ``adjoint_cost``, a torch autograd function whose
backward is the discrete adjoint); ``synth`` holds the seeded synthetic inputs.
"""
from .capi import (COST_DOMAIN, COST_SENSORS, FP64_BATCHED, FP64_PLAIN, MIXED, ST_ADJOINT, ST_CFL, ST_DIVERGENCE,
                   ST_NONFINITE, Batch, Config, Ensemble, EnvarError, adjoint_cost, default_config, header_symbols, lib,
                   revolve_plan)

__all__ = ["Batch", "Config", "Ensemble", "EnvarError", "adjoint_cost", "default_config", "header_symbols", "lib",
           "revolve_plan", "FP64_PLAIN", "FP64_BATCHED", "MIXED", "COST_DOMAIN", "COST_SENSORS", "ST_NONFINITE",
           "ST_DIVERGENCE", "ST_CFL", "ST_ADJOINT"]
