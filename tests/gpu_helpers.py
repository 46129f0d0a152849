"""Shared helpers of the GPU parity tests: run one case through the CUDA
library (C ABI) and through the CPU oracle on the same seeded input."""
from __future__ import annotations

import numpy as np
import pytest

from oracle.oracle import Oracle, Params as OParams
from paper_2012_11075_gb300 import wblbe


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_params(pr, scheme, precision=wblbe.FP64, rho0=0.0, rho_ref=float("nan")):
    return wblbe.Params(pr.nx, pr.ny, pr.tau, pr.kappa, pr.beta, pr.rho_l, pr.rho_g,
                        rho0=rho0, rho_ref=rho_ref, scheme=scheme, precision=precision)


def run_gpu(pr, scheme, steps, precision=wblbe.FP64, launch=None, rho0=0.0, rho=None):
    s = wblbe.Solver(gpu_params(pr, scheme, precision, rho0))
    if launch is not None:
        s.set_launch(*launch)
    s.init_rho(pr.rho if rho is None else rho)
    s.step(steps)
    f = s.get_populations()
    mom, st = s.moments()
    s.close()
    return f, mom, st


def run_oracle(pr, scheme, steps, rho0=0.0, rho=None):
    o = Oracle(OParams(pr.nx, pr.ny, pr.tau, pr.kappa, pr.beta, pr.rho_l, pr.rho_g, rho0, scheme))
    f = o.init(pr.rho if rho is None else rho)
    o.step(f, steps)
    return f, o.macro(f), o.stats(f)


def pop_error(f_gpu, f_orc):
    """max_x,i |df| / max_x,i |f| (global) and the worst per-direction
    max_x |df_i| / max_x |f_i|, taken over the directions whose largest
    population exceeds 1e-6 of the overall largest.  A direction below that
    floor (a well-balanced moving population that is still zero or at
    round-off level, e.g. in a state at rest) has no scale of its own; its
    error is bounded by the global norm."""
    scale = np.max(np.abs(f_orc))
    glob = np.max(np.abs(f_gpu - f_orc)) / scale
    per = 0.0
    for i in range(9):
        s = np.max(np.abs(f_orc[i]))
        if s > 1e-6 * scale:
            per = max(per, np.max(np.abs(f_gpu[i] - f_orc[i])) / s)
    return glob, per
