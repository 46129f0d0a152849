"""Stability map of the D2Q9 LBE over rho0, density ratio and tau.

Sec. III of Guo, arXiv 2012.11075 leaves the constant rho0 of the
well-balanced equilibrium (Eq. mFeq) free: it may change how stable the scheme
is, but not the equilibrium it reaches (the discrete balance of Sec. III does
not contain it).  This module runs a grid of stationary-droplet cases, one per
(rho0, density ratio, tau), as a single batch on the GPU and records for each
case whether it stayed finite for the whole step budget (and its final maximum
velocity) or after how many steps it became non-finite.

Every case: an n x n periodic lattice, one droplet of radius n/4 at the
centre with the tanh profile of Eq. Tanh, rho_l = 1, rho_g = 1/ratio,
interface width W (beta = 8 kappa / (W (rho_l - rho_g))^2).

The linear limit the map runs into is known in closed form.  Linearised
about a uniform rest state, the well-balanced update (Eq. mFeq, Eq. mFi,
BGK, streaming) leaves the density field that alternates along one lattice
axis (wave number pi) neutral: its central gradients vanish.  With a slow
modulation q along the other axis its eigenvalue becomes
1 + S (w^2 - 8 w + 8) / (6 w (w - 2)) q^2 + O(q^4), w = 1/tau,
S = rho (psi_0''(rho) + 4 kappa).  It grows for tau < (2 + sqrt 2) / 4,
whatever the free energy.
"""
from __future__ import annotations

import itertools
import math

from . import workloads as wl
from .wblbe import FP64, WELL_BALANCED, Batch, Params

RHO0_MODES = ("zero", "gas", "mean")
STATE_NAMES = {1: "converged", 2: "stable", 3: "unstable"}

# relaxation time below which the well-balanced scheme has a growing bulk mode
WB_TAU_LIMIT = 0.5 + math.sqrt(2.0) / 4.0


def bulk_mode_growth(tau: float, rho: float, d2psi: float, kappa: float, q: float) -> float:
    """|lambda| - 1 per step of the well-balanced bulk mode that alternates
    along one axis and is modulated with wave number q along the other, to
    second order in q, about a uniform rest state of density rho
    (d2psi = psi_0''(rho)).  Positive means growth."""
    w = 1.0 / tau
    s = rho * (d2psi + 4.0 * kappa)
    return s * (w * w - 8.0 * w + 8.0) / (6.0 * w * (w - 2.0)) * q * q


def rho0_value(mode: str, rho_l: float, rho_g: float) -> float:
    """rho0 for a named choice: 0 (the paper's), the gas density, the mean."""
    if mode == "zero":
        return 0.0
    if mode == "gas":
        return rho_g
    if mode == "mean":
        return 0.5 * (rho_l + rho_g)
    raise ValueError(f"unknown rho0 mode {mode!r}")


def grid(ratios, taus, rho0_modes=RHO0_MODES):
    return list(itertools.product(rho0_modes, ratios, taus))


def stability_map(ratios=(2.0, 5.0, 10.0, 20.0, 50.0),
                  taus=(0.55, 0.6, 0.7, 0.8, 0.85, 0.9, 1.0, 1.2),
                  rho0_modes=RHO0_MODES, n=128, steps=50000, width=4.0, kappa=0.01,
                  scheme=WELL_BALANCED, precision=FP64, steps_per_launch=50,
                  tile_x=64, rows_per_tile=32, stream=None):
    """Run every (rho0 mode, ratio, tau) case for ``steps`` lattice steps (or
    until it becomes non-finite) and return one record per case:
    {rho0_mode, rho0, ratio, tau, state ('stable' or 'unstable'), steps,
    umax, mass}.  ``steps`` is rounded up to whole launches.  Growth near
    the stability limit is slow (the WB droplet at tau = 0.8, W = 4, fails
    only between steps 15000 and 30000, depending on the density ratio),
    hence the default."""
    cases = grid(ratios, taus, rho0_modes)
    params = []
    for mode, ratio, tau in cases:
        rho_l, rho_g = 1.0, 1.0 / ratio
        beta = wl.beta_for_width(kappa, width, rho_l, rho_g)
        params.append(Params(n, n, tau, kappa, beta, rho_l, rho_g,
                             rho0=rho0_value(mode, rho_l, rho_g), scheme=scheme,
                             precision=precision))
    probe = Batch(scheme=scheme, precision=precision, max_cases=1, arena_bytes=1 << 20,
                  stream=stream)
    per_case = probe.case_bytes(params[0])
    probe.close()
    b = Batch(scheme=scheme, precision=precision, max_cases=len(cases),
              max_tiles=1 << 16, max_case_nodes=n * n,
              arena_bytes=int(per_case * len(cases) * 1.02) + (1 << 20), tile_x=tile_x,
              rows_per_tile=rows_per_tile, steps_per_launch=steps_per_launch, stream=stream)
    try:
        ids = []
        for (mode, ratio, tau), p in zip(cases, params):
            rho = wl.droplet_field(n, n, [(n // 2, n // 2)], [n / 4.0], p.rho_l, p.rho_g, width)
            cid = b.admit(p, rho, 0.0, steps)      # tolerance 0: never "converged"
            if cid is None:
                raise MemoryError("stability map: batch refused a case")
            ids.append(cid)
        while b.counts()["running"] > 0:
            b.advance(1)
        out = []
        for (mode, ratio, tau), p, cid in zip(cases, params, ids):
            info = b.info(cid)
            out.append({"rho0_mode": mode, "rho0": p.rho0, "ratio": ratio, "tau": tau,
                        "state": STATE_NAMES.get(info["state"], str(info["state"])),
                        "steps": info["steps"], "umax": info["stats"]["umax"],
                        "mass": info["stats"]["mass"]})
        return out
    finally:
        b.close()


def format_table(records) -> str:
    """Text table: one block per rho0 mode, ratios as rows, taus as columns;
    a cell is the final max|u| of a stable case or 'x@steps' for an
    unstable one."""
    modes = sorted({r["rho0_mode"] for r in records}, key=RHO0_MODES.index)
    ratios = sorted({r["ratio"] for r in records})
    taus = sorted({r["tau"] for r in records})
    by = {(r["rho0_mode"], r["ratio"], r["tau"]): r for r in records}
    lines = []
    for m in modes:
        lines.append(f"rho0 = {m}")
        lines.append("ratio  " + "".join(f"{t:>12g}" for t in taus))
        for q in ratios:
            cells = []
            for t in taus:
                r = by.get((m, q, t))
                if r is None:
                    cells.append(f"{'-':>12}")
                elif r["state"] == "unstable":
                    cells.append(f"{'x@' + str(r['steps']):>12}")
                else:
                    cells.append(f"{r['umax']:12.2e}")
            lines.append(f"{q:<7g}" + "".join(cells))
    return "\n".join(lines)
