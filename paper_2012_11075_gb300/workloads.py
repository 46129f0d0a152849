"""Seeded synthetic inputs: initial density fields and parameter sets.

This module holds the problem statements only (lattice sizes, free-energy
parameters, initial density profiles, random case mixes).  It contains none
of the lattice Boltzmann arithmetic, so both the CUDA library's tests and the
CPU oracle can be fed from it.

Profiles follow Sec. IV of Guo, arXiv 2012.11075: a flat liquid/vapour slab
with the tanh profile of Eq. Tanh, and a circular droplet with the same
radial profile.  The interface width is W = sqrt(8 kappa / beta) /
(rho_l - rho_g); ``beta_for_width`` inverts it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def beta_for_width(kappa: float, width: float, rho_l: float, rho_g: float) -> float:
    return 8.0 * kappa / (width * (rho_l - rho_g)) ** 2


@dataclass
class Problem:
    """One case: lattice, physical parameters and the initial density."""
    nx: int
    ny: int
    tau: float
    kappa: float
    beta: float
    rho_l: float
    rho_g: float
    rho: np.ndarray = field(repr=False)
    rho0: float = 0.0
    name: str = ""


def slab_profile(ny: int, rho_l: float, rho_g: float, width: float,
                 centre: float, half: float) -> np.ndarray:
    """rho(y) = rho_m + (Delta/2) tanh(2(|y - centre| - half)/W): vapour in the
    band |y - centre| < half, liquid outside, two interfaces."""
    y = np.arange(ny, dtype=np.float64)
    rm, d = 0.5 * (rho_l + rho_g), rho_l - rho_g
    return rm + 0.5 * d * np.tanh(2.0 * (np.abs(y - centre) - half) / width)


def flat_interface(nx=4, ny=256, rho_l=1.0, rho_g=0.1, kappa=0.01, width=4.0,
                   tau=0.8) -> Problem:
    """Flat two-interface slab: rho(y) = 0.55 + 0.45 tanh(2(|y-128|-64)/W) at
    the default sizes (periodic D2Q9 4 x 256, W = 4, tau = 0.8)."""
    prof = slab_profile(ny, rho_l, rho_g, width, ny / 2, ny / 4)
    rho = np.repeat(prof[:, None], nx, axis=1).copy()
    return Problem(nx, ny, tau, kappa, beta_for_width(kappa, width, rho_l, rho_g),
                   rho_l, rho_g, rho, name=f"flat_{nx}x{ny}")


def paper_flat(seed=2012, eps=0.01) -> Problem:
    """The 1D flat-interface run of Sec. IV.A: 21 x 101 periodic, liquid in
    25 <= y <= 75, rho_l = 1, rho_v = 0.2, beta = 0.01, kappa = 0.0128,
    tau = 0.85, tanh profile (Eq. Tanh) times (1 + eps r), r ~ U(-1, 1)."""
    nx, ny, rho_l, rho_g, beta, kappa = 21, 101, 1.0, 0.2, 0.01, 0.0128
    width = math.sqrt(8 * kappa / beta) / (rho_l - rho_g)
    y = np.arange(ny, dtype=np.float64)
    prof = rho_g + 0.5 * (rho_l - rho_g) * (np.tanh(2 * (y - 25) / width)
                                            - np.tanh(2 * (y - 75) / width))
    rng = np.random.default_rng(seed)
    r = rng.uniform(-1.0, 1.0, size=(ny, nx))
    rho = prof[:, None] * (1.0 + eps * r)
    return Problem(nx, ny, 0.85, kappa, beta, rho_l, rho_g, rho, name="paper_flat_21x101")


def droplet_field(nx: int, ny: int, centres, radii, rho_l: float, rho_g: float,
                  width: float) -> np.ndarray:
    """Liquid droplets in vapour.  Each node takes the profile
    rho_m - (Delta/2) tanh(2(r - R)/W) of the droplet whose surface is
    nearest (largest density), r the minimum-image periodic distance."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    rm, d = 0.5 * (rho_l + rho_g), rho_l - rho_g
    rho = np.full((ny, nx), rho_g, dtype=np.float64)
    for (cx, cy), R in zip(centres, radii):
        dx = np.abs(x - cx)
        dx = np.minimum(dx, nx - dx)
        dy = np.abs(y - cy)
        dy = np.minimum(dy, ny - dy)
        r = np.sqrt(dx * dx + dy * dy)
        rho = np.maximum(rho, rm - 0.5 * d * np.tanh(2.0 * (r - R) / width))
    return rho


def droplet(n=256, radius=40.0, tau=1.0, rho_l=1.0, rho_g=0.1, kappa=0.01,
            width=4.0, nx=None, ny=None) -> Problem:
    """Stationary droplet centred at (nx//2, ny//2) (periodic D2Q9)."""
    nx = nx or n
    ny = ny or n
    rho = droplet_field(nx, ny, [(nx // 2, ny // 2)], [radius], rho_l, rho_g, width)
    return Problem(nx, ny, tau, kappa, beta_for_width(kappa, width, rho_l, rho_g),
                   rho_l, rho_g, rho, name=f"droplet_{nx}x{ny}_R{radius:g}")


def paper_droplet() -> Problem:
    """The droplet of Sec. IV.B: 100 x 100, R = 25, centred, parameters of
    Sec. IV.A (no perturbation)."""
    beta, kappa, rho_l, rho_g = 0.01, 0.0128, 1.0, 0.2
    width = math.sqrt(8 * kappa / beta) / (rho_l - rho_g)
    rho = droplet_field(100, 100, [(50, 50)], [25.0], rho_l, rho_g, width)
    return Problem(100, 100, 0.85, kappa, beta, rho_l, rho_g, rho, name="paper_droplet_100")


def random_droplets(n: int, count: int, rmin: float, rmax: float, width: float,
                    seed: int, max_tries: int = 200000):
    """Non-overlapping droplet centres/radii on an n x n periodic lattice:
    radii U[rmin, rmax], centres uniform, rejected unless every pair keeps a
    minimum-image gap >= R_a + R_b + 2W."""
    rng = np.random.default_rng(seed)
    centres, radii = [], []
    tries = 0
    while len(centres) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place droplets")
        R = rng.uniform(rmin, rmax)
        c = rng.uniform(0, n, size=2)
        ok = True
        for (px, py), pr in zip(centres, radii):
            dx = abs(c[0] - px); dx = min(dx, n - dx)
            dy = abs(c[1] - py); dy = min(dy, n - dy)
            if math.hypot(dx, dy) < R + pr + 2 * width:
                ok = False
                break
        if ok:
            centres.append((float(c[0]), float(c[1])))
            radii.append(float(R))
    return centres, radii


def large_domain(n=4096, count=64, ratio=10.0, width=5.0, kappa=0.01, tau=0.7,
                 seed=20121107) -> Problem:
    """Large-domain throughput case: n x n periodic, `count` droplets with
    radii U[16, 64] at seeded non-overlapping centres, rho_l = 1,
    rho_g = 1/ratio, kappa = 0.01, W = 5, tau = 0.7."""
    rho_l, rho_g = 1.0, 1.0 / ratio
    centres, radii = random_droplets(n, count, 16.0, 64.0, width, seed)
    rho = droplet_field(n, n, centres, radii, rho_l, rho_g, width)
    return Problem(n, n, tau, kappa, beta_for_width(kappa, width, rho_l, rho_g),
                   rho_l, rho_g, rho, name=f"droplets{count}_{n}x{n}_ratio{ratio:g}")


def batched_case_specs(count=512, seed=4, side_min=64, side_max=512):
    """Parameters of uneven independent cases, without their fields: sides
    log-uniform in [side_min, side_max] (independently in x and y), flat slab
    or droplet 50/50, radius/side U[0.1, 0.3], density ratio U[2, 50] with
    rho_l = 1, tau U[0.55, 1.2], kappa U[0.005, 0.02], W in {3, 4, 5}."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx = int(round(math.exp(rng.uniform(math.log(side_min), math.log(side_max)))))
        ny = int(round(math.exp(rng.uniform(math.log(side_min), math.log(side_max)))))
        kind = "flat" if rng.uniform() < 0.5 else "droplet"
        frac = rng.uniform(0.1, 0.3)
        ratio = rng.uniform(2.0, 50.0)
        tau = rng.uniform(0.55, 1.2)
        kappa = rng.uniform(0.005, 0.02)
        width = float(rng.choice([3.0, 4.0, 5.0]))
        out.append(dict(k=k, nx=nx, ny=ny, kind=kind, frac=frac, rho_l=1.0, rho_g=1.0 / ratio,
                        tau=tau, kappa=kappa, width=width,
                        beta=beta_for_width(kappa, width, 1.0, 1.0 / ratio)))
    return out


def case_field(spec) -> np.ndarray:
    """Initial density of a case spec (flat slab or centred droplet)."""
    nx, ny = spec["nx"], spec["ny"]
    if spec["kind"] == "flat":
        prof = slab_profile(ny, spec["rho_l"], spec["rho_g"], spec["width"], ny / 2,
                            spec["frac"] * ny)
        return np.repeat(prof[:, None], nx, axis=1).copy()
    R = spec["frac"] * min(nx, ny)
    return droplet_field(nx, ny, [(nx // 2, ny // 2)], [R], spec["rho_l"], spec["rho_g"],
                         spec["width"])


def case_problem(spec) -> Problem:
    return Problem(spec["nx"], spec["ny"], spec["tau"], spec["kappa"], spec["beta"],
                   spec["rho_l"], spec["rho_g"], case_field(spec),
                   name=f"case{spec['k']}_{spec['kind']}_{spec['nx']}x{spec['ny']}")


def batched_cases(count=512, seed=4, side_min=64, side_max=512):
    """The uneven case mix with fields (see batched_case_specs)."""
    return [case_problem(s) for s in batched_case_specs(count, seed, side_min, side_max)]
