"""Closed forms and an LBE-free solver for the equilibrium state of Sec. I/IV.

TEST INFRASTRUCTURE ONLY (see ``oracle.py``).  Nothing here runs the lattice
Boltzmann update: these are the independent references that the oracle's
converged states are pinned to.

* ``coexistence``: the saturation densities of the double well (Eq. doubleWell)
  are its two minima, where mu_0 = 0 and p_0 = 0 (Eq. EOS).
* ``interface_width``, ``beta_for_width``: the flat-interface solution of
  kappa rho'^2 / 2 = psi_0 is the tanh profile of Eq. Tanh with width
  W = sqrt(8 kappa / beta) / (rho_l - rho_v).
* ``surface_tension``: sigma = (rho_l - rho_v)^3 sqrt(2 beta kappa) / 6
  (Sec. IV.B), the excess free energy of that profile.
* ``discrete_flat_equilibrium``: the discrete equilibrium state
  S = {mu = const, u = 0} of Sec. I for a density that varies along y only,
  with mu discretised by the same 3-point Laplacian the 2D isotropic stencil
  reduces to, found by Newton's method at fixed mass.  It does not use the
  LBE at all.
"""
from __future__ import annotations

import numpy as np


def psi0(rho, beta, rho_l, rho_g):
    """Eq. doubleWell."""
    return beta * (rho - rho_l) ** 2 * (rho - rho_g) ** 2


def mu0(rho, beta, rho_l, rho_g):
    """d psi0 / d rho, expanded."""
    return 2.0 * beta * (rho - rho_l) * (rho - rho_g) * (2.0 * rho - rho_l - rho_g)


def dmu0(rho, beta, rho_l, rho_g):
    """d^2 psi0 / d rho^2."""
    a, b = rho - rho_l, rho - rho_g
    return 2.0 * beta * (b * b + 4.0 * a * b + a * a)


def p0(rho, beta, rho_l, rho_g):
    """p_0 = rho mu_0 - psi_0 (Eq. EOS read with the factor rho)."""
    return rho * mu0(rho, beta, rho_l, rho_g) - psi0(rho, beta, rho_l, rho_g)


def beta_for_width(kappa, width, rho_l, rho_g):
    """beta such that sqrt(8 kappa / beta) / (rho_l - rho_g) = width."""
    return 8.0 * kappa / (width * (rho_l - rho_g)) ** 2


def interface_width(kappa, beta, rho_l, rho_g):
    return np.sqrt(8.0 * kappa / beta) / (rho_l - rho_g)


def surface_tension(kappa, beta, rho_l, rho_g):
    """sigma = (rho_l - rho_v)^3 sqrt(2 beta kappa) / 6 (Sec. IV.B)."""
    return (rho_l - rho_g) ** 3 * np.sqrt(2.0 * beta * kappa) / 6.0


def tanh_slab(y, y1, y2, width, rho_l, rho_g):
    """Eq. Tanh: liquid between y1 and y2, vapour outside (continuous solution)."""
    return rho_g + 0.5 * (rho_l - rho_g) * (np.tanh(2.0 * (y - y1) / width)
                                            - np.tanh(2.0 * (y - y2) / width))


def discrete_flat_equilibrium(rho_init, kappa, beta, rho_l, rho_g,
                              symmetric=True, tol=1e-15, max_iter=100):
    """Solve mu_0(rho_j) - kappa (rho_{j+1} - 2 rho_j + rho_{j-1}) = mu_bar,
    sum_j rho_j = sum_j rho_init_j on a periodic 1D lattice, by Newton's method
    started from rho_init.

    With ``symmetric`` the solution is sought among profiles with
    rho_j = rho_{-j} (mod N), which removes the translation mode a periodic
    slab has; rho_init must have that symmetry.  Returns (rho, mu_bar)."""
    r0 = np.asarray(rho_init, dtype=np.float64)
    n = r0.size
    mass = r0.sum()
    if symmetric:
        assert np.allclose(r0, r0[(-np.arange(n)) % n], atol=1e-14, rtol=0)
        m = n // 2 + 1                       # free unknowns rho_0 .. rho_{n//2}
        full_of = np.array([min(j, n - j) for j in range(n)])   # index map
    else:
        m = n
        full_of = np.arange(n)
    # expansion matrix E (n x m): rho_full = E @ rho_red
    E = np.zeros((n, m))
    E[np.arange(n), full_of] = 1.0
    # periodic 3-point Laplacian on the full lattice
    lap = -2.0 * np.eye(n) + np.roll(np.eye(n), 1, axis=1) + np.roll(np.eye(n), -1, axis=1)
    red = r0[:m].copy() if symmetric else r0.copy()
    mu_bar = float(np.mean(mu0(r0, beta, rho_l, rho_g) - kappa * lap @ r0))
    for _ in range(max_iter):
        rf = E @ red
        res = np.empty(n + 1)
        res[:n] = mu0(rf, beta, rho_l, rho_g) - kappa * (lap @ rf) - mu_bar
        res[n] = rf.sum() - mass
        J = np.zeros((n + 1, m + 1))
        J[:n, :m] = (np.diag(dmu0(rf, beta, rho_l, rho_g)) - kappa * lap) @ E
        J[:n, m] = -1.0
        J[n, :m] = E.sum(axis=0)
        # overdetermined when symmetric (mirror rows repeat): least squares
        delta = np.linalg.lstsq(J, -res, rcond=None)[0]
        red += delta[:m]
        mu_bar += delta[m]
        if np.max(np.abs(delta)) < tol:
            break
    return E @ red, mu_bar
