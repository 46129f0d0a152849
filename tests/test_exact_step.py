"""An exact-rational restatement of the lattice update, pinning the FP64 oracle.

Independent of the oracle's C code: the update of Sec. II (standard LBE) and
Sec. III (well-balanced LBE) of Guo, arXiv 2012.11075 is written out again
here in ``fractions.Fraction`` arithmetic on tiny periodic lattices (3x3 and
two non-square ones, so the stencils wrap onto their own nodes and a swapped
x/y index shows).  Parameters and initial densities are binary fractions, so
``Fraction(float)`` gives the oracle's inputs exactly and the exact result
differs from the oracle's only by FP64 rounding.

Per node, in the paper's order:
  rho = sum_i f_i                                    (Eq. rhoU)
  mu  = dpsi0/drho - kappa L[rho],  psi0 = beta (rho-rho_l)^2 (rho-rho_g)^2
        (Eq. doubleWell; L the isotropic 9-point Laplacian)
  F   = -rho grad mu                 (WB, Eq. mF)
      = cs^2 grad rho - rho grad mu  (standard, potential form of Sec. II)
  u   = (sum_i c_i f_i + F/2) / rho  (Eq. rhoU)
  f^eq: Eq. mFeq (WB) / Eq. feq (standard, with the sign reading of the
        quadratic terms that the moment conditions require)
  F_i: Eq. mFi (WB, D = 2) / Eq. Fi (standard)
  f*_i = f_i - (f_i - f^eq_i)/tau + (1 - 1/(2 tau)) F_i, then f*_i moves to x + c_i
        (Eq. D2Q9, collision term with the relaxation sign).
Gradients are 3 sum_i w_i c_i phi(x + c_i), the Laplacian
6 sum_i w_i (phi(x + c_i) - phi(x)) (isotropic central scheme, cs^2 = 1/3).

The two variants of the standard LBE that Sec. II compares: the pressure-form
force F = grad(cs^2 rho - p_0) + kappa rho grad(lap rho) with
p_0 = rho mu_0 - psi_0 (the sign of the last term is the reading under which
the two forms agree, as the paper states they do), and the forcing term of
Guo's textbook F_i = (c_i - u).F f_i^eq / (cs^2 rho); and the radius-2
gradient for F whose weights (4/15, 1/10, 1/120 on the shells |e|^2 = 1, 2,
4) make the lattice moments isotropic to sixth order.
"""
from fractions import Fraction as Q

import numpy as np
import pytest

from oracle.oracle import (STANDARD, STANDARD_E6, STANDARD_PRESSURE, STANDARD_TEXTBOOK,
                           WELL_BALANCED, Oracle, Params)

C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
WT = [Q(4, 9)] + [Q(1, 9)] * 4 + [Q(1, 36)] * 4
CS2 = Q(1, 3)


def _at(phi, x, y):
    ny, nx = len(phi), len(phi[0])
    return phi[y % ny][x % nx]


def _grad(phi, x, y):
    gx = sum(WT[i] * cx * _at(phi, x + cx, y + cy) for i, (cx, cy) in enumerate(C)) / CS2
    gy = sum(WT[i] * cy * _at(phi, x + cx, y + cy) for i, (cx, cy) in enumerate(C)) / CS2
    return gx, gy


E6 = [((1, 0), Q(4, 15)), ((0, 1), Q(4, 15)), ((-1, 0), Q(4, 15)), ((0, -1), Q(4, 15)),
      ((1, 1), Q(1, 10)), ((-1, 1), Q(1, 10)), ((-1, -1), Q(1, 10)), ((1, -1), Q(1, 10)),
      ((2, 0), Q(1, 120)), ((0, 2), Q(1, 120)), ((-2, 0), Q(1, 120)), ((0, -2), Q(1, 120))]


def _grad6(phi, x, y):
    gx = sum(w * ex * _at(phi, x + ex, y + ey) for (ex, ey), w in E6)
    gy = sum(w * ey * _at(phi, x + ex, y + ey) for (ex, ey), w in E6)
    return gx, gy


def _lap(phi, x, y):
    return 2 / CS2 * sum(WT[i] * (_at(phi, x + cx, y + cy) - phi[y][x])
                         for i, (cx, cy) in enumerate(C))


def _feq(wb, rho0, rho, ux, uy):
    uu = ux * ux + uy * uy
    out = []
    for i, (cx, cy) in enumerate(C):
        cu = cx * ux + cy * uy
        poly = cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2)
        if not wb:
            out.append(WT[i] * rho * (1 + poly))
        elif i == 0:
            out.append(rho - (1 - WT[0]) * rho0 - WT[0] * rho * uu / (2 * CS2))
        else:
            out.append(WT[i] * (rho0 + rho * poly))
    return out


def _forcing(wb, ux, uy, Fx, Fy, grx, gry):
    # (u G):(c c - cs^2 I) = (c.u)(c.G) - cs^2 u.G
    Gx, Gy = (Fx + CS2 * grx, Fy + CS2 * gry) if wb else (Fx, Fy)
    out = []
    for i, (cx, cy) in enumerate(C):
        cu, cF, cG = cx * ux + cy * uy, cx * Fx + cy * Fy, cx * Gx + cy * Gy
        t = cF / CS2 + (cu * cG - CS2 * (ux * Gx + uy * Gy)) / (CS2 * CS2)
        if wb:
            t += Q(1, 2) * ((cx * cx + cy * cy) / CS2 - 2) * (ux * grx + uy * gry)
        out.append(WT[i] * t)
    return out


def exact_init(rho, wb, rho0):
    ny, nx = len(rho), len(rho[0])
    f = [[[None] * nx for _ in range(ny)] for _ in range(9)]
    for y in range(ny):
        for x in range(nx):
            for i, v in enumerate(_feq(wb, rho0, rho[y][x], Q(0), Q(0))):
                f[i][y][x] = v
    return f


def _forcing_textbook(rho, ux, uy, Fx, Fy):
    feq = _feq(False, 0, rho, ux, uy)
    return [((cx - ux) * Fx + (cy - uy) * Fy) * feq[i] / (CS2 * rho)
            for i, (cx, cy) in enumerate(C)]


def exact_step(f, tau, kappa, beta, rl, rg, rho0, wb, variant=None):
    ny, nx = len(f[0]), len(f[0][0])
    rho = [[sum(f[i][y][x] for i in range(9)) for x in range(nx)] for y in range(ny)]
    mu = [[2 * beta * (r - rl) * (r - rg) * (2 * r - rl - rg) - kappa * _lap(rho, x, y)
           for x, r in enumerate(row)] for y, row in enumerate(rho)]
    if variant == "pressure":
        def p0(r):
            psi = beta * (r - rl) ** 2 * (r - rg) ** 2
            return r * 2 * beta * (r - rl) * (r - rg) * (2 * r - rl - rg) - psi
        A = [[CS2 * r - p0(r) for r in row] for row in rho]
        lap = [[_lap(rho, x, y) for x in range(nx)] for y in range(ny)]
    out = [[[None] * nx for _ in range(ny)] for _ in range(9)]
    for y in range(ny):
        for x in range(nx):
            r = rho[y][x]
            grad = _grad6 if variant == "e6" else _grad
            gmx, gmy = grad(mu, x, y)
            grx, gry = grad(rho, x, y)
            Fx, Fy = -r * gmx, -r * gmy
            if not wb:
                Fx, Fy = Fx + CS2 * grx, Fy + CS2 * gry
            if variant == "pressure":
                gAx, gAy = _grad(A, x, y)
                gLx, gLy = _grad(lap, x, y)
                Fx, Fy = gAx + kappa * r * gLx, gAy + kappa * r * gLy
            jx = sum(cx * f[i][y][x] for i, (cx, _) in enumerate(C))
            jy = sum(cy * f[i][y][x] for i, (_, cy) in enumerate(C))
            ux, uy = (jx + Fx / 2) / r, (jy + Fy / 2) / r
            feq = _feq(wb, rho0, r, ux, uy)
            if variant == "textbook":
                Fi = _forcing_textbook(r, ux, uy, Fx, Fy)
            else:
                Fi = _forcing(wb, ux, uy, Fx, Fy, grx, gry)
            for i, (cx, cy) in enumerate(C):
                post = f[i][y][x] - (f[i][y][x] - feq[i]) / tau + (1 - 1 / (2 * tau)) * Fi[i]
                out[i][(y + cy) % ny][(x + cx) % nx] = post
    return out


def _as_float(f):
    return np.array([[[float(v) for v in row] for row in plane] for plane in f])


CASES = [
    # nx, ny, scheme, rho0, tau
    (3, 3, WELL_BALANCED, 0.0, 0.75),
    (3, 3, STANDARD, 0.0, 0.75),
    (4, 3, WELL_BALANCED, 0.375, 1.25),
    (3, 5, STANDARD, 0.0, 0.625),
    (3, 5, WELL_BALANCED, 0.0, 2.0),
    (3, 3, STANDARD_PRESSURE, 0.0, 0.75),
    (4, 3, STANDARD_PRESSURE, 0.0, 1.25),
    (3, 3, STANDARD_TEXTBOOK, 0.0, 0.75),
    (3, 5, STANDARD_TEXTBOOK, 0.0, 0.625),
    (5, 5, STANDARD_E6, 0.0, 0.75),
    (3, 6, STANDARD_E6, 0.0, 1.25),
]
VARIANT = {STANDARD_PRESSURE: "pressure", STANDARD_TEXTBOOK: "textbook", STANDARD_E6: "e6"}


@pytest.mark.parametrize("nx,ny,scheme,rho0,tau", CASES)
def test_oracle_matches_exact_rational_steps(nx, ny, scheme, rho0, tau):
    kappa, beta, rl, rg = 0.015625, 0.0078125, 1.0, 0.125
    rng = np.random.default_rng(100 + nx * 10 + ny + 7 * scheme)
    # binary-fraction densities in [rho_g, rho_l]: exactly representable
    rho_f = (8 + rng.integers(0, 57, size=(ny, nx))) / 64.0
    rho_q = [[Q(float(v)) for v in row] for row in rho_f]
    wb = scheme == WELL_BALANCED
    p = Params(nx, ny, tau, kappa, beta, rl, rg, rho0=rho0, scheme=scheme)
    orc = Oracle(p)

    f = orc.init(rho_f)
    fq = exact_init(rho_q, wb, Q(rho0))
    # one rounding of w_i rho (the weights are not binary fractions)
    np.testing.assert_allclose(f, _as_float(fq), rtol=2.3e-16, atol=0)

    args = (Q(tau), Q(kappa), Q(beta), Q(rl), Q(rg), Q(rho0), wb, VARIANT.get(scheme))
    # the textbook term divides by rho each step, which makes the exact
    # denominators grow fast: two steps there (u != 0 from the first on)
    for step in range(2 if scheme == STANDARD_TEXTBOOK else 3):
        fq = exact_step(fq, *args)
        orc.step(f, 1)
        fe = _as_float(fq)
        scale = np.abs(fe).max()
        err = np.abs(f - fe).max() / scale
        assert err < 1e-14, (step, err)
    # the exact update conserves mass exactly
    total0 = sum(sum(row) for row in rho_q)
    total = sum(fq[i][y][x] for i in range(9) for y in range(ny) for x in range(nx))
    assert total == total0
