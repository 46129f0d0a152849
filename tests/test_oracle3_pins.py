"""Pins of the three-dimensional (D3Q19) FP64 oracle to what the paper and
the mathematics fix.

The paper's construction (Sec. III) is written for any dimension D: the
well-balanced equilibrium of Eq. mFeq, F = -rho grad(mu) of Eq. mF and the
forcing term of Eq. mFi, whose isotropic term carries D.  Pinned here:
  * the lattice moments of D3Q19 up to fourth order (what the moment
    identities need);
  * the moment identities of Sec. III with D = 3 (WB) and of Sec. II
    (standard) at random states;
  * the stencils: exact on quadratics, reducing to the 1D central forms on
    fields that vary along one axis;
  * uniform states (rest, uniform flow) are fixed points; mass is conserved;
    axis permutations and mirrors commute with the update;
  * a flat interface along one axis relaxes, in the WB scheme, to the
    LBE-free discrete equilibrium mu = const of the 1D problem (the same
    Newton solution as in 2D, since the 3D stencils reduce to 1D);
  * one to two steps against an exact-rational restatement of the update
    (``fractions.Fraction``) on tiny periodic lattices;
  * the FP64 conditioning of the WB moving populations (the oracle against
    its build that sums rho in pairs), as for D2Q9.
"""
from fractions import Fraction as Q

import numpy as np
import pytest

from oracle import equilibrium as eq
from oracle import oracle3 as o3

CX, CY, CZ, W = o3.lattice()
C3 = list(zip(CX.tolist(), CY.tolist(), CZ.tolist()))
CS2 = 1.0 / 3.0


def _params(**kw):
    base = dict(nx=6, ny=5, nz=4, tau=0.85, kappa=0.0128, beta=0.01, rho_l=1.0, rho_g=0.2,
                rho0=0.0, scheme=o3.WELL_BALANCED)
    base.update(kw)
    return o3.Params(**base)


def test_d3q19_lattice_moments():
    c = np.stack([CX, CY, CZ], axis=1).astype(float)
    assert len(set(C3)) == 19 and C3[0] == (0, 0, 0)
    assert abs(W.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", W, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", W, c, c), CS2 * np.eye(3), atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", W, c, c, c), 0, atol=1e-16)
    d = np.eye(3)
    want4 = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                        + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", W, c, c, c, c), want4, atol=1e-16)
    opp = [C3.index((-x, -y, -z)) for (x, y, z) in C3]
    assert all(W[i] == W[opp[i]] for i in range(19))


@pytest.mark.parametrize("rho0", [0.0, 0.37])
def test_well_balanced_moment_identities_d3(rho0):
    """Sec. III with D = 3: sum f^eq = rho, sum c f^eq = rho u,
    sum c c f^eq = rho u u (no pressure: the WB equilibrium carries none),
    sum c c c f^eq = cs^2 rho [u I]; sum F_i = 0, sum c F_i = F,
    sum c c F_i = [u F] + cs^2 ([u grad rho] + (u . grad rho) I)."""
    o = o3.Oracle3(_params(rho0=rho0))
    c = np.stack([CX, CY, CZ], axis=1).astype(float)
    rng = np.random.default_rng(3)
    for _ in range(20):
        rho = rng.uniform(0.05, 1.2)
        u = rng.uniform(-0.1, 0.1, 3)
        F = rng.uniform(-0.01, 0.01, 3)
        g = rng.uniform(-0.2, 0.2, 3)
        fe = o.feq(rho, u)
        Fi = o.forcing(u, F, g)
        d = np.eye(3)
        tol = 1e-15
        assert abs(fe.sum() - rho) < tol
        assert np.allclose(c.T @ fe, rho * u, atol=tol)
        assert np.allclose(np.einsum("i,ia,ib->ab", fe, c, c), rho * np.outer(u, u) +
                           rho0 * CS2 * d, atol=tol)
        uI = (np.einsum("a,bc->abc", u, d) + np.einsum("b,ac->abc", u, d)
              + np.einsum("c,ab->abc", u, d))
        assert np.allclose(np.einsum("i,ia,ib,ic->abc", fe, c, c, c), CS2 * rho * uI, atol=tol)
        assert abs(Fi.sum()) < tol
        assert np.allclose(c.T @ Fi, F, atol=tol)
        want = (np.outer(u, F) + np.outer(F, u)
                + CS2 * (np.outer(u, g) + np.outer(g, u) + (u @ g) * d))
        assert np.allclose(np.einsum("i,ia,ib->ab", Fi, c, c), want, atol=tol)


def test_standard_moment_identities_d3():
    o = o3.Oracle3(_params(scheme=o3.STANDARD))
    c = np.stack([CX, CY, CZ], axis=1).astype(float)
    rng = np.random.default_rng(4)
    for _ in range(10):
        rho = rng.uniform(0.05, 1.2)
        u = rng.uniform(-0.1, 0.1, 3)
        F = rng.uniform(-0.01, 0.01, 3)
        fe, Fi = o.feq(rho, u), o.forcing(u, F, np.zeros(3))
        assert abs(fe.sum() - rho) < 1e-15
        assert np.allclose(np.einsum("i,ia,ib->ab", fe, c, c),
                           rho * np.outer(u, u) + CS2 * rho * np.eye(3), atol=1e-15)
        assert abs(Fi.sum()) < 1e-15 and np.allclose(c.T @ Fi, F, atol=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", Fi, c, c),
                           np.outer(u, F) + np.outer(F, u), atol=1e-15)


def test_stencils_exact_on_quadratics_and_reduce_to_1d():
    p = _params(nx=7, ny=6, nz=5)
    o = o3.Oracle3(p)
    z, y, x = np.meshgrid(np.arange(5), np.arange(6), np.arange(7), indexing="ij")
    # periodic quadratics are not periodic: test at an interior node of a
    # field that is a quadratic around it
    phi = 0.3 + 0.1 * x - 0.2 * y + 0.05 * z + 0.01 * x * x + 0.02 * y * z - 0.03 * z * z
    lap = o.laplacian(phi)
    gx, gy, gz = o.gradient(phi)
    k = (2, 3, 3)
    X, Y, Z = 3, 3, 2
    assert abs(lap[k] - (0.02 - 0.06)) < 1e-13
    assert abs(gx[k] - (0.1 + 0.02 * X)) < 1e-13
    assert abs(gy[k] - (-0.2 + 0.02 * Z)) < 1e-13
    assert abs(gz[k] - (0.05 + 0.02 * Y - 0.06 * Z)) < 1e-13
    # a field varying along x only: the 3-point Laplacian and central difference
    s = np.sin(2 * np.pi * np.arange(7) / 7)
    phi = np.broadcast_to(s, (5, 6, 7)).copy()
    lap, (gx, gy, gz) = o.laplacian(phi), o.gradient(phi)
    assert np.allclose(lap[0, 0], np.roll(s, -1) + np.roll(s, 1) - 2 * s, atol=1e-15)
    assert np.allclose(gx[0, 0], (np.roll(s, -1) - np.roll(s, 1)) / 2, atol=1e-15)
    assert np.allclose(gy, 0, atol=1e-16) and np.allclose(gz, 0, atol=1e-16)


@pytest.mark.parametrize("scheme", [o3.STANDARD, o3.WELL_BALANCED])
def test_uniform_states_fixed_and_mass_conserved(scheme):
    p = _params(scheme=scheme, rho0=0.3 if scheme == o3.WELL_BALANCED else 0.0)
    o = o3.Oracle3(p)
    f = o.init(np.full((4, 5, 6), 0.7))
    f0 = f.copy()
    o.step(f, 20)
    assert np.max(np.abs(f - f0)) < 1e-14          # rho = sum of 19 rounds by an ulp
    # uniform flow: f^eq at a uniform u is preserved (F = 0)
    u = np.array([0.03, -0.02, 0.01])
    fe = o.feq(0.7, u)
    f = np.broadcast_to(fe[:, None, None, None], (19, 4, 5, 6)).copy()
    g = f.copy()
    o.step(g, 10)
    assert np.max(np.abs(g - f)) < 1e-14
    # mass on a random field
    rng = np.random.default_rng(5)
    f = o.init(0.6 + 0.3 * rng.uniform(-1, 1, (4, 5, 6)))
    m0 = o.stats(f)["mass"]
    o.step(f, 200)
    assert abs(o.stats(f)["mass"] - m0) < 1e-13 * m0


@pytest.mark.parametrize("scheme", [o3.STANDARD, o3.WELL_BALANCED])
def test_axis_permutations_and_mirrors_commute(scheme):
    o = o3.Oracle3(_params(scheme=scheme, nx=5, ny=5, nz=5))
    rng = np.random.default_rng(6)
    rho = 0.6 + 0.3 * rng.uniform(-1, 1, (5, 5, 5))
    base = o.init(rho)
    o.step(base, 7)

    def transform(f, perm, flip):
        # a field transform and the matching permutation of the directions
        T = np.eye(3)[list(perm)] * np.array([-1 if fl else 1 for fl in flip])[:, None]
        out = np.empty_like(f)
        for i, c in enumerate(C3):
            j = C3.index(tuple(int(v) for v in T @ np.array(c)))
            g = f[i]                                    # axes (z, y, x)
            g = np.transpose(g, [2 - a for a in perm][::-1])
            for ax, fl in enumerate(flip):
                if fl:
                    g = np.flip(g, axis=2 - ax)
                    g = np.roll(g, 1, axis=2 - ax)
            out[j] = g
        return out

    for perm, flip in (((1, 0, 2), (0, 0, 0)), ((2, 1, 0), (0, 0, 0)), ((0, 1, 2), (1, 0, 0)),
                       ((0, 1, 2), (0, 1, 1))):
        f = transform(o.init(rho), perm, flip)
        o.step(f, 7)
        assert np.max(np.abs(f - transform(base, perm, flip))) < 1e-14, (perm, flip)


def test_wb_flat_interface_reaches_discrete_equilibrium():
    """A slab along x (nx = 21, one node in y and z): the WB scheme relaxes to
    the Newton solution of mu_0(rho_j) - kappa (rho_j+1 - 2 rho_j + rho_j-1)
    = const, sum rho fixed (the 3D stencils reduce to the 1D ones)."""
    n = 21
    xs = np.arange(n, dtype=float)
    d = np.minimum(xs, n - xs)
    prof = 0.55 + 0.45 * np.tanh(2 * (d - n / 4) / 4.0)
    beta = eq.beta_for_width(0.01, 4.0, 1.0, 0.1)
    p = o3.Params(n, 1, 1, 0.8, 0.01, beta, 1.0, 0.1, 0.0, o3.WELL_BALANCED)
    o = o3.Oracle3(p)
    f = o.init(prof[None, None, :].copy())
    o.step(f, 40000)
    m = o.macro(f)
    rN, _ = eq.discrete_flat_equilibrium(prof, 0.01, beta, 1.0, 0.1)
    assert np.max(np.abs(m["rho"][0, 0] - rN)) < 1e-10
    assert np.max(np.abs(m["u"])) < 1e-13


# ---- exact-rational restatement of one step (independent of the C code) ----

WQ = [Q(1, 3)] + [Q(1, 18)] * 6 + [Q(1, 36)] * 12
QCS2 = Q(1, 3)


def _at(phi, x, y, z):
    nz, ny, nx = len(phi), len(phi[0]), len(phi[0][0])
    return phi[z % nz][y % ny][x % nx]


def _exact_step(f, tau, kappa, beta, rl, rg, rho0, wb):
    nz, ny, nx = len(f[0]), len(f[0][0]), len(f[0][0][0])
    R = range
    rho = [[[sum(f[i][z][y][x] for i in R(19)) for x in R(nx)] for y in R(ny)] for z in R(nz)]

    def lap(phi, x, y, z):
        return 2 / QCS2 * sum(WQ[i] * (_at(phi, x + cx, y + cy, z + cz) - phi[z][y][x])
                              for i, (cx, cy, cz) in enumerate(C3))

    def grad(phi, x, y, z):
        return [sum(WQ[i] * c[a] * _at(phi, x + c[0], y + c[1], z + c[2])
                    for i, c in enumerate(C3)) / QCS2 for a in R(3)]

    def mu0(r):
        a, b = r - rl, r - rg
        return 2 * beta * a * b * b + 2 * beta * a * a * b

    mu = [[[mu0(rho[z][y][x]) - kappa * lap(rho, x, y, z) for x in R(nx)] for y in R(ny)]
          for z in R(nz)]
    out = [[[[None] * nx for _ in R(ny)] for _ in R(nz)] for _ in R(19)]
    om, kf = 1 / tau, 1 - 1 / (2 * tau)
    for z in R(nz):
        for y in R(ny):
            for x in R(nx):
                r = rho[z][y][x]
                gm, gr = grad(mu, x, y, z), grad(rho, x, y, z)
                F = [-r * gm[a] if wb else QCS2 * gr[a] - r * gm[a] for a in R(3)]
                j = [sum(C3[i][a] * f[i][z][y][x] for i in R(19)) for a in R(3)]
                u = [(j[a] + F[a] / 2) / r for a in R(3)]
                uu = sum(v * v for v in u)
                G = [F[a] + QCS2 * gr[a] for a in R(3)] if wb else F
                ug = sum(u[a] * gr[a] for a in R(3))
                for i, c in enumerate(C3):
                    cu = sum(c[a] * u[a] for a in R(3))
                    poly = cu / QCS2 + cu * cu / (2 * QCS2 * QCS2) - uu / (2 * QCS2)
                    if not wb:
                        fe = WQ[i] * r * (1 + poly)
                    elif i == 0:
                        fe = r - (1 - WQ[0]) * rho0 - WQ[0] * r * uu / (2 * QCS2)
                    else:
                        fe = WQ[i] * (rho0 + r * poly)
                    cF = sum(c[a] * F[a] for a in R(3))
                    cG = sum(c[a] * G[a] for a in R(3))
                    uG = sum(u[a] * G[a] for a in R(3))
                    t = cF / QCS2 + (cu * cG - QCS2 * uG) / (QCS2 * QCS2)
                    if wb:
                        t += Q(1, 2) * (sum(v * v for v in c) / QCS2 - 3) * ug
                    fi = f[i][z][y][x]
                    out[i][(z + c[2]) % nz][(y + c[1]) % ny][(x + c[0]) % nx] = \
                        fi - om * (fi - fe) + kf * WQ[i] * t
    return out


@pytest.mark.parametrize("scheme,rho0,shape", [(o3.WELL_BALANCED, 0.0, (3, 3, 3)),
                                               (o3.WELL_BALANCED, 0.5, (4, 3, 2)),
                                               (o3.STANDARD, 0.0, (2, 3, 4))])
def test_two_steps_against_exact_rational_restatement(scheme, rho0, shape):
    nz, ny, nx = shape
    tau, kappa, beta, rl, rg = Q(4, 5), Q(1, 128), Q(1, 64), Q(1), Q(1, 8)
    rho = [[[Q(1) - Q(3, 8) * Q((x + 2 * y + 3 * z) % 5, 4) for x in range(nx)]
            for y in range(ny)] for z in range(nz)]
    wb = scheme == o3.WELL_BALANCED
    p = o3.Params(nx, ny, nz, float(tau), float(kappa), float(beta), float(rl), float(rg),
                  rho0, scheme)
    o = o3.Oracle3(p)
    f = o.init(np.array([[[float(v) for v in row] for row in sl] for sl in rho]))
    # the exact initial state is f^eq(rho, 0): rational, and equal to the oracle's
    fq = [[[[Q(v) for v in row] for row in sl] for sl in f[i]] for i in range(19)]
    for _ in range(2):
        fq = _exact_step(fq, tau, kappa, beta, rl, rg, Q(rho0), wb)
    o.step(f, 2)
    err = max(abs(float(fq[i][z][y][x]) - f[i, z, y, x]) for i in range(19)
              for z in range(nz) for y in range(ny) for x in range(nx))
    assert err < 1e-14, err


def test_fp64_conditioning_matches_d2q9_finding():
    """The oracle and its pairwise-density build: round-off level in the
    global norm after 500 WB steps of a 3D droplet, more than 1e-12 of their
    size on some moving populations."""
    n = 12
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2)
    beta = eq.beta_for_width(0.01, 4.0, 1.0, 0.1)
    rho = 0.55 - 0.45 * np.tanh(2 * (r - 3.5) / 4.0)
    p = o3.Params(n, n, n, 0.9, 0.01, beta, 1.0, 0.1, 0.0, o3.WELL_BALANCED)
    fs = []
    for pw in (False, True):
        o = o3.Oracle3(p, pairwise_density=pw)
        f = o.init(rho)
        o.step(f, 500)
        fs.append(f)
    a, b = fs
    scale = np.abs(a).max()
    assert np.abs(a - b).max() / scale < 1e-13
    assert not np.array_equal(a, b)
