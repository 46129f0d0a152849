"""The constant rho0 of the well-balanced equilibrium on the GPU (Sec. III):
it leaves the equilibrium state unchanged, and the stability map over
(rho0, density ratio, tau) runs through the batched kernel.  Host-side table
formatting, and a slow transverse instability of the WB flat interface at
tau = 0.8 on the oracle, are checked on the CPU."""
import numpy as np
import pytest

from paper_2012_11075_gb300 import stability


def test_rho0_values_and_table_layout():
    assert stability.rho0_value("zero", 1.0, 0.1) == 0.0
    assert stability.rho0_value("gas", 1.0, 0.1) == 0.1
    assert stability.rho0_value("mean", 1.0, 0.1) == pytest.approx(0.55)
    with pytest.raises(ValueError):
        stability.rho0_value("liquid", 1.0, 0.1)
    recs = [{"rho0_mode": m, "ratio": q, "tau": t, "state": s, "steps": 500, "umax": 1e-6}
            for m in ("zero", "gas") for q in (2.0, 10.0) for t in (0.6, 1.0)
            for s in (["unstable"] if (q == 10.0 and t == 0.6) else ["stable"])]
    txt = stability.format_table(recs)
    assert txt.count("rho0 =") == 2 and txt.count("x@500") == 2
    assert len(stability.grid((2, 10), (0.6, 1.0))) == 3 * 2 * 2


@pytest.mark.gpu
@pytest.mark.parametrize("rho0", [0.1, 0.55])
def test_equilibrium_does_not_depend_on_rho0_on_gpu(rho0):
    """FP64 WB slab (1 x 21, tau = 0.8) run to max|u| < 1e-13 and 50000 steps
    with rho0 = rho_g and the mean density: the density is the Newton
    solution of the discrete equilibrium (which has no rho0), to 1e-10."""
    from tests.gpu_helpers import gpu_params, need_gpu
    need_gpu()
    from oracle import equilibrium as eq
    from paper_2012_11075_gb300 import wblbe
    from paper_2012_11075_gb300 import workloads as wl
    ny = 21
    y = np.arange(ny, dtype=float)
    d = np.minimum(y, ny - y)
    prof = 0.55 + 0.45 * np.tanh(2 * (d - ny / 4) / 4.0)
    beta = wl.beta_for_width(0.01, 4.0, 1.0, 0.1)
    pr = wl.Problem(1, ny, 0.8, 0.01, beta, 1.0, 0.1, prof[:, None].copy())
    s = wblbe.Solver(gpu_params(pr, wblbe.WELL_BALANCED, rho0=rho0))
    s.init_rho(pr.rho)
    code, done, st = s.run_until_equilibrium(1e-13, 200000, 1000)
    assert code == wblbe.OK and st["umax"] < 1e-13
    s.step(50000 - done if done < 50000 else 0)
    m, st = s.moments()
    s.close()
    rN, _ = eq.discrete_flat_equilibrium(prof, 0.01, beta, 1.0, 0.1)
    assert st["mu_max"] - st["mu_min"] < 1e-13
    assert np.max(np.abs(m["rho"][:, 0] - rN)) < 1e-10


@pytest.mark.gpu
def test_small_stability_map_runs_every_case():
    """A 2 x 2 x 3 map (ratio 2 and 10, tau 0.6 and 1.0, three rho0 choices)
    on 64^2 droplets for 2000 steps: every case ends stable or unstable with
    its step count, and the mild corner (ratio 2, tau 1.0) is stable with a
    small spurious velocity for every rho0."""
    from tests.gpu_helpers import need_gpu
    need_gpu()
    recs = stability.stability_map(ratios=(2.0, 10.0), taus=(0.6, 1.0), n=64, steps=2000,
                                   steps_per_launch=50)
    assert len(recs) == 12
    for r in recs:
        assert r["state"] in ("stable", "unstable")
        if r["state"] == "stable":
            assert r["steps"] == 2000 and np.isfinite(r["umax"])
        else:
            assert 0 < r["steps"] <= 2000
    for r in recs:
        if r["ratio"] == 2.0 and r["tau"] == 1.0:
            assert r["state"] == "stable" and r["umax"] < 1e-3, r


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rho0_is_an_exact_offset_on_gpu(precision):
    """On the GPU, as on the oracle, the WB state with rho0 = 0.3 equals the
    rho0 = 0 state plus the constant vector b = rho0 (-(1-w0), w_1..w_8)
    after 1000 steps of the 256^2 droplet: the periodic dynamics do not see
    rho0 (FP64 to 1e-12; FP32-shifted to its storage rounding)."""
    from tests.gpu_helpers import need_gpu, run_gpu
    need_gpu()
    from paper_2012_11075_gb300 import wblbe
    from paper_2012_11075_gb300 import workloads as wl
    prec = wblbe.FP64 if precision == "fp64" else wblbe.FP32_SHIFTED
    pr = wl.droplet(n=256, radius=40.0, tau=1.0)
    f0, _, _ = run_gpu(pr, wblbe.WELL_BALANCED, 1000, precision=prec, rho0=0.0)
    f3, _, _ = run_gpu(pr, wblbe.WELL_BALANCED, 1000, precision=prec, rho0=0.3)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    b = np.concatenate([[-(1 - w[0]) * 0.3], w[1:] * 0.3])
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert np.max(np.abs(f3 - f0 - b[:, None, None])) < tol


@pytest.mark.parametrize("tau,grows", [(0.8, True), (0.85, False)])
def test_wb_flat_interface_transverse_mode(tau, grows):
    """Oracle (CPU, FP64): the WB flat slab 4 x 201 (ratio 10, W = 4) seeded
    with a density perturbation of 1e-10 that alternates along x.  At
    tau = 0.8 the x-alternating mode grows exponentially (about x8 per 4000
    steps), at tau = 0.85 it decays.  Runs that keep exact x-uniformity never
    seed this mode, which is why the deterministic slab at tau = 0.8 stays
    finite while any per-step noise (e.g. stochastic rounding) destroys it."""
    from oracle.oracle import Oracle, Params, WELL_BALANCED
    from paper_2012_11075_gb300 import workloads as wl
    pr = wl.flat_interface(nx=4, ny=201, tau=tau)
    o = Oracle(Params(pr.nx, pr.ny, tau, pr.kappa, pr.beta, pr.rho_l, pr.rho_g, 0.0,
                      WELL_BALANCED))
    rho = pr.rho + 1e-10 * (-1.0) ** np.arange(4)[None, :] * \
        np.random.default_rng(7).uniform(-1, 1, (201, 1))
    f = o.init(rho)

    def amp():
        r = o.macro(f)["rho"]
        return np.max(np.abs(r - r.mean(axis=1, keepdims=True)))

    o.step(f, 4000)
    a0 = amp()
    o.step(f, 16000)
    a1 = amp()
    if grows:
        assert a1 > 1e3 * a0, (a0, a1)
    else:
        assert a1 < a0, (a0, a1)


def _amplification(o, f0, mx, my, eps=1e-6):
    """9 x 9 amplification matrix of the oracle's step linearised about the
    uniform state f0, for the lattice wave number 2 pi (mx, my) / n: the
    responses to cos and sin perturbations of each population (central
    differences), read at node (0, 0)."""
    n = f0.shape[1]
    y, x = np.mgrid[0:n, 0:n]
    ph = 2 * np.pi * (mx * x + my * y) / n
    G = np.zeros((9, 9), complex)
    for i in range(9):
        parts = []
        for wave in (np.cos(ph), np.sin(ph)):
            fp, fm = f0.copy(), f0.copy()
            fp[i] += eps * wave
            fm[i] -= eps * wave
            o.step(fp, 1)
            o.step(fm, 1)
            parts.append((fp - fm)[:, 0, 0] / (2 * eps))
        G[:, i] = parts[0] + 1j * parts[1]
    return G


@pytest.mark.parametrize("scheme_name,tau,unstable", [("wb", 0.80, True), ("wb", 0.90, False),
                                                      ("standard", 0.60, False)])
def test_bulk_linear_stability(scheme_name, tau, unstable):
    """von Neumann analysis of the oracle's step about a uniform bulk state
    (liquid, ratio 10, W = 4, kappa = 0.01) on a 64^2 lattice, along
    k = (pi, k_y).  The WB scheme amplifies the x-alternating density mode
    with a slow modulation in y for tau below about 0.854 (at tau = 0.8 by
    about 5e-4 per step, the growth seen at the slab's interfaces); at
    tau = 0.9 every mode is bounded.  The standard scheme, whose equilibrium
    carries the pressure, shows no such mode."""
    from oracle import equilibrium as eq
    from oracle.oracle import STANDARD, WELL_BALANCED, Oracle, Params
    n, kappa, width = 64, 0.01, 4.0
    beta = eq.beta_for_width(kappa, width, 1.0, 0.1)
    scheme = WELL_BALANCED if scheme_name == "wb" else STANDARD
    o = Oracle(Params(n, n, tau, kappa, beta, 1.0, 0.1, 0.0, scheme))
    f0 = o.init(np.full((n, n), 1.0))
    growth = max(np.abs(np.linalg.eigvals(_amplification(o, f0, n // 2, my))).max() - 1.0
                 for my in (1, 2, 3, 4, 6, 8))
    if unstable:
        assert growth > 1e-4, growth
    else:
        assert growth < 1e-8, growth


@pytest.mark.parametrize("tau", [0.7, 0.8, 0.9, 1.2])
def test_bulk_mode_matches_second_order_formula(tau):
    """Linearised about a uniform rest state, the WB amplification matrix at
    k = (pi, 0) has the simple eigenvalue 1 (the x-alternating density field,
    which feels no force).  Second-order perturbation in the modulation
    k_y = q gives
        lambda = 1 + S (w^2 - 8 w + 8) / (6 w (w - 2)) q^2 + O(q^4),
    w = 1/tau, S = rho (psi_0''(rho) + 4 kappa): growth for w > 4 - 2 sqrt 2,
    i.e. tau < (2 + sqrt 2) / 4, whatever the free energy.  The oracle's
    eigenvalue at q = 2 pi / 128 agrees with it to 1 %."""
    from oracle import equilibrium as eq
    from oracle.oracle import WELL_BALANCED, Oracle, Params
    n, kappa, width, rho = 128, 0.01, 4.0, 1.0
    beta = eq.beta_for_width(kappa, width, 1.0, 0.1)
    o = Oracle(Params(n, n, tau, kappa, beta, 1.0, 0.1, 0.0, WELL_BALANCED))
    f0 = o.init(np.full((n, n), rho))
    lam = np.linalg.eigvals(_amplification(o, f0, n // 2, 1))
    got = lam[np.argmin(np.abs(lam - 1.0))] - 1.0
    q = 2 * np.pi / n
    want = stability.bulk_mode_growth(tau, rho, eq.dmu0(rho, beta, 1.0, 0.1), kappa, q)
    assert (want > 0) == (tau < stability.WB_TAU_LIMIT)
    assert abs(got.imag) < 1e-12
    assert abs(got.real - want) < 0.01 * abs(want), (got, want)


def test_bulk_mode_formula_is_derived():
    """The formula pinned above, derived symbolically from the linearised
    update (tests/bulk_mode_derivation.py, which shares no code with the
    oracle or the CUDA path): at k = (pi, q) the eigenvalue 1 moves by
    S (w^2 - 8 w + 8) / (6 w (w - 2)) q^2, which changes sign at
    w = 4 -+ 2 sqrt 2, and the eigenvalue -1 shrinks in modulus for w < 2."""
    sp = pytest.importorskip("sympy")
    from tests import bulk_mode_derivation as d
    om, S, lam1, lam2, a2 = d.second_order(1)
    assert lam1 == 0
    assert sp.simplify(lam2 - S * (om ** 2 - 8 * om + 8) / (6 * om * (om - 2))) == 0
    roots = sorted(sp.solve(sp.Eq(a2, 0), om), key=lambda r: float(r))
    assert [sp.nsimplify(r) for r in roots] == [4 - 2 * sp.sqrt(2), 4 + 2 * sp.sqrt(2)]
    om, S, lam1, lam2, a2 = d.second_order(-1)
    assert lam1 == 0 and sp.simplify(a2 - (om - 2) / (3 * om)) == 0
