"""The batched persistent kernel and its scheduler (C ABI wblbe_batch_*).

Each case's per-node arithmetic is the single-lattice kernel's, so a case
advanced inside any mix, with any tile shape or steps per launch, must equal
the same case run alone, bit for bit, and the FP64 path must match the
oracle as the single-lattice path does (1e-12 of the largest population)."""
import math

import numpy as np
import pytest

from oracle.oracle import WELL_BALANCED, STANDARD
from paper_2012_11075_gb300 import wblbe
from paper_2012_11075_gb300 import workloads as wl
from tests.gpu_helpers import check_per_direction, gpu_params, need_gpu, pop_error, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    wblbe.load_library()


def _mix(seed=7, count=6):
    """A few uneven cases: odd and even sides, flat and droplet, ratio 2-10."""
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(count):
        nx = int(rng.integers(40, 300))
        ny = int(rng.integers(40, 300))
        ratio = float(rng.uniform(2.0, 10.0))
        tau = float(rng.uniform(0.8, 1.2))
        if k % 2:
            pr = wl.droplet(radius=0.25 * min(nx, ny), tau=tau, rho_g=1.0 / ratio, nx=nx, ny=ny)
        else:
            pr = wl.flat_interface(nx=nx, ny=ny, rho_g=1.0 / ratio, tau=tau)
        cases.append(pr)
    return cases


def _solo_solver(pr, precision, steps):
    s = wblbe.Solver(gpu_params(pr, WELL_BALANCED, precision))
    s.init_rho(pr.rho)
    s.step(steps)
    f = s.get_populations()
    s.close()
    return f


@pytest.mark.parametrize("precision", [wblbe.FP32_SHIFTED, wblbe.FP64])
def test_case_in_mix_equals_case_alone_bitwise(precision):
    cases = _mix()
    steps_per_launch, launches = 4, 9
    mix = wblbe.Batch(precision=precision, max_cases=16, arena_bytes=1 << 28, tile_x=64,
                      rows_per_tile=24, steps_per_launch=steps_per_launch)
    ids = [mix.admit(gpu_params(pr, WELL_BALANCED, precision), pr.rho, 0.0, 10 ** 9)
           for pr in cases]
    assert None not in ids
    mix.advance(launches)
    for pr, cid in zip(cases, ids):
        f_mix = mix.get_populations(cid, (pr.ny, pr.nx))
        alone = wblbe.Batch(precision=precision, max_cases=1, arena_bytes=1 << 26, tile_x=128,
                            rows_per_tile=16, steps_per_launch=3)
        aid = alone.admit(gpu_params(pr, WELL_BALANCED, precision), pr.rho, 0.0, 10 ** 9)
        alone.advance(12)                  # the same 36 steps in another shape
        f_alone = alone.get_populations(aid, (pr.ny, pr.nx))
        alone.close()
        assert np.array_equal(f_mix, f_alone), pr.name
        assert np.array_equal(f_mix, _solo_solver(pr, precision, 36)), pr.name
        assert mix.info(cid)["steps"] == 36
    mix.close()


def test_batch_fp64_matches_oracle():
    cases = _mix(seed=11, count=3)
    b = wblbe.Batch(precision=wblbe.FP64, max_cases=4, arena_bytes=1 << 27, tile_x=64,
                    rows_per_tile=16, steps_per_launch=5)
    ids = [b.admit(gpu_params(pr, WELL_BALANCED), pr.rho, 0.0, 10 ** 9) for pr in cases]
    b.advance(40)
    for pr, cid in zip(cases, ids):
        fo, mo, so = run_oracle(pr, WELL_BALANCED, 200)
        fg = b.get_populations(cid, (pr.ny, pr.nx))
        glob, _ = pop_error(fg, fo)
        assert glob < 1e-12, (pr.name, glob)
        check_per_direction(fg, fo, lambda: run_oracle(pr, WELL_BALANCED, 200,
                                                       pairwise_density=True)[0])
        m, st = b.fetch(cid, (pr.ny, pr.nx))
        assert np.max(np.abs(m["rho"] - mo["rho"])) < 1e-12
        assert st["mass"] == pytest.approx(so["mass"], rel=1e-13)
    b.close()


def test_admission_refusal_and_slot_reuse():
    pr = wl.droplet(n=128, radius=30.0)
    p = gpu_params(pr, WELL_BALANCED, wblbe.FP32_SHIFTED)
    one = wblbe.Batch(max_cases=2, arena_bytes=1 << 26).case_bytes(p)
    b = wblbe.Batch(max_cases=2, arena_bytes=one + 4096)
    a = b.admit(p, pr.rho, 0.0, 100)
    assert a is not None
    assert b.admit(p, pr.rho, 0.0, 100) is None        # arena full
    b.retire(a)
    c = b.admit(p, pr.rho, 0.0, 100)
    assert c is not None and c != a
    assert b.counts()["resident"] == 1
    b.close()
    b = wblbe.Batch(max_cases=1, arena_bytes=1 << 27)
    assert b.admit(p, pr.rho, 0.0, 100) is not None
    assert b.admit(p, pr.rho, 0.0, 100) is None        # no slot
    b.close()


def test_cases_stop_on_convergence_budget_and_instability():
    pr = wl.droplet(n=64, radius=16.0, tau=0.9, rho_g=0.2)
    p = gpu_params(pr, WELL_BALANCED, wblbe.FP64)
    b = wblbe.Batch(precision=wblbe.FP64, max_cases=4, arena_bytes=1 << 26, tile_x=64,
                    rows_per_tile=16, steps_per_launch=10)
    loose = b.admit(p, pr.rho, 1.0, 10 ** 6)           # below tolerance at the first check
    budget = b.admit(p, pr.rho, 0.0, 30)               # stops after 30 steps
    bad_rho = pr.rho.copy()
    bad_rho[3, 5] = math.nan
    bad = b.admit(p, bad_rho, 0.0, 10 ** 6)
    live = b.admit(p, pr.rho, 0.0, 10 ** 6)
    b.advance(1)
    assert b.info(loose)["state"] == wblbe.CASE_CONVERGED
    assert b.info(bad)["state"] == wblbe.CASE_UNSTABLE
    assert b.info(live)["state"] == wblbe.CASE_RUNNING
    b.advance(3)
    assert b.info(budget)["state"] == wblbe.CASE_MAXSTEPS and b.info(budget)["steps"] == 30
    assert b.info(live)["steps"] == 40 and b.info(loose)["steps"] == 10
    assert sorted(b.poll()) == sorted([loose, bad, budget])
    assert b.poll() == []
    b.close()


def test_wait_limit_timeout_is_reported_and_context_survives():
    """A neighbour wait forced to give up (one spin) stops the launch with
    ETIMEOUT; nothing is left in flight and the device stays usable."""
    torch = need_gpu()
    pr = wl.droplet(n=256, radius=60.0, tau=1.0)
    p = gpu_params(pr, WELL_BALANCED, wblbe.FP32_SHIFTED)
    b = wblbe.Batch(max_cases=2, arena_bytes=1 << 27, tile_x=64, rows_per_tile=16,
                    steps_per_launch=8)
    b.admit(p, pr.rho, 0.0, 10 ** 6)
    b.set_wait_limit(1)
    with pytest.raises(wblbe.WblbeError) as e:
        b.advance(1)
    assert e.value.status == wblbe.ETIMEOUT
    b.close()
    torch.cuda.synchronize()
    b = wblbe.Batch(max_cases=2, arena_bytes=1 << 27)
    cid = b.admit(p, pr.rho, 0.0, 10 ** 6)
    b.advance(2)
    assert b.info(cid)["state"] == wblbe.CASE_RUNNING
    b.close()


def test_serving_results_equal_alone_and_in_the_mix():
    """Requests served together (arriving while others run, admitted as room
    frees up) end in exactly the state each reaches when served alone."""
    from paper_2012_11075_gb300 import serve
    reqs = serve.make_requests(rate=400.0, duration=0.05, seed=21, precision=wblbe.FP32_SHIFTED,
                               scheme=wblbe.WELL_BALANCED, side_min=32, side_max=160,
                               umax_tol=1e-4, max_steps=400)
    assert len(reqs) >= 8
    got = {}

    def keep(req, batch):
        got[req.rid] = (batch.get_populations(req.case_id, (req.params.ny, req.params.nx)),
                        req.steps, req.state)

    b = wblbe.Batch(max_cases=4, arena_bytes=1 << 26, max_case_nodes=160 * 160, tile_x=64,
                    rows_per_tile=16, steps_per_launch=8)
    srv = serve.Server(b, on_finish=keep)
    rep = srv.run(reqs, duration=0.0, drain=True)
    b.close()
    assert len(rep.completed) == len(reqs) and rep.summary()["p99_latency_s"] > 0
    for r in reqs:
        assert not callable(r.rho)          # every request was admitted
        solo = wblbe.Batch(max_cases=1, arena_bytes=1 << 25, max_case_nodes=160 * 160,
                           tile_x=64, rows_per_tile=16, steps_per_launch=8)
        cid = solo.admit(r.params, r.rho, r.umax_tol, r.max_steps)
        while solo.info(cid)["state"] == wblbe.CASE_RUNNING:
            solo.advance(1)
        f = solo.get_populations(cid, (r.params.ny, r.params.nx))
        info = solo.info(cid)
        solo.close()
        f_mix, steps, state = got[r.rid]
        assert steps == info["steps"] and state == info["state"], r.rid
        assert np.array_equal(f_mix, f), r.rid


def test_full_mix_in_bench_configuration_sampled_against_solo():
    """The benchmark's batched workload at full size (all 512 uneven cases,
    tile 128 x 32, 64 steps per launch) for two launches: sampled cases
    equal their single-lattice runs bit for bit (non-finite values too, for a
    case that became unstable), and every case reports its step count."""
    specs = wl.batched_case_specs(count=512, seed=4)

    def params(sp):
        return wblbe.Params(sp["nx"], sp["ny"], sp["tau"], sp["kappa"], sp["beta"],
                            sp["rho_l"], sp["rho_g"], scheme=WELL_BALANCED,
                            precision=wblbe.FP32_SHIFTED)

    probe = wblbe.Batch(max_cases=1, arena_bytes=1 << 20)
    total = sum(probe.case_bytes(params(sp)) for sp in specs)
    probe.close()
    b = wblbe.Batch(max_cases=512, max_tiles=1 << 18, max_case_nodes=512 * 512,
                    arena_bytes=int(total * 1.02) + (1 << 20), tile_x=128, rows_per_tile=32,
                    steps_per_launch=64)
    ids = [b.admit(params(sp), wl.case_field(sp), 0.0, 10 ** 9) for sp in specs]
    assert None not in ids
    b.advance(2)
    for k in (0, 97, 203, 301, 444, 511):
        sp, cid = specs[k], ids[k]
        info = b.info(cid)
        assert info["steps"] == 128 or info["state"] == wblbe.CASE_UNSTABLE
        f_mix = b.get_populations(cid, (sp["ny"], sp["nx"]))
        s = wblbe.Solver(params(sp))
        s.init_rho(wl.case_field(sp))
        s.step(info["steps"])
        f_solo = s.get_populations()
        s.close()
        assert np.array_equal(f_mix, f_solo, equal_nan=True), k
    b.close()
