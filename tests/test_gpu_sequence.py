"""wblbe_run_sequence (the overlapped host-I/O form of init_rho + step +
moments) against the same calls made one state at a time: every output
density bit for bit, every statistics record equal, and the handle left
holding the last state.  Both precisions and schemes, a ragged lattice,
step counts that cross the captured-graph chunk, pinned and pageable host
memory, repeated pointers, and the argument checks."""
import ctypes

import numpy as np
import pytest

from paper_2012_11075_gb300 import wblbe
from paper_2012_11075_gb300 import workloads as wl
from tests.gpu_helpers import gpu_params, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    wblbe.load_library()


def _inputs(pr, n, seed):
    """n distinct initial densities: the problem's field, shifted and mildly
    perturbed (bounded well inside the two phases' range)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        r = np.roll(pr.rho, (3 * k, 5 * k), axis=(0, 1))
        out.append(np.ascontiguousarray(r + 1e-3 * rng.uniform(-1, 1, r.shape)))
    return out


def _one_at_a_time(params, inputs, nsteps):
    s = wblbe.Solver(params)
    rhos, stats = [], []
    for r in inputs:
        s.init_rho(r)
        s.step(nsteps)
        m, st = s.moments()
        rhos.append(m["rho"])
        stats.append(st)
    s.close()
    return rhos, stats


@pytest.mark.parametrize("shape", [(96, 80), (37, 13)])
@pytest.mark.parametrize("scheme,precision", [(wblbe.WELL_BALANCED, wblbe.FP32_SHIFTED),
                                              (wblbe.WELL_BALANCED, wblbe.FP64),
                                              (wblbe.STANDARD, wblbe.FP64)])
def test_sequence_equals_one_state_at_a_time(shape, scheme, precision):
    import torch
    nx, ny = shape
    pr = wl.droplet(n=max(nx, ny), radius=max(nx, ny) / 5, tau=1.0)
    pr = wl.Problem(nx, ny, pr.tau, pr.kappa, pr.beta, pr.rho_l, pr.rho_g,
                    np.ascontiguousarray(pr.rho[:ny, :nx]))
    params = gpu_params(pr, scheme, precision)
    nsteps = 150
    inputs = _inputs(pr, 3, nx * ny)
    ref_rho, ref_stats = _one_at_a_time(params, inputs, nsteps)

    s = wblbe.Solver(params)
    pinned_in = [torch.from_numpy(r).pin_memory() for r in inputs]
    pinned_out = [torch.empty(pr.rho.shape, dtype=torch.float64).pin_memory() for _ in inputs]
    stats = s.run_sequence(pinned_in, nsteps, pinned_out)
    for k in range(3):
        assert np.array_equal(pinned_out[k].numpy(), ref_rho[k]), k
        for key in ("mass", "mass_drift_rel", "umax", "mu_min", "mu_max", "kinetic",
                    "nonfinite", "step"):
            assert stats[k][key] == ref_stats[k][key], (k, key)
    # the handle holds the last state, with that state's mass reference
    m, st = s.moments()
    assert np.array_equal(m["rho"], ref_rho[-1])
    assert st["mass_drift_rel"] == ref_stats[-1]["mass_drift_rel"]
    assert s.steps == nsteps
    # pageable memory and repeated pointers: the same results
    outs = [np.empty(pr.rho.shape) for _ in range(2)]
    stats2 = s.run_sequence([inputs[0], inputs[1], inputs[0]], nsteps,
                            [outs[0], outs[1], outs[0]])
    assert np.array_equal(outs[0], ref_rho[0]) and np.array_equal(outs[1], ref_rho[1])
    assert stats2[2]["umax"] == ref_stats[0]["umax"]
    s.close()


def test_sequence_argument_checks():
    pr = wl.droplet(n=64, radius=12.0, tau=1.0)
    params = gpu_params(pr, wblbe.WELL_BALANCED, wblbe.FP64)
    s = wblbe.Solver(params)
    lib = s.lib
    cp = params.c()
    need = int(lib.wblbe_sequence_scratch_bytes(ctypes.byref(cp)))
    assert need >= 4 * 64 * 64 * 8
    assert int(lib.wblbe_sequence_scratch_bytes(None)) == 0
    assert s.run_sequence([], 10, []) == []            # n = 0: nothing to do
    import torch
    scratch = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    r = np.ascontiguousarray(pr.rho)
    o = np.empty_like(r)
    pin = (ctypes.c_void_p * 1)(r.ctypes.data)
    pout = (ctypes.c_void_p * 1)(o.ctypes.data)
    base = scratch.data_ptr()
    aligned = (base + 255) // 256 * 256

    def call(n, steps, sp, nbytes, rin=pin, rout=pout):
        return lib.wblbe_run_sequence(s.h, n, ctypes.cast(rin, ctypes.c_void_p), steps,
                                      ctypes.cast(rout, ctypes.c_void_p), None,
                                      ctypes.c_void_p(sp), nbytes)

    assert call(1, 5, aligned, need - 8) == wblbe.EINVAL          # short
    assert call(1, 5, aligned + 8, need) == wblbe.EINVAL          # misaligned
    assert call(-1, 5, aligned, need) == wblbe.EINVAL
    assert call(1, -5, aligned, need) == wblbe.EINVAL
    nul = (ctypes.c_void_p * 1)(None)
    assert call(1, 5, aligned, need, rin=nul) == wblbe.EINVAL
    assert call(1, 5, aligned, need) == wblbe.OK
    s.init_rho(r)
    s.step(5)
    m, _ = s.moments()
    assert np.array_equal(o, m["rho"])
    s.close()
