"""The allocation-free statistics entry point, wblbe_moments_noalloc.

Callers that cannot allocate device memory (hosts whose own allocator has
reserved the whole device and forbids cudaMalloc, plug-ins and callbacks
that only receive buffers) use it to get rho, u, mu and the stats of a
population state they hold.  It keeps its reduction scratch in a fixed array
inside the library, so this test checks it against the regular entry point
(wblbe_moments on a handle holding the same state) on two calls in a row,
the second after the state has moved on, on a lattice of whole CTA tiles,
on ragged and tiny lattices, and at the exact size limit of the scratch.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from oracle.oracle import STANDARD, WELL_BALANCED
from paper_2012_11075_gb300 import wblbe
from paper_2012_11075_gb300 import workloads as wl
from tests.gpu_helpers import gpu_params, need_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-12          # the FP64 parity tolerance of the other GPU tests


def _noalloc(lib, params, f_dev, torch):
    ny, nx = params.ny, params.nx
    outs = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(4)]
    st = wblbe.CStats()
    cp = params.c()
    code = lib.wblbe_moments_noalloc(ctypes.byref(cp), ctypes.c_void_p(f_dev.data_ptr()),
                                     *[ctypes.c_void_p(o.data_ptr()) for o in outs],
                                     ctypes.byref(st),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == wblbe.OK, lib.wblbe_noalloc_last_error().decode()
    torch.cuda.synchronize()
    return dict(zip(("rho", "ux", "uy", "mu"), [o.cpu().numpy() for o in outs])), st.as_dict()


def _compare(ref, ref_st, got, st, pr):
    # u = (j + F/2) / rho with j a sum of populations of order 1/9 in another
    # order than the handle's kernel: an absolute floor of 1e-15 covers that
    # round-off where the velocity itself is tiny (as the other FP64 tests)
    for k in ("rho", "ux", "uy"):
        scale = np.max(np.abs(ref[k]))
        assert np.max(np.abs(got[k] - ref[k])) <= max(TOL * scale, 1e-15), k
    mu_scale = 2 * pr.beta * (pr.rho_l - pr.rho_g) ** 3
    assert np.max(np.abs(got["mu"] - ref["mu"])) <= TOL * mu_scale
    assert st["mass"] == pytest.approx(ref_st["mass"], rel=1e-13)
    assert st["umax"] == pytest.approx(ref_st["umax"], rel=1e-9)
    assert st["kinetic"] == pytest.approx(ref_st["kinetic"], rel=1e-9)
    assert st["mu_min"] == pytest.approx(ref_st["mu_min"], rel=1e-9, abs=1e-15)
    assert st["mu_max"] == pytest.approx(ref_st["mu_max"], rel=1e-9, abs=1e-15)
    assert st["nonfinite"] == 0


def _random_problem(nx, ny, seed):
    rng = np.random.default_rng(seed)
    rho = 0.6 + 0.3 * rng.uniform(-1, 1, (ny, nx))
    return wl.Problem(nx, ny, 0.85, 0.0128, 0.01, 1.0, 0.2, rho, name=f"rand{nx}x{ny}")


@pytest.mark.parametrize("shape", [(96, 80), (37, 13), (3, 5)])
@pytest.mark.parametrize("scheme", [WELL_BALANCED, STANDARD])
def test_noalloc_moments_match_regular_entry_point_twice(scheme, shape):
    """96 x 80 is whole 32 x 8 tiles; 37 x 13 leaves partial tiles on both
    axes (threads outside the lattice feed neutral records into the
    reduction); 3 x 5 is narrower than the 2-node density halo, which wraps
    onto the lattice itself."""
    torch = need_gpu()
    lib = wblbe.load_library()
    nx, ny = shape
    if shape == (96, 80):
        pr = wl.droplet(n=96, radius=24.0, tau=0.85, rho_g=0.2, nx=96, ny=80)
    else:
        pr = _random_problem(nx, ny, seed=nx * 100 + ny)
    params = gpu_params(pr, scheme)
    s = wblbe.Solver(params)
    s.init_rho(pr.rho)
    for steps in (150, 250):                       # two calls in a row
        s.step(steps)
        ref, ref_st = s.moments()
        f = torch.from_numpy(s.get_populations()).cuda()
        got, st = _noalloc(lib, params, f, torch)
        _compare(ref, ref_st, got, st, pr)
    s.close()


def test_noalloc_accepts_the_largest_lattice_and_rejects_one_record_more():
    """The scratch holds 16384 per-CTA records of 32 x 8 nodes.  2048 x 2048
    needs exactly 16384 and must run (and agree with wblbe_moments);
    160 x 26216 needs 5 x 3277 = 16385 and must be refused before any work."""
    torch = need_gpu()
    lib = wblbe.load_library()
    pr = wl.droplet(n=2048, radius=400.0, tau=1.0)
    params = gpu_params(pr, WELL_BALANCED)
    s = wblbe.Solver(params)
    s.init_rho(pr.rho)
    s.step(20)
    ref, ref_st = s.moments()
    f = torch.from_numpy(s.get_populations()).cuda()
    s.close()
    got, st = _noalloc(lib, params, f, torch)
    _compare(ref, ref_st, got, st, pr)
    del f
    over = gpu_params(pr, WELL_BALANCED)
    over.nx, over.ny = 160, 26216
    cp = over.c()
    small = torch.zeros(16, dtype=torch.float64, device="cuda")   # never read
    code = lib.wblbe_moments_noalloc(ctypes.byref(cp), ctypes.c_void_p(small.data_ptr()),
                                     None, None, None, None, ctypes.byref(wblbe.CStats()), None)
    assert code == wblbe.ENOMEM
    assert b"16385" in lib.wblbe_noalloc_last_error()


def test_noalloc_rejects_oversized_lattice_and_fp32():
    torch = need_gpu()
    lib = wblbe.load_library()
    pr = wl.droplet(n=16, radius=4.0)
    f = torch.zeros((9, 16, 16), dtype=torch.float64, device="cuda")
    big = gpu_params(pr, WELL_BALANCED)
    big.nx, big.ny = 8192, 8192                   # needs 256 * 1024 records
    cp = big.c()
    st = wblbe.CStats()
    code = lib.wblbe_moments_noalloc(ctypes.byref(cp), ctypes.c_void_p(f.data_ptr()),
                                     None, None, None, None, ctypes.byref(st), None)
    assert code == wblbe.ENOMEM
    assert b"scratch" in lib.wblbe_noalloc_last_error()
    p32 = gpu_params(pr, WELL_BALANCED, wblbe.FP32_SHIFTED).c()
    code = lib.wblbe_moments_noalloc(ctypes.byref(p32), ctypes.c_void_p(f.data_ptr()),
                                     None, None, None, None, ctypes.byref(st), None)
    assert code == wblbe.EINVAL
