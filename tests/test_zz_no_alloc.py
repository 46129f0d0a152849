"""The allocation-free statistics entry point, wblbe_moments_noalloc.

Callers that cannot allocate device memory (graph-capture regions, hosts
whose allocator owns the whole device, plug-ins that only receive buffers)
use it to get rho, u, mu and the stats of a population state they hold.  It
keeps its reduction scratch in a fixed array inside the library, so this
test checks it against the regular entry point (wblbe_moments on a handle
holding the same state) on two calls in a row, the second after the state
has moved on.  This file is collected last on purpose.
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


@pytest.mark.parametrize("scheme", [WELL_BALANCED, STANDARD])
def test_noalloc_moments_match_regular_entry_point_twice(scheme):
    torch = need_gpu()
    lib = wblbe.load_library()
    pr = wl.droplet(n=96, radius=24.0, tau=0.85, rho_g=0.2, nx=96, ny=80)
    params = gpu_params(pr, scheme)
    s = wblbe.Solver(params)
    s.init_rho(pr.rho)
    for steps in (150, 250):                       # two calls in a row
        s.step(steps)
        ref, ref_st = s.moments()
        f = torch.from_numpy(s.get_populations()).cuda()
        got, st = _noalloc(lib, params, f, torch)
        for k in ("rho", "ux", "uy"):
            scale = np.max(np.abs(ref[k]))
            assert np.max(np.abs(got[k] - ref[k])) <= TOL * max(scale, 1e-300), k
        mu_scale = 2 * pr.beta * (pr.rho_l - pr.rho_g) ** 3
        assert np.max(np.abs(got["mu"] - ref["mu"])) <= TOL * mu_scale
        assert st["mass"] == pytest.approx(ref_st["mass"], rel=1e-13)
        assert st["umax"] == pytest.approx(ref_st["umax"], rel=1e-9)
        assert st["kinetic"] == pytest.approx(ref_st["kinetic"], rel=1e-9)
        assert st["mu_min"] == pytest.approx(ref_st["mu_min"], rel=1e-9, abs=1e-15)
        assert st["mu_max"] == pytest.approx(ref_st["mu_max"], rel=1e-9, abs=1e-15)
        assert st["nonfinite"] == 0
    s.close()


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
