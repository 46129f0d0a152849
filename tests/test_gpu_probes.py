"""The measurement aids of the library, through the C ABI: the float64
reciprocal the update uses for 1/rho (Eq. rhoU) against the IEEE quotient,
and the FP64 fused multiply-add probe that sets the FP64 ceiling."""
import ctypes

import numpy as np
import pytest

from paper_2012_11075_gb300 import wblbe
from tests.gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def _ulps(a, b):
    """Distance in units in the last place between positive doubles."""
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_fp64_reciprocal_within_one_ulp_of_ieee_division():
    """1/x from the hardware seed plus one third-order refinement, over
    densities log-uniform in [1e-3, 1e2] (every valid state's range, with
    margin) and around powers of two: within one ulp of the correctly
    rounded quotient, and equal to it for nearly every x.  The seed alone
    is far coarser (measured and reported in the assertion message)."""
    torch = need_gpu()
    lib = wblbe.load_library()
    rng = np.random.default_rng(7)
    x = np.exp(rng.uniform(np.log(1e-3), np.log(1e2), 1 << 20))
    p2 = 2.0 ** np.arange(-10, 7)
    x = np.concatenate([x, p2, np.nextafter(p2, 0), np.nextafter(p2, 10), [0.1, 1 / 3, 0.55]])
    xd = torch.from_numpy(x).cuda()
    seed, ref = torch.empty_like(xd), torch.empty_like(xd)
    code = lib.wblbe_probe_reciprocal(ctypes.c_void_p(xd.data_ptr()),
                                      ctypes.c_void_p(seed.data_ptr()),
                                      ctypes.c_void_p(ref.data_ptr()), x.size,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == wblbe.OK
    torch.cuda.synchronize()
    want = 1.0 / x
    got = ref.cpu().numpy()
    seed_rel = np.max(np.abs(seed.cpu().numpy() * x - 1.0))
    u = _ulps(got, want)
    assert u.max() <= 1, (u.max(), seed_rel)
    assert np.mean(u == 0) > 0.999, (np.mean(u == 0), seed_rel)
    assert seed_rel < 1e-5


def test_fp64_fma_probe_runs_and_rejects_bad_shapes():
    torch = need_gpu()
    lib = wblbe.load_library()
    out = torch.empty(4 * 128, dtype=torch.float64, device="cuda")
    assert lib.wblbe_probe_fp64_fma(ctypes.c_void_p(out.data_ptr()), 4, 128, 100, None) == wblbe.OK
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all()) and float(out.min()) > 0
    assert lib.wblbe_probe_fp64_fma(ctypes.c_void_p(out.data_ptr()), 4, 100, 100, None) == wblbe.EINVAL
    assert lib.wblbe_probe_reciprocal(None, None, None, 4, None) == wblbe.EINVAL
