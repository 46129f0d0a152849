"""GPU parity of the comparison variants of the standard LBE (Sec. II): the
pressure-form interaction force, the textbook forcing term and the
sixth-order isotropic gradient in the force (FP64 only), through the C ABI
against the FP64 oracle (same tolerances as the main schemes), plus the
batch API's refusal of them."""
import numpy as np
import pytest

from oracle.oracle import STANDARD_E6, STANDARD_PRESSURE, STANDARD_TEXTBOOK
from paper_2012_11075_gb300 import wblbe
from paper_2012_11075_gb300 import workloads as wl
from tests.gpu_helpers import need_gpu, pop_error, run_gpu, run_oracle
from tests.test_gpu_parity import FP32_POP_TOL, FP32_RHO_TOL, FP32_U_TOL, _check_fp64

pytestmark = pytest.mark.gpu
VARIANTS = [STANDARD_PRESSURE, STANDARD_TEXTBOOK]
FP64_VARIANTS = VARIANTS + [STANDARD_E6]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    wblbe.load_library()


def test_codes_match_the_c_abi():
    assert (wblbe.STANDARD_PRESSURE, wblbe.STANDARD_TEXTBOOK, wblbe.STANDARD_E6) == (
        STANDARD_PRESSURE, STANDARD_TEXTBOOK, STANDARD_E6)


@pytest.mark.parametrize("scheme", FP64_VARIANTS)
def test_fp64_paper_flat_interface(scheme):
    """The 21 x 101 noisy slab of Sec. IV.A (rho_v = 0.2, tau = 0.85)."""
    _check_fp64(wl.paper_flat(), scheme, 1000)


@pytest.mark.parametrize("scheme", FP64_VARIANTS)
def test_fp64_paper_droplet(scheme):
    _check_fp64(wl.paper_droplet(), scheme, 1000)


@pytest.mark.parametrize("shape", [(3, 3), (1, 17), (17, 1), (5, 2), (67, 129), (257, 33)])
@pytest.mark.parametrize("scheme", FP64_VARIANTS)
def test_fp64_ragged_and_tiny_lattices(shape, scheme):
    nx, ny = shape
    rng = np.random.default_rng(nx * 1000 + ny)
    rho = 0.6 + 0.3 * rng.uniform(-1, 1, (ny, nx))
    pr = wl.Problem(nx, ny, 0.85, 0.0128, 0.01, 1.0, 0.2, rho, name=f"rand{nx}x{ny}")
    _check_fp64(pr, scheme, 100)


@pytest.mark.parametrize("scheme", VARIANTS)
def test_fp64_launch_shapes_bitwise(scheme):
    """Launch shape (strip width, rows per CTA) does not change the result."""
    pr = wl.paper_droplet()
    ref, _, _ = run_gpu(pr, scheme, 200)
    for launch in [(32, 7), (64, 13), (256, 100)]:
        f, _, _ = run_gpu(pr, scheme, 200, launch=launch)
        assert np.array_equal(f, ref), launch


@pytest.mark.parametrize("scheme", VARIANTS)
def test_fp32_shifted_against_oracle(scheme):
    pr = wl.paper_droplet()
    fg, mg, sg = run_gpu(pr, scheme, 1000, precision=wblbe.FP32_SHIFTED)
    fo, mo, so = run_oracle(pr, scheme, 1000)
    glob, _ = pop_error(fg, fo)
    assert glob < FP32_POP_TOL, glob
    assert np.max(np.abs(mg["rho"] - mo["rho"])) < FP32_RHO_TOL
    assert np.max(np.abs(mg["ux"] - mo["ux"])) < FP32_U_TOL
    assert np.max(np.abs(mg["uy"] - mo["uy"])) < FP32_U_TOL
    assert abs(sg["mass"] - so["mass"]) < 1e-5 * so["mass"]


def test_batch_refuses_the_variants():
    for scheme in FP64_VARIANTS:
        with pytest.raises(Exception):
            wblbe.Batch(scheme=scheme, max_cases=1, arena_bytes=1 << 20)
