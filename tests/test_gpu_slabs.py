"""One lattice split into row slabs (wblbe_slabs_*), through the C ABI on
one GPU: every slab is advanced from its own rows and 3 ghost rows on each
side, exchanged by one copy kernel after every step (the slabs' kernels run
side by side on forked streams; chunks of steps replay from a CUDA graph);
the result must equal
the single-lattice run bit for bit (populations, fields and the
order-independent statistics), in both precisions and for every number of
slabs, including one slab whose ghost rows wrap onto itself."""
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


def _both(pr, scheme, precision, nslabs, steps):
    a = wblbe.Solver(gpu_params(pr, scheme, precision))
    a.init_rho(pr.rho)
    a.step(steps)
    b = wblbe.Slabs(gpu_params(pr, scheme, precision), nslabs)
    b.init_rho(pr.rho)
    b.step(steps)
    out = (a.get_populations(), b.get_populations(), a.moments(), b.moments())
    assert a.steps == b.steps == steps
    a.close()
    b.close()
    return out


@pytest.mark.parametrize("precision", [wblbe.FP64, wblbe.FP32_SHIFTED])
@pytest.mark.parametrize("nslabs", [1, 2, 3, 7])
def test_slabs_equal_single_lattice_bitwise(precision, nslabs):
    pr = wl.droplet(n=160, radius=36.0, tau=0.9, nx=160, ny=150)
    fa, fb, (ma, sa), (mb, sb) = _both(pr, wblbe.WELL_BALANCED, precision, nslabs, 67)
    assert np.array_equal(fa, fb)
    for k in ("rho", "ux", "uy", "mu"):
        assert np.array_equal(ma[k], mb[k]), k
    assert sa["umax"] == sb["umax"] and sa["mu_min"] == sb["mu_min"]
    assert sa["mu_max"] == sb["mu_max"] and not sb["nonfinite"]
    assert sb["mass"] == pytest.approx(sa["mass"], rel=1e-14)


@pytest.mark.parametrize("scheme", [wblbe.STANDARD, wblbe.STANDARD_PRESSURE,
                                    wblbe.STANDARD_TEXTBOOK])
def test_slabs_other_schemes_ragged_lattice(scheme):
    """A width that is no multiple of 4 (element copies) and an odd height;
    the standard scheme and its Sec. II variants."""
    rng = np.random.default_rng(5)
    rho = 0.6 + 0.3 * rng.uniform(-1, 1, (61, 67))
    pr = wl.Problem(67, 61, 0.85, 0.0128, 0.01, 1.0, 0.2, rho, name="rand67x61")
    fa, fb, (ma, _), (mb, _) = _both(pr, scheme, wblbe.FP64, 4, 40)
    assert np.array_equal(fa, fb)
    assert np.array_equal(ma["mu"], mb["mu"])


def test_slabs_refuse_thin_slabs_and_the_e6_variant():
    pr = wl.droplet(n=32, radius=8.0)
    with pytest.raises(wblbe.WblbeError):
        wblbe.Slabs(gpu_params(pr, wblbe.WELL_BALANCED), 12)     # slabs of 2 rows
    with pytest.raises(wblbe.WblbeError):
        wblbe.Slabs(gpu_params(pr, wblbe.STANDARD_E6), 2)


@pytest.mark.parametrize("precision", [wblbe.FP64, wblbe.FP32_SHIFTED])
def test_slabs_graph_chunks_and_direct_steps(precision):
    """Steps issued in uneven chunks (1, 20, 17, 33: graph replays starting
    from either buffer, and direct steps) equal the single lattice stepped
    the same way, bit for bit, and count their steps and launches."""
    pr = wl.droplet(n=96, radius=20.0, tau=0.9, nx=96, ny=90)
    a = wblbe.Solver(gpu_params(pr, wblbe.WELL_BALANCED, precision))
    b = wblbe.Slabs(gpu_params(pr, wblbe.WELL_BALANCED, precision), 5)
    a.init_rho(pr.rho)
    b.init_rho(pr.rho)
    l0 = b.kernel_launches
    for n in (1, 20, 17, 33):
        a.step(n)
        b.step(n)
    assert a.steps == b.steps == 71
    # 71 steps of 5 slab kernels and one exchange each, plus one step-base
    # kernel per graph replay of 16 steps: 1 -> 1 direct; 20 -> 1 direct
    # (the state is in the second buffer), 1 replay, 3 direct; 17 -> 1
    # direct, 1 replay; 33 -> 2 replays, 1 direct
    assert b.kernel_launches - l0 == 71 * 6 + 4
    assert np.array_equal(a.get_populations(), b.get_populations())
    a.close()
    b.close()
