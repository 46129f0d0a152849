"""The C-ABI library builds, loads without a GPU and exports every entry
point include/wblbe.h declares; host-only entry points validate arguments."""
import ctypes
import math
import re
from pathlib import Path

import pytest

from paper_2012_11075_gb300 import wblbe

HEADER = Path(__file__).resolve().parents[1] / "include" / "wblbe.h"


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    return sorted(set(re.findall(r"\b(wblbe_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for required in ("wblbe_create", "wblbe_set_params", "wblbe_init_rho", "wblbe_step",
                     "wblbe_run_until_equilibrium", "wblbe_moments", "wblbe_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = wblbe.load_library()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(declared_functions()) <= set(wblbe._SIGNATURES)


def _params(**kw):
    base = dict(nx=64, ny=48, tau=0.8, kappa=0.01, beta=0.006, rho_l=1.0, rho_g=0.1)
    base.update(kw)
    return wblbe.Params(**base)


def test_workspace_bytes_on_host():
    lib = wblbe.load_library()
    p64 = _params().c()
    p32 = _params(precision=wblbe.FP32_SHIFTED).c()
    b64 = lib.wblbe_workspace_bytes(ctypes.byref(p64))
    b32 = lib.wblbe_workspace_bytes(ctypes.byref(p32))
    # two population buffers of 9 planes (rows padded to 128 bytes) at least
    assert b64 >= 2 * 9 * 48 * 64 * 8
    assert b32 >= 2 * 9 * 48 * 64 * 4
    assert b64 % 256 == 0 and b32 % 256 == 0
    assert b32 < b64


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=-1), dict(tau=0.5), dict(tau=math.nan),
                                 dict(kappa=-1e-3), dict(beta=0.0), dict(rho_g=0.0),
                                 dict(rho_l=0.05), dict(scheme=7), dict(precision=3)])
def test_invalid_parameters_rejected_on_host(bad):
    lib = wblbe.load_library()
    p = _params(**bad).c()
    assert lib.wblbe_workspace_bytes(ctypes.byref(p)) == 0
    h = ctypes.c_void_p()
    st = lib.wblbe_create(ctypes.byref(p), ctypes.c_void_p(256), 1 << 30, None, ctypes.byref(h))
    assert st == wblbe.EINVAL
    assert lib.wblbe_last_error(None)


def test_null_handle_calls_return_einval():
    lib = wblbe.load_library()
    assert lib.wblbe_step(None, 1) == wblbe.EINVAL
    assert lib.wblbe_destroy(None) == wblbe.EINVAL
    assert lib.wblbe_init_rho(None, None, 0) == wblbe.EINVAL
    assert lib.wblbe_moments(None, None, None, None, None, 0, None) == wblbe.EINVAL
    assert lib.wblbe_step_count(None) == -1


def test_largest_lattice_and_plane_offset_limit():
    """Plane offsets are 32-bit: a lattice whose padded plane reaches 2^31
    elements is rejected on the host; 32768 x 32768 (2^30 nodes, 2 x 77 GB in
    FP64) is accepted, and its workspace covers both population buffers."""
    lib = wblbe.load_library()
    ok = _params(nx=32768, ny=32768).c()
    b = lib.wblbe_workspace_bytes(ctypes.byref(ok))
    assert b >= 2 * 9 * 32768 * 32768 * 8
    for nx, ny in [(65536, 32768), (46340, 46341)]:
        p = _params(nx=nx, ny=ny).c()
        assert lib.wblbe_workspace_bytes(ctypes.byref(p)) == 0, (nx, ny)


@pytest.mark.parametrize("shape", [(0, 0), (0, 5), (5, 0)])
def test_empty_lattices_rejected(shape):
    lib = wblbe.load_library()
    p = _params(nx=shape[0], ny=shape[1]).c()
    assert lib.wblbe_workspace_bytes(ctypes.byref(p)) == 0


@pytest.mark.parametrize("scheme", [wblbe.STANDARD_PRESSURE, wblbe.STANDARD_TEXTBOOK,
                                    wblbe.STANDARD_E6])
def test_variant_schemes_single_lattice_only(scheme):
    """The Sec. II comparison variants are valid for a single lattice and
    refused by the batch API (before any device work)."""
    lib = wblbe.load_library()
    p = _params(scheme=scheme).c()
    assert lib.wblbe_workspace_bytes(ctypes.byref(p)) > 0
    cfg = wblbe.CBatchConfig(128, 32, 1)
    h = ctypes.c_void_p()
    st = lib.wblbe_batch_create(scheme, wblbe.FP64, 4, 64, 4096, ctypes.c_void_p(256), 1 << 30,
                                None, ctypes.byref(cfg), ctypes.byref(h))
    assert st == wblbe.EINVAL and not h.value
    assert b"single lattices" in lib.wblbe_batch_last_error(None)


def test_e6_scheme_is_fp64_only():
    lib = wblbe.load_library()
    p = _params(scheme=wblbe.STANDARD_E6, precision=wblbe.FP32_SHIFTED).c()
    assert lib.wblbe_workspace_bytes(ctypes.byref(p)) == 0


def test_workspace_too_small_is_enomem():
    """The library borrows its workspace: one below wblbe_workspace_bytes is
    refused with ENOMEM before any device work."""
    lib = wblbe.load_library()
    p = _params().c()
    need = lib.wblbe_workspace_bytes(ctypes.byref(p))
    h = ctypes.c_void_p()
    st = lib.wblbe_create(ctypes.byref(p), ctypes.c_void_p(256), need - 256, None,
                          ctypes.byref(h))
    assert st == wblbe.ENOMEM and not h.value
    assert b"needs" in lib.wblbe_last_error(None)


def test_batch_host_side_validation():
    """Batch sizes, case sizes, configurations and NULL handles are checked on
    the host, before any device work."""
    lib = wblbe.load_library()
    assert lib.wblbe_batch_workspace_bytes(0, 64, 4096, 1 << 20) == 0
    assert lib.wblbe_batch_workspace_bytes(4, 0, 4096, 1 << 20) == 0
    assert lib.wblbe_batch_workspace_bytes(4, 64, 63, 1 << 20) == 0
    ok = lib.wblbe_batch_workspace_bytes(4, 64, 4096, 1 << 20)
    assert ok > (1 << 20) and ok % 256 == 0
    small = _params(nx=7, ny=64).c()
    assert lib.wblbe_batch_case_bytes(ctypes.byref(small)) == 0      # nx < 8
    case = _params(nx=64, ny=48, precision=wblbe.FP32_SHIFTED).c()
    assert lib.wblbe_batch_case_bytes(ctypes.byref(case)) >= 2 * 9 * 64 * 48 * 4
    h = ctypes.c_void_p()
    for cfg in (wblbe.CBatchConfig(96, 32, 1), wblbe.CBatchConfig(128, 2, 1),
                wblbe.CBatchConfig(128, 32, 0)):
        st = lib.wblbe_batch_create(wblbe.WELL_BALANCED, wblbe.FP32_SHIFTED, 4, 64, 4096,
                                    ctypes.c_void_p(256), ok, None, ctypes.byref(cfg),
                                    ctypes.byref(h))
        assert st == wblbe.EINVAL and not h.value
    cfg = wblbe.CBatchConfig(128, 32, 1)
    st = lib.wblbe_batch_create(wblbe.WELL_BALANCED, 7, 4, 64, 4096, ctypes.c_void_p(256), ok,
                                None, ctypes.byref(cfg), ctypes.byref(h))
    assert st == wblbe.EINVAL                                          # unknown precision
    st = lib.wblbe_batch_create(wblbe.WELL_BALANCED, wblbe.FP64, 4, 64, 4096,
                                ctypes.c_void_p(100), ok, None, ctypes.byref(cfg),
                                ctypes.byref(h))
    assert st == wblbe.EINVAL and b"aligned" in lib.wblbe_batch_last_error(None)
    n = ctypes.c_int32()
    assert lib.wblbe_batch_advance(None, 1) == wblbe.EINVAL
    assert lib.wblbe_batch_poll(None, None, 0, ctypes.byref(n)) == wblbe.EINVAL
    assert lib.wblbe_batch_retire(None, 0) == wblbe.EINVAL
    assert lib.wblbe_batch_destroy(None) == wblbe.EINVAL
