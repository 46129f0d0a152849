"""Thin ctypes binding of the C ABI in include/wblbe.h.

Argument marshalling only: every step of the method runs in the CUDA library
``libwblbe.so``.  PyTorch supplies the device workspace (a uint8 tensor the
handle borrows) and the CUDA stream.  If the library is missing the import
fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import _build

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ENOTCONVERGED = range(7)
STANDARD, WELL_BALANCED = 0, 1
FP64, FP32_SHIFTED = 0, 1

_STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EUNSTABLE",
                 5: "ETIMEOUT", 6: "ENOTCONVERGED"}


class WblbeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class CParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("tau", ctypes.c_double), ("kappa", ctypes.c_double),
                ("beta", ctypes.c_double), ("rho_l", ctypes.c_double),
                ("rho_g", ctypes.c_double), ("rho0", ctypes.c_double),
                ("rho_ref", ctypes.c_double),
                ("scheme", ctypes.c_int32), ("precision", ctypes.c_int32)]


class CStats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("mass", ctypes.c_double),
                ("mass_drift_rel", ctypes.c_double), ("umax", ctypes.c_double),
                ("mu_min", ctypes.c_double), ("mu_max", ctypes.c_double),
                ("kinetic", ctypes.c_double), ("nonfinite", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class CLaunch(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int32), ("rows_per_cta", ctypes.c_int32)]


# Every entry point declared in include/wblbe.h with its ctypes signature.
_H = ctypes.c_void_p
_P = ctypes.c_void_p
_SIGNATURES = {
    "wblbe_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(CParams)]),
    "wblbe_create": (ctypes.c_int, [ctypes.POINTER(CParams), _P, ctypes.c_size_t, _P,
                                    ctypes.POINTER(_H)]),
    "wblbe_set_params": (ctypes.c_int, [_H, ctypes.POINTER(CParams)]),
    "wblbe_set_launch": (ctypes.c_int, [_H, ctypes.POINTER(CLaunch)]),
    "wblbe_get_launch": (ctypes.c_int, [_H, ctypes.POINTER(CLaunch)]),
    "wblbe_init_rho": (ctypes.c_int, [_H, _P, ctypes.c_int32]),
    "wblbe_step": (ctypes.c_int, [_H, ctypes.c_int64]),
    "wblbe_run_until_equilibrium": (ctypes.c_int, [_H, ctypes.c_double, ctypes.c_int64,
                                                   ctypes.c_int64,
                                                   ctypes.POINTER(ctypes.c_int64),
                                                   ctypes.POINTER(CStats)]),
    "wblbe_moments": (ctypes.c_int, [_H, _P, _P, _P, _P, ctypes.c_int32,
                                     ctypes.POINTER(CStats)]),
    "wblbe_get_populations": (ctypes.c_int, [_H, _P, ctypes.c_int32]),
    "wblbe_set_populations": (ctypes.c_int, [_H, _P, ctypes.c_int32]),
    "wblbe_step_count": (ctypes.c_int64, [_H]),
    "wblbe_kernel_launches": (ctypes.c_int64, [_H]),
    "wblbe_destroy": (ctypes.c_int, [_H]),
    "wblbe_last_error": (ctypes.c_char_p, [_H]),
    "wblbe_moments_noalloc": (ctypes.c_int, [ctypes.POINTER(CParams), _P, _P, _P, _P, _P,
                                             ctypes.POINTER(CStats), _P]),
    "wblbe_noalloc_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load_library(build: bool = True) -> ctypes.CDLL:
    """Load libwblbe.so (building it first if needed).  Raises if it cannot
    be built or loaded: there is no fallback implementation."""
    global _lib
    if _lib is None:
        path = _build.build() if build else _build.LIB_PATH
        if not path.exists():
            raise ImportError(f"CUDA library {path} is missing; run __graft_entry__.build()")
        lib = ctypes.CDLL(str(path))
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


@dataclass
class Params:
    """The paper's statement of the problem (Sec. IV) plus scheme/precision."""
    nx: int
    ny: int
    tau: float
    kappa: float
    beta: float
    rho_l: float
    rho_g: float
    rho0: float = 0.0
    rho_ref: float = math.nan
    scheme: int = WELL_BALANCED
    precision: int = FP64

    def c(self) -> CParams:
        return CParams(self.nx, self.ny, self.tau, self.kappa, self.beta, self.rho_l,
                       self.rho_g, self.rho0, self.rho_ref, self.scheme, self.precision)


def workspace_bytes(params: Params) -> int:
    cp = params.c()
    return int(load_library().wblbe_workspace_bytes(ctypes.byref(cp)))


def _ptr(x) -> int:
    """Device or host address of a torch tensor or numpy array."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Solver:
    """One lattice case on the current CUDA device.

    The workspace is a torch uint8 tensor owned by this object; the stream is
    ``stream`` (a torch.cuda.Stream) or torch's current stream."""

    def __init__(self, params: Params, stream=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.params = params
        if not torch.cuda.is_available():
            raise RuntimeError("wblbe needs a CUDA device")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nbytes = workspace_bytes(params)
        if nbytes == 0:
            raise WblbeError(EINVAL, "invalid parameters")
        # torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self._cp = params.c()
        h = ctypes.c_void_p()
        st = self.lib.wblbe_create(ctypes.byref(self._cp), ctypes.c_void_p(self.workspace.data_ptr()),
                                   nbytes, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise WblbeError(st, self.lib.wblbe_last_error(None).decode())
        self.h = h

    # -- helpers ---------------------------------------------------------------------
    def _check(self, st: int, allow=(OK,)) -> int:
        if st not in allow:
            raise WblbeError(st, self.lib.wblbe_last_error(self.h).decode())
        return st

    @property
    def shape(self):
        return (self.params.ny, self.params.nx)

    def close(self):
        if getattr(self, "h", None):
            self._check(self.lib.wblbe_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API ---------------------------------------------------------------------------
    def set_params(self, params: Params):
        self._cp = params.c()
        self._check(self.lib.wblbe_set_params(self.h, ctypes.byref(self._cp)))
        self.params = params

    def set_launch(self, tile_x: int, rows_per_cta: int):
        l = CLaunch(tile_x, rows_per_cta)
        self._check(self.lib.wblbe_set_launch(self.h, ctypes.byref(l)))

    def get_launch(self):
        l = CLaunch()
        self._check(self.lib.wblbe_get_launch(self.h, ctypes.byref(l)))
        return l.tile_x, l.rows_per_cta

    def init_rho(self, rho):
        """rho: float64 (ny, nx) as a numpy array or CPU tensor (host memory,
        pinned or not) or a CUDA tensor (device memory)."""
        if isinstance(rho, np.ndarray):
            rho = np.ascontiguousarray(rho, dtype=np.float64)
            assert rho.shape == self.shape
            self._check(self.lib.wblbe_init_rho(self.h, ctypes.c_void_p(rho.ctypes.data), 0))
        else:
            assert rho.dtype == self._torch.float64 and rho.is_contiguous()
            assert tuple(rho.shape) == self.shape
            self._check(self.lib.wblbe_init_rho(self.h, ctypes.c_void_p(rho.data_ptr()),
                                                1 if rho.is_cuda else 0))

    def moments_into(self, rho=None, ux=None, uy=None, mu=None) -> dict:
        """Write the requested fields into caller tensors/arrays (all on the
        host or all on the device) and return the stats."""
        outs = [rho, ux, uy, mu]
        given = [o for o in outs if o is not None]
        on_dev = bool(given) and not isinstance(given[0], np.ndarray) and given[0].is_cuda
        ptrs = [None if o is None else ctypes.c_void_p(_ptr(o)) for o in outs]
        st = CStats()
        self._check(self.lib.wblbe_moments(self.h, *ptrs, 1 if on_dev else 0, ctypes.byref(st)))
        return st.as_dict()

    def step(self, n: int = 1):
        self._check(self.lib.wblbe_step(self.h, int(n)))

    def run_until_equilibrium(self, umax_tol: float, max_steps: int, check_every: int = 1000):
        done = ctypes.c_int64()
        st = CStats()
        code = self._check(self.lib.wblbe_run_until_equilibrium(
            self.h, umax_tol, int(max_steps), int(check_every), ctypes.byref(done), ctypes.byref(st)),
            allow=(OK, ENOTCONVERGED, EUNSTABLE))
        return code, int(done.value), st.as_dict()

    def stats(self) -> dict:
        st = CStats()
        self._check(self.lib.wblbe_moments(self.h, None, None, None, None, 1, ctypes.byref(st)))
        return st.as_dict()

    def moments(self, device: bool = False):
        """rho, ux, uy, mu as numpy arrays (device=False) or CUDA tensors."""
        st = CStats()
        if device:
            t = self._torch
            outs = [t.empty(self.shape, dtype=t.float64, device="cuda") for _ in range(4)]
            self._check(self.lib.wblbe_moments(self.h, *[ctypes.c_void_p(o.data_ptr()) for o in outs],
                                               1, ctypes.byref(st)))
        else:
            outs = [np.empty(self.shape) for _ in range(4)]
            self._check(self.lib.wblbe_moments(self.h, *[ctypes.c_void_p(o.ctypes.data) for o in outs],
                                               0, ctypes.byref(st)))
        return dict(zip(("rho", "ux", "uy", "mu"), outs)), st.as_dict()

    def get_populations(self) -> np.ndarray:
        f = np.empty((9,) + self.shape)
        self._check(self.lib.wblbe_get_populations(self.h, ctypes.c_void_p(f.ctypes.data), 0))
        return f

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9,) + self.shape
        self._check(self.lib.wblbe_set_populations(self.h, ctypes.c_void_p(f.ctypes.data), 0))

    @property
    def steps(self) -> int:
        return int(self.lib.wblbe_step_count(self.h))

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.wblbe_kernel_launches(self.h))
