"""Thin ctypes binding of the C ABI in include/wblbe.h.

Argument marshalling only: every step of the method runs in the CUDA library
``libwblbe.so``.  PyTorch supplies the device workspace (a uint8 tensor the
handle borrows) and the CUDA stream.  If the library is missing the import
fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass
from pathlib import Path
from typing import Optional

import numpy as np

from . import _build

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ENOTCONVERGED = range(7)
STANDARD, WELL_BALANCED = 0, 1
# variants of the standard scheme compared in Sec. II (single lattices only;
# STANDARD_E6 in FP64 only)
STANDARD_PRESSURE, STANDARD_TEXTBOOK, STANDARD_E6 = 2, 3, 4
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


class CBatchConfig(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int32), ("rows_per_tile", ctypes.c_int32),
                ("steps_per_launch", ctypes.c_int32)]


class CCaseInfo(ctypes.Structure):
    _fields_ = [("case_id", ctypes.c_int64), ("state", ctypes.c_int32),
                ("steps", ctypes.c_int64), ("stats", CStats)]


CASE_RUNNING, CASE_CONVERGED, CASE_MAXSTEPS, CASE_UNSTABLE = range(4)


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
    "wblbe_set_step_count": (ctypes.c_int, [_H, ctypes.c_int64]),
    "wblbe_sequence_scratch_bytes": (ctypes.c_size_t, [_P]),
    "wblbe_run_sequence": (ctypes.c_int, [_H, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P,
                                          ctypes.c_size_t]),
    "wblbe_kernel_launches": (ctypes.c_int64, [_H]),
    "wblbe_destroy": (ctypes.c_int, [_H]),
    "wblbe_last_error": (ctypes.c_char_p, [_H]),
    "wblbe_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32,
                                                      ctypes.c_int64, ctypes.c_size_t]),
    "wblbe_batch_case_bytes": (ctypes.c_size_t, [ctypes.POINTER(CParams)]),
    "wblbe_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int64, _P, ctypes.c_size_t,
                                          _P, ctypes.POINTER(CBatchConfig), ctypes.POINTER(_H)]),
    "wblbe_batch_set_config": (ctypes.c_int, [_H, ctypes.POINTER(CBatchConfig)]),
    "wblbe_batch_get_config": (ctypes.c_int, [_H, ctypes.POINTER(CBatchConfig)]),
    "wblbe_batch_set_wait_limit": (ctypes.c_int, [_H, ctypes.c_int64]),
    "wblbe_batch_admit": (ctypes.c_int, [_H, ctypes.POINTER(CParams), _P, ctypes.c_double,
                                         ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "wblbe_batch_advance": (ctypes.c_int, [_H, ctypes.c_int32]),
    "wblbe_batch_poll": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]),
    "wblbe_batch_case_info": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.POINTER(CCaseInfo)]),
    "wblbe_batch_fetch": (ctypes.c_int, [_H, ctypes.c_int64, _P, _P, _P, _P,
                                         ctypes.POINTER(CStats)]),
    "wblbe_batch_get_populations": (ctypes.c_int, [_H, ctypes.c_int64, _P]),
    "wblbe_batch_retire": (ctypes.c_int, [_H, ctypes.c_int64]),
    "wblbe_batch_counts": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "wblbe_batch_kernel_launches": (ctypes.c_int64, [_H]),
    "wblbe_batch_destroy": (ctypes.c_int, [_H]),
    "wblbe_batch_last_error": (ctypes.c_char_p, [_H]),
    "wblbe_slabs_rows": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]),
    "wblbe_slabs_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(CParams), ctypes.c_int32]),
    "wblbe_slabs_create": (ctypes.c_int, [ctypes.POINTER(CParams), ctypes.c_int32, _P,
                                          ctypes.c_size_t, _P, ctypes.POINTER(_H)]),
    "wblbe_slabs_init_rho": (ctypes.c_int, [_H, _P, ctypes.c_int32]),
    "wblbe_slabs_step": (ctypes.c_int, [_H, ctypes.c_int64]),
    "wblbe_slabs_moments": (ctypes.c_int, [_H, _P, _P, _P, _P, ctypes.c_int32,
                                           ctypes.POINTER(CStats)]),
    "wblbe_slabs_get_populations": (ctypes.c_int, [_H, _P, ctypes.c_int32]),
    "wblbe_slabs_step_count": (ctypes.c_int64, [_H]),
    "wblbe_slabs_kernel_launches": (ctypes.c_int64, [_H]),
    "wblbe_slabs_destroy": (ctypes.c_int, [_H]),
    "wblbe_slabs_last_error": (ctypes.c_char_p, [_H]),
    "wblbe3_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "wblbe3_create": (ctypes.c_int, [ctypes.c_void_p, _P, ctypes.c_size_t, _P,
                                     ctypes.POINTER(_H)]),
    "wblbe3_init_rho": (ctypes.c_int, [_H, _P, ctypes.c_int32]),
    "wblbe3_step": (ctypes.c_int, [_H, ctypes.c_int64]),
    "wblbe3_moments": (ctypes.c_int, [_H, _P, _P, _P, ctypes.c_int32, ctypes.POINTER(CStats)]),
    "wblbe3_get_populations": (ctypes.c_int, [_H, _P, ctypes.c_int32]),
    "wblbe3_step_count": (ctypes.c_int64, [_H]),
    "wblbe3_kernel_launches": (ctypes.c_int64, [_H]),
    "wblbe3_destroy": (ctypes.c_int, [_H]),
    "wblbe3_last_error": (ctypes.c_char_p, [_H]),
    "wblbe_moments_noalloc": (ctypes.c_int, [ctypes.POINTER(CParams), _P, _P, _P, _P, _P,
                                             ctypes.POINTER(CStats), _P]),
    "wblbe_noalloc_last_error": (ctypes.c_char_p, []),
    "wblbe_debug_bounds_errors": (ctypes.c_uint, [ctypes.c_int32]),
    "wblbe_probe_fp64_fma": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            _P]),
    "wblbe_probe_reciprocal": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P]),
}

_lib = None


def load_library(build: bool = True) -> ctypes.CDLL:
    """Load libwblbe.so (building it first if needed).  Raises if it cannot
    be built or loaded: there is no fallback implementation."""
    global _lib
    if _lib is None:
        # WBLBE_LIBRARY selects another build of the library, e.g. the
        # bounds-checked one (_build.build(debug_bounds=True))
        override = os.environ.get("WBLBE_LIBRARY")
        if override:
            path = Path(override)
        else:
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


def _require(cond: bool, what: str):
    """Argument check that stays active under ``python -O``: the C side reads
    and writes as many elements as the lattice has, so a wrong shape, dtype
    or layout must never reach it."""
    if not cond:
        raise ValueError(what)


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
            _require(rho.shape == self.shape, f"rho must have shape {self.shape}")
            self._check(self.lib.wblbe_init_rho(self.h, ctypes.c_void_p(rho.ctypes.data), 0))
        else:
            _require(rho.dtype == self._torch.float64 and rho.is_contiguous(),
                     "rho must be a contiguous float64 tensor")
            _require(tuple(rho.shape) == self.shape, f"rho must have shape {self.shape}")
            self._check(self.lib.wblbe_init_rho(self.h, ctypes.c_void_p(rho.data_ptr()),
                                                1 if rho.is_cuda else 0))

    def moments_into(self, rho=None, ux=None, uy=None, mu=None) -> dict:
        """Write the requested fields into caller tensors/arrays (all on the
        host or all on the device) and return the stats."""
        outs = [rho, ux, uy, mu]
        given = [o for o in outs if o is not None]
        on_dev = bool(given) and not isinstance(given[0], np.ndarray) and given[0].is_cuda
        for o in given:
            if isinstance(o, np.ndarray):
                ok = o.dtype == np.float64 and o.flags.c_contiguous and o.flags.writeable
                dev = False
            else:
                ok = o.dtype == self._torch.float64 and o.is_contiguous()
                dev = o.is_cuda
            _require(ok and tuple(o.shape) == self.shape,
                     f"outputs must be contiguous writable float64 of shape {self.shape}")
            _require(dev == on_dev, "outputs must be all on the host or all on the device")
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
        _require(f.shape == (9,) + self.shape, f"f must have shape {(9,) + self.shape}")
        self._check(self.lib.wblbe_set_populations(self.h, ctypes.c_void_p(f.ctypes.data), 0))

    @property
    def steps(self) -> int:
        return int(self.lib.wblbe_step_count(self.h))

    def run_sequence(self, rho_in, nsteps: int, rho_out) -> list:
        """Relax len(rho_in) initial states one after another, each for nsteps
        steps from f = f^eq(rho, 0), with the host copies overlapping the
        computation (page-locked CPU tensors or numpy arrays; pinned memory
        is what lets the copies overlap).  rho_in, rho_out: equal-length
        lists of host float64 (ny, nx) arrays/tensors (entries may repeat;
        rho_out entries must be writable).  Returns the stats of each final
        state.  The device scratch is allocated once per solver."""
        _require(len(rho_in) == len(rho_out), "rho_in and rho_out must have the same length")
        n = len(rho_in)

        def host_ptr(a, writable):
            if isinstance(a, np.ndarray):
                ok = (a.dtype == np.float64 and a.flags.c_contiguous
                      and (a.flags.writeable or not writable))
                ptr = a.ctypes.data
            else:
                ok = (a.dtype == self._torch.float64 and a.is_contiguous()
                      and not a.is_cuda)
                ptr = a.data_ptr()
            _require(ok and tuple(a.shape) == self.shape,
                     f"states must be contiguous host float64 arrays of shape {self.shape}")
            return ptr

        pin = (ctypes.c_void_p * max(n, 1))(*[host_ptr(a, False) for a in rho_in])
        pout = (ctypes.c_void_p * max(n, 1))(*[host_ptr(a, True) for a in rho_out])
        need = int(self.lib.wblbe_sequence_scratch_bytes(ctypes.byref(self._cp)))
        if getattr(self, "_seq_scratch", None) is None or self._seq_scratch.numel() < need:
            self._seq_scratch = self._torch.empty(need, dtype=self._torch.uint8, device="cuda")
        stats = (CStats * max(n, 1))()
        self._check(self.lib.wblbe_run_sequence(
            self.h, n, ctypes.cast(pin, ctypes.c_void_p), int(nsteps),
            ctypes.cast(pout, ctypes.c_void_p), ctypes.cast(stats, ctypes.c_void_p),
            ctypes.c_void_p(self._seq_scratch.data_ptr()), self._seq_scratch.numel()))
        return [stats[k].as_dict() for k in range(n)]

    def set_step_count(self, step: int):
        """Restore the step counter (e.g. when resuming a checkpoint); in FP32
        well-balanced runs it also seeds the stochastic rounding."""
        self._check(self.lib.wblbe_set_step_count(self.h, int(step)))

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.wblbe_kernel_launches(self.h))


class Batch:
    """Many independent cases resident on the device, advanced together by
    the persistent batched kernel (C ABI wblbe_batch_*).

    ``arena_bytes`` of device memory hold the cases' populations; admission
    returns None (the caller queues the request) when no slot, arena range
    or tile-table room is free."""

    def __init__(self, scheme=WELL_BALANCED, precision=FP32_SHIFTED, max_cases=64,
                 max_tiles=1 << 15, max_case_nodes=1 << 20, arena_bytes=1 << 30,
                 tile_x=128, rows_per_tile=32, steps_per_launch=1, stream=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("wblbe needs a CUDA device")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nbytes = int(self.lib.wblbe_batch_workspace_bytes(max_cases, max_tiles, max_case_nodes,
                                                          arena_bytes))
        if nbytes == 0:
            raise WblbeError(EINVAL, "invalid batch sizes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        cfg = CBatchConfig(tile_x, rows_per_tile, steps_per_launch)
        h = ctypes.c_void_p()
        st = self.lib.wblbe_batch_create(scheme, precision, max_cases, max_tiles, max_case_nodes,
                                         ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                         ctypes.c_void_p(self.stream.cuda_stream),
                                         ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise WblbeError(st, self.lib.wblbe_batch_last_error(None).decode())
        self.h = h
        self.scheme, self.precision = scheme, precision
        self._shapes = {}                      # case id -> (ny, nx) of an admitted case

    def _check(self, st, allow=(OK,)):
        if st not in allow:
            raise WblbeError(st, self.lib.wblbe_batch_last_error(self.h).decode())
        return st

    def _shape_of(self, case_id: int, shape):
        """The case's (ny, nx); a shape given by the caller must match it."""
        known = self._shapes.get(int(case_id))
        if known is None:
            raise WblbeError(EINVAL, f"unknown case {case_id}")
        if shape is not None:
            _require(tuple(shape) == known, f"case {case_id} has shape {known}")
        return known

    def close(self):
        if getattr(self, "h", None):
            self._check(self.lib.wblbe_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, tile_x, rows_per_tile, steps_per_launch):
        cfg = CBatchConfig(tile_x, rows_per_tile, steps_per_launch)
        self._check(self.lib.wblbe_batch_set_config(self.h, ctypes.byref(cfg)))

    def get_config(self):
        cfg = CBatchConfig()
        self._check(self.lib.wblbe_batch_get_config(self.h, ctypes.byref(cfg)))
        return cfg.tile_x, cfg.rows_per_tile, cfg.steps_per_launch

    def set_wait_limit(self, spins):
        self._check(self.lib.wblbe_batch_set_wait_limit(self.h, int(spins)))

    def case_bytes(self, params: Params) -> int:
        cp = params.c()
        return int(self.lib.wblbe_batch_case_bytes(ctypes.byref(cp)))

    def admit(self, params: Params, rho, umax_tol: float, max_steps: int):
        """Returns the case id, or None when the batch is full (ENOMEM)."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        _require(rho.shape == (params.ny, params.nx), "rho must have shape (ny, nx)")
        cp = params.c()
        cid = ctypes.c_int64()
        st = self._check(self.lib.wblbe_batch_admit(self.h, ctypes.byref(cp),
                                                    ctypes.c_void_p(rho.ctypes.data),
                                                    float(umax_tol), int(max_steps),
                                                    ctypes.byref(cid)), allow=(OK, ENOMEM))
        if st == ENOMEM:
            return None
        self._shapes[int(cid.value)] = (params.ny, params.nx)
        return int(cid.value)

    def advance(self, launches: int = 1):
        self._check(self.lib.wblbe_batch_advance(self.h, int(launches)))

    def poll(self, cap: int = 4096):
        ids = (ctypes.c_int64 * cap)()
        n = ctypes.c_int32()
        self._check(self.lib.wblbe_batch_poll(self.h, ids, cap, ctypes.byref(n)))
        return [int(ids[k]) for k in range(n.value)]

    def info(self, case_id: int) -> dict:
        ci = CCaseInfo()
        self._check(self.lib.wblbe_batch_case_info(self.h, int(case_id), ctypes.byref(ci)))
        return {"case_id": ci.case_id, "state": ci.state, "steps": ci.steps,
                "stats": ci.stats.as_dict()}

    def fetch(self, case_id: int, shape=None):
        outs = [np.empty(self._shape_of(case_id, shape)) for _ in range(4)]
        st = CStats()
        self._check(self.lib.wblbe_batch_fetch(self.h, int(case_id),
                                               *[ctypes.c_void_p(o.ctypes.data) for o in outs],
                                               ctypes.byref(st)))
        return dict(zip(("rho", "ux", "uy", "mu"), outs)), st.as_dict()

    def get_populations(self, case_id: int, shape=None) -> np.ndarray:
        f = np.empty((9,) + self._shape_of(case_id, shape))
        self._check(self.lib.wblbe_batch_get_populations(self.h, int(case_id),
                                                         ctypes.c_void_p(f.ctypes.data)))
        return f

    def retire(self, case_id: int):
        self._check(self.lib.wblbe_batch_retire(self.h, int(case_id)))
        self._shapes.pop(int(case_id), None)

    def counts(self) -> dict:
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        fr = ctypes.c_size_t()
        self._check(self.lib.wblbe_batch_counts(self.h, ctypes.byref(a), ctypes.byref(b),
                                                ctypes.byref(c), ctypes.byref(fr)))
        return {"resident": a.value, "running": b.value, "tiles": c.value,
                "arena_free": fr.value}

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.wblbe_batch_kernel_launches(self.h))


def debug_bounds_errors(reset: bool = False) -> int:
    """Out-of-bounds accesses seen by a bounds-checked build of the library
    on the current device (0xFFFFFFFF: the loaded library has no checks)."""
    return int(load_library().wblbe_debug_bounds_errors(1 if reset else 0))


def slab_rows(ny: int, nslabs: int) -> list:
    """First global row of every slab of a lattice split into nslabs row
    slabs (the library's partition; the last entry is ny).  Host only."""
    out = (ctypes.c_int32 * (nslabs + 1))()
    st = load_library().wblbe_slabs_rows(int(ny), int(nslabs), out)
    if st != OK:
        raise WblbeError(st, load_library().wblbe_slabs_last_error(None).decode())
    return list(out)


class Slabs:
    """One lattice split into row slabs on the current CUDA device, each
    advanced with 3 ghost rows on each side that are exchanged every step
    (wblbe_slabs_*).  Same interface and results as Solver."""

    def __init__(self, params: Params, nslabs: int, stream=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.params = params
        self.nslabs = int(nslabs)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._cp = params.c()
        nbytes = int(self.lib.wblbe_slabs_workspace_bytes(ctypes.byref(self._cp), self.nslabs))
        if nbytes == 0:
            raise WblbeError(EINVAL, "invalid parameters or slab count")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        st = self.lib.wblbe_slabs_create(ctypes.byref(self._cp), self.nslabs,
                                         ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise WblbeError(st, self.lib.wblbe_slabs_last_error(None).decode())
        self.h = h

    def _check(self, st: int) -> int:
        if st != OK:
            raise WblbeError(st, self.lib.wblbe_slabs_last_error(self.h).decode())
        return st

    @property
    def shape(self):
        return (self.params.ny, self.params.nx)

    def close(self):
        if getattr(self, "h", None):
            self._check(self.lib.wblbe_slabs_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_rho(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        _require(rho.shape == self.shape, f"rho must have shape {self.shape}")
        self._check(self.lib.wblbe_slabs_init_rho(self.h, ctypes.c_void_p(rho.ctypes.data), 0))

    def step(self, n: int = 1):
        self._check(self.lib.wblbe_slabs_step(self.h, int(n)))

    def moments(self):
        st = CStats()
        outs = [np.empty(self.shape) for _ in range(4)]
        self._check(self.lib.wblbe_slabs_moments(self.h, *[ctypes.c_void_p(o.ctypes.data)
                                                           for o in outs], 0, ctypes.byref(st)))
        return dict(zip(("rho", "ux", "uy", "mu"), outs)), st.as_dict()

    def stats(self) -> dict:
        st = CStats()
        self._check(self.lib.wblbe_slabs_moments(self.h, None, None, None, None, 1,
                                                 ctypes.byref(st)))
        return st.as_dict()

    def get_populations(self) -> np.ndarray:
        f = np.empty((9,) + self.shape)
        self._check(self.lib.wblbe_slabs_get_populations(self.h, ctypes.c_void_p(f.ctypes.data), 0))
        return f

    @property
    def steps(self) -> int:
        return int(self.lib.wblbe_slabs_step_count(self.h))

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.wblbe_slabs_kernel_launches(self.h))


class CParams3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("tau", ctypes.c_double), ("kappa", ctypes.c_double),
                ("beta", ctypes.c_double), ("rho_l", ctypes.c_double),
                ("rho_g", ctypes.c_double), ("rho0", ctypes.c_double),
                ("scheme", ctypes.c_int32), ("precision", ctypes.c_int32)]


# D3Q19 direction order of the wblbe3_* entry points (rest, axes, edges in
# opposite pairs)
D3Q19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
         (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
         (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


@dataclass
class Params3:
    """The three-dimensional (D3Q19) problem: lattice, tau, the free-energy
    parameters, rho0 of Eq. mFeq, the scheme and the precision (FP64, or
    FP32_SHIFTED: float32 deviations from the rest equilibrium at rho_g)."""
    nx: int
    ny: int
    nz: int
    tau: float
    kappa: float
    beta: float
    rho_l: float
    rho_g: float
    rho0: float = 0.0
    scheme: int = WELL_BALANCED
    precision: int = FP64

    def c(self) -> CParams3:
        return CParams3(self.nx, self.ny, self.nz, self.tau, self.kappa, self.beta, self.rho_l,
                        self.rho_g, self.rho0, self.scheme, self.precision)


class Solver3:
    """One D3Q19 lattice (FP64 or FP32-shifted) on the current CUDA device
    (wblbe3_*)."""

    def __init__(self, params: Params3, stream=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.params = params
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._cp = params.c()
        nbytes = int(self.lib.wblbe3_workspace_bytes(ctypes.byref(self._cp)))
        if nbytes == 0:
            raise WblbeError(EINVAL, "invalid parameters")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        st = self.lib.wblbe3_create(ctypes.byref(self._cp),
                                    ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise WblbeError(st, self.lib.wblbe3_last_error(None).decode())
        self.h = h

    def _check(self, st: int) -> int:
        if st != OK:
            raise WblbeError(st, self.lib.wblbe3_last_error(self.h).decode())
        return st

    @property
    def shape(self):
        return (self.params.nz, self.params.ny, self.params.nx)

    def close(self):
        if getattr(self, "h", None):
            self._check(self.lib.wblbe3_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_rho(self, rho):
        if isinstance(rho, np.ndarray):
            rho = np.ascontiguousarray(rho, dtype=np.float64)
            _require(rho.shape == self.shape, f"rho must have shape {self.shape}")
            self._check(self.lib.wblbe3_init_rho(self.h, ctypes.c_void_p(rho.ctypes.data), 0))
        else:
            _require(rho.dtype == self._torch.float64 and rho.is_contiguous()
                     and tuple(rho.shape) == self.shape, f"rho must be float64 {self.shape}")
            self._check(self.lib.wblbe3_init_rho(self.h, ctypes.c_void_p(rho.data_ptr()),
                                                 1 if rho.is_cuda else 0))

    def step(self, n: int = 1):
        self._check(self.lib.wblbe3_step(self.h, int(n)))

    def moments(self):
        st = CStats()
        rho, mu = np.empty(self.shape), np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        self._check(self.lib.wblbe3_moments(self.h, ctypes.c_void_p(rho.ctypes.data),
                                            ctypes.c_void_p(u.ctypes.data),
                                            ctypes.c_void_p(mu.ctypes.data), 0, ctypes.byref(st)))
        return {"rho": rho, "u": u, "mu": mu}, st.as_dict()

    def stats(self) -> dict:
        st = CStats()
        self._check(self.lib.wblbe3_moments(self.h, None, None, None, 1, ctypes.byref(st)))
        return st.as_dict()

    def get_populations(self) -> np.ndarray:
        f = np.empty((19,) + self.shape)
        self._check(self.lib.wblbe3_get_populations(self.h, ctypes.c_void_p(f.ctypes.data), 0))
        return f

    @property
    def steps(self) -> int:
        return int(self.lib.wblbe3_step_count(self.h))

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.wblbe3_kernel_launches(self.h))
