"""ctypes shim over the FP64 C oracle of the three-dimensional (D3Q19) form
of the well-balanced LBE and of the standard LBE, ``wblbe3_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the benchmark's CPU legs may import this module.  It imports nothing from
the CUDA package and the CUDA package imports nothing from here.

Population arrays have shape (19, nz, ny, nx); scalar fields (nz, ny, nx);
vector fields (3, nz, ny, nx).  A population array holds f_i(x, t) after
streaming and before collision.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "wblbe3_oracle.c"
BUILD_DIR = HERE / "_build"
LIB_PATH = BUILD_DIR / f"liboracle3_{platform.machine()}.so"
LIB_PAIRWISE_PATH = BUILD_DIR / f"liboracle3_pairwise_{platform.machine()}.so"

STANDARD = 0
WELL_BALANCED = 1
Q = 19


def build(force: bool = False, pairwise_density: bool = False) -> Path:
    """Compile the C oracle (plain gcc, no FMA contraction) if needed;
    ``pairwise_density`` builds its rounding-sensitivity variant."""
    BUILD_DIR.mkdir(exist_ok=True)
    path = LIB_PAIRWISE_PATH if pairwise_density else LIB_PATH
    if force or not path.exists() or path.stat().st_mtime < SRC.stat().st_mtime:
        tmp = path.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(
            ["gcc", "-O3", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
             *(["-DORC_DENSITY_PAIRWISE"] if pairwise_density else []),
             "-fPIC", "-shared", "-o", str(tmp), str(SRC), "-lm"])
        os.replace(tmp, path)
    return path


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau", ctypes.c_double), ("kappa", ctypes.c_double),
                ("beta", ctypes.c_double), ("rho_l", ctypes.c_double),
                ("rho_g", ctypes.c_double), ("rho0", ctypes.c_double),
                ("scheme", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("umax", ctypes.c_double),
                ("mu_min", ctypes.c_double), ("mu_max", ctypes.c_double),
                ("kinetic", ctypes.c_double), ("nonfinite", ctypes.c_int)]


_libs = {}


def _load(pairwise_density: bool = False):
    if pairwise_density not in _libs:
        lib = ctypes.CDLL(str(build(pairwise_density=pairwise_density)))
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        pp = ctypes.POINTER(_Params)
        lib.o3_lattice.argtypes = [ip, ip, ip, dp]
        lib.o3_mu0.argtypes = [pp, ctypes.c_double]
        lib.o3_mu0.restype = ctypes.c_double
        lib.o3_laplacian.argtypes = [pp, dp, dp]
        lib.o3_gradient.argtypes = [pp, dp, dp, dp, dp]
        lib.o3_feq.argtypes = [pp, ctypes.c_double, dp, dp]
        lib.o3_forcing.argtypes = [pp, dp, dp, dp, dp]
        lib.o3_macro.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        lib.o3_init.argtypes = [pp, dp, dp]
        lib.o3_step.argtypes = [pp, dp, ctypes.c_long]
        lib.o3_step.restype = ctypes.c_int
        lib.o3_stats_of.argtypes = [pp, dp, ctypes.POINTER(_Stats)]
        _libs[pairwise_density] = lib
    return _libs[pairwise_density]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lattice():
    """The D3Q19 velocity set (cx, cy, cz as int arrays) and weights."""
    lib = _load()
    cx, cy, cz = ((ctypes.c_int * Q)() for _ in range(3))
    w = (ctypes.c_double * Q)()
    lib.o3_lattice(cx, cy, cz, w)
    return np.array(cx), np.array(cy), np.array(cz), np.array(w)


@dataclass
class Params:
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

    def _c(self) -> _Params:
        return _Params(self.nx, self.ny, self.nz, self.tau, self.kappa, self.beta,
                       self.rho_l, self.rho_g, self.rho0, self.scheme)


class Oracle3:
    """FP64 CPU oracle of the D3Q19 scheme, bound to one parameter set."""

    def __init__(self, params: Params, pairwise_density: bool = False):
        self.p = params
        self._cp = params._c()
        self._lib = _load(pairwise_density)

    @property
    def shape(self):
        return (self.p.nz, self.p.ny, self.p.nx)

    def mu0(self, rho: float) -> float:
        return self._lib.o3_mu0(ctypes.byref(self._cp), float(rho))

    def laplacian(self, phi) -> np.ndarray:
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        out = np.empty_like(phi)
        self._lib.o3_laplacian(ctypes.byref(self._cp), _ptr(phi), _ptr(out))
        return out

    def gradient(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        g = [np.empty_like(phi) for _ in range(3)]
        self._lib.o3_gradient(ctypes.byref(self._cp), _ptr(phi), *[_ptr(a) for a in g])
        return g

    def feq(self, rho, u) -> np.ndarray:
        out = np.empty(Q)
        self._lib.o3_feq(ctypes.byref(self._cp), float(rho),
                         _ptr(np.ascontiguousarray(u, dtype=np.float64)), _ptr(out))
        return out

    def forcing(self, u, F, grho) -> np.ndarray:
        out = np.empty(Q)
        args = [_ptr(np.ascontiguousarray(v, dtype=np.float64)) for v in (u, F, grho)]
        self._lib.o3_forcing(ctypes.byref(self._cp), *args, _ptr(out))
        return out

    def init(self, rho) -> np.ndarray:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        assert rho.shape == self.shape
        f = np.empty((Q,) + self.shape)
        self._lib.o3_init(ctypes.byref(self._cp), _ptr(rho), _ptr(f))
        return f

    def step(self, f: np.ndarray, nsteps: int = 1) -> np.ndarray:
        assert f.shape == (Q,) + self.shape
        if self._lib.o3_step(ctypes.byref(self._cp), _ptr(f), int(nsteps)) != 0:
            raise MemoryError("oracle step: out of memory")
        return f

    def macro(self, f: np.ndarray) -> dict:
        out = {"rho": np.empty(self.shape), "mu": np.empty(self.shape),
               "u": np.empty((3,) + self.shape), "F": np.empty((3,) + self.shape),
               "grho": np.empty((3,) + self.shape)}
        self._lib.o3_macro(ctypes.byref(self._cp), _ptr(f), _ptr(out["rho"]), _ptr(out["mu"]),
                           _ptr(out["u"]), _ptr(out["F"]), _ptr(out["grho"]))
        return out

    def stats(self, f: np.ndarray) -> dict:
        st = _Stats()
        self._lib.o3_stats_of(ctypes.byref(self._cp), _ptr(f), ctypes.byref(st))
        return {"mass": st.mass, "umax": st.umax, "mu_min": st.mu_min, "mu_max": st.mu_max,
                "kinetic": st.kinetic, "nonfinite": bool(st.nonfinite)}
