"""ctypes shim over the FP64 C oracle in ``wblbe_oracle.c``.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain FP64 CPU restatement
of the standard LBE (Sec. II) and the well-balanced LBE (Sec. III) of Guo,
arXiv 2012.11075, against which the CUDA library is checked.  Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this module.  It imports nothing from the CUDA package and the CUDA package
imports nothing from here.

Every function works on numpy float64 arrays.  Population arrays have shape
(9, ny, nx) (direction, row, column); scalar fields have shape (ny, nx).
The state held by a population array is f_i(x, t) *after* streaming and
*before* collision, i.e. the left-hand side of Eq. D2Q9 at time t.
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
SRC = HERE / "wblbe_oracle.c"
BUILD_DIR = HERE / "_build"
LIB_PATH = BUILD_DIR / f"liboracle_{platform.machine()}.so"
# timing-only build with the row loops split over threads (same arithmetic)
LIB_OMP_PATH = BUILD_DIR / f"liboracle_omp_{platform.machine()}.so"
# rounding-sensitivity build: the density summed in another order (tests only)
LIB_PAIRWISE_PATH = BUILD_DIR / f"liboracle_pairwise_{platform.machine()}.so"

STANDARD = 0
WELL_BALANCED = 1
# variants of the standard LBE compared in Sec. II
STANDARD_PRESSURE = 2      # pressure-form interaction force
STANDARD_TEXTBOOK = 3           # forcing term of Guo's textbook
STANDARD_E6 = 4            # 6th-order isotropic gradient in the force

# D2Q9 velocity set and weights as the paper states them (Sec. II), kept here
# for tests that need to name a direction.
CX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
CY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
W = (4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36)


def build(force: bool = False, openmp: bool = False, pairwise_density: bool = False) -> Path:
    """Compile the C oracle (plain gcc, no FMA contraction) if needed.
    ``openmp`` builds the timing-only variant whose row loops run on all
    host threads; every node is computed as in the serial build.
    ``pairwise_density`` builds the rounding-sensitivity variant that sums
    rho = sum_i f_i in pairs (nothing else differs)."""
    assert not (openmp and pairwise_density)
    BUILD_DIR.mkdir(exist_ok=True)
    path = LIB_OMP_PATH if openmp else (LIB_PAIRWISE_PATH if pairwise_density else LIB_PATH)
    if force or not path.exists() or path.stat().st_mtime < SRC.stat().st_mtime:
        tmp = path.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(
            ["gcc", "-O3", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
             *(["-fopenmp"] if openmp else []),
             *(["-DORC_DENSITY_PAIRWISE"] if pairwise_density else []),
             "-fPIC", "-shared", "-o", str(tmp), str(SRC), "-lm"])
        os.replace(tmp, path)
    return path


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("tau", ctypes.c_double), ("kappa", ctypes.c_double),
                ("beta", ctypes.c_double), ("rho_l", ctypes.c_double),
                ("rho_g", ctypes.c_double), ("rho0", ctypes.c_double),
                ("scheme", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("umax", ctypes.c_double),
                ("mu_min", ctypes.c_double), ("mu_max", ctypes.c_double),
                ("kinetic", ctypes.c_double), ("nonfinite", ctypes.c_int)]


_libs = {}


def _load(openmp: bool = False, pairwise_density: bool = False):
    key = (openmp, pairwise_density)
    if key not in _libs:
        lib = ctypes.CDLL(str(build(openmp=openmp, pairwise_density=pairwise_density)))
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        for name in ("orc_psi0", "orc_mu0", "orc_p0"):
            fn = getattr(lib, name)
            fn.argtypes = [pp, ctypes.c_double]
            fn.restype = ctypes.c_double
        lib.orc_laplacian.argtypes = [pp, dp, dp]
        lib.orc_gradient.argtypes = [pp, dp, dp, dp]
        lib.orc_gradient6.argtypes = [pp, dp, dp, dp]
        lib.orc_feq.argtypes = [pp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_forcing.argtypes = [pp] + [ctypes.c_double] * 6 + [dp]
        lib.orc_macro.argtypes = [pp, dp] + [dp] * 8
        lib.orc_init.argtypes = [pp, dp, dp]
        lib.orc_step.argtypes = [pp, dp, ctypes.c_long]
        lib.orc_step.restype = ctypes.c_int
        lib.orc_stats_of.argtypes = [pp, dp, ctypes.POINTER(_Stats)]
        _libs[key] = lib
    return _libs[key]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Params:
    """The paper's statement of the problem (Sec. IV) plus the scheme switch.

    rho0 is the numerical constant of Eq. mFeq (the paper sets it to 0)."""
    nx: int
    ny: int
    tau: float
    kappa: float
    beta: float
    rho_l: float
    rho_g: float
    rho0: float = 0.0
    scheme: int = WELL_BALANCED

    def _c(self) -> _Params:
        return _Params(self.nx, self.ny, self.tau, self.kappa, self.beta,
                       self.rho_l, self.rho_g, self.rho0, self.scheme)


class Oracle:
    """FP64 CPU oracle bound to one parameter set."""

    def __init__(self, params: Params, openmp: bool = False, pairwise_density: bool = False):
        """``openmp``: use the timing build whose loops run on all host
        threads (for the benchmark's all-cores baseline); same results.
        ``pairwise_density``: use the rounding-sensitivity build (the density
        summed in another order), which measures the FP64 conditioning of
        the update."""
        self.p = params
        self._cp = params._c()
        self._lib = _load(openmp, pairwise_density)

    # -- free energy (Eq. doubleWell, Eq. EOS) --------------------------------
    def psi0(self, rho: float) -> float:
        return self._lib.orc_psi0(ctypes.byref(self._cp), float(rho))

    def mu0(self, rho: float) -> float:
        return self._lib.orc_mu0(ctypes.byref(self._cp), float(rho))

    def p0(self, rho: float) -> float:
        return self._lib.orc_p0(ctypes.byref(self._cp), float(rho))

    # -- stencils ------------------------------------------------------------------
    def _field(self, phi) -> np.ndarray:
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        assert phi.shape == (self.p.ny, self.p.nx)
        return phi

    def laplacian(self, phi) -> np.ndarray:
        phi = self._field(phi)
        out = np.empty_like(phi)
        self._lib.orc_laplacian(ctypes.byref(self._cp), _ptr(phi), _ptr(out))
        return out

    def gradient(self, phi):
        phi = self._field(phi)
        gx, gy = np.empty_like(phi), np.empty_like(phi)
        self._lib.orc_gradient(ctypes.byref(self._cp), _ptr(phi), _ptr(gx), _ptr(gy))
        return gx, gy

    def gradient6(self, phi):
        """The radius-2, 6th-order isotropic gradient of the E6 variant."""
        phi = self._field(phi)
        gx, gy = np.empty_like(phi), np.empty_like(phi)
        self._lib.orc_gradient6(ctypes.byref(self._cp), _ptr(phi), _ptr(gx), _ptr(gy))
        return gx, gy

    # -- per-node formulas ---------------------------------------------------------
    def feq(self, rho, ux, uy) -> np.ndarray:
        out = np.empty(9)
        self._lib.orc_feq(ctypes.byref(self._cp), rho, ux, uy, _ptr(out))
        return out

    def forcing(self, ux, uy, Fx, Fy, grx=0.0, gry=0.0) -> np.ndarray:
        out = np.empty(9)
        self._lib.orc_forcing(ctypes.byref(self._cp), ux, uy, Fx, Fy, grx, gry, _ptr(out))
        return out

    # -- lattice operations -----------------------------------------------------
    def init(self, rho) -> np.ndarray:
        rho = self._field(rho)
        f = np.empty((9, self.p.ny, self.p.nx))
        self._lib.orc_init(ctypes.byref(self._cp), _ptr(rho), _ptr(f))
        return f

    def step(self, f: np.ndarray, nsteps: int = 1) -> np.ndarray:
        """Advance f in place by nsteps time steps; returns f."""
        assert f.shape == (9, self.p.ny, self.p.nx)
        if self._lib.orc_step(ctypes.byref(self._cp), _ptr(f), int(nsteps)) != 0:
            raise MemoryError("oracle step: out of memory")
        return f

    def macro(self, f: np.ndarray) -> dict:
        """rho, mu, u, F and grad(rho) of the state f (Eq. rhoU, Eq. mF / Sec. II)."""
        names = ("rho", "mu", "ux", "uy", "Fx", "Fy", "grx", "gry")
        out = {k: np.empty((self.p.ny, self.p.nx)) for k in names}
        self._lib.orc_macro(ctypes.byref(self._cp), _ptr(f), *[_ptr(out[k]) for k in names])
        return out

    def stats(self, f: np.ndarray) -> dict:
        st = _Stats()
        self._lib.orc_stats_of(ctypes.byref(self._cp), _ptr(f), ctypes.byref(st))
        return {"mass": st.mass, "umax": st.umax, "mu_min": st.mu_min,
                "mu_max": st.mu_max, "kinetic": st.kinetic,
                "nonfinite": bool(st.nonfinite)}
