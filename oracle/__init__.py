"""FP64 CPU oracle for the D2Q9 + NSBC update (Euser & Vuik, arXiv 2005.08674).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package.

The solver itself is plain C (``lbm_oracle.c``), built with
``-O2 -ffp-contract=off`` and driven through ctypes.  ``reflection.py`` holds
the energy measure used to quantify reflections.  Which paper passage each
function follows is stated in the C file's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_LIB_OMP = os.path.join(_HERE, "liblbm_oracle_omp.so")
_lock = threading.Lock()
_libs = {}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into ``oracle/liblbm_oracle.so`` (gcc, no FMA
    contraction).  ``openmp=True`` builds ``liblbm_oracle_omp.so`` from the same
    source with the row loop split over threads (bit-identical results)."""
    out = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu99", "-fPIC",
             *(["-fopenmp"] if openmp else []), "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def lib(openmp: bool = False):
    with _lock:
        if openmp not in _libs:
            # a test may point the oracle at a deliberately broken build of the
            # same source, to show that the pins catch the planted mistake
            override = os.environ.get("LBM_ORACLE_LIB")
            L = ctypes.CDLL(override if override else build(openmp=openmp))
            L.or_create.restype = ctypes.c_void_p
            L.or_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.or_destroy.argtypes = [ctypes.c_void_p]
            L.or_set_nsbc.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int]
            L.or_set_periodic.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
            L.or_set_corner_mode.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.or_set_velocity_edge.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double]
            L.or_set_collision.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
            L.or_mrt_matrix.argtypes = [ctypes.c_void_p, _dp]
            L.or_init.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
            L.or_set_f.argtypes = [ctypes.c_void_p, _dp]
            L.or_get_f.argtypes = [ctypes.c_void_p, _dp]
            L.or_macros.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
            L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.or_steps.restype = ctypes.c_long
            L.or_steps.argtypes = [ctypes.c_void_p]
            L.or_equilibrium.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
            L.or_lattice.argtypes = [_ip, _ip, _dp, _ip]
            L.or_set_storage.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
            _libs[openmp] = L
    return _libs[openmp]


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def equilibrium(rho: float, ux: float, uy: float) -> np.ndarray:
    """Eq. (feq_1) at one state; returns the 9 populations."""
    out = np.zeros(9)
    lib().or_equilibrium(rho, ux, uy, _p(out))
    return out


def lattice():
    """(cx, cy, w, opposite) exactly as the oracle uses them."""
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = np.zeros(9)
    opp = (ctypes.c_int * 9)()
    lib().or_lattice(cx, cy, _p(w), opp)
    return np.array(cx[:]), np.array(cy[:]), w, np.array(opp[:])


class Oracle:
    """One FP64 simulation: nx x ny nodes, NSBC on every non-periodic edge."""

    def __init__(self, nx: int, ny: int, tau: float, farfield_rho: float = 1.0,
                 farfield_u=(0.0, 0.0), gamma: float = 0.6, beta: float = 0.0,
                 kappa: float = 3.0, grad_order: int = 1, periodic=(False, False),
                 collision: str = "bgk", mrt_rates=None, openmp: bool = False, velocity_edges=None,
                 corner_mode: int = 0):
        """velocity_edges: {side: (ux, uy)} with side 0 left, 1 right, 2 bottom, 3 top.
        corner_mode: 0 = diagonal normal at corners, 1 = mean of the m_c the two
        edges meeting at the corner predict (readings of Sec. 5, silent on corners)."""
        self._L = lib(openmp)
        h = self._L.or_create(nx, ny, tau, farfield_rho, farfield_u[0], farfield_u[1])
        if not h:
            raise ValueError(f"oracle rejected nx={nx} ny={ny} tau={tau}")
        self._h = ctypes.c_void_p(h)
        self.nx, self.ny, self.tau = nx, ny, tau
        self._L.or_set_nsbc(self._h, gamma, beta, kappa, grad_order)
        self._L.or_set_corner_mode(self._h, int(corner_mode))
        self._L.or_set_periodic(self._h, int(periodic[0]), int(periodic[1]))
        for side, (vx, vy) in (velocity_edges or {}).items():
            self._L.or_set_velocity_edge(self._h, int(side), 1, float(vx), float(vy))
        if collision == "mrt":
            r = np.ascontiguousarray(mrt_rates, dtype=np.float64)
            assert r.shape == (9,)
            self._L.or_set_collision(self._h, 1, _p(r))
        elif collision != "bgk":
            raise ValueError(collision)

    def close(self):
        if getattr(self, "_h", None):
            self._L.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, ux, uy):
        """f := f^eq(rho, u) at every node; fields [ny][nx]."""
        rho, ux, uy = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
        for a in (rho, ux, uy):
            assert a.shape == (self.ny, self.nx)
        self._L.or_init(self._h, _p(rho), _p(ux), _p(uy))
        return self

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx)
        self._L.or_set_f(self._h, _p(f))
        return self

    def get_f(self) -> np.ndarray:
        f = np.zeros((9, self.ny, self.nx))
        self._L.or_get_f(self._h, _p(f))
        return f

    def step(self, n: int = 1):
        self._L.or_step(self._h, int(n))
        return self

    STORAGE_FORMATS = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}

    def storage(self, fmt: str, far_field_shift: bool = True):
        """Storage emulation (a test instrument): from now on, and at once, every
        population is kept as its deviation from f^eq(m_0) (or from w_i)
        rounded through `fmt` (f32, f16 scaled by 2^12, bf16); "f64" is off.
        All arithmetic stays double, so the difference to a plain run is what
        the narrower storage alone loses."""
        self._L.or_set_storage(self._h, self.STORAGE_FORMATS[fmt], int(bool(far_field_shift)))
        return self

    @property
    def steps(self) -> int:
        return int(self._L.or_steps(self._h))

    def macros(self):
        """(rho, ux, uy) of the stored post-collision state, each [ny][nx]."""
        rho = np.zeros((self.ny, self.nx))
        ux = np.zeros_like(rho)
        uy = np.zeros_like(rho)
        self._L.or_macros(self._h, _p(rho), _p(ux), _p(uy))
        return rho, ux, uy

    def mrt_matrix(self) -> np.ndarray:
        M = np.zeros(81)
        self._L.or_mrt_matrix(self._h, _p(M))
        return M.reshape(9, 9)
