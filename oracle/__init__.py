"""Plain FP64 CPU oracle of the coupled LB step of arXiv 2603.22902 (Sections 2-3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library: it has its own C source (``lbo.c``), its own
header and its own parameter structure.

Inputs come from plain Python objects (``workloads.Case``-like: attributes
``nx, ny, N, phases, sigma, ...`` and initial fields), so the oracle never sees
anything produced by the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbo.c")
_HDR = os.path.join(_HERE, "lbo.h")
_LIB = os.path.join(_HERE, "liblbo.so")
_LIB_OMP = os.path.join(_HERE, "liblbo_omp.so")   # the same source built with -fopenmp
_lock = threading.Lock()
_lib = None
_lib_omp = None

MAXN = 4
PERIODIC, WALL, OUTFLOW = 0, 1, 2
ADIABATIC, DIRICHLET = 0, 1


def build(force: bool = False, omp: bool = False) -> str:
    """Compile ``lbo.c`` into ``liblbo.so`` (plain gcc, no contraction of a*b+c); with
    omp=True into ``liblbo_omp.so`` with -fopenmp (the per-cell loops run in threads and
    give bitwise the same results; used only to time the oracle on several cores)."""
    lib = _LIB_OMP if omp else _LIB
    stale = (not os.path.exists(lib)) or any(
        os.path.getmtime(p) > os.path.getmtime(lib) for p in (_SRC, _HDR))
    if force or stale:
        tmp = lib + ".tmp"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC"] + \
              (["-fopenmp"] if omp else []) + ["-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return lib


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("N", ctypes.c_int),
        ("rho_l", ctypes.c_double * MAXN), ("rho_s", ctypes.c_double * MAXN),
        ("mu_l", ctypes.c_double * MAXN), ("mu_s", ctypes.c_double * MAXN),
        ("lam_l", ctypes.c_double * MAXN), ("lam_s", ctypes.c_double * MAXN),
        ("cp_l", ctypes.c_double * MAXN), ("cp_s", ctypes.c_double * MAXN),
        ("latent", ctypes.c_double * MAXN),
        ("sigma", ctypes.c_double * (MAXN * MAXN)),
        ("eps", ctypes.c_double), ("mobility", ctypes.c_double),
        ("T_sol", ctypes.c_double), ("T_liq", ctypes.c_double),
        ("rho_ref", ctypes.c_double), ("cp_ref", ctypes.c_double),
        ("u_solid", ctypes.c_double * 2), ("accel", ctypes.c_double * 2),
        ("bc", ctypes.c_int * 4), ("tbc", ctypes.c_int * 4),
        ("T_wall", ctypes.c_double * 4),
        ("wet_cos", (ctypes.c_double * (MAXN * MAXN)) * 4),
        ("two_phase_textbook", ctypes.c_int),
        ("penalty_literal", ctypes.c_int),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


def _load(omp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if omp else _lib) is None:
            lib = ctypes.CDLL(build(omp=omp))
            lib.lbo_create.restype = ctypes.c_void_p
            lib.lbo_create.argtypes = [ctypes.POINTER(Params), _DP, _DP, _DP, _DP]
            lib.lbo_destroy.argtypes = [ctypes.c_void_p]
            lib.lbo_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            lib.lbo_steps.argtypes = [ctypes.c_void_p]
            lib.lbo_steps.restype = ctypes.c_long
            lib.lbo_fields.argtypes = [ctypes.c_void_p] + [_DP] * 9
            lib.lbo_populations.argtypes = [ctypes.c_void_p, _DP, _DP, _DP]
            lib.lbo_enthalpy_map.argtypes = [ctypes.POINTER(Params), _DP, ctypes.c_double] + [_DP] * 5
            lib.lbo_inverse_map.argtypes = [ctypes.POINTER(Params), _DP, ctypes.c_double]
            lib.lbo_inverse_map.restype = ctypes.c_double
            lib.lbo_stencil.argtypes = [ctypes.POINTER(Params), _DP, _DP, _DP, _DP]
            if omp:
                _lib_omp = lib
            else:
                _lib = lib
    return _lib_omp if omp else _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def make_params(case, two_phase_textbook: bool = False, penalty_literal: bool = False) -> Params:
    """Fill the oracle's parameter structure from a case description."""
    P = Params()
    P.nx, P.ny, P.N = case.nx, case.ny, case.N
    for p, ph in enumerate(case.phases):
        P.rho_l[p], P.rho_s[p] = ph["rho_l"], ph["rho_s"]
        P.mu_l[p], P.mu_s[p] = ph["mu_l"], ph["mu_s"]
        P.lam_l[p], P.lam_s[p] = ph["lam_l"], ph["lam_s"]
        P.cp_l[p], P.cp_s[p] = ph["cp_l"], ph["cp_s"]
        P.latent[p] = ph["latent"]
    sig = np.asarray(case.sigma, dtype=np.float64)
    for p in range(case.N):
        for q in range(case.N):
            P.sigma[p * MAXN + q] = sig[p, q]
    P.eps, P.mobility = case.eps, case.mobility
    P.T_sol, P.T_liq = case.T_sol, case.T_liq
    P.rho_ref, P.cp_ref = case.rho_ref, case.cp_ref
    P.u_solid[0], P.u_solid[1] = case.u_solid
    P.accel[0], P.accel[1] = case.accel
    for side in range(4):
        P.bc[side] = case.bc[side]
        P.tbc[side] = case.tbc[side]
        P.T_wall[side] = case.T_wall[side]
        wc = np.asarray(case.wet_cos[side], dtype=np.float64).reshape(case.N, case.N)
        for p in range(case.N):
            for q in range(case.N):
                P.wet_cos[side][p * MAXN + q] = wc[p, q]
    P.two_phase_textbook = 1 if two_phase_textbook else 0
    P.penalty_literal = 1 if penalty_literal else 0
    return P


class Oracle:
    """The CPU oracle on one case: ``step(n)`` then ``fields()``."""

    def __init__(self, case, two_phase_textbook: bool = False, penalty_literal: bool = False, omp: bool = False):
        self._lib = _load(omp)
        self.case = case
        self.N, self.nx, self.ny = case.N, case.nx, case.ny
        self._P = make_params(case, two_phase_textbook, penalty_literal)
        phi = np.ascontiguousarray(case.phi, dtype=np.float64)
        T = np.ascontiguousarray(case.T, dtype=np.float64)
        ux = np.ascontiguousarray(case.ux, dtype=np.float64)
        uy = np.ascontiguousarray(case.uy, dtype=np.float64)
        h = self._lib.lbo_create(ctypes.byref(self._P), _ptr(phi), _ptr(T), _ptr(ux), _ptr(uy))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.lbo_destroy(h)
            self._h = None

    def step(self, n: int = 1):
        self._lib.lbo_step(self._h, int(n))
        return self

    @property
    def steps(self) -> int:
        return int(self._lib.lbo_steps(self._h))

    def fields(self) -> dict:
        """phi[N,ny,nx], T, H (specific), fl, ux, uy, p, rho, rhoH as float64 arrays."""
        ny, nx, N = self.ny, self.nx, self.N
        out = {k: np.empty((ny, nx)) for k in ("T", "H", "fl", "ux", "uy", "p", "rho", "rhoH")}
        out["phi"] = np.empty((N, ny, nx))
        self._lib.lbo_fields(self._h, _ptr(out["phi"]), _ptr(out["T"]), _ptr(out["H"]),
                             _ptr(out["fl"]), _ptr(out["ux"]), _ptr(out["uy"]), _ptr(out["p"]),
                             _ptr(out["rho"]), _ptr(out["rhoH"]))
        return out

    def populations(self):
        ny, nx, N = self.ny, self.nx, self.N
        f = np.empty((9, ny, nx))
        g = np.empty((N, 9, ny, nx))
        h = np.empty((9, ny, nx))
        self._lib.lbo_populations(self._h, _ptr(f), _ptr(g), _ptr(h))
        return f, g, h


def enthalpy_map(case, phi, rhoH):
    """eq. H on one cell: returns (f_l, T, rho, psi, chi)."""
    lib = _load()
    P = make_params(case)
    ph = np.ascontiguousarray(phi, dtype=np.float64)
    out = [ctypes.c_double() for _ in range(5)]
    lib.lbo_enthalpy_map(ctypes.byref(P), _ptr(ph), float(rhoH),
                         *[ctypes.cast(ctypes.pointer(o), _DP) for o in out])
    return tuple(o.value for o in out)


def inverse_map(case, phi, T):
    lib = _load()
    P = make_params(case)
    ph = np.ascontiguousarray(phi, dtype=np.float64)
    return float(lib.lbo_inverse_map(ctypes.byref(P), _ptr(ph), float(T)))


def stencil(case, field):
    """Isotropic gradient and Laplacian of one scalar field with the case's boundary rules."""
    lib = _load()
    P = make_params(case)
    a = np.ascontiguousarray(field, dtype=np.float64)
    gx, gy, lap = (np.empty_like(a) for _ in range(3))
    lib.lbo_stencil(ctypes.byref(P), _ptr(a), _ptr(gx), _ptr(gy), _ptr(lap))
    return gx, gy, lap
