"""FP64 serial oracle of the explicit finite-volume step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product library never does: it shares
no code with the oracle, and the oracle never calls the library.

``build()`` compiles ``gg_oracle.c`` with gcc (serial, IEEE double, no FMA
contraction, no architecture flags, so x86-64 and aarch64 give the same bits)
into ``liboracle_gg.so`` next to this file; the functions below are thin
ctypes wrappers taking float64 numpy arrays of shape (ny, nx).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_gg.so")
_FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or out of date."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *_FLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def build_openmp() -> Optional[str]:
    """The same source built with -fopenmp (the row loop of the step runs on
    every host core), for the multi-core CPU baseline; None if the compiler
    has no OpenMP."""
    lib = os.path.join(_HERE, "liboracle_gg_omp.so")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".{os.getpid()}.tmp"
        r = subprocess.run(["gcc", *_FLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, lib)
    return lib


def threads() -> int:
    """Threads the loaded library's step runs on."""
    return int(_load().ggo_threads())


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("no_reaction", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("delta", ctypes.c_double), ("rho", ctypes.c_double),
        ("D", ctypes.c_double), ("c", ctypes.c_double), ("dt", ctypes.c_double),
    ]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    if True:
        P = ctypes.POINTER(_Problem)
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.ggo_coefficients.argtypes = [i64, _D, _D, _D, _D, _D, _D]
        lib.ggo_coefficients.restype = None
        lib.ggo_lambda_max.argtypes = [i64, _D, _D, _D]
        lib.ggo_lambda_max.restype = dbl
        lib.ggo_dt_max.argtypes = [dbl] * 7
        lib.ggo_dt_max.restype = dbl
        lib.ggo_tumour_operator.argtypes = [i32, i32, dbl, dbl, _D, _D, _D]
        lib.ggo_tumour_operator.restype = None
        lib.ggo_acid_operator.argtypes = [i32, i32, dbl, dbl, _D, _D, _D, _D, _D]
        lib.ggo_acid_operator.restype = None
        lib.ggo_step.argtypes = [P, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        lib.ggo_step.restype = None
        lib.ggo_run.argtypes = [P, _D, _D, _D, _D, _D, _D, i64]
        lib.ggo_run.restype = ctypes.c_int
        lib.ggo_adaptive_dt.argtypes = [P, dbl, dbl, _D, _D, _D]
        lib.ggo_adaptive_dt.restype = dbl
        lib.ggo_run_adaptive.argtypes = [P, _D, _D, _D, dbl, dbl, i64, _D, _D, _D, i64, _D, _D]
        lib.ggo_run_adaptive.restype = ctypes.c_int
        lib.ggo_diagnostics.argtypes = [i32, i32, dbl, dbl, _D, _D, _D, dbl, _D]
        lib.ggo_diagnostics.restype = None
        lib.ggo_step_vjp.argtypes = [P, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        lib.ggo_step_vjp.restype = ctypes.c_int
        lib.ggo_adjoint.argtypes = [P, _D, _D, _D, _D, _D, _D, i64, _D, _D, _D, _D, _D, _D, _D]
        lib.ggo_adjoint.restype = ctypes.c_int
        lib.ggo_coefficients_vjp.argtypes = [i64, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        lib.ggo_coefficients_vjp.restype = None
        lib.ggo_front_rays.argtypes = [i32, i32, dbl, dbl, _D, _D, i32, i32, dbl, dbl, dbl, _D]
        lib.ggo_front_rays.restype = None
        lib.ggo_front_speed.argtypes = [_D, _D, dbl, _D]
        lib.ggo_front_speed.restype = None
        lib.ggo_threads.argtypes = []
        lib.ggo_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def use_library(path: Optional[str]):
    """Point the wrappers at another build of gg_oracle.c (None: the default
    build).  Used by the tests that plant mistakes in a copy of the oracle."""
    global _lib
    _lib = None if path is None else _configure(ctypes.CDLL(path))


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


@dataclass
class Setup:
    """Grid, rates and time step of one oracle run."""
    nx: int
    ny: int
    delta: float
    rho: float
    D: float
    c: float
    dt: float
    no_reaction: bool = False
    lx: float = 1.0
    ly: float = 1.0

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dy(self) -> float:
        return self.ly / self.ny

    def struct(self) -> _Problem:
        return _Problem(self.nx, self.ny, int(self.no_reaction), 0, self.dx, self.dy,
                        self.delta, self.rho, self.D, self.c, self.dt)


def coefficients(theta, l1, l2):
    """eq. (2): (a11, a12, a22) of A = R(theta) diag(l1, l2) R(theta)^T."""
    theta, l1, l2 = _f64(theta), _f64(l1), _f64(l2)
    a11, a12, a22 = (np.empty_like(theta) for _ in range(3))
    _load().ggo_coefficients(theta.size, _p(theta), _p(l1), _p(l2), _p(a11), _p(a12), _p(a22))
    return a11, a12, a22


def lambda_max(a11, a12, a22) -> float:
    a11, a12, a22 = _f64(a11), _f64(a12), _f64(a22)
    return float(_load().ggo_lambda_max(a11.size, _p(a11), _p(a12), _p(a22)))


def dt_max(dx, dy, Lambda, delta, rho, D, c) -> float:
    return float(_load().ggo_dt_max(dx, dy, Lambda, delta, rho, D, c))


def stable_dt(nx, ny, a11, a12, a22, delta, rho, D, c, cfl=0.9, lx=1.0, ly=1.0) -> float:
    """CFL * dt_max with Lambda = max(lambda_max(A), D) (the oracle's step rule)."""
    lam = lambda_max(a11, a12, a22)
    return cfl * dt_max(lx / nx, ly / ny, lam, delta, rho, D, c)


def tumour_operator(U, V, dx, dy):
    """Table 1: D1(V; U)."""
    U, V = _f64(U), _f64(V)
    ny, nx = U.shape
    out = np.empty_like(U)
    _load().ggo_tumour_operator(nx, ny, dx, dy, _p(U), _p(V), _p(out))
    return out


def acid_operator(a11, a12, a22, W, dx, dy):
    """Table 2: D2(W; A) with the zero-flux boundary reading."""
    a11, a12, a22, W = _f64(a11), _f64(a12), _f64(a22), _f64(W)
    ny, nx = W.shape
    out = np.empty_like(W)
    _load().ggo_acid_operator(nx, ny, dx, dy, _p(a11), _p(a12), _p(a22), _p(W), _p(out))
    return out


def step(s: Setup, a11, a12, a22, U, V, W):
    """One step of eq. (3); returns new (U, V, W)."""
    a11, a12, a22, U, V, W = (_f64(x) for x in (a11, a12, a22, U, V, W))
    Uo, Vo, Wo = np.empty_like(U), np.empty_like(V), np.empty_like(W)
    st = s.struct()
    _load().ggo_step(ctypes.byref(st), _p(a11), _p(a12), _p(a22), _p(U), _p(V), _p(W),
                     _p(Uo), _p(Vo), _p(Wo))
    return Uo, Vo, Wo


def run(s: Setup, a11, a12, a22, U, V, W, nsteps: int):
    """nsteps steps of eq. (3) from (U, V, W); returns the final (U, V, W)."""
    a11, a12, a22 = _f64(a11), _f64(a12), _f64(a22)
    U, V, W = (np.array(x, dtype=np.float64, order="C") for x in (U, V, W))
    st = s.struct()
    rc = _load().ggo_run(ctypes.byref(st), _p(a11), _p(a12), _p(a22), _p(U), _p(V), _p(W), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle run: allocation failed")
    return U, V, W


def adaptive_dt(s: Setup, lambda_a: float, cfl: float, U, V, W) -> float:
    """Delta t_k of the adaptive step rule on the state (U, V, W)."""
    U, V, W = _f64(U), _f64(V), _f64(W)
    st = s.struct()
    return float(_load().ggo_adaptive_dt(ctypes.byref(st), float(lambda_a), float(cfl), _p(U), _p(V), _p(W)))


def run_adaptive(s: Setup, a11, a12, a22, lambda_a: float, cfl: float, every: int, U, V, W, nsteps: int):
    """nsteps steps with Delta t_k recomputed every `every` steps; returns
    (U, V, W), the time advanced and the last Delta t_k."""
    a11, a12, a22 = _f64(a11), _f64(a12), _f64(a22)
    U, V, W = (np.array(x, dtype=np.float64, order="C") for x in (U, V, W))
    st = s.struct()
    t, dt = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = _load().ggo_run_adaptive(ctypes.byref(st), _p(a11), _p(a12), _p(a22), float(lambda_a), float(cfl),
                                  int(every), _p(U), _p(V), _p(W), int(nsteps), ctypes.byref(t), ctypes.byref(dt))
    if rc != 0:
        raise MemoryError("oracle run: allocation failed")
    return (U, V, W), t.value, dt.value


def diagnostics(U, V, W, dx, dy, eps=0.01):
    """Integrals, minima, maxima, non-finite count, tumour and gap areas."""
    U, V, W = _f64(U), _f64(V), _f64(W)
    ny, nx = U.shape
    out = np.zeros(12)
    _load().ggo_diagnostics(nx, ny, dx, dy, _p(U), _p(V), _p(W), eps, _p(out))
    return dict(mass=out[0:3].copy(), min=out[3:6].copy(), max=out[6:9].copy(),
                nonfinite=int(out[9]), tumour_area=float(out[10]), gap_area=float(out[11]))


def front_rays(U, V, dx, dy, i0, j0, v_front=0.5, u_edge=0.5, eps=0.01):
    """Front, healthy edge, gap width and ray integrals of V and U along the
    east, west, north and south rays from cell (i0, j0) (Section 2's fronts
    and interstitial gap; definitions in ggo_front_rays)."""
    U, V = _f64(U), _f64(V)
    ny, nx = U.shape
    out = np.zeros(20)
    _load().ggo_front_rays(nx, ny, dx, dy, _p(U), _p(V), int(i0), int(j0), v_front, u_edge, eps, _p(out))
    return dict(front=out[0:4].copy(), edge=out[4:8].copy(), gap=out[8:12].copy(),
                mass_v=out[12:16].copy(), mass_u=out[16:20].copy())


def _front_vec(f):
    return np.ascontiguousarray(np.concatenate([f["front"], f["edge"], f["gap"], f["mass_v"], f["mass_u"]]))


def front_speed(before, after, elapsed):
    """LeVeque-Yee space-averaged front speed along each ray from two
    front_rays results taken `elapsed` time units apart."""
    b, a = _front_vec(before), _front_vec(after)
    out = np.zeros(4)
    _load().ggo_front_speed(_p(b), _p(a), float(elapsed), _p(out))
    return out


def step_vjp(s: Setup, a11, a12, a22, U, V, W, lamU, lamV, lamW):
    """Transpose of one step's Jacobian: returns (lamU, lamV, lamW) at t_k and
    the parameter gradients (ga11, ga12, ga22, gs[4])."""
    a11, a12, a22, U, V, W = (_f64(x) for x in (a11, a12, a22, U, V, W))
    lu, lv, lw = (np.array(x, dtype=np.float64, order="C") for x in (lamU, lamV, lamW))
    g1, g2, g3 = np.zeros_like(U), np.zeros_like(U), np.zeros_like(U)
    gs = np.zeros(4)
    st = s.struct()
    rc = _load().ggo_step_vjp(ctypes.byref(st), _p(a11), _p(a12), _p(a22), _p(U), _p(V), _p(W),
                              _p(lu), _p(lv), _p(lw), _p(g1), _p(g2), _p(g3), _p(gs))
    if rc != 0:
        raise MemoryError("oracle vjp: allocation failed")
    return (lu, lv, lw), (g1, g2, g3), gs


def adjoint(s: Setup, a11, a12, a22, U0, V0, W0, nsteps, lamU, lamV, lamW):
    """Discrete adjoint of nsteps steps (all states stored).  Returns
    (dL/dU0, dL/dV0, dL/dW0), (dL/da11, dL/da12, dL/da22), dL/d(delta,rho,D,c)."""
    a11, a12, a22, U0, V0, W0 = (_f64(x) for x in (a11, a12, a22, U0, V0, W0))
    lu, lv, lw = (np.array(x, dtype=np.float64, order="C") for x in (lamU, lamV, lamW))
    g1, g2, g3 = np.zeros_like(U0), np.zeros_like(U0), np.zeros_like(U0)
    gs = np.zeros(4)
    st = s.struct()
    rc = _load().ggo_adjoint(ctypes.byref(st), _p(a11), _p(a12), _p(a22), _p(U0), _p(V0), _p(W0),
                             int(nsteps), _p(lu), _p(lv), _p(lw), _p(g1), _p(g2), _p(g3), _p(gs))
    if rc != 0:
        raise MemoryError("oracle adjoint: allocation failed")
    return (lu, lv, lw), (g1, g2, g3), gs


def coefficients_vjp(theta, l1, l2, ga11, ga12, ga22):
    """Chain rule of eq. (2) from dL/d(a11, a12, a22) to dL/d(theta, l1, l2)."""
    theta, l1, l2, ga11, ga12, ga22 = (_f64(x) for x in (theta, l1, l2, ga11, ga12, ga22))
    gt, g1, g2 = np.empty_like(theta), np.empty_like(theta), np.empty_like(theta)
    _load().ggo_coefficients_vjp(theta.size, _p(theta), _p(l1), _p(l2), _p(ga11), _p(ga12), _p(ga22),
                                 _p(gt), _p(g1), _p(g2))
    return gt, g1, g2


def misfit(V, Vstar, dx, dy) -> float:
    """L = 1/2 dx dy sum (V - V*)^2, the final-state misfit."""
    d = _f64(V) - _f64(Vstar)
    return 0.5 * dx * dy * float(np.sum(d * d))


def misfit_grad(V, Vstar, dx, dy):
    """dL/dV of ``misfit``."""
    return dx * dy * (_f64(V) - _f64(Vstar))


def setup_for(problem, dt: Optional[float] = None, no_reaction: bool = False) -> "tuple[Setup, tuple]":
    """Setup and (a11, a12, a22) of a synthetic problem (dt from the CFL rule
    unless given)."""
    a = coefficients(problem.theta, problem.lambda1, problem.lambda2)
    if dt is None:
        dt = stable_dt(problem.nx, problem.ny, *a, problem.delta, problem.rho, problem.D, problem.c,
                       cfl=problem.cfl, lx=problem.lx, ly=problem.ly)
    s = Setup(problem.nx, problem.ny, problem.delta, problem.rho, problem.D, problem.c, dt,
              no_reaction, problem.lx, problem.ly)
    return s, a
