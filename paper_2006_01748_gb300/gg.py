"""ctypes binding of libgg.so (include/gg.h), argument marshalling only.

The functions ``gg_create`` ... ``gg_batch_destroy`` mirror the C entry
points one to one; ``GGSim`` and ``GGBatch`` wrap them with numpy / torch
arrays and raise ``GGError`` on a non-zero status.  Every step of the method
runs in the CUDA kernels of libgg.so: there is no CPU fallback, and loading
fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgg.so")

GG_OK = 0
GG_ERR_ARG = -1
GG_ERR_NOT_SPD = -2
GG_ERR_CFL = -3
GG_ERR_OOM = -4
GG_ERR_CUDA = -5
GG_ERR_NONFINITE = -6
GG_ERR_TIMEOUT = -7
GG_ERR_STATE = -8

GG_FP64_PLAIN = 0
GG_FP32 = 1
GG_FP32_KAHAN = 2
PRECISIONS = {"fp64": GG_FP64_PLAIN, "fp64_plain": GG_FP64_PLAIN, "fp32": GG_FP32, "fp32_kahan": GG_FP32_KAHAN}

FIELDS = {"u": 0, "v": 1, "w": 2, "comp_u": 3, "comp_v": 4, "comp_w": 5, "a11": 6, "a12": 7, "a22": 8,
          "face_x": 9, "face_y": 10, "cross": 11}

# launch-plan kinds of gg_set_plan / gg_plan_info: shared-memory wavefront,
# warp-register wavefront (one column per lane), the plain FP64 kernel, and
# the paired-column warp wavefront (two columns per lane)
PLAN_KINDS = {"smem": 0, "warp": 1, "warp2": 3}
PLAN_NAMES = {0: "smem", 1: "warp", 2: "fp64", 3: "warp2"}
# ensemble launch modes of gg_batch_set_plan / gg_batch_launch_info
BATCH_MODES = ["persistent", "passes", "passes2"]

GG_FLAG_NO_REACTION = 1
GG_FLAG_ALLOW_UNSTABLE = 2


class gg_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("lx", ctypes.c_double), ("ly", ctypes.c_double)]


class gg_params(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("rho", ctypes.c_double), ("D", ctypes.c_double),
                ("c", ctypes.c_double), ("cfl", ctypes.c_double), ("dt", ctypes.c_double),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("steps_per_pass", ctypes.c_int32), ("adapt_every", ctypes.c_int32)]


class gg_diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 3), ("min", ctypes.c_double * 3), ("max", ctypes.c_double * 3),
                ("nonfinite", ctypes.c_int64), ("tumour_area", ctypes.c_double), ("gap_area", ctypes.c_double),
                ("gap_eps", ctypes.c_double)]


class gg_front(ctypes.Structure):
    _fields_ = [("front", ctypes.c_double * 4), ("edge", ctypes.c_double * 4), ("gap", ctypes.c_double * 4),
                ("mass_v", ctypes.c_double * 4), ("mass_u", ctypes.c_double * 4)]


class GGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

# name: (restype, argtypes)
_SIGNATURES = {
    "gg_create": (ctypes.c_int, [ctypes.POINTER(gg_grid), ctypes.POINTER(gg_params), _VP, _VP, _VP, _VP, _VP, _VP,
                                 _VP, ctypes.POINTER(_VP)]),
    "gg_step": (ctypes.c_int, [_VP, _I64]),
    "gg_read": (ctypes.c_int, [_VP, _I32, _VP, _I32, _I32]),
    "gg_write": (ctypes.c_int, [_VP, _I32, _VP, _I32, _I32]),
    "gg_diagnostics": (ctypes.c_int, [_VP, ctypes.POINTER(gg_diag)]),
    "gg_diagnostics_eps": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.POINTER(gg_diag)]),
    "gg_diagnostics_noalloc": (ctypes.c_int, [_VP, _VP, _VP, _I32, _I32, _I32, _I32, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, _VP, ctypes.POINTER(gg_diag)]),
    "gg_adjoint": (ctypes.c_int, [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _DP, _I64]),
    "gg_adjoint_release": (ctypes.c_int, [_VP]),
    "gg_front_rays": (ctypes.c_int, [_VP, _I32, _I32, ctypes.c_double, ctypes.c_double, ctypes.c_double, _VP]),
    "gg_front_speed": (ctypes.c_int, [_VP, _I32, _I32, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      _VP, _VP, _DP]),
    "gg_autotune": (ctypes.c_int, [_VP, _I64, ctypes.POINTER(_I32)]),
    "gg_set_plan": (ctypes.c_int, [_VP, _I32, _I32, _I32, _I32]),
    "gg_plan_info": (ctypes.c_int, [_VP, ctypes.POINTER(_I32)]),
    "gg_dt": (ctypes.c_double, [_VP]),
    "gg_dt_max": (ctypes.c_double, [_VP]),
    "gg_time": (ctypes.c_double, [_VP]),
    "gg_step_count": (_I64, [_VP]),
    "gg_steps_per_pass": (_I32, [_VP]),
    "gg_last_error": (ctypes.c_char_p, [_VP]),
    "gg_error_string": (ctypes.c_char_p, [_I32]),
    "gg_destroy": (ctypes.c_int, [_VP]),
    "gg_batch_create": (ctypes.c_int, [_I32, ctypes.POINTER(gg_grid), ctypes.POINTER(gg_params),
                                       ctypes.POINTER(_VP), _VP, ctypes.POINTER(_VP)]),
    "gg_batch_step": (ctypes.c_int, [_VP, _I64]),
    "gg_batch_read": (ctypes.c_int, [_VP, _I32, _I32, _VP, _I32, _I32]),
    "gg_batch_diagnostics": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(gg_diag)]),
    "gg_batch_dt": (ctypes.c_double, [_VP, _I32]),
    "gg_batch_autotune": (ctypes.c_int, [_VP, _I64, ctypes.POINTER(_I32)]),
    "gg_batch_set_barrier_timeout": (ctypes.c_int, [_VP, ctypes.c_double, _I32]),
    "gg_batch_steps_per_pass": (_I32, [_VP]),
    "gg_batch_launch_info": (ctypes.c_int, [_VP, ctypes.POINTER(_I32)]),
    "gg_batch_set_plan": (ctypes.c_int, [_VP, _I32, _I32, _I32]),
    "gg_batch_last_error": (ctypes.c_char_p, [_VP]),
    "gg_batch_destroy": (ctypes.c_int, [_VP]),
    "gg_probe_fma_rate": (ctypes.c_int, [_I32, _I64, _I32, _VP, _DP]),
}


def lib():
    """Load libgg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2006_01748_gb300.build() "
                               "(nvcc, sm_103a); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


# ---------------------------------------------------------------- thin C mirrors

def gg_create(grid, params, theta, lambda1, lambda2, u0, v0, w0, stream=None):
    out = _VP()
    rc = lib().gg_create(ctypes.byref(grid), ctypes.byref(params), theta, lambda1, lambda2, u0, v0, w0,
                         stream, ctypes.byref(out))
    return rc, out


def gg_step(sim, nsteps):
    return lib().gg_step(sim, int(nsteps))


def gg_read(sim, field, dst, dst_on_device, dst_fp64):
    return lib().gg_read(sim, field, dst, dst_on_device, dst_fp64)


def gg_write(sim, field, src, src_on_device, src_fp64):
    return lib().gg_write(sim, field, src, src_on_device, src_fp64)


def gg_diagnostics(sim, eps=None):
    d = gg_diag()
    if eps is None:
        rc = lib().gg_diagnostics(sim, ctypes.byref(d))
    else:
        rc = lib().gg_diagnostics_eps(sim, float(eps), ctypes.byref(d))
    return rc, d


def gg_adjoint(sim, nsteps, dLdu, dLdv, dLdw, g_theta, g_l1, g_l2, g_u0, g_v0, g_w0, g_scalars, checkpoint_every=0):
    return lib().gg_adjoint(sim, int(nsteps), dLdu, dLdv, dLdw, g_theta, g_l1, g_l2, g_u0, g_v0, g_w0,
                            g_scalars, int(checkpoint_every))


def gg_front_rays(sim, i0, j0, v_front, u_edge, eps):
    f = gg_front()
    rc = lib().gg_front_rays(sim, int(i0), int(j0), float(v_front), float(u_edge), float(eps), ctypes.byref(f))
    return rc, f


def gg_front_speed(sim, i0, j0, nsteps, v_front, u_edge, eps):
    b, a = gg_front(), gg_front()
    sp = np.zeros(4)
    rc = lib().gg_front_speed(sim, int(i0), int(j0), int(nsteps), float(v_front), float(u_edge), float(eps),
                              ctypes.byref(b), ctypes.byref(a), sp.ctypes.data_as(_DP))
    return rc, b, a, sp


def front_dict(f: gg_front) -> Dict:
    return dict(front=np.array(f.front[:]), edge=np.array(f.edge[:]), gap=np.array(f.gap[:]),
                mass_v=np.array(f.mass_v[:]), mass_u=np.array(f.mass_u[:]))


def gg_adjoint_release(sim):
    return lib().gg_adjoint_release(sim)


def gg_dt(sim):
    return lib().gg_dt(sim)


def gg_dt_max(sim):
    return lib().gg_dt_max(sim)


def gg_step_count(sim):
    return lib().gg_step_count(sim)


def gg_steps_per_pass(sim):
    return lib().gg_steps_per_pass(sim)


def gg_last_error(sim=None):
    r = lib().gg_last_error(sim)
    return r.decode() if r else ""


def gg_error_string(status):
    return lib().gg_error_string(int(status)).decode()


def gg_destroy(sim):
    return lib().gg_destroy(sim)


def gg_probe_fma_rate(kind, iters, waves=4, stream=None):
    """Measured FMA rate (flop/s) of kind 0 FP64, 1 FP32, 2 packed FP32 pairs."""
    out = ctypes.c_double(0.0)
    rc = lib().gg_probe_fma_rate(int(kind), int(iters), int(waves), stream, ctypes.byref(out))
    return rc, out.value


# ---------------------------------------------------------------- helpers

def _f64_host(a, n) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def _check(rc, sim=None, what="libgg"):
    if rc != GG_OK:
        msg = gg_last_error(sim) or gg_error_string(rc)
        raise GGError(rc, f"{what}: {msg}")


def make_params(delta, rho, D, c, precision="fp32_kahan", dt=0.0, cfl=0.9, steps_per_pass=0,
                no_reaction=False, allow_unstable=False, adapt_every=0) -> gg_params:
    p = gg_params()
    p.delta, p.rho, p.D, p.c = float(delta), float(rho), float(D), float(c)
    p.cfl, p.dt = float(cfl), float(dt)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.flags = (GG_FLAG_NO_REACTION if no_reaction else 0) | (GG_FLAG_ALLOW_UNSTABLE if allow_unstable else 0)
    p.steps_per_pass = int(steps_per_pass)
    p.adapt_every = int(adapt_every)
    return p


def diag_dict(d: gg_diag) -> Dict:
    return dict(mass=np.array(d.mass[:]), min=np.array(d.min[:]), max=np.array(d.max[:]),
                nonfinite=int(d.nonfinite), tumour_area=d.tumour_area, gap_area=d.gap_area, gap_eps=d.gap_eps)


class GGSim:
    """One simulation of eq. (3) on the GPU (owns a gg_sim*)."""

    def __init__(self, nx, ny, theta, lambda1, lambda2, u0, v0, w0, delta, rho, D, c,
                 precision="fp32_kahan", dt=0.0, cfl=0.9, steps_per_pass=0, no_reaction=False,
                 allow_unstable=False, lx=1.0, ly=1.0, stream=None, adapt_every=0):
        self._sim = None
        n = int(nx) * int(ny)
        self.nx, self.ny = int(nx), int(ny)
        arrs = [_f64_host(a, n) for a in (theta, lambda1, lambda2, u0, v0, w0)]
        grid = gg_grid(self.nx, self.ny, float(lx), float(ly))
        self.params = make_params(delta, rho, D, c, precision, dt, cfl, steps_per_pass, no_reaction, allow_unstable,
                                  adapt_every)
        self.precision = self.params.precision
        self._stream = stream if stream is not None else _current_stream()
        rc, sim = gg_create(grid, self.params, *[a.ctypes.data_as(_VP) for a in arrs], stream=self._stream)
        _check(rc, None, "gg_create")
        self._sim = sim

    @classmethod
    def from_problem(cls, prob, precision="fp32_kahan", **kw):
        return cls(prob.nx, prob.ny, prob.theta, prob.lambda1, prob.lambda2, prob.u0, prob.v0, prob.w0,
                   prob.delta, prob.rho, prob.D, prob.c, precision=precision, cfl=prob.cfl,
                   lx=prob.lx, ly=prob.ly, **kw)

    @property
    def handle(self):
        return self._sim

    @property
    def dt(self) -> float:
        return gg_dt(self._sim)

    @property
    def dt_max(self) -> float:
        return gg_dt_max(self._sim)

    @property
    def steps(self) -> int:
        return gg_step_count(self._sim)

    @property
    def time(self) -> float:
        """Simulated time advanced since creation (sum of the steps taken)."""
        return lib().gg_time(self._sim)

    @property
    def steps_per_pass(self) -> int:
        return gg_steps_per_pass(self._sim)

    def step(self, nsteps: int):
        _check(gg_step(self._sim, nsteps), self._sim, "gg_step")

    def plan(self) -> Dict:
        info = (_I32 * 4)()
        _check(lib().gg_plan_info(self._sim, info), self._sim, "gg_plan_info")
        return dict(kind=PLAN_NAMES[info[0]], T=info[1], bx=info[2], by=info[3])

    def set_plan(self, kind: str = "warp", T: int = 1, strip: int = 0, chunk: int = 0):
        _check(lib().gg_set_plan(self._sim, PLAN_KINDS[kind], int(T), int(strip), int(chunk)),
               self._sim, "gg_set_plan")

    def autotune(self, trial_steps: int = 24) -> Dict:
        chosen = (_I32 * 4)()
        _check(lib().gg_autotune(self._sim, int(trial_steps), chosen), self._sim, "gg_autotune")
        return dict(T=chosen[0], kind=PLAN_NAMES[chosen[1]], bx=chosen[2], by=chosen[3])

    def read(self, field: str = "v", fp64: bool = True, out=None):
        """Copy a field; into a new host numpy array, into ``out`` when it is
        a C-contiguous host numpy array of nx*ny float32/float64 values (for
        instance one backed by pinned memory), or into ``out`` when it is a
        contiguous torch CUDA tensor of nx*ny float32/float64 values."""
        f = FIELDS[field]
        if out is None or isinstance(out, np.ndarray):
            a = out if out is not None else np.empty((self.ny, self.nx), dtype=np.float64 if fp64 else np.float32)
            assert a.flags.c_contiguous and a.size == self.nx * self.ny and a.dtype in (np.float32, np.float64)
            is64 = a.dtype == np.float64
            _check(gg_read(self._sim, f, a.ctypes.data_as(_VP), 0, 1 if is64 else 0), self._sim, "gg_read")
            return a
        import torch
        assert out.is_cuda and out.is_contiguous() and out.numel() == self.nx * self.ny
        is64 = out.dtype == torch.float64
        _check(gg_read(self._sim, f, ctypes.c_void_p(out.data_ptr()), 1, 1 if is64 else 0), self._sim, "gg_read")
        return out

    def write(self, field: str, src):
        f = FIELDS[field]
        try:
            import torch
            if isinstance(src, torch.Tensor) and src.is_cuda:
                assert src.is_contiguous() and src.numel() == self.nx * self.ny
                is64 = src.dtype == torch.float64
                _check(gg_write(self._sim, f, ctypes.c_void_p(src.data_ptr()), 1, 1 if is64 else 0),
                       self._sim, "gg_write")
                return
        except ImportError:
            pass
        a = np.ascontiguousarray(src)
        is64 = a.dtype == np.float64
        if not is64:
            a = a.astype(np.float32)
        _check(gg_write(self._sim, f, a.ctypes.data_as(_VP), 0, 1 if is64 else 0), self._sim, "gg_write")

    def diagnostics(self, eps: Optional[float] = None, check: bool = True) -> Dict:
        rc, d = gg_diagnostics(self._sim, eps)
        if check and rc not in (GG_OK, GG_ERR_NONFINITE):
            _check(rc, self._sim, "gg_diagnostics")
        out = diag_dict(d)
        out["status"] = rc
        return out

    def adjoint(self, nsteps: int, dLdu=None, dLdv=None, dLdw=None, checkpoint_every: int = 0,
                outputs=("theta", "lambda1", "lambda2", "u0", "v0", "w0")):
        """Discrete adjoint of ``nsteps`` steps from the current state.

        dLdu/dLdv/dLdw: contiguous float32 CUDA tensors of nx*ny values
        (dL/d(U,V,W) after the last step) or None.  Returns a dict of float32
        CUDA tensors of shape (ny, nx) for the requested outputs and
        ``scalars`` = dL/d(delta, rho, D, c) as a float64 numpy array.  The
        simulation is left at step ``nsteps``."""
        import torch
        n = self.nx * self.ny

        def ptr(t):
            if t is None:
                return None
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == n
            return ctypes.c_void_p(t.data_ptr())

        res = {name: torch.empty((self.ny, self.nx), dtype=torch.float32, device="cuda") for name in outputs}
        gs = np.zeros(4)
        rc = gg_adjoint(self._sim, nsteps, ptr(dLdu), ptr(dLdv), ptr(dLdw),
                        *(ptr(res.get(k)) for k in ("theta", "lambda1", "lambda2", "u0", "v0", "w0")),
                        gs.ctypes.data_as(_DP), checkpoint_every)
        _check(rc, self._sim, "gg_adjoint")
        res["scalars"] = gs
        return res

    def front_rays(self, i0: int, j0: int, v_front: float = 0.5, u_edge: float = 0.5, eps: float = 0.01) -> Dict:
        """Tumour front, healthy edge, gap width and ray integrals of V and U
        along the east, west, north and south rays from cell (i0, j0)."""
        rc, f = gg_front_rays(self._sim, i0, j0, v_front, u_edge, eps)
        _check(rc, self._sim, "gg_front_rays")
        return front_dict(f)

    def front_speed(self, i0: int, j0: int, nsteps: int, v_front: float = 0.5, u_edge: float = 0.5,
                    eps: float = 0.01):
        """Advance nsteps and return (before, after, speed[4]) with the
        LeVeque-Yee space-averaged front speed along each ray."""
        rc, b, a, sp = gg_front_speed(self._sim, i0, j0, nsteps, v_front, u_edge, eps)
        _check(rc, self._sim, "gg_front_speed")
        return front_dict(b), front_dict(a), sp

    def release_adjoint(self):
        """Free the adjoint workspace (checkpoints, stash and kept states)."""
        _check(gg_adjoint_release(self._sim), self._sim, "gg_adjoint_release")

    def state(self, fp64: bool = True):
        return tuple(self.read(f, fp64) for f in ("u", "v", "w"))

    def close(self):
        if self._sim is not None:
            gg_destroy(self._sim)
            self._sim = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class GGBatch:
    """An ensemble of independent simulations advanced by one persistent,
    graph-captured launch (owns a gg_batch*)."""

    def __init__(self, problems: Sequence, precision="fp32_kahan", steps_per_pass=0, stream=None):
        n = len(problems)
        self.problems = list(problems)
        grids = (gg_grid * n)()
        params = (gg_params * n)()
        keep = []
        ptrs = (_VP * (6 * n))()
        for k, p in enumerate(problems):
            grids[k] = gg_grid(p.nx, p.ny, p.lx, p.ly)
            params[k] = make_params(p.delta, p.rho, p.D, p.c, precision, cfl=p.cfl, steps_per_pass=steps_per_pass)
            for m, a in enumerate((p.theta, p.lambda1, p.lambda2, p.u0, p.v0, p.w0)):
                arr = _f64_host(a, p.nx * p.ny)
                keep.append(arr)
                ptrs[6 * k + m] = arr.ctypes.data_as(_VP)
        self._stream = stream if stream is not None else _current_stream()
        out = _VP()
        rc = lib().gg_batch_create(n, grids, params, ptrs, self._stream, ctypes.byref(out))
        if rc != GG_OK:
            raise GGError(rc, "gg_batch_create failed")
        self._b = out
        self.n = n

    @property
    def handle(self):
        return self._b

    @property
    def steps_per_pass(self) -> int:
        return lib().gg_batch_steps_per_pass(self._b)

    def _check(self, rc, what):
        if rc != GG_OK:
            msg = lib().gg_batch_last_error(self._b)
            raise GGError(rc, f"{what}: {msg.decode() if msg else gg_error_string(rc)}")

    def autotune(self, trial_steps: int = 8):
        chosen = (_I32 * 4)()
        self._check(lib().gg_batch_autotune(self._b, int(trial_steps), chosen), "gg_batch_autotune")
        return dict(T=chosen[0], bx=chosen[1], by=chosen[2], threads=chosen[3], mode=self.launch_info()["mode"])

    def step(self, nsteps: int):
        self._check(lib().gg_batch_step(self._b, int(nsteps)), "gg_batch_step")

    def dt(self, inst: int) -> float:
        return lib().gg_batch_dt(self._b, inst)

    def launch_info(self) -> Dict:
        info = (_I32 * 8)()
        self._check(lib().gg_batch_launch_info(self._b, info), "gg_batch_launch_info")
        return dict(T=info[0], bx=info[1], by=info[2], threads=info[3], ctas=info[4], tiles=info[5],
                    graph=bool(info[6]), mode=BATCH_MODES[info[7]])

    def set_plan(self, mode: str = "persistent", T: int = 1, chunk: int = 0):
        """mode "persistent" (cooperative kernel, grid barrier between passes),
        "passes" (one launch of one warp per one-column tile per pass) or
        "passes2" (the same with the paired-column tiles)."""
        self._check(lib().gg_batch_set_plan(self._b, BATCH_MODES.index(mode), int(T), int(chunk)),
                    "gg_batch_set_plan")

    def read(self, inst: int, field: str = "v", fp64: bool = True):
        p = self.problems[inst]
        a = np.empty((p.ny, p.nx), dtype=np.float64 if fp64 else np.float32)
        self._check(lib().gg_batch_read(self._b, inst, FIELDS[field], a.ctypes.data_as(_VP), 0, 1 if fp64 else 0),
                    "gg_batch_read")
        return a

    def read_status(self, inst: int, field: str = "v"):
        p = self.problems[inst]
        a = np.empty((p.ny, p.nx), dtype=np.float64)
        return lib().gg_batch_read(self._b, inst, FIELDS[field], a.ctypes.data_as(_VP), 0, 1)

    def diagnostics(self, inst: int) -> Dict:
        d = gg_diag()
        rc = lib().gg_batch_diagnostics(self._b, inst, ctypes.byref(d))
        if rc not in (GG_OK, GG_ERR_NONFINITE):
            self._check(rc, "gg_batch_diagnostics")
        out = diag_dict(d)
        out["status"] = rc
        return out

    def set_barrier_timeout(self, seconds: float, extra_arrivals: int = 0):
        self._check(lib().gg_batch_set_barrier_timeout(self._b, float(seconds), int(extra_arrivals)),
                    "gg_batch_set_barrier_timeout")

    def close(self):
        if getattr(self, "_b", None) is not None:
            lib().gg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
