"""torch.autograd.Function around the forward step and its discrete adjoint.

``GGStepFn.apply(theta, lambda1, lambda2, scalars, u0, v0, w0, nsteps, dt,
precision)`` advances eq. (3) nsteps steps on the GPU and returns the final
(U, V, W) as float32 CUDA tensors of shape (ny, nx).  Its backward runs
gg_adjoint (sqrt(N) checkpointing) and returns gradients for theta, lambda1,
lambda2 (per cell), scalars = (delta, rho, D, c) and the initial fields.
dt is held fixed: pass it explicitly, or it is taken from the step rule of
the forward inputs and not differentiated.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gg


def _host64(t: torch.Tensor) -> np.ndarray:
    return np.ascontiguousarray(t.detach().to("cpu", torch.float64).numpy())


class GGStepFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, lambda1, lambda2, scalars, u0, v0, w0, nsteps: int, dt: float = 0.0,
                precision: str = "fp32_kahan", checkpoint_every: int = 0):
        ny, nx = theta.shape
        sc = _host64(scalars)
        host = [_host64(x) for x in (theta, lambda1, lambda2, u0, v0, w0)]
        sim = gg.GGSim(nx, ny, *host, *sc, precision=precision, dt=dt)
        dt_used = sim.dt
        sim.step(nsteps)
        outs = [sim.read(f, out=torch.empty(nx * ny, dtype=torch.float32, device="cuda")).view(ny, nx)
                for f in "uvw"]
        sim.close()
        ctx.host = host
        ctx.sc = sc
        ctx.meta = (nx, ny, int(nsteps), dt_used, precision, int(checkpoint_every))
        ctx.like = [(x.dtype, x.device) for x in (theta, lambda1, lambda2, scalars, u0, v0, w0)]
        return tuple(outs)

    @staticmethod
    def backward(ctx, gu, gv, gw):
        nx, ny, nsteps, dt, precision, ck = ctx.meta
        sim = gg.GGSim(nx, ny, *ctx.host, *ctx.sc, precision=precision, dt=dt)

        def prep(g):
            return None if g is None else g.detach().to("cuda", torch.float32).contiguous().view(-1)

        r = sim.adjoint(nsteps, prep(gu), prep(gv), prep(gw), checkpoint_every=ck)
        sim.close()
        grads = [r["theta"], r["lambda1"], r["lambda2"], torch.from_numpy(r["scalars"]), r["u0"], r["v0"], r["w0"]]
        out = [g.to(dtype=dt_, device=dev) for g, (dt_, dev) in zip(grads, ctx.like)]
        return (*out, None, None, None, None)
