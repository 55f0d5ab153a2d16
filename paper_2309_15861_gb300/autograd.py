"""torch.autograd bridge for the atmosphere parameters.

theta = (c_1 .. c_L, K, L0): the layer scale heights (m), the refractivity
coefficient (cm^3/g) and the extinction length (m); the layer b_i, the
layer edges, the random numbers and the bunch counts stay fixed.  The
forward runs the CUDA path at theta and returns the hits' arrival x_rel,
y_rel, t and the soft-edged per-telescope yields; the backward calls the
tangent-linear adjoint kernels (clight_trace_adjoint) with the upstream
gradients.  All arithmetic happens in the library's kernels.
"""
from __future__ import annotations

import copy
import dataclasses

import numpy as np
import torch

from . import ClightError, Context, ERR_HIT_CAPACITY, HIT_DTYPE, OK
from . import inputs as I


@dataclasses.dataclass
class Engine:
    """Everything the function needs besides theta."""
    ctx: Context
    workload: I.Workload
    d_segs: torch.Tensor
    soft_s: float = 0.5
    soft_w: float = 20.0
    capacity: int = 1 << 20
    hits: torch.Tensor = None        # filled by the forward


def atmosphere_at(base: I.Atmosphere, theta) -> I.Atmosphere:
    a = copy.deepcopy(base)
    L = a.n_layers
    th = [float(v) for v in theta]
    a.c = th[:L]
    a.K = th[L]
    a.L0 = th[L + 1]
    return a


def theta_of(atm: I.Atmosphere) -> torch.Tensor:
    return torch.tensor(list(atm.c) + [atm.K, atm.L0], dtype=torch.float64)


class AtmosphereResponse(torch.autograd.Function):
    """(x_rel, y_rel, t of every hit; soft yield of every (shower, telescope)) as a function of theta."""

    @staticmethod
    def forward(fctx, theta, eng: Engine):
        w = eng.workload
        eng.ctx.set_atmosphere(atmosphere_at(w.atmosphere, theta.detach().cpu().numpy()))
        eng.ctx.set_params(w.params)
        n = len(w.segments)
        dev = eng.d_segs.device
        while True:
            hits = torch.empty(eng.capacity * 48, dtype=torch.uint8, device=dev)
            code, nh, st = eng.ctx.trace(eng.d_segs, n, w.n_showers, hits, eng.capacity, raise_on_error=False)
            if code == ERR_HIT_CAPACITY:
                eng.capacity = nh + 1024
                continue
            if code != OK:
                raise ClightError(code, "AtmosphereResponse.forward")
            break
        hits = hits[: nh * 48]
        eng.hits = hits
        rec = hits.view(-1, 48)
        f32 = rec.view(torch.float32).view(-1, 12) if nh else torch.empty(0, 12, dtype=torch.float32, device=dev)
        x = f32[:, 4].clone()
        y = f32[:, 5].clone()
        t = rec.view(torch.float64).view(-1, 6)[:, 5].clone() if nh else torch.empty(0, dtype=torch.float64, device=dev)
        ng = w.n_showers * len(w.telescopes)
        Y = torch.zeros(ng, dtype=torch.float64, device=dev)
        eng.ctx.trace_adjoint(eng.d_segs, n, w.n_showers, hits, nh, soft_s=eng.soft_s, soft_w=eng.soft_w, d_yield=Y)
        fctx.eng = eng
        fctx.theta = theta.detach().clone()
        fctx.nh = nh
        return x, y, t, Y

    @staticmethod
    def backward(fctx, gx, gy, gt, gY):
        eng = fctx.eng
        w = eng.workload
        eng.ctx.set_atmosphere(atmosphere_at(w.atmosphere, fctx.theta.numpy()))
        dev = eng.d_segs.device
        f = lambda g: None if g is None else g.detach().to(device=dev, dtype=torch.float32).contiguous()
        gY_ = None if gY is None else gY.detach().to(device=dev, dtype=torch.float64).contiguous()
        grad = eng.ctx.trace_adjoint(eng.d_segs, len(w.segments), w.n_showers, eng.hits, fctx.nh,
                                     gx=f(gx), gy=f(gy), gt=f(gt), gY=gY_, soft_s=eng.soft_s, soft_w=eng.soft_w)
        L = w.atmosphere.n_layers
        return torch.tensor(grad[: L + 2], dtype=torch.float64), None


def hits_to_numpy(hits: torch.Tensor) -> np.ndarray:
    return hits.cpu().numpy().view(HIT_DTYPE).copy()
