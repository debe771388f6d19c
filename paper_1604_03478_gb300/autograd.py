"""torch.autograd.Function around the recorded run and its adjoint.

``melt_front(dTh, Ra, ...)`` runs a cavity for `steps` steps with the
heated-wall temperature Th + dTh (one value per column) and returns the final
front S as a torch tensor; ``backward`` calls the library's hand-written
adjoint (lbm_melt_tape_backward) with dL/dS and returns dL/d(dTh) and dL/dRa.
All arithmetic runs in the CUDA library; this is argument marshalling.
"""
from __future__ import annotations

import numpy as np
import torch

from .cavity import Cavity


class MeltFront(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dTh, Ra, spec, steps, ckpt_every):
        spec = dict(spec)
        n = (spec.pop("nx"), spec.pop("ny"), spec.pop("nz"))
        Th = spec.get("Th", 1.0)
        cav = Cavity(*n, Ra=float(Ra), derive=True, **spec)
        cav.set_hot_wall((Th + dTh.detach().to("cpu", torch.float64).numpy()).astype(np.float32))
        cav.tape_forward(int(steps), int(ckpt_every))
        S = cav.get(T=False, u=False, lf=False)[2]
        ctx.cav = cav
        ctx.device = dTh.device
        ctx.shape = dTh.shape
        return torch.as_tensor(S, dtype=torch.float64, device=dTh.device)

    @staticmethod
    def backward(ctx, gS):
        cav = ctx.cav
        dth, par = cav.tape_backward(gS.detach().to("cpu", torch.float64).numpy())
        cav.close()
        ctx.cav = None
        g_th = torch.as_tensor(dth, dtype=torch.float64, device=ctx.device).reshape(ctx.shape)
        g_ra = torch.tensor(par["Ra"], dtype=torch.float64, device=ctx.device)
        return g_th, g_ra, None, None, None


def melt_front(dTh, Ra, spec, steps, ckpt_every=0):
    """Final front S(x, z) of a run with wall temperature Th + dTh; spec
    holds the other Cavity arguments (nx, ny, nz, face, Pr, Ste, Ma, s0, ...)."""
    return MeltFront.apply(dTh, Ra, spec, steps, ckpt_every)
