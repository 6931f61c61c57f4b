"""torch.autograd.Function over the library's discrete adjoint.

`ensemble_objective(params, ...)` runs an ensemble from its 24 parameters per sample
for `nsteps` steps and returns J [M] (kinetic energy or enstrophy per sample at the
final step); backward multiplies the incoming gradient by dJ/dX computed by the
hand-written adjoint kernels (mclbm_grad).  Forward and reverse run on the GPU; the
parameters live on the host (they enter the library as host arrays).
"""
import numpy as np
import torch

from . import mclbm as _m
from .ensemble import Ensemble

OBJECTIVES = {"energy": 0, "enstrophy": 1}


class _EnsembleObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, cfg):
        X = params.detach().to("cpu", torch.float64).contiguous().numpy()
        M = X.shape[0]
        ens = Ensemble(cfg["N"], M, Re=cfg.get("Re"), nu=cfg.get("nu"), Ma=cfg["Ma"], precision=cfg["precision"],
                       pattern="pull", device=cfg.get("device"), stream=cfg.get("stream")).init(X)
        need = _m.mclbm_grad_required_bytes(ens.ctx, cfg["nsteps"], cfg["ckpt_every"])
        buf = torch.empty(need + 256, dtype=torch.uint8, device=ens.device)
        ens._enter(buf)
        ptr = (buf.data_ptr() + 255) // 256 * 256
        J, G = _m.mclbm_grad(ens.ctx, OBJECTIVES[cfg["objective"]], cfg["nsteps"], cfg["ckpt_every"], ptr, need, M)
        ctx.save_for_backward(torch.from_numpy(G))
        return torch.from_numpy(J).to(params.dtype)

    @staticmethod
    def backward(ctx, grad_J):
        (G,) = ctx.saved_tensors
        return (grad_J.to(torch.float64)[:, None] * G).to(grad_J.dtype), None


def ensemble_objective(params, N, Ma, nsteps, Re=None, nu=None, objective="energy", precision="fp32", ckpt_every=50,
                       device=None, stream=None):
    """J [M] of the ensemble started from `params` [M][24] (CPU tensor); differentiable in params."""
    cfg = dict(N=N, Ma=Ma, Re=Re, nu=nu, nsteps=int(nsteps), objective=objective, precision=precision,
               ckpt_every=int(ckpt_every), device=device, stream=stream)
    return _EnsembleObjective.apply(params, cfg)
