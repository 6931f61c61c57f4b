"""torch.autograd.Function over the library's discrete adjoint.

`ensemble_objective(params, ...)` runs an ensemble from its 24 parameters per sample
for `nsteps` steps and returns J [M] (kinetic energy or enstrophy per sample at the
final step).  The forward pass is a plain stepped run (the stepper and the energy
reduction, nothing else), so evaluating J costs one forward run whether or not a
backward pass follows.  Backward re-runs the ensemble from the saved parameters
through mclbm_grad (forward with checkpoints, segment recomputation, the hand-written
adjoint kernels, parameter reduction) and multiplies the incoming gradient by dJ/dX.
Both use the same stepper launches, so J of the two runs is the same to the bit.  The
parameters live on the host (they enter the library as host arrays).
"""
import torch
from torch.autograd.function import once_differentiable

from . import mclbm as _m
from .ensemble import Ensemble

OBJECTIVES = {"energy": 0, "enstrophy": 1}


def _ensemble(cfg, X):
    return Ensemble(cfg["N"], X.shape[0], Re=cfg.get("Re"), nu=cfg.get("nu"), Ma=cfg["Ma"],
                    precision=cfg["precision"], pattern="pull", device=cfg.get("device"),
                    stream=cfg.get("stream")).init(X)


def objective_values(cfg, X):
    """J [M] of a plain stepped run from parameters X [M][24] (numpy FP64)."""
    ens = _ensemble(cfg, X).step(cfg["nsteps"])
    if cfg["objective"] == "enstrophy":
        return ens.energy(enstrophy=True)[1]
    return ens.energy()


def objective_and_gradient(cfg, X):
    """(J [M], dJ/dX [M][24]) through the adjoint (mclbm_grad)."""
    ens = _ensemble(cfg, X)
    need = _m.mclbm_grad_required_bytes(ens.ctx, cfg["nsteps"], cfg["ckpt_every"])
    buf = torch.empty(need + 256, dtype=torch.uint8, device=ens.device)
    ens._enter(buf)
    ptr = (buf.data_ptr() + 255) // 256 * 256
    return _m.mclbm_grad(ens.ctx, OBJECTIVES[cfg["objective"]], cfg["nsteps"], cfg["ckpt_every"], ptr, need,
                         X.shape[0])


class _EnsembleObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, cfg):
        X = params.detach().to("cpu", torch.float64).contiguous().numpy()
        ctx.cfg = cfg
        ctx.save_for_backward(params)
        return torch.from_numpy(objective_values(cfg, X)).to(params.dtype)

    @staticmethod
    @once_differentiable
    def backward(ctx, grad_J):
        (params,) = ctx.saved_tensors
        X = params.detach().to("cpu", torch.float64).contiguous().numpy()
        _, G = objective_and_gradient(ctx.cfg, X)
        G = torch.from_numpy(G)
        return (grad_J.to("cpu", torch.float64)[:, None] * G).to(grad_J.dtype), None


def ensemble_objective(params, N, Ma, nsteps, Re=None, nu=None, objective="energy", precision="fp32", ckpt_every=50,
                       device=None, stream=None):
    """J [M] of the ensemble started from `params` [M][24] (CPU tensor); differentiable in params.
    The gradient is computed only when a backward pass asks for it."""
    if objective not in OBJECTIVES:
        raise ValueError(f"objective must be one of {sorted(OBJECTIVES)}")
    cfg = dict(N=N, Ma=Ma, Re=Re, nu=nu, nsteps=int(nsteps), objective=objective, precision=precision,
               ckpt_every=int(ckpt_every), device=device, stream=stream)
    return _EnsembleObjective.apply(params, cfg)
