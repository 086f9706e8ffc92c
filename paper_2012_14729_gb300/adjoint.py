"""Differentiable run of the phase-field LBM (adjoint pattern).

``PFLBMRun.apply(phi0, sigma, M, spec)`` advances ``spec.nsteps`` steps from
phi0 with surface tension sigma and mobility M and returns phi_T.  Its backward
calls the hand-written discrete adjoint of the CUDA library
(``pflbm_adjoint_run``): the forward is recomputed from checkpoints taken every
``spec.ckpt_every`` steps and the adjoint runs backwards through each segment,
giving dJ/dphi0, dJ/dsigma and dJ/dM for any objective J of phi_T.  PyTorch
provides memory, streams and the objective's own gradient; every step of the
method and of its adjoint runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import pflbm


@dataclass
class RunSpec:
    nx: int
    ny: int
    wall_y: bool
    nsteps: int
    ckpt_every: int = 200
    params: dict = field(default_factory=dict)  # every parameter except sigma and M


def _domain(spec: RunSpec, sigma: float, M: float, stream):
    d = pflbm.Domain(spec.nx, spec.ny, wall_y=spec.wall_y, stream=stream)
    d.set_params(**{**spec.params, "sigma": float(sigma), "M": float(M)})
    return d


class PFLBMRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, sigma, M, spec: RunSpec):
        stream = torch.cuda.current_stream()
        phi0 = phi0.detach().to(torch.float32).contiguous()
        d = _domain(spec, sigma.item(), M.item(), stream)
        pflbm.pflbm_init_phi(d.h, phi0)
        pflbm.pflbm_step(d.h, spec.nsteps)
        out = torch.empty((len(pflbm.FIELDS), spec.ny, spec.nx), dtype=torch.float32,
                          device=phi0.device)
        pflbm.pflbm_read_fields(d.h, out)
        ctx.save_for_backward(phi0, sigma, M)
        ctx.spec = spec
        return out[0].clone()

    @staticmethod
    def backward(ctx, g_phiT):
        phi0, sigma, M = ctx.saved_tensors
        spec = ctx.spec
        stream = torch.cuda.current_stream()
        d = _domain(spec, sigma.item(), M.item(), stream)
        nbytes = pflbm.pflbm_adjoint_scratch_bytes(d.h, spec.nsteps, spec.ckpt_every)
        scratch = torch.empty(nbytes, dtype=torch.uint8, device=phi0.device)
        dphi0 = torch.empty_like(phi0)
        ds, dm = pflbm.pflbm_adjoint_run(d.h, phi0, spec.nsteps, spec.ckpt_every,
                                         g_phiT.to(torch.float32).contiguous(), dphi0, scratch)
        return (dphi0, torch.tensor(ds, dtype=sigma.dtype, device=sigma.device),
                torch.tensor(dm, dtype=M.dtype, device=M.device), None)


def run(phi0, sigma, M, spec: RunSpec):
    """phi_T as a differentiable function of (phi0, sigma, M)."""
    return PFLBMRun.apply(phi0, sigma, M, spec)
