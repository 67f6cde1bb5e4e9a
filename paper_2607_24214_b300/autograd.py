"""The QS-PIC run as a differentiable function of its seed: a torch.autograd.Function whose
forward and backward run on the GPU through the C ABI (qsa_grad_forward, qsa_grad_backward).

    loss = QSAFunction.apply(amplitudes, alphas, params, n_steps, step_ckpt)

amplitudes: the seeded transverse modes' amplitudes a_m (one per params.modes entry);
alphas: each beam species' density ratio alpha_s.  loss is 1/2 sum (B_x^2 + B_y^2) dx dy dxi
over the slices and cells of the final sweep after n_steps beam steps: the transverse
magnetic (filamentation) energy whose growth the paper's linear theory (Eqs. 3-5) ties to
alpha and to the seed.  The backward pass is the discrete adjoint of the FP64 scheme (beam
checkpoints every step_ckpt steps, each segment recomputed and recorded slice by slice), so
the gradient is that of the forward value to rounding.  Argument marshalling only.
"""
from __future__ import annotations

import torch

from . import config
from .qsa import QSA


def with_seed(p: config.Params, amplitudes, alphas) -> config.Params:
    """params with the modes' amplitudes and the species' alpha replaced, on the FP64 path."""
    import copy
    q = copy.deepcopy(p)
    for m, a in zip(q.modes, amplitudes):
        m.amplitude = float(a)
    for s, a in zip(q.species, alphas):
        s.alpha = float(a)
    return q.with_(precision="fp64")


class QSAFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, amplitudes, alphas, p, n_steps, step_ckpt=10):
        q = QSA(with_seed(p, amplitudes.detach().cpu().tolist(), alphas.detach().cpu().tolist()))
        loss = q.grad_forward(n_steps, step_ckpt)
        ctx.q = q
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        q = ctx.q
        dm, da = q.grad_backward(float(g))
        q.close()
        ctx.q = None
        return (torch.as_tensor(dm, dtype=torch.float64), torch.as_tensor(da, dtype=torch.float64),
                None, None, None)
