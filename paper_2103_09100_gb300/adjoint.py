"""Receiver misfit as a differentiable function of the cell moduli.

``misfit(E, solver, n_steps, rec_dof, data)`` returns
J(E) = 1/2 sum_{n=1..N} sum_r (U_n[rec_r] - data[n-1, r])^2 for the
undamped explicit solver started from rest, as a torch scalar whose
gradient with respect to E (one modulus per cell) comes from the GPU
discrete adjoint (``sbx_adjoint``): the forward run keeps a checkpoint every
``ckpt_every`` steps and the reverse sweep recomputes each segment.  The
forward call already computes dJ/dE; ``backward`` only scales it.
"""
from __future__ import annotations

import numpy as np
import torch


class ModulusMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E, solver, n_steps, rec_dof, data, ckpt_every):
        solver.set_modulus(E.detach().to(torch.float64).cpu().numpy())
        solver.initial()
        J, grad = solver.adjoint(n_steps, rec_dof, data, ckpt_every)
        ctx.save_for_backward(torch.from_numpy(grad).to(E.dtype))
        return E.new_tensor(J)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return gJ * grad.to(gJ.device), None, None, None, None, None


def misfit(E, solver, n_steps, rec_dof, data, ckpt_every=64):
    return ModulusMisfit.apply(E, solver, int(n_steps), np.asarray(rec_dof, np.int64),
                               np.asarray(data, np.float64), int(ckpt_every))
