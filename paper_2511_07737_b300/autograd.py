"""``SatObjective``: the binarised R = P A layer of Fig. 3 as a torch.autograd.Function.

forward(z) evaluates, in the library's kernels, the per-variable normaliser
(Eq. 5), the binarisation (Eq. 2; deterministic or Philox at step ``t_bin``),
R = P A (Eq. 1), SmoothMin (Eq. 4) and L = -sum_i S_i (Eq. 3) for every
instance of the problem.  backward applies the hand-written adjoint: the
straight-through estimator (or the exact sigmoid chain rule of the relaxed
layer) followed by the chain rule through Eq. 5.  The returned loss is the sum
of the instances' losses; S is returned as a non-differentiable output.

The state passed in serves as workspace (bits, normaliser, histograms, gamma
tables); its optimiser moments are not touched.
"""
from __future__ import annotations

import torch

from . import turbosat as ts


class SatObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z: torch.Tensor, state: "ts.State", hp: "ts.tsat_hparams", t_bin: int = 0):
        if not z.is_cuda or z.dtype != torch.float32 or not z.is_contiguous():
            raise ValueError("z must be a contiguous float32 CUDA tensor of shape (n_vars, n_samples)")
        n_inst = state.prob.info["n_inst"]
        if tuple(z.shape) != (state.prob.info["n_vars"], state.N):
            raise ValueError(f"z has shape {tuple(z.shape)}, expected {(state.prob.info['n_vars'], state.N)}")
        S = torch.empty(n_inst * state.N, device=z.device, dtype=torch.float32)
        L = torch.empty(n_inst, device=z.device, dtype=torch.float32)
        ts.tsat_forward(state.h, hp, z, int(t_bin), S, L)
        ctx.save_for_backward(z)
        ctx.state = state
        ctx.hp = hp
        ctx.mark_non_differentiable(S)
        return L.sum(), S

    @staticmethod
    def backward(ctx, dL, dS):
        (z,) = ctx.saved_tensors
        grad = torch.empty_like(z)
        ts.tsat_backward(ctx.state.h, ctx.hp, z, 1.0, grad)
        return grad.mul_(dL), None, None, None


def sat_objective(z: torch.Tensor, state: "ts.State", hp: "ts.tsat_hparams", t_bin: int = 0):
    """Functional form: returns (loss, S)."""
    return SatObjective.apply(z, state, hp, t_bin)
