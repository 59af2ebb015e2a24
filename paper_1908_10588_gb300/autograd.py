"""torch.autograd bridge of the differentiable 2TDVP form.

`population(g, ...)` returns the population P_k(t) of one electronic state
after a 2TDVP propagation from the product state, as a differentiable
function of a tensor g of linear vibronic couplings g^I_ij (Eq. Helvib_2).
Forward and gradient both run in the library (tdvp2_population_gradient: the
forward sweeps, the costate sweeps backwards in time and the coupling
contractions on the GPU); this module only writes the coupling values into
the model, builds the MPO and hands the gradient to autograd.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import binding as B


def _model_with(model: dict, params, values) -> dict:
    m = copy.deepcopy(model)
    g1 = np.array(m["g1"], dtype=float)
    for (I, i, j), v in zip(params, values):
        g1[I, i, j] = float(v)
        g1[I, j, i] = float(v)
    m["g1"] = g1
    return m


class PopulationFunction(torch.autograd.Function):
    """P_k(t)(g): forward and dP_k/dg in one library call; backward scales
    the stored gradient by the incoming one."""

    @staticmethod
    def forward(ctx, g, model, params, init_index, el_state, dt_fs, n_steps, m_max, dtype, eps, zero_floor,
                checkpoint_every, pad_full):
        vals = g.detach().cpu().numpy().astype(np.float64)
        mpo = B.Mpo(_model_with(model, params, vals))
        mps = B.Mps(mpo, init_index, m_cap=m_max, dtype=dtype, pad_full=pad_full)
        pops, grad = mps.population_gradient(dt_fs, n_steps, params, el_state, m_max, eps=eps,
                                             zero_floor=zero_floor, checkpoint_every=checkpoint_every)
        mps.close()
        mpo.close()
        ctx.save_for_backward(torch.as_tensor(grad, dtype=g.dtype, device=g.device))
        return torch.as_tensor(pops[el_state], dtype=g.dtype, device=g.device)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return (gout * grad,) + (None,) * 12


def population(g, model: dict, params, el_state: int, dt_fs: float, n_steps: int, m_max: int,
               init_index=None, dtype: int = B.VB_FP64, eps: float = 0.0, zero_floor: float = 1e-14,
               checkpoint_every: int = 10, pad_full: bool = False):
    """Differentiable P_el_state(n_steps * dt) for coupling values g (1-D
    tensor, one per parameter (mode, i, j) in params)."""
    if init_index is None:
        raise ValueError("init_index: the product state's basis index on every site")
    return PopulationFunction.apply(g, model, list(params), list(init_index), int(el_state), float(dt_fs),
                                    int(n_steps), int(m_max), int(dtype), float(eps), float(zero_floor),
                                    int(checkpoint_every), bool(pad_full))
