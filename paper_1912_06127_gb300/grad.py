"""d<O_j(t)>/d(h, J) of a TDVP quench behind torch.autograd.Function.

The library advances, with every local operation of the sweep, the tangent of
the state along d/dh and d/dJ (forward-mode differentiation, in FP64;
tdvp_step_tangent in include/tdvp.h). With two parameters the forward mode
costs two tangent sweeps, keeps no per-step state and needs no checkpoints: the
whole Jacobian d<O_j(t)>/d(h, J) is known when the forward pass ends, and the
backward pass only contracts it with the incoming gradient.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

from . import tdvp


@dataclasses.dataclass
class Quench:
    """A quench from a fixed initial state: model, initial state and sweep settings."""
    kind: int
    N: int
    alpha: float
    n_exp: int
    dt: float
    n_steps: int
    chi_max: int
    eps: float = 1e-12
    krylov_max: int = 16
    krylov_tol: float = 1e-12
    seg_len: Optional[Sequence[int]] = None
    basis_state: Optional[Sequence[int]] = None      # product initial state, or
    tensors: Optional[Sequence[np.ndarray]] = None   # raw site tensors (brought to canonical form)
    obs: int = tdvp.OBS_SZ
    n_quad: int = 6
    x: Optional[np.ndarray] = None                   # fitted exponentials (fitted here if None)
    lam: Optional[np.ndarray] = None

    def run(self, h: float, J: float):
        """(<O_j(t)> [N], d<O_j(t)>/d(h, J) [N, 2])."""
        if self.x is None or self.lam is None:
            self.x, self.lam = tdvp.fit_power_law(self.alpha, self.n_exp, self.N - 1)
        mpo = tdvp.build_mpo(self.kind, self.N, self.alpha, J, h, self.n_exp, self.x, self.lam)
        dmpos = [tdvp.build_mpo_derivative(mpo, tdvp.PARAM_H), tdvp.build_mpo_derivative(mpo, tdvp.PARAM_J)]
        if self.tensors is not None:
            mps = tdvp.init_mps_tensors(self.tensors, self.chi_max, 1e-14)
        else:
            mps = tdvp.init_mps(self.N, self.basis_state, self.chi_max)
        tan = tdvp.Tangent(mps, 2)
        p = tdvp.step_params(self.dt, self.chi_max, eps=self.eps, krylov_max=self.krylov_max,
                             krylov_tol=self.krylov_tol, seg_len=self.seg_len)
        tdvp.step_tangent(mps, mpo, tan, dmpos, p, self.n_steps, n_quad=self.n_quad)
        val, der = tdvp.measure_tangent(mps, tan, self.obs)
        return val, der.T.copy()


def _autograd_function():
    import torch

    class QuenchObservable(torch.autograd.Function):
        """<O_j(t)> of a Quench as a differentiable function of the scalars h and J."""

        @staticmethod
        def forward(ctx, h, J, quench: Quench):
            val, jac = quench.run(float(h), float(J))
            ctx.save_for_backward(torch.as_tensor(jac, dtype=torch.float64))
            return torch.as_tensor(val, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            (jac,) = ctx.saved_tensors
            g = g.to(torch.float64).cpu()
            return (g * jac[:, 0]).sum(), (g * jac[:, 1]).sum(), None

    return QuenchObservable


def observable(h, J, quench: Quench):
    """<O_j(t)> (torch float64 tensor [N]); differentiable in h and J (0-dim tensors)."""
    return _autograd_function().apply(h, J, quench)
