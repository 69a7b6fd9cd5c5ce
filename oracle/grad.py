"""Derivative of the TDVP time evolution with respect to the model parameters (oracle).

Test infrastructure (see oracle/__init__.py): never imported by the product path.

The paper evolves in time only; d<O_j(t)>/d(h, J) is the derivative of the
discrete algorithm of oracle.tdvp (the symmetric sweep of Sec. III A/B with the
truncated split of Fig. 5) as a function of the transverse field h and the
coupling J. This module restates that algorithm with plain PyTorch FP64 CPU
operations and lets torch's forward-mode automatic differentiation carry the
tangents (torch.autograd.forward_ad):

  * W(J, h) = W(0, 0) + J dW/dJ + h dW/dh: the MPO tensor of Sec. II C is
    affine in J (which multiplies every x_k) and in h (the field block);
  * H2_eff and H1_eff (Fig. 4) are formed as explicit matrices (small sizes
    only) and exponentiated with torch.linalg.matrix_exp: the exact local
    exponential that a converged Lanczos run approximates (Eq. 18, Eq. 20);
  * the split (Fig. 5) is torch.linalg.svd with the kept rank taken from
    oracle.tdvp.truncation_rank on the current singular values, so the
    derivative is the one at fixed truncation;
  * observables from the explicit 2^N state vector.

Nothing here is blocked, fused or reordered: the ops run in the order of
oracle.tdvp.build_schedule, one at a time.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch
import torch.autograd.forward_ad as fwAD

from .models import SX, SY, SZ, build_mpo_site, mpo_boundaries
from .mps import MPS
from .tdvp import Params, build_schedule, execution_order, truncation_rank

C128 = torch.complex128


def _t(a: np.ndarray) -> torch.Tensor:
    return torch.as_tensor(np.asarray(a), dtype=C128)


def _primal(x: torch.Tensor) -> torch.Tensor:
    return fwAD.unpack_dual(x).primal


def mpo_affine(kind: int, x: np.ndarray, lam: np.ndarray) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """(W(0,0), dW/dJ, dW/dh) of the MPO tensor of Sec. II C (exact: W is affine in J and h)."""
    W00 = build_mpo_site(kind, 0.0, 0.0, x, lam)
    WJ = build_mpo_site(kind, 1.0, 0.0, x, lam) - W00
    Wh = build_mpo_site(kind, 0.0, 1.0, x, lam) - W00
    return _t(W00), _t(WJ), _t(Wh)


# environments (Fig. 3, Eq. 19 and its mirror image), [bra, mpo, ket]
def env_left(beta, A, W):
    return torch.einsum("asb,awx,wvst,xty->bvy", A.conj(), beta, W, A)


def env_right(gamma, B, W):
    return torch.einsum("asb,wvst,bvy,xty->awx", B.conj(), W, gamma, B)


def heff2_matrix(L, W, R):
    """H2_eff as a matrix over (a, s1, s2, b) (Fig. 4a)."""
    a, b, d = L.shape[0], R.shape[0], W.shape[2]
    H = torch.einsum("awx,wvsp,vuqr,buy->asqbxpry", L, W, W, R)
    n = a * d * d * b
    return H.reshape(n, n)


def heff1_matrix(L, W, R):
    """H1_eff as a matrix over (a, s, b) (Fig. 4b)."""
    a, b, d = L.shape[0], R.shape[0], W.shape[2]
    H = torch.einsum("awx,wvst,bvy->asbxty", L, W, R)
    n = a * d * b
    return H.reshape(n, n)


def expm_apply(H, v, t):
    """exp(-i t H) v with the exact matrix exponential."""
    return (torch.linalg.matrix_exp(-1j * t * H) @ v.reshape(-1)).reshape(v.shape)


class Sweep:
    """The state of oracle.tdvp.Engine as torch tensors: Psi, V, beta, gamma, W."""

    def __init__(self, mps: MPS, W: torch.Tensor):
        self.Psi: List[torch.Tensor] = [_t(p) for p in mps.Psi]
        self.V: List[torch.Tensor] = [torch.as_tensor(v, dtype=torch.float64) for v in mps.V]
        self.W = W
        self.ranks: List[Tuple[int, int]] = []   # (bond, kept rank) of every split
        N = len(self.Psi)
        left, right = mpo_boundaries(W.shape[0])
        self.beta: List[Optional[torch.Tensor]] = [None] * N
        self.gamma: List[Optional[torch.Tensor]] = [None] * N
        self.beta[0] = _t(left)
        self.gamma[N - 1] = _t(right)
        for j in range(N - 1):
            self.beta[j + 1] = env_left(self.beta[j], self.A(j), W)
        for j in range(N - 2, -1, -1):
            self.gamma[j] = env_right(self.gamma[j + 1], self.B(j), W)

    def A(self, j):
        return self.Psi[j] * self.V[j].to(C128)[None, None, :]

    def B(self, j):
        return self.V[j].to(C128)[:, None, None] * self.Psi[j + 1]

    def fwd2(self, j: int, t: float, env: str, p: Params) -> None:
        theta = torch.einsum("asc,c,cub->asub", self.Psi[j], self.V[j].to(C128), self.Psi[j + 1])
        theta = expm_apply(heff2_matrix(self.beta[j], self.W, self.gamma[j + 1]), theta, t)
        a, d1, d2, b = theta.shape
        U, s, Vh = torch.linalg.svd(theta.reshape(a * d1, d2 * b), full_matrices=False)
        chi, _ = truncation_rank(_primal(s).numpy(), p.chi_max, p.w_max, p.eps)
        lam = s[:chi]
        self.Psi[j] = (U[:, :chi] * lam[None, :].to(C128)).reshape(a, d1, chi)
        self.V[j] = 1.0 / lam
        self.Psi[j + 1] = (lam[:, None].to(C128) * Vh[:chi]).reshape(chi, d2, b)
        self.ranks.append((j, chi))
        if "L" in env:
            self.beta[j + 1] = env_left(self.beta[j], self.A(j), self.W)
        if "R" in env:
            self.gamma[j] = env_right(self.gamma[j + 1], self.B(j), self.W)

    def back1(self, j: int, t: float) -> None:
        self.Psi[j] = expm_apply(heff1_matrix(self.beta[j], self.W, self.gamma[j]), self.Psi[j], t)

    def step(self, p: Params, n_steps: int) -> None:
        N = len(self.Psi)
        tau = 0.5 * p.dt
        sched = build_schedule(N, p.seg_len if p.seg_len else [N], p.merge_turning)
        for _ in range(n_steps):
            for half in sched:
                for op in execution_order(half, "stage"):
                    if op.kind == "fwd2":
                        self.fwd2(op.j, op.tfac * tau, op.env, p)
                    else:
                        self.back1(op.j, -op.tfac * tau)

    def state_vector(self) -> torch.Tensor:
        N = len(self.Psi)
        M = [self.A(j) for j in range(N - 1)] + [self.Psi[N - 1]]
        v = M[0].reshape(M[0].shape[1], M[0].shape[2])
        for Mj in M[1:]:
            v = torch.einsum("pa,asb->psb", v, Mj).reshape(-1, Mj.shape[2])
        return v.reshape(-1)


def local_expectations(psi: torch.Tensor, op: np.ndarray, N: int) -> torch.Tensor:
    """<psi|O_j|psi> / <psi|psi> for every site j from the state vector (site 0 most significant)."""
    O = _t(op)
    nrm = torch.vdot(psi, psi).real
    out = []
    for j in range(N):
        T = psi.reshape(2 ** j, 2, 2 ** (N - 1 - j))
        OT = torch.einsum("st,atb->asb", O, T)
        out.append(torch.vdot(T.reshape(-1), OT.reshape(-1)).real / nrm)
    return torch.stack(out)


OPS = {"z": SZ, "x": SX, "y": SY}


def evolve_observable(kind: int, x: np.ndarray, lam: np.ndarray, J, h, mps0: MPS, p: Params, n_steps: int,
                      obs: str = "z") -> Tuple[torch.Tensor, List[Tuple[int, int]]]:
    """<O_j(t)> after n_steps of TDVP from mps0 with W(J, h); J and h may be dual tensors."""
    W00, WJ, Wh = mpo_affine(kind, x, lam)
    W = W00 + J * WJ + h * Wh
    sw = Sweep(mps0, W)
    sw.step(p, n_steps)
    return local_expectations(sw.state_vector(), OPS[obs], len(sw.Psi)), sw.ranks


def jacobian(kind: int, x: np.ndarray, lam: np.ndarray, J: float, h: float, mps0: MPS, p: Params,
             n_steps: int, obs: str = "z") -> Tuple[np.ndarray, np.ndarray, List[Tuple[int, int]]]:
    """(<O_j(t)>, d<O_j(t)>/d(h, J) as an [N, 2] array, (bond, kept rank) of every split)
    by forward-mode AD, one pass per parameter."""
    cols = []
    value = None
    ranks: List[Tuple[int, int]] = []
    for dh, dJ in ((1.0, 0.0), (0.0, 1.0)):
        with fwAD.dual_level():
            Jd = fwAD.make_dual(torch.tensor(float(J), dtype=torch.float64), torch.tensor(dJ, dtype=torch.float64))
            hd = fwAD.make_dual(torch.tensor(float(h), dtype=torch.float64), torch.tensor(dh, dtype=torch.float64))
            out, ranks = evolve_observable(kind, x, lam, Jd, hd, mps0, p, n_steps, obs)
            pr, tg = fwAD.unpack_dual(out)
            value = pr.numpy().copy()
            cols.append(tg.numpy().copy())
    return value, np.stack(cols, axis=1), ranks


def final_dims(ranks: Sequence[Tuple[int, int]], n_bonds: int, initial: Sequence[int]) -> List[int]:
    """Bond dimensions after a run, from the (bond, rank) record of its splits."""
    dims = list(initial)
    for j, chi in ranks:
        dims[j] = chi
    assert len(dims) == n_bonds
    return dims
