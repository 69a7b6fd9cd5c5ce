"""One-site TDVP (1TDVP) and the hybrid two-site -> one-site scheme, plain FP64 (oracle).

Test infrastructure (see oracle/__init__.py): never imported by the product path.

The paper defines the one-site tangent-space projector (Eq. proj1site: a sum of
one-site terms minus a sum of bond terms) and the 1TDVP it leads to: a
Lie-Trotter-Suzuki splitting that evolves one site tensor forward, then the bond
matrix backward, sweeping like one-site DMRG, at fixed bond dimension (Sec. II).
Its discussion proposes a parallel one-site variant and the hybrid scheme that
switches from 2TDVP to 1TDVP once chi_max is reached. This module is the serial
1TDVP step in the inverse canonical gauge of oracle.tdvp, our reading:

left-to-right half (tau = dt/2), for j = 0 .. N-2:
  Psi_j <- exp(-i tau H1_eff(j)) Psi_j                       (site term, forward)
  Psi_j = U S W^H  (as a (chi_{j-1} d) x chi_j matrix, no truncation)
  A_j = U, beta_{j+1} from A_j; C = S W^H (the bond matrix)
  C <- exp(+i tau H0_eff(j)) C                               (bond term, backward)
  C = u s v^H: Psi_j = U u s, V_j = 1/s, Psi_{j+1} <- s v^H V_j(old) Psi_{j+1}
  beta_{j+1} rebuilt from Psi_j V_j
then the last site forward by 2 tau (the two halves' turning terms merged), and
the right-to-left half as the mirror image, ending with site 0 forward by tau.
gamma_0 is rebuilt at the start of a step (after a two-site step it is stale).
H0_eff(j) C = sum beta_{j+1}[a,w,a'] C[a',b'] gamma_j[b,w,b'] (Fig. 4 without W).
"""
from __future__ import annotations

from typing import Callable

import numpy as np

from .tdvp import Engine, Params, env_left, env_right, heff1_apply, lanczos_expm


def heff0_apply(L: np.ndarray, R: np.ndarray, C: np.ndarray) -> np.ndarray:
    """y = H0_eff C, y[a,b] = sum L[a,w,a'] C[a',b'] R[b,w,b']."""
    return np.einsum("awx,xy,bwy->ab", L, C, R)


def _svd(M: np.ndarray):
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    k = max(1, int(np.count_nonzero(s > 1e-14 * np.linalg.norm(s))))
    return U[:, :k], s[:k], Vh[:k]


def _expm(apply: Callable[[np.ndarray], np.ndarray], x: np.ndarray, t: float, p: Params) -> np.ndarray:
    y, _ = lanczos_expm(apply, x, t, p.krylov_max, p.krylov_tol)
    return y


def site_forward(eng: Engine, j: int, t: float, p: Params) -> None:
    L, R, W = eng.beta[j], eng.gamma[j], eng.W
    eng.mps.Psi[j] = _expm(lambda x: heff1_apply(L, W, R, x), eng.mps.Psi[j], t, p)


def bond_backward_right(eng: Engine, j: int, tau: float, p: Params) -> None:
    """Split site j, evolve the bond matrix of bond j by +tau backward, move it into site j+1."""
    mps, W = eng.mps, eng.W
    a, d, b = mps.Psi[j].shape
    U, S, Wh = _svd(mps.Psi[j].reshape(a * d, b))
    k = len(S)
    A = U.reshape(a, d, k)
    eng.beta[j + 1] = env_left(eng.beta[j], A, W)
    C = S[:, None] * Wh
    L, R = eng.beta[j + 1], eng.gamma[j]
    C = _expm(lambda x: heff0_apply(L, R, x), C, -tau, p)
    u, s, vh = _svd(C)
    Vold = mps.V[j]
    mps.Psi[j] = np.einsum("xsk,kq->xsq", A, u * s[None, :])
    mps.V[j] = 1.0 / s
    mps.Psi[j + 1] = np.einsum("qb,b,bsc->qsc", s[:, None] * vh, Vold, mps.Psi[j + 1])
    eng.beta[j + 1] = env_left(eng.beta[j], eng._A(j), W)


def bond_backward_left(eng: Engine, j: int, tau: float, p: Params) -> None:
    """Split site j, evolve the bond matrix of bond j-1 by +tau backward, move it into site j-1."""
    mps, W = eng.mps, eng.W
    a, d, b = mps.Psi[j].shape
    U, S, Wh = _svd(mps.Psi[j].reshape(a, d * b))
    k = len(S)
    Bj = Wh.reshape(k, d, b)
    eng.gamma[j - 1] = env_right(eng.gamma[j], Bj, W)
    C = U * S[None, :]
    L, R = eng.beta[j], eng.gamma[j - 1]
    C = _expm(lambda x: heff0_apply(L, R, x), C, -tau, p)
    u, s, vh = _svd(C)
    Vold = mps.V[j - 1]
    mps.Psi[j] = np.einsum("qk,ksb->qsb", s[:, None] * vh, Bj)
    mps.V[j - 1] = 1.0 / s
    mps.Psi[j - 1] = np.einsum("xsa,a,aq->xsq", mps.Psi[j - 1], Vold, u * s[None, :])
    eng.gamma[j - 1] = env_right(eng.gamma[j], eng._B(j - 1), W)


def step1(eng: Engine, p: Params, n_steps: int = 1) -> None:
    """n_steps symmetric 1TDVP steps (serial sweep, see the module docstring)."""
    N = eng.mps.N
    tau = 0.5 * p.dt
    for _ in range(n_steps):
        # gamma_0 as the current state has it (a preceding two-site half ends
        # with the pair (0, 1) and leaves gamma_0 behind)
        eng.gamma[0] = env_right(eng.gamma[1], eng._B(0), eng.W)
        for j in range(N - 1):
            site_forward(eng, j, tau, p)
            bond_backward_right(eng, j, tau, p)
        site_forward(eng, N - 1, 2 * tau, p)
        for j in range(N - 1, 0, -1):
            bond_backward_left(eng, j, tau, p)
            site_forward(eng, j - 1, tau, p)


def saturated(eng: Engine, chi_max: int) -> bool:
    """Every bond at min(chi_max, the largest dimension the bond can have)."""
    N, d = eng.mps.N, eng.mps.Psi[0].shape[1]
    for j, v in enumerate(eng.mps.V):
        full = min(d ** (j + 1), d ** (N - 1 - j))
        if len(v) < min(chi_max, full):
            return False
    return True


def step_hybrid(eng: Engine, p: Params, n_steps: int = 1) -> int:
    """The hybrid scheme: a two-site step while some bond can still grow, a one-site
    step once all are saturated. Returns the number of one-site steps taken."""
    n1 = 0
    for _ in range(n_steps):
        if saturated(eng, p.chi_max):
            step1(eng, p, 1)
            n1 += 1
        else:
            eng.step(p, 1)
    return n1
