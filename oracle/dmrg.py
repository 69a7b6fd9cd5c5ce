"""Two-site DMRG ground states with the TDVP building blocks, plain FP64 (oracle).

Test infrastructure (see oracle/__init__.py): never imported by the product path.

The paper prepares the initial states of its Ising, XY and XXX benchmarks with
two-site DMRG (Sec. IV and the Supplemental Material: the same Lanczos
settings as the exponentiation, ARPACK as eigensolver) and notes that a TDVP
time step has the sweeping pattern and cost of a two-site DMRG sweep
(Sec. II C, Sec. III A). It prints no DMRG algorithm, so this is the textbook
one (White's two-site update in the MPS formulation): at each pair the
two-site state is replaced by the lowest eigenvector of H2_eff, found by
Lanczos on the tridiagonal projection, then re-split and the environments
updated exactly as in the TDVP sweep. No backward one-site step.

Reading: the local eigensolver is an unrestarted Lanczos with full
re-orthogonalisation started from the current two-site state, at most kmax
vectors, stopped on breakdown or when the residual estimate
beta_{j+1} |z_j| (z the lowest Ritz vector) falls below tol; the new state
keeps the norm of the old one (no renormalisation, as in the TDVP sweep).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Tuple

import numpy as np
import scipy.linalg

from .tdvp import BREAKDOWN_REL, Engine, env_left, env_right, heff2_apply, split_two_site


@dataclasses.dataclass
class GroundInfo:
    n_vectors: int
    energy: float
    residual: float


def tridiag_ground(alpha: np.ndarray, beta: np.ndarray) -> Tuple[float, np.ndarray]:
    """Lowest eigenpair of the real symmetric tridiagonal T = tridiag(beta, alpha, beta)."""
    if len(alpha) == 1:
        return float(alpha[0]), np.array([1.0])
    theta, Q = scipy.linalg.eigh_tridiagonal(np.asarray(alpha, float), np.asarray(beta, float))
    return float(theta[0]), Q[:, 0]


def lanczos_ground(apply_h: Callable[[np.ndarray], np.ndarray], theta: np.ndarray, kmax: int,
                   tol: float) -> Tuple[np.ndarray, GroundInfo]:
    """Lowest eigenvector of H (only products H v) in the Krylov space of theta,
    returned with the norm of theta, and its Ritz value."""
    shape = theta.shape
    v0 = theta.reshape(-1)
    beta0 = np.linalg.norm(v0)
    if beta0 == 0.0:
        return theta.copy(), GroundInfo(0, 0.0, 0.0)
    Vs = [v0 / beta0]
    alpha: List[float] = []
    beta: List[float] = []
    e0, z = 0.0, np.array([1.0])
    res = 0.0
    for j in range(kmax):
        w = apply_h(Vs[j].reshape(shape)).reshape(-1)
        # two classical Gram-Schmidt passes (full re-orthogonalisation)
        h = np.array([np.vdot(Vs[i], w) for i in range(j + 1)])
        w = w - sum(h[i] * Vs[i] for i in range(j + 1))
        g = np.array([np.vdot(Vs[i], w) for i in range(j + 1)])
        w = w - sum(g[i] * Vs[i] for i in range(j + 1))
        alpha.append(float((h[j] + g[j]).real))
        b = float(np.linalg.norm(w))
        e0, z = tridiag_ground(np.array(alpha), np.array(beta))
        res = b * abs(z[j])
        scale = abs(alpha[j]) + (beta[j - 1] if j > 0 else 0.0)
        if b <= BREAKDOWN_REL * scale:
            break
        if tol > 0.0 and res < tol:
            break
        if j + 1 == kmax:
            break
        beta.append(b)
        Vs.append(w / b)
    y = beta0 * sum(z[i] * Vs[i] for i in range(len(z)))
    return y.reshape(shape), GroundInfo(len(z), e0, res)


@dataclasses.dataclass
class DmrgParams:
    chi_max: int
    w_max: float = 0.0
    eps: float = 1e-12
    krylov_max: int = 8
    krylov_tol: float = 1e-6


@dataclasses.dataclass
class DmrgStats:
    energy: float = 0.0
    w_total: float = 0.0
    chi_max_seen: int = 0
    krylov_vectors: int = 0
    energies: List[float] = dataclasses.field(default_factory=list)


def dmrg_update(eng: Engine, j: int, env: str, p: DmrgParams, st: DmrgStats) -> float:
    """Ground-state update of pair (j, j+1): Theta -> lowest eigenvector of H2_eff,
    re-split (Fig. 5) and the environment of the sweep direction rebuilt."""
    mps, W = eng.mps, eng.W
    theta = np.einsum("asc,c,cub->asub", mps.Psi[j], mps.V[j], mps.Psi[j + 1])
    L, R = eng.beta[j], eng.gamma[j + 1]
    theta2, info = lanczos_ground(lambda x: heff2_apply(L, W, W, R, x), theta, p.krylov_max, p.krylov_tol)
    Psi_L, Vn, Psi_R, w, _ = split_two_site(theta2, p.chi_max, p.w_max, p.eps)
    mps.Psi[j], mps.V[j], mps.Psi[j + 1] = Psi_L, Vn, Psi_R
    if "L" in env:
        eng.beta[j + 1] = env_left(eng.beta[j], eng._A(j), W)
    if "R" in env:
        eng.gamma[j] = env_right(eng.gamma[j + 1], eng._B(j), W)
    st.w_total += w
    st.chi_max_seen = max(st.chi_max_seen, len(Vn))
    st.krylov_vectors += info.n_vectors
    st.energy = info.energy
    return info.energy


def dmrg(eng: Engine, p: DmrgParams, n_sweeps: int) -> DmrgStats:
    """n_sweeps serial two-site DMRG sweeps (left to right over the pairs
    0..N-2 rebuilding left environments, then right to left rebuilding right
    environments). stats.energy is the last Ritz value; stats.energies holds
    it after every sweep."""
    N = eng.mps.N
    st = DmrgStats()
    for _ in range(n_sweeps):
        for j in range(N - 1):
            dmrg_update(eng, j, "L", p, st)
        for j in range(N - 2, -1, -1):
            dmrg_update(eng, j, "R", p, st)
        st.energies.append(st.energy)
    return st
