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

import dataclasses
from typing import Callable, Dict, List, Tuple

import numpy as np

from .tdvp import (Engine, Params, env_left, env_right, heff1_apply, heff2_apply, lanczos_expm,
                   segment_bounds, split_two_site, sweeps_right_first)


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
    step once all are saturated, both with the segments of p.seg_len (serial
    without). Returns the number of one-site steps taken."""
    n1 = 0
    for _ in range(n_steps):
        if saturated(eng, p.chi_max):
            step1_segmented(eng, p, 1)
            n1 += 1
        else:
            eng.step(p, 1)
    return n1


# ---------------------------------------------------------------------------
# Segmented (parallel) one-site TDVP, our reading of the paper's outlook on a
# parallel 1TDVP. The chain is cut into the segments of the two-site scheme
# (Sec. III B; directions, turning rules and waits as in oracle.tdvp.build_half)
# and every segment runs the one-site sweep above over its own sites. The two
# sites of a boundary are evolved together, as in the two-site scheme: the
# left segment forms Theta = Psi_e V_e Psi_{e+1} (V = Lambda^-1, Sec. III B),
# evolves it with H2_eff and splits it back at the bond's current dimension.
# That pair step stands for the site terms of e and e+1 and the bond term
# between them, so neither segment evolves its boundary site on its own: a
# segment that leaves a boundary starts with the bond next to it. Boundaries
# where the first half's sweeps converge get their pair step once by 2 tau at
# the end of the first half (twice tau without merging); those where the
# sweeps start get tau before the first half and tau after the second. With
# one segment this is exactly step1; at full bond dimension it is exact, like
# the serial sweep.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Op1:
    seg: int
    kind: str        # "site" (forward, site j), "bond_r" / "bond_l" (bond_backward_right(j) /
                     # bond_backward_left(j)), "pair" (boundary pair j, j+1)
    j: int
    tfac: int        # time in units of tau = dt/2
    stage: int = -1
    deps: Tuple[int, ...] = ()


def build_half1(N: int, seg_len: List[int], half: int, merge: int) -> List[Op1]:
    """Ops of one half of a segmented one-site time step, in stage order."""
    segs = segment_bounds(N, seg_len)
    p = len(segs)
    turn = 2 if (half == 1 and merge) else 1
    per_seg: List[List[Op1]] = [[] for _ in range(p)]
    start_boundary: Dict[int, Op1] = {}
    end_boundary: Dict[int, Op1] = {}
    for k, (s, e) in enumerate(segs):
        right = sweeps_right_first(k, p) if half == 1 else not sweeps_right_first(k, p)
        q = per_seg[k]
        if right:
            if s == 0 and (half == 1 or not merge):
                q.append(Op1(k, "site", 0, 1))
            last_site = e if e == N - 1 else e - 1   # a boundary site is in the pair step
            for j in range(s, e):
                q.append(Op1(k, "bond_r", j, 1))
                if j + 1 <= last_site:
                    turning = (j + 1 == e) and (e == N - 1)
                    q.append(Op1(k, "site", j + 1, turn if turning else 1))
            if e < N - 1:
                op = Op1(k, "pair", e, turn)
                q.append(op)
                end_boundary[k] = op
        else:
            if e == N - 1:
                if half == 1 or not merge:
                    q.append(Op1(k, "site", N - 1, 1))
            elif half == 1 or not merge:
                op = Op1(k, "pair", e, 1)
                q.append(op)
                start_boundary[k] = op
            first_site = s if s == 0 else s + 1
            for j in range(e, s, -1):
                q.append(Op1(k, "bond_l", j, 1))
                if j - 1 >= first_site:
                    turning = (j - 1 == s) and (s == 0)
                    q.append(Op1(k, "site", j - 1, turn if turning else 1))
    changed = True
    while changed:
        changed = False
        for k in range(p):
            prev = -1
            for i, op in enumerate(per_seg[k]):
                st = prev + 1
                if i == 0 and (k - 1) in start_boundary:
                    st = max(st, start_boundary[k - 1].stage + 1)
                if op is end_boundary.get(k):
                    st = max(st, per_seg[k + 1][-1].stage + 1)
                if st != op.stage:
                    op.stage = st
                    changed = True
                prev = op.stage
    ops = [op for k in range(p) for op in per_seg[k]]
    ops.sort(key=lambda o: (o.stage, o.seg))
    index = {id(o): i for i, o in enumerate(ops)}
    for k in range(p):
        for i, op in enumerate(per_seg[k]):
            deps = []
            if i > 0:
                deps.append(index[id(per_seg[k][i - 1])])
            if i == 0 and (k - 1) in start_boundary:
                deps.append(index[id(start_boundary[k - 1])])
            if op is end_boundary.get(k):
                deps.append(index[id(per_seg[k + 1][-1])])
            op.deps = tuple(deps)
    return ops


def boundary_pair(eng: Engine, e: int, t: float, p: Params) -> None:
    """Sites e, e+1 evolved together by t (Eq. 18 with Theta = Psi_e V_e Psi_{e+1})
    and split back at the bond's current dimension (the relative cutoff p.eps
    still applies); beta_{e+1} and gamma_e rebuilt."""
    mps, W = eng.mps, eng.W
    chi = len(mps.V[e])
    theta = np.einsum("asc,c,cub->asub", mps.Psi[e], mps.V[e], mps.Psi[e + 1])
    L, R = eng.beta[e], eng.gamma[e + 1]
    theta2, _ = lanczos_expm(lambda x: heff2_apply(L, W, W, R, x), theta, t, p.krylov_max, p.krylov_tol)
    Psi_L, Vn, Psi_R, _, _ = split_two_site(theta2, chi, 0.0, p.eps)
    mps.Psi[e], mps.V[e], mps.Psi[e + 1] = Psi_L, Vn, Psi_R
    eng.beta[e + 1] = env_left(eng.beta[e], eng._A(e), W)
    eng.gamma[e] = env_right(eng.gamma[e + 1], eng._B(e), W)


def run_op1(eng: Engine, op: Op1, p: Params) -> None:
    t = op.tfac * 0.5 * p.dt
    if op.kind == "site":
        site_forward(eng, op.j, t, p)
    elif op.kind == "bond_r":
        bond_backward_right(eng, op.j, t, p)
    elif op.kind == "bond_l":
        bond_backward_left(eng, op.j, t, p)
    else:
        boundary_pair(eng, op.j, t, p)


def step1_segmented(eng: Engine, p: Params, n_steps: int = 1) -> None:
    """n_steps symmetric one-site steps with the segments of p.seg_len (one
    segment: the serial sweep of step1). At the start of a step the chain-end
    environment that the first half reads first is rebuilt from the current
    state, as step1 does for gamma_0 (a two-site half that ends moving away
    from a chain end leaves that end's environment behind): gamma_0 when the
    first segment starts at site 0, beta_{N-1} when the last one starts at
    site N-1."""
    N = eng.mps.N
    seg = p.seg_len if p.seg_len else [N]
    halves = [build_half1(N, seg, 1, p.merge_turning), build_half1(N, seg, 2, p.merge_turning)]
    nseg = len(seg)
    for _ in range(n_steps):
        if sweeps_right_first(0, nseg):
            eng.gamma[0] = env_right(eng.gamma[1], eng._B(0), eng.W)
        if not sweeps_right_first(nseg - 1, nseg):
            eng.beta[N - 1] = env_left(eng.beta[N - 2], eng._A(N - 2), eng.W)
        for half in halves:
            for op in half:
                run_op1(eng, op, p)
