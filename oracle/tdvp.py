"""Serial and segmented (parallel) two-site TDVP, plain FP64 (oracle).

Test infrastructure (see oracle/__init__.py): never imported by the product path.

Follows Sec. III of the paper:
  * effective environments beta_j (left of site j) and gamma_j (right of site j),
    Fig. 3; beta_{j+1} from beta_j, Psi_j V_j and W_j (Eq. 19), gamma_j mirrored;
  * two-site forward step Theta' = exp(-i H2_eff dt/2) Theta (Eq. 18), with
    Theta = Psi_j V_j Psi_{j+1} and H2_eff built from beta_j, W_j, W_{j+1},
    gamma_{j+1} (Fig. 4a);
  * Lanczos exponentiation (Park and Light) needing only H_eff . theta;
  * truncated SVD re-split Psi_L = A' L', Psi_R = L' B', V' = L'^-1 (Fig. 5) with
    the discarded-weight rule (Eq. 22, Sec. III C) and the relative cutoff
    eps * lambda_1 (Sec. III D);
  * one-site backward step Theta1' = exp(+i H1_eff dt/2) Theta1 (Eq. 20);
  * serial sweep (Sec. III A, Fig. 2, App. A) and the Stoudenmire-White segment
    scheme (Sec. III B, Figs. 6-7, App. B).

Index conventions: environments are [bra, mpo, ket]; MPO tensors are
W[w_left, w_right, s_out, s_in]; two-site states are [chi_l, d, d, chi_r].
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np
import scipy.linalg

from .models import mpo_boundaries
from .mps import MPS


# ---------------------------------------------------------------------------
# Environments (Fig. 3, Eq. 19)
# ---------------------------------------------------------------------------

def env_left(beta: np.ndarray, A: np.ndarray, W: np.ndarray) -> np.ndarray:
    """beta_{j+1}[b, w', b'] = sum conj(A[a,s,b]) beta_j[a,w,a'] W[w,w',s,s'] A[a',s',b'] (Eq. 19),
    with A = Psi_j V_j."""
    X1 = np.einsum("awx,xty->awty", beta, A)
    X2 = np.einsum("wvst,awty->asvy", W, X1)
    return np.einsum("asb,asvy->bvy", A.conj(), X2)


def env_right(gamma: np.ndarray, B: np.ndarray, W: np.ndarray) -> np.ndarray:
    """gamma_j[a, w, a'] = sum conj(B[a,s,b]) W[w,w',s,s'] gamma_{j+1}[b,w',b'] B[a',s',b'],
    with B = V_j Psi_{j+1} (the mirror image of Eq. 19)."""
    Y1 = np.einsum("xty,bvy->xtbv", B, gamma)
    Y2 = np.einsum("wvst,xtbv->wxsb", W, Y1)
    return np.einsum("asb,wxsb->awx", B.conj(), Y2)


# ---------------------------------------------------------------------------
# Effective Hamiltonians (Fig. 4)
# ---------------------------------------------------------------------------

def heff2_apply(L: np.ndarray, W1: np.ndarray, W2: np.ndarray, R: np.ndarray,
                theta: np.ndarray) -> np.ndarray:
    """y = H2_eff theta, y[a,s1,s2,b] = sum L[a,w,a'] W1[w,v,s1,t1] W2[v,u,s2,t2] R[b,u,b'] theta[a',t1,t2,b']."""
    T1 = np.einsum("awx,xtuy->awtuy", L, theta)
    T2 = np.einsum("wvst,awtuy->asvuy", W1, T1)
    T3 = np.einsum("vzqu,asvuy->asqzy", W2, T2)
    return np.einsum("asqzy,bzy->asqb", T3, R)


def heff1_apply(L: np.ndarray, W: np.ndarray, R: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """y = H1_eff theta, y[a,s,b] = sum L[a,w,a'] W[w,v,s,t] R[b,v,b'] theta[a',t,b']."""
    T1 = np.einsum("awx,xty->awty", L, theta)
    T2 = np.einsum("wvst,awty->asvy", W, T1)
    return np.einsum("asvy,bvy->asb", T2, R)


def heff2_dense(L, W1, W2, R) -> np.ndarray:
    """Explicit matrix of H2_eff (small sizes only; used by pins)."""
    a, _, _ = L.shape
    b = R.shape[0]
    d = W1.shape[2]
    n = a * d * d * b
    H = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[i] = 1.0
        H[:, i] = heff2_apply(L, W1, W2, R, e.reshape(a, d, d, b)).reshape(-1)
    return H


# ---------------------------------------------------------------------------
# Lanczos exponentiation (Park and Light; Sec. III A)
# ---------------------------------------------------------------------------

BREAKDOWN_REL = 1e-12


def tridiag_expm_e0(alpha: np.ndarray, beta: np.ndarray, t: float) -> np.ndarray:
    """c = exp(-i t T) e_0 for the real symmetric tridiagonal T = tridiag(beta, alpha, beta)."""
    k = len(alpha)
    if k == 1:
        return np.array([np.exp(-1j * t * alpha[0])])
    theta, Q = scipy.linalg.eigh_tridiagonal(np.asarray(alpha, float), np.asarray(beta, float))
    return Q @ (np.exp(-1j * t * theta) * Q[0, :])


@dataclasses.dataclass
class KrylovInfo:
    n_vectors: int
    breakdown: bool
    err: float


def lanczos_expm(apply_h: Callable[[np.ndarray], np.ndarray], theta: np.ndarray, t: float,
                 kmax: int, tol: float) -> Tuple[np.ndarray, KrylovInfo]:
    """exp(-i t H) theta using only products H v (Park and Light).

    Krylov basis with full re-orthogonalisation (two classical Gram-Schmidt
    passes per vector). After j+1 vectors the coefficients
    c = exp(-i t T_{j+1}) e_0 give the a-posteriori error estimate
    beta_{j+1} |c_j|. Stops at kmax vectors, when the estimate is below tol
    (tol = 0 disables this), or on breakdown beta_{j+1} <= 1e-12 (|alpha_j| + beta_j),
    i.e. an invariant subspace. Returns ||theta|| sum_i c_i v_i.
    """
    shape = theta.shape
    v0 = theta.reshape(-1)
    beta0 = np.linalg.norm(v0)
    if beta0 == 0.0:
        return theta.copy(), KrylovInfo(0, True, 0.0)
    Vs = [v0 / beta0]
    alpha: List[float] = []
    beta: List[float] = []
    c = np.array([1.0 + 0j])
    breakdown = False
    err = 0.0
    for j in range(kmax):
        w = apply_h(Vs[j].reshape(shape)).reshape(-1)
        h = np.array([np.vdot(Vs[i], w) for i in range(j + 1)])
        w = w - sum(h[i] * Vs[i] for i in range(j + 1))
        g = np.array([np.vdot(Vs[i], w) for i in range(j + 1)])
        w = w - sum(g[i] * Vs[i] for i in range(j + 1))
        alpha.append(float((h[j] + g[j]).real))
        b = float(np.linalg.norm(w))
        c = tridiag_expm_e0(np.array(alpha), np.array(beta), t)
        err = b * abs(c[j])
        scale = abs(alpha[j]) + (beta[j - 1] if j > 0 else 0.0)
        if b <= BREAKDOWN_REL * scale:
            breakdown = True
            break
        if tol > 0.0 and err < tol:
            break
        if j + 1 == kmax:
            break
        beta.append(b)
        Vs.append(w / b)
    y = beta0 * sum(c[i] * Vs[i] for i in range(len(c)))
    return y.reshape(shape), KrylovInfo(len(c), breakdown, err)


# ---------------------------------------------------------------------------
# Truncated split (Fig. 5, Eq. 22, Sec. III D)
# ---------------------------------------------------------------------------

def truncation_rank(s: np.ndarray, chi_max: int, w_max: float, eps: float) -> Tuple[int, float]:
    """Kept rank chi and discarded weight w for descending singular values s.

    chi_w = smallest rank with sum_{j >= chi_w} s_j^2 <= w_max (Eq. 22);
    chi = min(chi_w, chi_max) (Sec. III C), further limited to the values
    above eps * s_0 (Sec. III D) and to those above the FP64 rounding level
    1e-14 * ||s||_2 (= ||Theta'||_F): values at the noise level are numerical
    zeros, thrown away before Lambda is inverted (Sec. II B and its footnote),
    whatever eps. At least one value is kept.
    """
    n = len(s)
    sq = s.astype(np.float64) ** 2
    tail = np.zeros(n + 1)
    for k in range(n - 1, -1, -1):
        tail[k] = tail[k + 1] + sq[k]
    chi_w = n
    for k in range(1, n + 1):
        if tail[k] <= w_max:
            chi_w = k
            break
    n_eps = int(np.count_nonzero(s > eps * s[0])) if s[0] > 0 else 1
    n_noise = int(np.count_nonzero(s > 1e-14 * np.sqrt(sq.sum())))
    chi = max(1, min(chi_w, chi_max, n_eps, n_noise))
    return chi, float(tail[chi])


def split_two_site(theta: np.ndarray, chi_max: int, w_max: float, eps: float):
    """Theta' -> (Psi_L, V, Psi_R, w) with Psi_L = A' L', Psi_R = L' B', V = 1/L' (Fig. 5)."""
    a, d1, d2, b = theta.shape
    U, s, Vh = np.linalg.svd(theta.reshape(a * d1, d2 * b), full_matrices=False)
    chi, w = truncation_rank(s, chi_max, w_max, eps)
    lam = s[:chi]
    Psi_L = (U[:, :chi] * lam[None, :]).reshape(a, d1, chi)
    Psi_R = (lam[:, None] * Vh[:chi]).reshape(chi, d2, b)
    return Psi_L, 1.0 / lam, Psi_R, w, s


# ---------------------------------------------------------------------------
# The state of a run: MPS, MPO, environments
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    dt: float
    chi_max: int
    w_max: float = 0.0
    eps: float = 1e-12
    krylov_max: int = 8
    krylov_tol: float = 1e-6
    seg_len: Optional[List[int]] = None
    merge_turning: int = 1


@dataclasses.dataclass
class Stats:
    w_total: float = 0.0
    chi_max_seen: int = 0
    krylov_vectors: int = 0
    n_fwd2: int = 0
    n_back1: int = 0


class Engine:
    """Holds MPS, MPO (the same W on every site) and the cached environments."""

    def __init__(self, mps: MPS, W: np.ndarray):
        self.mps = mps
        self.W = W
        N = mps.N
        m = W.shape[0]
        left, right = mpo_boundaries(m)
        self.beta: List[Optional[np.ndarray]] = [None] * N
        self.gamma: List[Optional[np.ndarray]] = [None] * N
        self.beta[0] = left
        self.gamma[N - 1] = right
        # Initial environments: all beta from the left, all gamma from the
        # right (Sec. III A: computed once at the start; Sec. III B: each
        # partition needs the ones of its own sites).
        for j in range(N - 1):
            self.beta[j + 1] = env_left(self.beta[j], self._A(j), W)
        for j in range(N - 2, -1, -1):
            self.gamma[j] = env_right(self.gamma[j + 1], self._B(j), W)
        self.stats = Stats()

    def _A(self, j: int) -> np.ndarray:
        return self.mps.Psi[j] * self.mps.V[j][None, None, :]

    def _B(self, j: int) -> np.ndarray:
        """V_j Psi_{j+1}."""
        return self.mps.V[j][:, None, None] * self.mps.Psi[j + 1]

    # -- local operations ---------------------------------------------------
    def fwd2(self, j: int, t: float, env: str, p: Params) -> None:
        """Two-site forward step on pair (j, j+1) by time t (Eq. 18), re-split (Fig. 5),
        then rebuild beta_{j+1} ('L') and/or gamma_j ('R')."""
        mps, W = self.mps, self.W
        theta = np.einsum("asc,c,cub->asub", mps.Psi[j], mps.V[j], mps.Psi[j + 1])
        L, R = self.beta[j], self.gamma[j + 1]
        theta2, info = lanczos_expm(lambda x: heff2_apply(L, W, W, R, x), theta, t,
                                    p.krylov_max, p.krylov_tol)
        Psi_L, Vn, Psi_R, w, _ = split_two_site(theta2, p.chi_max, p.w_max, p.eps)
        mps.Psi[j], mps.V[j], mps.Psi[j + 1] = Psi_L, Vn, Psi_R
        if "L" in env:
            self.beta[j + 1] = env_left(self.beta[j], self._A(j), W)
        if "R" in env:
            self.gamma[j] = env_right(self.gamma[j + 1], self._B(j), W)
        st = self.stats
        st.w_total += w
        st.chi_max_seen = max(st.chi_max_seen, len(Vn))
        st.krylov_vectors += info.n_vectors
        st.n_fwd2 += 1

    def back1(self, j: int, t: float, p: Params) -> None:
        """One-site step on site j by time t (Eq. 20 uses t = -dt/2)."""
        L, R, W = self.beta[j], self.gamma[j], self.W
        psi, info = lanczos_expm(lambda x: heff1_apply(L, W, R, x), self.mps.Psi[j], t,
                                 p.krylov_max, p.krylov_tol)
        self.mps.Psi[j] = psi
        self.stats.krylov_vectors += info.n_vectors
        self.stats.n_back1 += 1

    def run_op(self, op: "Op", p: Params) -> None:
        tau = 0.5 * p.dt
        if op.kind == "fwd2":
            self.fwd2(op.j, op.tfac * tau, op.env, p)
        else:
            self.back1(op.j, -op.tfac * tau, p)

    def step(self, p: Params, n_steps: int = 1, order: str = "stage") -> Stats:
        N = self.mps.N
        seg = p.seg_len if p.seg_len else [N]
        sched = build_schedule(N, seg, p.merge_turning)
        for _ in range(n_steps):
            for half in sched:
                for op in execution_order(half, order):
                    self.run_op(op, p)
        return self.stats


# ---------------------------------------------------------------------------
# Sweep schedule: serial (Sec. III A, Fig. 2, App. A) and segmented
# (Sec. III B, Figs. 6-7, App. B; the activity diagrams themselves are not in
# the text, so the rules below are our reading of the prose)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Op:
    seg: int
    kind: str          # "fwd2" (pair j, j+1) or "back1" (site j)
    j: int
    tfac: int          # forward time in units of tau = dt/2 (1 or 2); back1: 1
    env: str = ""      # after fwd2: "L" builds beta_{j+1}, "R" builds gamma_j
    boundary: bool = False
    deps: Tuple[int, ...] = ()   # indices (within the half) of ops it waits for
    stage: int = -1


def segment_bounds(N: int, seg_len: List[int]) -> List[Tuple[int, int]]:
    assert sum(seg_len) == N, "segment lengths must add up to N"
    out, s = [], 0
    for n in seg_len:
        assert n >= 2, "a partition holds at least two sites (Sec. III B)"
        out.append((s, s + n - 1))
        s += n
    return out


def sweeps_right_first(k: int, p: int) -> bool:
    """Direction of segment k in the first half of a step (Sec. III B, Fig. 6).

    The two central segments sweep away from the centre first and neighbours
    alternate: segment k sweeps right iff k and p//2 have the same parity.
    For p = 1 this is the serial left-to-right first sweep.
    """
    return (k % 2) == ((p // 2) % 2)


def build_half(N: int, seg_len: List[int], half: int, merge: int) -> List[Op]:
    """Ops of one half of a time step, in stage order, with cross-segment waits.

    Per segment [s, e] sweeping right: pairs (s..e-1) interleaved with back1 of
    the site they share, as in the serial sweep (Fig. 2). The boundary pair
    (e, e+1) is updated by the left segment (Sec. III B). Turning pairs where
    a half ends (chain ends in half 1, converging boundaries in half 1) are
    evolved once by 2 tau when merge is on (App. A); pairs where half 1 starts
    (a chain end or a diverging boundary) get tau at the start of half 1 and
    tau at the end of half 2. A segment that leaves a boundary starts with
    back1 of its boundary site. Leftward sweeps are the mirror image.
    """
    segs = segment_bounds(N, seg_len)
    p = len(segs)
    per_seg: List[List[Op]] = [[] for _ in range(p)]
    turn = 2 if (half == 1 and merge) else 1
    start_boundary: Dict[int, Op] = {}
    end_boundary: Dict[int, Op] = {}
    for k, (s, e) in enumerate(segs):
        right = sweeps_right_first(k, p) if half == 1 else not sweeps_right_first(k, p)
        q = per_seg[k]
        if right:
            if s == 0:
                if half == 1 or not merge:
                    q.append(Op(k, "fwd2", 0, 1, "L"))
                first_back = 1
            else:
                first_back = s
            for j in range(first_back, e):
                q.append(Op(k, "back1", j, 1))
                last = (j == e - 1) and (e == N - 1)
                q.append(Op(k, "fwd2", j, turn if last else 1, "R" if last else "L"))
            if e < N - 1:
                q.append(Op(k, "back1", e, 1))
                op = Op(k, "fwd2", e, turn, "LR", boundary=True)
                q.append(op)
                end_boundary[k] = op
        else:
            if e == N - 1:
                if half == 1 or not merge:
                    q.append(Op(k, "fwd2", N - 2, 1, "R"))
                first_back = N - 2
            else:
                if half == 1 or not merge:
                    op = Op(k, "fwd2", e, 1, "LR", boundary=True)
                    q.append(op)
                    start_boundary[k] = op
                first_back = e
            for j in range(first_back, s, -1):
                q.append(Op(k, "back1", j, 1))
                last = (j - 1 == s) and (s == 0)
                q.append(Op(k, "fwd2", j - 1, turn if last else 1, "L" if last else "R"))
            if s > 0:
                q.append(Op(k, "back1", s, 1))
    # stage assignment (as soon as possible)
    done_stage: Dict[int, int] = {}
    for k in range(p):
        for i, op in enumerate(per_seg[k]):
            op.stage = -1
    # iterate to a fixed point: stage = max(previous in queue, dependencies) + 1
    changed = True
    while changed:
        changed = False
        for k in range(p):
            prev = -1
            for i, op in enumerate(per_seg[k]):
                st = prev + 1
                if i == 0 and (k - 1) in start_boundary:
                    # right neighbour of a start-of-half boundary op waits for it
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


def build_schedule(N: int, seg_len: List[int], merge: int = 1) -> List[List[Op]]:
    return [build_half(N, seg_len, 1, merge), build_half(N, seg_len, 2, merge)]


def execution_order(ops: List[Op], order: str) -> List[Op]:
    """'stage': stage by stage; 'segment': segment-major topological order (any
    order that respects the waits gives the same result)."""
    if order == "stage":
        return ops
    remaining = list(range(len(ops)))
    done = set()
    out = []
    while remaining:
        # pick the highest-numbered segment whose next op is ready
        best = None
        for i in remaining:
            if all(d in done for d in ops[i].deps):
                if best is None or ops[i].seg > ops[best].seg:
                    best = i
        out.append(ops[best])
        done.add(best)
        remaining.remove(best)
    return out
