"""Model definitions for the oracle: spin operators, the power-law fit and the MPO.

Test infrastructure (see oracle/__init__.py): never imported by the product path.

Sec. II C: long-range power laws 1/r^alpha are approximated by a sum of
n_exp exponentials, f(r) ~ sum_k x_k lam_k^r, which gives an MPO of bond
dimension m = n_H * n_exp + 2 (n_H = number of long-range terms).
The paper uses the method of Pirvu et al. (appendix of their MPO paper); the
fit below is the same shift-invariance (matrix-pencil) idea: the samples
f(1..R) are arranged in a Hankel matrix, its dominant right singular
subspace is shift invariant under multiplication by diag(lam), and the
exponents lam_k are the eigenvalues of that shift; the weights x_k then
follow by linear least squares.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
ID2 = np.eye(2, dtype=np.complex128)

ISING, XY, XXX = 0, 1, 2


def model_terms(kind: int) -> Tuple[List[Tuple[np.ndarray, np.ndarray]], np.ndarray]:
    """Long-range terms (A_t, B_t) and the on-site field operator F.

    Sec. IV: Ising uses sigma^z sigma^z with a sigma^x field (Eq. 25); XY uses
    sigma^x sigma^x + sigma^y sigma^y (Eq. 27); XXX uses S.S = (1/4) sigma.sigma
    (Eq. 31). Signs and prefactors are carried by J and h.
    """
    if kind == ISING:
        return [(SZ, SZ)], SX
    if kind == XY:
        return [(SX, SX), (SY, SY)], SX
    if kind == XXX:
        return [(0.5 * SX, 0.5 * SX), (0.5 * SY, 0.5 * SY), (0.5 * SZ, 0.5 * SZ)], SX
    raise ValueError(kind)


def fit_exponentials(f: np.ndarray, n_exp: int) -> Tuple[np.ndarray, np.ndarray]:
    """Fit samples f(1..R) by sum_k x_k lam_k^r (shift-invariance / matrix pencil).

    Steps: Hankel matrix Y[i, j] = f(1 + i + j); SVD; keep the n_exp dominant
    right singular vectors Q; lam = eig(pinv(Q[:-1]) Q[1:]); x from least squares.
    If R is too small for n_exp exponentials the missing ones get x = 0.
    """
    f = np.asarray(f, dtype=np.float64)
    r_max = len(f)
    r = np.arange(1, r_max + 1, dtype=np.float64)
    K = int(n_exp)
    L = r_max // 2                      # pencil parameter
    rows = r_max - L
    k_eff = min(K, L, rows)
    Y = np.array([[f[i + j] for j in range(L + 1)] for i in range(rows)])
    _, _, Vh = np.linalg.svd(Y)
    Q = Vh[:k_eff].conj().T             # (L+1) x k_eff
    shift = np.linalg.pinv(Q[:-1]) @ Q[1:]
    lam = np.linalg.eigvals(shift).astype(np.complex128)
    P = lam[None, :] ** r[:, None]
    x = np.linalg.lstsq(P, f.astype(np.complex128), rcond=None)[0]
    if k_eff < K:                       # pad with inert exponentials
        pad = K - k_eff
        lam = np.concatenate([lam, np.full(pad, 0.5, dtype=np.complex128)])
        x = np.concatenate([x, np.zeros(pad, dtype=np.complex128)])
    return x.astype(np.complex128), lam.astype(np.complex128)


def fit_power_law(alpha: float, n_exp: int, r_max: int) -> Tuple[np.ndarray, np.ndarray]:
    """Approximate f(r) = r^-alpha on r = 1..r_max by sum_k x_k lam_k^r (Sec. II C)."""
    r = np.arange(1, r_max + 1, dtype=np.float64)
    return fit_exponentials(r ** (-float(alpha)), n_exp)


def fit_exponentials_lm(f: np.ndarray, x0: np.ndarray, lam0: np.ndarray, relative: bool):
    """Levenberg-Marquardt least squares for real x_k, lam_k in f(r) ~ sum_k x_k lam_k^r
    (the alternative fit of the Supplemental Material's power-law section, with its
    lsqnonlin stopping values: step 1e-6, function 1e-14, 10000 evaluations), residuals
    e_r weighted by 1 or 1/f(r). The minimiser is scipy's MINPACK Levenberg-Marquardt.
    Returns (x, lam, rms of the weighted residuals)."""
    import scipy.optimize
    f = np.asarray(f, dtype=np.float64)
    r = np.arange(1, len(f) + 1, dtype=np.float64)
    K = len(x0)
    w = 1.0 / f if relative else np.ones_like(f)

    def res(p):
        return w * ((p[None, :K] * p[None, K:] ** r[:, None]).sum(axis=1) - f)

    def jac(p):
        Jx = p[None, K:] ** r[:, None]
        Jl = p[None, :K] * r[:, None] * p[None, K:] ** (r[:, None] - 1)
        return w[:, None] * np.hstack([Jx, Jl])

    p0 = np.concatenate([np.real(x0), np.real(lam0)]).astype(np.float64)
    out = scipy.optimize.least_squares(res, p0, jac=jac, method="lm", xtol=1e-6, ftol=1e-14, max_nfev=10000)
    p = out.x
    if not (np.all(np.abs(p[K:]) < 1) and np.all(p[K:] != 0)) or (res(p) ** 2).sum() > (res(p0) ** 2).sum():
        p = p0
    return p[:K].astype(np.complex128), p[K:].astype(np.complex128), float(np.sqrt(np.mean(res(p) ** 2)))


def fit_power_law_lm(alpha: float, n_exp: int, r_max: int, relative: bool = True):
    """Levenberg-Marquardt fit of r^-alpha on r = 1..r_max, started from fit_power_law."""
    r = np.arange(1, r_max + 1, dtype=np.float64)
    x0, lam0 = fit_power_law(alpha, n_exp, r_max)
    return fit_exponentials_lm(r ** (-float(alpha)), x0, lam0, relative)


def couplings(x: np.ndarray, lam: np.ndarray, r_max: int) -> np.ndarray:
    """V(r) = sum_k x_k lam_k^r for r = 1..r_max (index r-1)."""
    r = np.arange(1, r_max + 1)
    return (x[None, :] * lam[None, :] ** r[:, None]).sum(axis=1)


def build_mpo_site(kind: int, J: float, h: float, x: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """One bulk MPO tensor W[w_left, w_right, s_out, s_in] (Sec. II C).

    Finite-state-machine layout (our reading; the paper gives only m):
    index m-1 = "nothing placed yet", index 0 = "all placed".
      W[m-1, m-1] = 1, W[0, 0] = 1, W[m-1, 0] = h F
      for term t, exponential k, channel c = 1 + t K + k:
        W[m-1, c] = A_t, W[c, c] = lam_k 1, W[c, 0] = J x_k lam_k B_t
    A string A_i ... B_j then carries J x_k lam_k^(j-i), i.e. J V(j-i).
    The chain is closed by the row vector e_{m-1} on the left and the column
    vector e_0 on the right.
    """
    terms, F = model_terms(kind)
    K = len(lam)
    m = len(terms) * K + 2
    W = np.zeros((m, m, 2, 2), dtype=np.complex128)
    W[0, 0] = ID2
    W[m - 1, m - 1] = ID2
    W[m - 1, 0] = h * F
    for t, (A, B) in enumerate(terms):
        for k in range(K):
            c = 1 + t * K + k
            W[m - 1, c] = A
            W[c, c] = lam[k] * ID2
            W[c, 0] = J * x[k] * lam[k] * B
    return W


def mpo_boundaries(m: int) -> Tuple[np.ndarray, np.ndarray]:
    """Left and right boundary environments [1, m, 1] (Fig. 3: beta_1, gamma_N trivial)."""
    left = np.zeros((1, m, 1), dtype=np.complex128)
    left[0, m - 1, 0] = 1.0
    right = np.zeros((1, m, 1), dtype=np.complex128)
    right[0, 0, 0] = 1.0
    return left, right


def mpo_to_dense(W: np.ndarray, N: int) -> np.ndarray:
    """Contract N copies of W between the boundary vectors into a 2^N x 2^N matrix."""
    m = W.shape[0]
    row = [W[m - 1, w].copy() for w in range(m)]   # operator strings after site 1
    for _ in range(1, N):
        dim = row[0].shape[0] * 2
        new = [np.zeros((dim, dim), dtype=np.complex128) for _ in range(m)]
        for w1 in range(m):
            for w2 in range(m):
                if np.any(W[w1, w2]):
                    new[w2] += np.kron(row[w1], W[w1, w2])
        row = new
    return row[0]


def site_operator(op: np.ndarray, j: int, N: int) -> np.ndarray:
    out = np.array([[1.0 + 0j]])
    for i in range(N):
        out = np.kron(out, op if i == j else ID2)
    return out


def dense_hamiltonian(kind: int, N: int, J: float, h: float, V: np.ndarray) -> np.ndarray:
    """H = sum_{i<j} J V(j-i) sum_t A_t(i) B_t(j) + h sum_i F(i) from Pauli strings.

    Built independently of the MPO (operator Kronecker products), for exact
    diagonalisation and for pinning the MPO.
    """
    terms, F = model_terms(kind)
    dim = 2 ** N
    H = np.zeros((dim, dim), dtype=np.complex128)
    ops_A = [[site_operator(A, i, N) for i in range(N)] for (A, _) in terms]
    ops_B = [[site_operator(B, i, N) for i in range(N)] for (_, B) in terms]
    for i in range(N):
        for j in range(i + 1, N):
            for t in range(len(terms)):
                H += J * V[j - i - 1] * (ops_A[t][i] @ ops_B[t][j])
        H += h * site_operator(F, i, N)
    return H
