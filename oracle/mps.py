"""MPS in the inverse canonical gauge, for the oracle (Sec. II A/B).

Test infrastructure (see oracle/__init__.py): never imported by the product path.

|psi> = Psi_1 V_1 Psi_2 V_2 ... V_{N-1} Psi_N with V_j = Lambda_j^{-1} (Eq. 9).
Site tensors Psi_j have shape [chi_{j-1}, d, chi_j] (chi_0 = chi_N = 1, indices
here are 0-based: sites 0..N-1, bonds 0..N-2, bond j between sites j, j+1).
V[j] holds the diagonal of V_j as a real vector.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from .models import SX, SY, SZ


@dataclasses.dataclass
class MPS:
    Psi: List[np.ndarray]
    V: List[np.ndarray]

    @property
    def N(self) -> int:
        return len(self.Psi)

    def copy(self) -> "MPS":
        return MPS([p.copy() for p in self.Psi], [v.copy() for v in self.V])

    def bond_dims(self) -> List[int]:
        return [len(v) for v in self.V]

    def matrices(self) -> List[np.ndarray]:
        """M_j = Psi_j V_j (j < N-1) and M_N = Psi_N, so that |psi> = M_1 ... M_N."""
        out = []
        for j, P in enumerate(self.Psi):
            if j < self.N - 1:
                out.append(P * self.V[j][None, None, :])
            else:
                out.append(P)
        return out


def product_state(states: np.ndarray, d: int = 2) -> MPS:
    """Basis product state (chi = 1 everywhere, V = 1); index 0 = spin up."""
    Psi = []
    for s in states:
        t = np.zeros((1, d, 1), dtype=np.complex128)
        t[0, int(s), 0] = 1.0
        Psi.append(t)
    V = [np.ones(1) for _ in range(len(states) - 1)]
    return MPS(Psi, V)


def _truncate_count(s: np.ndarray, chi_max: int, eps: float) -> int:
    keep = int(np.count_nonzero(s > eps * s[0])) if s[0] > 0 else 1
    return max(1, min(keep, chi_max))


def canonicalize(raw: List[np.ndarray], chi_max: int, eps: float = 1e-14) -> MPS:
    """Bring raw site tensors to the inverse canonical gauge (Sec. II B) and normalise.

    A left-to-right sweep of SVDs makes every tensor left-orthonormal; a
    right-to-left sweep then yields the Schmidt values Lambda_j at every bond
    and right-orthonormal B_j, so that Psi_j = Lambda_{j-1} B_j and
    V_j = Lambda_j^{-1} (the construction described after Eq. 9). Bonds are
    cut to chi_max and to singular values above eps * lambda_1.
    The initial state must be orthonormal (Sec. III D); this provides it.
    """
    N = len(raw)
    A = [t.astype(np.complex128).copy() for t in raw]
    for j in range(N - 1):
        a, d, b = A[j].shape
        U, s, Vh = np.linalg.svd(A[j].reshape(a * d, b), full_matrices=False)
        k = _truncate_count(s, chi_max, eps)
        A[j] = U[:, :k].reshape(a, d, k)
        carry = s[:k, None] * Vh[:k]
        A[j + 1] = np.einsum("kb,bsc->ksc", carry, A[j + 1])
    nrm = np.linalg.norm(A[N - 1])
    A[N - 1] = A[N - 1] / nrm
    Psi: List[Optional[np.ndarray]] = [None] * N
    V: List[Optional[np.ndarray]] = [None] * (N - 1)
    C = A[N - 1]
    for j in range(N - 1, 0, -1):
        a, d, b = C.shape
        U, s, Vh = np.linalg.svd(C.reshape(a, d * b), full_matrices=False)
        k = _truncate_count(s, chi_max, eps)
        B = Vh[:k].reshape(k, d, b)
        Psi[j] = s[:k, None, None] * B
        V[j - 1] = 1.0 / s[:k]
        C = np.einsum("asb,bk->ask", A[j - 1], U[:, :k] * s[None, :k])
    Psi[0] = C
    return MPS(Psi, V)


# ---------------------------------------------------------------------------
# Measurement by full transfer-matrix contraction (exact in any gauge).
# ---------------------------------------------------------------------------

def _left_norm_envs(M: List[np.ndarray]) -> List[np.ndarray]:
    E = [np.ones((1, 1), dtype=np.complex128)]
    for Mj in M:
        E.append(np.einsum("asb,ax,xsy->by", Mj.conj(), E[-1], Mj))
    return E


def _right_norm_envs(M: List[np.ndarray]) -> List[np.ndarray]:
    N = len(M)
    E = [None] * (N + 1)
    E[N] = np.ones((1, 1), dtype=np.complex128)
    for j in range(N - 1, -1, -1):
        E[j] = np.einsum("asb,by,xsy->ax", M[j].conj(), E[j + 1], M[j])
    return E


def norm2(mps: MPS) -> float:
    M = mps.matrices()
    return float(_left_norm_envs(M)[-1][0, 0].real)


def expect_local(mps: MPS, op: np.ndarray) -> np.ndarray:
    """<psi|O_j|psi> / <psi|psi> for every site j (single-site observables)."""
    M = mps.matrices()
    Lf = _left_norm_envs(M)
    Rf = _right_norm_envs(M)
    nrm = Lf[-1][0, 0].real
    out = np.empty(len(M))
    for j, Mj in enumerate(M):
        val = np.einsum("asb,ax,st,xty,by->", Mj.conj(), Lf[j], op, Mj, Rf[j + 1])
        out[j] = val.real / nrm
    return out


def expect_sz(mps: MPS) -> np.ndarray:
    return expect_local(mps, SZ)


def expect_sx(mps: MPS) -> np.ndarray:
    return expect_local(mps, SX)


def expect_sy(mps: MPS) -> np.ndarray:
    return expect_local(mps, SY)


def energy(mps: MPS, W: np.ndarray) -> float:
    """<psi|H|psi>/<psi|psi> with the MPO tensor W on every site."""
    M = mps.matrices()
    m = W.shape[0]
    E = np.zeros((1, m, 1), dtype=np.complex128)
    E[0, m - 1, 0] = 1.0
    for Mj in M:
        X1 = np.einsum("awx,xty->awty", E, Mj)
        X2 = np.einsum("wvst,awty->asvy", W, X1)
        E = np.einsum("asb,asvy->bvy", Mj.conj(), X2)
    return float((E[0, 0, 0] / norm2(mps)).real)


def overlap(a: MPS, b: MPS) -> complex:
    """<a|b> by transfer matrices."""
    Ma, Mb = a.matrices(), b.matrices()
    E = np.ones((1, 1), dtype=np.complex128)
    for A, B in zip(Ma, Mb):
        E = np.einsum("asb,ax,xsy->by", A.conj(), E, B)
    return complex(E[0, 0])


def apply_site_op(mps: MPS, op: np.ndarray, j: int) -> MPS:
    """O_j |psi> with O acting on the physical index of Psi_j (the excitation
    sigma^z_k |psi_0> of the dynamical correlation function, Sec. IV). A unitary O
    keeps the inverse canonical gauge."""
    out = mps.copy()
    out.Psi[j] = np.einsum("st,atb->asb", op, mps.Psi[j])
    return out


def mixed_local(a: MPS, b: MPS, op: np.ndarray) -> np.ndarray:
    """<a|O_j|b> for every site j (complex, not normalised), by transfer
    matrices with a in the bra and b in the ket."""
    Ma, Mb = a.matrices(), b.matrices()
    N = len(Ma)
    L = [np.ones((1, 1), dtype=np.complex128)]
    for A, B in zip(Ma, Mb):
        L.append(np.einsum("asb,ax,xsy->by", A.conj(), L[-1], B))
    R = [None] * (N + 1)
    R[N] = np.ones((1, 1), dtype=np.complex128)
    for j in range(N - 1, -1, -1):
        R[j] = np.einsum("asb,by,xsy->ax", Ma[j].conj(), R[j + 1], Mb[j])
    return np.array([np.einsum("asb,ax,st,xty,by->", Ma[j].conj(), L[j], op, Mb[j], R[j + 1])
                     for j in range(N)])


def infidelity(a: MPS, b: MPS) -> float:
    """I = 1 - |<a|b>| / sqrt(<a|a><b|b>) (Eq. 24)."""
    return 1.0 - abs(overlap(a, b)) / np.sqrt(norm2(a) * norm2(b))


def from_dense(v: np.ndarray, N: int, chi_max: int, d: int = 2) -> MPS:
    """A state vector (site 0 most significant) as an MPS in the inverse canonical
    gauge: exact left-to-right SVD factorisation into raw tensors, then canonicalize."""
    raw = []
    rest = np.asarray(v, dtype=np.complex128).reshape(1, -1)
    for j in range(N - 1):
        a = rest.shape[0]
        U, s, Vh = np.linalg.svd(rest.reshape(a * d, -1), full_matrices=False)
        k = int(np.count_nonzero(s > 1e-15 * s[0]))
        raw.append(U[:, :k].reshape(a, d, k))
        rest = s[:k, None] * Vh[:k]
    raw.append(rest.reshape(rest.shape[0], d, 1))
    return canonicalize(raw, chi_max)


def to_dense(mps: MPS) -> np.ndarray:
    """State vector (site 0 most significant), for small N only."""
    M = mps.matrices()
    v = M[0].reshape(M[0].shape[1], M[0].shape[2])
    for Mj in M[1:]:
        v = np.einsum("pa,asb->psb", v, Mj).reshape(-1, Mj.shape[2])
    return v.reshape(-1)
