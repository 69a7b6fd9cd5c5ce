"""Exact diagonalisation of the dense 2^N Hamiltonian (oracle pin, N <= 12).

Test infrastructure (see oracle/__init__.py): never imported by the product path.
psi(t) = U exp(-i E t) U^dagger psi0 with H = U E U^dagger from numpy's eigh.
"""
from __future__ import annotations

import numpy as np

from .models import SZ, site_operator


class ExactEvolution:
    def __init__(self, H: np.ndarray):
        Hh = 0.5 * (H + H.conj().T)
        self.E, self.U = np.linalg.eigh(Hh)

    def evolve(self, psi0: np.ndarray, t: float) -> np.ndarray:
        c = self.U.conj().T @ psi0
        return self.U @ (np.exp(-1j * self.E * t) * c)


def product_vector(states) -> np.ndarray:
    v = np.array([1.0 + 0j])
    for s in states:
        e = np.zeros(2, dtype=np.complex128)
        e[int(s)] = 1.0
        v = np.kron(v, e)
    return v


def expect_local_dense(psi: np.ndarray, op: np.ndarray, N: int) -> np.ndarray:
    out = np.empty(N)
    nrm = np.vdot(psi, psi).real
    for j in range(N):
        out[j] = np.vdot(psi, site_operator(op, j, N) @ psi).real / nrm
    return out


def expect_sz_dense(psi: np.ndarray, N: int) -> np.ndarray:
    return expect_local_dense(psi, SZ, N)
