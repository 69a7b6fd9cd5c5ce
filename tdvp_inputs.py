"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds workload definitions (model parameters, chain partitions,
time-step settings) and seeded random-number draws only. It contains none of
the method's arithmetic: no MPO construction, no coupling fit, no contraction,
no decomposition. Both the CPU oracle and the CUDA library receive what this
module produces as plain arrays and numbers.

The workloads are synthetic quenches shaped like the paper's long-range spin
chains (Sec. IV): the transverse-field Ising chain (Sec. IV A), the XY chain
(Sec. IV B) and the 1/r^2 Heisenberg (XXX) chain (Sec. IV C).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

# model kinds (same integer codes as the C-ABI header)
ISING = 0
XY = 1
XXX = 2

# precision codes (same integer codes as the C-ABI header)
FP64 = 0
TF32 = 1
TF32X3 = 2


@dataclasses.dataclass
class Model:
    """A long-range spin-1/2 chain H = sum_{i<j} J f(j-i) sum_t A_t(i) B_t(j) + h sum_i F(i).

    f(r) = 1/r^alpha is approximated by n_exp exponentials (Sec. II C), so the MPO
    bond dimension is m = n_terms * n_exp + 2.
    kind: ISING (terms sz.sz, field sx), XY (sx.sx + sy.sy), XXX (S.S with S = sigma/2).
    """
    kind: int
    N: int
    alpha: float
    J: float
    h: float
    n_exp: int

    @property
    def n_terms(self) -> int:
        return {ISING: 1, XY: 2, XXX: 3}[self.kind]

    @property
    def m(self) -> int:
        return self.n_terms * self.n_exp + 2


@dataclasses.dataclass
class StepParams:
    dt: float
    chi_max: int
    w_max: float = 0.0
    eps: float = 1e-12
    krylov_max: int = 8
    krylov_tol: float = 1e-6
    precision: int = FP64
    seg_len: Optional[List[int]] = None  # None or [N] -> one segment (serial)
    merge_turning: int = 1


@dataclasses.dataclass
class Workload:
    name: str
    model: Model
    params: StepParams
    n_steps: int
    init: str          # "all_up", "neel" or "random"
    chi_init: int = 1  # bond dimension of a random initial state
    seed: int = 0


def basis_state(kind: str, N: int) -> np.ndarray:
    """Product-state occupation list; basis index 0 is spin up (sigma^z = +1)."""
    if kind == "all_up":
        return np.zeros(N, dtype=np.int32)
    if kind == "all_down":
        return np.ones(N, dtype=np.int32)
    if kind == "neel":
        return (np.arange(N) % 2).astype(np.int32)
    raise ValueError(kind)


def single_flip(N: int, site: int, background: int = 1) -> np.ndarray:
    """All spins in `background` except one flipped spin at `site`."""
    s = np.full(N, background, dtype=np.int32)
    s[site] = 1 - background
    return s


def bond_dims(N: int, chi: int, d: int = 2) -> List[int]:
    """Bond dimensions chi_j (j = 0..N-2) of a saturated MPS capped at chi:
    chi_j = min(chi, d^(j+1), d^(N-1-j))."""
    out = []
    for j in range(N - 1):
        left = j + 1
        right = N - 1 - j
        c = chi
        for e in (left, right):
            c = min(c, d ** min(e, 60))
        out.append(int(c))
    return out


def random_mps_tensors(N: int, chi: int, seed: int, d: int = 2) -> List[np.ndarray]:
    """Seeded complex-Gaussian site tensors [chi_{j-1}, d, chi_j] (boundary dims 1)."""
    rng = np.random.default_rng(seed)
    dims = [1] + bond_dims(N, chi, d) + [1]
    out = []
    for j in range(N):
        shape = (dims[j], d, dims[j + 1])
        t = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        out.append(np.ascontiguousarray(t, dtype=np.complex128))
    return out


def random_complex(shape: Sequence[int], seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)


def random_real(shape: Sequence[int], seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape).astype(np.float64)


def even_partition(N: int, p: int) -> List[int]:
    base = N // p
    extra = N - base * p
    return [base + (1 if k < extra else 0) for k in range(p)]


# ---------------------------------------------------------------------------
# The five workloads. Partitions for p > 1 are the paper's own uneven ones
# (Supplemental Material, partition tables) where the sizes match.
# ---------------------------------------------------------------------------

def tfim_n10_quench() -> Workload:
    """Long-range TFIM, N=10, alpha=3, J=1, h=1, 4 exponentials (m=6), all up,
    dt=0.01 x 100, chi_max=32 (no truncation), one segment, FP64."""
    return Workload(
        name="tfim_n10_a3_m6_chi32_p1",
        model=Model(ISING, 10, 3.0, 1.0, 1.0, 4),
        params=StepParams(dt=0.01, chi_max=32, eps=1e-12, seg_len=None),
        n_steps=100, init="all_up")


def xy_n51_quench() -> Workload:
    """Long-range XY, N=51, alpha=1.5, 6 exponentials (m=14), Neel start,
    dt=0.02 x 200, chi_max=128, relative cutoff 1e-10, 4 segments 13/13/13/12."""
    return Workload(
        name="xy_n51_a1.5_m14_chi128_p4",
        model=Model(XY, 51, 1.5, 1.0, 0.0, 6),
        params=StepParams(dt=0.02, chi_max=128, eps=1e-10, seg_len=[13, 13, 13, 12]),
        n_steps=200, init="neel")


def tfim_n101_quench(precision: int = TF32X3) -> Workload:
    """Long-range TFIM, N=101, alpha=1.5, J=1, h=0.5, 8 exponentials (m=10),
    dt=0.01, chi_max=256, 8 segments 15 / 12 x 6 / 14 (the paper's 101-site
    partition), contractions in TF32 / 3xTF32 or FP64."""
    return Workload(
        name="tfim_n101_a1.5_m10_chi256_p8",
        model=Model(ISING, 101, 1.5, 1.0, 0.5, 8),
        params=StepParams(dt=0.01, chi_max=256, eps=1e-12,
                          seg_len=[15, 12, 12, 12, 12, 12, 12, 14], precision=precision),
        n_steps=300, init="all_up")


def tfim_n41_derivative() -> Workload:
    return Workload(
        name="tfim_n41_a3_m8_chi64_p1",
        model=Model(ISING, 41, 3.0, 1.0, 1.0, 6),
        params=StepParams(dt=0.02, chi_max=64, eps=1e-12),
        n_steps=100, init="all_up")


def xxx_n201_quench() -> Workload:
    return Workload(
        name="xxx_n201_a2_m32_chi256_p16",
        model=Model(XXX, 201, 2.0, 1.0, 0.0, 10),
        params=StepParams(dt=0.05, chi_max=256, eps=1e-12,
                          seg_len=[65, 12] + [4] * 12 + [12, 64],
                          precision=TF32X3),
        n_steps=400, init="random", chi_init=16, seed=0)
