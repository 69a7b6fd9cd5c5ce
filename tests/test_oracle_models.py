"""Pins for the oracle's model layer: power-law fit, MPO, dense Hamiltonian, ED.

CPU only. Each check is against something other than the oracle itself:
closed forms, the paper's printed fit errors, or an independent construction.
"""
import json
import os

import numpy as np
import pytest

from oracle import ed, models
from oracle.models import ISING, XXX, XY, SX, SZ

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fit_recovers_exact_exponential_sums():
    # Samples that ARE a sum of exponentials must be recovered exactly.
    r = np.arange(1, 41)
    for lam_true, x_true in [([0.7], [1.3]), ([0.8, 0.3], [0.5, 2.0]), ([0.9, -0.4], [1.0, 0.25])]:
        f = sum(x * l ** r for x, l in zip(x_true, lam_true))
        x, lam = models.fit_exponentials(f, len(lam_true))
        order = np.argsort(lam.real)
        assert np.allclose(lam[order], np.sort(lam_true), atol=1e-10)
        assert np.allclose(x[order], np.array(x_true)[np.argsort(lam_true)], atol=1e-9)


def test_fit_power_law_matches_paper_error_bounds():
    with open(os.path.join(HERE, "golden", "paper_fit_errors.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        x, lam = models.fit_power_law(c["alpha"], c["n_exp"], c["r_max"])
        r = np.arange(1, c["r_max"] + 1)
        f = r ** (-c["alpha"])
        V = models.couplings(x, lam, c["r_max"])
        assert np.abs(V - f).max() <= c["max_abs"], c
        if c["max_rel"] is not None:
            assert (np.abs(V - f) / f).max() <= c["max_rel"], c
        assert np.abs(V.imag).max() < 1e-12


def test_fit_pads_when_range_is_short():
    x, lam = models.fit_power_law(3.0, 8, 5)
    assert len(x) == 8 and len(lam) == 8
    V = models.couplings(x, lam, 5)
    # only two exponentials fit in 5 samples; the padded ones carry x = 0
    assert np.count_nonzero(x) == 2
    assert np.allclose(V.real, np.arange(1, 6) ** -3.0, atol=1e-3)


@pytest.mark.parametrize("kind", [ISING, XY, XXX])
def test_mpo_equals_pauli_string_hamiltonian(kind):
    N = 7
    x, lam = models.fit_power_law(1.7, 3, N - 1)
    J, h = 0.8, 0.45
    W = models.build_mpo_site(kind, J, h, x, lam)
    assert W.shape[0] == models.model_terms(kind)[0].__len__() * 3 + 2
    Hm = models.mpo_to_dense(W, N)
    Hd = models.dense_hamiltonian(kind, N, J, h, models.couplings(x, lam, N - 1))
    assert np.abs(Hm - Hd).max() < 1e-13
    assert np.abs(Hd - Hd.conj().T).max() < 1e-12


def test_mpo_catches_wrong_power():
    # A W with lam_k on the decay channel but without the closing lam_k gives
    # x_k lam_k^(r-1): it must not match the dense H (guards the exponent).
    N = 5
    x, lam = models.fit_power_law(2.0, 2, N - 1)
    W = models.build_mpo_site(ISING, 1.0, 0.0, x, lam)
    Wbad = W.copy()
    for k in range(2):
        Wbad[1 + k, 0] = x[k] * SZ
    Hd = models.dense_hamiltonian(ISING, N, 1.0, 0.0, models.couplings(x, lam, N - 1))
    assert np.abs(models.mpo_to_dense(Wbad, N) - Hd).max() > 1e-3


def test_ed_ising_h0_closed_form():
    # h = 0 Ising from |+x>^N: <sx_j(t)> = prod_{k != j} cos(2 J V(|j-k|) t)
    N = 8
    x, lam = models.fit_power_law(1.5, 4, N - 1)
    V = models.couplings(x, lam, N - 1).real
    H = models.dense_hamiltonian(ISING, N, 1.0, 0.0, V)
    ev = ed.ExactEvolution(H)
    plus = np.ones(2 ** N, dtype=np.complex128) / np.sqrt(2 ** N)
    t = 0.7
    psi = ev.evolve(plus, t)
    sx = ed.expect_local_dense(psi, SX, N)
    cf = np.array([np.prod([np.cos(2 * V[abs(j - k) - 1] * t) for k in range(N) if k != j])
                   for j in range(N)])
    assert np.abs(sx - cf).max() < 1e-12


@pytest.mark.parametrize("kind", [XY, XXX])
def test_ed_single_magnon_closed_form(kind):
    # One flipped spin in an all-down chain: an N x N hopping problem.
    N = 9
    x, lam = models.fit_power_law(1.5, 4, N - 1)
    V = models.couplings(x, lam, N - 1).real
    H = models.dense_hamiltonian(kind, N, 1.0, 0.0, V)
    H1 = single_magnon_matrix(kind, V, N)
    states = np.ones(N, dtype=int)
    states[3] = 0
    psi = ed.ExactEvolution(H).evolve(ed.product_vector(states), 0.9)
    c0 = np.zeros(N)
    c0[3] = 1.0
    e, U = np.linalg.eigh(H1)
    ct = U @ (np.exp(-1j * e * 0.9) * (U.T @ c0))
    assert np.abs(ed.expect_sz_dense(psi, N) - (-1 + 2 * np.abs(ct) ** 2)).max() < 1e-12


def single_magnon_matrix(kind, V, N):
    """Closed-form one-magnon Hamiltonian (textbook): XY hops with 2V(r);
    XXX hops with V(r)/2 and carries the Ising diagonal of S^z S^z."""
    H1 = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            if i != j:
                H1[i, j] = (2.0 if kind == XY else 0.5) * V[abs(i - j) - 1]
    if kind == XXX:
        E0 = 0.25 * sum(V[abs(i - j) - 1] for i in range(N) for j in range(i + 1, N))
        for j in range(N):
            H1[j, j] = E0 - 0.5 * sum(V[abs(j - k) - 1] for k in range(N) if k != j)
    return H1


def test_lm_fit_recovers_exact_exponential_sums():
    r = np.arange(1, 61, dtype=float)
    x = np.array([0.7, -0.2, 0.05])
    lam = np.array([0.9, 0.6, 0.3])
    f = (x[None, :] * lam[None, :] ** r[:, None]).sum(1)
    for relative in (False, True):
        xf, lf, rms = models.fit_exponentials_lm(f, x * 1.05, lam * 0.98, relative)
        assert rms < 1e-11
        order = np.argsort(-lf.real)
        assert np.allclose(lf.real[order], lam, atol=1e-8) and np.allclose(xf.real[order], x, atol=1e-8)


def test_lm_fit_improves_on_the_shift_invariance_start():
    # the Supplemental Material's comparison: 1/r^2 on r = 1..200 with 9 exponentials;
    # the relative least-squares fit holds over a longer distance (smaller relative error)
    alpha, K, R = 2.0, 9, 200
    r = np.arange(1, R + 1, dtype=float)
    f = r ** -alpha
    x0, l0 = models.fit_power_law(alpha, K, R)
    e0 = (x0[None, :] * l0[None, :] ** r[:, None]).sum(1).real - f
    for relative in (False, True):
        x, lam, rms = models.fit_power_law_lm(alpha, K, R, relative)
        e = (x[None, :] * lam[None, :] ** r[:, None]).sum(1).real - f
        w = 1 / f if relative else np.ones(R)
        assert np.sqrt(np.mean((w * e) ** 2)) <= np.sqrt(np.mean((w * e0) ** 2)) + 1e-18
        assert abs(rms - np.sqrt(np.mean((w * e) ** 2))) < 1e-15
        assert np.all(np.abs(lam) < 1)
    x, lam, _ = models.fit_power_law_lm(alpha, K, R, True)
    e = (x[None, :] * lam[None, :] ** r[:, None]).sum(1).real - f
    assert np.abs(e / f).max() < 0.5 * np.abs(e0 / f).max()
