"""Pins for the oracle's two-site DMRG (ground-state) mode.

CPU only. The tridiagonal eigenpair is checked against the closed form of the
path-graph matrix; the Lanczos ground state against dense diagonalisation of
an explicit effective Hamiltonian; the sweeps against exact diagonalisation of
the full 2^N Hamiltonian (N = 10, bonds at full rank) and against the
variational bound when truncated.
"""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import dmrg as D
from oracle import models
from oracle import mps as M
from oracle import tdvp as T
from oracle.models import ISING, XXX


def test_tridiag_ground_closed_form():
    # tridiag(b, a, b) of size k: eigenvalues a + 2b cos(pi j / (k + 1)), eigenvectors sin(pi i j / (k + 1))
    for k in (1, 2, 5, 12):
        a, b = 0.3, -0.7
        e, z = D.tridiag_ground(np.full(k, a), np.full(k - 1, b))
        j = 1 if b < 0 else k
        assert abs(e - (a + 2 * b * np.cos(np.pi * j / (k + 1)))) < 1e-13
        ref = np.sin(np.pi * np.arange(1, k + 1) * j / (k + 1))
        ref /= np.linalg.norm(ref)
        assert abs(abs(np.dot(z, ref)) - 1.0) < 1e-12


def _small_heff(seed):
    x, lam = models.fit_power_law(2.0, 3, 9)
    W = models.build_mpo_site(ISING, 1.0, 0.7, x, lam)
    m, d, a, b = W.shape[0], 2, 3, 4
    rng = np.random.default_rng(seed)

    def herm(shape):
        X = I.random_complex(shape, int(rng.integers(1 << 30)))
        return 0.5 * (X + np.conj(np.transpose(X, (2, 1, 0))))
    L, R = herm((a, m, a)), herm((b, m, b))
    return W, L, R, (a, d, d, b)


def test_lanczos_ground_full_krylov_is_exact():
    W, L, R, shape = _small_heff(3)
    H = T.heff2_dense(L, W, W, R)
    H = 0.5 * (H + H.conj().T)
    E, U = np.linalg.eigh(H)
    th = I.random_complex(shape, 4)
    y, info = D.lanczos_ground(lambda v: T.heff2_apply(L, W, W, R, v), th, kmax=H.shape[0], tol=0.0)
    v = y.reshape(-1)
    assert abs(info.energy - E[0]) < 1e-10
    assert abs(np.linalg.norm(v) - np.linalg.norm(th)) < 1e-12      # norm of the input kept
    assert abs(abs(np.vdot(U[:, 0], v)) - np.linalg.norm(v)) < 1e-8   # the ground state, up to a phase
    r = H @ v - info.energy * v
    assert np.linalg.norm(r) < 1e-8 * np.linalg.norm(v)


def test_lanczos_ground_ritz_value_is_variational():
    W, L, R, shape = _small_heff(5)
    H = T.heff2_dense(L, W, W, R)
    E0 = np.linalg.eigvalsh(0.5 * (H + H.conj().T))[0]
    th = I.random_complex(shape, 6)
    prev = np.inf
    for k in range(1, 8):
        _, info = D.lanczos_ground(lambda v: T.heff2_apply(L, W, W, R, v), th, kmax=k, tol=0.0)
        assert info.energy >= E0 - 1e-12
        assert info.energy <= prev + 1e-12          # Ritz values decrease with the Krylov dimension
        prev = info.energy


@pytest.mark.parametrize("kind,h,alpha", [(ISING, 1.0, 3.0), (XXX, 0.0, 2.0)])
def test_dmrg_matches_ed_ground_energy(kind, h, alpha):
    N = 10
    x, lam = models.fit_power_law(alpha, 4, N - 1)
    W = models.build_mpo_site(kind, 1.0, h, x, lam)
    H = models.dense_hamiltonian(kind, N, 1.0, h, models.couplings(x, lam, N - 1))
    E = np.linalg.eigvalsh(0.5 * (H + H.conj().T))
    state = M.canonicalize(I.random_mps_tensors(N, 4, seed=1), 32)
    eng = T.Engine(state, W)
    st = D.dmrg(eng, D.DmrgParams(chi_max=32, krylov_max=12, krylov_tol=0.0), 4)
    nrm = M.norm2(eng.mps)
    assert abs(st.energy - E[0]) < 1e-9 * abs(E[0])
    # the Ritz value is the energy of the state the sweep leaves behind
    assert abs(M.energy(eng.mps, W) - st.energy) < 1e-9 * abs(E[0])
    assert abs(nrm - 1.0) < 1e-12


def test_dmrg_truncated_is_variational_and_converges():
    N = 10
    x, lam = models.fit_power_law(3.0, 4, N - 1)
    W = models.build_mpo_site(ISING, 1.0, 1.0, x, lam)
    H = models.dense_hamiltonian(ISING, N, 1.0, 1.0, models.couplings(x, lam, N - 1))
    E0 = np.linalg.eigvalsh(0.5 * (H + H.conj().T))[0]
    eng = T.Engine(M.canonicalize(I.random_mps_tensors(N, 2, seed=2), 4), W)
    st = D.dmrg(eng, D.DmrgParams(chi_max=4, krylov_max=10, krylov_tol=0.0), 6)
    es = np.array(st.energies)
    assert np.all(es >= E0 - 1e-12)
    assert es[-1] - E0 < 1e-3 * abs(E0)        # chi = 4 is close for this gapped chain
    assert abs(es[-1] - es[-2]) < 1e-8 * abs(E0)
