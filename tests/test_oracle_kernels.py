"""Pins for the oracle's local operations against dense brute force.

CPU only. H_eff is checked against X^dagger H X with the dense Hamiltonian built
from Pauli strings (independent of the MPO and of the environment code); the
Lanczos exponential against scipy's expm; the split against its definition;
measurements against a dense state vector.
"""
import numpy as np
import pytest
import scipy.linalg

import tdvp_inputs as I
from oracle import models
from oracle import mps as M
from oracle import tdvp as T
from oracle.models import ISING, XXX, XY, SX, SY, SZ


def random_state(N, chi, seed):
    return M.canonicalize(I.random_mps_tensors(N, chi, seed), chi)


def left_basis(mps, j):
    """Orthonormal basis of sites < j as columns [d^j, chi_{j-1}] from A_i = Psi_i V_i."""
    X = np.ones((1, 1), dtype=np.complex128)
    for i in range(j):
        A = mps.Psi[i] * mps.V[i][None, None, :]
        X = np.einsum("pa,asb->psb", X, A).reshape(-1, A.shape[2])
    return X


def right_basis(mps, j):
    """Orthonormal basis of sites > j as rows [chi_j, d^(N-1-j)] from B_i = V_{i-1} Psi_i."""
    N = mps.N
    Y = np.ones((1, 1), dtype=np.complex128)
    for i in range(N - 1, j, -1):
        B = mps.V[i - 1][:, None, None] * mps.Psi[i]
        Y = np.einsum("asb,bq->asq", B, Y).reshape(B.shape[0], -1)
    return Y


@pytest.mark.parametrize("kind", [ISING, XY, XXX])
def test_heff2_equals_projected_hamiltonian(kind):
    N, chi, j = 7, 5, 2
    x, lam = models.fit_power_law(1.3, 2, N - 1)
    W = models.build_mpo_site(kind, 0.9, 0.35, x, lam)
    mps = random_state(N, chi, seed=11)
    eng = T.Engine(mps, W)
    Hd = models.dense_hamiltonian(kind, N, 0.9, 0.35, models.couplings(x, lam, N - 1))
    XL = left_basis(mps, j)
    XR = right_basis(mps, j + 1)
    assert np.allclose(XL.conj().T @ XL, np.eye(XL.shape[1]), atol=1e-12)
    assert np.allclose(XR @ XR.conj().T, np.eye(XR.shape[0]), atol=1e-12)
    X = np.kron(np.kron(XL, np.eye(4)), XR.T)
    Hproj = X.conj().T @ Hd @ X
    Heff = T.heff2_dense(eng.beta[j], W, W, eng.gamma[j + 1])
    assert np.abs(Hproj - Heff).max() < 1e-12
    assert np.abs(Heff - Heff.conj().T).max() < 1e-12


def test_heff1_equals_projected_hamiltonian():
    N, chi, j = 6, 4, 3
    x, lam = models.fit_power_law(2.0, 2, N - 1)
    W = models.build_mpo_site(ISING, 1.0, 0.6, x, lam)
    mps = random_state(N, chi, seed=3)
    eng = T.Engine(mps, W)
    Hd = models.dense_hamiltonian(ISING, N, 1.0, 0.6, models.couplings(x, lam, N - 1))
    X = np.kron(np.kron(left_basis(mps, j), np.eye(2)), right_basis(mps, j).T)
    Hproj = X.conj().T @ Hd @ X
    a, b = eng.beta[j].shape[0], eng.gamma[j].shape[0]
    n = a * 2 * b
    Heff = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[i] = 1
        Heff[:, i] = T.heff1_apply(eng.beta[j], W, eng.gamma[j], e.reshape(a, 2, b)).reshape(-1)
    assert np.abs(Hproj - Heff).max() < 1e-12


def test_env_update_matches_transfer_definition():
    # Left env from an explicit sum over a (bra, ket) product basis.
    rng = np.random.default_rng(0)
    m, a, b = 4, 3, 5
    beta = rng.standard_normal((a, m, a)) + 1j * rng.standard_normal((a, m, a))
    A = rng.standard_normal((a, 2, b)) + 1j * rng.standard_normal((a, 2, b))
    W = rng.standard_normal((m, m, 2, 2)) + 1j * rng.standard_normal((m, m, 2, 2))
    out = T.env_left(beta, A, W)
    ref = np.zeros((b, m, b), dtype=np.complex128)
    for bb in range(b):
        for v in range(m):
            for bp in range(b):
                acc = 0
                for aa in range(a):
                    for w in range(m):
                        for ap in range(a):
                            for s in range(2):
                                for sp in range(2):
                                    acc += (np.conj(A[aa, s, bb]) * beta[aa, w, ap]
                                            * W[w, v, s, sp] * A[ap, sp, bp])
                ref[bb, v, bp] = acc
    assert np.abs(out - ref).max() < 1e-12
    # right env is the mirror image: reversing the chain maps one onto the other
    gam = rng.standard_normal((b, m, b)) + 1j * rng.standard_normal((b, m, b))
    Wt = W.transpose(1, 0, 2, 3)
    r1 = T.env_right(gam, A, W)
    r2 = T.env_left(gam, A.transpose(2, 1, 0), Wt)
    assert np.abs(r1 - r2).max() < 1e-12


@pytest.mark.parametrize("t", [0.05, -0.05, 0.3])
def test_lanczos_matches_expm(t):
    rng = np.random.default_rng(5)
    n = 24
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = 0.5 * (A + A.conj().T)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = scipy.linalg.expm(-1j * t * H) @ v
    y, info = T.lanczos_expm(lambda x: H @ x, v, t, kmax=16, tol=0.0)
    assert np.abs(y - ref).max() < 1e-10 * np.linalg.norm(v)
    assert info.n_vectors == 16
    y2, info2 = T.lanczos_expm(lambda x: H @ x, v, t, kmax=24, tol=1e-12)
    assert np.abs(y2 - ref).max() < 1e-9 * np.linalg.norm(v)
    assert info2.n_vectors < 24


def test_lanczos_breakdown_on_invariant_subspace():
    # H acts on a 3-dim invariant subspace containing v: exact after 3 vectors.
    H = np.diag([1.0, -2.0, 0.5, 3.0, 7.0]).astype(np.complex128)
    v = np.array([1, 1j, 0.5, 0, 0], dtype=np.complex128)
    y, info = T.lanczos_expm(lambda x: H @ x, v, 0.4, kmax=8, tol=0.0)
    assert info.breakdown and info.n_vectors == 3
    assert np.abs(y - scipy.linalg.expm(-0.4j * H) @ v).max() < 1e-13


def test_tridiag_expm_single_and_pair():
    c = T.tridiag_expm_e0(np.array([2.0]), np.array([]), 0.3)
    assert np.allclose(c, [np.exp(-0.6j)])
    c = T.tridiag_expm_e0(np.array([1.0, -1.0]), np.array([0.5]), 0.7)
    Tm = np.array([[1.0, 0.5], [0.5, -1.0]])
    assert np.allclose(c, scipy.linalg.expm(-0.7j * Tm)[:, 0], atol=1e-14)


def test_truncation_rank_rules():
    s = np.array([1.0, 0.5, 1e-3, 1e-7, 1e-13])
    # eps cut only
    assert T.truncation_rank(s, 10, 0.0, 1e-12)[0] == 4
    # chi_max cut
    chi, w = T.truncation_rank(s, 2, 0.0, 1e-12)
    assert chi == 2 and np.isclose(w, 1e-6 + 1e-14 + 1e-26)
    # discarded-weight rule (Eq. 22): smallest chi with tail weight <= w_max
    assert T.truncation_rank(s, 10, 1e-6 + 2e-14, 0.0)[0] == 2
    assert T.truncation_rank(s, 10, 1e-13, 0.0)[0] == 3
    # at least one value is kept
    assert T.truncation_rank(np.array([0.0, 0.0]), 4, 1.0, 1e-12)[0] == 1
    # numerical zeros (below 1e-14 of the norm) are dropped even at eps = 0,
    # and their weight counts as discarded
    s2 = np.array([1.0, 0.5, 2e-14, 5e-15, 0.0])
    chi, w = T.truncation_rank(s2, 10, 0.0, 0.0)
    assert chi == 3 and abs(w - 5e-15 ** 2) < 1e-40
    chi, w = T.truncation_rank(np.array([1.0, 0.5, 1e-15]), 10, 0.0, 0.0)
    assert chi == 2 and abs(w - 1e-30) < 1e-44


def test_split_reconstructs_and_orders():
    theta = I.random_complex((3, 2, 2, 4), seed=7)
    Psi_L, Vb, Psi_R, w, s = T.split_two_site(theta, 16, 0.0, 0.0)
    rec = np.einsum("asc,c,cub->asub", Psi_L, Vb, Psi_R)
    assert np.abs(rec - theta).max() < 1e-13
    assert np.all(np.diff(s) <= 0)
    # left isometry A = Psi_L V and right isometry B = V Psi_R
    A = (Psi_L * Vb[None, None, :]).reshape(-1, len(Vb))
    B = (Vb[:, None, None] * Psi_R).reshape(len(Vb), -1)
    assert np.allclose(A.conj().T @ A, np.eye(len(Vb)), atol=1e-13)
    assert np.allclose(B @ B.conj().T, np.eye(len(Vb)), atol=1e-13)
    Psi_L, Vb, Psi_R, w, s = T.split_two_site(theta, 2, 0.0, 0.0)
    assert np.isclose(w, np.sum(s[2:] ** 2))


def test_measure_matches_dense_vector():
    N = 6
    mps = random_state(N, 4, seed=21)
    # rescale a bond to make the state unnormalised and the gauge non-trivial
    mps.Psi[2] = mps.Psi[2] * 1.7
    v = M.to_dense(mps)
    nrm = np.vdot(v, v).real
    assert np.isclose(M.norm2(mps), nrm, rtol=1e-13)
    for op, fn in ((SZ, M.expect_sz), (SX, M.expect_sx), (SY, M.expect_sy)):
        ref = [np.vdot(v, models.site_operator(op, j, N) @ v).real / nrm for j in range(N)]
        assert np.abs(fn(mps) - np.array(ref)).max() < 1e-13
    x, lam = models.fit_power_law(1.5, 3, N - 1)
    W = models.build_mpo_site(XY, 1.0, 0.2, x, lam)
    Hd = models.dense_hamiltonian(XY, N, 1.0, 0.2, models.couplings(x, lam, N - 1))
    assert np.isclose(M.energy(mps, W), np.vdot(v, Hd @ v).real / nrm, rtol=1e-12)
    other = random_state(N, 4, seed=22)
    v2 = M.to_dense(other)
    assert np.isclose(M.overlap(mps, other), np.vdot(v, v2), rtol=1e-12)
    assert M.infidelity(mps, mps) < 1e-14


def test_canonicalize_gives_inverse_canonical_gauge():
    mps = random_state(8, 6, seed=2)
    assert np.isclose(M.norm2(mps), 1.0, atol=1e-13)
    for j in range(mps.N - 1):
        A = (mps.Psi[j] * mps.V[j][None, None, :]).reshape(-1, len(mps.V[j]))
        B = (mps.V[j][:, None, None] * mps.Psi[j + 1]).reshape(len(mps.V[j]), -1)
        assert np.allclose(A.conj().T @ A, np.eye(A.shape[1]), atol=1e-12)
        assert np.allclose(B @ B.conj().T, np.eye(B.shape[0]), atol=1e-12)
        assert np.all(np.diff(1.0 / mps.V[j]) <= 1e-15)


def test_apply_site_op_and_mixed_local_match_dense_vectors():
    N = 6
    a = M.canonicalize(I.random_mps_tensors(N, 4, seed=21), 8)
    b = M.canonicalize(I.random_mps_tensors(N, 3, seed=22), 8)
    va, vb = M.to_dense(a), M.to_dense(b)
    for op in (models.SZ, models.SX, models.SY):
        got = M.mixed_local(a, b, op)
        ref = np.array([np.vdot(va, models.site_operator(op, j, N) @ vb) for j in range(N)])
        assert np.abs(got - ref).max() < 1e-13
    c = M.apply_site_op(b, models.SY, 2)
    assert np.abs(M.to_dense(c) - models.site_operator(models.SY, 2, N) @ vb).max() < 1e-14
    # a unitary keeps the norm and the gauge (the state stays normalised)
    assert abs(M.norm2(c) - M.norm2(b)) < 1e-13
