"""Pins for the oracle's derivative d<O_j(t)>/d(h, J) of the TDVP evolution.

CPU only. The forward-mode derivative of oracle/grad.py is pinned three ways,
none of which re-derives it:
  * its forward values equal those of the numpy sweep of oracle/tdvp.py
    (itself pinned against exact diagonalisation), with the same kept ranks;
  * it equals central finite differences of the numpy sweep (step 1e-5) at
    fixed truncation, on a truncated run with and without segments;
  * at full rank it equals the exact derivative of <psi(t)|O_j|psi(t)> for the
    dense 2^N Hamiltonian, computed with the Frechet derivative of the matrix
    exponential (scipy.linalg.expm_frechet).
"""
import numpy as np
import pytest
import scipy.linalg

import tdvp_inputs as I
from oracle import ed, models
from oracle import grad as G
from oracle import mps as M
from oracle import tdvp as T
from oracle.models import ISING, XY, SX, SZ


def setup(kind, N, alpha, K, chi0, chi, seed):
    x, lam = models.fit_power_law(alpha, K, N - 1)
    mps0 = M.canonicalize(I.random_mps_tensors(N, chi0, seed=seed), chi, 1e-14)
    return x, lam, mps0


def numpy_run(kind, x, lam, J, h, mps0, p, n_steps, op=SZ):
    eng = T.Engine(mps0.copy(), models.build_mpo_site(kind, J, h, x, lam))
    eng.step(p, n_steps)
    return M.expect_local(eng.mps, op), eng


def test_forward_matches_numpy_sweep():
    kind, J, h = ISING, 1.0, 0.7
    x, lam, mps0 = setup(kind, 8, 2.0, 4, 3, 6, seed=11)
    p = T.Params(dt=0.05, chi_max=6, eps=1e-12, krylov_max=24, krylov_tol=0.0)
    ref, eng = numpy_run(kind, x, lam, J, h, mps0, p, 3)
    val, jac, ranks = G.jacobian(kind, x, lam, J, h, mps0, p, 3)
    assert np.abs(val - ref).max() < 1e-11
    assert eng.mps.bond_dims() == G.final_dims(ranks, 7, mps0.bond_dims())
    assert jac.shape == (8, 2) and np.all(np.isfinite(jac))


@pytest.mark.parametrize("kind,seg,obs", [(ISING, None, "z"), (ISING, [4, 4], "x"), (XY, [3, 5], "z")])
def test_jacobian_matches_central_differences(kind, seg, obs):
    J, h = 1.0, 0.6
    x, lam, mps0 = setup(kind, 8, 2.5, 3, 3, 6, seed=5)
    p = T.Params(dt=0.04, chi_max=6, eps=1e-12, krylov_max=24, krylov_tol=0.0, seg_len=seg)
    n = 3
    op = {"z": SZ, "x": SX}[obs]
    val, jac, ranks = G.jacobian(kind, x, lam, J, h, mps0, p, n, obs)
    kept = [r for _, r in ranks]
    assert max(kept) == 6 and G.final_dims(ranks, 7, mps0.bond_dims())[3] == 6   # truncation active (full: 16)
    d = 1e-5
    fd = np.zeros_like(jac)
    for c, (dh, dJ) in enumerate(((d, 0.0), (0.0, d))):
        plus, ep = numpy_run(kind, x, lam, J + dJ, h + dh, mps0, p, n, op)
        minus, em = numpy_run(kind, x, lam, J - dJ, h - dh, mps0, p, n, op)
        assert ep.mps.bond_dims() == em.mps.bond_dims()      # fixed truncation
        fd[:, c] = (plus - minus) / (2 * d)
    scale = np.abs(jac).max()
    assert scale > 1e-3
    assert np.abs(jac - fd).max() < 1e-7 * scale


@pytest.mark.parametrize("kind,h", [(ISING, 0.8), (XY, 0.3)])
def test_full_rank_jacobian_is_the_exact_derivative(kind, h):
    N, J, t_steps, dt = 6, 1.0, 4, 0.05
    x, lam, mps0 = setup(kind, N, 2.0, 3, 8, 8, seed=2)
    p = T.Params(dt=dt, chi_max=8, eps=1e-14, krylov_max=24, krylov_tol=0.0)
    val, jac, _ = G.jacobian(kind, x, lam, J, h, mps0, p, t_steps)
    V = models.couplings(x, lam, N - 1)
    H = models.dense_hamiltonian(kind, N, J, h, V)
    dH = [models.dense_hamiltonian(kind, N, 0.0, 1.0, V), models.dense_hamiltonian(kind, N, 1.0, 0.0, V)]
    t = t_steps * dt
    psi0 = M.to_dense(mps0)
    psi0 = psi0 / np.linalg.norm(psi0)
    exact_val = None
    for c in range(2):
        E, L = scipy.linalg.expm_frechet(-1j * t * H, -1j * t * dH[c])
        psi, dpsi = E @ psi0, L @ psi0
        O = [models.site_operator(SZ, j, N) for j in range(N)]
        exact_val = np.array([np.vdot(psi, Oj @ psi).real for Oj in O])
        exact_d = np.array([2 * np.vdot(psi, Oj @ dpsi).real for Oj in O])
        assert np.abs(jac[:, c] - exact_d).max() < 1e-9
    assert np.abs(val - exact_val).max() < 1e-10
