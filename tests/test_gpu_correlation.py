"""GPU parity of the pieces of the dynamical correlation function of the 1/r^2
XXX quench: one-site operator application, MPS copy and mixed expectations
<a|O_j|b> against the oracle; and C(r - k, t) = e^{-i E0 t} <psi0|sz_r|psi(t)>
of the 1/r^2 XXX chain from a GPU DMRG ground state, against the oracle's run
of the same DMRG and sweep (1e-8) and against exact diagonalisation (1e-6,
set by the DMRG convergence)."""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import dmrg as D
from oracle import ed, models
from oracle import mps as M
from oracle import tdvp as T
from oracle.models import XXX, SX, SY, SZ

from gpu_util import lib, torch_or_skip

pytestmark = pytest.mark.gpu


def test_expect_mixed_copy_and_site_op():
    torch_or_skip()
    tdvp = lib()
    N = 8
    ra, rb = I.random_mps_tensors(N, 4, seed=21), I.random_mps_tensors(N, 3, seed=22)
    a, b = tdvp.init_mps_tensors(ra, 8, 1e-14), tdvp.init_mps_tensors(rb, 8, 1e-14)
    oa, ob = M.canonicalize(ra, 8, 1e-14), M.canonicalize(rb, 8, 1e-14)
    for code, op in ((tdvp.OBS_SZ, SZ), (tdvp.OBS_SX, SX), (tdvp.OBS_SY, SY)):
        assert np.abs(tdvp.expect_mixed(a, b, code) - M.mixed_local(oa, ob, op)).max() < 1e-12
    c = tdvp.mps_copy(b)
    tdvp.apply_site_op(c, 2, SY)
    ref = M.mixed_local(oa, M.apply_site_op(ob, SY, 2), SZ)
    assert np.abs(tdvp.expect_mixed(a, c, tdvp.OBS_SZ) - ref).max() < 1e-12
    # the copy is independent of its source
    assert np.abs(tdvp.expect_mixed(a, b, tdvp.OBS_SZ) - M.mixed_local(oa, ob, SZ)).max() < 1e-12
    assert abs(tdvp.norm(c) - tdvp.norm(b)) < 1e-12


def test_correlation_function_xxx():
    torch_or_skip()
    tdvp = lib()
    N, alpha, K, k, dt, n, chi = 10, 2.0, 4, 4, 0.05, 8, 32
    x, lam = models.fit_power_law(alpha, K, N - 1)
    mpo = tdvp.build_mpo(XXX, N, alpha, 1.0, 0.0, K, x, lam)
    raw = I.random_mps_tensors(N, 4, seed=0)
    gs = tdvp.init_mps_tensors(raw, chi, 1e-14)
    tdvp.dmrg(gs, mpo, tdvp.dmrg_params(chi, krylov_max=24, krylov_tol=0.0), 6)
    E0 = tdvp.energy(gs, mpo)
    psi = tdvp.mps_copy(gs)
    tdvp.apply_site_op(psi, k, SZ)
    p = tdvp.step_params(dt, chi, eps=1e-14, krylov_max=24, krylov_tol=0.0)
    tdvp.step(psi, mpo, p, n)
    t = n * dt
    C = np.exp(-1j * E0 * t) * tdvp.expect_mixed(gs, psi, tdvp.OBS_SZ)
    # the oracle: the same DMRG from the same state, the same sweep
    W = models.build_mpo_site(XXX, 1.0, 0.0, x, lam)
    eng = T.Engine(M.canonicalize(raw, chi, 1e-14), W)
    D.dmrg(eng, D.DmrgParams(chi_max=chi, krylov_max=24, krylov_tol=0.0), 6)
    ogs = eng.mps.copy()
    oE0 = M.energy(ogs, W)
    ev = T.Engine(M.apply_site_op(ogs, SZ, k), W)
    ev.step(T.Params(dt=dt, chi_max=chi, eps=1e-14, krylov_max=24, krylov_tol=0.0), n)
    oC = np.exp(-1j * oE0 * t) * M.mixed_local(ogs, ev.mps, SZ)
    assert abs(E0 - oE0) < 1e-10 * abs(oE0)
    assert np.abs(C - oC).max() < 1e-8
    # exact diagonalisation
    H = models.dense_hamiltonian(XXX, N, 1.0, 0.0, models.couplings(x, lam, N - 1))
    H = 0.5 * (H + H.conj().T)
    E, U = np.linalg.eigh(H)
    psi0 = U[:, 0]
    psi_t = ed.ExactEvolution(H).evolve(models.site_operator(SZ, k, N) @ psi0, t)
    ref = np.exp(-1j * E[0] * t) * np.array([np.vdot(psi0, models.site_operator(SZ, r, N) @ psi_t)
                                               for r in range(N)])
    assert abs(E0 - E[0]) < 1e-9 * abs(E[0])
    assert np.abs(C - ref).max() < 1e-6
