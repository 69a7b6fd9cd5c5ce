"""Pin for the dynamical correlation function of the 1/r^2 XXX chain (the quantity of the 201-site quench).

CPU only. C(r, t) = e^{-i E0 t} <psi0| sigma^z_r |psi(t)>, |psi(t)> = e^{-iHt} sigma^z_k |psi0>
(Sec. IV, Eq. of the Haldane-Shastry comparison), from the oracle's sweep at full rank started
at the exact ground state, against the same expression with the dense Hamiltonian.
"""
import numpy as np

from oracle import ed, models
from oracle import mps as M
from oracle import tdvp as T
from oracle.models import XXX, SZ


def test_correlation_full_rank_matches_ed():
    N, alpha, K, k, dt, n = 8, 2.0, 4, 3, 0.05, 8
    x, lam = models.fit_power_law(alpha, K, N - 1)
    W = models.build_mpo_site(XXX, 1.0, 0.0, x, lam)
    H = models.dense_hamiltonian(XXX, N, 1.0, 0.0, models.couplings(x, lam, N - 1))
    H = 0.5 * (H + H.conj().T)
    E, U = np.linalg.eigh(H)
    assert E[1] - E[0] > 1e-3                      # non-degenerate ground state
    psi0 = U[:, 0]
    gs = M.from_dense(psi0, N, 16)
    assert abs(M.energy(gs, W) - E[0]) < 1e-12
    exc = M.apply_site_op(gs, SZ, k)
    eng = T.Engine(exc.copy(), W)
    p = T.Params(dt=dt, chi_max=16, eps=1e-14, krylov_max=24, krylov_tol=0.0)
    eng.step(p, n)
    t = n * dt
    C = np.exp(-1j * E[0] * t) * M.mixed_local(gs, eng.mps, SZ)
    ev = ed.ExactEvolution(H)
    psi_t = ev.evolve(models.site_operator(SZ, k, N) @ psi0, t)
    ref = np.exp(-1j * E[0] * t) * np.array([np.vdot(psi0, models.site_operator(SZ, r, N) @ psi_t)
                                               for r in range(N)])
    assert np.abs(C - ref).max() < 1e-9
    # at t = 0 it is the static correlation <sz_r sz_k>, real, 1 on the diagonal
    C0 = M.mixed_local(gs, exc, SZ)
    assert abs(C0[k] - 1.0) < 1e-12 and np.abs(C0.imag).max() < 1e-12
