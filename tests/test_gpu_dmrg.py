"""GPU parity of tdvp_dmrg (two-site DMRG ground states) against the oracle.

The CUDA path and the oracle run the same sweeps from the same seeded state
with the same couplings and a fixed Krylov dimension. FP64 energies must agree
to 1e-10 and observables to 1e-9: each update takes the lowest Ritz vector,
whose sensitivity to rounding grows with the inverse Ritz gap, so over tens of
updates rounding differences in the state reach ~1e-10 while the energy,
stationary at the ground state, stays at rounding level. The mixed-precision
run (3xTF32 contractions, environments included) agrees to 1e-5.
"""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import dmrg as D
from oracle import models
from oracle import mps as M
from oracle import tdvp as T
from oracle.models import ISING, XXX

from gpu_util import lib, torch_or_skip
from test_gpu_sweep import compare

pytestmark = pytest.mark.gpu


def run_pair(kind, N, alpha, J, h, K, chi, sweeps, chi0=4, kmax=12, tol=0.0, prec=0, seed=1):
    torch_or_skip()
    tdvp = lib()
    x, lam = models.fit_power_law(alpha, K, N - 1)
    W = models.build_mpo_site(kind, J, h, x, lam)
    mpo = tdvp.build_mpo(kind, N, alpha, J, h, K, x, lam)
    raw = I.random_mps_tensors(N, chi0, seed=seed)
    mps = tdvp.init_mps_tensors(raw, chi, 1e-14)
    st = tdvp.dmrg(mps, mpo, tdvp.dmrg_params(chi, krylov_max=kmax, krylov_tol=tol, precision=prec), sweeps)
    eng = T.Engine(M.canonicalize(raw, chi, 1e-14), W)
    ost = D.dmrg(eng, D.DmrgParams(chi_max=chi, krylov_max=kmax, krylov_tol=tol), sweeps)
    return tdvp, mps, mpo, eng, W, st, ost


@pytest.mark.parametrize("kind,h,alpha", [(ISING, 1.0, 3.0), (XXX, 0.0, 2.0)])
def test_dmrg_full_rank_fp64(kind, h, alpha):
    tdvp, mps, mpo, eng, W, st, ost = run_pair(kind, 10, alpha, 1.0, h, 4, 32, 3)
    assert abs(st.energy - ost.energy) < 1e-10 * abs(ost.energy)
    compare(tdvp, mps, mpo, eng, W, 1e-9)
    assert st.n_updates == 3 * 2 * 9


def test_dmrg_truncated_fp64():
    tdvp, mps, mpo, eng, W, st, ost = run_pair(ISING, 12, 2.0, 1.0, 0.8, 4, 6, 3)
    assert list(mps.bond_dims()) == eng.mps.bond_dims()
    assert abs(st.energy - ost.energy) < 1e-10 * abs(ost.energy)
    assert abs(st.w_total - ost.w_total) < 1e-12
    compare(tdvp, mps, mpo, eng, W, 1e-9)


def test_dmrg_production_krylov_reaches_ed():
    # the paper's local-solver settings (8 vectors, tolerance 1e-6) with more sweeps
    N = 10
    x, lam = models.fit_power_law(3.0, 4, N - 1)
    H = models.dense_hamiltonian(ISING, N, 1.0, 1.0, models.couplings(x, lam, N - 1))
    E0 = np.linalg.eigvalsh(0.5 * (H + H.conj().T))[0]
    tdvp, mps, mpo, eng, W, st, ost = run_pair(ISING, N, 3.0, 1.0, 1.0, 4, 32, 6, kmax=8, tol=1e-6)
    assert abs(st.energy - E0) < 1e-8 * abs(E0)
    assert abs(tdvp.energy(mps, mpo) - E0) < 1e-8 * abs(E0)


def test_dmrg_mixed_precision():
    tdvp, mps, mpo, eng, W, st, ost = run_pair(XXX, 10, 2.0, 1.0, 0.0, 4, 32, 3, prec=2)
    assert abs(st.energy - ost.energy) < 1e-5 * abs(ost.energy)
    g = tdvp.measure(mps, tdvp.OBS_SZ)
    assert np.abs(g - M.expect_sz(eng.mps)).max() < 1e-5
