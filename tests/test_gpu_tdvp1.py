"""GPU parity of the one-site TDVP step (tdvp_step1, serial and segmented) and
the hybrid scheme (tdvp_step_hybrid) against the oracle (oracle/tdvp1.py,
pinned in test_oracle_tdvp1.py): the same FP64 sweep with a fixed Krylov
dimension, so observables agree to 1e-10; at full rank both are the exact
evolution."""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import ed, models
from oracle import mps as M
from oracle import tdvp as T
from oracle import tdvp1 as T1
from oracle.models import ISING, XY

from gpu_util import lib, torch_or_skip
from test_gpu_sweep import compare

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,h,N,chi0,chi", [(ISING, 0.6, 10, 4, 4), (XY, 0.2, 9, 3, 6)])
def test_one_site_matches_oracle(kind, h, N, chi0, chi):
    torch_or_skip()
    tdvp = lib()
    x, lam = models.fit_power_law(2.0, 4, N - 1)
    W = models.build_mpo_site(kind, 1.0, h, x, lam)
    mpo = tdvp.build_mpo(kind, N, 2.0, 1.0, h, 4, x, lam)
    raw = I.random_mps_tensors(N, chi0, seed=7)
    mps = tdvp.init_mps_tensors(raw, chi, 1e-14)
    eng = T.Engine(M.canonicalize(raw, chi, 1e-14), W)
    dims = list(mps.bond_dims())
    assert dims == eng.mps.bond_dims()
    p = tdvp.step_params(0.05, chi, eps=0.0, krylov_max=24, krylov_tol=0.0)
    tdvp.step1(mps, mpo, p, 4)
    T1.step1(eng, T.Params(dt=0.05, chi_max=chi, eps=0.0, krylov_max=24, krylov_tol=0.0), 4)
    assert list(mps.bond_dims()) == dims == eng.mps.bond_dims()
    compare(tdvp, mps, mpo, eng, W, 1e-10)


def test_one_site_full_rank_is_exact():
    torch_or_skip()
    tdvp = lib()
    N = 8
    x, lam = models.fit_power_law(3.0, 4, N - 1)
    mpo = tdvp.build_mpo(ISING, N, 3.0, 1.0, 0.7, 4, x, lam)
    H = models.dense_hamiltonian(ISING, N, 1.0, 0.7, models.couplings(x, lam, N - 1))
    raw = I.random_mps_tensors(N, 16, seed=3)
    mps = tdvp.init_mps_tensors(raw, 16, 1e-14)
    v0 = M.to_dense(M.canonicalize(raw, 16, 1e-14))
    tdvp.step1(mps, mpo, tdvp.step_params(0.05, 16, eps=0.0, krylov_max=24, krylov_tol=0.0), 6)
    ref = ed.ExactEvolution(H).evolve(v0, 0.3)
    want = np.array([np.vdot(ref, models.site_operator(models.SZ, j, N) @ ref).real for j in range(N)])
    assert np.abs(tdvp.measure(mps, tdvp.OBS_SZ) - want).max() < 1e-9


@pytest.mark.parametrize("seg", [None, [4, 4]], ids=["serial", "segments"])
def test_hybrid_matches_oracle(seg):
    torch_or_skip()
    tdvp = lib()
    N, chi = 8, 4
    x, lam = models.fit_power_law(3.0, 4, N - 1)
    W = models.build_mpo_site(ISING, 1.0, 1.0, x, lam)
    mpo = tdvp.build_mpo(ISING, N, 3.0, 1.0, 1.0, 4, x, lam)
    up = I.basis_state("all_up", N)
    mps = tdvp.init_mps(N, up, chi)
    eng = T.Engine(M.product_state(up), W)
    n1 = tdvp.step_hybrid(mps, mpo, tdvp.step_params(0.05, chi, krylov_max=24, krylov_tol=0.0, seg_len=seg), 12)
    on1 = T1.step_hybrid(eng, T.Params(dt=0.05, chi_max=chi, krylov_max=24, krylov_tol=0.0, seg_len=seg), 12)
    assert n1 == on1 and 0 < n1 < 12
    assert list(mps.bond_dims()) == eng.mps.bond_dims()
    compare(tdvp, mps, mpo, eng, W, 1e-10)


@pytest.mark.parametrize("seg", [[5, 5], [3, 3, 4], [2, 3, 2, 3]])
def test_segmented_one_site_matches_oracle(seg):
    """tdvp_step1 with segments (one-site sweeps inside the segments, two-site
    boundary pairs at the bonds' current dimension, all segments of a stage
    batched) against the oracle's step1_segmented, below full rank."""
    torch_or_skip()
    tdvp = lib()
    N, chi = 10, 4
    x, lam = models.fit_power_law(2.0, 4, N - 1)
    W = models.build_mpo_site(ISING, 1.0, 0.6, x, lam)
    mpo = tdvp.build_mpo(ISING, N, 2.0, 1.0, 0.6, 4, x, lam)
    raw = I.random_mps_tensors(N, chi, seed=7)
    mps = tdvp.init_mps_tensors(raw, chi, 1e-14)
    eng = T.Engine(M.canonicalize(raw, chi, 1e-14), W)
    dims = list(mps.bond_dims())
    p = tdvp.step_params(0.05, chi, krylov_max=24, krylov_tol=0.0, seg_len=seg)
    st = tdvp.step1(mps, mpo, p, 4)
    T1.step1_segmented(eng, T.Params(dt=0.05, chi_max=chi, krylov_max=24, krylov_tol=0.0, seg_len=seg), 4)
    assert list(mps.bond_dims()) == dims == eng.mps.bond_dims()
    assert st.n_fwd2 > 0
    compare(tdvp, mps, mpo, eng, W, 1e-10)


def test_segmented_one_site_full_rank_is_exact():
    torch_or_skip()
    tdvp = lib()
    N = 8
    x, lam = models.fit_power_law(3.0, 4, N - 1)
    mpo = tdvp.build_mpo(ISING, N, 3.0, 1.0, 0.7, 4, x, lam)
    H = models.dense_hamiltonian(ISING, N, 1.0, 0.7, models.couplings(x, lam, N - 1))
    raw = I.random_mps_tensors(N, 16, seed=3)
    v0 = M.to_dense(M.canonicalize(raw, 16, 1e-14))
    ref = ed.ExactEvolution(H).evolve(v0, 0.3)
    want = np.array([np.vdot(ref, models.site_operator(models.SZ, j, N) @ ref).real for j in range(N)])
    for seg in ([4, 4], [2, 2, 2, 2]):
        mps = tdvp.init_mps_tensors(raw, 16, 1e-14)
        tdvp.step1(mps, mpo, tdvp.step_params(0.05, 16, krylov_max=24, krylov_tol=0.0, seg_len=seg), 6)
        assert np.abs(tdvp.measure(mps, tdvp.OBS_SZ) - want).max() < 1e-9, seg
        assert abs(tdvp.norm(mps) - 1.0) < 1e-11
