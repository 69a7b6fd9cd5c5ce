"""Parity of the CUDA sweep with the oracle at the sizes the workloads name.

* The 10-site Ising quench (alpha = 3, J = h = 1, 4 exponentials, all up,
  dt = 0.01, chi_max = 32 = full rank) for its whole run of 100 steps: the
  FP64 GPU path against the oracle's sweep (1e-10) and against exact
  diagonalisation of the same fitted 1024 x 1024 Hamiltonian, every 10 steps.
* The 51-site XY quench (alpha = 1.5, 6 exponentials, m = 14, Neel start,
  dt = 0.02, chi_max = 128, relative cutoff 1e-10, segments 13/13/13/12; the
  shape of Sec. IV B) for as many steps as the oracle finishes in about a
  minute: all three spin components, the norm and the energy after every step
  at 1e-10, with bond dimensions reaching chi_max.
* The mixed-precision path against the FP64 GPU path on a 41-site Ising chain
  with every bond at chi = 64 and 8 segments, after each of 20 steps:
  <sigma^z_j> within 1e-5, the accuracy the mixed path is held to.
Both sides use a fixed Krylov dimension (10 vectors, tolerance 0) where the
comparison with the oracle is at 1e-10, so that they take the same number of Lanczos steps.
"""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import ed
from oracle import models
from oracle import mps as M
from oracle import tdvp as T

from gpu_util import lib, torch_or_skip

pytestmark = pytest.mark.gpu


def _compare_all(tdvp, mps, mpo, omps, W, tol):
    errs = {}
    for obs, fn in ((tdvp.OBS_SZ, M.expect_sz), (tdvp.OBS_SX, M.expect_sx), (tdvp.OBS_SY, M.expect_sy)):
        errs[obs] = float(np.abs(tdvp.measure(mps, obs) - fn(omps)).max())
    errs["norm"] = abs(tdvp.norm(mps) - M.norm2(omps))
    e_ref = M.energy(omps, W)
    errs["energy"] = abs(tdvp.energy(mps, mpo) - e_ref) / max(1.0, abs(e_ref))
    bad = {k: v for k, v in errs.items() if not v < tol}
    assert not bad, bad
    return errs


def test_tfim_n10_full_run_matches_oracle_and_ed():
    torch_or_skip()
    tdvp = lib()
    w = I.tfim_n10_quench()
    m, prm = w.model, w.params
    N = m.N
    x, lam = models.fit_power_law(m.alpha, m.n_exp, N - 1)
    W = models.build_mpo_site(m.kind, m.J, m.h, x, lam)
    H = models.dense_hamiltonian(m.kind, N, m.J, m.h, models.couplings(x, lam, N - 1))
    exact = ed.ExactEvolution(H)
    st = I.basis_state(w.init, N)
    v0 = ed.product_vector(st)
    mpo = tdvp.build_mpo(m.kind, N, m.alpha, m.J, m.h, m.n_exp, x, lam)
    mps = tdvp.init_mps(N, st, prm.chi_max)
    eng = T.Engine(M.product_state(st), W)
    p = tdvp.step_params(dt=prm.dt, chi_max=prm.chi_max, eps=prm.eps, krylov_max=10, krylov_tol=0.0)
    op = T.Params(dt=prm.dt, chi_max=prm.chi_max, eps=prm.eps, krylov_max=10, krylov_tol=0.0)
    e0 = tdvp.energy(mps, mpo)
    assert w.n_steps == 100
    for k in range(1, w.n_steps // 10 + 1):
        tdvp.step(mps, mpo, p, 10)
        eng.step(op, 10)
        _compare_all(tdvp, mps, mpo, eng.mps, W, 1e-10)
        ref = ed.expect_sz_dense(exact.evolve(v0, 10 * k * prm.dt), N)
        assert np.abs(tdvp.measure(mps, tdvp.OBS_SZ) - ref).max() < 1e-9, k
        # full rank: the integrator is exact, the norm and energy are kept to rounding
        assert abs(tdvp.norm(mps) - 1.0) < 1e-12
        assert abs(tdvp.energy(mps, mpo) - e0) < 1e-9
    assert list(mps.bond_dims()) == eng.mps.bond_dims()


def test_xy_n51_matches_oracle_at_full_size():
    torch_or_skip()
    tdvp = lib()
    w = I.xy_n51_quench()
    m, prm = w.model, w.params
    N = m.N
    x, lam = models.fit_power_law(m.alpha, m.n_exp, N - 1)
    W = models.build_mpo_site(m.kind, m.J, m.h, x, lam)
    st = I.basis_state(w.init, N)
    mpo = tdvp.build_mpo(m.kind, N, m.alpha, m.J, m.h, m.n_exp, x, lam)
    mps = tdvp.init_mps(N, st, prm.chi_max)
    eng = T.Engine(M.product_state(st), W)
    p = tdvp.step_params(dt=prm.dt, chi_max=prm.chi_max, w_max=prm.w_max, eps=prm.eps, krylov_max=10,
                         krylov_tol=0.0, seg_len=prm.seg_len)
    op = T.Params(dt=prm.dt, chi_max=prm.chi_max, w_max=prm.w_max, eps=prm.eps, krylov_max=10, krylov_tol=0.0,
                  seg_len=prm.seg_len)
    w_gpu = 0.0
    for k in range(3):
        stt = tdvp.step(mps, mpo, p, 1)
        w_gpu += stt.w_total
        eng.step(op, 1)
        _compare_all(tdvp, mps, mpo, eng.mps, W, 1e-10)
        assert list(mps.bond_dims()) == eng.mps.bond_dims(), k
    assert max(mps.bond_dims()) == prm.chi_max
    assert abs(w_gpu - eng.stats.w_total) < 1e-10 * max(1.0, eng.stats.w_total)


def test_mixed_precision_series_stays_within_1e5_of_fp64():
    """The mixed path (3xTF32 H_eff on the tensor cores, double-float
    environment updates, mixed SVD) against the FP64 GPU path on a 41-site Ising
    chain (alpha = 1.5, h = 0.5, 8 exponentials) with every bond at chi = 64
    and 8 segments, from the same seeded state, after each of 20 steps:
    <sigma^z_j> within 1e-5 (the accuracy the mixed path is held to), energies
    within 1e-6 relative, discarded weights within 5 %."""
    torch_or_skip()
    tdvp = lib()
    N, chi, steps = 41, 64, 20
    seg = [6, 5, 5, 5, 5, 5, 5, 5]
    x, lam = models.fit_power_law(1.5, 8, N - 1)
    mpo = tdvp.build_mpo(models.ISING, N, 1.5, 1.0, 0.5, 8, x, lam)
    raw = I.random_mps_tensors(N, chi, seed=5)
    runs = {}
    for prec in (I.TF32X3, I.FP64):
        mps = tdvp.init_mps_tensors(raw, chi, 1e-14)
        p = tdvp.step_params(dt=0.01, chi_max=chi, eps=1e-12, krylov_max=8, krylov_tol=1e-6, precision=prec,
                             seg_len=seg)
        e0 = tdvp.energy(mps, mpo)
        sz, en, wt = [], [], []
        for _ in range(steps):
            st = tdvp.step(mps, mpo, p, 1)
            sz.append(tdvp.measure(mps, tdvp.OBS_SZ))
            en.append(tdvp.energy(mps, mpo))
            wt.append(st.w_total)
        runs[prec] = (np.array(sz), np.array(en), np.cumsum(wt), e0)
        del mps
    sz_m, en_m, w_m, e0_m = runs[I.TF32X3]
    sz_d, en_d, w_d, e0_d = runs[I.FP64]
    assert abs(e0_m - e0_d) < 1e-12 * max(1.0, abs(e0_d))
    err = np.abs(sz_m - sz_d).max(axis=1)
    assert err.max() < 1e-5, err
    assert np.abs(en_m - en_d).max() < 1e-6 * max(1.0, abs(e0_d)), en_m - en_d
    assert np.all(np.abs(w_m - w_d) <= 0.05 * w_d + 1e-12)
