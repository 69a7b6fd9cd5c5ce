"""End-to-end GPU parity of tdvp_step against the oracle's sweep.

The CUDA path (all segments of a stage batched) and the oracle run the same
schedule on the same seeded inputs with the same couplings; FP64 observables
must agree to 1e-10, the mixed-precision runs to their stated tolerance.
"""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import models
from oracle import mps as M
from oracle import tdvp as T

from gpu_util import lib, torch_or_skip
from test_oracle_tdvp import w_state

pytestmark = pytest.mark.gpu


def run_pair(kind, N, alpha, J, h, K, init, dt, steps, chi, seg=None, eps=1e-12, kmax=10, tol=0.0,
             prec=0, w_max=0.0, merge=1, raw=None):
    torch_or_skip()
    tdvp = lib()
    x, lam = models.fit_power_law(alpha, K, N - 1)
    W = models.build_mpo_site(kind, J, h, x, lam)
    mpo = tdvp.build_mpo(kind, N, alpha, J, h, K, x, lam)
    if raw is None:
        mps = tdvp.init_mps(N, init, chi)
        omps = M.product_state(init)
    else:
        mps = tdvp.init_mps_tensors(raw, chi, 1e-14)
        omps = M.canonicalize(raw, chi, 1e-14)
    p = tdvp.step_params(dt=dt, chi_max=chi, w_max=w_max, eps=eps, krylov_max=kmax, krylov_tol=tol,
                         precision=prec, seg_len=seg, merge_turning=merge)
    st = tdvp.step(mps, mpo, p, steps)
    eng = T.Engine(omps, W)
    eng.step(T.Params(dt=dt, chi_max=chi, w_max=w_max, eps=eps, krylov_max=kmax, krylov_tol=tol, seg_len=seg,
                      merge_turning=merge), steps)
    return tdvp, mps, mpo, eng, W, st


def compare(tdvp, mps, mpo, eng, W, tol):
    for obs, fn in ((tdvp.OBS_SZ, M.expect_sz), (tdvp.OBS_SX, M.expect_sx), (tdvp.OBS_SY, M.expect_sy)):
        g = tdvp.measure(mps, obs)
        r = fn(eng.mps)
        assert np.abs(g - r).max() < tol, (obs, np.abs(g - r).max())
    assert abs(tdvp.norm(mps) - M.norm2(eng.mps)) < tol
    assert abs(tdvp.energy(mps, mpo) - M.energy(eng.mps, W)) < tol * max(1.0, abs(M.energy(eng.mps, W)))


def test_sweep_serial_tfim_n10_fp64():
    w = I.tfim_n10_quench()
    m = w.model
    tdvp, mps, mpo, eng, W, st = run_pair(m.kind, m.N, m.alpha, m.J, m.h, m.n_exp,
                                          I.basis_state("all_up", m.N), 0.01, 20, 32)
    compare(tdvp, mps, mpo, eng, W, 1e-10)
    assert list(mps.bond_dims()) == eng.mps.bond_dims()
    assert abs(st.w_total - eng.stats.w_total) < 1e-14
    assert st.n_fwd2 == eng.stats.n_fwd2 and st.n_back1 == eng.stats.n_back1


@pytest.mark.parametrize("seg", [[5, 5], [2, 3, 3, 2], [3, 3, 4]])
def test_sweep_segments_tfim_n10_fp64(seg):
    w = I.tfim_n10_quench()
    m = w.model
    tdvp, mps, mpo, eng, W, st = run_pair(m.kind, m.N, m.alpha, m.J, m.h, m.n_exp,
                                          I.basis_state("all_up", m.N), 0.01, 10, 32, seg=seg)
    compare(tdvp, mps, mpo, eng, W, 1e-10)
    assert st.n_stages > 0


def test_sweep_xy_neel_segments_fp64():
    N = 12
    tdvp, mps, mpo, eng, W, st = run_pair(models.XY, N, 1.5, 1.0, 0.0, 4, I.basis_state("neel", N), 0.02, 8,
                                          64, seg=[3, 3, 3, 3])
    compare(tdvp, mps, mpo, eng, W, 1e-10)


def test_sweep_truncated_ising_fp64():
    # truncation by chi_max (bonds cut at 6) with a transverse field (no symmetry,
    # no degenerate multiplets at the cut)
    N = 12
    tdvp, mps, mpo, eng, W, st = run_pair(models.ISING, N, 2.0, 1.0, 0.9, 3, I.basis_state("neel", N), 0.05, 6,
                                          6, seg=[6, 6])
    assert max(mps.bond_dims()) == 6
    compare(tdvp, mps, mpo, eng, W, 1e-10)
    assert abs(st.w_total - eng.stats.w_total) < 1e-10 * max(1.0, eng.stats.w_total)


def test_sweep_random_state_xxx_fp64():
    N = 10
    raw = I.random_mps_tensors(N, 6, seed=0)
    tdvp, mps, mpo, eng, W, st = run_pair(models.XXX, N, 2.0, 1.0, 0.0, 3, None, 0.02, 4, 16, seg=[4, 6],
                                          raw=raw)
    compare(tdvp, mps, mpo, eng, W, 1e-10)


def test_sweep_single_magnon_merge_off():
    N = 12
    c = I.random_complex((N,), seed=1)
    c /= np.linalg.norm(c)
    tdvp, mps, mpo, eng, W, st = run_pair(models.XY, N, 1.5, 1.0, 0.0, 6, None, 0.02, 10, 8, seg=[6, 6],
                                          merge=0, raw=w_state(c))
    compare(tdvp, mps, mpo, eng, W, 1e-10)


def test_sweep_production_krylov():
    # the paper's Lanczos settings: at most 8 vectors, tolerance 1e-6
    w = I.tfim_n10_quench()
    m = w.model
    tdvp, mps, mpo, eng, W, st = run_pair(m.kind, m.N, m.alpha, m.J, m.h, m.n_exp,
                                          I.basis_state("all_up", m.N), 0.01, 10, 32, kmax=8, tol=1e-6)
    compare(tdvp, mps, mpo, eng, W, 1e-7)


@pytest.mark.parametrize("prec,tol", [(2, 1e-5), (1, 2e-3)], ids=["tf32x3", "tf32"])
def test_sweep_mixed_precision(prec, tol):
    w = I.tfim_n10_quench()
    m = w.model
    tdvp, mps, mpo, eng, W, st = run_pair(m.kind, m.N, m.alpha, m.J, m.h, m.n_exp,
                                          I.basis_state("all_up", m.N), 0.01, 20, 32, seg=[5, 5], prec=prec)
    g = tdvp.measure(mps, tdvp.OBS_SZ)
    assert np.abs(g - M.expect_sz(eng.mps)).max() < tol


def test_overlap_and_infidelity_between_runs():
    torch_or_skip()
    tdvp = lib()
    N = 10
    x, lam = models.fit_power_law(3.0, 4, N - 1)
    mpo = tdvp.build_mpo(models.ISING, N, 3.0, 1.0, 1.0, 4, x, lam)
    a = tdvp.init_mps(N, I.basis_state("all_up", N), 32)
    b = tdvp.init_mps(N, I.basis_state("all_up", N), 32)
    tdvp.step(a, mpo, tdvp.step_params(0.02, 32, krylov_max=10, krylov_tol=0.0), 5)
    tdvp.step(b, mpo, tdvp.step_params(0.02, 32, krylov_max=10, krylov_tol=0.0, seg_len=[5, 5]), 5)
    ov = tdvp.overlap(a, b)
    infid = 1 - abs(ov) / np.sqrt(tdvp.norm(a) * tdvp.norm(b))
    W = models.build_mpo_site(models.ISING, 1.0, 1.0, x, lam)
    ea = T.Engine(M.product_state(I.basis_state("all_up", N)), W)
    ea.step(T.Params(dt=0.02, chi_max=32, krylov_max=10, krylov_tol=0.0), 5)
    eb = T.Engine(M.product_state(I.basis_state("all_up", N)), W)
    eb.step(T.Params(dt=0.02, chi_max=32, krylov_max=10, krylov_tol=0.0, seg_len=[5, 5]), 5)
    assert abs(ov - M.overlap(ea.mps, eb.mps)) < 1e-11
    assert abs(infid - M.infidelity(ea.mps, eb.mps)) < 1e-11


def test_step_rejects_bad_params():
    torch_or_skip()
    tdvp = lib()
    N = 6
    mpo = tdvp.build_mpo(models.ISING, N, 2.0, 1.0, 1.0, 2)
    mps = tdvp.init_mps(N, [0] * N, 8)
    with pytest.raises(tdvp.TdvpError):
        tdvp.step(mps, mpo, tdvp.step_params(0.01, 8, seg_len=[1, 5]), 1)
    with pytest.raises(tdvp.TdvpError):
        tdvp.step(mps, mpo, tdvp.step_params(0.01, 8, krylov_max=40), 1)
    with pytest.raises(tdvp.TdvpError):
        tdvp.step(mps, mpo, tdvp.step_params(-0.01, 8), 1)
    other = tdvp.build_mpo(models.ISING, N + 1, 2.0, 1.0, 1.0, 2)
    with pytest.raises(tdvp.TdvpError):
        tdvp.step(mps, other, tdvp.step_params(0.01, 8), 1)


def test_full_size_mixed_step_matches_fp64_step():
    """The benchmark's workload (N = 101, chi = 256, 8 segments, 8 Krylov
    vectors, tolerance 1e-6) from its seeded random state: one mixed-precision
    (3xTF32) step and one plain FP64 step must give <sigma^z_j> within 1e-5 (the
    mixed path's accuracy target). The norm and the discarded weight (a sum of
    ~1e-6 remainders over 200 splits, each carrying the contractions' ~1e-7
    relative error of Theta') are compared loosely."""
    torch_or_skip()
    tdvp = lib()
    w = I.tfim_n101_quench()
    mdl, prm = w.model, w.params
    mpo = tdvp.build_mpo(mdl.kind, mdl.N, mdl.alpha, mdl.J, mdl.h, mdl.n_exp)
    raw = I.random_mps_tensors(mdl.N, prm.chi_max, seed=0)
    out = {}
    for prec in (I.TF32X3, I.FP64):
        mps = tdvp.init_mps_tensors(raw, prm.chi_max, 1e-14)
        p = tdvp.step_params(dt=prm.dt, chi_max=prm.chi_max, w_max=prm.w_max, eps=prm.eps,
                             krylov_max=prm.krylov_max, krylov_tol=prm.krylov_tol, precision=prec,
                             seg_len=prm.seg_len, merge_turning=1)
        st = tdvp.step(mps, mpo, p, 1)
        out[prec] = (tdvp.measure(mps, tdvp.OBS_SZ), tdvp.norm(mps), st.w_total, st.chi_max_seen)
        del mps
    (sz_m, n_m, w_m, c_m), (sz_d, n_d, w_d, c_d) = out[I.TF32X3], out[I.FP64]
    assert c_m == c_d == prm.chi_max
    assert np.abs(sz_m - sz_d).max() < 1e-5
    assert abs(n_m - n_d) < 1e-5
    assert abs(w_m - w_d) < 0.05 * w_d


def test_reorthonormalize_keeps_the_state():
    """tdvp_reorthonormalize (Sec. III D) after a segmented run: the state is
    unchanged up to its norm (observables to 1e-12), normalised (to 1e-10), and
    back in the inverse canonical gauge (Psi_j = A_j Lambda_j = Lambda_{j-1} B_j
    with A_j, B_j isometries); a serial run continued after it matches the
    oracle's uninterrupted run."""
    torch_or_skip()
    N = 12
    tdvp, mps, mpo, eng, W, st = run_pair(models.XY, N, 1.5, 1.0, 0.3, 4, I.basis_state("neel", N), 0.05, 6,
                                          64, seg=[3, 3, 3, 3])
    before = [tdvp.measure(mps, o) for o in (tdvp.OBS_SZ, tdvp.OBS_SX)]
    tdvp.reorthonormalize(mps)
    after = [tdvp.measure(mps, o) for o in (tdvp.OBS_SZ, tdvp.OBS_SX)]
    for b, a in zip(before, after):
        assert np.abs(a - b).max() < 1e-12
    assert abs(tdvp.norm(mps) - 1.0) < 1e-10
    # Psi_j = A_j Lambda_j = Lambda_{j-1} B_j: the Gram matrices of Psi_j over its
    # right / left bond are Lambda^2. The check ties the SVDs of two neighbouring
    # bonds together, and with Schmidt values down to ~1e-5 their vectors are
    # determined to ~eps lambda_1 / lambda_i in FP64: 1e-10 of lambda_1^2
    for j in range(N - 1):
        psi = mps.site(j)
        lam = 1.0 / mps.bond(j)
        A = psi.reshape(-1, len(lam))
        assert np.abs(A.conj().T @ A - np.diag(lam ** 2)).max() < 1e-10 * lam.max() ** 2
    for j in range(1, N):
        psi = mps.site(j)
        lam = 1.0 / mps.bond(j - 1)
        B = psi.reshape(len(lam), -1)
        assert np.abs(B @ B.conj().T - np.diag(lam ** 2)).max() < 1e-10 * lam.max() ** 2
    # serial: 4 steps, reorthonormalise, 4 more == 8 uninterrupted oracle steps
    x, lam = models.fit_power_law(2.0, 4, N - 1)
    mpo2 = tdvp.build_mpo(models.ISING, N, 2.0, 1.0, 0.8, 4, x, lam)
    s = tdvp.init_mps(N, I.basis_state("all_up", N), 64)
    p = tdvp.step_params(dt=0.02, chi_max=64, krylov_max=10, krylov_tol=0.0)
    tdvp.step(s, mpo2, p, 4)
    tdvp.reorthonormalize(s)
    tdvp.step(s, mpo2, p, 4)
    e = T.Engine(M.product_state(I.basis_state("all_up", N)), models.build_mpo_site(models.ISING, 1.0, 0.8, x, lam))
    e.step(T.Params(dt=0.02, chi_max=64, krylov_max=10, krylov_tol=0.0), 8)
    assert np.abs(tdvp.measure(s, tdvp.OBS_SZ) - M.expect_sz(e.mps)).max() < 1e-10


@pytest.mark.parametrize("N,chi,seg", [(2, 4, None), (3, 4, None), (4, 1, None), (6, 8, [2, 4]), (7, 8, [3, 4])])
def test_sweep_edge_cases(N, chi, seg):
    """Smallest chains (a single pair; three sites), bond dimension 1 (a product
    state kept a product state), segments of two sites and an odd chain length:
    the same schedule and results as the oracle."""
    tdvp, mps, mpo, eng, W, st = run_pair(models.ISING, N, 2.0, 1.0, 0.7, 2, I.basis_state("neel", N), 0.05, 3,
                                          chi, seg=seg)
    compare(tdvp, mps, mpo, eng, W, 1e-10)
    assert list(mps.bond_dims()) == eng.mps.bond_dims()
    assert st.n_fwd2 == eng.stats.n_fwd2 and st.n_back1 == eng.stats.n_back1


def test_xy_n51_full_size_properties():
    """The 51-site XY quench at its full size (XY, N = 51, chi_max = 128, eps = 1e-10, four
    segments 13/13/13/12, Neel start): the XY Hamiltonian conserves the total
    S^z (+1 for the odd chain's Neel state) to rounding; the energy of the TDVP state is conserved up
    to the truncation, and the norm drops by about the discarded weight."""
    torch_or_skip()
    tdvp = lib()
    w = I.xy_n51_quench()
    mdl, prm = w.model, w.params
    mpo = tdvp.build_mpo(mdl.kind, mdl.N, mdl.alpha, mdl.J, mdl.h, mdl.n_exp)
    mps = tdvp.init_mps(mdl.N, I.basis_state("neel", mdl.N), prm.chi_max)
    e0 = tdvp.energy(mps, mpo)
    sz0 = tdvp.measure(mps, tdvp.OBS_SZ).sum()
    p = tdvp.step_params(dt=prm.dt, chi_max=prm.chi_max, w_max=prm.w_max, eps=prm.eps, krylov_max=10,
                         krylov_tol=0.0, seg_len=prm.seg_len)
    st = tdvp.step(mps, mpo, p, 20)
    sz = tdvp.measure(mps, tdvp.OBS_SZ)
    assert abs(sz0 - 1.0) < 1e-12 and abs(sz.sum() - sz0) < 1e-9
    assert abs(tdvp.energy(mps, mpo) - e0) < 1e-3 * max(1.0, abs(e0))
    nrm = tdvp.norm(mps)
    assert nrm <= 1.0 + 1e-10
    assert st.chi_max_seen <= prm.chi_max
