"""Pins for the oracle's one-site TDVP (1TDVP) and the hybrid 2TDVP -> 1TDVP scheme.

CPU only. At full bond dimension the one-site projector is the identity, so the
split steps compose to the exact evolution: 1TDVP must reproduce exact
diagonalisation. Below full rank the scheme is symplectic at fixed bond
dimension: norm and energy are conserved (to the Krylov accuracy) and the bond
dimensions do not change. The hybrid scheme switches once every bond is full.
"""
import numpy as np

import tdvp_inputs as I
from oracle import ed, models
from oracle import mps as M
from oracle import tdvp as T
from oracle import tdvp1 as T1
from oracle.models import ISING, XY


def setup(kind, N, alpha, K, h, chi0, chi, seed):
    x, lam = models.fit_power_law(alpha, K, N - 1)
    W = models.build_mpo_site(kind, 1.0, h, x, lam)
    H = models.dense_hamiltonian(kind, N, 1.0, h, models.couplings(x, lam, N - 1))
    mps = M.canonicalize(I.random_mps_tensors(N, chi0, seed=seed), chi, 1e-14)
    return W, H, mps


def test_full_rank_one_site_tdvp_is_exact():
    N = 8
    W, H, mps = setup(ISING, N, 3.0, 4, 0.7, 16, 16, 3)
    v0 = M.to_dense(mps)
    eng = T.Engine(mps, W)
    p = T.Params(dt=0.05, chi_max=16, krylov_max=24, krylov_tol=0.0)
    T1.step1(eng, p, 6)
    ref = ed.ExactEvolution(H).evolve(v0, 6 * p.dt)
    for op in (models.SZ, models.SX):
        got = M.expect_local(eng.mps, op)
        want = np.array([np.vdot(ref, models.site_operator(op, j, N) @ ref).real for j in range(N)])
        assert np.abs(got - want).max() < 1e-9
    assert abs(M.infidelity(eng.mps, M.from_dense(ref, N, 16))) < 1e-10


def test_one_site_tdvp_conserves_norm_energy_and_bond_dimensions():
    for kind, h in ((ISING, 0.6), (XY, 0.2)):
        W, H, mps = setup(kind, 10, 2.0, 4, h, 4, 4, 7)
        dims = mps.bond_dims()
        assert max(dims) == 4 and dims != [min(2 ** (j + 1), 2 ** (9 - j)) for j in range(9)]
        eng = T.Engine(mps, W)
        E0 = M.energy(eng.mps, W)
        p = T.Params(dt=0.05, chi_max=4, krylov_max=24, krylov_tol=0.0)
        T1.step1(eng, p, 8)
        assert eng.mps.bond_dims() == dims
        assert abs(M.norm2(eng.mps) - 1.0) < 1e-12
        assert abs(M.energy(eng.mps, W) - E0) < 1e-10 * max(1.0, abs(E0))


def test_hybrid_switches_when_bonds_saturate():
    N = 8
    x, lam = models.fit_power_law(3.0, 4, N - 1)
    W = models.build_mpo_site(ISING, 1.0, 1.0, x, lam)
    eng = T.Engine(M.product_state(I.basis_state("all_up", N)), W)
    p = T.Params(dt=0.05, chi_max=4, krylov_max=24, krylov_tol=0.0)
    E0 = M.energy(eng.mps, W)
    n1 = T1.step_hybrid(eng, p, 12)
    assert 0 < n1 < 12
    assert T1.saturated(eng, 4)
    assert abs(M.norm2(eng.mps) - 1.0) < 1e-10
    assert abs(M.energy(eng.mps, W) - E0) < 1e-3 * abs(E0)


# ---- segmented (parallel) one-site TDVP ----

def _copy(mps):
    import copy
    return copy.deepcopy(mps)


def test_segmented_one_site_with_one_segment_is_the_serial_sweep():
    W, H, mps = setup(ISING, 8, 3.0, 4, 0.7, 6, 6, 11)
    a, b = T.Engine(_copy(mps), W), T.Engine(_copy(mps), W)
    p = T.Params(dt=0.05, chi_max=6, krylov_max=16, krylov_tol=0.0)
    T1.step1(a, p, 3)
    T1.step1_segmented(b, p, 3)
    for x, y in zip(a.mps.Psi, b.mps.Psi):
        assert np.array_equal(x, y)


def test_segmented_schedule_covers_every_term_once_per_step():
    """Per time step every site term acts forward for dt (one-site steps, or its
    share of a boundary pair step) and every bond term backward for dt (a bond
    step, or inside a boundary pair step)."""
    for N, seg in ((10, [10]), (10, [5, 5]), (10, [3, 3, 4]), (11, [2, 3, 3, 3]), (12, [2, 2, 2, 2, 2, 2])):
        for merge in (0, 1):
            site = np.zeros(N)
            bond = np.zeros(N - 1)
            for half in (1, 2):
                for op in T1.build_half1(N, seg, half, merge):
                    if op.kind == "site":
                        site[op.j] += op.tfac
                    elif op.kind == "bond_r":
                        bond[op.j] += op.tfac
                    elif op.kind == "bond_l":
                        bond[op.j - 1] += op.tfac
                    else:
                        site[op.j] += op.tfac
                        site[op.j + 1] += op.tfac
                        bond[op.j] += op.tfac
            assert np.all(site == 2) and np.all(bond == 2), (N, seg, merge, site, bond)


def test_segmented_one_site_is_exact_at_full_rank():
    N = 8
    W, H, mps = setup(ISING, N, 3.0, 4, 0.7, 16, 16, 3)
    v0 = M.to_dense(mps)
    ref = ed.expect_sz_dense(ed.ExactEvolution(H).evolve(v0, 0.3), N)
    for seg in ([4, 4], [2, 3, 3], [2, 2, 2, 2]):
        eng = T.Engine(_copy(mps), W)
        T1.step1_segmented(eng, T.Params(dt=0.05, chi_max=16, krylov_max=24, krylov_tol=0.0, seg_len=seg), 6)
        assert np.abs(M.expect_sz(eng.mps) - ref).max() < 1e-11, seg
        assert abs(M.norm2(eng.mps) - 1.0) < 1e-12


def test_segmented_one_site_below_full_rank():
    """Bond dimensions are kept; the boundary pair steps cut back to them, so the
    norm and energy drift by the discarded weight, which falls in proportion to
    dt over a fixed time (a cut per boundary and step, each of order dt^2)."""
    W, H, mps = setup(ISING, 10, 2.0, 4, 0.6, 4, 4, 7)
    dims = mps.bond_dims()
    E0 = M.energy(mps, W)
    drift = []
    for dt, n in ((0.05, 4), (0.025, 8)):
        eng = T.Engine(_copy(mps), W)
        T1.step1_segmented(eng, T.Params(dt=dt, chi_max=4, krylov_max=24, krylov_tol=0.0, seg_len=[3, 3, 4]), n)
        assert eng.mps.bond_dims() == dims
        assert M.norm2(eng.mps) <= 1.0 + 1e-12
        drift.append(abs(M.energy(eng.mps, W) - E0))
    assert drift[0] < 1e-2 and 0.4 * drift[0] < drift[1] < 0.6 * drift[0]


def test_hybrid_with_segments_switches_and_matches_serial_at_full_rank():
    """The hybrid scheme with segments: two-site steps until every bond is full,
    then segmented one-site steps. From the product state the first two-site
    steps are not exact (the bonds grow with the evolution; 2.3e-8 for the
    serial hybrid here); once every bond is full both schemes are, so the
    segmented hybrid stays as close to exact diagonalisation as the serial one."""
    N = 8
    x, lam = models.fit_power_law(3.0, 4, N - 1)
    W = models.build_mpo_site(ISING, 1.0, 1.0, x, lam)
    H = models.dense_hamiltonian(ISING, N, 1.0, 1.0, models.couplings(x, lam, N - 1))
    st = I.basis_state("all_up", N)
    eng = T.Engine(M.product_state(st), W)
    p = T.Params(dt=0.05, chi_max=16, krylov_max=24, krylov_tol=0.0, seg_len=[4, 4])
    n1 = T1.step_hybrid(eng, p, 10)
    assert 0 < n1 < 10
    ref = ed.expect_sz_dense(ed.ExactEvolution(H).evolve(ed.product_vector(st), 0.5), N)
    assert np.abs(M.expect_sz(eng.mps) - ref).max() < 1e-7
