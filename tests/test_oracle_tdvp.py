"""Pins for the oracle's sweeps against exact diagonalisation and closed forms.

CPU only. The serial sweep must reproduce ED where the two-site projector is
exact (full-rank bonds), converge at second order in dt on a single-magnon
state (closed-form N x N solution), and conserve norm and energy without
truncation. The segment schedule is checked for its invariants and for
independence of the execution order.
"""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import ed, models
from oracle import mps as M
from oracle import tdvp as T
from oracle.models import ISING, XXX, XY

from test_oracle_models import single_magnon_matrix


def tfim_n10_setup(N=10):
    w = I.tfim_n10_quench()
    mdl = w.model
    x, lam = models.fit_power_law(mdl.alpha, mdl.n_exp, N - 1)
    W = models.build_mpo_site(mdl.kind, mdl.J, mdl.h, x, lam)
    H = models.dense_hamiltonian(mdl.kind, N, mdl.J, mdl.h, models.couplings(x, lam, N - 1))
    return W, H


def test_serial_matches_ed_full_rank():
    N = 10
    W, H = tfim_n10_setup(N)
    st = I.basis_state("all_up", N)
    eng = T.Engine(M.product_state(st), W)
    p = T.Params(dt=0.01, chi_max=32, krylov_max=10, krylov_tol=0.0)
    exact = ed.ExactEvolution(H)
    v0 = ed.product_vector(st)
    E0 = M.energy(eng.mps, W)
    for n in range(1, 21):
        eng.step(p, 1)
        if n % 10 == 0:
            ref = ed.expect_sz_dense(exact.evolve(v0, n * p.dt), N)
            assert np.abs(M.expect_sz(eng.mps) - ref).max() < 1e-9
            assert abs(M.norm2(eng.mps) - 1.0) < 1e-12
            assert abs(M.energy(eng.mps, W) - E0) < 1e-9
    assert eng.stats.w_total < 1e-20


def test_serial_production_krylov_within_1e5():
    # the paper's Lanczos settings (8 vectors, tol 1e-6)
    N = 10
    W, H = tfim_n10_setup(N)
    st = I.basis_state("all_up", N)
    eng = T.Engine(M.product_state(st), W)
    p = T.Params(dt=0.01, chi_max=32)
    for _ in range(10):
        eng.step(p, 1)
    ref = ed.expect_sz_dense(ed.ExactEvolution(H).evolve(ed.product_vector(st), 0.1), N)
    assert np.abs(M.expect_sz(eng.mps) - ref).max() < 1e-5


def w_state(c):
    """Single-magnon superposition sum_j c_j |down..up_j..down> as a chi = 2 MPS."""
    N = len(c)
    out = []
    for j in range(N):
        t = np.zeros((2, 2, 2), dtype=np.complex128)
        t[0, 1, 0] = 1.0
        t[0, 0, 1] = c[j]
        t[1, 1, 1] = 1.0
        if j == 0:
            t = t[:1]
        if j == N - 1:
            t = t[:, :, 1:]
        out.append(t)
    return out


def magnon_errors(kind, seg, dts, N=12, tf=0.4):
    x, lam = models.fit_power_law(1.5, 6, N - 1)
    V = models.couplings(x, lam, N - 1).real
    W = models.build_mpo_site(kind, 1.0, 0.0, x, lam)
    c = I.random_complex((N,), seed=1)
    c /= np.linalg.norm(c)
    e, U = np.linalg.eigh(single_magnon_matrix(kind, V, N))
    ct = U @ (np.exp(-1j * e * tf) * (U.conj().T @ c))
    exact = -1 + 2 * np.abs(ct) ** 2
    errs = []
    for dt in dts:
        eng = T.Engine(M.canonicalize(w_state(c), 8), W)
        p = T.Params(dt=dt, chi_max=8, krylov_max=12, krylov_tol=0.0, seg_len=seg)
        eng.step(p, int(round(tf / dt)))
        errs.append(np.abs(M.expect_sz(eng.mps) - exact).max())
        assert max(eng.mps.bond_dims()) == 2
    return np.array(errs)


@pytest.mark.parametrize("kind", [XY, XXX])
def test_serial_second_order_on_single_magnon(kind):
    # symmetric second-order splitting: error falls 4x when dt is halved
    errs = magnon_errors(kind, None, (0.04, 0.02, 0.01))
    ratios = errs[:-1] / errs[1:]
    assert np.all(np.abs(ratios - 4.0) < 0.1), ratios
    assert errs[-1] < 2e-5


def test_segments_converge_on_single_magnon():
    # p = 2: out-of-date environments add an O(dt) error (Sec. III D)
    errs = magnon_errors(XY, [6, 6], (0.04, 0.02, 0.01))
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 1.8), ratios
    assert errs[-1] < 1e-3


def serial_expected_ops(N):
    """Serial sweep of Sec. III A written out: pairs forward, shared sites
    backward, rightmost pair once by a full dt, then the mirror image."""
    h1 = [("fwd2", 0, 1)]
    for j in range(1, N - 1):
        h1 += [("back1", j, 1), ("fwd2", j, 2 if j == N - 2 else 1)]
    h2 = []
    for j in range(N - 2, 0, -1):
        h2 += [("back1", j, 1), ("fwd2", j - 1, 1)]
    return h1, h2


@pytest.mark.parametrize("N", [3, 5, 9])
def test_serial_schedule_is_sec3a_sweep(N):
    h1, h2 = T.build_schedule(N, [N], 1)
    assert [(o.kind, o.j, o.tfac) for o in h1] == serial_expected_ops(N)[0]
    assert [(o.kind, o.j, o.tfac) for o in h2] == serial_expected_ops(N)[1]
    assert [o.stage for o in h1] == list(range(len(h1)))


@pytest.mark.parametrize("seg", [[12], [6, 6], [3, 4, 5], [2, 3, 3, 4], [3, 3, 3, 3],
                                 [2, 2, 2, 2, 2, 2], [4, 2, 2, 4]])
@pytest.mark.parametrize("merge", [0, 1])
def test_schedule_invariants(seg, merge):
    N = sum(seg)
    sched = T.build_schedule(N, seg, merge)
    fw = np.zeros(N - 1)
    bk = np.zeros(N)
    for half in sched:
        stages = {}
        for o in half:
            if o.kind == "fwd2":
                fw[o.j] += o.tfac
            else:
                bk[o.j] += o.tfac
            stages.setdefault(o.stage, []).append(o)
            for d in o.deps:
                assert half[d].stage < o.stage
        for ops in stages.values():
            # a segment runs at most one op per stage; ops of a stage touch
            # disjoint sites
            assert len({o.seg for o in ops}) == len(ops)
            sites = [s for o in ops for s in ((o.j, o.j + 1) if o.kind == "fwd2" else (o.j,))]
            assert len(sites) == len(set(sites))
    # every pair forward by dt (2 tau), every interior site backward by dt
    assert np.all(fw == 2)
    assert np.all(bk[1:-1] == 2) and bk[0] == 0 and bk[-1] == 0


def test_boundary_ops_by_left_segment():
    seg = [3, 4, 5, 4]
    N = sum(seg)
    bounds = T.segment_bounds(N, seg)
    for half in T.build_schedule(N, seg, 1):
        for o in half:
            if o.boundary:
                s, e = bounds[o.seg]
                assert o.kind == "fwd2" and o.j == e and o.env == "LR"


def run_tfim_n10(seg, dt, tf, order="stage", merge=1, chi=32):
    N = 10
    W, _ = tfim_n10_setup(N)
    eng = T.Engine(M.product_state(I.basis_state("all_up", N)), W)
    p = T.Params(dt=dt, chi_max=chi, krylov_max=10, krylov_tol=0.0, seg_len=seg,
                 merge_turning=merge)
    eng.step(p, int(round(tf / dt)), order=order)
    return eng


def test_execution_order_independence():
    a = run_tfim_n10([2, 3, 3, 2], 0.02, 0.2, order="stage")
    b = run_tfim_n10([2, 3, 3, 2], 0.02, 0.2, order="segment")
    for x, y in zip(a.mps.Psi, b.mps.Psi):
        assert np.array_equal(x, y)


def test_segments_close_to_serial_and_improve_with_dt():
    infid = []
    for dt in (0.04, 0.02):
        s = run_tfim_n10(None, dt, 0.4)
        q = run_tfim_n10([5, 5], dt, 0.4)
        infid.append(M.infidelity(s.mps, q.mps))
    assert infid[0] < 1e-7 and infid[1] < infid[0]


def test_merge_off_also_matches_ed():
    N = 10
    W, H = tfim_n10_setup(N)
    eng = run_tfim_n10([5, 5], 0.01, 0.1, merge=0)
    ref = ed.expect_sz_dense(ed.ExactEvolution(H).evolve(
        ed.product_vector(I.basis_state("all_up", N)), 0.1), N)
    assert np.abs(M.expect_sz(eng.mps) - ref).max() < 1e-8


def test_truncated_run_reports_discarded_weight():
    eng = run_tfim_n10(None, 0.02, 0.4, chi=4)
    assert max(eng.mps.bond_dims()) == 4
    assert eng.stats.w_total > 0
    # no renormalisation: the norm shrinks by about the discarded weight
    assert abs((1 - M.norm2(eng.mps)) - eng.stats.w_total) < 0.5 * eng.stats.w_total + 1e-12
