"""GPU parity of the local operations (one per hot-path step) against the oracle.

Each test calls the CUDA library through its C ABI (kernel-level entry points
on torch device buffers) and compares element by element with the oracle on
the same seeded inputs: H_eff . theta (two- and one-site), the environment
updates, the Lanczos exponential and the truncated SVD split. FP64 must agree
to rounding (1e-12 relative); TF32 and 3xTF32 contractions to the precision of
their products (tolerances derived from the unit roundoffs 2^-11 and ~2^-22
times the length of the sums).
"""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import models
from oracle import tdvp as T

from gpu_util import dev, hermitian_env, host, lib, max_err, torch_or_skip

pytestmark = pytest.mark.gpu

FP64, TF32, TF32X3 = 0, 1, 2
TOL = {FP64: 1e-12, TF32: 6e-3, TF32X3: 3e-5}


def mpo_W(kind=models.ISING, alpha=1.5, K=3, N=20, J=1.0, h=0.5):
    x, lam = models.fit_power_law(alpha, K, N - 1)
    return models.build_mpo_site(kind, J, h, x, lam)


SIZES_2 = [(1, 1), (1, 2), (2, 1), (3, 5), (17, 9), (33, 64), (64, 64), (100, 37)]


@pytest.mark.parametrize("prec", [FP64, TF32, TF32X3], ids=["fp64", "tf32", "tf32x3"])
@pytest.mark.parametrize("chi_l,chi_r", SIZES_2)
def test_heff_two_site(prec, chi_l, chi_r):
    torch = torch_or_skip()
    tdvp = lib()
    W = mpo_W()
    m, d = W.shape[0], 2
    L = hermitian_env((chi_l, m, chi_l), 1)
    R = hermitian_env((chi_r, m, chi_r), 2)
    th = I.random_complex((chi_l, d, d, chi_r), 3)
    ref = T.heff2_apply(L, W, W, R, th)
    y = torch.zeros(ref.size, dtype=torch.complex128, device="cuda")
    tdvp.op_heff(prec, 2, chi_l, chi_r, m, d, W, dev(torch, L), dev(torch, R), dev(torch, th), y)
    out = host(y).reshape(ref.shape)
    assert max_err(out, ref) < TOL[prec], (prec, chi_l, chi_r, max_err(out, ref))


@pytest.mark.parametrize("prec", [FP64, TF32, TF32X3], ids=["fp64", "tf32", "tf32x3"])
@pytest.mark.parametrize("kind", [models.ISING, models.XY, models.XXX])
@pytest.mark.parametrize("chi_l,chi_r", [(1, 1), (5, 3), (40, 71), (128, 128)])
def test_heff_one_site(prec, kind, chi_l, chi_r):
    torch = torch_or_skip()
    tdvp = lib()
    W = mpo_W(kind=kind, K=2)
    m, d = W.shape[0], 2
    L = hermitian_env((chi_l, m, chi_l), 4)
    R = hermitian_env((chi_r, m, chi_r), 5)
    th = I.random_complex((chi_l, d, chi_r), 6)
    ref = T.heff1_apply(L, W, R, th)
    y = torch.zeros(ref.size, dtype=torch.complex128, device="cuda")
    tdvp.op_heff(prec, 1, chi_l, chi_r, m, d, W, dev(torch, L), dev(torch, R), dev(torch, th), y)
    assert max_err(host(y).reshape(ref.shape), ref) < TOL[prec]


ENV_TOL_DD = 1e-12  # mixed modes' default double-float environments (~48 bits)


@pytest.mark.parametrize("env_tc", [False, True], ids=["env_dd", "env_tc"])
@pytest.mark.parametrize("prec", [FP64, TF32, TF32X3], ids=["fp64", "tf32", "tf32x3"])
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("chi_l,chi_r", [(1, 2), (2, 4), (7, 13), (64, 50), (128, 128)])
def test_env_update(env_tc, prec, side, chi_l, chi_r):
    """Environment updates: FP64; the mixed modes' default double-float GEMMs
    (to ~1e-12); and, switched to the tensor cores, the mode's products."""
    torch = torch_or_skip()
    tdvp = lib()
    if env_tc and prec == FP64:
        pytest.skip("the FP64 path has one environment update")
    W = mpo_W(kind=models.XY, K=3)
    m, d = W.shape[0], 2
    A = I.random_complex((chi_l, d, chi_r), 7)
    if side == 0:
        env = hermitian_env((chi_l, m, chi_l), 8)
        ref = T.env_left(env, A, W)
    else:
        env = hermitian_env((chi_r, m, chi_r), 9)
        ref = T.env_right(env, A, W)
    out = torch.zeros(ref.size, dtype=torch.complex128, device="cuda")
    tdvp.set_env_tensor_cores(env_tc)
    try:
        tdvp.op_env(prec, side, chi_l, chi_r, m, d, W, dev(torch, env), dev(torch, A), out)
    finally:
        tdvp.set_env_tensor_cores(False)
    tol = TOL[prec] if (env_tc or prec == FP64) else ENV_TOL_DD
    assert max_err(host(out).reshape(ref.shape), ref) < tol


@pytest.mark.parametrize("nsite", [1, 2])
@pytest.mark.parametrize("t", [0.005, -0.005, 0.05])
@pytest.mark.parametrize("chi_l,chi_r", [(1, 1), (2, 2), (9, 14), (48, 48)])
def test_expm_fixed_krylov(nsite, t, chi_l, chi_r):
    torch = torch_or_skip()
    tdvp = lib()
    W = mpo_W()
    m, d = W.shape[0], 2
    L = hermitian_env((chi_l, m, chi_l), 10)
    R = hermitian_env((chi_r, m, chi_r), 11)
    shape = (chi_l, d, d, chi_r) if nsite == 2 else (chi_l, d, chi_r)
    th = I.random_complex(shape, 12)
    if nsite == 2:
        fn = lambda x: T.heff2_apply(L, W, W, R, x)  # noqa: E731
    else:
        fn = lambda x: T.heff1_apply(L, W, R, x)  # noqa: E731
    ref, info = T.lanczos_expm(fn, th, t, kmax=10, tol=0.0)
    y = torch.zeros(th.size, dtype=torch.complex128, device="cuda")
    nv = tdvp.op_expm(FP64, nsite, chi_l, chi_r, m, d, W, dev(torch, L), dev(torch, R), dev(torch, th), y,
                      t, 10, 0.0)
    assert nv == info.n_vectors
    assert max_err(host(y).reshape(shape), ref) < 1e-11


def test_expm_breakdown_on_product_state():
    # a one-site problem with chi = 1 lives in a d-dimensional space: the
    # Krylov basis is exhausted after at most 2 vectors
    torch = torch_or_skip()
    tdvp = lib()
    W = mpo_W()
    m, d = W.shape[0], 2
    L = np.zeros((1, m, 1), complex)
    L[0, m - 1, 0] = 1
    R = np.zeros((1, m, 1), complex)
    R[0, 0, 0] = 1
    th = I.random_complex((1, d, 1), 13)
    ref, info = T.lanczos_expm(lambda x: T.heff1_apply(L, W, R, x), th, 0.3, kmax=8, tol=0.0)
    y = torch.zeros(th.size, dtype=torch.complex128, device="cuda")
    nv = tdvp.op_expm(FP64, 1, 1, 1, m, d, W, dev(torch, L), dev(torch, R), dev(torch, th), y, 0.3, 8, 0.0)
    assert info.breakdown and nv == info.n_vectors <= 2
    assert max_err(host(y).reshape(th.shape), ref) < 1e-13


@pytest.mark.parametrize("prec", [TF32, TF32X3], ids=["tf32", "tf32x3"])
def test_expm_mixed_precision(prec):
    torch = torch_or_skip()
    tdvp = lib()
    W = mpo_W()
    m, d = W.shape[0], 2
    L = hermitian_env((32, m, 32), 14)
    R = hermitian_env((20, m, 20), 15)
    th = I.random_complex((32, d, d, 20), 16)
    ref, _ = T.lanczos_expm(lambda x: T.heff2_apply(L, W, W, R, x), th, 0.005, kmax=8, tol=0.0)
    y = torch.zeros(th.size, dtype=torch.complex128, device="cuda")
    tdvp.op_expm(prec, 2, 32, 20, m, d, W, dev(torch, L), dev(torch, R), dev(torch, th), y, 0.005, 8, 0.0)
    assert max_err(host(y).reshape(th.shape), ref) < TOL[prec]


def decaying_matrix(rows, cols, seed, rank=None, decay=0.75):
    U = np.linalg.qr(I.random_complex((rows, rows), seed))[0]
    Vh = np.linalg.qr(I.random_complex((cols, cols), seed + 1))[0]
    n = min(rows, cols)
    s = decay ** np.arange(n)
    if rank is not None:
        s[rank:] = 0.0
    return (U[:, :n] * s) @ Vh[:n], s


@pytest.mark.parametrize("rows,cols", [(1, 1), (2, 2), (4, 2), (2, 4), (8, 8), (33, 20), (20, 33),
                                       (64, 64), (130, 96)])
@pytest.mark.parametrize("chi_max,w_max,eps", [(1000, 0.0, 0.0), (5, 0.0, 1e-12), (1000, 1e-6, 0.0),
                                               (1000, 0.0, 1e-3)])
def test_split(rows, cols, chi_max, w_max, eps):
    torch = torch_or_skip()
    tdvp = lib()
    theta, _ = decaying_matrix(rows, cols, 20)
    n = min(rows, cols)
    s_ref = np.linalg.svd(theta, compute_uv=False)
    chi_ref, w_ref = T.truncation_rank(s_ref, chi_max, w_max, eps)
    PsiL = torch.zeros(rows * n, dtype=torch.complex128, device="cuda")
    PsiR = torch.zeros(n * cols, dtype=torch.complex128, device="cuda")
    V = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = torch.zeros(n, dtype=torch.float64, device="cuda")
    chi, w = tdvp.op_split(rows, cols, dev(torch, theta), chi_max, w_max, eps, PsiL, V, PsiR, s)
    assert chi == chi_ref
    assert abs(w - w_ref) <= 1e-14 + 1e-12 * w_ref
    sg = s.cpu().numpy()
    assert np.abs(sg - s_ref).max() < 1e-13 * s_ref[0]
    pl = host(PsiL)[: rows * chi].reshape(rows, chi)
    pr = host(PsiR)[: chi * cols].reshape(chi, cols)
    v = V.cpu().numpy()[:chi]
    # FP64 SVDs agree to absolute accuracy ~ eps * lambda_1 (relative only for large values)
    assert np.allclose(1.0 / v, s_ref[:chi], rtol=1e-12, atol=1e-13 * s_ref[0])
    A = pl * v[None, :]
    B = v[:, None] * pr
    assert np.abs(A.conj().T @ A - np.eye(chi)).max() < 1e-12
    assert np.abs(B @ B.conj().T - np.eye(chi)).max() < 1e-12
    rec = (pl * v[None, :]) @ pr
    U, sv, Vh = np.linalg.svd(theta)
    best = (U[:, :chi] * sv[:chi]) @ Vh[:chi]
    assert np.abs(rec - best).max() < 1e-12


@pytest.mark.parametrize("eps", [1e-12, 0.0])
@pytest.mark.parametrize("rows,cols", [(24, 40), (40, 24), (4, 4)])
def test_split_rank_deficient(eps, rows, cols):
    # exact zeros: the numerically-zero values (below 1e-14 ||theta||_F) are
    # dropped even with eps = 0, and the kept vectors are orthonormal
    torch = torch_or_skip()
    tdvp = lib()
    rank = 2 if rows == 4 else 5
    theta, s_true = decaying_matrix(rows, cols, 30, rank=rank)
    n = min(rows, cols)
    PsiL = torch.zeros(rows * n, dtype=torch.complex128, device="cuda")
    PsiR = torch.zeros(n * cols, dtype=torch.complex128, device="cuda")
    V = torch.zeros(n, dtype=torch.float64, device="cuda")
    chi, w = tdvp.op_split(rows, cols, dev(torch, theta), 100, 0.0, eps, PsiL, V, PsiR)
    assert chi == rank and w < 1e-26
    v = V.cpu().numpy()[:rank]
    assert np.allclose(1.0 / v, s_true[:rank], rtol=1e-12)
    A = host(PsiL)[: rows * chi].reshape(rows, chi) * v[None, :]
    B = v[:, None] * host(PsiR)[: chi * cols].reshape(chi, cols)
    assert np.abs(A.conj().T @ A - np.eye(chi)).max() < 1e-12
    assert np.abs(B @ B.conj().T - np.eye(chi)).max() < 1e-12


def gapped_matrix(n, n_big, seed, deg=1):
    """Spectrum of an evolved two-site state: n_big values from 1 down to 6.5e-3
    (the previous bond's Schmidt values), then a tail from 7e-4 down to 4e-6
    (weight the time step moved into new directions); deg > 1 repeats each
    value deg times (symmetry multiplets)."""
    U = np.linalg.qr(I.random_complex((n, n), seed))[0]
    Vh = np.linalg.qr(I.random_complex((n, n), seed + 1))[0]
    big = np.repeat(np.geomspace(1.0, 6.5e-3, n_big // deg), deg)
    tail = np.repeat(np.geomspace(7e-4, 4e-6, (n - n_big) // deg), deg)
    s = np.concatenate([big, tail])
    return (U * s) @ Vh, s


@pytest.mark.parametrize("n,chi_max,w_max,deg", [(160, 80, 0.0, 1), (160, 80, 0.0, 2), (160, 86, 0.0, 1),
                                                  (160, 200, 1e-9, 1), (96, 200, 0.0, 1)])
def test_split_tail_rule(n, chi_max, w_max, deg):
    """Without s_out the SVD skips rotations between vectors that the truncation
    discards; the kept triplets, chi and the discarded weight must not change."""
    torch = torch_or_skip()
    tdvp = lib()
    theta, _ = gapped_matrix(n, n // 2, 90 + deg, deg)
    s_ref = np.linalg.svd(theta, compute_uv=False)
    chi_ref, w_ref = T.truncation_rank(s_ref, chi_max, w_max, 1e-12)
    outs = []
    for with_s in (False, True):
        PsiL = torch.zeros(n * n, dtype=torch.complex128, device="cuda")
        PsiR = torch.zeros(n * n, dtype=torch.complex128, device="cuda")
        V = torch.zeros(n, dtype=torch.float64, device="cuda")
        s = torch.zeros(n, dtype=torch.float64, device="cuda") if with_s else None
        chi, w = tdvp.op_split(n, n, dev(torch, theta), chi_max, w_max, 1e-12, PsiL, V, PsiR, s)
        assert chi == chi_ref
        # singular values agree to ~1e-15 s_1 (absolute): bound on the sum of squares
        assert abs(w - w_ref) <= 1e-12 * w_ref + 2e-15 * s_ref[0] * np.sqrt(n * w_ref) + 1e-28
        v = V.cpu().numpy()[:chi]
        assert np.allclose(1.0 / v, s_ref[:chi], rtol=1e-12, atol=1e-13 * s_ref[0])
        pl = host(PsiL)[: n * chi].reshape(n, chi)
        pr = host(PsiR)[: chi * n].reshape(chi, n)
        A = pl * v[None, :]
        B = v[:, None] * pr
        assert np.abs(A.conj().T @ A - np.eye(chi)).max() < 1e-12
        assert np.abs(B @ B.conj().T - np.eye(chi)).max() < 1e-12
        rec = (pl * v[None, :]) @ pr
        outs.append(rec)
        if deg == 1:  # a unique best rank-chi approximation
            U, sv, Vh = np.linalg.svd(theta)
            best = (U[:, :chi] * sv[:chi]) @ Vh[:chi]
            assert np.abs(rec - best).max() < 1e-12
    assert np.abs(outs[0] - outs[1]).max() < 1e-12


@pytest.mark.parametrize("n,chi_max", [(160, 80), (512, 256)])
def test_split_mixed_precision_path(n, chi_max):
    """The mixed path's SVD (FP32 sweeps, double-float finishing sweeps, FP32
    block-rotation updates of the unitary factor) at the full bond size of the
    benchmark: kept values, isometries and the truncated product to the ~1e-8
    its orthogonality target allows."""
    torch = torch_or_skip()
    tdvp = lib()
    theta, _ = gapped_matrix(n, n // 2, 95)
    s_ref = np.linalg.svd(theta, compute_uv=False)
    chi_ref, w_ref = T.truncation_rank(s_ref, chi_max, 0.0, 1e-12)
    PsiL = torch.zeros(n * n, dtype=torch.complex128, device="cuda")
    PsiR = torch.zeros(n * n, dtype=torch.complex128, device="cuda")
    V = torch.zeros(n, dtype=torch.float64, device="cuda")
    chi, w = tdvp.op_split(n, n, dev(torch, theta), chi_max, 0.0, 1e-12, PsiL, V, PsiR, None, precision=TF32X3)
    assert chi == chi_ref
    # w is a small remainder of ||theta||^2: its error is set by the unitarity
    # of the transformed vectors (~1e-10 here), relative to ||theta||^2
    assert abs(w - w_ref) <= 1e-10 * np.sum(s_ref ** 2)
    v = V.cpu().numpy()[:chi]
    assert np.allclose(1.0 / v, s_ref[:chi], rtol=1e-7, atol=1e-10 * s_ref[0])
    pl = host(PsiL)[: n * chi].reshape(n, chi)
    pr = host(PsiR)[: chi * n].reshape(chi, n)
    A = pl * v[None, :]
    B = v[:, None] * pr
    assert np.abs(A.conj().T @ A - np.eye(chi)).max() < 1e-7
    assert np.abs(B @ B.conj().T - np.eye(chi)).max() < 1e-7
    U, sv, Vh = np.linalg.svd(theta)
    best = (U[:, :chi] * sv[:chi]) @ Vh[:chi]
    assert np.abs((pl * v[None, :]) @ pr - best).max() < 1e-7 * s_ref[0]


@pytest.mark.parametrize("prec", [FP64, TF32X3], ids=["fp64", "tf32x3"])
def test_heff_full_size_sampled(prec):
    """H_eff at the chi = 256, m = 10 (N = 101 Ising, 8 exponentials) size of the
    benchmark, checked on sampled outputs computed one by one."""
    torch = torch_or_skip()
    tdvp = lib()
    x, lam = models.fit_power_law(1.5, 8, 100)
    W = models.build_mpo_site(models.ISING, 1.0, 0.5, x, lam)
    m, d, chi = W.shape[0], 2, 256
    L = hermitian_env((chi, m, chi), 40)
    R = hermitian_env((chi, m, chi), 41)
    th = I.random_complex((chi, d, d, chi), 42)
    y = torch.zeros(th.size, dtype=torch.complex128, device="cuda")
    tdvp.op_heff(prec, 2, chi, chi, m, d, W, dev(torch, L), dev(torch, R), dev(torch, th), y)
    out = host(y).reshape(th.shape)
    rng = np.random.default_rng(43)
    W12 = np.einsum("wvst,vuqr->wusqtr", W, W)  # [w, w'', s1, s2, t1, t2]
    errs = []
    scale = []
    for _ in range(12):
        a, s1, s2, b = rng.integers(chi), rng.integers(d), rng.integers(d), rng.integers(chi)
        # y[a,s1,s2,b] = sum L[a,w,a'] W12[w,w'',s1,s2,t1,t2] R[b,w'',b'] th[a',t1,t2,b']
        X = np.einsum("wx,xtuy->wtuy", L[a], th)                 # [w, t1, t2, b']
        Y = np.einsum("vy,wtuy->wtuv", R[b], X)                  # [w, t1, t2, w'']
        val = np.einsum("wvtu,wtuv->", W12[:, :, s1, s2], Y)
        errs.append(abs(out[a, s1, s2, b] - val))
        scale.append(abs(val))
    assert max(errs) < TOL[prec] * 10 * np.sqrt(np.mean(np.square(scale))), (max(errs), np.mean(scale))
