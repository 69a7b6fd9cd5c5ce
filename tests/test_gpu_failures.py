"""Failure detection on the GPU, in forms that fault and hang nothing.

The norm-error monitoring of Sec. III D has a device-side counterpart here: the
kernels record NaN, zero norms and given-up waits in a status word that the
host reads after each stage, and the entry points turn it into an error code.
These tests make each failure on the host side -- a NaN or an all-zero tensor
in the caller's input, a NaN model parameter, a grid-barrier wait whose poll
limit is set to zero so that it gives up at once -- and check the code that
comes back, and that the next well-formed call on the same context succeeds.
"""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import models
from oracle import tdvp as T

from gpu_util import dev, lib, max_err, torch_or_skip

pytestmark = pytest.mark.gpu

EINVAL, ENUMERIC, ETIMEOUT = -1, -4, -5


def _healthy_run(tdvp):
    """A short serial run that must succeed after a failure."""
    N = 6
    mpo = tdvp.build_mpo(models.ISING, N, 2.0, 1.0, 0.8, 2)
    mps = tdvp.init_mps(N, I.basis_state("all_up", N), 8)
    tdvp.step(mps, mpo, tdvp.step_params(0.02, 8, krylov_max=10, krylov_tol=0.0), 2)
    assert abs(tdvp.norm(mps) - 1.0) < 1e-10


def test_nan_in_initial_tensors_is_enumeric():
    torch_or_skip()
    tdvp = lib()
    raw = I.random_mps_tensors(8, 4, seed=3)
    raw[3] = raw[3].copy()
    raw[3].flat[5] = complex(np.nan, 0.0)
    with pytest.raises(tdvp.TdvpError) as e:
        tdvp.init_mps_tensors(raw, 8)
    assert e.value.code == ENUMERIC
    _healthy_run(tdvp)


def test_zero_state_is_enumeric():
    torch_or_skip()
    tdvp = lib()
    raw = [np.zeros_like(a) for a in I.random_mps_tensors(6, 3, seed=4)]
    with pytest.raises(tdvp.TdvpError) as e:
        tdvp.init_mps_tensors(raw, 8)
    assert e.value.code == ENUMERIC
    _healthy_run(tdvp)


def test_nan_field_then_step_is_enumeric():
    """A NaN transverse field reaches H_eff in the first local update; the
    Lanczos recurrence sees it and the step returns TDVP_ENUMERIC."""
    torch_or_skip()
    tdvp = lib()
    N = 8
    mpo = tdvp.build_mpo(models.ISING, N, 2.0, 1.0, float("nan"), 2)
    mps = tdvp.init_mps(N, I.basis_state("all_up", N), 8)
    with pytest.raises(tdvp.TdvpError) as e:
        tdvp.step(mps, mpo, tdvp.step_params(0.02, 8, krylov_max=8, krylov_tol=0.0, seg_len=[4, 4]), 1)
    assert e.value.code == ENUMERIC
    _healthy_run(tdvp)


def test_nan_state_in_expm_and_split_is_enumeric():
    torch = torch_or_skip()
    tdvp = lib()
    x, lam = models.fit_power_law(1.5, 3, 19)
    W = models.build_mpo_site(models.ISING, 1.0, 0.5, x, lam)
    m, d, chi = W.shape[0], 2, 12
    L = I.random_complex((chi, m, chi), 30)
    L = 0.5 * (L + L.conj().transpose(2, 1, 0))
    R = I.random_complex((chi, m, chi), 31)
    R = 0.5 * (R + R.conj().transpose(2, 1, 0))
    th = I.random_complex((chi, d, d, chi), 32)
    th.flat[7] = complex(0.0, np.nan)
    y = torch.zeros(th.size, dtype=torch.complex128, device="cuda")
    with pytest.raises(tdvp.TdvpError) as e:
        tdvp.op_expm(0, 2, chi, chi, m, d, W, dev(torch, L), dev(torch, R), dev(torch, th), y, 0.01, 8, 0.0)
    assert e.value.code == ENUMERIC
    n = chi * d
    PsiL = torch.zeros(n * n, dtype=torch.complex128, device="cuda")
    PsiR = torch.zeros(n * n, dtype=torch.complex128, device="cuda")
    V = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(tdvp.TdvpError) as e:
        tdvp.op_split(n, n, dev(torch, th.reshape(n, n)), n, 0.0, 1e-12, PsiL, V, PsiR)
    assert e.value.code == ENUMERIC
    _healthy_run(tdvp)


def test_nan_time_step_is_rejected():
    torch_or_skip()
    tdvp = lib()
    N = 6
    mpo = tdvp.build_mpo(models.ISING, N, 2.0, 1.0, 0.8, 2)
    mps = tdvp.init_mps(N, I.basis_state("all_up", N), 8)
    with pytest.raises(tdvp.TdvpError) as e:
        tdvp.step(mps, mpo, tdvp.step_params(float("nan"), 8), 1)
    assert e.value.code == EINVAL


def test_grid_barrier_wait_gives_up_and_returns_etimeout():
    """With a poll limit of zero, the first block of the SVD's cooperative
    Jacobi launch to reach a grid barrier gives up at once (a 512 x 512 split
    runs 16 blocks, so some block always waits), raises the abort word that
    sends every other block home at its next barrier, and the split returns
    TDVP_ETIMEOUT. With the default limit restored, the same split succeeds
    and agrees with LAPACK."""
    torch = torch_or_skip()
    tdvp = lib()
    n = 512
    U = np.linalg.qr(I.random_complex((n, n), 33))[0]
    Vh = np.linalg.qr(I.random_complex((n, n), 34))[0]
    s = 0.97 ** np.arange(n)
    theta = (U * s) @ Vh
    PsiL = torch.zeros(n * n, dtype=torch.complex128, device="cuda")
    PsiR = torch.zeros(n * n, dtype=torch.complex128, device="cuda")
    V = torch.zeros(n, dtype=torch.float64, device="cuda")
    th = dev(torch, theta)
    try:
        tdvp.set_wait_limit(0)
        with pytest.raises(tdvp.TdvpError) as e:
            tdvp.op_split(n, n, th, 256, 0.0, 1e-12, PsiL, V, PsiR)
        assert e.value.code == ETIMEOUT
    finally:
        tdvp.set_wait_limit(-1)
    s_out = torch.zeros(n, dtype=torch.float64, device="cuda")
    chi, w = tdvp.op_split(n, n, th, 256, 0.0, 1e-12, PsiL, V, PsiR, s_out)
    chi_ref, w_ref = T.truncation_rank(s, 256, 0.0, 1e-12)
    assert chi == chi_ref
    assert max_err(s_out.cpu().numpy(), s) < 1e-13
    _healthy_run(tdvp)
