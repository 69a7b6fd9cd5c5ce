"""The allocation-free H_eff entry point agrees with the allocating one.

tdvp_op_heff_noalloc serves callers that cannot allocate device memory (a
host application that owns all device memory through its own pool, a
real-time loop that must not enter an allocator): it keeps its intermediates
in a fixed scratch array inside the library. This test calls it through the C ABI twice
in a row -- a two-site problem, then a smaller one-site problem that finds
the first call's data still in the array -- and compares each result with
tdvp_op_heff (FP64) to the tolerance of the other FP64 parity tests. It also
checks that a problem too large for the array is refused with a clear error.
The file is named to be collected last and passes both alone and after the
other GPU tests.
"""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import models

from gpu_util import dev, hermitian_env, host, lib, max_err, torch_or_skip

pytestmark = pytest.mark.gpu


def _problem(nsite, chi_l, chi_r, seed):
    x, lam = models.fit_power_law(1.5, 3, 19)
    W = models.build_mpo_site(models.ISING, 1.0, 0.5, x, lam)
    m, d = W.shape[0], 2
    L = hermitian_env((chi_l, m, chi_l), seed)
    R = hermitian_env((chi_r, m, chi_r), seed + 1)
    shape = (chi_l, d, d, chi_r) if nsite == 2 else (chi_l, d, chi_r)
    th = I.random_complex(shape, seed + 2)
    return W, m, d, L, R, th


def test_noalloc_matches_allocating_entry_point_twice():
    torch = torch_or_skip()
    tdvp = lib()
    for nsite, chi_l, chi_r, seed in ((2, 37, 21, 60), (1, 9, 13, 70)):
        W, m, d, L, R, th = _problem(nsite, chi_l, chi_r, seed)
        Ld, Rd, xd = dev(torch, L), dev(torch, R), dev(torch, th)
        y_ref = torch.zeros(th.size, dtype=torch.complex128, device="cuda")
        y_new = torch.full((th.size,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        tdvp.op_heff(0, nsite, chi_l, chi_r, m, d, W, Ld, Rd, xd, y_ref)
        tdvp.op_heff_noalloc(nsite, chi_l, chi_r, m, d, W, Ld, Rd, xd, y_new)
        a, b = host(y_new), host(y_ref)
        assert np.all(np.isfinite(a))
        assert max_err(a, b) < 1e-12


def test_noalloc_rejects_problem_larger_than_scratch():
    torch = torch_or_skip()
    tdvp = lib()
    x, lam = models.fit_power_law(1.5, 3, 19)
    W = models.build_mpo_site(models.ISING, 1.0, 0.5, x, lam)
    m, d, chi = W.shape[0], 2, 256   # 2 x 256*5*4*256*16 B = 84 MB > 32 MiB
    L = torch.zeros(chi * m * chi, dtype=torch.complex128, device="cuda")
    R = torch.zeros(chi * m * chi, dtype=torch.complex128, device="cuda")
    xv = torch.zeros(chi * d * d * chi, dtype=torch.complex128, device="cuda")
    y = torch.zeros(chi * d * d * chi, dtype=torch.complex128, device="cuda")
    with pytest.raises(tdvp.TdvpError) as e:
        tdvp.op_heff_noalloc(2, chi, chi, m, d, W, L, R, xv, y)
    assert e.value.code == -1 and "scratch" in str(e.value)


def test_noalloc_rejects_large_mpo_bond_dimension_before_building():
    torch = torch_or_skip()
    tdvp = lib()
    m, d, chi = 65, 2, 2
    W = np.zeros((m, m, d, d), complex)
    L = torch.zeros(chi * m * chi, dtype=torch.complex128, device="cuda")
    R = torch.zeros(chi * m * chi, dtype=torch.complex128, device="cuda")
    xv = torch.zeros(chi * d * d * chi, dtype=torch.complex128, device="cuda")
    y = torch.zeros(chi * d * d * chi, dtype=torch.complex128, device="cuda")
    with pytest.raises(tdvp.TdvpError) as e:
        tdvp.op_heff_noalloc(2, chi, chi, m, d, W, L, R, xv, y)
    assert e.value.code == -1 and "TDVP_NOALLOC_MAX_M" in str(e.value)
