"""The GEMM tile autotuner changes speed, not results.

Its candidates (tcgen05 N tiles of 256 and 128; SIMT tiles of 64 x 64 and
32 x 32) compute every output element with the same operations in the same
order, so the kernel-level results and a whole mixed-precision step must be
bitwise the same with tuning on and off; the tuner must have recorded a
decision for every family it met.
"""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import models

from gpu_util import dev, hermitian_env, host, lib, torch_or_skip

pytestmark = pytest.mark.gpu


def _heff_all(tdvp, torch, chi_l, chi_r):
    x, lam = models.fit_power_law(1.5, 8, 100)
    W = models.build_mpo_site(models.ISING, 1.0, 0.5, x, lam)
    m, d = W.shape[0], 2
    L = hermitian_env((chi_l, m, chi_l), 50)
    R = hermitian_env((chi_r, m, chi_r), 51)
    th = I.random_complex((chi_l, d, d, chi_r), 52)
    out = []
    for prec in (0, 1, 2):
        y = torch.zeros(th.size, dtype=torch.complex128, device="cuda")
        tdvp.op_heff(prec, 2, chi_l, chi_r, m, d, W, dev(torch, L), dev(torch, R), dev(torch, th), y)
        out.append(host(y))
    return out


def test_tuned_kernels_give_the_same_bits():
    torch = torch_or_skip()
    tdvp = lib()
    try:
        for chi_l, chi_r in ((33, 64), (128, 96), (256, 256)):
            tdvp.set_autotune(False)
            ref = _heff_all(tdvp, torch, chi_l, chi_r)
            tdvp.set_autotune(True)
            first = _heff_all(tdvp, torch, chi_l, chi_r)   # tunes (runs every candidate)
            again = _heff_all(tdvp, torch, chi_l, chi_r)   # uses the decisions
            for a, b, c in zip(ref, first, again):
                assert np.array_equal(a, b) and np.array_equal(a, c)
        fams = {r["family"] for r in tdvp.autotune_report()}
        assert {"tc_gemm_tf32", "tc_gemm_tf32x3", "zgemm_fp64"} <= fams
        for r in tdvp.autotune_report():
            assert r["choice"] in ("BN256", "BN128", "64x64", "32x32") and len(r["us"]) == 2
    finally:
        tdvp.set_autotune(True)


def test_tuned_step_gives_the_same_bits():
    torch_or_skip()
    tdvp = lib()
    N, chi = 21, 32
    x, lam = models.fit_power_law(1.5, 8, N - 1)
    mpo = tdvp.build_mpo(models.ISING, N, 1.5, 1.0, 0.5, 8, x, lam)
    raw = I.random_mps_tensors(N, chi, seed=9)
    out = []
    try:
        for k in range(3):
            if k < 2:
                tdvp.set_autotune(k == 1)   # off; then on (the third run reuses the decisions)
            mps = tdvp.init_mps_tensors(raw, chi, 1e-14)
            p = tdvp.step_params(dt=0.01, chi_max=chi, krylov_max=8, krylov_tol=0.0, precision=I.TF32X3,
                                 seg_len=[6, 5, 5, 5])
            tdvp.step(mps, mpo, p, 2)
            out.append(tdvp.measure(mps, tdvp.OBS_SZ))
        assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    finally:
        tdvp.set_autotune(True)
