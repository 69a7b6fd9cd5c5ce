"""GPU parity of the derivative d<O_j(t)>/d(h, J) (tdvp_step_tangent).

Against the oracle's forward-mode derivative (oracle/grad.py: exact local
exponentials, torch's SVD derivative) on truncated runs with and without
segments, to 1e-6 relative (expected ~1e-9: the GPU exponentials are Lanczos
runs converged to rounding, the Frechet integral a 6-point Gauss-Legendre
rule, and the GPU SVD derivative the closed form at fixed kept rank). Against
central differences (step 1e-5) of tdvp_step itself on a product-state quench
with growing bonds; and through the torch.autograd.Function.
"""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import grad as G
from oracle import models
from oracle import mps as M
from oracle import tdvp as T
from oracle.models import ISING, XY

from gpu_util import lib, torch_or_skip

pytestmark = pytest.mark.gpu


def gpu_quench(tdvp, kind, N, alpha, K, x, lam, J, h, init, chi, dt, n_steps, eps=1e-12, kmax=24, tol=0.0,
               seg=None, obs=None, n_quad=6):
    mpo = tdvp.build_mpo(kind, N, alpha, J, h, K, x, lam)
    dm = [tdvp.build_mpo_derivative(mpo, tdvp.PARAM_H), tdvp.build_mpo_derivative(mpo, tdvp.PARAM_J)]
    mps = tdvp.init_mps_tensors(init, chi, 1e-14) if isinstance(init, list) else tdvp.init_mps(N, init, chi)
    tan = tdvp.Tangent(mps, 2)
    p = tdvp.step_params(dt, chi, eps=eps, krylov_max=kmax, krylov_tol=tol, seg_len=seg)
    tdvp.step_tangent(mps, mpo, tan, dm, p, n_steps, n_quad=n_quad)
    val, der = tdvp.measure_tangent(mps, tan, tdvp.OBS_SZ if obs is None else obs)
    return val, der.T, mps


def gpu_plain(tdvp, kind, N, alpha, K, x, lam, J, h, init, chi, dt, n_steps, eps=1e-12, kmax=24, tol=0.0,
              seg=None, obs=None):
    mpo = tdvp.build_mpo(kind, N, alpha, J, h, K, x, lam)
    mps = tdvp.init_mps_tensors(init, chi, 1e-14) if isinstance(init, list) else tdvp.init_mps(N, init, chi)
    p = tdvp.step_params(dt, chi, eps=eps, krylov_max=kmax, krylov_tol=tol, seg_len=seg)
    tdvp.step(mps, mpo, p, n_steps)
    return tdvp.measure(mps, tdvp.OBS_SZ if obs is None else obs), list(mps.bond_dims())


@pytest.mark.parametrize("kind,seg,obs", [(ISING, None, "z"), (ISING, [4, 4], "x"), (XY, [3, 5], "z"),
                                          (ISING, None, "y")])
def test_tangent_matches_oracle_jacobian(kind, seg, obs):
    torch_or_skip()
    tdvp = lib()
    N, alpha, K, J, h = 8, 2.5, 3, 1.0, 0.6
    x, lam = models.fit_power_law(alpha, K, N - 1)
    raw = I.random_mps_tensors(N, 3, seed=5)
    mps0 = M.canonicalize(raw, 6, 1e-14)
    p = T.Params(dt=0.04, chi_max=6, eps=1e-12, krylov_max=24, krylov_tol=0.0, seg_len=seg)
    oval, ojac, _ = G.jacobian(kind, x, lam, J, h, mps0, p, 3, obs)
    code = {"z": tdvp.OBS_SZ, "x": tdvp.OBS_SX, "y": tdvp.OBS_SY}[obs]
    val, jac, mps = gpu_quench(tdvp, kind, N, alpha, K, x, lam, J, h, raw, 6, 0.04, 3, seg=seg, obs=code)
    assert np.abs(val - oval).max() < 1e-10
    scale = np.abs(ojac).max()
    assert scale > 1e-3
    err = np.abs(jac - ojac).max() / scale
    assert err < 1e-6, err


def test_tangent_matches_gpu_central_differences():
    torch_or_skip()
    tdvp = lib()
    N, alpha, K, J, h, chi, dt, n = 16, 3.0, 6, 1.0, 1.0, 12, 0.02, 12
    x, lam = models.fit_power_law(alpha, K, N - 1)
    up = I.basis_state("all_up", N)
    val, jac, mps = gpu_quench(tdvp, ISING, N, alpha, K, x, lam, J, h, up, chi, dt, n, tol=1e-13)
    dims = list(mps.bond_dims())
    assert max(dims) == chi                       # truncation active in the middle
    d = 1e-5
    for c, (dh, dJ) in enumerate(((d, 0.0), (0.0, d))):
        plus, dp = gpu_plain(tdvp, ISING, N, alpha, K, x, lam, J + dJ, h + dh, up, chi, dt, n, tol=1e-13)
        minus, dm = gpu_plain(tdvp, ISING, N, alpha, K, x, lam, J - dJ, h - dh, up, chi, dt, n, tol=1e-13)
        assert dp == dims and dm == dims          # fixed truncation
        fd = (plus - minus) / (2 * d)
        scale = np.abs(fd).max()
        assert scale > 1e-3
        assert np.abs(jac[:, c] - fd).max() < 1e-6 * scale, (c, np.abs(jac[:, c] - fd).max() / scale)


def test_primal_of_tangent_step_is_tdvp_step():
    torch_or_skip()
    tdvp = lib()
    N, alpha, K = 10, 2.0, 4
    x, lam = models.fit_power_law(alpha, K, N - 1)
    up = I.basis_state("all_up", N)
    val, _, mps = gpu_quench(tdvp, ISING, N, alpha, K, x, lam, 1.0, 0.8, up, 8, 0.02, 5, seg=[5, 5])
    ref, dims = gpu_plain(tdvp, ISING, N, alpha, K, x, lam, 1.0, 0.8, up, 8, 0.02, 5, seg=[5, 5])
    assert list(mps.bond_dims()) == dims
    assert np.abs(val - ref).max() < 1e-12


def test_autograd_function():
    torch = torch_or_skip()
    from paper_1912_06127_gb300 import grad as PG
    tdvp = lib()
    N = 8
    q = PG.Quench(kind=ISING, N=N, alpha=3.0, n_exp=4, dt=0.02, n_steps=5, chi_max=8,
                  basis_state=I.basis_state("all_up", N), krylov_max=24, krylov_tol=0.0)
    h = torch.tensor(0.9, dtype=torch.float64, requires_grad=True)
    J = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    out = PG.observable(h, J, q)
    loss = out[N // 2]
    gh, gJ = torch.autograd.grad(loss, (h, J))
    val, jac = q.run(0.9, 1.0)
    assert abs(float(loss) - val[N // 2]) < 1e-14
    assert abs(float(gh) - jac[N // 2, 0]) < 1e-14 and abs(float(gJ) - jac[N // 2, 1]) < 1e-14
    # central differences of the forward pass
    d = 1e-5
    fd = (q.run(0.9 + d, 1.0)[0][N // 2] - q.run(0.9 - d, 1.0)[0][N // 2]) / (2 * d)
    assert abs(float(gh) - fd) < 1e-6 * max(1e-3, abs(fd))
