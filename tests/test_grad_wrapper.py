"""CPU test of the autograd plumbing of paper_1912_06127_gb300/grad.py: the
Function's backward contracts the Jacobian that the forward pass returned with
the incoming gradient (the library call is replaced by a fixed Jacobian)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1912_06127_gb300 import grad as PG  # noqa: E402


class FixedQuench(PG.Quench):
    def run(self, h, J):
        N = self.N
        val = np.arange(N) * h + J
        jac = np.stack([np.arange(N, dtype=float), np.ones(N)], axis=1)   # d/dh, d/dJ
        return val, jac


def test_backward_contracts_the_jacobian():
    q = FixedQuench(kind=0, N=5, alpha=3.0, n_exp=4, dt=0.01, n_steps=1, chi_max=4, basis_state=[0] * 5)
    h = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    J = torch.tensor(1.2, dtype=torch.float64, requires_grad=True)
    out = PG.observable(h, J, q)
    assert torch.allclose(out, torch.arange(5, dtype=torch.float64) * 0.3 + 1.2)
    w = torch.tensor([0.5, -1.0, 2.0, 0.0, 3.0], dtype=torch.float64)
    gh, gJ = torch.autograd.grad((w * out).sum(), (h, J))
    assert abs(float(gh) - float((w * torch.arange(5)).sum())) < 1e-14
    assert abs(float(gJ) - float(w.sum())) < 1e-14
