"""Helpers for the GPU parity tests: build/load the library, move seeded
inputs to the device, and compare with the oracle."""
import numpy as np
import pytest

import tdvp_inputs as I


def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_06127_gb300 import tdvp
    return tdvp


def torch_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def host(t):
    return t.cpu().numpy()


def hermitian_env(shape, seed):
    """Random environment [chi, m, chi] whose slices env[:, w, :] are Hermitian
    (as for a Hermitian MPO), seeded."""
    a = I.random_complex(shape, seed)
    return 0.5 * (a + a.conj().transpose(2, 1, 0))


def max_err(a, b):
    """Element-wise error of `a` against the reference `b`: max |a - b| over
    all elements, relative to max |b|. Every element is checked at the scale
    of the largest one, so a wrong or missing tile fails even where its
    entries are small."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    assert a.shape == b.shape, (a.shape, b.shape)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
