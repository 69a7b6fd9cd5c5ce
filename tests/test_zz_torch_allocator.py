"""The allocator hook (tdvp_set_allocator): with torch's caching allocator
registered, the library's device memory comes from torch, and a sweep gives the
same observables as with cudaMalloc; blocks are returned through the allocator
that handed them out. The registration checks run on the CPU."""
import gc

import numpy as np
import pytest

import tdvp_inputs as I
from oracle import models

from gpu_util import lib, torch_or_skip


def test_allocator_registration_rules():
    tdvp = lib()
    L = tdvp.lib()
    assert L.tdvp_set_allocator(tdvp._ALLOC(), tdvp._FREE(), None) == 0
    assert L.tdvp_set_allocator(tdvp._ALLOC(lambda n, c: None), tdvp._FREE(), None) == -1


@pytest.mark.gpu
def test_torch_allocator_hook():
    torch = torch_or_skip()
    tdvp = lib()
    N = 8
    x, lam = models.fit_power_law(3.0, 4, N - 1)
    up = I.basis_state("all_up", N)

    def run():
        mpo = tdvp.build_mpo(models.ISING, N, 3.0, 1.0, 1.0, 4, x, lam)
        mps = tdvp.init_mps(N, up, 8)
        tdvp.step(mps, mpo, tdvp.step_params(0.05, 8, krylov_max=10, krylov_tol=0.0), 3)
        return mpo, mps, tdvp.measure(mps, tdvp.OBS_SZ)

    _, _, ref = run()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    tdvp.use_torch_allocator(True)
    try:
        mpo, mps, sz = run()
        during = torch.cuda.memory_allocated()
        del mpo, mps
        gc.collect()
        after = torch.cuda.memory_allocated()
    finally:
        tdvp.use_torch_allocator(False)
    assert during > before            # the library's buffers came from torch
    assert after < during             # and went back to it
    assert np.abs(sz - ref).max() < 1e-13
