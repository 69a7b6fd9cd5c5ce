"""Plain FP64 CPU oracle of parallel two-site TDVP (test infrastructure).

This package is test infrastructure. Only `tests/`, `__graft_entry__.smoke()`
and the `cpu_baseline` / `--impl reference` legs of `bench.py` may import it.
The product path (the CUDA library and its Python binding) never imports it,
and it never imports the product path. The two share nothing except the
seeded input module `tdvp_inputs`, which holds no arithmetic of the method.

Every function is written for clarity against the paper, not for speed:
explicit einsum contractions, numpy's LAPACK SVD, a plain Lanczos loop.

Modules
  models  -- Pauli operators, power-law fit (Sec. II C), MPO (Sec. II C), dense H
  mps     -- inverse canonical gauge state (Sec. II B), measurement, overlap
  tdvp    -- environments (Fig. 3), H_eff (Fig. 4), Lanczos exponential (Eq. 18/20),
             truncated split (Fig. 5, Sec. III C/D), serial and segmented sweeps
             (Sec. III A/B, App. A/B)
  ed      -- exact diagonalisation of the dense 2^N Hamiltonian
  dmrg    -- two-site DMRG ground states with the same building blocks
  tdvp1   -- one-site TDVP (Eq. proj1site) and the hybrid two-site -> one-site scheme
  grad    -- d<O_j(t)>/d(h, J) of the sweep: the same steps in PyTorch FP64 CPU
             operations, differentiated by forward-mode automatic differentiation

Parity status: every function is pinned by a test in tests/test_oracle_*.py
against a closed form, a brute-force dense calculation or exact
diagonalisation, except where a docstring says "parity unpinned".
"""
