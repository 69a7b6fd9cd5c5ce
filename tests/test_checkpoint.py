"""CPU tests of the checkpoint format (paper_1912_06127_gb300/checkpoint.py):
arrays and metadata survive a round trip, inconsistent files are refused, and
the raw tensors a resume hands to the library represent the saved state (checked
with the oracle's canonicalisation and dense vectors)."""
import numpy as np
import pytest

import tdvp_inputs as I
from oracle import mps as M
from paper_1912_06127_gb300 import checkpoint as C


def test_round_trip_and_state(tmp_path):
    st = M.canonicalize(I.random_mps_tensors(7, 4, seed=3), 6)
    p = str(tmp_path / "s.npz")
    C.write_arrays(p, st.Psi, st.V, {"step": 12, "t": 0.24, "model": {"kind": 0, "h": 1.0}})
    sites, bonds, meta = C.read_arrays(p)
    assert meta["step"] == 12 and meta["model"]["h"] == 1.0 and meta["N"] == 7
    for a, b in zip(sites + bonds, st.Psi + st.V):
        assert np.array_equal(a, b)
    back = M.canonicalize(C.raw_tensors(sites, bonds), 6)
    v0, v1 = M.to_dense(st), M.to_dense(back)
    assert abs(abs(np.vdot(v0, v1)) - np.linalg.norm(v0) * np.linalg.norm(v1)) < 1e-12
    assert back.bond_dims() == st.bond_dims()


def test_inconsistent_files_are_refused(tmp_path):
    st = M.canonicalize(I.random_mps_tensors(5, 2, seed=1), 4)
    p = str(tmp_path / "bad.npz")
    bonds = list(st.V)
    bonds[1] = np.concatenate([bonds[1], [1.0]])
    C.write_arrays(p, st.Psi, bonds, {})
    with pytest.raises(ValueError):
        C.read_arrays(p)
    q = str(tmp_path / "other.npz")
    np.savez(q, header=np.frombuffer(b'{"format": "x"}', dtype=np.uint8))
    with pytest.raises(ValueError):
        C.read_arrays(q)
