"""Checkpoint and resume of a state (Psi_j, V_j, chi_j) with its metadata.

The paper re-ran its final 201-site state for an extra time step, i.e. it saved
and reloaded states. A checkpoint holds the site tensors Psi_j and the bond
vectors V_j = 1/Lambda_j of the inverse canonical gauge (Sec. II B) as read
back from the library, and free-form metadata (model parameters, step counter,
time). Resuming builds the raw tensors Psi_j V_j (the last site as it is) and
hands them to tdvp_init_mps_tensors, which brings them to the inverse canonical
gauge again; environments are rebuilt on the first step (as after a
reorthonormalisation, Sec. III D).
"""
from __future__ import annotations

import json
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import tdvp

FORMAT = "tdvp-mps-checkpoint-1"


def write_arrays(path: str, sites: Sequence[np.ndarray], bonds: Sequence[np.ndarray], meta: Dict) -> None:
    """Host arrays to an .npz file (site j as site_j, bond j as bond_j)."""
    arrays = {"site_%d" % j: np.ascontiguousarray(s, dtype=np.complex128) for j, s in enumerate(sites)}
    arrays.update({"bond_%d" % j: np.ascontiguousarray(b, dtype=np.float64) for j, b in enumerate(bonds)})
    header = dict(meta)
    header["format"] = FORMAT
    header["N"] = len(sites)
    arrays["header"] = np.frombuffer(json.dumps(header).encode(), dtype=np.uint8)
    with open(path, "wb") as fh:
        np.savez(fh, **arrays)


def read_arrays(path: str) -> Tuple[List[np.ndarray], List[np.ndarray], Dict]:
    with np.load(path) as z:
        header = json.loads(bytes(z["header"]).decode())
        if header.get("format") != FORMAT:
            raise ValueError("not a checkpoint of this library: %r" % header.get("format"))
        N = int(header["N"])
        sites = [z["site_%d" % j].copy() for j in range(N)]
        bonds = [z["bond_%d" % j].copy() for j in range(N - 1)]
    for j in range(N - 1):
        if sites[j].shape[2] != len(bonds[j]) or sites[j + 1].shape[0] != len(bonds[j]):
            raise ValueError("inconsistent bond dimension at bond %d" % j)
    return sites, bonds, header


def raw_tensors(sites: Sequence[np.ndarray], bonds: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Psi_j V_j for j < N-1 and Psi_N: the state |psi> = M_1 ... M_N in any gauge."""
    out = [sites[j] * bonds[j][None, None, :] for j in range(len(bonds))]
    out.append(np.asarray(sites[-1]))
    return out


def save(path: str, mps: "tdvp.Mps", **meta) -> None:
    N, _ = mps.size()
    write_arrays(path, [mps.site(j) for j in range(N)], [mps.bond(j) for j in range(N - 1)], meta)


def load(path: str, chi_cap: int) -> Tuple["tdvp.Mps", Dict]:
    sites, bonds, header = read_arrays(path)
    return tdvp.init_mps_tensors(raw_tensors(sites, bonds), chi_cap, 1e-14), header
