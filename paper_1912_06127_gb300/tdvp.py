"""Thin ctypes binding of libtdvp (include/tdvp.h); argument marshalling only.

Every computation runs inside the CUDA library. PyTorch is used for device
buffers and streams of the kernel-level calls (tensors are passed by their
data pointers). The functions keep the C names without the `tdvp_` prefix.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdvp.so")

ISING, XY, XXX = 0, 1, 2
FP64, TF32, TF32X3 = 0, 1, 2
OBS_SZ, OBS_SX, OBS_SY = 0, 1, 2
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENUMERIC", -5: "ETIMEOUT", -6: "ESTATE"}


class TdvpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class Model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("N", ctypes.c_int), ("alpha", ctypes.c_double),
                ("J", ctypes.c_double), ("h", ctypes.c_double), ("n_exp", ctypes.c_int),
                ("x", ctypes.POINTER(ctypes.c_double)), ("lam", ctypes.POINTER(ctypes.c_double))]


class StepParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("chi_max", ctypes.c_int), ("w_max", ctypes.c_double),
                ("eps", ctypes.c_double), ("krylov_max", ctypes.c_int), ("krylov_tol", ctypes.c_double),
                ("precision", ctypes.c_int), ("n_seg", ctypes.c_int),
                ("seg_len", ctypes.POINTER(ctypes.c_int)), ("merge_turning", ctypes.c_int)]


class StepStats(ctypes.Structure):
    _fields_ = [("w_total", ctypes.c_double), ("chi_max_seen", ctypes.c_int), ("n_stages", ctypes.c_int),
                ("krylov_vectors", ctypes.c_int64), ("n_fwd2", ctypes.c_int64), ("n_back1", ctypes.c_int64),
                ("heff_flops", ctypes.c_double), ("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class DmrgParams(ctypes.Structure):
    _fields_ = [("chi_max", ctypes.c_int), ("w_max", ctypes.c_double), ("eps", ctypes.c_double),
                ("krylov_max", ctypes.c_int), ("krylov_tol", ctypes.c_double), ("precision", ctypes.c_int)]


class DmrgStats(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("w_total", ctypes.c_double), ("chi_max_seen", ctypes.c_int),
                ("krylov_vectors", ctypes.c_int64), ("n_updates", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p
_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_allocator_keep = None  # the registered callbacks must outlive their use
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    """Load libtdvp.so (built by `__graft_entry__.build()`); fails loudly if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libtdvp.so is not built (run __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "tdvp_last_error": ([], ctypes.c_char_p),
        "tdvp_version": ([], ctypes.c_char_p),
        "tdvp_device_ok": ([], ctypes.c_int),
        "tdvp_set_allocator": ([_ALLOC, _FREE, _P], ctypes.c_int),
        "tdvp_fit_power_law": ([ctypes.c_double, ctypes.c_int, ctypes.c_int, _D, _D], ctypes.c_int),
        "tdvp_build_mpo": ([ctypes.POINTER(Model), ctypes.POINTER(_P)], ctypes.c_int),
        "tdvp_couplings": ([ctypes.c_int, _D, _D, ctypes.c_int, _D], ctypes.c_int),
        "tdvp_mpo_couplings": ([_P, ctypes.c_int, _D], ctypes.c_int),
        "tdvp_fit_power_law_lm": ([ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D],
                                  ctypes.c_int),
        "tdvp_mpo_dims": ([_P, _I, _I], ctypes.c_int),
        "tdvp_mpo_tensor": ([_P, _D, _D, _D], ctypes.c_int),
        "tdvp_free_mpo": ([_P], None),
        "tdvp_init_mps": ([ctypes.c_int, ctypes.c_int, _I, ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
        "tdvp_init_mps_tensors": ([ctypes.c_int, ctypes.c_int, _I, ctypes.POINTER(_D), ctypes.c_int,
                                   ctypes.c_double, ctypes.POINTER(_P)], ctypes.c_int),
        "tdvp_mps_bond_dims": ([_P, _I], ctypes.c_int),
        "tdvp_mps_get_site": ([_P, ctypes.c_int, _D], ctypes.c_int),
        "tdvp_mps_get_bond": ([_P, ctypes.c_int, _D], ctypes.c_int),
        "tdvp_mps_size": ([_P, _I, _I], ctypes.c_int),
        "tdvp_free_mps": ([_P], None),
        "tdvp_step": ([_P, _P, ctypes.POINTER(StepParams), ctypes.c_int, ctypes.POINTER(StepStats), _P],
                      ctypes.c_int),
        "tdvp_measure": ([_P, ctypes.c_int, _D], ctypes.c_int),
        "tdvp_step1": ([_P, _P, ctypes.POINTER(StepParams), ctypes.c_int, ctypes.POINTER(StepStats), _P],
                       ctypes.c_int),
        "tdvp_step_hybrid": ([_P, _P, ctypes.POINTER(StepParams), ctypes.c_int, ctypes.POINTER(StepStats), _P],
                             ctypes.c_int),
        "tdvp_reorthonormalize": ([_P, ctypes.c_double], ctypes.c_int),
        "tdvp_dmrg": ([_P, _P, ctypes.POINTER(DmrgParams), ctypes.c_int, ctypes.POINTER(DmrgStats), _P],
                      ctypes.c_int),
        "tdvp_norm": ([_P, _D], ctypes.c_int),
        "tdvp_energy": ([_P, _P, _D], ctypes.c_int),
        "tdvp_overlap": ([_P, _P, _D], ctypes.c_int),
        "tdvp_op_heff": ([ctypes.c_int] * 6 + [_D, _P, _P, _P, _P, _P], ctypes.c_int),
        "tdvp_op_env": ([ctypes.c_int] * 6 + [_D, _P, _P, _P, _P], ctypes.c_int),
        "tdvp_op_expm": ([ctypes.c_int] * 6 + [_D, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_double, _I, _P], ctypes.c_int),
        "tdvp_op_split": ([ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                           _P, _P, _P, _P, _I, _D, _P], ctypes.c_int),
        "tdvp_op_split_prec": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                           _P, _P, _P, _P, _I, _D, _P], ctypes.c_int),
        "tdvp_schedule": ([ctypes.c_int, ctypes.c_int, _I, ctypes.c_int, ctypes.c_int, _I, ctypes.c_int],
                          ctypes.c_int),
        "tdvp_schedule1": ([ctypes.c_int, ctypes.c_int, _I, ctypes.c_int, ctypes.c_int, _I, ctypes.c_int],
                           ctypes.c_int),
        "tdvp_exchange_plan": ([ctypes.c_int, ctypes.c_int, _I, _I, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I,
                                ctypes.c_int], ctypes.c_int),
        "tdvp_tridiag_expm": ([ctypes.c_int, _D, _D, ctypes.c_double, _D], ctypes.c_int),
        "tdvp_profile": ([ctypes.c_int], ctypes.c_int),
        "tdvp_profile_read_aux": ([ctypes.c_int, _D], ctypes.c_int),
        "tdvp_op_heff_noalloc": ([ctypes.c_int] * 5 + [_D, _P, _P, _P, _P, _P], ctypes.c_int),
        "tdvp_set_wait_limit": ([ctypes.c_longlong], ctypes.c_int),
        "tdvp_set_autotune": ([ctypes.c_int], ctypes.c_int),
        "tdvp_set_env_tensor_cores": ([ctypes.c_int], ctypes.c_int),
        "tdvp_autotune_report": ([ctypes.c_char_p, ctypes.c_int], ctypes.c_int),
        "tdvp_profile_read": ([ctypes.c_int, ctypes.c_char_p, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int64),
                               _D, _D], ctypes.c_int),
        "tdvp_build_mpo_derivative": ([_P, ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
        "tdvp_tangent_create": ([_P, ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
        "tdvp_free_tangent": ([_P], None),
        "tdvp_step_tangent": ([_P, _P, _P, ctypes.POINTER(_P), ctypes.POINTER(StepParams), ctypes.c_int,
                               ctypes.c_int, ctypes.POINTER(StepStats), _P], ctypes.c_int),
        "tdvp_measure_tangent": ([_P, _P, ctypes.c_int, _D, _D], ctypes.c_int),
        "tdvp_gauss_legendre": ([ctypes.c_int, _D, _D], ctypes.c_int),
        "tdvp_mps_copy": ([_P, ctypes.POINTER(_P)], ctypes.c_int),
        "tdvp_apply_site_op": ([_P, ctypes.c_int, _D], ctypes.c_int),
        "tdvp_expect_mixed": ([_P, _P, ctypes.c_int, _D], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device memory through torch's caching allocator
    (enable=False: back to cudaMalloc / cudaFree for new blocks). Blocks taken
    from torch go back to torch when their handle is released, so release the
    library's handles while torch is still alive (not at interpreter exit)."""
    global _allocator_keep
    if not enable:
        _check(lib().tdvp_set_allocator(_ALLOC(), _FREE(), None))
        return
    import torch

    def alloc(n, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(n)))
        except Exception:
            return None

    def free(p, ctx):
        torch.cuda.caching_allocator_delete(p)

    cbs = (_ALLOC(alloc), _FREE(free))
    _check(lib().tdvp_set_allocator(cbs[0], cbs[1], None))
    _allocator_keep = (cbs, _allocator_keep)  # earlier callbacks may still own blocks


def last_error() -> str:
    return lib().tdvp_last_error().decode()


def version() -> str:
    return lib().tdvp_version().decode()


def device_ok() -> bool:
    return bool(lib().tdvp_device_ok())


def _check(rc: int) -> int:
    if rc < 0:
        raise TdvpError(rc, last_error())
    return rc


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _cplx_out(n: int) -> np.ndarray:
    return np.zeros(n, dtype=np.complex128)


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _ptr(t) -> int:
    """Device pointer of a contiguous torch tensor (complex128 / float64 / int32)."""
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return t.data_ptr()


# ---------------------------------------------------------------------------
def fit_power_law(alpha: float, n_exp: int, r_max: int):
    x = _cplx_out(n_exp)
    lam = _cplx_out(n_exp)
    _check(lib().tdvp_fit_power_law(alpha, n_exp, r_max, _dptr(x.view(np.float64)), _dptr(lam.view(np.float64))))
    return x, lam


def fit_power_law_lm(alpha: float, n_exp: int, r_max: int, relative: bool = True):
    """(x, lam, rms) of the Levenberg-Marquardt fit of r^-alpha on r = 1..r_max."""
    x = _cplx_out(n_exp)
    lam = _cplx_out(n_exp)
    rms = ctypes.c_double(0.0)
    _check(lib().tdvp_fit_power_law_lm(alpha, n_exp, r_max, 1 if relative else 0, _dptr(x.view(np.float64)),
                                       _dptr(lam.view(np.float64)), ctypes.byref(rms)))
    return x, lam, rms.value


def couplings(x: np.ndarray, lam: np.ndarray, r_max: int) -> np.ndarray:
    """V(r) = sum_k x_k lam_k^r for r = 1..r_max (complex)."""
    xa = np.ascontiguousarray(x, dtype=np.complex128)
    la = np.ascontiguousarray(lam, dtype=np.complex128)
    out = _cplx_out(r_max)
    _check(lib().tdvp_couplings(len(xa), _dptr(xa.view(np.float64)), _dptr(la.view(np.float64)), r_max,
                                _dptr(out.view(np.float64))))
    return out


class Mpo:
    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tdvp_free_mpo(self.handle)
            self.handle = None

    def dims(self):
        m, d = ctypes.c_int(), ctypes.c_int()
        _check(lib().tdvp_mpo_dims(self.handle, ctypes.byref(m), ctypes.byref(d)))
        return m.value, d.value

    def couplings(self, r_max: int) -> np.ndarray:
        out = _cplx_out(r_max)
        _check(lib().tdvp_mpo_couplings(self.handle, r_max, _dptr(out.view(np.float64))))
        return out

    def tensor(self, n_exp: int):
        m, d = self.dims()
        W = _cplx_out(m * m * d * d)
        x = _cplx_out(n_exp)
        lam = _cplx_out(n_exp)
        _check(lib().tdvp_mpo_tensor(self.handle, _dptr(W.view(np.float64)), _dptr(x.view(np.float64)),
                                     _dptr(lam.view(np.float64))))
        return W.reshape(m, m, d, d), x, lam


def build_mpo(kind: int, N: int, alpha: float, J: float, h: float, n_exp: int,
              x: Optional[np.ndarray] = None, lam: Optional[np.ndarray] = None) -> Mpo:
    m = Model(kind, N, alpha, J, h, n_exp, None, None)
    keep = []
    if x is not None and lam is not None:
        xa = np.ascontiguousarray(x, dtype=np.complex128)
        la = np.ascontiguousarray(lam, dtype=np.complex128)
        keep = [xa, la]
        m.x = _dptr(xa.view(np.float64))
        m.lam = _dptr(la.view(np.float64))
    h_ = ctypes.c_void_p()
    _check(lib().tdvp_build_mpo(ctypes.byref(m), ctypes.byref(h_)))
    del keep
    return Mpo(h_)


class Mps:
    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tdvp_free_mps(self.handle)
            self.handle = None

    def size(self):
        N, d = ctypes.c_int(), ctypes.c_int()
        _check(lib().tdvp_mps_size(self.handle, ctypes.byref(N), ctypes.byref(d)))
        return N.value, d.value

    def bond_dims(self) -> np.ndarray:
        N, _ = self.size()
        out = np.zeros(N - 1, dtype=np.int32)
        _check(lib().tdvp_mps_bond_dims(self.handle, out.ctypes.data_as(_I)))
        return out

    def site(self, j: int) -> np.ndarray:
        N, d = self.size()
        dims = [1] + list(self.bond_dims()) + [1]
        out = _cplx_out(dims[j] * d * dims[j + 1])
        _check(lib().tdvp_mps_get_site(self.handle, j, _dptr(out.view(np.float64))))
        return out.reshape(dims[j], d, dims[j + 1])

    def bond(self, j: int) -> np.ndarray:
        out = np.zeros(int(self.bond_dims()[j]), dtype=np.float64)
        _check(lib().tdvp_mps_get_bond(self.handle, j, _dptr(out)))
        return out


def init_mps(N: int, basis_state: Sequence[int], chi_cap: int, d: int = 2) -> Mps:
    s = np.ascontiguousarray(basis_state, dtype=np.int32)
    h_ = ctypes.c_void_p()
    _check(lib().tdvp_init_mps(N, d, s.ctypes.data_as(_I), chi_cap, ctypes.byref(h_)))
    return Mps(h_)


def init_mps_tensors(tensors: Sequence[np.ndarray], chi_cap: int, eps: float = 1e-14) -> Mps:
    N = len(tensors)
    d = tensors[0].shape[1]
    dims = np.array([t.shape[0] for t in tensors] + [tensors[-1].shape[2]], dtype=np.int32)
    arrs = [np.ascontiguousarray(t, dtype=np.complex128) for t in tensors]
    ptrs = (_D * N)(*[_dptr(a.view(np.float64)) for a in arrs])
    h_ = ctypes.c_void_p()
    _check(lib().tdvp_init_mps_tensors(N, d, dims.ctypes.data_as(_I), ptrs, chi_cap, eps, ctypes.byref(h_)))
    return Mps(h_)


def step_params(dt: float, chi_max: int, w_max: float = 0.0, eps: float = 1e-12, krylov_max: int = 8,
                krylov_tol: float = 1e-6, precision: int = FP64, seg_len: Optional[Sequence[int]] = None,
                merge_turning: int = 1):
    seg = np.ascontiguousarray(seg_len if seg_len else [], dtype=np.int32)
    p = StepParams(dt, chi_max, w_max, eps, krylov_max, krylov_tol, precision, len(seg),
                   seg.ctypes.data_as(_I) if len(seg) else None, merge_turning)
    p._seg = seg  # keep alive
    return p


def step(mps: Mps, mpo: Mpo, params: StepParams, n_steps: int = 1, stream=None,
         stats: Optional[StepStats] = None) -> StepStats:
    st = stats if stats is not None else StepStats()
    _check(lib().tdvp_step(mps.handle, mpo.handle, ctypes.byref(params), n_steps, ctypes.byref(st),
                           _stream(stream)))
    return st


def step1(mps: Mps, mpo: Mpo, params: StepParams, n_steps: int = 1, stream=None,
          stats: Optional[StepStats] = None) -> StepStats:
    """One-site TDVP steps (FP64, fixed bond dimension; segmented when params has segments)."""
    st = stats if stats is not None else StepStats()
    _check(lib().tdvp_step1(mps.handle, mpo.handle, ctypes.byref(params), n_steps, ctypes.byref(st),
                            _stream(stream)))
    return st


def step_hybrid(mps: Mps, mpo: Mpo, params: StepParams, n_steps: int = 1, stream=None,
                stats: Optional[StepStats] = None) -> int:
    """Two-site steps until every bond is full, then one-site steps; returns the one-site count."""
    st = stats if stats is not None else StepStats()
    return _check(lib().tdvp_step_hybrid(mps.handle, mpo.handle, ctypes.byref(params), n_steps, ctypes.byref(st),
                                         _stream(stream)))


def dmrg_params(chi_max: int, w_max: float = 0.0, eps: float = 1e-12, krylov_max: int = 8,
                krylov_tol: float = 1e-6, precision: int = FP64) -> DmrgParams:
    return DmrgParams(chi_max, w_max, eps, krylov_max, krylov_tol, precision)


def dmrg(mps: Mps, mpo: Mpo, params: DmrgParams, n_sweeps: int = 1, stream=None) -> DmrgStats:
    st = DmrgStats()
    _check(lib().tdvp_dmrg(mps.handle, mpo.handle, ctypes.byref(params), n_sweeps, ctypes.byref(st),
                           _stream(stream)))
    return st


def reorthonormalize(mps: Mps, eps: float = 1e-14) -> None:
    _check(lib().tdvp_reorthonormalize(mps.handle, eps))


def measure(mps: Mps, obs: int = OBS_SZ) -> np.ndarray:
    N, _ = mps.size()
    out = np.zeros(N, dtype=np.float64)
    _check(lib().tdvp_measure(mps.handle, obs, _dptr(out)))
    return out


def mps_copy(mps: Mps) -> Mps:
    h_ = ctypes.c_void_p()
    _check(lib().tdvp_mps_copy(mps.handle, ctypes.byref(h_)))
    return Mps(h_)


def apply_site_op(mps: Mps, j: int, op: np.ndarray) -> None:
    """O_j |psi> in place (op: d x d complex, [s_out][s_in])."""
    o = np.ascontiguousarray(op, dtype=np.complex128)
    _check(lib().tdvp_apply_site_op(mps.handle, j, _dptr(o.view(np.float64))))


def expect_mixed(a: Mps, b: Mps, obs: int = OBS_SZ) -> np.ndarray:
    """<a|O_j|b> for every site (complex, not normalised)."""
    N, _ = a.size()
    out = np.zeros(2 * N, dtype=np.float64)
    _check(lib().tdvp_expect_mixed(a.handle, b.handle, obs, _dptr(out)))
    return out.view(np.complex128).copy()


def norm(mps: Mps) -> float:
    out = np.zeros(1)
    _check(lib().tdvp_norm(mps.handle, _dptr(out)))
    return float(out[0])


def energy(mps: Mps, mpo: Mpo) -> float:
    out = np.zeros(1)
    _check(lib().tdvp_energy(mps.handle, mpo.handle, _dptr(out)))
    return float(out[0])


def overlap(a: Mps, b: Mps) -> complex:
    out = np.zeros(2)
    _check(lib().tdvp_overlap(a.handle, b.handle, _dptr(out)))
    return complex(out[0], out[1])


# ---- derivatives with respect to the model parameters -------------------------
PARAM_H, PARAM_J = 0, 1


def build_mpo_derivative(mpo: Mpo, param: int) -> Mpo:
    """dW/d(param) of `mpo` (PARAM_H or PARAM_J) as an MPO handle."""
    h_ = ctypes.c_void_p()
    _check(lib().tdvp_build_mpo_derivative(mpo.handle, param, ctypes.byref(h_)))
    d = Mpo(h_)
    d._base = mpo  # the derivative refers to its MPO
    return d


class Tangent:
    """Tangent of an MPS in n_dir parameter directions (zero when created)."""

    def __init__(self, mps: Mps, n_dir: int):
        h_ = ctypes.c_void_p()
        _check(lib().tdvp_tangent_create(mps.handle, n_dir, ctypes.byref(h_)))
        self.handle = h_
        self.mps = mps
        self.n_dir = n_dir

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tdvp_free_tangent(self.handle)
            self.handle = None


def step_tangent(mps: Mps, mpo: Mpo, tan: Tangent, dmpos: Sequence[Mpo], params: StepParams, n_steps: int = 1,
                 n_quad: int = 6, stream=None, stats: Optional[StepStats] = None) -> StepStats:
    st = stats if stats is not None else StepStats()
    arr = (_P * len(dmpos))(*[d.handle for d in dmpos])
    _check(lib().tdvp_step_tangent(mps.handle, mpo.handle, tan.handle, arr, ctypes.byref(params), n_quad, n_steps,
                                   ctypes.byref(st), _stream(stream)))
    return st


def measure_tangent(mps: Mps, tan: Tangent, obs: int = OBS_SZ):
    """(<O_j> [N], d<O_j> [n_dir, N])."""
    N, _ = mps.size()
    val = np.zeros(N, dtype=np.float64)
    der = np.zeros((tan.n_dir, N), dtype=np.float64)
    _check(lib().tdvp_measure_tangent(mps.handle, tan.handle, obs, _dptr(val), _dptr(der)))
    return val, der


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _check(lib().tdvp_gauss_legendre(n, _dptr(x), _dptr(w)))
    return x, w


# ---- kernel-level operations (torch device tensors) -------------------------
def op_heff(precision, nsite, chi_l, chi_r, m, d, W, L, R, x, y, stream=None):
    Wh = np.ascontiguousarray(W, dtype=np.complex128)
    _check(lib().tdvp_op_heff(precision, nsite, chi_l, chi_r, m, d, _dptr(Wh.view(np.float64)), _ptr(L),
                              _ptr(R), _ptr(x), _ptr(y), _stream(stream)))


def op_heff_noalloc(nsite, chi_l, chi_r, m, d, W, L, R, x, y, stream=None):
    """FP64 H_eff . x using only the library's fixed scratch array (no device allocation)."""
    Wh = np.ascontiguousarray(W, dtype=np.complex128)
    _check(lib().tdvp_op_heff_noalloc(nsite, chi_l, chi_r, m, d, _dptr(Wh.view(np.float64)), _ptr(L), _ptr(R),
                                      _ptr(x), _ptr(y), _stream(stream)))


def op_env(precision, side, chi_l, chi_r, m, d, W, env, A, out, stream=None):
    Wh = np.ascontiguousarray(W, dtype=np.complex128)
    _check(lib().tdvp_op_env(precision, side, chi_l, chi_r, m, d, _dptr(Wh.view(np.float64)), _ptr(env),
                             _ptr(A), _ptr(out), _stream(stream)))


def op_expm(precision, nsite, chi_l, chi_r, m, d, W, L, R, x, y, t, kmax, tol, stream=None) -> int:
    Wh = np.ascontiguousarray(W, dtype=np.complex128)
    nv = ctypes.c_int(0)
    _check(lib().tdvp_op_expm(precision, nsite, chi_l, chi_r, m, d, _dptr(Wh.view(np.float64)), _ptr(L),
                              _ptr(R), _ptr(x), _ptr(y), t, kmax, tol, ctypes.byref(nv), _stream(stream)))
    return nv.value


def op_split(rows, cols, theta, chi_max, w_max, eps, Psi_L, V, Psi_R, s_out=None, stream=None, precision=FP64):
    chi = ctypes.c_int(0)
    w = ctypes.c_double(0)
    _check(lib().tdvp_op_split_prec(precision, rows, cols, _ptr(theta), chi_max, w_max, eps, _ptr(Psi_L), _ptr(V),
                                    _ptr(Psi_R), _ptr(s_out) if s_out is not None else None, ctypes.byref(chi),
                                    ctypes.byref(w), _stream(stream)))
    return chi.value, w.value


# ---- host-only utilities -----------------------------------------------------
def schedule(N: int, seg_len: Optional[Sequence[int]], merge_turning: int, half: int) -> np.ndarray:
    seg = np.ascontiguousarray(seg_len if seg_len else [N], dtype=np.int32)
    n = _check(lib().tdvp_schedule(N, len(seg), seg.ctypes.data_as(_I), merge_turning, half, None, 0))
    out = np.zeros((n, 7), dtype=np.int32)
    _check(lib().tdvp_schedule(N, len(seg), seg.ctypes.data_as(_I), merge_turning, half,
                               out.ctypes.data_as(_I), n))
    return out


def schedule1(N: int, seg_len: Optional[Sequence[int]], merge_turning: int, half: int) -> np.ndarray:
    """Stage schedule of a segmented one-site half step (tdvp_schedule1)."""
    seg = np.ascontiguousarray(seg_len if seg_len else [N], dtype=np.int32)
    n = _check(lib().tdvp_schedule1(N, len(seg), seg.ctypes.data_as(_I), merge_turning, half, None, 0))
    out = np.zeros((n, 7), dtype=np.int32)
    _check(lib().tdvp_schedule1(N, len(seg), seg.ctypes.data_as(_I), merge_turning, half,
                                out.ctypes.data_as(_I), n))
    return out


def exchange_plan(N: int, seg_len: Sequence[int], seg_rank: Sequence[int], scheme: int, merge_turning: int,
                  half: int) -> np.ndarray:
    """Messages of a half step with the segments on several ranks (tdvp_exchange_plan):
    rows (stage, after, src, dst, tensor, j), tensor 0 = Psi_j, 1 = V_j, 2 = beta_j, 3 = gamma_j."""
    seg = np.ascontiguousarray(seg_len, dtype=np.int32)
    rk = np.ascontiguousarray(seg_rank, dtype=np.int32)
    n = _check(lib().tdvp_exchange_plan(N, len(seg), seg.ctypes.data_as(_I), rk.ctypes.data_as(_I), scheme,
                                        merge_turning, half, None, 0))
    out = np.zeros((n, 6), dtype=np.int32)
    _check(lib().tdvp_exchange_plan(N, len(seg), seg.ctypes.data_as(_I), rk.ctypes.data_as(_I), scheme,
                                    merge_turning, half, out.ctypes.data_as(_I), n))
    return out


def tridiag_expm(alpha: np.ndarray, beta: np.ndarray, t: float) -> np.ndarray:
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta if len(beta) else [0.0], dtype=np.float64)
    out = _cplx_out(len(a))
    _check(lib().tdvp_tridiag_expm(len(a), _dptr(a), _dptr(b), t, _dptr(out.view(np.float64))))
    return out


def set_env_tensor_cores(enable: bool) -> None:
    """Mixed modes: environment updates on the tensor cores (True) or in double-float (False, default)."""
    _check(lib().tdvp_set_env_tensor_cores(1 if enable else 0))


def set_autotune(enable: bool) -> None:
    """Per-shape GEMM tile autotuning on (default) or off (fixed tiles); clears the decisions."""
    _check(lib().tdvp_set_autotune(1 if enable else 0))


def autotune_report() -> list:
    """The autotuner's decisions so far (family, shape bucket, choice, microseconds per candidate)."""
    import json
    n = _check(lib().tdvp_autotune_report(None, 0))
    buf = ctypes.create_string_buffer(n + 1)
    lib().tdvp_autotune_report(buf, n + 1)
    return json.loads(buf.value.decode())


def set_wait_limit(spins: int) -> None:
    """Polls a grid-barrier wait of the SVD sweeps makes before giving up
    (TDVP_ETIMEOUT); spins < 0 restores the default."""
    _check(lib().tdvp_set_wait_limit(int(spins)))


# ---- profiling -----------------------------------------------------------------
def profile(enable: bool) -> None:
    _check(lib().tdvp_profile(1 if enable else 0))


def profile_read() -> dict:
    """{kernel kind: {"ms", "launches", "flops", "bytes"}} accumulated since profile(True)."""
    n = _check(lib().tdvp_profile_read(-1, None, 0, None, None, None, None))
    out = {}
    for i in range(n):
        name = ctypes.create_string_buffer(64)
        ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        la = ctypes.c_int64()
        _check(lib().tdvp_profile_read(i, name, 64, ctypes.byref(ms), ctypes.byref(la), ctypes.byref(fl),
                                       ctypes.byref(by)))
        aux = ctypes.c_double()
        _check(lib().tdvp_profile_read_aux(i, ctypes.byref(aux)))
        out[name.value.decode()] = {"ms": ms.value, "launches": la.value, "flops": fl.value, "bytes": by.value,
                                    "aux": aux.value}
    return out
