"""Thin Python binding of the C-ABI in include/hf.h (argument marshalling only).

Every computation runs in the CUDA library ``_build/libhf.so``; if it is not
built, loading fails with an error instead of falling back to anything else.
PyTorch supplies device memory and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import math
import os
import sys

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhf.so")

HF_OK = 0
HF_E_INVALID = -1
HF_E_UNSUPPORTED = -2
HF_E_NOMEM = -3
HF_E_CUDA = -4
HF_E_TIMEOUT = -5
HF_E_NOCONV = -6
HF_PTR_HOST = 0
HF_PTR_DEVICE = 1
HF_TIMING = 2
HF_FP64_ONLY = 8
HF_DENSITY_SCREEN = 16
HF_RYS = 32
HF_OBARA_SAIKA = 64
NUM_CLASSES = 21

CLASS_NAMES = []
for _X, _xn in enumerate(["ss", "ps", "pp", "ds", "dp", "dd"]):
    for _Y, _yn in enumerate(["ss", "ps", "pp", "ds", "dp", "dd"][: _X + 1]):
        CLASS_NAMES.append(f"({_xn}|{_yn})")

PAIR_L = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
CLASS_KERNELS = [f"k_eri_{PAIR_L[X][0]}{PAIR_L[X][1]}{PAIR_L[Y][0]}{PAIR_L[Y][1]}"
                 for X in range(6) for Y in range(X + 1)]

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


class Geometry_c(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("Z", _i32p), ("xyz", _f64p)]


class Basis_c(ctypes.Structure):
    _fields_ = [("n_shells", ctypes.c_int32), ("atom", _i32p), ("l", _i32p), ("nprim", _i32p),
                ("exps", _f64p), ("coefs", _f64p), ("coefs_p", _f64p)]


HF_SP_SHELL = -1


def _basis_c(basis, keep: list):
    """hf_basis of an inputs.Basis; the arrays it points to are appended to ``keep``."""
    at, l, npr = _as_i32(basis.atom), _as_i32(basis.l), _as_i32(basis.nprim)
    ex, co = _as_f64(basis.exps), _as_f64(basis.coefs)
    cp = getattr(basis, "coefs_p", None)
    cp = _as_f64(cp) if cp is not None else None
    keep += [at, l, npr, ex, co, cp]
    return Basis_c(int(l.shape[0]), at.ctypes.data_as(_i32p), l.ctypes.data_as(_i32p), npr.ctypes.data_as(_i32p),
                   ex.ctypes.data_as(_f64p), co.ctypes.data_as(_f64p),
                   cp.ctypes.data_as(_f64p) if cp is not None else None)


class Thresholds_c(ctypes.Structure):
    _fields_ = [("schwarz_tau", ctypes.c_double), ("fp32_cutoff", ctypes.c_double), ("prim_tau", ctypes.c_double)]


class Stats_c(ctypes.Structure):
    _fields_ = [("quartets_unscreened", ctypes.c_int64), ("quartets_fp64", ctypes.c_int64),
                ("quartets_fp32", ctypes.c_int64),
                ("class_quartets_fp64", ctypes.c_int64 * NUM_CLASSES),
                ("class_quartets_fp32", ctypes.c_int64 * NUM_CLASSES),
                ("flops_fp64", ctypes.c_double), ("flops_fp32", ctypes.c_double),
                ("ms_class_fp64", ctypes.c_float * NUM_CLASSES), ("ms_class_fp32", ctypes.c_float * NUM_CLASSES),
                ("ms_eri", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("class_flops_fp64", ctypes.c_double * NUM_CLASSES), ("class_flops_fp32", ctypes.c_double * NUM_CLASSES),
                ("kernels_launched", ctypes.c_int32), ("prim_quartets_fp64", ctypes.c_int64),
                ("prim_quartets_fp32", ctypes.c_int64)]


class SystemInfo_c(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("n_shells", ctypes.c_int32), ("n_bf", ctypes.c_int32),
                ("n_electrons", ctypes.c_int32), ("n_pairs", ctypes.c_int64), ("n_significant_pairs", ctypes.c_int64),
                ("quartets_unscreened", ctypes.c_int64), ("quartets_fp64", ctypes.c_int64),
                ("quartets_fp32", ctypes.c_int64), ("E_nn", ctypes.c_double), ("Q_max", ctypes.c_double),
                ("device_bytes", ctypes.c_int64)]


class Peaks_c(ctypes.Structure):
    _fields_ = [("fp64_fma_gflops", ctypes.c_double), ("fp32_fma_gflops", ctypes.c_double),
                ("red_add_f64_random_gops", ctypes.c_double), ("red_add_f64_coalesced_gops", ctypes.c_double),
                ("sm_max_mhz", ctypes.c_double), ("num_sms", ctypes.c_int32), ("pad", ctypes.c_int32)]


class ScfOpts_c(ctypes.Structure):
    _fields_ = [("n_occ", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("e_tol", ctypes.c_double),
                ("d_tol", ctypes.c_double), ("diis_size", ctypes.c_int32), ("diis_off", ctypes.c_int32),
                ("mixed_switch", ctypes.c_double), ("incremental", ctypes.c_int32), ("rebuild_every", ctypes.c_int32),
                ("incremental_switch", ctypes.c_double)]


class ScfResult_c(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("E_nn", ctypes.c_double), ("iterations", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("last_dE", ctypes.c_double), ("last_dP", ctypes.c_double),
                ("seconds_total", ctypes.c_double), ("seconds_fock", ctypes.c_double),
                ("seconds_diag", ctypes.c_double), ("jacobi_sweeps", ctypes.c_int32), ("n_kept", ctypes.c_int32),
                ("s_min", ctypes.c_double), ("mixed_iterations", ctypes.c_int32), ("full_builds", ctypes.c_int32)]


class BatchInfo_c(ctypes.Structure):
    _fields_ = [("n_mol", ctypes.c_int32), ("packed_len", ctypes.c_int64), ("n_bf_total", ctypes.c_int64),
                ("quartets", ctypes.c_int64), ("class_quartets", ctypes.c_int64 * NUM_CLASSES),
                ("block", ctypes.c_int32 * NUM_CLASSES), ("chunk", ctypes.c_int32 * NUM_CLASSES),
                ("blocks_per_sm", ctypes.c_int32 * NUM_CLASSES)]


HF_BATCH_SEQUENTIAL = 4


class TrainOpts_c(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float), ("pad", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class HFError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__(f"{where}: status {code} ({msg})")
        self.code = code


_lib = None


def load_library():
    """Load libhf.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_1708_00033_gb300.build() on a machine with nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    lib.hf_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
    lib.hf_destroy.argtypes = [vp]
    lib.hf_destroy.restype = None
    lib.hf_strerror.argtypes = [ctypes.c_int]
    lib.hf_strerror.restype = ctypes.c_char_p
    lib.hf_last_error.argtypes = []
    lib.hf_last_error.restype = ctypes.c_char_p
    lib.hf_system_create.argtypes = [vp, ctypes.POINTER(Geometry_c), ctypes.POINTER(Basis_c),
                                     ctypes.POINTER(Thresholds_c), ctypes.POINTER(vp)]
    lib.hf_system_destroy.argtypes = [vp]
    lib.hf_system_destroy.restype = None
    lib.hf_system_get_info.argtypes = [vp, ctypes.POINTER(SystemInfo_c)]
    lib.hf_one_electron.argtypes = [vp, vp, vp, ctypes.c_int]
    lib.hf_fock_build.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Stats_c),
                                  ctypes.c_int]
    lib.hf_fock_build_noalloc.argtypes = [vp, vp, vp, vp, vp]
    lib.hf_fock_build_partial.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int]
    lib.hf_system_set_fock_copies.argtypes = [vp, ctypes.c_int32]
    lib.hf_measure_peaks.argtypes = [vp, ctypes.POINTER(Peaks_c)]
    lib.hf_scf_run.argtypes = [vp, ctypes.POINTER(ScfOpts_c), vp, vp, vp, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ScfResult_c), ctypes.c_int]
    lib.hf_eigh.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_int]
    lib.hf_batch_create.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Geometry_c), ctypes.POINTER(Basis_c),
                                    ctypes.POINTER(Thresholds_c), ctypes.POINTER(vp)]
    lib.hf_batch_destroy.argtypes = [vp]
    lib.hf_batch_destroy.restype = None
    lib.hf_batch_get_info.argtypes = [vp, ctypes.POINTER(BatchInfo_c)]
    lib.hf_batch_offsets.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.hf_fock_build_batch.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float),
                                        ctypes.c_int]
    lib.hf_batch_tune.argtypes = [vp, ctypes.c_char_p, ctypes.c_int64]
    lib.hf_model_num_params.restype = ctypes.c_int64
    lib.hf_model_num_params.argtypes = []
    lib.hf_model_create.argtypes = [vp, vp, ctypes.POINTER(vp)]
    lib.hf_model_destroy.argtypes = [vp]
    lib.hf_model_destroy.restype = None
    lib.hf_model_get_weights.argtypes = [vp, vp, vp]
    lib.hf_model_forward.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int]
    lib.hf_model_train_step.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                        ctypes.c_int]
    lib.hf_guess_features.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
    lib.hf_guess_predict.argtypes = [vp, vp, vp, ctypes.c_int]
    lib.hf_guess_targets.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    lib.hf_guess_train.argtypes = [vp, ctypes.c_int64, vp, vp, vp, ctypes.POINTER(TrainOpts_c), vp, ctypes.c_int]
    lib.hf_fock_assemble.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    _lib = lib
    return lib


def _check(rc, where):
    if rc != HF_OK:
        lib = load_library()
        raise HFError(rc, where, lib.hf_last_error().decode() or lib.hf_strerror(rc).decode())


def _torch():
    import torch
    return torch


class Context:
    """hf_create: one device, one stream (torch's current stream by default)."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._h = ctypes.c_void_p()
        _check(load_library().hf_create(ctypes.byref(self._h), self.device, ctypes.c_void_p(handle)), "hf_create")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().hf_destroy(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():  # the CUDA runtime may already be gone
            return
        try:
            self.close()
        except Exception:
            pass


def _as_i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _as_f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class System:
    """hf_system_create: one molecule with its screening plan."""

    def __init__(self, ctx: Context, geom: _inputs.Geometry, basis: _inputs.Basis, schwarz_tau: float = 0.0,
                 fp32_cutoff: float = 0.0, prim_tau: float = 0.0):
        self.ctx = ctx
        Z, xyz = _as_i32(geom.Z), _as_f64(geom.xyz)
        keep = []
        g = Geometry_c(int(Z.shape[0]), Z.ctypes.data_as(_i32p), xyz.ctypes.data_as(_f64p))
        b = _basis_c(basis, keep)
        th = Thresholds_c(float(schwarz_tau), float(fp32_cutoff), float(prim_tau))
        self._h = ctypes.c_void_p()
        _check(load_library().hf_system_create(ctx._h, ctypes.byref(g), ctypes.byref(b), ctypes.byref(th),
                                               ctypes.byref(self._h)), "hf_system_create")
        self.info = self.get_info()
        self.n_bf = self.info["n_bf"]

    def get_info(self) -> dict:
        inf = SystemInfo_c()
        _check(load_library().hf_system_get_info(self._h, ctypes.byref(inf)), "hf_system_get_info")
        return {k: getattr(inf, k) for k, _ in SystemInfo_c._fields_}

    def set_fock_copies(self, copies: int):
        """hf_system_set_fock_copies: 1 = one shared accumulator pair, >1 = per-block private copies."""
        _check(load_library().hf_system_set_fock_copies(self._h, int(copies)), "hf_system_set_fock_copies")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().hf_system_destroy(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def one_electron(self, device: bool = False):
        N = self.n_bf
        if device:
            torch = _torch()
            S = torch.empty((N, N), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
            H = torch.empty_like(S)
            _check(load_library().hf_one_electron(self._h, S.data_ptr(), H.data_ptr(), HF_PTR_DEVICE),
                   "hf_one_electron")
            return S, H
        S, H = np.empty((N, N)), np.empty((N, N))
        _check(load_library().hf_one_electron(self._h, S.ctypes.data, H.ctypes.data, HF_PTR_HOST), "hf_one_electron")
        return S, H

    def fock_build(self, P, F=None, J=None, K=None, want_J=False, want_K=False, energy=True, stats=False,
                   timing=False, rys=None, fp64_only=False):
        """hf_fock_build.  ``P`` may be a numpy array (host path: copies in the
        timed call) or a CUDA float64 tensor (device path).  Output buffers may
        be passed to avoid allocation.  rys: True for Rys quadrature in all five
        L >= 6 classes (HF_RYS), False for Obara-Saika in every class
        (HF_OBARA_SAIKA), None for the per-class default.  Returns a dict with
        F, J, K, E_elec and optionally stats."""
        N = self.n_bf
        lib = load_library()
        flags = (HF_TIMING if timing else 0) | _method_flags(rys) | (HF_FP64_ONLY if fp64_only else 0)
        is_dev = hasattr(P, "is_cuda") and P.is_cuda
        if is_dev:
            torch = _torch()
            if P.dtype != torch.float64 or not P.is_contiguous() or tuple(P.shape) != (N, N):
                raise ValueError("P must be a contiguous float64 N x N CUDA tensor")
            flags |= HF_PTR_DEVICE
            if F is None:
                F = torch.empty_like(P)
            if want_J and J is None:
                J = torch.empty_like(P)
            if want_K and K is None:
                K = torch.empty_like(P)
            ptr = lambda t: t.data_ptr() if t is not None else None  # noqa: E731
            p_ptr = P.data_ptr()
        else:
            P = _as_f64(P)
            if P.shape != (N, N):
                raise ValueError("P must be N x N")
            if F is None:
                F = np.empty((N, N))
            if want_J and J is None:
                J = np.empty((N, N))
            if want_K and K is None:
                K = np.empty((N, N))
            ptr = lambda a: a.ctypes.data if a is not None else None  # noqa: E731
            p_ptr = P.ctypes.data
        e = ctypes.c_double(0.0)
        st = Stats_c()
        rc = lib.hf_fock_build(self._h, p_ptr, ptr(F), ptr(J), ptr(K), ctypes.byref(e) if energy else None,
                               ctypes.byref(st) if (stats or timing) else None, flags)
        _check(rc, "hf_fock_build")
        out = {"F": F, "J": J, "K": K, "E_elec": e.value if energy else None}
        if stats or timing:
            out["stats"] = stats_dict(st)
        return out


class Batch:
    """hf_batch_create: many molecules built together in one graph-captured step."""

    def __init__(self, ctx: Context, geoms, bases, schwarz_tau: float = 0.0, prim_tau: float = 0.0):
        self.ctx = ctx
        n = len(geoms)
        keep = []
        G = (Geometry_c * n)()
        Bs = (Basis_c * n)()
        for m, (g, b) in enumerate(zip(geoms, bases)):
            arrs = [_as_i32(g.Z), _as_f64(g.xyz)]
            keep.append(arrs)
            G[m] = Geometry_c(int(arrs[0].shape[0]), arrs[0].ctypes.data_as(_i32p), arrs[1].ctypes.data_as(_f64p))
            Bs[m] = _basis_c(b, keep)
        th = Thresholds_c(float(schwarz_tau), 0.0, float(prim_tau))
        self._h = ctypes.c_void_p()
        _check(load_library().hf_batch_create(ctx._h, n, G, Bs, ctypes.byref(th), ctypes.byref(self._h)),
               "hf_batch_create")
        self.n_mol = n
        off = (ctypes.c_int64 * (n + 1))()
        _check(load_library().hf_batch_offsets(self._h, off), "hf_batch_offsets")
        self.offsets = np.array(list(off), dtype=np.int64)
        self.n_bf = [math.isqrt(int(self.offsets[m + 1] - self.offsets[m])) for m in range(n)]  # blocks are N_m^2

    def info(self) -> dict:
        inf = BatchInfo_c()
        _check(load_library().hf_batch_get_info(self._h, ctypes.byref(inf)), "hf_batch_get_info")
        d = {k: getattr(inf, k) for k, _ in BatchInfo_c._fields_}
        for k in ("class_quartets", "block", "chunk", "blocks_per_sm"):
            d[k] = list(d[k])
        return d

    def tune(self, cache_path: str | None = None, sample_quartets: int = 0):
        _check(load_library().hf_batch_tune(self._h, cache_path.encode() if cache_path else None,
                                            int(sample_quartets)), "hf_batch_tune")

    def fock_build(self, P, F, energies: bool = False, sequential: bool = False):
        """Packed P in, packed F out (CUDA tensors or numpy arrays); returns (ms, E_elec or None)."""
        is_dev = hasattr(P, "is_cuda") and P.is_cuda
        flags = (HF_PTR_DEVICE if is_dev else 0) | (HF_BATCH_SEQUENTIAL if sequential else 0)
        ptr = (lambda t: t.data_ptr()) if is_dev else (lambda a: a.ctypes.data)
        E = np.zeros(self.n_mol) if energies else None
        ms = ctypes.c_float(0.0)
        _check(load_library().hf_fock_build_batch(self._h, ptr(P), ptr(F), E.ctypes.data_as(_f64p) if energies else None,
                                                  ctypes.byref(ms), flags), "hf_fock_build_batch")
        return ms.value, E

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().hf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Model:
    """hf_model_create: the learned-guess MLP (weights live on the device)."""

    N_FEAT, WIDTH, N_OUT = 16, 256, 325

    def __init__(self, ctx: Context, weights: np.ndarray):
        self.ctx = ctx
        w = np.ascontiguousarray(weights, dtype=np.float32)
        if w.size != num_params():
            raise ValueError("weight vector has the wrong length")
        self._h = ctypes.c_void_p()
        _check(load_library().hf_model_create(ctx._h, w.ctypes.data, ctypes.byref(self._h)), "hf_model_create")

    def weights(self, gradients: bool = False) -> np.ndarray:
        out = np.empty(num_params(), dtype=np.float32)
        if gradients:
            _check(load_library().hf_model_get_weights(self._h, None, out.ctypes.data), "hf_model_get_weights")
        else:
            _check(load_library().hf_model_get_weights(self._h, out.ctypes.data, None), "hf_model_get_weights")
        return out

    def forward(self, X):
        """X [n, 16]: numpy (host path) or CUDA float32 tensor (device path)."""
        if hasattr(X, "is_cuda") and X.is_cuda:
            torch = _torch()
            Y = torch.empty((X.shape[0], self.N_OUT), dtype=torch.float32, device=X.device)
            _check(load_library().hf_model_forward(self._h, int(X.shape[0]), X.data_ptr(), Y.data_ptr(),
                                                   HF_PTR_DEVICE), "hf_model_forward")
            return Y
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.empty((X.shape[0], self.N_OUT), dtype=np.float32)
        _check(load_library().hf_model_forward(self._h, int(X.shape[0]), X.ctypes.data, Y.ctypes.data, HF_PTR_HOST),
               "hf_model_forward")
        return Y

    def train_step(self, X, T, mask, lr: float) -> float:
        """One Adam step on CUDA float32 tensors; returns the minibatch loss."""
        loss = ctypes.c_float(0.0)
        _check(load_library().hf_model_train_step(self._h, int(X.shape[0]), X.data_ptr(), T.data_ptr(),
                                                  mask.data_ptr(), float(lr), ctypes.byref(loss), HF_PTR_DEVICE),
               "hf_model_train_step")
        return float(loss.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().hf_model_destroy(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def num_params() -> int:
    return int(load_library().hf_model_num_params())


def guess_features(system: "System"):
    """Host arrays X [n_pairs, 16] float32 and meta [n_pairs, 4] int32."""
    n = ctypes.c_int64(0)
    _check(load_library().hf_guess_features(system._h, None, None, ctypes.byref(n), 0), "hf_guess_features")
    X = np.empty((n.value, 16), dtype=np.float32)
    meta = np.empty((n.value, 4), dtype=np.int32)
    _check(load_library().hf_guess_features(system._h, X.ctypes.data, meta.ctypes.data, ctypes.byref(n), HF_PTR_HOST),
           "hf_guess_features")
    return X, meta


def guess_predict(model: Model, system: "System") -> np.ndarray:
    P = np.empty((system.n_bf, system.n_bf))
    _check(load_library().hf_guess_predict(model._h, system._h, P.ctypes.data, HF_PTR_HOST), "hf_guess_predict")
    return P


def scf(system: "System", n_occ: int = 0, max_iter: int = 100, e_tol: float = 1e-9, d_tol: float = 1e-6,
        diis_size: int = 8, P_guess=None, raise_on_noconv: bool = True, mixed_switch: float = 1e-5,
        incremental: bool = False, rebuild_every: int = 8, incremental_switch: float = 1e-5) -> dict:
    """hf_scf_run with host arrays; returns energy, density, orbital energies and timings."""
    N = system.n_bf
    o = ScfOpts_c(int(n_occ), int(max_iter), float(e_tol), float(d_tol), int(diis_size), 1 if diis_size == 0 else 0,
                  float(mixed_switch), 1 if incremental else 0, int(rebuild_every), float(incremental_switch))
    P_out = np.empty((N, N))
    eps = np.zeros(N)
    en = np.zeros(max_iter)
    res = ScfResult_c()
    Pg = None if P_guess is None else _as_f64(P_guess)
    rc = load_library().hf_scf_run(system._h, ctypes.byref(o), Pg.ctypes.data if Pg is not None else None,
                                   P_out.ctypes.data, eps.ctypes.data, en.ctypes.data_as(_f64p), ctypes.byref(res),
                                   HF_PTR_HOST)
    if rc != HF_E_NOCONV or raise_on_noconv:
        _check(rc, "hf_scf_run")
    out = {k: getattr(res, k) for k, _ in ScfResult_c._fields_}
    out.update(P=P_out, eps=eps[: res.n_kept], energies=en[: res.iterations].copy(), status=rc)
    return out


def eigh(ctx: Context, A) -> tuple:
    """hf_eigh on a host matrix: eigenvalues ascending and eigenvectors as columns."""
    A = _as_f64(A)
    n = A.shape[0]
    w = np.empty(n)
    V = np.empty((n, n))
    _check(load_library().hf_eigh(ctx._h, n, A.ctypes.data, w.ctypes.data, V.ctypes.data, HF_PTR_HOST), "hf_eigh")
    return w, V


def measure_peaks(ctx: "Context") -> dict:
    """hf_measure_peaks: FP64/FP32 FMA and FP64 atomic-add throughput of this GPU."""
    out = Peaks_c()
    _check(load_library().hf_measure_peaks(ctx._h, ctypes.byref(out)), "hf_measure_peaks")
    return {k: getattr(out, k) for k, _ in Peaks_c._fields_ if k != "pad"}


def fock_build_noalloc(system: "System", P, F, J=None, K=None):
    """hf_fock_build_noalloc: device tensors in and out, no allocation in the call."""
    ptr = lambda t: t.data_ptr() if t is not None else None  # noqa: E731
    _check(load_library().hf_fock_build_noalloc(system._h, ptr(P), ptr(F), ptr(J), ptr(K)), "hf_fock_build_noalloc")
    return F


def _is_dev(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def _method_flags(rys) -> int:
    """ERI method flags: True -> HF_RYS, False -> HF_OBARA_SAIKA, None -> 0 (the per-class default)."""
    return 0 if rys is None else (HF_RYS if rys else HF_OBARA_SAIKA)


def fock_build_partial(system: "System", P, shard: int = 0, n_shards: int = 1, density_screen: bool = False,
                       fp64_only: bool = False, J=None, K=None, rys=None):
    """hf_fock_build_partial: (J_shard, K_shard).  ``P`` is a numpy array (host path) or a contiguous float64
    CUDA tensor (device path, outputs are CUDA tensors).  density_screen also skips quartets whose Schwarz
    bound times the largest |P| of the six blocks they touch is below the Schwarz threshold."""
    N = system.n_bf
    flags = (HF_DENSITY_SCREEN if density_screen else 0) | (HF_FP64_ONLY if fp64_only else 0) | _method_flags(rys)
    if _is_dev(P):
        torch = _torch()
        if P.dtype != torch.float64 or not P.is_contiguous() or tuple(P.shape) != (N, N):
            raise ValueError("P must be a contiguous float64 N x N CUDA tensor")
        J = torch.empty_like(P) if J is None else J
        K = torch.empty_like(P) if K is None else K
        _check(load_library().hf_fock_build_partial(system._h, P.data_ptr(), int(shard), int(n_shards), J.data_ptr(),
                                                    K.data_ptr(), flags | HF_PTR_DEVICE), "hf_fock_build_partial")
        return J, K
    P = _as_f64(P)
    J = np.empty((N, N)) if J is None else J
    K = np.empty((N, N)) if K is None else K
    _check(load_library().hf_fock_build_partial(system._h, P.ctypes.data, int(shard), int(n_shards), J.ctypes.data,
                                                K.ctypes.data, flags | HF_PTR_HOST), "hf_fock_build_partial")
    return J, K


def fock_assemble(system: "System", J, K, P=None, energy: bool = False):
    """hf_fock_assemble: F = H + J - K/2 (and E_elec from P) from J and K summed over every shard.
    Host arrays or CUDA tensors (all of one kind).  Returns (F, E_elec or None)."""
    N = system.n_bf
    e = ctypes.c_double(0.0)
    if energy and P is None:
        raise ValueError("the energy needs the density P")
    if _is_dev(J):
        torch = _torch()
        F = torch.empty_like(J)
        _check(load_library().hf_fock_assemble(system._h, P.data_ptr() if P is not None else None, J.data_ptr(),
                                               K.data_ptr(), F.data_ptr(), ctypes.byref(e) if energy else None,
                                               HF_PTR_DEVICE), "hf_fock_assemble")
    else:
        J, K = _as_f64(J), _as_f64(K)
        Pp = _as_f64(P) if P is not None else None
        F = np.empty((N, N))
        _check(load_library().hf_fock_assemble(system._h, Pp.ctypes.data if Pp is not None else None, J.ctypes.data,
                                               K.ctypes.data, F.ctypes.data, ctypes.byref(e) if energy else None,
                                               HF_PTR_HOST), "hf_fock_assemble")
    return F, (e.value if energy else None)


def assemble_shards(system: "System", J_part, K_part, all_reduce_sum, P=None, energy: bool = False,
                    assemble=None):
    """F of a sharded build from this rank's partial J and K.

    ``all_reduce_sum`` returns the sum of an array or tensor over the ranks
    (for example an NCCL or gloo allreduce): the reduction the paper performs
    with ddi_gsumf.  ``assemble`` (default: the library's hf_fock_assemble)
    then forms F (and E_elec from P).  Returns (F, J, K, E_elec or None)."""
    J = all_reduce_sum(J_part)
    K = all_reduce_sum(K_part)
    F, E = (assemble or fock_assemble)(system, J, K, P=P, energy=energy)
    return F, J, K, E


def sharded_fock_build(system: "System", P, rank: int, world: int, all_reduce_sum, energy: bool = True,
                       build_partial=None, assemble=None):
    """One rank's part of a Fock build sharded over ``world`` ranks (Algorithms 2/3 with ddi_gsumf): the
    quartet shard ``rank`` of every class (hf_fock_build_partial), one sum of J and one of K over the ranks,
    and the assembly of F.  Every rank returns the full (F, J, K, E_elec).  ``build_partial`` and
    ``assemble`` default to the library calls."""
    J, K = (build_partial or fock_build_partial)(system, P, rank, world)
    return assemble_shards(system, J, K, all_reduce_sum, P=P, energy=energy, assemble=assemble)


def guess_targets(system: "System", P):
    """hf_guess_targets on a host density: T and mask [n_pairs, 325] float32 host arrays."""
    n = ctypes.c_int64(0)
    _check(load_library().hf_guess_features(system._h, None, None, ctypes.byref(n), 0), "hf_guess_features")
    P = _as_f64(P)
    T = np.empty((n.value, Model.N_OUT), dtype=np.float32)
    M = np.empty((n.value, Model.N_OUT), dtype=np.float32)
    _check(load_library().hf_guess_targets(system._h, P.ctypes.data, T.ctypes.data, M.ctypes.data, HF_PTR_HOST),
           "hf_guess_targets")
    return T, M


def guess_train(model: "Model", X, T, mask, steps: int, batch: int = 2048, lr: float = 1e-3, seed: int = 0):
    """hf_guess_train on a dataset in CUDA float32 tensors; returns the per-step minibatch losses."""
    losses = np.zeros(int(steps), dtype=np.float32)
    o = TrainOpts_c(int(steps), int(batch), float(lr), 0, int(seed))
    _check(load_library().hf_guess_train(model._h, int(X.shape[0]), X.data_ptr(), T.data_ptr(), mask.data_ptr(),
                                         ctypes.byref(o), losses.ctypes.data, HF_PTR_DEVICE), "hf_guess_train")
    return losses


def stats_dict(st: Stats_c) -> dict:
    d = {k: getattr(st, k) for k, _ in Stats_c._fields_}
    for k in ("class_quartets_fp64", "class_quartets_fp32", "ms_class_fp64", "ms_class_fp32", "class_flops_fp64",
              "class_flops_fp32"):
        d[k] = list(d[k])
    return d


def exported_symbols() -> list[str]:
    """Names declared in include/hf.h (functions only)."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "hf.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"\b(hf_[a-z_0-9]+)\s*\(", txt)))
