"""ctypes binding of libxbar (C ABI in include/xbar.h): argument marshalling only.

Every step of the solve runs in libxbar.so's CUDA kernels.  Arrays may be
torch tensors (CUDA or CPU, float64, contiguous) or numpy float64 arrays; the
library itself decides whether each pointer is host or device memory.  If the
library cannot be loaded every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

XBAR_OK, XBAR_EINVAL, XBAR_ENOMEM, XBAR_ECUDA, XBAR_ESTATE, XBAR_ENOTCONV, XBAR_ETIMEOUT = range(7)
XBAR_FP64, XBAR_FP32_IR = 0, 1
STATUS_NAMES = {0: "XBAR_OK", 1: "XBAR_EINVAL", 2: "XBAR_ENOMEM", 3: "XBAR_ECUDA", 4: "XBAR_ESTATE",
                5: "XBAR_ENOTCONV", 6: "XBAR_ETIMEOUT"}
PRECISIONS = {"fp64": XBAR_FP64, "fp32_ir": XBAR_FP32_IR}


class XbarError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("max_rel_dI", ctypes.c_double), ("resid_inf", ctypes.c_double),
                ("err_est", ctypes.c_double), ("n_fallback", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PHASES = ["assemble", "factor", "sweep", "resid", "update", "output"]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int * 6), ("ms", ctypes.c_double * 6)]

    def as_dict(self):
        return {ph: {"launches": int(self.launches[k]), "ms": float(self.ms[k])} for k, ph in enumerate(PHASES)}


class TileDesc(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("N", ctypes.c_int), ("G", ctypes.c_void_p), ("R_s", ctypes.c_double),
                ("R_w", ctypes.c_double), ("R_b", ctypes.c_double), ("R_sense", ctypes.c_double)]


OPTIONS = {"sweep_kernel": 0, "factor_kernel": 1, "algorithm": 2, "cr_products": 3, "wait_limit_ns": 4,
           "orientation": 5, "eager_assembly": 6}
ALGORITHMS = {"thomas": 0, "cr": 1}
ORIENTATIONS = {"auto": -1, "columns": 0, "rows": 1}
_VALUE_NAMES = {"algorithm": ALGORITHMS, "orientation": ORIENTATIONS}

_lib = None
_vp = ctypes.c_void_p


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libxbar.so (building it first if needed); raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build._stale()):
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libxbar.so not found at {path}; run paper_2410_19993_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.xbar_assemble.argtypes = [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, _vp, ctypes.POINTER(_vp)]
    lib.xbar_factor.argtypes = [_vp, ctypes.c_int]
    lib.xbar_solve.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int,
                               ctypes.POINTER(SolveInfo)]
    lib.xbar_sync.argtypes = [_vp]
    lib.xbar_set_conductances.argtypes = [_vp, _vp]
    lib.xbar_solve_noalloc.argtypes = [_vp, ctypes.c_int, _vp, _vp]
    lib.xbar_transfer_matrix.argtypes = [_vp, ctypes.c_double, ctypes.c_int, _vp, ctypes.POINTER(SolveInfo)]
    lib.xbar_solve_transfer.argtypes = [_vp, ctypes.c_int, _vp, _vp]
    lib.xbar_set_option.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    lib.xbar_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(TileDesc), _vp, ctypes.POINTER(_vp)]
    lib.xbar_batch_run.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_vp),
                                   ctypes.POINTER(_vp), ctypes.c_double, ctypes.c_int, ctypes.POINTER(SolveInfo)]
    lib.xbar_batch_autotune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_char_p]
    lib.xbar_batch_tile.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(_vp)]
    lib.xbar_batch_destroy.argtypes = [_vp]
    lib.xbar_profile_enable.argtypes = [_vp, ctypes.c_int]
    lib.xbar_profile_read.argtypes = [_vp, ctypes.POINTER(Profile), ctypes.c_int]
    lib.xbar_destroy.argtypes = [_vp]
    _pp, _ip = ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int)
    lib.xbar_surrogate_create.argtypes = ([ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [ctypes.c_int]
                                          + [ctypes.c_double] * 2 + [ctypes.c_uint, _vp, _pp])
    lib.xbar_surrogate_params.argtypes = [_vp, _vp, _vp, _ip]
    lib.xbar_surrogate_scaling.argtypes = [_vp, _vp, _vp]
    lib.xbar_surrogate_grad.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp]
    lib.xbar_surrogate_train.argtypes = [_vp, ctypes.c_int, _pp, _ip, _pp, _pp, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_uint, _vp]
    lib.xbar_surrogate_calibrate.argtypes = [_vp, ctypes.c_int, _pp, _ip, _pp, _pp, ctypes.c_double, _vp]
    lib.xbar_surrogate_predict.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, _vp]
    lib.xbar_surrogate_solve.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_double, _vp,
                                         ctypes.POINTER(SolveInfo)]
    lib.xbar_surrogate_destroy.argtypes = [_vp]
    lib.xbar_last_error.restype = ctypes.c_char_p
    lib.xbar_version.restype = ctypes.c_char_p
    for f in ("xbar_assemble", "xbar_factor", "xbar_solve", "xbar_sync", "xbar_destroy", "xbar_set_conductances",
              "xbar_profile_enable", "xbar_profile_read", "xbar_solve_noalloc", "xbar_set_option",
              "xbar_transfer_matrix", "xbar_solve_transfer",
              "xbar_batch_create", "xbar_batch_run", "xbar_batch_autotune", "xbar_batch_tile",
              "xbar_batch_destroy", "xbar_surrogate_create", "xbar_surrogate_params", "xbar_surrogate_grad",
              "xbar_surrogate_scaling",
              "xbar_surrogate_train", "xbar_surrogate_calibrate", "xbar_surrogate_predict",
              "xbar_surrogate_solve", "xbar_surrogate_destroy"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def last_error() -> str:
    return load().xbar_last_error().decode()


def _check(status):
    if status != XBAR_OK:
        raise XbarError(status, last_error())


def _ptr(a, dtype=np.float64):
    """Data pointer of a contiguous torch tensor or numpy array of `dtype` (None -> NULL)."""
    if a is None:
        return None
    name = np.dtype(dtype).name
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != getattr(torch, name) or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {name} tensor")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a contiguous {name} numpy array")
    return a.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def _cuda_index(a):
    """CUDA device index of a torch tensor, or None for host memory (numpy or CPU tensors)."""
    dev = getattr(a, "device", None)
    if dev is None or getattr(dev, "type", None) != "cuda":
        return None
    return dev.index if dev.index is not None else 0


def _check_shape(name, a, shape, device):
    """Refuse (ValueError) an array whose shape or device does not match what the C call will
    assume: the library receives a bare pointer and would read or write past its end."""
    if a is None:
        return
    if tuple(int(d) for d in a.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(a.shape)}, expected {tuple(shape)}")
    idx = _cuda_index(a)
    if idx is not None and device is not None and idx != device:
        raise ValueError(f"{name} is on cuda:{idx}, the handle on cuda:{device}")


def _current_device():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_device()
    except ImportError:
        pass
    return None


@dataclass
class Crossbar:
    """Handle of one assembled crossbar (xbar_assemble); factor() then solve() any number of batches."""
    M: int
    N: int
    handle: int
    device: int = None  # CUDA device the handle was created on (None: unknown)

    @classmethod
    def assemble(cls, G, Rs, Rw, Rb, Rsense, stream=None):
        if len(G.shape) != 2:
            raise ValueError(f"G must be M x N, got shape {tuple(G.shape)}")
        M, N = int(G.shape[0]), int(G.shape[1])
        dev = _cuda_index(G)
        if dev is None:
            dev = _current_device()
        elif dev != _current_device():
            raise ValueError(f"G is on cuda:{dev}, the current device is cuda:{_current_device()}")
        lib = load()
        h = _vp()
        _check(lib.xbar_assemble(M, N, _ptr(G), Rs, Rw, Rb, Rsense, _stream_ptr(stream), ctypes.byref(h)))
        return cls(M, N, h.value, dev)

    def _check_batch(self, V, I, vWL=None, vBL=None):
        if len(V.shape) != 2:
            raise ValueError(f"V must be B x M, got shape {tuple(V.shape)}")
        B = int(V.shape[0])
        _check_shape("V", V, (B, self.M), self.device)
        _check_shape("I", I, (B, self.N), self.device)
        _check_shape("vWL", vWL, (B, self.M, self.N), self.device)
        _check_shape("vBL", vBL, (B, self.M, self.N), self.device)
        return B

    def factor(self, precision="fp64"):
        _check(load().xbar_factor(self.handle, PRECISIONS.get(precision, precision)))
        return self

    def solve(self, V, I, vWL=None, vBL=None, tol=1e-8, max_iter=10, raise_on_error=True):
        """xbar_solve: V [B x M] -> I [B x N] (+ node voltages [B x M x N]); returns (status, info dict)."""
        B = self._check_batch(V, I, vWL, vBL)
        info = SolveInfo()
        st = load().xbar_solve(self.handle, B, _ptr(V), _ptr(I), _ptr(vWL), _ptr(vBL), tol, max_iter,
                               ctypes.byref(info))
        if raise_on_error:
            _check(st)
        return st, info.as_dict()

    def solve_noalloc(self, V, I, raise_on_error=True):
        """xbar_solve_noalloc: FP64 substitution with library-internal fixed scratch (device V, I only)."""
        B = self._check_batch(V, I)
        st = load().xbar_solve_noalloc(self.handle, B, _ptr(V), _ptr(I))
        if raise_on_error:
            _check(st)
        return st

    def transfer_matrix(self, tol=1e-9, max_iter=10, Geff=None, raise_on_error=True):
        """xbar_transfer_matrix: G_eff (M x N) of the current factorization from M unit solves (cached
        until the next factor); optionally copied into Geff. Returns (status, info dict)."""
        info = SolveInfo()
        _check_shape("Geff", Geff, (self.M, self.N), self.device)
        st = load().xbar_transfer_matrix(self.handle, tol, max_iter, _ptr(Geff), ctypes.byref(info))
        if raise_on_error:
            _check(st)
        return st, info.as_dict()

    def solve_transfer(self, V, I, raise_on_error=True):
        """xbar_solve_transfer: I = V G_eff (currents only), one FP64 product."""
        B = self._check_batch(V, I)
        st = load().xbar_solve_transfer(self.handle, B, _ptr(V), _ptr(I))
        if raise_on_error:
            _check(st)
        return st

    def set_option(self, name, value):
        """xbar_set_option: 'sweep_kernel' (0 CUDA cores, 1 tensor cores) / 'factor_kernel' (0 group,
        1 cluster) / 'algorithm' (0 or 'thomas', 1 or 'cr') / 'cr_products' (0 CUDA cores, 1 tensor cores)
        / 'wait_limit_ns' / 'orientation' (-1 or 'auto', 0 or 'columns', 1 or 'rows'; FP64 factors)."""
        value = _VALUE_NAMES.get(name, {}).get(value, value)
        _check(load().xbar_set_option(self.handle, OPTIONS[name], int(value)))
        return self

    def set_conductances(self, G):
        _check_shape("G", G, (self.M, self.N), self.device)
        _check(load().xbar_set_conductances(self.handle, _ptr(G)))
        return self

    def profile_enable(self, on=True):
        _check(load().xbar_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self, reset=True):
        pr = Profile()
        _check(load().xbar_profile_read(self.handle, ctypes.byref(pr), 1 if reset else 0))
        return pr.as_dict()

    def sync(self):
        _check(load().xbar_sync(self.handle))

    def destroy(self):
        if self.handle:
            load().xbar_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Batch:
    """xbar_batch_*: many tiles factored and solved by one CUDA-graph launch (device buffers only)."""

    def __init__(self, tiles, stream=None):
        """tiles: list of (G [M x N], R_s, R_w, R_b, R_sense)."""
        lib = load()
        self._G = [t[0] for t in tiles]
        arr = (TileDesc * len(tiles))()
        for k, (G, Rs, Rw, Rb, Rse) in enumerate(tiles):
            arr[k] = TileDesc(int(G.shape[0]), int(G.shape[1]), _ptr(G), Rs, Rw, Rb, Rse)
        h = _vp()
        _check(lib.xbar_batch_create(len(tiles), arr, _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h.value
        self.T = len(tiles)

    def autotune(self, precision, B, cache_path=None):
        Barr = (ctypes.c_int * self.T)(*[int(b) for b in B])
        _check(load().xbar_batch_autotune(self.handle, PRECISIONS.get(precision, precision), Barr,
                                          cache_path.encode() if cache_path else None))

    def run(self, precision, Vs, Is, tol=1e-8, max_iter=6, raise_on_error=True):
        """Vs[t]: B_t x M_t, Is[t]: B_t x N_t (CUDA float64 tensors); returns (status, [info dicts])."""
        T = self.T
        Barr = (ctypes.c_int * T)(*[int(v.shape[0]) for v in Vs])
        Varr = (_vp * T)(*[_ptr(v) for v in Vs])
        Iarr = (_vp * T)(*[_ptr(i) for i in Is])
        infos = (SolveInfo * T)()
        st = load().xbar_batch_run(self.handle, PRECISIONS.get(precision, precision), Barr, Varr, Iarr, tol,
                                   max_iter, infos)
        if raise_on_error:
            _check(st)
        return st, [infos[k].as_dict() for k in range(T)]

    def tile_handle(self, t):
        h = _vp()
        _check(load().xbar_batch_tile(self.handle, t, ctypes.byref(h)))
        return h.value

    def destroy(self):
        if self.handle:
            load().xbar_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Surrogate:
    """xbar_surrogate_*: the learned per-column estimate of the currents, with exact fallback."""

    def __init__(self, M, N, circuit, passes=2, g_scale=1e-4, v_scale=0.5, seed=0, stream=None):
        """circuit: (R_s, R_w, R_b, R_sense) of the crossbars modelled; passes: line-model passes."""
        h = _vp()
        _check(load().xbar_surrogate_create(int(M), int(N), *[float(r) for r in circuit], int(passes), g_scale,
                                            v_scale, seed, _stream_ptr(stream), ctypes.byref(h)))
        self.passes = int(passes)
        self.handle = h.value
        self.M, self.N = int(M), int(N)

    def n_params(self):
        n = ctypes.c_int()
        _check(load().xbar_surrogate_params(self.handle, None, None, ctypes.byref(n)))
        return n.value

    def get_params(self):
        out = np.empty(self.n_params(), dtype=np.float32)
        _check(load().xbar_surrogate_params(self.handle, _ptr(out, np.float32), None, None))
        return out

    def set_params(self, P):
        P = np.ascontiguousarray(P, dtype=np.float32)
        _check(load().xbar_surrogate_params(self.handle, None, _ptr(P, np.float32), None))

    def scaling(self, mu=None, sigma=None, c=None):
        """Get (and, given values, first set) the scalars (mu, sigma, c) around the network."""
        cur = np.zeros(3)
        _check(load().xbar_surrogate_scaling(self.handle, None, _ptr(cur)))
        if mu is not None or sigma is not None or c is not None:
            new = np.array([cur[0] if mu is None else mu, cur[1] if sigma is None else sigma,
                            cur[2] if c is None else c], dtype=np.float64)
            _check(load().xbar_surrogate_scaling(self.handle, _ptr(new), _ptr(cur)))
        return tuple(float(v) for v in cur)

    def grad(self, X, y):
        """X: R x 3M float32 features, y: R targets q -> (loss[2], flat gradient float32)."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        loss = np.zeros(2)
        g = np.empty(self.n_params(), dtype=np.float32)
        _check(load().xbar_surrogate_grad(self.handle, int(X.shape[0]), _ptr(X, np.float32), _ptr(y, np.float32),
                                          _ptr(loss), _ptr(g, np.float32)))
        return loss, g

    @staticmethod
    def _maps(Gs, Vs, Is):
        n = len(Gs)
        Garr = (_vp * n)(*[_ptr(G) for G in Gs])
        Varr = (_vp * n)(*[_ptr(V) for V in Vs])
        Iarr = (_vp * n)(*[_ptr(I) for I in Is])
        Barr = (ctypes.c_int * n)(*[int(V.shape[0]) for V in Vs])
        return n, Garr, Barr, Varr, Iarr

    def train(self, Gs, Vs, Is, epochs=10, batch_rows=4096, lr=1e-3, seed=0):
        """Gs[m]: M x N, Vs[m]: B_m x M, Is[m]: B_m x N exact currents -> losses [epochs x 2]."""
        n, Garr, Barr, Varr, Iarr = self._maps(Gs, Vs, Is)
        losses = np.zeros((max(epochs, 1), 2))
        _check(load().xbar_surrogate_train(self.handle, n, Garr, Barr, Varr, Iarr, int(epochs), int(batch_rows), lr,
                                           seed, _ptr(losses)))
        return losses[:epochs]

    def calibrate(self, Gs, Vs, Is, quantile=0.99):
        n, Garr, Barr, Varr, Iarr = self._maps(Gs, Vs, Is)
        c = ctypes.c_double()
        _check(load().xbar_surrogate_calibrate(self.handle, n, Garr, Barr, Varr, Iarr, quantile, ctypes.byref(c)))
        return c.value

    def predict(self, G, V, I, err_est=None):
        _check(load().xbar_surrogate_predict(self.handle, _ptr(G), int(V.shape[0]), _ptr(V), _ptr(I),
                                             _ptr(err_est)))

    def solve(self, exact, V, I, bound=0.01, err_est=None, raise_on_error=True):
        """Predict for the map of Crossbar `exact`, solving vectors above `bound` exactly (device tensors)."""
        info = SolveInfo()
        st = load().xbar_surrogate_solve(self.handle, exact.handle, int(V.shape[0]), _ptr(V), _ptr(I), bound,
                                         _ptr(err_est), ctypes.byref(info))
        if raise_on_error:
            _check(st)
        return st, info.as_dict()

    def destroy(self):
        if self.handle:
            load().xbar_surrogate_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def exported_symbols():
    """Names declared in include/xbar.h (every one must be exported by libxbar.so)."""
    import re
    hdr = open(os.path.join(os.path.dirname(_build.HERE), "include", "xbar.h")).read()
    return sorted(set(re.findall(r"^\s*(?:xbar_status|const char\*)\s+(xbar_\w+)\s*\(", hdr, re.M)))
