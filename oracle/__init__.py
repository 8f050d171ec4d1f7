"""CPU FP64 oracle for the XbarSim crossbar nodal solve (arXiv 2410.19993).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports this package, and this package imports nothing from it.

The arithmetic lives in ``xref.c`` (plain C, FP64, ``-ffp-contract=off``):
banded LU without pivoting of the nodal matrix in the paper's interleaved
ordering (Sec. II-B, Sec. II-C).  This module only marshals numpy arrays and
adds two thin compositions:

* ``solve``: assemble, decompose once, substitute every input vector of the
  batch (Sec. III-A: one decomposition per batch), extract outputs.
* ``transfer_matrix``: the M x N matrix of bit-line currents produced by unit
  input vectors.  By linearity of the nodal system (I depends linearly on V
  through the right-hand side of Eq. 5), ``I = V @ transfer_matrix`` exactly
  up to rounding; this lets large batches be checked without one substitution
  per vector.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xref.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libxref.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile xref.c into oracle/_build/libxref.so with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    """Declare the C signatures on a loaded libxref (also used on test copies of it)."""
    lib.xref_assemble_band.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
    lib.xref_rhs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _dp]
    lib.xref_lu_band.argtypes = [ctypes.c_longlong, ctypes.c_int, _dp]
    lib.xref_solve_band.argtypes = [ctypes.c_longlong, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                    ctypes.c_int]
    lib.xref_extract.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                 ctypes.c_double, _dp, _dp, _dp, _dp, _dp]
    lib.xref_half_bandwidth.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.xref_num_threads.argtypes = []
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    return int(_load().xref_num_threads())


def half_bandwidth(M: int, N: int) -> int:
    return int(_load().xref_half_bandwidth(M, N))


def assemble_band(M, N, G, Rs, Rw, Rb, Rsense):
    """Nodal matrix (Eqs. 1-7) in band storage, shape (2MN, 4N+1); returns (ab, p)."""
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(M, N)
    p = 2 * N
    ab = np.zeros((2 * M * N, 2 * p + 1), dtype=np.float64)
    rc = _load().xref_assemble_band(M, N, _ptr(G), Rs, Rw, Rb, Rsense, _ptr(ab))
    if rc != 0:
        raise ValueError(f"xref_assemble_band failed (rc={rc}): -1 invalid arguments, "
                         "-2 a node index outside the matrix or its band")
    return ab, p


def band_to_dense(ab, p):
    """Expand band storage to a dense matrix (tests on tiny crossbars only)."""
    k = ab.shape[0]
    A = np.zeros((k, k))
    for r in range(k):
        for c in range(max(0, r - p), min(k, r + p + 1)):
            A[r, c] = ab[r, c - r + p]
    return A


def rhs(M, N, V, Rs):
    """Nodal current vectors for a batch V[B x M]: g_s*V_i at WL(i,1) (Eq. 5)."""
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1, M)
    out = np.zeros((V.shape[0], 2 * M * N))
    _load().xref_rhs(M, N, V.shape[0], _ptr(V), Rs, _ptr(out))
    return out


def lu_band(ab, p):
    """In-place LU without pivoting (Sec. II-C); returns the same array."""
    rc = _load().xref_lu_band(ab.shape[0], p, _ptr(ab))
    if rc != 0:
        raise ZeroDivisionError(f"zero pivot at row {rc}")
    return ab


def solve_band(lu, p, b, nthreads: int = 0):
    """Forward/back substitution of every row of b[B x k] (Sec. II-C)."""
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    x = x.reshape(-1, lu.shape[0])
    _load().xref_solve_band(lu.shape[0], p, _ptr(lu), x.shape[0], _ptr(x), nthreads)
    return x


@dataclass
class Factor:
    M: int
    N: int
    Rs: float
    Rw: float
    Rb: float
    Rsense: float
    lu: np.ndarray
    p: int


def factor(M, N, G, Rs, Rw, Rb, Rsense) -> Factor:
    """Assemble and decompose once (one decomposition serves a whole batch, Sec. III-A)."""
    ab, p = assemble_band(M, N, G, Rs, Rw, Rb, Rsense)
    return Factor(M, N, Rs, Rw, Rb, Rsense, lu_band(ab, p), p)


def solve_factored(f: Factor, V, voltages: bool = False, nthreads: int = 0):
    """Substitute each input vector of V[B x M]; returns a dict of outputs.

    Keys: ``I`` [B x N] bit-line termination currents; ``Isrc`` [B x M] source
    currents; with ``voltages``: ``vWL``, ``vBL`` [B x M x N]; ``x`` the raw
    node-voltage vectors [B x 2MN] in the interleaved ordering.
    """
    M, N = f.M, f.N
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1, M)
    B = V.shape[0]
    x = solve_band(f.lu, f.p, rhs(M, N, V, f.Rs), nthreads)
    I = np.zeros((B, N))
    Isrc = np.zeros((B, M))
    vWL = np.zeros((B, M, N)) if voltages else None
    vBL = np.zeros((B, M, N)) if voltages else None
    _load().xref_extract(M, N, B, _ptr(x), f.Rs, f.Rsense, _ptr(V), _ptr(I), _ptr(vWL), _ptr(vBL),
                         _ptr(Isrc))
    out = {"I": I, "Isrc": Isrc}
    if voltages:
        out.update(vWL=vWL, vBL=vBL, x=x)
    return out


def solve(M, N, G, Rs, Rw, Rb, Rsense, V, voltages: bool = False, nthreads: int = 0):
    """Assemble, decompose, substitute and extract for a batch V[B x M]."""
    return solve_factored(factor(M, N, G, Rs, Rw, Rb, Rsense), V, voltages, nthreads)


def transfer_matrix(f: Factor, nthreads: int = 0):
    """G_eff[i, j] = I_j for the unit input vector V = e_i (M substitutions).

    The nodal system is linear in V, so the currents of any batch are
    ``V @ G_eff`` (exact up to rounding).
    """
    return solve_factored(f, np.eye(f.M), nthreads=nthreads)["I"]
