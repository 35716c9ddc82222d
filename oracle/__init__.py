"""CPU parity oracle for the banded Cholesky library (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and it
imports nothing from the library.  Every routine is a plain serial FP64 loop
in ``bchol_oracle.c`` (compiled with ``-O2 -ffp-contract=off``).

Band arrays are numpy float64 arrays of shape (ldab, n) in Fortran order, so
``ab[d, j]`` is LAPACK's ``AB(1+d, 1+j)`` = A(j+d, j) of the lower band.

Paper: Liu, Fredriksson, Markidis, "Parallel Cholesky Factorization for
Banded Matrices using OpenMP Tasks" (arXiv 2305.04635).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bchol_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (serial, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_pbtrf.argtypes = [I, I, P, I]
        lib.oracle_pbtrf.restype = I
        lib.oracle_pbtrs.argtypes = [I, I, I, P, I, P, I]
        lib.oracle_pbtrs.restype = I
        lib.oracle_logdet.argtypes = [I, P, I]
        lib.oracle_logdet.restype = D
        lib.oracle_sbmv.argtypes = [I, I, I, P, I, P, I, P, I]
        lib.oracle_sbmv.restype = I
        lib.oracle_backward_error.argtypes = [I, I, P, I, P, I]
        lib.oracle_backward_error.restype = D
        lib.oracle_llt_residual_sampled.argtypes = [I, I, P, I, P, I, I, P, P, P]
        lib.oracle_llt_residual_sampled.restype = None
        lib.oracle_sbmv_residual_sampled.argtypes = [I, I, P, I, P, P, I, P, P]
        lib.oracle_sbmv_residual_sampled.restype = None
        lib.oracle_flops_eq1.argtypes = [ctypes.c_int64, ctypes.c_int64]
        lib.oracle_flops_eq1.restype = ctypes.c_uint64
        lib.oracle_inverse_band.argtypes = [I, I, P, I, P, I, P]
        lib.oracle_inverse_band.restype = None
        lib.oracle_band_grad_sampled.argtypes = [I, I, P, I, P, P, D, I, P, P, P, P]
        lib.oracle_band_grad_sampled.restype = None
        _lib = lib
    return _lib


def _band(ab: np.ndarray) -> np.ndarray:
    if ab.dtype != np.float64 or ab.ndim != 2 or not ab.flags.f_contiguous:
        raise ValueError("band array must be a Fortran-ordered float64 (ldab, n) array")
    return ab


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def pbtrf(ab: np.ndarray, k: int) -> tuple[np.ndarray, int]:
    """Return (L band, info): the left-looking band Cholesky of Algorithm 2 on a copy of `ab`."""
    L = np.array(_band(ab), order="F", copy=True)
    ldab, n = L.shape
    info = _load().oracle_pbtrf(n, k, _ptr(L), ldab)
    if info < 0:
        raise ValueError("oracle_pbtrf: argument error")
    return L, int(info)


def pbtrs(l_band: np.ndarray, k: int, b: np.ndarray) -> np.ndarray:
    """X = A^{-1} B from the factor band (forward then back substitution). B: (n,) or (n, nrhs)."""
    _band(l_band)
    ldab, n = l_band.shape
    vec = b.ndim == 1
    X = np.array(b.reshape(n, -1), dtype=np.float64, order="F", copy=True)
    rc = _load().oracle_pbtrs(n, k, X.shape[1], _ptr(l_band), ldab, _ptr(X), max(1, n))
    if rc < 0:
        raise ValueError("oracle_pbtrs: argument error")
    return X[:, 0].copy() if vec else X


def logdet(l_band: np.ndarray) -> float:
    """log det A = 2 sum log L_ii."""
    _band(l_band)
    ldab, n = l_band.shape
    return float(_load().oracle_logdet(n, _ptr(l_band), ldab))


def sbmv(a_band: np.ndarray, k: int, x: np.ndarray) -> np.ndarray:
    """y = A x for the symmetric band matrix held by its lower band."""
    _band(a_band)
    ldab, n = a_band.shape
    vec = x.ndim == 1
    X = np.array(x.reshape(n, -1), dtype=np.float64, order="F", copy=True)
    Y = np.zeros_like(X, order="F")
    _load().oracle_sbmv(n, k, X.shape[1], _ptr(a_band), ldab, _ptr(X), max(1, n), _ptr(Y), max(1, n))
    return Y[:, 0].copy() if vec else Y


def backward_error(a_band: np.ndarray, l_band: np.ndarray, k: int) -> float:
    """||A - L L^T||_F / ||A||_F with compensated (Dot2) residual entries."""
    _band(a_band)
    _band(l_band)
    n = a_band.shape[1]
    return float(_load().oracle_backward_error(n, k, _ptr(a_band), a_band.shape[0], _ptr(l_band),
                                               l_band.shape[0]))


def llt_residual_sampled(a_band, l_band, k, rows, cols) -> np.ndarray:
    """(A - L L^T)(rows[q], cols[q]) for sampled band positions (rows >= cols), by Dot2."""
    _band(a_band)
    _band(l_band)
    n = a_band.shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros(rows.size)
    _load().oracle_llt_residual_sampled(n, k, _ptr(a_band), a_band.shape[0], _ptr(l_band), l_band.shape[0],
                                        rows.size, _ptr(rows), _ptr(cols), _ptr(out))
    return out


def sbmv_residual_sampled(a_band, k, x, b, rows) -> np.ndarray:
    """b_i - (A x)_i for sampled rows, by Dot2."""
    _band(a_band)
    n = a_band.shape[1]
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros(rows.size)
    _load().oracle_sbmv_residual_sampled(n, k, _ptr(a_band), a_band.shape[0], _ptr(x), _ptr(b), rows.size,
                                         _ptr(rows), _ptr(out))
    return out


def flops_eq1_bruteforce(N: int, k: int) -> int:
    """Eq. (1) summed term by term (O(N k^2); small cases only)."""
    return int(_load().oracle_flops_eq1(N, k))


def inverse_band(l_band: np.ndarray, k: int) -> np.ndarray:
    """Lower band of A^{-1}, column by column from A s = e_j."""
    _band(l_band)
    ldab, n = l_band.shape
    sig = np.zeros((k + 1, n), order="F")
    work = np.zeros(max(1, n))
    _load().oracle_inverse_band(n, k, _ptr(l_band), ldab, _ptr(sig), k + 1, _ptr(work))
    return sig


def band_grad_sampled(l_band, k, x, bbar, ldbar, rows, cols) -> np.ndarray:
    """d f / d ab(rows-cols, cols) for f(x, log det A), x = A^{-1} b, given bbar = A^{-1} xbar."""
    _band(l_band)
    ldab, n = l_band.shape
    x = np.ascontiguousarray(x, dtype=np.float64)
    bbar = np.ascontiguousarray(bbar, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros(rows.size)
    work = np.zeros(max(1, n))
    _load().oracle_band_grad_sampled(n, k, _ptr(l_band), ldab, _ptr(x), _ptr(bbar), float(ldbar), rows.size,
                                     _ptr(rows), _ptr(cols), _ptr(out), _ptr(work))
    return out
