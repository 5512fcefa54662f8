"""FP64 CPU oracle for dense -> compact band reduction (sy2sb, ge2gb).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, one-reflector-at-a-time statement of
what the reduction computes (Section 2.1, Eqs. updateA0-updateA2syr2k, read unblocked;
Section 3.1, Eqs. updateB-updateD, read unblocked), written in ``oracle.c``.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  The library never does, and nothing here is shared with the CUDA path.

Arrays are NumPy float64 in column-major (Fortran) order.  Every function copies its
input and returns new arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-shared", "-fPIC", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, dp, c_int = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        lib.oracle_sy2sb.argtypes = [i64, i64, dp, i64, dp, i64]
        lib.oracle_sy2sb.restype = c_int
        lib.oracle_ge2gb.argtypes = [i64, i64, i64, dp, i64, dp, dp, i64]
        lib.oracle_ge2gb.restype = c_int
        lib.oracle_ge2bb.argtypes = [i64, i64, i64, dp, i64, dp, dp, i64]
        lib.oracle_ge2bb.restype = c_int
        lib.oracle_sb2st.argtypes = [i64, i64, dp, i64, dp, dp]
        lib.oracle_sb2st.restype = c_int
        lib.oracle_tridiag_eig.argtypes = [i64, dp, dp, dp]
        lib.oracle_tridiag_eig.restype = c_int
        lib.oracle_gb2bd.argtypes = [i64, i64, dp, i64, dp, dp]
        lib.oracle_gb2bd.restype = c_int
        lib.oracle_bd_singular_values.argtypes = [i64, dp, dp, dp]
        lib.oracle_bd_singular_values.restype = c_int
        lib.oracle_jacobi_eig.argtypes = [i64, dp, i64, dp]
        lib.oracle_jacobi_eig.restype = c_int
        lib.oracle_jacobi_svd.argtypes = [i64, i64, dp, i64, dp]
        lib.oracle_jacobi_svd.restype = c_int
        lib.oracle_set_threads.argtypes = [c_int]
        lib.oracle_set_threads.restype = c_int
        lib.oracle_get_threads.argtypes = []
        lib.oracle_get_threads.restype = c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(t: int) -> int:
    """Threads used by the sweeps (<= 0: all available).  Returns the value in effect."""
    return _load().oracle_set_threads(int(t))


def get_threads() -> int:
    return _load().oracle_get_threads()


def sy2sb(A: np.ndarray, w: int, ncols: int = -1):
    """Reduce symmetric A (lower triangle read) to band form with bandwidth w.

    Returns (Aout, tau): Aout's lower triangle holds the band and the reflectors below
    it (packed); tau has max(n-w, 0) entries.  ``ncols >= 0`` stops after that many
    reflectors (used to time a bounded sample).
    """
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    assert A.shape == (n, n)
    tau = np.zeros(max(n - w, 0) + 1, dtype=np.float64)
    info = _load().oracle_sy2sb(n, w, _ptr(A), max(n, 1), _ptr(tau), ncols)
    if info != 0:
        raise ValueError(f"oracle_sy2sb: info={info}")
    return A, tau[: max(n - w, 0)]


def ge2gb(A: np.ndarray, w: int, ncols: int = -1):
    """Reduce general A (m x n, m >= n) to upper triangular band with upper bandwidth w.

    Returns (Aout, tauq[n], taup[max(n-w,0)]).
    """
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    m, n = A.shape
    tauq = np.zeros(n + 1, dtype=np.float64)
    taup = np.zeros(max(n - w, 0) + 1, dtype=np.float64)
    info = _load().oracle_ge2gb(m, n, w, _ptr(A), max(m, 1), _ptr(tauq), _ptr(taup), ncols)
    if info != 0:
        raise ValueError(f"oracle_ge2gb: info={info}")
    return A, tauq[:n], taup[: max(n - w, 0)]


def ge2bb(A: np.ndarray, w: int, ncols: int = -1):
    """Reduce general A (m x n) to a band with lower and upper bandwidth w (Section 3.3).

    Returns (Aout, tauq[max(min(n, m-w), 0)], taup[max(min(m, n-w), 0)]); the band
    |i - j| <= w of Aout holds B, left reflector c has v in Aout(c+w+1:m, c), right
    reflector c has v in Aout(c, c+w+1:n).
    """
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    m, n = A.shape
    nlq, nrq = max(min(n, m - w), 0), max(min(m, n - w), 0)
    tauq = np.zeros(nlq + 1, dtype=np.float64)
    taup = np.zeros(nrq + 1, dtype=np.float64)
    info = _load().oracle_ge2bb(m, n, w, _ptr(A), max(m, 1), _ptr(tauq), _ptr(taup), ncols)
    if info != 0:
        raise ValueError(f"oracle_ge2bb: info={info}")
    return A, tauq[:nlq], taup[:nrq]


def ge2gb_wide(A: np.ndarray, w: int):
    """Reduce a wide A (m x n, m < n) to LOWER band form with lower bandwidth w.

    Section 3.1 assumes m >= n.  For m < n the reduction is read on the transpose:
    A^T (n x m, tall) = U' B' V'^T by ``ge2gb``, so A = V' B'^T U'^T with B'^T lower band
    (LAPACK's bidiagonal reduction gives a lower bidiagonal for m < n in the same way).
    Returns (Aout, tauq[max(m-w,0)], taup[m]): the lower band 0 <= i-j <= w of Aout holds
    B; left reflector c (acting on rows c+w..m-1, A = Q B P^T, Q = H_0 H_1 ...) has beta on
    Aout(c+w, c) and v in Aout(c+w+1:m, c) with tauq[c]; right reflector c (acting on
    columns c..n-1, P = G_0 G_1 ...) has beta on Aout(c, c) and v in Aout(c, c+1:n) with
    taup[c].
    """
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    m, n = A.shape
    if m > n:
        raise ValueError("ge2gb_wide: m must be < n (use ge2gb for m >= n)")
    T, tq_t, tp_t = ge2gb(np.asfortranarray(A.T), w)
    return np.asfortranarray(T.T), tp_t, tq_t


def sb2st(A: np.ndarray, w: int):
    """Symmetric band (lower triangle, bandwidth w) -> tridiagonal by bulge chasing with
    Householder reflectors (the second stage after the band form).  Returns (d, e)."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    d = np.zeros(max(n, 1))
    e = np.zeros(max(n - 1, 1))
    info = _load().oracle_sb2st(n, w, _ptr(A), max(n, 1), _ptr(d), _ptr(e))
    if info != 0:
        raise ValueError(f"oracle_sb2st: info={info}")
    return d[:n], e[: max(n - 1, 0)]


def tridiag_eig(d: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Eigenvalues (ascending) of the symmetric tridiagonal (d, e) by bisection on Sturm
    counts."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    n = d.shape[0]
    ee = np.zeros(max(n, 1))
    ee[: max(n - 1, 0)] = e[: max(n - 1, 0)]
    lam = np.zeros(max(n, 1))
    info = _load().oracle_tridiag_eig(n, _ptr(d if n else np.zeros(1)), _ptr(ee), _ptr(lam))
    if info != 0:
        raise ValueError(f"oracle_tridiag_eig: info={info}")
    return lam[:n]


def gb2bd(A: np.ndarray, w: int):
    """Upper band (upper triangle, upper bandwidth w) -> upper bidiagonal by bulge chasing
    with Householder reflectors (the SVD's second stage).  Returns (d, e): the diagonal
    and the superdiagonal."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    d = np.zeros(max(n, 1))
    e = np.zeros(max(n - 1, 1))
    info = _load().oracle_gb2bd(n, w, _ptr(A), max(n, 1), _ptr(d), _ptr(e))
    if info != 0:
        raise ValueError(f"oracle_gb2bd: info={info}")
    return d[:n], e[: max(n - 1, 0)]


def bd_singular_values(d: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Singular values (descending) of the upper bidiagonal (d, e), by bisection on its
    Golub-Kahan tridiagonal."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.shape[0]
    ee = np.zeros(max(n, 1))
    ee[: max(n - 1, 0)] = np.asarray(e, dtype=np.float64)[: max(n - 1, 0)]
    sig = np.zeros(max(n, 1))
    info = _load().oracle_bd_singular_values(n, _ptr(d if n else np.zeros(1)), _ptr(ee), _ptr(sig))
    if info != 0:
        raise ValueError(f"oracle_bd_singular_values: info={info}")
    return sig[:n]


def jacobi_eig(A: np.ndarray) -> np.ndarray:
    """Eigenvalues (ascending) of a small symmetric matrix by cyclic Jacobi."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    lam = np.zeros(max(n, 1))
    sweeps = _load().oracle_jacobi_eig(n, _ptr(A), max(n, 1), _ptr(lam))
    if sweeps < 0:
        raise RuntimeError("oracle_jacobi_eig did not converge")
    return np.sort(lam[:n])


def jacobi_svd(A: np.ndarray) -> np.ndarray:
    """Singular values (descending) of a small m x n matrix, m >= n, by one-sided Jacobi."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    m, n = A.shape
    sig = np.zeros(max(n, 1))
    sweeps = _load().oracle_jacobi_svd(m, n, _ptr(A), max(m, 1), _ptr(sig))
    if sweeps < 0:
        raise RuntimeError("oracle_jacobi_svd did not converge")
    return np.sort(sig[:n])[::-1]
