"""Pins of the SVD second-stage oracle (CPU only): upper band -> upper bidiagonal by
bulge chasing (oracle.gb2bd) and the singular values of an upper bidiagonal
(oracle.bd_singular_values).

What fixes them without re-typing their steps:

* Orthogonal equivalence.  B = U^T A V keeps the singular values of the band (LAPACK's
  dense SVD, a different algorithm, and the oracle's one-sided Jacobi on tiny inputs)
  and its Frobenius norm (sum d^2 + sum e^2 = ||A||_F^2).  A dropped term, a wrong sign,
  a reflector from the wrong row or column, or an application window that misses a
  nonzero breaks the singular values.
* Special cases.  w = 1 is already bidiagonal: no reflector acts, d and e are the input
  bit for bit, and so is a bidiagonal input under a wider nominal w (every reflector
  meets a zero tail).  n = 3, w = 2 by hand: the first right reflector on [a01, a02] gives
  e0 = -sign(a01) hypot(a01, a02) (the larfg convention) and leaves a00; the trailing
  2 x 2 block keeps the singular values of A(1:3, 1:3).
* Closed form for the singular values: the upper bidiagonal with d = e = 1 of order n has
  2 cos(k pi / (2n + 1)), k = 1 .. n.  A diagonal has its absolute values.

The last tests compile copies of the oracle with planted mistakes and check that these
pins reject them.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

_ORACLE_C = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")


class _Lib:
    def __init__(self, lib):
        i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.oracle_gb2bd.argtypes = [i64, i64, dp, i64, dp, dp]
        lib.oracle_gb2bd.restype = ctypes.c_int
        lib.oracle_bd_singular_values.argtypes = [i64, dp, dp, dp]
        lib.oracle_bd_singular_values.restype = ctypes.c_int
        self.lib = lib

    @staticmethod
    def _p(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def gb2bd(self, A, w):
        A = np.array(A, dtype=np.float64, order="F", copy=True)
        n = A.shape[0]
        d, e = np.zeros(max(n, 1)), np.zeros(max(n - 1, 1))
        assert self.lib.oracle_gb2bd(n, w, self._p(A), max(n, 1), self._p(d), self._p(e)) == 0
        return d[:n], e[: max(n - 1, 0)]

    def bd_sv(self, d, e):
        d = np.ascontiguousarray(d, dtype=np.float64)
        n = d.shape[0]
        ee = np.zeros(max(n, 1))
        ee[: n - 1] = e
        s = np.zeros(max(n, 1))
        assert self.lib.oracle_bd_singular_values(n, self._p(d), self._p(ee), self._p(s)) == 0
        return s[:n]


def _real():
    return _Lib(oracle._load())


def upper_band(n, w, seed):
    rng = np.random.default_rng(seed)
    A = np.triu(rng.standard_normal((n, n)))
    return np.triu(A) - np.triu(A, w + 1)


def bidiag(d, e):
    return np.diag(d) + np.diag(e, 1)


def equivalence_holds(lib, n, w, seed):
    A = upper_band(n, w, seed)
    d, e = lib.gb2bd(A, w)
    if not (np.all(np.isfinite(d)) and np.all(np.isfinite(e))):
        return False
    sa = np.linalg.svd(A, compute_uv=False)
    sb = np.linalg.svd(bidiag(d, e), compute_uv=False)
    nrm = max(sa.max(), 1e-300)
    ok = np.max(np.abs(sb - sa)) <= 50 * n * 2.0 ** -53 * nrm
    ok = ok and abs((d @ d + e @ e) - np.sum(A * A)) <= 1e-13 * n * np.sum(A * A)
    return bool(ok)


@pytest.mark.parametrize("n,w", [(20, 4), (33, 5), (17, 16), (100, 8), (3, 2), (150, 31), (64, 63), (41, 2)])
def test_bidiagonal_is_an_orthogonal_equivalence_of_the_band(n, w):
    assert equivalence_holds(_real(), n, w, 10 * n + w)


def test_small_against_one_sided_jacobi():
    for n, w in [(6, 3), (9, 4), (12, 11)]:
        A = upper_band(n, w, n + w)
        d, e = oracle.gb2bd(A, w)
        sj = np.sort(oracle.jacobi_svd(bidiag(d, e)))[::-1]
        sa = np.sort(oracle.jacobi_svd(A))[::-1]
        assert np.max(np.abs(sj - sa)) <= 1e-13 * sa.max()


def test_bandwidth_one_is_left_alone():
    A = upper_band(40, 1, 3)
    d, e = oracle.gb2bd(A, 1)
    assert np.array_equal(d, np.diag(A)) and np.array_equal(e, np.diag(A, 1))
    d2, e2 = oracle.gb2bd(A, 5)
    assert np.array_equal(d2, d) and np.array_equal(e2, e)


def test_order_three_by_hand():
    a00, a01, a02, a11, a12, a22 = 1.5, -3.0, 4.0, 0.25, -2.0, 7.0
    A = np.array([[a00, a01, a02], [0.0, a11, a12], [0.0, 0.0, a22]])
    d, e = oracle.gb2bd(A, 2)
    assert d[0] == a00
    assert e[0] == pytest.approx(-np.sign(a01) * np.hypot(a01, a02), rel=0, abs=1e-15)  # +5
    s_tail = np.linalg.svd(np.array([[d[1], e[1]], [0.0, d[2]]]), compute_uv=False)
    assert np.allclose(s_tail, np.linalg.svd(A[1:, 1:], compute_uv=False), rtol=0, atol=1e-14)


def test_empty_and_tiny_orders():
    d, e = oracle.gb2bd(np.zeros((0, 0)), 3)
    assert d.shape == (0,) and e.shape == (0,)
    d, e = oracle.gb2bd(np.array([[2.0]]), 3)
    assert d.tolist() == [2.0] and e.shape == (0,)
    d, e = oracle.gb2bd(np.array([[1.0, 2.0], [0.0, -1.0]]), 4)
    assert d.tolist() == [1.0, -1.0] and e.tolist() == [2.0]


# --------------------------------------------------------------------------- singular values
def sv_pins_hold(lib):
    ok = True
    for n in (1, 2, 7, 64, 257):
        s = lib.bd_sv(np.ones(n), np.ones(n - 1))
        ref = 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (2 * n + 1))
        ok = ok and np.max(np.abs(s - ref)) <= 1e-14
    dg = np.array([3.0, -1.0, 2.5, 0.0, -7.0])
    ok = ok and np.max(np.abs(lib.bd_sv(dg, np.zeros(4)) - np.sort(np.abs(dg))[::-1])) <= 4 * 2.0 ** -53 * 7.0
    rng = np.random.default_rng(5)
    for n in (10, 200):
        d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
        ref = np.linalg.svd(bidiag(d, e), compute_uv=False)
        ok = ok and np.max(np.abs(lib.bd_sv(d, e) - ref)) <= 1e-13 * ref.max()
    return bool(ok)


def test_bidiagonal_singular_value_pins():
    assert sv_pins_hold(_real())


# --------------------------------------------------------------------------- planted mistakes
_MUTANTS = {
    # the chase's next range starts w - 1 after the previous one instead of w
    "chase_offset": [("            r = a;\n            a += w;\n        }\n    }\n    for (int64_t i = 0; i < n; ++i) d[i] = AT(M, n, i, i);\n    for (int64_t i = 0; i + 1 < n; ++i) e[i] = AT(M, n, i, i + 1);",
                      "            r = a;\n            a += w - 1;\n        }\n    }\n    for (int64_t i = 0; i < n; ++i) d[i] = AT(M, n, i, i);\n    for (int64_t i = 0; i + 1 < n; ++i) e[i] = AT(M, n, i, i + 1);")],
    # the right reflector skips the rows below its range (the lower bulge is never made)
    "right_window": [("int64_t lo = a - 2 * w > 0 ? a - 2 * w : 0, hi = end + w < n ? end + w : n;",
                      "int64_t lo = a - 2 * w > 0 ? a - 2 * w : 0, hi = a;")],
    # the left reflector is taken from the column after its range start
    "left_column": [("            house(len, &AT(M, n, a, a), 1, &t);", "            house(len, &AT(M, n, a, a + 1), 1, &t);")],
    # the Golub-Kahan tridiagonal drops the last diagonal entry of the bidiagonal
    "gk_last": [("    for (int64_t i = 0; i < n; ++i) {\n        o[2 * i] = d[i];", "    for (int64_t i = 0; i + 1 < n; ++i) {\n        o[2 * i] = d[i];")],
}


def _build_mutant(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(_ORACLE_C).read()
    for old, new in _MUTANTS[name]:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    c = tmp_path / f"oracle_{name}.c"
    so = tmp_path / f"liboracle_{name}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", str(so), str(c), "-lm"], check=True, capture_output=True)
    return _Lib(ctypes.CDLL(str(so)))


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_pins_reject_a_planted_mistake(tmp_path, name):
    lib = _build_mutant(tmp_path, name)
    with np.errstate(all="ignore"):
        if name.startswith("gk"):
            assert not sv_pins_hold(lib)
        else:
            assert not all(equivalence_holds(lib, n, w, 10 * n + w) for n, w in [(33, 5), (100, 8), (150, 31)])
