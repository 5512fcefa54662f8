"""Pins of the second-stage oracle (CPU only): band -> tridiagonal by bulge chasing
(oracle.sb2st) and the eigenvalues of a symmetric tridiagonal by bisection
(oracle.tridiag_eig).

What fixes them without re-typing their steps:

* Orthogonal similarity.  The tridiagonal T = Q^T B Q has the eigenvalues of the band B
  (LAPACK's dense eigvalsh, a different algorithm, within the backward-error bound), its
  trace, and its Frobenius norm (sum d^2 + 2 sum e^2 = ||B||_F^2).  A dropped term, a
  wrong sign or a reflector applied on the wrong range breaks the eigenvalues.
* Special cases.  w = 1 is already tridiagonal: no reflector acts, d and e are the input
  bit for bit.  n = 3, w = 2: one reflector on [a10; a20] gives e0 = -sign(a10) hypot(a10,
  a20) (the larfg convention) and the trailing 2 x 2 block is fixed by trace and
  determinant.  A band that is already tridiagonal plus zeros stays as it is.
* Closed form for the eigenvalues: tridiag(-1, 2, -1) of order n has
  2 - 2 cos(k pi / (n + 1)).  A diagonal T (e = 0) has its sorted diagonal (to the
  bisection's stopping width, a few units in the last place of max |T|).  LAPACK's
  eigvalsh_tridiagonal on random T.  The Wilkinson matrix W21+ has close pairs.

The last tests compile copies of the oracle with planted mistakes (a chase step on the
wrong range, a Sturm count off by one) and check that these pins reject them.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads

_ORACLE_C = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")


class _Lib:
    def __init__(self, lib):
        i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.oracle_sb2st.argtypes = [i64, i64, dp, i64, dp, dp]
        lib.oracle_sb2st.restype = ctypes.c_int
        lib.oracle_tridiag_eig.argtypes = [i64, dp, dp, dp]
        lib.oracle_tridiag_eig.restype = ctypes.c_int
        self.lib = lib

    @staticmethod
    def _p(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def sb2st(self, A, w):
        A = np.array(A, dtype=np.float64, order="F", copy=True)
        n = A.shape[0]
        d, e = np.zeros(max(n, 1)), np.zeros(max(n - 1, 1))
        assert self.lib.oracle_sb2st(n, w, self._p(A), max(n, 1), self._p(d), self._p(e)) == 0
        return d[:n], e[: max(n - 1, 0)]

    def tridiag_eig(self, d, e):
        d = np.ascontiguousarray(d, dtype=np.float64)
        n = d.shape[0]
        ee = np.zeros(max(n, 1))
        ee[: n - 1] = e
        lam = np.zeros(max(n, 1))
        assert self.lib.oracle_tridiag_eig(n, self._p(d), self._p(ee), self._p(lam)) == 0
        return lam[:n]


def _real():
    return _Lib(oracle._load())


def band_of(n, w, seed):
    A = workloads.sym_gaussian(n, seed)
    i, j = np.indices((n, n))
    A[np.abs(i - j) > w] = 0.0
    return A


def similarity_holds(lib, n, w, seed):
    A = band_of(n, w, seed)
    d, e = lib.sb2st(np.tril(A), w)
    la = np.linalg.eigvalsh(A)
    lt = sl.eigvalsh_tridiagonal(d, e)
    nrm = max(np.abs(la).max(), 1e-300)
    ok = np.max(np.abs(lt - la)) <= 50 * n * 2.0 ** -53 * nrm
    ok = ok and abs(d.sum() - np.trace(A)) <= 1e-13 * n * nrm
    ok = ok and abs((d @ d + 2 * e @ e) - np.sum(A * A)) <= 1e-13 * n * np.sum(A * A)
    return bool(ok)


@pytest.mark.parametrize("n,w", [(20, 4), (33, 5), (17, 16), (100, 8), (3, 2), (150, 31), (64, 63)])
def test_tridiagonal_is_an_orthogonal_similarity_of_the_band(n, w):
    assert similarity_holds(_real(), n, w, 10 * n + w)


def test_bandwidth_one_is_left_alone():
    A = band_of(40, 1, 3)
    d, e = oracle.sb2st(np.tril(A), 1)
    assert np.array_equal(d, np.diag(A)) and np.array_equal(e, np.diag(A, -1))
    # a wider nominal bandwidth over a tridiagonal input changes nothing either (every
    # reflector meets a zero tail: tau = 0)
    d2, e2 = oracle.sb2st(np.tril(A), 5)
    assert np.array_equal(d2, d) and np.array_equal(e2, e)


def test_order_three_by_hand():
    a00, a10, a20, a11, a21, a22 = 1.5, -3.0, 4.0, 0.25, -2.0, 7.0
    A = np.array([[a00, a10, a20], [a10, a11, a21], [a20, a21, a22]])
    d, e = oracle.sb2st(np.tril(A), 2)
    assert d[0] == a00
    assert e[0] == pytest.approx(-np.sign(a10) * np.hypot(a10, a20), rel=0, abs=1e-15)  # beta = +5
    # the trailing 2 x 2 block is orthogonally similar to A(1:3, 1:3)
    tr, det = a11 + a22, a11 * a22 - a21 * a21
    assert d[1] + d[2] == pytest.approx(tr, abs=1e-14)
    assert d[1] * d[2] - e[1] ** 2 == pytest.approx(det, abs=1e-13)
    # reflector H = I - tau v v^T on [a10; a20] = [-3; 4]: beta = 5, H [-3; 4] = [5; 0]
    v = np.array([1.0, 4.0 / (-3.0 - 5.0)])
    tau = (5.0 + 3.0) / 5.0
    H = np.eye(2) - tau * np.outer(v, v)
    B = H @ A[1:, 1:] @ H
    assert np.allclose([d[1], d[2], e[1]], [B[0, 0], B[1, 1], B[1, 0]], rtol=0, atol=1e-14)


def test_empty_and_tiny_orders():
    d, e = oracle.sb2st(np.zeros((0, 0)), 3)
    assert d.shape == (0,) and e.shape == (0,)
    d, e = oracle.sb2st(np.array([[2.0]]), 3)
    assert d.tolist() == [2.0] and e.shape == (0,)
    A = np.array([[1.0, 2.0], [2.0, -1.0]])
    d, e = oracle.sb2st(np.tril(A), 4)
    assert d.tolist() == [1.0, -1.0] and e.tolist() == [2.0]


# --------------------------------------------------------------------------- eigenvalues
def eig_pins_hold(lib):
    ok = True
    for n in (1, 2, 7, 64, 257):
        lam = lib.tridiag_eig(np.full(n, 2.0), np.full(n - 1, -1.0))
        ref = 2.0 - 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
        ok = ok and np.max(np.abs(lam - np.sort(ref))) <= 1e-14
    dg = np.array([3.0, -1.0, 2.5, 0.0, -7.0, 2.5])  # bisection stops within 4 ulps of max |T|
    ok = ok and np.max(np.abs(lib.tridiag_eig(dg, np.zeros(5)) - np.sort(dg))) <= 4 * 2.0 ** -53 * 7.0
    rng = np.random.default_rng(5)
    for n in (10, 200):
        d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
        ref = sl.eigvalsh_tridiagonal(d, e)
        ok = ok and np.max(np.abs(lib.tridiag_eig(d, e) - ref)) <= 1e-13 * np.abs(ref).max()
    # Wilkinson W21+: d = |10 - i|, e = 1; its two largest eigenvalues agree to 14 digits
    d = np.abs(10.0 - np.arange(21))
    lam = lib.tridiag_eig(d, np.ones(20))
    ref = sl.eigvalsh_tridiagonal(d, np.ones(20))
    ok = ok and np.max(np.abs(lam - ref)) <= 1e-13 * 11.0
    return bool(ok)


def test_tridiagonal_eigenvalue_pins():
    assert eig_pins_hold(_real())


def test_eigenvalue_scale_range():
    """Entries near 2^+-500 (the squares in the Sturm recurrence stay in range)."""
    for s in (-500, 500):
        c = np.ldexp(1.0, s)
        lam = oracle.tridiag_eig(np.full(9, 2.0 * c), np.full(8, -c))
        ref = c * (2.0 - 2.0 * np.cos(np.arange(1, 10) * np.pi / 10))
        assert np.max(np.abs(lam - ref)) <= 1e-14 * 4 * c


# --------------------------------------------------------------------------- planted mistakes
_MUTANTS = {
    # the chase's next range starts w - 1 after the previous one instead of w
    "chase_offset": [("            col = s;\n            s += w;", "            col = s;\n            s += w - 1;")],
    # the bulge's right application skips the rows below the reflector's range
    "right_window": [("int64_t lo = s - 2 * w > 0 ? s - 2 * w : 0, hi = end + 2 * w < n ? end + 2 * w : n;",
                      "int64_t lo = s - 2 * w > 0 ? s - 2 * w : 0, hi = end;")],
    # a Sturm count that also counts the first term's sign the wrong way
    "sturm_first": [("    if (fabs(q) < pivmin) q = -pivmin;\n    if (q < 0.0) ++neg;\n    for",
                     "    if (fabs(q) < pivmin) q = -pivmin;\n    if (q > 0.0) ++neg;\n    for")],
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
        if name.startswith("sturm"):
            assert not eig_pins_hold(lib)
        else:
            assert not all(similarity_holds(lib, n, w, 10 * n + w) for n, w in [(33, 5), (100, 8), (150, 31)])
