"""Pins of the oracle's overflow- and underflow-safe norm (CPU only).

The reflector of Section 2.1 / 3.1 needs ||x2||_2 for a column that may hold entries
near the ends of the FP64 range; the oracle computes it as amax * sqrt(sum (x_i/amax)^2)
so that no square overflows or underflows.  Two facts of the mathematics pin that part
without re-typing its formula:

* Power-of-two equivariance.  Multiplying A by 2^s multiplies every intermediate of the
  reduction by 2^s (sums, norms, the band) or leaves it unchanged (v, tau), and a
  product or quotient by a power of two is exact in IEEE arithmetic while nothing
  overflows or underflows.  So the oracle on 2^s A must return exactly 2^s times the
  band and bit-identical reflectors and tau.  With s = +-600 the plain sum of squares
  would overflow (2^1200) or underflow (2^-1200), so an unscaled or wrongly scaled norm
  breaks the identity.
* Closed forms.  A column [3 t, x2] with x2 = [t', t', t', 4 t] (t' far below t) has
  ||x|| = 5 t to the last bit, beta = -5 t, tau = 8/5 and v = x2 / (8 t), whatever the
  power of two t, so the band entry, tau and v are known exactly for t = 2^600 and
  t = 2^-600.

The last tests compile copies of the oracle with planted mistakes in that norm (no
scaling; the maximum taken over only part of the vector) and check that these pins
reject them.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import workloads

_ORACLE_C = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")


# --------------------------------------------------------------------------- runners
class _Lib:
    """ctypes view of an oracle shared library (the real one, or a mutant copy)."""

    def __init__(self, lib):
        i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.oracle_sy2sb.argtypes = [i64, i64, dp, i64, dp, i64]
        lib.oracle_sy2sb.restype = ctypes.c_int
        lib.oracle_ge2gb.argtypes = [i64, i64, i64, dp, i64, dp, dp, i64]
        lib.oracle_ge2gb.restype = ctypes.c_int
        self.lib = lib

    @staticmethod
    def _p(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def sy2sb(self, A, w):
        A = np.array(A, dtype=np.float64, order="F", copy=True)
        n = A.shape[0]
        tau = np.zeros(max(n - w, 0) + 1)
        assert self.lib.oracle_sy2sb(n, w, self._p(A), max(n, 1), self._p(tau), -1) == 0
        return A, tau[: max(n - w, 0)]

    def ge2gb(self, A, w):
        A = np.array(A, dtype=np.float64, order="F", copy=True)
        m, n = A.shape
        tq, tp = np.zeros(n + 1), np.zeros(max(n - w, 0) + 1)
        assert self.lib.oracle_ge2gb(m, n, w, self._p(A), max(m, 1), self._p(tq), self._p(tp), -1) == 0
        return A, tq[:n], tp[: max(n - w, 0)]


def _real():
    return _Lib(oracle._load())


# --------------------------------------------------------------------------- the pins
def equivariance_holds(lib, s, n=40, w=3, m=36, ng=28, wg=2):
    """The oracle on 2^s A returns 2^s B and bit-identical v and tau (sy2sb and ge2gb)."""
    scale = np.ldexp(1.0, s)
    A = workloads.sym_gaussian(n, 101)
    A0, t0 = lib.sy2sb(A, w)
    A1, t1 = lib.sy2sb(A * scale, w)
    i, j = np.indices((n, n))
    band, refl = (i - j >= 0) & (i - j <= w), i - j > w
    ok = np.array_equal(A1[band], A0[band] * scale) and np.array_equal(A1[refl], A0[refl])
    ok = ok and np.array_equal(t1, t0)
    G = workloads.gen_gaussian(m, ng, 102)
    G0, q0, p0 = lib.ge2gb(G, wg)
    G1, q1, p1 = lib.ge2gb(G * scale, wg)
    i, j = np.indices((m, ng))
    gband = (j - i >= 0) & (j - i <= wg)
    ok = ok and np.array_equal(G1[gband], G0[gband] * scale) and np.array_equal(G1[~gband], G0[~gband])
    return bool(ok and np.array_equal(q1, q0) and np.array_equal(p1, p0))


def _column_case(t, tiny):
    """x = [3t; tiny, tiny, tiny, 4t] as column 0 of a symmetric matrix (n = 6, w = 1)
    that is zero elsewhere, and the same column as a 5 x 2 general matrix."""
    x = np.array([3.0 * t, tiny, tiny, tiny, 4.0 * t])
    A = np.zeros((6, 6))
    A[1:, 0] = x
    A[0, 1:] = x
    G = np.zeros((5, 2))
    G[:, 0] = x
    return A, G, x


def closed_form_holds(lib, s):
    t = np.ldexp(1.0, s)
    # ||x2|| = 4t exactly (3 tiny^2 is far below half an ulp of 16 t^2); for t = 2^600 the
    # small entries are 2^-600 of the large one, so a norm scaled by a maximum that misses
    # the large entry squares 2^602 and overflows
    tiny = np.ldexp(1.0, s - 600) if s > 0 else np.ldexp(1.0, s - 100)
    A, G, x = _column_case(t, tiny)
    beta, tau, v = -5.0 * t, 8.0 / 5.0, x[1:] / (8.0 * t)  # alpha - beta = 8t: v is exact
    Ao, to = lib.sy2sb(A, 1)
    ok = Ao[1, 0] == beta and to[0] == tau and np.array_equal(Ao[2:, 0], v) and np.all(to[1:] == 0.0)
    Go, qo, po = lib.ge2gb(G, 1)
    ok = ok and Go[0, 0] == beta and qo[0] == tau and np.array_equal(Go[1:, 0], v)
    return bool(ok)


@pytest.mark.parametrize("s", [-600, 600])
def test_power_of_two_scaling_is_exact(s):
    assert equivariance_holds(_real(), s)


@pytest.mark.parametrize("s", [-600, 600])
def test_norm_closed_form_beyond_the_square_range(s):
    assert closed_form_holds(_real(), s)


def test_unscaled_squares_would_fail_here():
    """The cases above lie where the plain sum of squares leaves the FP64 range."""
    with np.errstate(over="ignore", under="ignore"):
        big = np.ldexp(1.0, 600)
        assert np.isinf(np.float64(4.0 * big) ** 2)
        small = np.ldexp(1.0, -600)
        assert np.float64(4.0 * small) ** 2 == 0.0


# --------------------------------------------------------------------------- planted mistakes
_MUTANTS = {
    # the textbook sum of squares with no scaling
    "no_scaling": [("double t = x[i * inc] / amax;", "double t = x[i * inc];"),
                   ("return amax * sqrt(s);", "return sqrt(s);")],
    # the maximum taken over the first half of the vector only
    "max_of_first_half": [("for (int64_t i = 0; i < len; ++i) {\n        double a = fabs(x[i * inc]);",
                           "for (int64_t i = 0; i < (len + 1) / 2; ++i) {\n        double a = fabs(x[i * inc]);")],
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
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", str(so), str(c), "-lm"], check=True,
                   capture_output=True)
    return _Lib(ctypes.CDLL(str(so)))


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_pins_reject_a_planted_norm_mistake(tmp_path, name):
    lib = _build_mutant(tmp_path, name)
    with np.errstate(all="ignore"):
        caught = [not equivariance_holds(lib, s) for s in (-600, 600)]
        caught += [not closed_form_holds(lib, s) for s in (-600, 600)]
    assert any(caught), name
    # and the mutant still agrees with the real oracle to rounding on O(1) data, where every
    # older pin passes: only the pins of this file tell them apart
    A = workloads.sym_gaussian(30, 7)
    Ar, tr = _real().sy2sb(A, 2)
    Am, tm = lib.sy2sb(A, 2)
    np.testing.assert_allclose(np.tril(Am), np.tril(Ar), rtol=0, atol=1e-12)
    np.testing.assert_allclose(tm, tr, rtol=0, atol=1e-12)
