"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Section 2.1 (symmetric band, A = Q B Q^T) and Section 3.1 (triangular band,
A = U B V^T): band shape, reconstruction through independently formed factors,
orthogonality, preserved spectra (against LAPACK and against the oracle's own Jacobi,
which is itself pinned to closed forms), hand-derived small cases and the Householder
sign convention.  A final group plants mistakes in oracle outputs and shows that these
pins catch them.
"""
import numpy as np
import pytest

import oracle
import workloads
from checks import U64, gen_band, gen_form_uv, gen_report, sym_band, sym_form_q, sym_report, sym_probe_backward


# --------------------------------------------------------------------------- Jacobi
def test_jacobi_eig_closed_form_2x2():
    # eigenvalues of [[a, b], [b, d]] are (a+d)/2 +- sqrt(((a-d)/2)^2 + b^2)
    a, b, d = 3.0, -2.0, 0.5
    lam = oracle.jacobi_eig(np.array([[a, b], [b, d]]))
    r = np.hypot((a - d) / 2, b)
    np.testing.assert_allclose(lam, [(a + d) / 2 - r, (a + d) / 2 + r], rtol=0, atol=4 * U64 * 4)


def test_jacobi_eig_known_spectrum_and_lapack():
    A, lam = workloads.sym_known_spectrum(40, 3, 4)
    got = oracle.jacobi_eig(A)
    assert np.max(np.abs(got - lam)) < 1e-14
    assert np.max(np.abs(got - np.linalg.eigvalsh(A))) < 1e-14
    d = np.array([5.0, -1.0, 0.0, 2.5])
    np.testing.assert_array_equal(oracle.jacobi_eig(np.diag(d)), np.sort(d))


def test_jacobi_svd_closed_form_and_lapack():
    # singular values of [[3, 0], [4, 5]] are sqrt(45) and sqrt(5)
    s = oracle.jacobi_svd(np.array([[3.0, 0.0], [4.0, 5.0]]))
    np.testing.assert_allclose(s, [np.sqrt(45.0), np.sqrt(5.0)], rtol=1e-15)
    A, sig = workloads.gen_known_singular(30, 20, 2)
    got = oracle.jacobi_svd(A)
    assert np.max(np.abs(got - sig)) < 1e-14
    G = workloads.gen_gaussian(25, 18, 9)
    np.testing.assert_allclose(oracle.jacobi_svd(G), np.linalg.svd(G, compute_uv=False), rtol=1e-13)


# --------------------------------------------------------------------------- closed forms
def test_sy2sb_hand_case_n3_w1():
    """One reflector on [a10; a20] of a 3x3 symmetric matrix, evaluated exactly."""
    sp = pytest.importorskip("sympy")
    Aint = [[4, 1, 2], [1, 2, 0], [2, 0, 3]]
    A = sp.Matrix(Aint)
    alpha, x2 = A[1, 0], A[2, 0]
    beta = -sp.sqrt(alpha ** 2 + x2 ** 2)  # alpha > 0
    tau = (beta - alpha) / beta
    v = sp.Matrix([1, x2 / (alpha - beta)])
    H = sp.eye(3)
    H[1:, 1:] = sp.eye(2) - tau * v * v.T
    # H maps the column to beta e1 and is orthogonal
    assert sp.simplify((H[1:, 1:] * sp.Matrix([alpha, x2]) - sp.Matrix([beta, 0]))).is_zero_matrix
    B = (H * A * H).applyfunc(sp.nsimplify)
    Bf = np.array(B.evalf(30).tolist(), dtype=np.float64)
    Aout, t = oracle.sy2sb(np.array(Aint, dtype=np.float64), 1)
    assert t.shape == (2,)
    np.testing.assert_allclose(t[0], float(tau.evalf(30)), rtol=4 * U64)
    assert t[1] == 0.0  # length-1 reflector
    np.testing.assert_allclose(Aout[2, 0], float(v[1].evalf(30)), rtol=4 * U64)
    for (i, j) in [(0, 0), (1, 0), (1, 1), (2, 1), (2, 2)]:
        assert abs(Aout[i, j] - Bf[i, j]) <= 8 * U64 * 6.0, (i, j)
    assert Aout[1, 0] == pytest.approx(-np.sqrt(5.0), rel=2 * U64)


def test_ge2gb_hand_case_3x2_w1():
    """m=3, n=2, w=1: only left reflectors; B(0,0) = -sign(a00)||A(:,0)||."""
    sp = pytest.importorskip("sympy")
    Aint = [[-2, 1], [1, 3], [2, -1]]
    A = sp.Matrix(Aint)
    x = A[:, 0]
    beta0 = sp.sqrt(x.dot(x))  # alpha = -2 < 0  ->  beta = +||x||
    tau0 = (beta0 - x[0]) / beta0
    v0 = sp.Matrix([1, x[1] / (x[0] - beta0), x[2] / (x[0] - beta0)])
    H0 = sp.eye(3) - tau0 * v0 * v0.T
    A1 = H0 * A
    y = A1[1:, 1]
    beta1 = (-1 if y[0] >= 0 else 1) * sp.sqrt(y.dot(y))
    Aout, tq, tp = oracle.ge2gb(np.array(Aint, dtype=np.float64), 1)
    assert tp.shape == (1,) and tp[0] == 0.0
    np.testing.assert_allclose(Aout[0, 0], float(beta0.evalf(30)), rtol=4 * U64)
    np.testing.assert_allclose(Aout[0, 1], float(A1[0, 1].evalf(30)), rtol=16 * U64)
    np.testing.assert_allclose(Aout[1, 1], float(beta1.evalf(30)), rtol=16 * U64)
    np.testing.assert_allclose(tq[0], float(tau0.evalf(30)), rtol=4 * U64)


def test_householder_conventions():
    # alpha = 0: beta = -||x|| (sign(0) = +1)
    A = np.zeros((3, 3))
    A[2, 0] = A[0, 2] = 3.0
    A[1, 1] = 1.0
    Aout, t = oracle.sy2sb(A, 1)
    assert Aout[1, 0] == -3.0 and t[0] == 1.0
    # column already reduced: tau = 0 and the matrix is unchanged
    A = np.diag([1.0, 2.0, 3.0, 4.0])
    A[1, 0] = A[0, 1] = 0.5
    Aout, t = oracle.sy2sb(A, 1)
    assert np.all(t == 0.0)
    np.testing.assert_array_equal(np.tril(Aout), np.tril(A))


def test_sy2sb_trivial_sizes():
    for n, w in [(0, 1), (1, 1), (2, 1), (5, 4), (5, 7)]:
        A = workloads.sym_gaussian(n, 1) if n else np.zeros((0, 0))
        Aout, t = oracle.sy2sb(A, w)
        assert t.shape == (max(n - w, 0),)
        assert np.all(t == 0.0)
        np.testing.assert_array_equal(np.tril(Aout), np.tril(A))


def test_sy2sb_single_reflector_n_eq_w_plus_2():
    n, w = 7, 5
    A = workloads.sym_gaussian(n, 2)
    Aout, t = oracle.sy2sb(A, w)
    assert t[0] != 0.0 and t[1] == 0.0
    x = A[w:, 0]
    assert Aout[w, 0] == pytest.approx(-np.sign(x[0]) * np.linalg.norm(x), rel=4 * U64)


# --------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("n,w", [(8, 1), (37, 2), (64, 5), (96, 16), (130, 32), (50, 49)])
def test_sy2sb_invariants(n, w):
    A = workloads.sym_gaussian(n, n + w)
    Aout, tau = oracle.sy2sb(A, w)
    r = sym_report(A, Aout, tau, w)
    assert r["backward"] < 20 * n * U64
    assert r["orth"] < 20 * n * U64
    assert r["eig"] < 20 * n * U64
    # the band output by the oracle: zeros outside the band of the full matrix it keeps
    i, j = np.indices((n, n))
    assert np.all(Aout[(j - i > w)] == 0.0)
    # explicitly recomputed Q^T A Q has negligible entries outside the band
    Q = sym_form_q(Aout, tau, w)
    QAQ = Q.T @ A @ Q
    off = np.abs(QAQ[np.abs(i - j) > w])
    assert off.size == 0 or off.max() < 20 * n * U64 * np.linalg.norm(A)
    # trace and Frobenius norm preserved
    B = sym_band(Aout, w)
    assert abs(np.trace(B) - np.trace(A)) < 20 * n * U64 * np.linalg.norm(A)
    assert abs(np.linalg.norm(B) - np.linalg.norm(A)) < 20 * n * U64 * np.linalg.norm(A)


def test_sy2sb_w1_is_tridiagonal_and_matches_jacobi():
    n = 48
    A = workloads.sym_gaussian(n, 11)
    Aout, tau = oracle.sy2sb(A, 1)
    B = sym_band(Aout, 1)
    assert np.count_nonzero(np.triu(B, 2)) == 0
    lam_j = oracle.jacobi_eig(A)
    assert np.max(np.abs(np.linalg.eigvalsh(B) - lam_j)) < 50 * n * U64 * np.linalg.norm(A, 2)
    assert np.max(np.abs(oracle.jacobi_eig(B) - lam_j)) < 50 * n * U64 * np.linalg.norm(A, 2)


def test_sy2sb_known_spectrum():
    A, lam = workloads.sym_known_spectrum(64, 0, 1)
    Aout, tau = oracle.sy2sb(A, 8)
    lam_b = oracle.jacobi_eig(sym_band(Aout, 8))
    assert np.max(np.abs(lam_b - lam)) < 20 * 64 * U64  # Weyl: ||E||_2 <= backward error


def test_sy2sb_probe_backward_matches_dense():
    n, w = 90, 6
    A = workloads.sym_gaussian(n, 3)
    Aout, tau = oracle.sy2sb(A, w)
    est = sym_probe_backward(A, Aout, tau, w)
    assert est < 20 * n * U64


def test_sy2sb_thread_count_does_not_change_results():
    A = workloads.sym_gaussian(200, 4)
    oracle.set_threads(1)
    a1, t1 = oracle.sy2sb(A, 8)
    oracle.set_threads(4)
    a4, t4 = oracle.sy2sb(A, 8)
    oracle.set_threads(1)
    np.testing.assert_array_equal(a1, a4)
    np.testing.assert_array_equal(t1, t4)


def test_sy2sb_sample_prefix_is_prefix():
    """Stopping after k reflectors gives the first k reflectors of the full run."""
    A = workloads.sym_gaussian(60, 6)
    af, tf = oracle.sy2sb(A, 4)
    ap, tp = oracle.sy2sb(A, 4, ncols=10)
    np.testing.assert_array_equal(tp[:10], tf[:10])
    np.testing.assert_array_equal(ap[:, :10], af[:, :10])


@pytest.mark.parametrize("m,n,w", [(6, 6, 1), (20, 12, 1), (40, 40, 3), (70, 33, 8), (64, 64, 16), (9, 9, 8)])
def test_ge2gb_invariants(m, n, w):
    A = workloads.gen_gaussian(m, n, m * n + w)
    Aout, tq, tp = oracle.ge2gb(A, w)
    assert tq.shape == (n,) and tp.shape == (max(n - w, 0),)
    r = gen_report(A, Aout, tq, tp, w)
    assert r["backward"] < 20 * m * U64
    assert r["orth_u"] < 20 * m * U64
    assert r["orth_v"] < 20 * m * U64
    assert r["sv"] < 20 * m * U64
    U, V = gen_form_uv(Aout, tq, tp, w)
    UAV = U.T @ A @ V
    i, j = np.indices((m, n))
    off = np.abs(UAV[(j - i > w) | (j < i)])
    assert off.max() < 20 * m * U64 * np.linalg.norm(A)


def test_ge2gb_w1_bidiagonal_and_jacobi():
    A = workloads.gen_gaussian(40, 30, 12)
    Aout, tq, tp = oracle.ge2gb(A, 1)
    B = gen_band(Aout, 1)
    i, j = np.indices(B.shape)
    assert np.all(B[(j - i > 1) | (i > j)] == 0.0)
    np.testing.assert_allclose(oracle.jacobi_svd(B), oracle.jacobi_svd(A), rtol=0, atol=1e-13 * np.linalg.norm(A, 2))


def test_ge2gb_known_singular_values():
    A, sig = workloads.gen_known_singular(50, 40, 7)
    Aout, tq, tp = oracle.ge2gb(A, 4)
    assert np.max(np.abs(oracle.jacobi_svd(gen_band(Aout, 4)) - sig)) < 20 * 50 * U64


def test_ge2gb_rejects_wide():
    with pytest.raises(ValueError):
        oracle.ge2gb(np.zeros((3, 4)), 1)


# --------------------------------------------------------------------------- planted mistakes
def _sym_ok(A, Aout, tau, w, tol):
    r = sym_report(A, Aout, tau, w)
    return r["backward"] < tol and r["eig"] < tol


@pytest.mark.parametrize("mistake", ["tau_sign", "drop_reflector", "v_sign", "v_shift", "band_transpose"])
def test_pins_catch_planted_mistakes_sy2sb(mistake):
    n, w = 24, 3
    A = workloads.sym_gaussian(n, 21)
    Aout, tau = oracle.sy2sb(A, w)
    tol = 20 * n * U64
    assert _sym_ok(A, Aout, tau, w, tol)
    Am, tm = Aout.copy(), tau.copy()
    if mistake == "tau_sign":
        tm[3] = -tm[3]
    elif mistake == "drop_reflector":
        tm[5] = 0.0
    elif mistake == "v_sign":
        Am[w + 5:, 2] *= -1.0
    elif mistake == "v_shift":
        Am[w + 2:, 1] = np.roll(Am[w + 2:, 1], 1)
    elif mistake == "band_transpose":
        Am[w, 0], Am[w - 1, 0] = Am[w - 1, 0], Am[w, 0]
    assert not _sym_ok(A, Am, tm, w, tol)


@pytest.mark.parametrize("mistake", ["tauq_sign", "taup_drop", "vp_sign"])
def test_pins_catch_planted_mistakes_ge2gb(mistake):
    m, n, w = 20, 16, 2
    A = workloads.gen_gaussian(m, n, 22)
    Aout, tq, tp = oracle.ge2gb(A, w)
    tol = 20 * m * U64
    assert gen_report(A, Aout, tq, tp, w)["backward"] < tol
    Am, tqm, tpm = Aout.copy(), tq.copy(), tp.copy()
    if mistake == "tauq_sign":
        tqm[2] = -tqm[2]
    elif mistake == "taup_drop":
        tpm[1] = 0.0
    elif mistake == "vp_sign":
        Am[3, 3 + w + 1:] *= -1.0
    assert gen_report(A, Am, tqm, tpm, w)["backward"] > tol


# --------------------------------------------------------------------------- frozen outputs
def _read_golden(name):
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    out, key, rows = {}, None, []
    for line in open(path):
        if line.startswith("#"):
            if key:
                out[key] = np.array(rows)
            key, rows = line.split()[1], []
        else:
            rows.append([float(x) for x in line.split()])
    out[key] = np.array(rows)
    return out


def test_oracle_matches_its_frozen_outputs():
    g = _read_golden("sy2sb_n12_w3.txt")
    Aout, tau = oracle.sy2sb(g["A"], 3)
    np.testing.assert_allclose(np.tril(Aout), g["Aout_lower"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(tau, g["tau"].ravel(), rtol=0, atol=1e-15)
    h = _read_golden("ge2gb_m10_n8_w2.txt")
    Gout, tq, tp = oracle.ge2gb(h["A"], 2)
    np.testing.assert_allclose(Gout, h["Aout"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(tq, h["tauq"].ravel(), rtol=0, atol=1e-15)
    np.testing.assert_allclose(tp, h["taup"].ravel(), rtol=0, atol=1e-15)
    s = _read_golden("sb2st_n14_w3.txt")
    d, e = oracle.sb2st(s["A_lower"], 3)
    np.testing.assert_allclose(d, s["d"].ravel(), rtol=0, atol=1e-14)
    np.testing.assert_allclose(e, s["e"].ravel(), rtol=0, atol=1e-14)
    u = _read_golden("gb2bd_n14_w3.txt")
    d, e = oracle.gb2bd(u["A_upper"], 3)
    np.testing.assert_allclose(d, u["d"].ravel(), rtol=0, atol=1e-14)
    np.testing.assert_allclose(e, u["e"].ravel(), rtol=0, atol=1e-14)


# --------------------------------------------------------------------------- wide (m < n)
from checks import wide_band, wide_report  # noqa: E402


@pytest.mark.parametrize("m,n,w", [(20, 33, 2), (17, 40, 5), (8, 9, 1), (30, 64, 16), (5, 12, 8)])
def test_ge2gb_wide_invariants(m, n, w):
    """A = Q B P^T with B lower band: reconstruction through independently formed Q and P,
    orthogonality, band shape, and the singular values of A (LAPACK)."""
    A = workloads.gen_gaussian(m, n, 300 + m + n + w)
    Aout, tq, tp = oracle.ge2gb_wide(A, w)
    assert tq.shape == (max(m - w, 0),) and tp.shape == (m,)
    r = wide_report(A, Aout, tq, tp, w)
    tol = 20 * n * U64
    assert r["backward"] < tol and r["orth_q"] < tol and r["orth_p"] < tol and r["sv"] < tol, r


def test_ge2gb_wide_w1_is_lower_bidiagonal():
    m, n = 12, 20
    A = workloads.gen_gaussian(m, n, 9)
    Aout, tq, tp = oracle.ge2gb_wide(A, 1)
    B = wide_band(Aout, 1)
    i, j = np.indices(B.shape)
    assert np.all(B[(i - j < 0) | (i - j > 1)] == 0.0)
    np.testing.assert_allclose(np.sort(np.abs(np.linalg.svd(B, compute_uv=False))),
                               np.sort(oracle.jacobi_svd(A.T)), rtol=0, atol=1e-13 * np.linalg.norm(A))


def test_ge2gb_wide_hand_case_2x3_w1():
    # A = [[a, b, c], [d, e, f]]: the right reflector of row 0 gives beta_0 = -sign(a) ||(a, b, c)||
    A = np.array([[3.0, 4.0, 12.0], [1.0, -2.0, 5.0]])
    Aout, tq, tp = oracle.ge2gb_wide(A, 1)
    assert Aout[0, 0] == pytest.approx(-13.0, rel=4 * U64)
    assert tp[0] == pytest.approx(1.0 + 3.0 / 13.0, rel=4 * U64)
    # the band's singular values are those of A
    np.testing.assert_allclose(np.linalg.svd(wide_band(Aout, 1), compute_uv=False),
                               np.linalg.svd(A, compute_uv=False), rtol=1e-14)


def test_pins_catch_planted_mistakes_wide():
    m, n, w = 14, 25, 3
    A = workloads.gen_gaussian(m, n, 23)
    Aout, tq, tp = oracle.ge2gb_wide(A, w)
    tol = 20 * n * U64
    assert wide_report(A, Aout, tq, tp, w)["backward"] < tol
    for mistake in ("tauq_sign", "taup_drop", "v_right_sign"):
        Am, tqm, tpm = Aout.copy(), tq.copy(), tp.copy()
        if mistake == "tauq_sign":
            tqm[1] = -tqm[1]
        elif mistake == "taup_drop":
            tpm[2] = 0.0
        else:
            Am[3, 5:] *= -1.0
        assert wide_report(A, Am, tqm, tpm, w)["backward"] > tol, mistake


# --------------------------------------------------------------------------- equal bandwidth (Section 3.3)
from checks import bb_band, bb_report  # noqa: E402


@pytest.mark.parametrize("m,n,w", [(30, 24, 3), (24, 30, 3), (40, 40, 1), (50, 35, 8), (17, 60, 5), (33, 33, 32)])
def test_ge2bb_invariants(m, n, w):
    """A = U B V^T with |i-j| <= w on B: reconstruction through independently formed U and
    V, orthogonality, band shape, and the singular values of A (LAPACK)."""
    A = workloads.gen_gaussian(m, n, 400 + m + n + w)
    Aout, tq, tp = oracle.ge2bb(A, w)
    assert tq.shape == (max(min(n, m - w), 0),) and tp.shape == (max(min(m, n - w), 0),)
    r = bb_report(A, Aout, tq, tp, w)
    tol = 20 * max(m, n) * U64
    assert r["backward"] < tol and r["orth_u"] < tol and r["orth_v"] < tol and r["sv"] < tol, r


def test_ge2bb_w1_is_tridiagonal_with_the_singular_values_of_A():
    m, n = 25, 18
    A = workloads.gen_gaussian(m, n, 11)
    Aout, tq, tp = oracle.ge2bb(A, 1)
    B = bb_band(Aout, 1)
    i, j = np.indices(B.shape)
    assert np.all(B[np.abs(i - j) > 1] == 0.0)
    np.testing.assert_allclose(np.sort(np.linalg.svd(B, compute_uv=False)), np.sort(oracle.jacobi_svd(A)),
                               rtol=0, atol=1e-13 * np.linalg.norm(A))


def test_ge2bb_hand_case_4x4_w2():
    # the first left reflector acts on rows 2..3 of column 0: beta = -sign(a20) ||(a20, a30)||
    A = np.array([[1.0, 2.0, 3.0, 4.0], [5.0, 6.0, 7.0, 8.0], [3.0, 1.0, 2.0, 5.0], [4.0, 9.0, 1.0, 2.0]])
    Aout, tq, tp = oracle.ge2bb(A, 2)
    assert Aout[2, 0] == pytest.approx(-5.0, rel=4 * U64)
    assert tq[0] == pytest.approx(1.0 + 3.0 / 5.0, rel=4 * U64)
    # column 0 above row 2 is untouched by it: the band keeps a00 and a10
    assert Aout[0, 0] == 1.0 and Aout[1, 0] == 5.0


def test_pins_catch_planted_mistakes_ge2bb():
    m, n, w = 30, 26, 4
    A = workloads.gen_gaussian(m, n, 29)
    Aout, tq, tp = oracle.ge2bb(A, w)
    tol = 20 * m * U64
    assert bb_report(A, Aout, tq, tp, w)["backward"] < tol
    for mistake in ("tauq_sign", "taup_drop", "vq_shift"):
        Am, tqm, tpm = Aout.copy(), tq.copy(), tp.copy()
        if mistake == "tauq_sign":
            tqm[2] = -tqm[2]
        elif mistake == "taup_drop":
            tpm[3] = 0.0
        else:
            Am[w + 3:, 1] = np.roll(Am[w + 3:, 1], 1)
        assert bb_report(A, Am, tqm, tpm, w)["backward"] > tol, mistake
