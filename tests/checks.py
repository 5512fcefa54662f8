"""Independent NumPy checks of packed band-reduction outputs (test helpers).

These routines read the packed layout (band + reflectors + tau) written by either the
oracle or the library, rebuild the orthogonal factors explicitly from the reflectors
and measure what the mathematics fixes: A = Q B Q^T (Section 2.1) or A = U B V^T
(Section 3.1), orthogonality, band shape and spectra.  They share no code with the
oracle or with the CUDA path.
"""
from __future__ import annotations

import numpy as np

U64 = np.finfo(np.float64).eps / 2  # unit roundoff 2^-53


def sym_band(Aout: np.ndarray, w: int) -> np.ndarray:
    """Dense symmetric band matrix from the lower band 0 <= i-j <= w of Aout."""
    n = Aout.shape[0]
    i, j = np.indices((n, n))
    L = np.where((i - j >= 0) & (i - j <= w), Aout, 0.0)
    return L + np.tril(L, -1).T


def sym_form_q(Aout: np.ndarray, tau: np.ndarray, w: int) -> np.ndarray:
    """Q = H_0 H_1 ... with H_c = I - tau_c v_c v_c^T acting on rows c+w..n-1,
    v_c = [1; Aout(c+w+1:n, c)]."""
    n = Aout.shape[0]
    Q = np.eye(n)
    for c in range(len(tau)):
        t = tau[c]
        if t == 0.0:
            continue
        r0 = c + w
        v = np.concatenate(([1.0], Aout[r0 + 1:, c]))
        Q[:, r0:] -= t * np.outer(Q[:, r0:] @ v, v)
    return Q


def sym_apply_qt(Aout: np.ndarray, tau: np.ndarray, w: int, X: np.ndarray) -> np.ndarray:
    """Q^T X through the reflectors, without forming Q."""
    X = np.array(X, dtype=np.float64, copy=True)
    for c in range(len(tau)):
        t = tau[c]
        if t == 0.0:
            continue
        r0 = c + w
        v = np.concatenate(([1.0], Aout[r0 + 1:, c]))
        X[r0:] -= t * np.outer(v, v @ X[r0:])
    return X


def sym_apply_q(Aout: np.ndarray, tau: np.ndarray, w: int, X: np.ndarray) -> np.ndarray:
    """Q X through the reflectors, without forming Q."""
    X = np.array(X, dtype=np.float64, copy=True)
    for c in reversed(range(len(tau))):
        t = tau[c]
        if t == 0.0:
            continue
        r0 = c + w
        v = np.concatenate(([1.0], Aout[r0 + 1:, c]))
        X[r0:] -= t * np.outer(v, v @ X[r0:])
    return X


def gen_band(Aout: np.ndarray, w: int) -> np.ndarray:
    """Upper triangular band 0 <= j-i <= w of an m x n packed output."""
    m, n = Aout.shape
    i, j = np.indices((m, n))
    return np.where((j - i >= 0) & (j - i <= w), Aout, 0.0)


def gen_form_uv(Aout: np.ndarray, tauq: np.ndarray, taup: np.ndarray, w: int):
    """U = Hq_0 Hq_1 ... (left reflectors, v below the diagonal) and V = Hp_0 Hp_1 ...
    (right reflectors acting on columns c+w.., v in row c right of column c+w)."""
    m, n = Aout.shape
    U = np.eye(m)
    for c in range(len(tauq)):
        t = tauq[c]
        if t == 0.0:
            continue
        v = np.concatenate(([1.0], Aout[c + 1:, c]))
        U[:, c:] -= t * np.outer(U[:, c:] @ v, v)
    V = np.eye(n)
    for c in range(len(taup)):
        t = taup[c]
        if t == 0.0:
            continue
        r0 = c + w
        v = np.concatenate(([1.0], Aout[c, r0 + 1:]))
        V[:, r0:] -= t * np.outer(V[:, r0:] @ v, v)
    return U, V


def sym_report(A: np.ndarray, Aout: np.ndarray, tau: np.ndarray, w: int) -> dict:
    """Backward error, orthogonality and eigenvalue error for a small sy2sb result."""
    A = np.tril(A) + np.tril(A, -1).T
    B = sym_band(Aout, w)
    Q = sym_form_q(Aout, tau, w)
    n = A.shape[0]
    fa = np.linalg.norm(A)
    lam_a = np.linalg.eigvalsh(A)
    lam_b = np.linalg.eigvalsh(B)
    return {
        "backward": np.linalg.norm(A - Q @ B @ Q.T) / fa if fa else 0.0,
        "orth": np.linalg.norm(Q.T @ Q - np.eye(n)),
        "eig": np.max(np.abs(lam_a - lam_b)) / max(np.max(np.abs(lam_a)), 1e-300) if n else 0.0,
    }


def gen_report(A: np.ndarray, Aout: np.ndarray, tauq, taup, w: int) -> dict:
    B = gen_band(Aout, w)
    U, V = gen_form_uv(Aout, tauq, taup, w)
    m, n = A.shape
    fa = np.linalg.norm(A)
    s_a = np.linalg.svd(A, compute_uv=False)
    s_b = np.linalg.svd(B, compute_uv=False)
    return {
        "backward": np.linalg.norm(A - U @ B @ V.T) / fa if fa else 0.0,
        "orth_u": np.linalg.norm(U.T @ U - np.eye(m)),
        "orth_v": np.linalg.norm(V.T @ V - np.eye(n)),
        "sv": np.max(np.abs(s_a - s_b)) / max(s_a[0], 1e-300) if n else 0.0,
    }


def sym_probe_backward(A: np.ndarray, Aout: np.ndarray, tau: np.ndarray, w: int, probes: int = 8,
                       seed: int = 5) -> float:
    """||(A - Q B Q^T) X||_F / ||A X||_F for Gaussian probes X (n x probes): a backward
    error estimate that needs neither Q nor B formed densely."""
    n = A.shape[0]
    X = np.random.Generator(np.random.PCG64(seed)).standard_normal((n, probes))
    Al = np.tril(A)
    AX = Al @ X + np.tril(A, -1).T @ X
    Y = sym_apply_qt(Aout, tau, w, X)
    # B Y with the band read from the lower band of Aout.
    BY = np.zeros_like(Y)
    for d in range(0, w + 1):
        diag = np.diagonal(Aout, -d)
        if d == 0:
            BY += diag[:, None] * Y
        else:
            BY[d:] += diag[:, None] * Y[:-d]
            BY[:-d] += diag[:, None] * Y[d:]
    QBY = sym_apply_q(Aout, tau, w, BY)
    return float(np.linalg.norm(AX - QBY) / np.linalg.norm(AX))


def gen_probe_backward(A: np.ndarray, Aout: np.ndarray, tauq: np.ndarray, taup: np.ndarray, w: int,
                       probes: int = 8, seed: int = 5) -> float:
    """||(A - U B V^T) X||_F / ||A X||_F for Gaussian probes X (n x probes), with U and V
    applied through the reflectors (ge2gb layout) and B read from the upper band."""
    m, n = A.shape
    X = np.random.Generator(np.random.PCG64(seed)).standard_normal((n, probes))
    AX = A @ X
    # Y = V^T X: V = Hp_0 Hp_1 ..., so V^T X applies Hp_0 first
    Y = np.array(X, copy=True)
    for c in range(len(taup)):
        t = taup[c]
        if t == 0.0:
            continue
        r0 = c + w
        v = np.concatenate(([1.0], Aout[c, r0 + 1:]))
        Y[r0:] -= t * np.outer(v, v @ Y[r0:])
    BY = np.zeros((m, probes))
    for d in range(0, w + 1):
        diag = np.diagonal(Aout, d)  # B(i, i+d)
        k = len(diag)
        BY[:k] += diag[:, None] * Y[d:d + k]
    # U BY: U = Hq_0 Hq_1 ..., applied last-first
    Z = BY
    for c in reversed(range(len(tauq))):
        t = tauq[c]
        if t == 0.0:
            continue
        v = np.concatenate(([1.0], Aout[c + 1:, c]))
        Z[c:] -= t * np.outer(v, v @ Z[c:])
    return float(np.linalg.norm(AX - Z) / np.linalg.norm(AX))


def wide_band(Aout: np.ndarray, w: int) -> np.ndarray:
    """Lower band 0 <= i-j <= w of an m x n (m < n) packed output."""
    m, n = Aout.shape
    i, j = np.indices((m, n))
    return np.where((i - j >= 0) & (i - j <= w), Aout, 0.0)


def wide_form_qp(Aout: np.ndarray, tauq: np.ndarray, taup: np.ndarray, w: int):
    """Q = H_0 H_1 ... (left reflectors on rows c+w.., v in column c below the band) and
    P = G_0 G_1 ... (right reflectors on columns c.., v in row c right of the diagonal)."""
    m, n = Aout.shape
    Q = np.eye(m)
    for c in range(len(tauq)):
        t = tauq[c]
        if t == 0.0:
            continue
        r0 = c + w
        v = np.concatenate(([1.0], Aout[r0 + 1:, c]))
        Q[:, r0:] -= t * np.outer(Q[:, r0:] @ v, v)
    P = np.eye(n)
    for c in range(len(taup)):
        t = taup[c]
        if t == 0.0:
            continue
        v = np.concatenate(([1.0], Aout[c, c + 1:]))
        P[:, c:] -= t * np.outer(P[:, c:] @ v, v)
    return Q, P


def wide_report(A: np.ndarray, Aout: np.ndarray, tauq, taup, w: int) -> dict:
    """Backward error, orthogonality and singular-value error of a wide (m < n) result."""
    B = wide_band(Aout, w)
    Q, P = wide_form_qp(Aout, tauq, taup, w)
    m, n = A.shape
    fa = np.linalg.norm(A)
    s_a = np.linalg.svd(A, compute_uv=False)
    s_b = np.linalg.svd(B, compute_uv=False)
    return {
        "backward": np.linalg.norm(A - Q @ B @ P.T) / fa if fa else 0.0,
        "orth_q": np.linalg.norm(Q.T @ Q - np.eye(m)),
        "orth_p": np.linalg.norm(P.T @ P - np.eye(n)),
        "sv": np.max(np.abs(s_a - s_b)) / max(s_a[0], 1e-300) if m else 0.0,
    }


def bb_band(Aout: np.ndarray, w: int) -> np.ndarray:
    """Band |i-j| <= w of an m x n packed equal-bandwidth output."""
    m, n = Aout.shape
    i, j = np.indices((m, n))
    return np.where(np.abs(i - j) <= w, Aout, 0.0)


def bb_form_uv(Aout: np.ndarray, tauq: np.ndarray, taup: np.ndarray, w: int):
    """U = Hq_0 Hq_1 ... (left reflector c on rows c+w.., v in column c below the band) and
    V = Hp_0 Hp_1 ... (right reflector c on columns c+w.., v in row c right of the band)."""
    m, n = Aout.shape
    U = np.eye(m)
    for c in range(len(tauq)):
        t = tauq[c]
        if t == 0.0:
            continue
        r0 = c + w
        v = np.concatenate(([1.0], Aout[r0 + 1:, c]))
        U[:, r0:] -= t * np.outer(U[:, r0:] @ v, v)
    V = np.eye(n)
    for c in range(len(taup)):
        t = taup[c]
        if t == 0.0:
            continue
        r0 = c + w
        v = np.concatenate(([1.0], Aout[c, r0 + 1:]))
        V[:, r0:] -= t * np.outer(V[:, r0:] @ v, v)
    return U, V


def bb_report(A: np.ndarray, Aout: np.ndarray, tauq, taup, w: int) -> dict:
    B = bb_band(Aout, w)
    U, V = bb_form_uv(Aout, tauq, taup, w)
    m, n = A.shape
    fa = np.linalg.norm(A)
    s_a = np.linalg.svd(A, compute_uv=False)
    s_b = np.linalg.svd(B, compute_uv=False)
    return {
        "backward": np.linalg.norm(A - U @ B @ V.T) / fa if fa else 0.0,
        "orth_u": np.linalg.norm(U.T @ U - np.eye(m)),
        "orth_v": np.linalg.norm(V.T @ V - np.eye(n)),
        "sv": np.max(np.abs(s_a - s_b)) / max(s_a[0], 1e-300) if min(m, n) else 0.0,
    }
