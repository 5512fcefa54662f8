"""The algebra of the grouped panel step (panel_qr4_kernel), on the CPU.

One grid-wide reduction gives, for a block of up to four columns i .. i+3, the sums of
every panel column against the block columns' tails (rows below the block) and the
block's explicit rows.  The kernel derives the block's Householder reflectors (Section
2.1's panel QR, LAPACK sign convention), their compact-WY factor and every other column's
update from those numbers alone.  Here the same derivation is restated in FP64 NumPy and
checked against column-by-column Householder QR: entrywise on well-conditioned panels,
and backward stable (Q R = P, Q orthogonal, W = -Y T) on panels with dependent columns,
where the reflectors themselves are set by rounding.  A planted sign error must fail.
"""
import numpy as np
import pytest


def larfg(alpha, xn2):
    if xn2 == 0.0:
        return alpha, 0.0, 1.0
    h = np.sqrt(alpha * alpha + xn2)
    beta = -h if alpha >= 0 else h
    return beta, 1.0 + abs(alpha) / h, (1.0 if alpha >= 0 else -1.0) / (abs(alpha) + h)


def householder_qr(P):
    """Column-by-column Householder QR: packed R and V, tau, and W = -Y T."""
    P = P.copy()
    J, bk = P.shape
    tau = np.zeros(bk)
    for c in range(bk):
        x2 = P[c + 1:, c]
        beta, t, scal = larfg(P[c, c], float(x2 @ x2)) if J - c > 1 else (P[c, c], 0.0, 1.0)
        v = np.concatenate([[1.0], x2 * scal])
        tau[c] = t
        if t != 0.0:
            P[c:, c + 1:] -= t * np.outer(v, v @ P[c:, c + 1:])
            P[c + 1:, c] = v[1:]
            P[c, c] = beta
    return P, tau, -unit_y(P) @ t_factor(unit_y(P), tau)


def unit_y(P):
    J, bk = P.shape
    Y = np.tril(P, -1)
    Y[np.arange(bk), np.arange(bk)] = 1.0
    return Y


def t_factor(Y, tau):
    bk = Y.shape[1]
    T = np.zeros((bk, bk))
    for c in range(bk):
        T[c, c] = tau[c]
        T[:c, c] = -tau[c] * T[:c, :c] @ (Y[:, :c].T @ Y[:, c])
    return T


def grouped_qr(P0, group=4, guard=0.125, sign=1.0):
    """The grouped step: per block, only the tail sums G, the explicit rows and the block's
    own quantities.  `sign` = -1 plants a mistake (the wrong sign of the transform)."""
    P = P0.copy()
    J, bk = P.shape
    tau = np.zeros(bk)
    W = np.zeros((J, bk))
    i = 0
    while i < bk:
        mt = max(1, min(group, bk - i, J - i - 1))
        lo = i + mt
        top = P[i:lo, :].copy()
        tails = P[lo:, i:lo].copy()
        G = tails.T @ P[lo:, :]
        Gb = G[:, i:lo]
        tb = [top[:, i + q].copy() for q in range(mt)]
        lam = np.zeros((mt, mt))
        V, C, TB, beta_k = [], [], [], []
        for k in range(mt):
            e = lam[k] + np.eye(mt)[k]
            n2t = float(e @ Gb @ e)
            if k > 0 and not n2t > guard * float(np.sum(e * e * np.diag(Gb))):
                break
            xn2 = n2t + float(tb[k][k + 1:] @ tb[k][k + 1:])
            beta, t, scal = larfg(tb[k][k], xn2) if J - (i + k) > 1 else (tb[k][k], 0.0, 1.0)
            v = np.zeros(mt)
            v[k + 1:] = scal * tb[k][k + 1:]
            V.append(v)
            C.append(scal * e)
            TB.append(tb[k].copy())
            beta_k.append(beta)
            tau[i + k] = t
            for q in range(k + 1, mt):
                eq = lam[q] + np.eye(mt)[q]
                z = sign * t * (tb[q][k] + v[k + 1:] @ tb[q][k + 1:] + C[k] @ Gb @ eq)
                tb[q][k] -= z
                tb[q][k + 1:] -= z * v[k + 1:]
                lam[q] -= z * C[k]
        meff = len(V)
        # compact-WY factor of the block from the in-block products of its reflectors
        Tb = np.zeros((meff, meff))
        gb = np.zeros((meff, meff))
        for k in range(meff):
            for q in range(k):
                gb[q, k] = V[q][k] + V[q][k + 1:] @ V[k][k + 1:] + C[q] @ Gb @ C[k]
            Tb[k, k] = tau[i + k]
            Tb[:k, k] = -tau[i + k] * Tb[:k, :k] @ gb[:k, k]
        # every column: w = V^T c, z = T^T w, c -= V z (tail: coefficients of the block tails)
        wdots = np.zeros((meff, bk))
        for c in range(bk):
            if i <= c < i + meff:
                continue
            w = np.array([top[k, c] + V[k][k + 1:] @ top[k + 1:, c] + C[k] @ G[:, c] for k in range(meff)])
            wdots[:, c] = w
            if c < i:
                continue
            z = Tb.T @ w
            for s in range(mt):
                P[i + s, c] = top[s, c] - sum(z[k] * (1.0 if k == s else V[k][s]) for k in range(min(meff, s + 1)))
            P[lo:, c] += tails @ (-sum(z[k] * C[k] for k in range(meff)))
        for k in range(meff):
            P[lo:, i + k] = tails @ C[k]
            P[i:i + k, i + k] = TB[k][:k]
            P[i + k, i + k] = beta_k[k]
            P[i + k + 1:lo, i + k] = V[k][k + 1:]
        for k in range(meff):  # W column recurrence with g = Y(:, 0:i+k)^T y_{i+k}
            col = i + k
            g = np.concatenate([wdots[k, :i], gb[:k, k]])
            y = np.zeros(J)
            y[col] = 1.0
            y[col + 1:] = P[col + 1:, col]
            W[:, col] = -tau[col] * (y + W[:, :col] @ g)
        i += meff
    return P, tau, W


def backward(P0, P, tau, W):
    J, bk = P0.shape
    Y = unit_y(P)
    Q = np.eye(J)
    for c in reversed(range(bk)):
        Q -= tau[c] * np.outer(Y[:, c], Y[:, c] @ Q)
    res = np.linalg.norm(Q[:, :bk] @ np.triu(P[:bk, :]) - P0) / np.linalg.norm(P0)
    orth = np.linalg.norm(Q.T @ Q - np.eye(J))
    werr = np.linalg.norm(W + Y @ t_factor(Y, tau)) / max(1.0, np.linalg.norm(Y @ t_factor(Y, tau)))
    return res, orth, werr


def panels(seed, kind):
    rng = np.random.default_rng(seed)
    J = int(rng.integers(8, 160))
    bk = int(rng.integers(1, min(J, 33)))
    P0 = rng.standard_normal((J, bk))
    if kind == "graded":
        P0 *= 10.0 ** rng.uniform(-8, 8, size=(1, bk))
    if kind == "zero_tails":
        P0[bk:, : bk // 2] = 0.0
    if kind == "dependent":
        P0[:, 1::2] = P0[:, 0::2][:, : P0[:, 1::2].shape[1]]
    return P0


@pytest.mark.parametrize("group", [2, 3, 4])
@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("kind", ["gaussian", "graded", "zero_tails"])
def test_grouped_step_matches_householder_qr(group, seed, kind):
    P0 = panels(seed, kind)
    Pr, tr, Wr = householder_qr(P0)
    P, t, W = grouped_qr(P0, group)
    scale = np.abs(P0).max(axis=0, keepdims=True)
    # R relative to its column's scale; reflector entries (at most 1 in magnitude) absolutely
    assert np.max(np.abs(np.triu(P - Pr)) / scale) < 1e-10
    assert np.max(np.abs(np.tril(P - Pr, -1))) < 1e-10
    assert np.max(np.abs(t - tr)) < 1e-12
    assert np.max(np.abs(W - Wr)) < 1e-10 * max(1.0, np.abs(Wr).max())


@pytest.mark.parametrize("group", [2, 4])
@pytest.mark.parametrize("seed", range(6))
def test_grouped_step_is_backward_stable_on_dependent_columns(group, seed):
    P0 = panels(seed, "dependent")
    res, orth, werr = backward(P0, *grouped_qr(P0, group))
    assert res < 1e-14 and orth < 1e-13 and werr < 1e-13, (res, orth, werr)


def test_a_planted_sign_error_is_caught():
    P0 = panels(3, "gaussian")
    if P0.shape[1] < 3:
        P0 = np.random.default_rng(5).standard_normal((60, 8))
    res, _, _ = backward(P0, *grouped_qr(P0, 4, sign=-1.0))
    assert res > 1e-3
