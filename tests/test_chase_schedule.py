"""The concurrency protocol of the two bulge-chasing kernels, checked on the CPU.

Both second-stage kernels run every sweep of the chase at once, one CTA per sweep, and
each sweep waits on a progress counter of the sweep before.  Correctness rests on a rule:
a sweep's step t may start once the sweep before has published a given count, and every
value a step reads is then final.  This file models each of the four chase kernels (the
shared-memory and the L2 kernel of each second stage) at the granularity at which it
touches the band store, in NumPy:

* what a step reads, it reads at its start (the blocks the shared-memory kernels stage
  after their wait), or, in the L2 kernels, at the moment one warp updates one vector;
* what it writes, it writes at the phase where the kernel writes it (the early column or
  row of the next step, the write-back, the diagonal block), and its counter goes up last;
* what it carries between steps stays private to the sweep.

Sweeps then advance one phase at a time in random order, each step starting only when the
kernel's wait would let it, and the band must come out bit for bit as the one-sweep-at-a-
time run gives it.  A lag one step shorter than the kernel's must show a difference for
some interleaving (the check can see a race), and the sequential model must agree with the
C oracle (it is the algorithm the oracle defines).
"""
import random

import numpy as np
import pytest

import oracle


def larfg(x):
    """Householder reflector of x, larfg convention: (v with v[0] = 1, tau, beta)."""
    alpha = x[0]
    xn = np.linalg.norm(x[1:])
    if xn == 0.0:
        return np.concatenate([[1.0], np.zeros(len(x) - 1)]), 0.0, alpha
    h = np.hypot(alpha, xn)
    beta = -h if alpha >= 0.0 else h
    return np.concatenate([[1.0], x[1:] / (alpha - beta)]), (beta - alpha) / beta, beta


# --------------------------------------------------------------------------- symmetric
def sym_sweep(M, n, w, c):
    """Sweep c of the symmetric chase (M: dense symmetric, updated in place).  Yields
    ('start', t) when step t would wait, then one item per write phase, ('done', t) when its
    counter goes up.  Step t stages its diagonal block and the rows below at its start; the
    column it annihilates and the bulge come from the step before (carried)."""
    col, s, t = c, c + 1, 0
    carry = None  # the rows below of the step before: rows [s, end) x columns [col, s)
    while True:
        end = min(s + w, n)
        ln = end - s
        if ln < 2:
            return
        yield ("start", t)
        nl = min(end + w, n) - end
        D = M[s:end, s:end].copy()
        L = M[end:end + nl, s:end].copy()
        if t == 0:
            x = M[s:end, col].copy()
            v, tau, beta = larfg(x)
            M[s:end, col] = 0.0
            M[s, col] = beta
            M[col, s:end] = M[s:end, col]
            yield ("column", t)
            B = np.zeros((ln, 0))
        else:
            v, tau = carry["v"], carry["tau"]
            B = carry["L"][:, 1:]  # rows [s, end), bulge columns (col, s)
        # the step's arithmetic on private copies
        if tau != 0.0:
            B = B - tau * np.outer(v, v @ B)
            L = L - tau * np.outer(L @ v, v)
            p = tau * (D @ v)
            K = p - 0.5 * tau * (p @ v) * v
            D = D - np.outer(v, K) - np.outer(K, v)
        nxt = None
        if nl >= 2:
            v2, tau2, beta2 = larfg(L[:, 0].copy())
            nxt = {"v": v2, "tau": tau2, "beta": beta2}
        # write-back phase: the bulge (final), the next step's column (beta, 0, ..)
        if B.shape[1]:
            M[s:end, col + 1:s] = B
            M[col + 1:s, s:end] = B.T
        if nxt is not None:
            M[end:end + nl, s] = 0.0
            M[end, s] = nxt["beta"]
            M[s, end:end + nl] = M[end:end + nl, s]
        elif nl == 1:
            M[end:end + nl, s:end] = L
            M[s:end, end:end + nl] = L.T
        yield ("writeback", t)
        M[s:end, s:end] = D
        yield ("diagonal", t)
        yield ("done", t)
        carry = None if nxt is None else {"v": nxt["v"], "tau": nxt["tau"], "L": L}
        col, s, t = s, s + w, t + 1


# --------------------------------------------------------------------------- bidiagonal
def bd_sweep(M, n, w, c):
    """Sweep c of the upper band -> bidiagonal chase (M: dense, in place), as the tile
    kernel runs it: the tile (rows (r, a + w) x columns [a, a + 2w), the entries of the
    step) is staged at the step's start and written back at its end, with the next step's
    right-reflector row already (beta, 0, ..)."""
    r, a, t = c, c + 1, 0
    saved = None
    while True:
        end = min(a + w, n)
        ln = end - a
        if ln < 2:
            return
        yield ("start", t)
        rend, cend = min(a + w, n), min(a + 2 * w, n)
        T = M[r + 1:rend, a:cend].copy()
        ia = a - r - 1
        if t == 0:
            v, tau, beta = larfg(M[r, a:end].copy())
            M[r, a:end] = 0.0
            M[r, a] = beta
            yield ("row", t)
        else:
            v, tau = saved
        if tau != 0.0:
            Y = T[:, 0:ln]
            T[:, 0:ln] = Y - tau * np.outer(Y @ v, v)
        vl, tl, bl = larfg(T[ia:ia + ln, 0].copy())
        T[ia:ia + ln, 0] = 0.0
        T[ia, 0] = bl
        if tl != 0.0:
            Z = T[ia:ia + ln, 1:]
            T[ia:ia + ln, 1:] = Z - tl * np.outer(vl, vl @ Z)
        nl = min(a + 2 * w, n) - (a + w)
        saved = None
        if nl >= 2:
            v2, tau2, beta2 = larfg(T[ia, w:w + nl].copy())
            T[ia, w:w + nl] = 0.0
            T[ia, w] = beta2
            saved = (v2, tau2)
        # write back the step's entries (the tile's top-right corner is not the step's)
        rows = np.arange(r + 1, rend)[:, None]
        cols = np.arange(a, cend)[None, :]
        mine = (cols < end) | ((rows >= a) & (rows < end))
        blk = M[r + 1:rend, a:cend]
        blk[mine] = T[mine]
        yield ("writeback", t)
        yield ("done", t)
        r, a, t = a, a + w, t + 1


# --------------------------------------------------------------------------- L2 kernels
def sym_sweep_l2(M, n, w, c):
    """Sweep c of the symmetric chase as the L2 kernel (w <= 128) runs it: every vector
    (a bulge column, a row below, a row of the diagonal block) is read and written back at
    its own moment, one warp at a time."""
    col, s, t = c, c + 1, 0
    while True:
        end = min(s + w, n)
        ln = end - s
        if ln < 2:
            return
        yield ("start", t)
        v, tau, beta = larfg(M[s:end, col].copy())
        M[s:end, col] = 0.0
        M[s, col] = beta
        M[col, s:end] = M[s:end, col]
        yield ("column", t)
        nl = min(end + w, n) - end
        if tau != 0.0:
            for j in range(col + 1, s):  # bulge columns: left application
                y = M[s:end, j].copy()
                M[s:end, j] = y - tau * (v @ y) * v
                M[j, s:end] = M[s:end, j]
                yield ("vector", t)
            for i in range(end, end + nl):  # rows below: right application
                y = M[i, s:end].copy()
                M[i, s:end] = y - tau * (y @ v) * v
                M[s:end, i] = M[i, s:end]
                yield ("vector", t)
            p = tau * (M[s:end, s:end] @ v)  # the diagonal block's matvec (reads)
            yield ("matvec", t)
            K = p - 0.5 * tau * (p @ v) * v
            D = M[s:end, s:end] - np.outer(v, K) - np.outer(K, v)
            M[s:end, s:end] = D
            yield ("diagonal", t)
        yield ("done", t)
        col, s, t = s, s + w, t + 1


def bd_sweep_l2(M, n, w, c):
    """Sweep c of the bidiagonal chase as the L2 kernel runs it: each row (right
    reflector) and column (left reflector) updated at its own moment."""
    r, a, t = c, c + 1, 0
    while True:
        end = min(a + w, n)
        ln = end - a
        if ln < 2:
            return
        yield ("start", t)
        v, tau, beta = larfg(M[r, a:end].copy())
        M[r, a:end] = 0.0
        M[r, a] = beta
        yield ("row", t)
        if tau != 0.0:
            for i in range(r + 1, min(a + w, n)):
                y = M[i, a:end].copy()
                M[i, a:end] = y - tau * (y @ v) * v
                yield ("vector", t)
        v, tau, beta = larfg(M[a:end, a].copy())
        M[a:end, a] = 0.0
        M[a, a] = beta
        yield ("column", t)
        if tau != 0.0:
            for j in range(a + 1, min(a + 2 * w, n)):
                y = M[a:end, j].copy()
                M[a:end, j] = y - tau * (v @ y) * v
                yield ("vector", t)
        yield ("done", t)
        r, a, t = a, a + w, t + 1


# --------------------------------------------------------------------------- scheduler
def run(M0, w, sweep, lag, seed=None):
    """All sweeps of the chase.  seed None: one sweep after the other.  Otherwise random
    interleaving of phases; sweep c's step t starts only when sweep c - 1 has counted t +
    lag (or has finished)."""
    M = M0.copy()
    n = M.shape[0]
    gens = {c: sweep(M, n, w, c) for c in range(max(n - 1, 0))}
    if seed is None:
        for c in sorted(gens):
            for _ in gens[c]:
                pass
        return M
    rng = random.Random(seed)
    prog = {c: 0 for c in gens}
    waiting = {c: True for c in gens}  # about to start a step
    done = set()
    pend = {c: None for c in gens}
    while len(done) < len(gens):
        runnable = []
        for c in gens:
            if c in done:
                continue
            if waiting[c] and c > 0 and (c - 1) not in done and prog[c - 1] < prog[c] + lag:
                continue
            runnable.append(c)
        c = rng.choice(runnable)
        try:
            kind, t = next(gens[c])
        except StopIteration:
            done.add(c)
            continue
        if kind == "start":
            waiting[c] = False
        elif kind == "done":
            prog[c] = t + 1
            waiting[c] = True
    return M


def sym_band(n, w, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    A = (G + G.T) / 2
    i, j = np.indices((n, n))
    A[np.abs(i - j) > w] = 0.0
    return A


def upper_band(n, w, seed):
    rng = np.random.default_rng(seed)
    A = np.triu(rng.standard_normal((n, n)))
    return np.triu(A) - np.triu(A, w + 1)


@pytest.mark.parametrize("n,w", [(30, 3), (41, 4), (37, 6), (24, 2)])
def test_symmetric_chase_two_step_lag_is_exact(n, w):
    A = sym_band(n, w, n + w)
    S = run(A, w, sym_sweep, 2)
    d, e = oracle.sb2st(np.tril(A), w)  # the model is the oracle's algorithm
    assert np.max(np.abs(np.diag(S) - d)) <= 1e-12 and np.max(np.abs(np.diag(S, -1) - e)) <= 1e-12
    for seed in range(12):
        assert np.array_equal(run(A, w, sym_sweep, 2, seed), S), seed


@pytest.mark.parametrize("n,w", [(30, 3), (41, 4), (37, 6), (24, 2)])
def test_bidiagonal_chase_two_step_lag_is_exact(n, w):
    A = upper_band(n, w, n + w)
    S = run(A, w, bd_sweep, 2)
    d, e = oracle.gb2bd(A, w)
    assert np.max(np.abs(np.diag(S) - d)) <= 1e-12 and np.max(np.abs(np.diag(S, 1) - e)) <= 1e-12
    for seed in range(12):
        assert np.array_equal(run(A, w, bd_sweep, 2, seed), S), seed


@pytest.mark.parametrize("sweep,band", [(sym_sweep, sym_band), (bd_sweep, upper_band)])
def test_a_shorter_lag_shows_a_race(sweep, band):
    """With sweeps only one step apart, some interleaving reads a value before the sweep
    ahead has finished with it, and the band differs: the checks above can see a race."""
    n, w = 30, 3
    A = band(n, w, 5)
    S = run(A, w, sweep, 2)
    assert any(not np.array_equal(run(A, w, sweep, 1, seed), S) for seed in range(12))


@pytest.mark.parametrize("sweep,band,ref", [(sym_sweep_l2, sym_band, "sb2st"), (bd_sweep_l2, upper_band, "gb2bd")])
def test_l2_kernels_three_step_lag_is_exact(sweep, band, ref):
    """The L2 kernels (w up to 128) wait for step t + 2 of the sweep before; each vector's
    update touches the band store at its own moment."""
    for n, w in [(30, 3), (37, 5)]:
        A = band(n, w, 3 * n + w)
        S = run(A, w, sweep, 3)
        if ref == "sb2st":
            d, e = oracle.sb2st(np.tril(A), w)
            off = np.diag(S, -1)
        else:
            d, e = oracle.gb2bd(A, w)
            off = np.diag(S, 1)
        assert np.max(np.abs(np.diag(S) - d)) <= 1e-12 and np.max(np.abs(off - e)) <= 1e-12
        for seed in range(12):
            assert np.array_equal(run(A, w, sweep, 3, seed), S), (n, w, seed)
        # one step less, and the single shared entry can be read too early
        assert any(not np.array_equal(run(A, w, sweep, 2, seed), S) for seed in range(24))
