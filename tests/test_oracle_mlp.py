"""Pins of the cost-model oracle (oracle/mlp.py) against facts fixed by the mathematics:
a complex-step derivative, a structured network with a closed-form output, the
small-weight linearisation, hidden-unit symmetries, and the closed forms of Adam's
first steps (Kingma & Ba 2015, Algorithm 1)."""
import numpy as np
import pytest

from oracle import mlp


def rand_params(D, H, seed, scale=0.5):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(mlp.param_count(D, H)) * scale


def rand_data(rows, D, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    return r.standard_normal((rows, D)), r.standard_normal(rows)


def test_param_count_layout():
    D, H = 5, 7
    p = np.arange(mlp.param_count(D, H), dtype=np.float64)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, D, H)
    assert W1.shape == (H, D) and W1[1, 0] == D  # row-major: W1[h, d] at h*D + d
    assert b1[0] == H * D
    assert W2.shape == (H, H) and W2[0, 1] == H * D + H + 1
    assert b2[0] == H * D + H + H * H
    assert w3[0] == H * D + 2 * H + H * H
    assert b3 == p.size - 1


def test_structured_network_closed_form():
    """Only W1[0, 1] = a, W2[0, 0] = c and w3[0] = 1 non-zero: y = tanh(c tanh(a x_1)).
    A transposed W1 or W2 would pick another input or unit and fail."""
    D, H = 3, 4
    p = np.zeros(mlp.param_count(D, H))
    W1, b1, W2, b2, w3, _ = mlp.unpack(p, D, H)
    a, c = 0.7, -1.3
    W1[0, 1] = a
    W2[0, 0] = c
    w3[0] = 1.0
    X, _ = rand_data(9, D, 1)
    assert np.allclose(mlp.forward(p, X, D, H), np.tanh(c * np.tanh(a * X[:, 1])), rtol=0, atol=1e-15)
    p[-1] = 0.25  # b3 shifts the output
    assert np.allclose(mlp.forward(p, X, D, H), np.tanh(c * np.tanh(a * X[:, 1])) + 0.25, rtol=0, atol=1e-15)


def test_small_weight_linearisation():
    """For weights of scale s, tanh(z) = z + O(z^3): y agrees with the linear network
    w3^T (W2 (W1 x + b1) + b2) + b3 to O(s^4) (the cube of a pre-activation times w3)."""
    D, H = 4, 6
    X, _ = rand_data(20, D, 2)
    for s in (1e-2, 1e-3):
        p = rand_params(D, H, 3, scale=s)
        W1, b1, W2, b2, w3, b3 = mlp.unpack(p, D, H)
        lin = (W2 @ (X @ W1.T + b1).T + b2[:, None]).T @ w3 + b3
        err = np.max(np.abs(mlp.forward(p, X, D, H) - lin))
        assert err < 50 * s ** 4, (s, err)


def test_hidden_unit_symmetries():
    """Permuting hidden units, or flipping the sign of a first-layer unit together with
    its outgoing weights (tanh is odd), leaves the output unchanged."""
    D, H = 3, 5
    p = rand_params(D, H, 4)
    X, _ = rand_data(11, D, 5)
    y = mlp.forward(p, X, D, H)
    q = p.copy()
    W1, b1, W2, b2, w3, _ = mlp.unpack(q, D, H)
    perm = np.array([2, 0, 4, 1, 3])
    W1[:] = W1[perm]
    b1[:] = b1[perm]
    W2[:] = W2[:, perm]
    assert np.allclose(mlp.forward(q, X, D, H), y, rtol=0, atol=1e-14)
    q = p.copy()
    W1, b1, W2, b2, w3, _ = mlp.unpack(q, D, H)
    W1[1] *= -1
    b1[1] *= -1
    W2[:, 1] *= -1
    assert np.allclose(mlp.forward(q, X, D, H), y, rtol=0, atol=1e-14)
    q = p.copy()
    W1, b1, W2, b2, w3, _ = mlp.unpack(q, D, H)
    perm2 = np.array([4, 3, 2, 1, 0])
    W2[:] = W2[perm2]
    b2[:] = b2[perm2]
    w3[:] = w3[perm2]
    assert np.allclose(mlp.forward(q, X, D, H), y, rtol=0, atol=1e-14)


def test_fd_gradient_matches_complex_step():
    """Complex-step derivative Im L(p + i h e_k) / h (exact to rounding for analytic L,
    an independent route to the gradient) against the oracle's central differences."""
    D, H = 4, 5
    p = rand_params(D, H, 6)
    X, t = rand_data(17, D, 7)
    g = mlp.fd_grad(p, X, t, D, H)
    hc = 1e-30
    cs = np.zeros_like(p)
    for k in range(p.size):
        q = p.astype(np.complex128)
        q[k] += 1j * hc
        e = mlp.forward(q, X, D, H) - t
        cs[k] = np.mean(e * e).imag / hc  # e*e, not |e|^2: keeps L analytic
    assert np.max(np.abs(g - cs)) <= 1e-7 * max(1.0, np.max(np.abs(cs)))


def test_fd_gradient_of_loss_in_b3_closed_form():
    """dL/db3 = 2 mean(y - t): the output bias enters y with coefficient 1."""
    D, H = 3, 4
    p = rand_params(D, H, 8)
    X, t = rand_data(13, D, 9)
    g = mlp.fd_grad(p, X, t, D, H)
    assert abs(g[-1] - 2 * np.mean(mlp.forward(p, X, D, H) - t)) < 1e-8


def test_adam_first_step_closed_form():
    """From m = v = 0 the bias-corrected moments are g and g^2: the step is
    -lr g / (|g| + eps), about lr in size whatever the gradient's scale."""
    g = np.array([3.0, -1e-3, 0.5, -7.0])
    p0 = np.array([1.0, 2.0, -1.0, 0.0])
    lr, eps = 0.01, 1e-8
    p1, m, v = mlp.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, lr, 0.9, 0.999, eps)
    assert np.allclose(p1, p0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_closed_form():
    """With the same gradient at every step the corrected moments stay g and g^2, so k
    steps move each parameter by k lr g / (|g| + eps)."""
    g = np.array([0.3, -2.0])
    p = np.array([0.0, 1.0])
    m = v = np.zeros(2)
    for k in range(1, 26):
        p, m, v = mlp.adam_step(p, g, m, v, k, 0.05, 0.8, 0.95, 1e-8)
    assert np.allclose(p, np.array([0.0, 1.0]) - 25 * 0.05 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_adam_minimises_quadratic():
    c = np.array([1.5, -0.5, 2.0])
    p = np.zeros(3)
    m = v = np.zeros(3)
    for k in range(1, 3001):
        p, m, v = mlp.adam_step(p, 2 * (p - c), m, v, k, 0.01)
    assert np.max(np.abs(p - c)) < 1e-3


@pytest.mark.parametrize("D,H", [(1, 1), (8, 16)])
def test_fd_gradient_of_zero_loss_is_zero(D, H):
    """At a perfect fit (targets = the model's own outputs) the loss has its minimum 0."""
    p = rand_params(D, H, 10)
    X, _ = rand_data(7, D, 11)
    t = mlp.forward(p, X, D, H)
    assert np.max(np.abs(mlp.fd_grad(p, X, t, D, H))) < 1e-9
