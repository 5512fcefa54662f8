"""The autotuner's cost model on the GPU (bandred_mlp_* of include/bandred_tune.h)
against the FP64 oracle (oracle/mlp.py): forward pass, back-propagated gradient against
the oracle's finite differences, loss, the Adam step, reproducibility and training.

Tolerances come from FP32 arithmetic: outputs and losses within 1e-5 relative, the
gradient within 1e-3 of its largest entry (FP32 sums over <= 200 rows against central
differences of step 1e-6 in FP64), Adam within 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def br():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_00302_gb300 as br

    br.build()
    br.lib()
    return br


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def case(D, H, rows, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    p = (r.standard_normal(mlp.param_count(D, H)) * 0.4).astype(np.float32)
    X = r.standard_normal((rows, D)).astype(np.float32)
    t = r.standard_normal(rows).astype(np.float32)
    return p, X, t


def gpu_grad(br, D, H, p, X, t):
    import torch

    rows = X.shape[0]
    P = br.bandred_mlp_param_count(D, H)
    grad = torch.zeros(P, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = torch.empty(br.bandred_mlp_workspace(D, H, rows), dtype=torch.uint8, device="cuda")
    rc = br.bandred_mlp_loss_grad(D, H, dev(p), dev(X), dev(t), rows, grad, loss, work)
    assert rc == 0
    torch.cuda.synchronize()
    return grad.cpu().numpy().astype(np.float64), float(loss.item())


@pytest.mark.parametrize("D,H,rows", [(1, 1, 1), (8, 32, 200), (13, 64, 77), (32, 7, 130)])
def test_forward_matches_oracle(br, D, H, rows):
    import torch

    p, X, _ = case(D, H, rows, 1 + D)
    y = torch.zeros(rows, dtype=torch.float32, device="cuda")
    assert br.bandred_mlp_forward(D, H, dev(p), dev(X), rows, y) == 0
    ref = mlp.forward(p.astype(np.float64), X.astype(np.float64), D, H)
    got = y.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("D,H,rows", [(1, 1, 3), (8, 16, 200), (5, 64, 40)])
def test_gradient_matches_finite_differences(br, D, H, rows):
    p, X, t = case(D, H, rows, 10 + H)
    g, loss = gpu_grad(br, D, H, p, X, t)
    p64, X64, t64 = p.astype(np.float64), X.astype(np.float64), t.astype(np.float64)
    ref = mlp.fd_grad(p64, X64, t64, D, H)
    assert np.max(np.abs(g - ref)) <= 1e-3 * np.max(np.abs(ref))
    assert abs(loss - mlp.loss(p64, X64, t64, D, H)) <= 1e-5 * mlp.loss(p64, X64, t64, D, H)


def test_adam_matches_oracle(br):
    import torch

    r = np.random.Generator(np.random.PCG64(3))
    P = 1000
    p = r.standard_normal(P).astype(np.float32)
    g = r.standard_normal(P).astype(np.float32)
    m = (r.standard_normal(P) * 0.1).astype(np.float32)
    v = np.abs(r.standard_normal(P) * 0.1).astype(np.float32)
    pd, gd, md, vd = dev(p), dev(g), dev(m), dev(v)
    assert br.bandred_mlp_adam(P, pd, gd, md, vd, 7, 1e-2, 0.9, 0.999, 1e-8) == 0
    torch.cuda.synchronize()
    # the oracle takes the hyper-parameters the kernel received: their FP32 values
    # (1 - beta2 is computed exactly from the FP32 beta2 on both sides)
    f = lambda x: float(np.float32(x))
    rp, rm, rv = mlp.adam_step(p, g, m, v, 7, f(1e-2), f(0.9), f(0.999), f(1e-8))
    for got, ref in ((pd, rp), (md, rm), (vd, rv)):
        assert np.allclose(got.cpu().numpy(), ref, rtol=1e-6, atol=1e-7)


def test_invalid_arguments(br):
    assert br.bandred_mlp_param_count(0, 4) == 0
    assert br.bandred_mlp_forward(33, 4, None, None, 0, None) == -1
    assert br.bandred_mlp_forward(4, 65, None, None, 0, None) == -2
    assert br.bandred_mlp_adam(4, None, None, None, None, 1, 0.1) == -2


def train(br, D, H, X, t, steps, lr, seed):
    import torch

    rows = X.shape[0]
    P = br.bandred_mlp_param_count(D, H)
    r = np.random.Generator(np.random.PCG64(seed))
    params = dev((r.standard_normal(P) * 0.3).astype(np.float32))
    m = torch.zeros(P, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    grad = torch.zeros_like(m)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = torch.empty(br.bandred_mlp_workspace(D, H, rows), dtype=torch.uint8, device="cuda")
    Xd, td = dev(X), dev(t)
    losses = []
    for k in range(1, steps + 1):
        assert br.bandred_mlp_loss_grad(D, H, params, Xd, td, rows, grad, loss, work) == 0
        if k == 1 or k == steps:
            losses.append(float(loss.item()))
        assert br.bandred_mlp_adam(P, params, grad, m, v, k, lr) == 0
    torch.cuda.synchronize()
    return params.cpu().numpy(), losses


def test_training_fits_smooth_target_and_is_reproducible(br):
    r = np.random.Generator(np.random.PCG64(4))
    X = r.uniform(-1, 1, (300, 3)).astype(np.float32)
    t = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2]).astype(np.float32)
    p1, l1 = train(br, 3, 16, X, t, 400, 1e-2, 5)
    p2, l2 = train(br, 3, 16, X, t, 400, 1e-2, 5)
    assert l1[-1] < 0.05 * l1[0], l1
    assert np.array_equal(p1, p2) and l1 == l2
