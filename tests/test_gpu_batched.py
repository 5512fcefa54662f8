"""Batched reductions of uneven matrices (lockstep launches, cluster panels, split
precision), against the oracle per matrix, and replayed from a captured CUDA graph.

Each matrix must meet the split-precision tolerances of the single-matrix path (bf16x6:
backward error <= 3e-5, spectrum of B within 2e-5 of the oracle's band relative to the
largest eigen/singular value); the graph replay must reproduce the eager run bit for bit
(the batched kernels sum in a fixed order).
"""
import numpy as np
import pytest

import oracle
import workloads
from checks import gen_band, gen_report, sym_band, sym_report
from gpu_util import to_dev, to_host

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


def sym_batch(seed=0, count=9):
    r = np.random.Generator(np.random.PCG64(seed))
    shapes = [(int(r.integers(40, 320)), int(r.choice([16, 32]))) for _ in range(count)] + [(34, 32), (18, 16)]
    mats = [workloads.sym_gaussian(n, seed=100 + q) for q, (n, _) in enumerate(shapes)]
    return shapes, mats


def gen_batch(seed=1, count=7):
    r = np.random.Generator(np.random.PCG64(seed))
    shapes = []
    for _ in range(count):
        n = int(r.integers(20, 260))
        shapes.append((int(r.integers(n, 2 * n + 1)), n, int(r.choice([16, 32]))))
    shapes.append((40, 40, 16))
    mats = [workloads.gen_gaussian(m, n, seed=200 + q) for q, (m, n, _) in enumerate(shapes)]
    return shapes, mats


def run_sy(br, shapes, mats, precision="bf16x6", graph=False):
    import torch

    dAs = [to_dev(a) for a in mats]
    taus = [torch.zeros(max(n - w, 0), dtype=torch.float64, device="cuda") for (n, w) in shapes]
    bt = br.SyBatch(dAs, [w for (_, w) in shapes], taus, br.make_opts(precision=precision))
    work = torch.empty(bt.workspace(), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert bt.plan(work) == 0, br.bandred_last_error()
    if not graph:
        assert bt.run(work, st) == 0, br.bandred_last_error()
    else:
        originals = [to_dev(a) for a in mats]
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                for d, o in zip(dAs, originals):
                    d.copy_(o)
                assert bt.run(work, st) == 0
        for _ in range(2):  # replay twice: the second replay starts from restored inputs
            g.replay()
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return [to_host(d) for d in dAs], [t.cpu().numpy() for t in taus]


def test_sy2sb_batched_matches_oracle(br):
    shapes, mats = sym_batch()
    outs, taus = run_sy(br, shapes, mats)
    for (n, w), A, Aout, tau in zip(shapes, mats, outs, taus):
        r = sym_report(A, Aout, tau, w)
        assert r["backward"] <= 3e-5 and r["orth"] <= 1e-13, (n, w, r)
        Ao, _ = oracle.sy2sb(A, w)
        lg = np.linalg.eigvalsh(sym_band(Aout, w))
        lo = np.linalg.eigvalsh(sym_band(Ao, w))
        assert np.max(np.abs(lg - lo)) <= 2e-5 * np.linalg.norm(A, 2), (n, w)


def test_sy2sb_batched_graph_replay_is_bitwise_identical(br):
    shapes, mats = sym_batch(seed=3, count=6)
    eager, te = run_sy(br, shapes, mats)
    graph, tg = run_sy(br, shapes, mats, graph=True)
    for a, b, x, y in zip(eager, graph, te, tg):
        np.testing.assert_array_equal(np.tril(a), np.tril(b))
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", ["bf16x3", "bf16x6"])
def test_ge2gb_batched_matches_oracle(br, precision):
    import torch

    shapes, mats = gen_batch()
    dAs = [to_dev(a) for a in mats]
    tqs = [torch.zeros(n, dtype=torch.float64, device="cuda") for (_, n, _) in shapes]
    tps = [torch.zeros(max(n - w, 0), dtype=torch.float64, device="cuda") for (_, n, w) in shapes]
    bt = br.GeBatch(dAs, [w for (_, _, w) in shapes], tqs, tps, br.make_opts(precision=precision))
    work = torch.empty(bt.workspace(), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert bt.plan(work) == 0, br.bandred_last_error()
    assert bt.run(work, st) == 0, br.bandred_last_error()
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    tb, ts = {"bf16x3": (2e-4, 1e-4), "bf16x6": (3e-5, 2e-5)}[precision]
    for (m, n, w), A, dA, tq, tp in zip(shapes, mats, dAs, tqs, tps):
        Aout = to_host(dA)
        r = gen_report(A, Aout, tq.cpu().numpy(), tp.cpu().numpy(), w)
        assert r["backward"] <= tb and r["orth_u"] <= 1e-13 and r["orth_v"] <= 1e-13, (m, n, w, r)
        Ao, _, _ = oracle.ge2gb(A, w)
        sg = np.linalg.svd(gen_band(Aout, w), compute_uv=False)
        so = np.linalg.svd(gen_band(Ao, w), compute_uv=False)
        assert np.max(np.abs(sg - so)) <= ts * so[0], (m, n, w)


def test_batched_rejects_fp64(br):
    import torch

    shapes, mats = sym_batch(count=2)
    dAs = [to_dev(a) for a in mats]
    taus = [torch.zeros(max(n - w, 0), dtype=torch.float64, device="cuda") for (n, w) in shapes]
    bt = br.SyBatch(dAs, [w for (_, w) in shapes], taus, br.make_opts(precision="fp64"))
    assert bt.workspace() == 0
    work = torch.empty(256, dtype=torch.uint8, device="cuda")
    assert bt.plan(work) == -1003  # BANDRED_ERR_UNSUPPORTED
