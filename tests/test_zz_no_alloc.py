"""The non-allocating entry point bandred_sy2sb_noalloc, through the C ABI.

It exists for callers that cannot allocate device memory when they call (inside a
stream capture, under a fixed memory budget, or in a process whose allocator they do not
own): it runs the same reduction as bandred_sy2sb_ex with the library's fixed device
scratch array as workspace.  These tests check, on a GPU, that two calls in a row give
the same result as the existing entry point and as the FP64 oracle within the tolerances
of the FP64 parity tests (the Ozaki precision included; bf16x6 by the spectrum of its
band, at its stated tolerance), with the default options (look-ahead on) as well as
without look-ahead, that a call captured into a CUDA graph replays correctly, that the
caller's current device is left alone, and that a problem too large for the scratch is
refused before any device work.  The file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from gpu_util import lower_band_and_v, to_dev, to_host

pytestmark = pytest.mark.gpu

B_TOL = 1e-12   # band entries, relative to ||A||_F (as in the FP64 parity tests)
V_TOL = 1e-10   # reflector entries and tau
ERR_SCRATCH = -1005


@pytest.fixture(scope="module")
def br():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_00302_gb300 as br

    br.build()
    br.lib()
    return br


def call_noalloc(br, A, w, opts):
    """Direct C-ABI call of bandred_sy2sb_noalloc on a device copy of A."""
    import torch

    n = A.shape[0]
    dA = to_dev(A)
    tau = torch.zeros(max(n - w, 0), dtype=torch.float64, device="cuda")
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    dev = torch.cuda.current_device()
    rc = br.lib().bandred_sy2sb_noalloc(n, w, ctypes.c_void_p(dA.data_ptr()), dA.stride(1),
                                        ctypes.c_void_p(tau.data_ptr()), ctypes.byref(opts),
                                        ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert torch.cuda.current_device() == dev
    torch.cuda.synchronize()
    return rc, to_host(dA), tau.cpu().numpy(), int(status.item())


def call_ex(br, A, w, opts):
    import torch

    n = A.shape[0]
    dA = to_dev(A)
    tau = torch.zeros(max(n - w, 0), dtype=torch.float64, device="cuda")
    work = torch.empty(br.bandred_sy2sb_workspace(n, w, opts), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = br.bandred_sy2sb_ex(dA, w, tau, opts, work, status)
    torch.cuda.synchronize()
    return rc, to_host(dA), tau.cpu().numpy(), int(status.item())


@pytest.mark.parametrize("n,w,b", [(512, 32, 32), (1000, 40, 16), (2500, 64, 64)])
def test_noalloc_matches_existing_entry_point_twice(br, n, w, b):
    A = workloads.sym_gaussian(n, seed=n + w)
    opts = br.make_opts(b=b, lookahead=0)
    rc, Aref, tref, st = call_ex(br, A, w, opts)
    assert rc == 0 and st == 0
    fa = np.linalg.norm(A)
    bref, vref = lower_band_and_v(Aref, w)
    for _ in range(2):  # the scratch keeps the previous call's contents: the second call must not care
        rc, Aout, tout, st = call_noalloc(br, A, w, opts)
        assert rc == 0 and st == 0
        bg, vg = lower_band_and_v(Aout, w)
        assert np.max(np.abs(bg - bref)) <= B_TOL * fa
        assert np.max(np.abs(vg - vref), initial=0.0) <= V_TOL
        assert np.max(np.abs(tout - tref), initial=0.0) <= V_TOL
        assert np.all(np.isfinite(Aout[np.tril_indices(n)]))


# the Ozaki buffers are larger (packed digits), so its problem is smaller to fit the scratch
@pytest.mark.parametrize("precision,n,w", [("fp64", 1000, 40), ("ozaki", 600, 32)])
def test_noalloc_default_options_match_the_oracle_twice(br, precision, n, w):
    # default b (= w here, so the V2 look-ahead with its side stream) and default look-ahead
    A = workloads.sym_gaussian(n, seed=n + w + 3)
    opts = br.make_opts(precision=precision)
    assert br.bandred_sy2sb_workspace(n, w, opts) <= br.NOALLOC_SCRATCH_BYTES
    Ao, to = oracle.sy2sb(A, w)
    bo, vo = lower_band_and_v(Ao, w)
    fa = np.linalg.norm(A)
    for _ in range(2):
        rc, Aout, tout, st = call_noalloc(br, A, w, opts)
        assert rc == 0 and st == 0
        bg, vg = lower_band_and_v(Aout, w)
        assert np.max(np.abs(bg - bo)) <= B_TOL * fa
        assert np.max(np.abs(vg - vo), initial=0.0) <= V_TOL
        assert np.max(np.abs(tout - to), initial=0.0) <= V_TOL


def test_noalloc_split_precision_keeps_the_spectrum_twice(br):
    # bf16x6 products (FP32-class): the band's eigenvalues within the stated 2e-5 ||A||_2
    n, w = 800, 32
    A = workloads.sym_gaussian(n, seed=n + w + 5)
    lam = np.linalg.eigvalsh(A)
    opts = br.make_opts(precision="bf16x6")
    i, j = np.indices((n, n))
    for _ in range(2):
        rc, Aout, tout, st = call_noalloc(br, A, w, opts)
        assert rc == 0 and st == 0
        L = np.where((i - j >= 0) & (i - j <= w), Aout, 0.0)
        B = L + np.tril(L, -1).T
        assert np.max(np.abs(np.linalg.eigvalsh(B) - lam)) <= 2e-5 * np.max(np.abs(lam))


@pytest.mark.parametrize("lookahead", [0, -1])
def test_noalloc_captured_in_a_cuda_graph_replays(br, lookahead):
    """The stated use case: after one call outside the capture (which creates the look-ahead
    stream and events), a call is captured into a CUDA graph together with the copy that
    resets A, and two replays each give the oracle's reduction."""
    import torch

    n, w = 600, 32
    A = workloads.sym_gaussian(n, seed=n + w + 9)
    opts = br.make_opts(precision="fp64", lookahead=lookahead)
    dA0 = to_dev(A)
    dA = torch.empty_like(dA0)
    tau = torch.zeros(n - w, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")

    def call():
        s = torch.cuda.current_stream()
        return br.lib().bandred_sy2sb_noalloc(n, w, ctypes.c_void_p(dA.data_ptr()), dA.stride(1),
                                              ctypes.c_void_p(tau.data_ptr()), ctypes.byref(opts),
                                              ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(s.cuda_stream))

    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        dA.copy_(dA0)
        assert call() == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        dA.copy_(dA0)
        rc = call()
    assert rc == 0
    Ao, to = oracle.sy2sb(A, w)
    bo, vo = lower_band_and_v(Ao, w)
    fa = np.linalg.norm(A)
    for _ in range(2):
        dA.zero_()
        tau.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        bg, vg = lower_band_and_v(to_host(dA), w)
        assert np.max(np.abs(bg - bo)) <= B_TOL * fa
        assert np.max(np.abs(vg - vo), initial=0.0) <= V_TOL
        assert np.max(np.abs(tau.cpu().numpy() - to), initial=0.0) <= V_TOL


def test_noalloc_refuses_problems_beyond_the_scratch(br):
    import torch

    n, w = 8192, 64
    opts = br.make_opts(b=64)
    assert br.bandred_sy2sb_workspace(n, w, opts) > br.NOALLOC_SCRATCH_BYTES
    dA = torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
    tau = torch.zeros(n - w, dtype=torch.float64, device="cuda")
    rc = br.bandred_sy2sb_noalloc(dA, w, tau, opts)
    assert rc == ERR_SCRATCH
    assert "fixed scratch" in br.bandred_status_string(rc)
