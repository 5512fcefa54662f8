"""The non-allocating entry point bandred_sy2sb_noalloc, through the C ABI.

It exists for callers that cannot allocate device memory when they call (inside a
stream capture, under a fixed memory budget, or in a process whose allocator they do not
own): it runs the same reduction as bandred_sy2sb_ex with the library's fixed device
scratch array as workspace.  These tests check, on a GPU, that two calls in a row give
the same result as the existing entry point within the tolerances of the FP64 parity
tests, and that a problem too large for the scratch is refused before any device work.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

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
    rc = br.lib().bandred_sy2sb_noalloc(n, w, ctypes.c_void_p(dA.data_ptr()), dA.stride(1),
                                        ctypes.c_void_p(tau.data_ptr()), ctypes.byref(opts),
                                        ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
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
