"""Split-precision tensor-core engine (tcgen05) against FP64 products, through the C ABI.

The engine forms FP64 products from bf16 slices with FP32 accumulation in tensor memory
(recombined in FP64 every 256 reduction steps).  Bounds checked per entry, relative to
(|A| |B|)_ij = sum_k |a_ik| |b_kj|:
  bf16x3 (2 slices, 3 products): slice error ~2^-16, FP32 accumulation <= 256 * 2^-24
  bf16x6 (3 slices, 6 products): slice error ~2^-24, same accumulation bound
The typical (RMS) relative error must also be well inside the bound, which a layout or
descriptor mistake (wrong operand element, transposed tile, dropped slice product) fails.
"""
import numpy as np
import pytest

from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

BOUND = {"bf16x3": 2.0 ** -13, "bf16x6": 2.0 ** -15}
RMS = {"bf16x3": 3e-5, "bf16x6": 3e-7}


@pytest.fixture(scope="module")
def br():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_00302_gb300 as br

    br.build()
    br.lib()
    return br


def rel_errors(C, Cref, absprod):
    e = np.abs(C - Cref) / np.maximum(absprod, 1e-300)
    return e.max(), np.sqrt(np.mean(e ** 2))


@pytest.mark.parametrize("precision", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("m,n,k,trans", [(128, 64, 32, 0), (300, 64, 1000, 0), (257, 33, 700, 1), (1000, 128, 4100, 0),
                                         (64, 64, 8000, 1), (5, 16, 3, 0)])
def test_gemm_split(br, precision, m, n, k, trans):
    import torch

    rng = np.random.Generator(np.random.PCG64(m + n + k))
    A = rng.standard_normal((k, m) if trans else (m, k))
    B = rng.standard_normal((k, n))
    dA, dB = to_dev(A), to_dev(B)
    dC = to_dev(np.full((m, n), np.nan))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert br.bandred_gemm_split(dA, dB, dC, precision, transA=bool(trans), dev_status=st) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Aop = A.T if trans else A
    C = to_host(dC)
    Cref = Aop @ B
    absprod = np.abs(Aop) @ np.abs(B)
    mx, rms = rel_errors(C, Cref, absprod)
    assert mx <= BOUND[precision], (mx, rms)
    assert rms <= RMS[precision], (mx, rms)


@pytest.mark.parametrize("precision", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("n,kb", [(128, 64), (300, 64), (513, 32), (1000, 16), (77, 5)])
def test_syr2k_split(br, precision, n, kb):
    import torch

    rng = np.random.Generator(np.random.PCG64(n * kb))
    X = rng.standard_normal((n, kb))
    Y = rng.standard_normal((n, kb))
    C0 = rng.standard_normal((n, n))
    Cu = C0.copy()
    Cu[np.triu_indices(n, 1)] = np.nan  # the upper triangle must stay untouched
    dX, dY, dC = to_dev(X), to_dev(Y), to_dev(Cu)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert br.bandred_syr2k_split(dX, dY, dC, precision, dev_status=st) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    C = to_host(dC)
    assert np.all(np.isnan(C[np.triu_indices(n, 1)]))
    ref = C0 + X @ Y.T + Y @ X.T
    absprod = np.abs(X) @ np.abs(Y.T) + np.abs(Y) @ np.abs(X.T)
    L = np.tril_indices(n)
    mx, rms = rel_errors(C[L] - C0[L], ref[L] - C0[L], absprod[L])
    assert mx <= BOUND[precision], (mx, rms)
    assert rms <= RMS[precision], (mx, rms)


def test_range_status(br):
    import torch

    A = np.ones((128, 32))
    A[3, 4] = 1e-300  # below the representable range of the slices
    B = np.ones((32, 16))
    dC = to_dev(np.zeros((128, 16)))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert br.bandred_gemm_split(to_dev(A), to_dev(B), dC, "bf16x6", dev_status=st) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 3  # BANDRED_DEV_RANGE
