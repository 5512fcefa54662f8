"""GB300-native reduction of dense FP64 matrices to compact band form.

Python binding of ``libbandred.so`` (the C ABI of ``include/bandred.h``): argument
marshalling only.  Every step of the reduction runs in the library's CUDA kernels;
PyTorch supplies device memory and streams.  There is no CPU fallback: when the library
is missing or no GPU is present, the calls raise.

Matrices are column-major FP64 CUDA tensors: ``A.stride(0) == 1`` and ``lda =
A.stride(1)`` (e.g. ``torch.from_numpy(np.asfortranarray(a)).cuda()`` or ``X.t()`` of a
contiguous ``X``).

Method: Rodriguez-Sanchez et al., "Look-Ahead in the Two-Sided Reduction to Compact
Band Forms for Symmetric Eigenvalue Problems and the SVD" (arXiv:1709.00302), Sections
2 (sy2sb) and 3 (ge2gb).
"""
from __future__ import annotations

import ctypes
import os

from ._build import LIB, build  # noqa: F401

__all__ = [
    "bandred_opts", "make_opts", "lib", "PRECISIONS",
    "bandred_sy2sb_workspace", "bandred_sy2sb_ex", "bandred_sy2sb", "bandred_sy2sb_noalloc",
    "bandred_ge2gb_workspace", "bandred_ge2gb_ex", "bandred_ge2gb",
    "bandred_status_string", "bandred_last_error", "bandred_profile_begin", "bandred_profile_end",
    "bandred_launch_count", "bandred_kernel_stat", "bandred_gemm_split", "bandred_gemm_split_workspace",
    "bandred_syr2k_split", "bandred_syr2k_split_workspace", "SyBatch", "GeBatch", "sy2sb", "ge2gb", "BandredError",
    "bandred_mlp_param_count", "bandred_mlp_workspace", "bandred_mlp_forward", "bandred_mlp_loss_grad",
    "bandred_mlp_adam",
]

PRECISIONS = {"fp64": 0, "bf16x3": 1, "bf16x6": 2, "ozaki": 3}


class bandred_opts(ctypes.Structure):
    _fields_ = [
        ("b", ctypes.c_int),
        ("lookahead", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("slices", ctypes.c_int),
        ("panel_ctas", ctypes.c_int),
        ("timeout_ms", ctypes.c_int),
        ("debug", ctypes.c_int),
        ("panel_group", ctypes.c_int),
        ("depth", ctypes.c_int),
        ("reserved", ctypes.c_int * 7),
    ]


class bandred_trace_record(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("iteration", ctypes.c_longlong),
        ("t0_ns", ctypes.c_ulonglong),
        ("t1_ns", ctypes.c_ulonglong),
    ]


class bandred_kernel_stat(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 32),
        ("launches", ctypes.c_longlong),
        ("ms", ctypes.c_double),
        ("flops", ctypes.c_double),
        ("bytes", ctypes.c_double),
    ]


class BandredError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = f"{where}: {code} ({bandred_status_string(code)})"
        if code == -1001 or code == -1004:
            msg += f": {bandred_last_error()}"
        super().__init__(msg)
        self.code = code


_lib = None


def lib():
    """The loaded libbandred.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_1709_00302_gb300.build()")
        L = ctypes.CDLL(LIB)
        i64, vp, sz, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        op = ctypes.POINTER(bandred_opts)
        L.bandred_default_opts.argtypes = [op]
        L.bandred_default_opts.restype = None
        L.bandred_status_string.argtypes = [ci]
        L.bandred_status_string.restype = ctypes.c_char_p
        L.bandred_last_error.argtypes = []
        L.bandred_last_error.restype = ctypes.c_char_p
        L.bandred_sy2sb_workspace.argtypes = [i64, i64, op]
        L.bandred_sy2sb_workspace.restype = sz
        L.bandred_sy2sb_ex.argtypes = [i64, i64, vp, i64, vp, op, vp, sz, vp, vp]
        L.bandred_sy2sb_ex.restype = ci
        L.bandred_sy2sb.argtypes = [i64, i64, vp, i64, vp, op, vp]
        L.bandred_sy2sb.restype = ci
        L.bandred_ge2gb_workspace.argtypes = [i64, i64, i64, op]
        L.bandred_ge2gb_workspace.restype = sz
        L.bandred_ge2gb_ex.argtypes = [i64, i64, i64, vp, i64, vp, vp, op, vp, sz, vp, vp]
        L.bandred_ge2gb_ex.restype = ci
        L.bandred_ge2gb.argtypes = [i64, i64, i64, vp, i64, vp, vp, op, vp]
        L.bandred_ge2gb.restype = ci
        L.bandred_gemm_split_workspace.argtypes = [i64, i64, i64, ci]
        L.bandred_gemm_split_workspace.restype = sz
        L.bandred_gemm_split.argtypes = [i64, i64, i64, vp, i64, ci, vp, i64, vp, i64, ci, vp, sz, vp, vp]
        L.bandred_gemm_split.restype = ci
        L.bandred_syr2k_split_workspace.argtypes = [i64, i64, ci]
        L.bandred_syr2k_split_workspace.restype = sz
        L.bandred_syr2k_split.argtypes = [i64, i64, vp, i64, vp, i64, vp, i64, ci, vp, sz, vp, vp]
        L.bandred_syr2k_split.restype = ci
        p64 = ctypes.POINTER(ctypes.c_int64)
        pvp = ctypes.POINTER(ctypes.c_void_p)
        L.bandred_sy2sb_batched_workspace.argtypes = [ci, p64, p64, op]
        L.bandred_sy2sb_batched_workspace.restype = sz
        L.bandred_sy2sb_batched_plan.argtypes = [ci, p64, p64, pvp, p64, pvp, op, vp, sz, vp]
        L.bandred_sy2sb_batched_plan.restype = ci
        L.bandred_sy2sb_batched_run.argtypes = [ci, p64, p64, pvp, p64, pvp, op, vp, sz, vp, vp]
        L.bandred_sy2sb_batched_run.restype = ci
        L.bandred_ge2gb_batched_workspace.argtypes = [ci, p64, p64, p64, op]
        L.bandred_ge2gb_batched_workspace.restype = sz
        L.bandred_ge2gb_batched_plan.argtypes = [ci, p64, p64, p64, pvp, p64, pvp, pvp, op, vp, sz, vp]
        L.bandred_ge2gb_batched_plan.restype = ci
        L.bandred_ge2gb_batched_run.argtypes = [ci, p64, p64, p64, pvp, p64, pvp, pvp, op, vp, sz, vp, vp]
        L.bandred_ge2gb_batched_run.restype = ci
        L.bandred_sy2sb_noalloc.argtypes = [i64, i64, vp, i64, vp, op, vp, vp]
        L.bandred_sy2sb_noalloc.restype = ci
        L.bandred_profile_begin.argtypes = []
        L.bandred_profile_begin.restype = ci
        L.bandred_profile_end.argtypes = [ctypes.POINTER(bandred_kernel_stat), ci]
        L.bandred_profile_end.restype = ci
        L.bandred_launch_count.argtypes = []
        L.bandred_launch_count.restype = ctypes.c_longlong
        L.bandred_trace_begin.argtypes = [vp, sz]
        L.bandred_trace_begin.restype = ci
        L.bandred_trace_end.argtypes = [ctypes.POINTER(bandred_trace_record), ci]
        L.bandred_trace_end.restype = ci
        L.bandred_panel_phase_trace.argtypes = [vp, ci]
        L.bandred_panel_phase_trace.restype = ci
        L.bandred_sb2st_phase_trace.argtypes = [vp, ci]
        L.bandred_sb2st_phase_trace.restype = ci
        L.bandred_form_workspace.argtypes = [i64, op]
        L.bandred_form_workspace.restype = sz
        L.bandred_sy2sb_form_q.argtypes = [i64, i64, vp, i64, vp, vp, i64, op, vp, sz, vp, vp]
        L.bandred_sy2sb_form_q.restype = ci
        L.bandred_ge2gb_form.argtypes = [i64, i64, i64, vp, i64, vp, ci, vp, i64, op, vp, sz, vp, vp]
        L.bandred_ge2gb_form.restype = ci
        L.bandred_ge2bb_workspace.argtypes = [i64, i64, i64, op]
        L.bandred_ge2bb_workspace.restype = sz
        L.bandred_ge2bb_ex.argtypes = [i64, i64, i64, vp, i64, vp, vp, op, vp, sz, vp, vp]
        L.bandred_ge2bb_ex.restype = ci
        L.bandred_ge2bb_form.argtypes = [i64, i64, i64, vp, i64, vp, ci, vp, i64, op, vp, sz, vp, vp]
        L.bandred_ge2bb_form.restype = ci
        L.bandred_sb2st_workspace.argtypes = [i64, i64]
        L.bandred_sb2st_workspace.restype = sz
        L.bandred_sb2st.argtypes = [i64, i64, vp, i64, vp, vp, op, vp, sz, vp, vp]
        L.bandred_sb2st.restype = ci
        L.bandred_sterf_workspace.argtypes = [i64]
        L.bandred_sterf_workspace.restype = sz
        L.bandred_sterf.argtypes = [i64, vp, vp, vp, vp, sz, vp]
        L.bandred_sterf.restype = ci
        L.bandred_gb2bd_workspace.argtypes = [i64, i64]
        L.bandred_gb2bd_workspace.restype = sz
        L.bandred_gb2bd.argtypes = [i64, i64, vp, i64, vp, vp, op, vp, sz, vp, vp]
        L.bandred_gb2bd.restype = ci
        L.bandred_bdsv_workspace.argtypes = [i64]
        L.bandred_bdsv_workspace.restype = sz
        L.bandred_bdsv.argtypes = [i64, vp, vp, vp, vp, sz, vp]
        L.bandred_bdsv.restype = ci
        L.bandred_newton_eval.argtypes = [i64, vp, vp, vp, vp]
        L.bandred_newton_eval.restype = ci
        L.bandred_fp64_probe.argtypes = [ci, ci, ci, vp, vp]
        L.bandred_fp64_probe.restype = ci
        # cost model of the autotuner (include/bandred_tune.h)
        f32 = ctypes.c_float
        L.bandred_mlp_param_count.argtypes = [ci, ci]
        L.bandred_mlp_param_count.restype = sz
        L.bandred_mlp_workspace.argtypes = [ci, ci, ci]
        L.bandred_mlp_workspace.restype = sz
        L.bandred_mlp_forward.argtypes = [ci, ci, vp, vp, ci, vp, vp]
        L.bandred_mlp_forward.restype = ci
        L.bandred_mlp_loss_grad.argtypes = [ci, ci, vp, vp, vp, ci, vp, vp, vp, sz, vp]
        L.bandred_mlp_loss_grad.restype = ci
        L.bandred_mlp_adam.argtypes = [ci, vp, vp, vp, vp, ci, f32, f32, f32, f32, vp]
        L.bandred_mlp_adam.restype = ci
        _lib = L
    return _lib


def make_opts(b: int = 0, lookahead: int = -1, precision="fp64", slices: int = 0, panel_ctas: int = 0,
              timeout_ms: int = 0, debug: int = 0, panel_group: int = 0, depth: int = 0) -> bandred_opts:
    o = bandred_opts()
    lib().bandred_default_opts(ctypes.byref(o))
    o.b = b
    o.lookahead = lookahead
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.slices = slices
    o.panel_ctas = panel_ctas
    o.timeout_ms = timeout_ms
    o.debug = debug
    o.panel_group = panel_group
    o.depth = depth
    return o


def bandred_status_string(code: int) -> str:
    return lib().bandred_status_string(int(code)).decode()


def bandred_last_error() -> str:
    return lib().bandred_last_error().decode()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _lda(A) -> int:
    import torch

    if A.dtype != torch.float64 or not A.is_cuda or A.dim() != 2:
        raise TypeError("A must be a 2-D float64 CUDA tensor")
    if A.shape[0] > 1 and A.stride(0) != 1:
        raise ValueError("A must be column-major (A.stride(0) == 1)")
    return max(A.stride(1), A.shape[0], 1)


def _opts_ref(opts):
    return None if opts is None else ctypes.byref(opts)


# ------------------------------------------------------------------ raw C-ABI calls
def bandred_sy2sb_workspace(n: int, w: int, opts: bandred_opts | None = None) -> int:
    return lib().bandred_sy2sb_workspace(n, w, _opts_ref(opts))


def bandred_sy2sb_ex(A, w: int, tau, opts, work, dev_status=None, stream=None) -> int:
    n = A.shape[0]
    return lib().bandred_sy2sb_ex(n, w, _ptr(A), _lda(A), _ptr(tau), _opts_ref(opts), _ptr(work),
                                  work.numel() * work.element_size() if work is not None else 0,
                                  _ptr(dev_status), _stream(stream))


def bandred_sy2sb(A, w: int, tau, opts=None, stream=None) -> int:
    return lib().bandred_sy2sb(A.shape[0], w, _ptr(A), _lda(A), _ptr(tau), _opts_ref(opts), _stream(stream))


NOALLOC_SCRATCH_BYTES = 16 << 20


def bandred_sy2sb_noalloc(A, w: int, tau, opts=None, dev_status=None, stream=None) -> int:
    """bandred_sy2sb_ex without a workspace argument, for callers that cannot allocate:
    the library's fixed device scratch array is used instead (see include/bandred.h)."""
    return lib().bandred_sy2sb_noalloc(A.shape[0], w, _ptr(A), _lda(A), _ptr(tau), _opts_ref(opts),
                                       _ptr(dev_status), _stream(stream))


def bandred_ge2gb_workspace(m: int, n: int, w: int, opts: bandred_opts | None = None) -> int:
    return lib().bandred_ge2gb_workspace(m, n, w, _opts_ref(opts))


def bandred_ge2gb_ex(A, w: int, tauq, taup, opts, work, dev_status=None, stream=None) -> int:
    m, n = A.shape
    return lib().bandred_ge2gb_ex(m, n, w, _ptr(A), _lda(A), _ptr(tauq), _ptr(taup), _opts_ref(opts), _ptr(work),
                                  work.numel() * work.element_size() if work is not None else 0,
                                  _ptr(dev_status), _stream(stream))


def bandred_ge2gb(A, w: int, tauq, taup, opts=None, stream=None) -> int:
    m, n = A.shape
    return lib().bandred_ge2gb(m, n, w, _ptr(A), _lda(A), _ptr(tauq), _ptr(taup), _opts_ref(opts), _stream(stream))


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def bandred_gemm_split_workspace(m: int, n: int, k: int, precision="bf16x6") -> int:
    return lib().bandred_gemm_split_workspace(m, n, k, _prec(precision))


def bandred_gemm_split(A, B, C, precision="bf16x6", transA=False, work=None, dev_status=None, stream=None) -> int:
    """C = op(A) B on the split-precision tensor-core engine (column-major CUDA tensors)."""
    import torch

    k, n = B.shape
    m = C.shape[0]
    if work is None:
        work = torch.empty(max(bandred_gemm_split_workspace(m, n, k, precision), 256), dtype=torch.uint8,
                           device=C.device)
    return lib().bandred_gemm_split(m, n, k, _ptr(A), _lda(A), 1 if transA else 0, _ptr(B), _lda(B), _ptr(C), _lda(C),
                                    _prec(precision), _ptr(work), work.numel(), _ptr(dev_status), _stream(stream))


def bandred_syr2k_split_workspace(n: int, kb: int, precision="bf16x6") -> int:
    return lib().bandred_syr2k_split_workspace(n, kb, _prec(precision))


def bandred_syr2k_split(X, Y, C, precision="bf16x6", work=None, dev_status=None, stream=None) -> int:
    """Lower triangle of C += X Y^T + Y X^T on the split-precision engine."""
    import torch

    n, kb = X.shape
    if work is None:
        work = torch.empty(max(bandred_syr2k_split_workspace(n, kb, precision), 256), dtype=torch.uint8,
                           device=C.device)
    return lib().bandred_syr2k_split(n, kb, _ptr(X), _lda(X), _ptr(Y), _lda(Y), _ptr(C), _lda(C), _prec(precision),
                                     _ptr(work), work.numel(), _ptr(dev_status), _stream(stream))


def bandred_profile_begin() -> int:
    return lib().bandred_profile_begin()


def bandred_profile_end(max_entries: int = 16) -> list:
    """Per-kernel-class stats since bandred_profile_begin(): list of dicts."""
    arr = (bandred_kernel_stat * max_entries)()
    n = lib().bandred_profile_end(arr, max_entries)
    if n < 0:
        raise BandredError(n, "bandred_profile_end")
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "ms": arr[i].ms,
             "flops": arr[i].flops, "bytes": arr[i].bytes} for i in range(n)]


def bandred_launch_count() -> int:
    return lib().bandred_launch_count()


# ------------------------------------------------------------------ cost model (bandred_tune.h)
def bandred_mlp_param_count(d_in: int, hidden: int) -> int:
    return lib().bandred_mlp_param_count(d_in, hidden)


def bandred_mlp_workspace(d_in: int, hidden: int, rows: int) -> int:
    return lib().bandred_mlp_workspace(d_in, hidden, rows)


def bandred_mlp_forward(d_in, hidden, params, X, rows, y, stream=None) -> int:
    return lib().bandred_mlp_forward(d_in, hidden, _ptr(params), _ptr(X), rows, _ptr(y), _stream(stream))


def bandred_mlp_loss_grad(d_in, hidden, params, X, t, rows, grad, loss, work, stream=None) -> int:
    return lib().bandred_mlp_loss_grad(d_in, hidden, _ptr(params), _ptr(X), _ptr(t), rows, _ptr(grad), _ptr(loss),
                                       _ptr(work), 0 if work is None else work.numel() * work.element_size(),
                                       _stream(stream))


def bandred_mlp_adam(count, params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> int:
    return lib().bandred_mlp_adam(count, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr, beta1, beta2, eps,
                                  _stream(stream))


# ------------------------------------------------------------------ batched
def _i64(vals):
    return (ctypes.c_int64 * max(len(vals), 1))(*[int(v) for v in vals])


def _ptrs(ts):
    return (ctypes.c_void_p * max(len(ts), 1))(*[t.data_ptr() if t is not None and t.numel() else 0 for t in ts])


class SyBatch:
    """Arguments of bandred_sy2sb_batched_* for lists of column-major CUDA matrices and
    tau vectors (kept alive by this object)."""

    def __init__(self, As, w, taus, opts=None):
        self.As, self.taus = As, taus
        self.n = _i64([a.shape[0] for a in As])
        self.w = _i64(w)
        self.lda = _i64([_lda(a) for a in As])
        self.A = _ptrs(As)
        self.tau = _ptrs(taus)
        self.count = len(As)
        self.opts = opts if opts is not None else make_opts(precision="bf16x6")

    def workspace(self):
        return lib().bandred_sy2sb_batched_workspace(self.count, self.n, self.w, ctypes.byref(self.opts))

    def plan(self, work, stream=None):
        return lib().bandred_sy2sb_batched_plan(self.count, self.n, self.w, self.A, self.lda, self.tau,
                                                ctypes.byref(self.opts), _ptr(work), work.numel(), _stream(stream))

    def run(self, work, dev_status=None, stream=None):
        return lib().bandred_sy2sb_batched_run(self.count, self.n, self.w, self.A, self.lda, self.tau,
                                               ctypes.byref(self.opts), _ptr(work), work.numel(), _ptr(dev_status),
                                               _stream(stream))


class GeBatch:
    """Arguments of bandred_ge2gb_batched_* (see SyBatch)."""

    def __init__(self, As, w, tauqs, taups, opts=None):
        self.As, self.tauqs, self.taups = As, tauqs, taups
        self.m = _i64([a.shape[0] for a in As])
        self.n = _i64([a.shape[1] for a in As])
        self.w = _i64(w)
        self.lda = _i64([_lda(a) for a in As])
        self.A = _ptrs(As)
        self.tauq = _ptrs(tauqs)
        self.taup = _ptrs(taups)
        self.count = len(As)
        self.opts = opts if opts is not None else make_opts(precision="bf16x6")

    def workspace(self):
        return lib().bandred_ge2gb_batched_workspace(self.count, self.m, self.n, self.w, ctypes.byref(self.opts))

    def plan(self, work, stream=None):
        return lib().bandred_ge2gb_batched_plan(self.count, self.m, self.n, self.w, self.A, self.lda, self.tauq,
                                                self.taup, ctypes.byref(self.opts), _ptr(work), work.numel(),
                                                _stream(stream))

    def run(self, work, dev_status=None, stream=None):
        return lib().bandred_ge2gb_batched_run(self.count, self.m, self.n, self.w, self.A, self.lda, self.tauq,
                                               self.taup, ctypes.byref(self.opts), _ptr(work), work.numel(),
                                               _ptr(dev_status), _stream(stream))


TRACE_KINDS = {0: "panel", 1: "rank_next_panel", 2: "rank_rest", 3: "x1_product", 4: "row_panel", 5: "left_update",
               6: "right_update", 7: "w_from_gram"}


def bandred_trace_begin(buf) -> int:
    """Arms the device trace with a device uint8 tensor (16 bytes per record)."""
    return lib().bandred_trace_begin(_ptr(buf), buf.numel() * buf.element_size())


def bandred_trace_end(max_records: int = 65536) -> list:
    """The records since bandred_trace_begin: dicts with kind, iteration, t0_ns, t1_ns."""
    arr = (bandred_trace_record * max_records)()
    n = lib().bandred_trace_end(arr, max_records)
    if n < 0:
        raise BandredError(n, "bandred_trace_end")
    return [{"kind": TRACE_KINDS.get(arr[i].kind, str(arr[i].kind)), "iteration": arr[i].iteration,
             "t0_ns": arr[i].t0_ns, "t1_ns": arr[i].t1_ns} for i in range(n)]


def _form_buffers(N: int, opts, device):
    import torch

    Q = torch.empty((N, N), dtype=torch.float64, device=device).t()  # column-major
    work = torch.empty(max(lib().bandred_form_workspace(N, ctypes.byref(opts)), 256), dtype=torch.uint8,
                       device=device)
    status = torch.zeros(1, dtype=torch.int32, device=device)
    return Q, work, status


def sy2sb_form_q(A, w: int, tau, opts: bandred_opts | None = None, stream=None):
    """Q (n x n, column-major CUDA tensor) of the finished sy2sb reduction held in A, tau."""
    n = A.shape[0]
    opts = make_opts() if opts is None else opts
    Q, work, status = _form_buffers(n, opts, A.device)
    rc = lib().bandred_sy2sb_form_q(n, w, _ptr(A), _lda(A), _ptr(tau), _ptr(Q), Q.stride(1), ctypes.byref(opts),
                                    _ptr(work), work.numel(), _ptr(status), _stream(stream))
    if rc != 0:
        raise BandredError(rc, "bandred_sy2sb_form_q")
    return Q, status


def ge2gb_form(A, w: int, tau, side: int, opts: bandred_opts | None = None, stream=None):
    """side 0: U (m x m; Q when m < n), side 1: V (n x n; P when m < n) of a finished ge2gb."""
    m, n = A.shape
    N = m if side == 0 else n
    opts = make_opts() if opts is None else opts
    Q, work, status = _form_buffers(N, opts, A.device)
    rc = lib().bandred_ge2gb_form(m, n, w, _ptr(A), _lda(A), _ptr(tau), side, _ptr(Q), Q.stride(1),
                                  ctypes.byref(opts), _ptr(work), work.numel(), _ptr(status), _stream(stream))
    if rc != 0:
        raise BandredError(rc, "bandred_ge2gb_form")
    return Q, status


def ge2bb(A, w: int, opts: bandred_opts | None = None, stream=None, check: bool = True):
    """In-place reduction of the column-major CUDA tensor A (m x n) to the band with lower
    and upper bandwidth w (Section 3.3).  Returns (A, tauq, taup, dev_status)."""
    import torch

    m, n = A.shape
    opts = make_opts() if opts is None else opts
    tauq = torch.zeros(max(min(n, m - w), 0), dtype=torch.float64, device=A.device)
    taup = torch.zeros(max(min(m, n - w), 0), dtype=torch.float64, device=A.device)
    work = torch.empty(max(lib().bandred_ge2bb_workspace(m, n, w, ctypes.byref(opts)), 256), dtype=torch.uint8,
                       device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    rc = lib().bandred_ge2bb_ex(m, n, w, _ptr(A), _lda(A), _ptr(tauq), _ptr(taup), ctypes.byref(opts), _ptr(work),
                                work.numel(), _ptr(status), _stream(stream))
    if rc != 0:
        raise BandredError(rc, "bandred_ge2bb_ex")
    if check:
        st = int(status.item())
        if st != 0:
            raise BandredError(st, "bandred_ge2bb_ex (device)")
    return A, tauq, taup, status


def ge2bb_form(A, w: int, tau, side: int, opts: bandred_opts | None = None, stream=None):
    """side 0: U (m x m), side 1: V (n x n) of a finished ge2bb."""
    m, n = A.shape
    N = m if side == 0 else n
    opts = make_opts() if opts is None else opts
    Q, work, status = _form_buffers(N, opts, A.device)
    rc = lib().bandred_ge2bb_form(m, n, w, _ptr(A), _lda(A), _ptr(tau), side, _ptr(Q), Q.stride(1),
                                  ctypes.byref(opts), _ptr(work), work.numel(), _ptr(status), _stream(stream))
    if rc != 0:
        raise BandredError(rc, "bandred_ge2bb_form")
    return Q, status


def sb2st(A, w: int, opts: bandred_opts | None = None, stream=None, check: bool = True):
    """Band -> tridiagonal by bulge chasing: the lower band (bandwidth w) of the
    column-major CUDA tensor A (n x n, read only).  Returns (d, e, dev_status)."""
    import torch

    n = A.shape[0]
    d = torch.zeros(max(n, 1), dtype=torch.float64, device=A.device)
    e = torch.zeros(max(n - 1, 1), dtype=torch.float64, device=A.device)
    work = torch.empty(max(lib().bandred_sb2st_workspace(n, w), 256), dtype=torch.uint8, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    rc = lib().bandred_sb2st(n, w, _ptr(A), _lda(A), _ptr(d), _ptr(e), None if opts is None else ctypes.byref(opts),
                             _ptr(work), work.numel(), _ptr(status), _stream(stream))
    if rc != 0:
        raise BandredError(rc, "bandred_sb2st")
    if check:
        st = int(status.item())
        if st != 0:
            raise BandredError(st, "bandred_sb2st (device)")
    return d[:n], e[: max(n - 1, 0)], status


def sterf(d, e, stream=None):
    """Eigenvalues (ascending) of the symmetric tridiagonal (d, e), CUDA tensors."""
    import torch

    n = d.shape[0]
    lam = torch.zeros(max(n, 1), dtype=torch.float64, device=d.device)
    work = torch.empty(max(lib().bandred_sterf_workspace(n), 256), dtype=torch.uint8, device=d.device)
    ee = e if e.numel() > 0 else torch.zeros(1, dtype=torch.float64, device=d.device)
    rc = lib().bandred_sterf(n, _ptr(d), _ptr(ee), _ptr(lam), _ptr(work), work.numel(), _stream(stream))
    if rc != 0:
        raise BandredError(rc, "bandred_sterf")
    return lam[:n]


def gb2bd(A, w: int, opts: bandred_opts | None = None, stream=None, check: bool = True):
    """Upper band -> upper bidiagonal by bulge chasing: the upper band (bandwidth w) of the
    column-major CUDA tensor A (its upper n x n triangle, read only; n = A.shape[1]).
    Returns (d, e, dev_status): the diagonal and the superdiagonal."""
    import torch

    n = A.shape[1]
    d = torch.zeros(max(n, 1), dtype=torch.float64, device=A.device)
    e = torch.zeros(max(n - 1, 1), dtype=torch.float64, device=A.device)
    work = torch.empty(max(lib().bandred_gb2bd_workspace(n, w), 256), dtype=torch.uint8, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    rc = lib().bandred_gb2bd(n, w, _ptr(A), _lda(A), _ptr(d), _ptr(e), None if opts is None else ctypes.byref(opts),
                             _ptr(work), work.numel(), _ptr(status), _stream(stream))
    if rc != 0:
        raise BandredError(rc, "bandred_gb2bd")
    if check:
        st = int(status.item())
        if st != 0:
            raise BandredError(st, "bandred_gb2bd (device)")
    return d[:n], e[: max(n - 1, 0)], status


def bdsv(d, e, stream=None):
    """Singular values (descending) of the upper bidiagonal (d, e), CUDA tensors."""
    import torch

    n = d.shape[0]
    sig = torch.zeros(max(n, 1), dtype=torch.float64, device=d.device)
    work = torch.empty(max(lib().bandred_bdsv_workspace(n), 256), dtype=torch.uint8, device=d.device)
    ee = e if e.numel() > 0 else torch.zeros(1, dtype=torch.float64, device=d.device)
    rc = lib().bandred_bdsv(n, _ptr(d), _ptr(ee), _ptr(sig), _ptr(work), work.numel(), _stream(stream))
    if rc != 0:
        raise BandredError(rc, "bandred_bdsv")
    return sig[:n]


def bandred_panel_phase_trace(buf) -> int:
    """Arms the phase timing of the next grid panel into the device int64 tensor buf (8 per step)."""
    return lib().bandred_panel_phase_trace(_ptr(buf), buf.numel() // 8)


def bandred_sb2st_phase_trace(buf) -> int:
    """Arms the phase timing of the next bulge chase (its middle sweep) into the device int64
    tensor buf (16 per step)."""
    return lib().bandred_sb2st_phase_trace(_ptr(buf), buf.numel() // 16)


def bandred_newton_eval(x, rsqrt=None, rcp=None, stream=None) -> int:
    """The panel kernels' Newton-Raphson 1/sqrt(x) and 1/x of the device FP64 tensor x."""
    return lib().bandred_newton_eval(x.numel(), _ptr(x), _ptr(rsqrt), _ptr(rcp), _stream(stream))


def bandred_fp64_probe(blocks: int, threads: int, iters: int, sink, stream=None) -> int:
    """FP64 FMA throughput probe (16 * blocks * threads * iters flops); sink: device FP64."""
    return lib().bandred_fp64_probe(blocks, threads, iters, _ptr(sink), _stream(stream))


# ------------------------------------------------------------------ conveniences
def sy2sb(A, w: int, opts: bandred_opts | None = None, stream=None, check: bool = True):
    """In-place symmetric band reduction of the column-major CUDA tensor A.

    Returns (A, tau, dev_status) with tau on the device; raises BandredError on a
    negative return code, and (when ``check``) synchronises to raise on a device status.
    """
    import torch

    n = A.shape[0]
    opts = make_opts() if opts is None else opts
    tau = torch.zeros(max(n - w, 0), dtype=torch.float64, device=A.device)
    work = torch.empty(max(bandred_sy2sb_workspace(n, w, opts), 256), dtype=torch.uint8, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    rc = bandred_sy2sb_ex(A, w, tau, opts, work, status, stream)
    if rc != 0:
        raise BandredError(rc, "bandred_sy2sb_ex")
    if check:
        st = int(status.item())
        if st != 0:
            raise BandredError(st, "bandred_sy2sb_ex (device)")
    return A, tau, status


def ge2gb(A, w: int, opts: bandred_opts | None = None, stream=None, check: bool = True):
    """In-place reduction of the column-major CUDA tensor A (m x n) to band form: upper
    triangular band for m >= n, lower band for m < n (see include/bandred.h).  Returns
    (A, tauq, taup, dev_status)."""
    import torch

    m, n = A.shape
    opts = make_opts() if opts is None else opts
    nq, np_ = (n, max(n - w, 0)) if m >= n else (max(m - w, 0), m)
    tauq = torch.zeros(nq, dtype=torch.float64, device=A.device)
    taup = torch.zeros(np_, dtype=torch.float64, device=A.device)
    work = torch.empty(max(bandred_ge2gb_workspace(m, n, w, opts), 256), dtype=torch.uint8, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    rc = bandred_ge2gb_ex(A, w, tauq, taup, opts, work, status, stream)
    if rc != 0:
        raise BandredError(rc, "bandred_ge2gb_ex")
    if check:
        st = int(status.item())
        if st != 0:
            raise BandredError(st, "bandred_ge2gb_ex (device)")
    return A, tauq, taup, status
