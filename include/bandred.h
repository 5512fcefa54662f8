/*
 * bandred: reduction of dense FP64 matrices to compact band form on NVIDIA GB300 (sm_103a).
 *
 * The operations follow Rodriguez-Sanchez, Catalan, Herrero, Quintana-Orti, Tomas,
 * "Look-Ahead in the Two-Sided Reduction to Compact Band Forms for Symmetric Eigenvalue
 * Problems and the SVD" (arXiv:1709.00302):
 *
 *   sy2sb  Section 2.1 (Eqs. updateA0, updateA1, updateA2, updateA2symm .. updateA2syr2k)
 *          with the look-ahead of Section 2.2 (Variants V1, 2b <= w, and V2, 2b > w):
 *          symmetric A = Q B Q^T, B symmetric with bandwidth w.
 *   ge2gb  Section 3.1 (Eqs. updateB, updateCD, updateC, updateD) with the look-ahead
 *          rules of Section 3.2 (w >= 3b for both overlaps):
 *          general A (m x n, m >= n) = U B V^T, B upper triangular with upper bandwidth w.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are FP64, column-major: A(i, j) = A[i + j * lda], 0-based.
 *  - Every pointer to matrix data, tau, workspace or status is DEVICE memory owned by the
 *    caller; nothing is freed by the library.  Sizes and option structs are host values.
 *  - Calls are stream-ordered on `stream` and, unless stated otherwise, return on the host
 *    before the device finishes.  The "_ex" and batched forms never allocate memory and
 *    never synchronise; they are safe to capture in a CUDA graph once the first call for
 *    that shape has been made (the first call on a device configures kernel attributes).
 *  - Reflectors follow the Householder convention of Golub & Van Loan as used by LAPACK:
 *    for x = [alpha; x2], beta = -sign(alpha) ||x||_2 with sign(0) = +1,
 *    tau = (beta - alpha) / beta, v = [1; x2 / (alpha - beta)], H = I - tau v v^T;
 *    when x2 = 0 (or x has length 1) tau = 0 and H = I.
 *  - Return value (LAPACK-style info): 0 on success; -i when the i-th argument is invalid;
 *    BANDRED_ERR_* (< -1000) for a CUDA error or an unusable workspace.  Device-side
 *    failures (a bounded wait that timed out) are written to the caller's `dev_status`
 *    (an int in device memory; 0 = OK, see BANDRED_DEV_*), readable after the stream has
 *    been synchronised.  NaN and Inf entries are not checked; they propagate.
 */
#ifndef BANDRED_H
#define BANDRED_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic of the trailing updates (panels, reflectors, T factors and the band
 * write-back are always FP64). */
enum bandred_precision {
    BANDRED_FP64 = 0,      /* FP64 FMA on the CUDA cores */
    BANDRED_BF16X3 = 1,    /* each FP64 operand split into bf16 slices; tensor-core
                              products hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM,
                              FP64 recombination (FP32-class accuracy) */
    BANDRED_BF16X6 = 2,    /* three bf16 slices, the six products of order <= 2 */
    BANDRED_OZAKI = 3      /* FP64-class accuracy on the tensor cores (Ozaki scheme): each
                              row of an operand scaled by a power of two and cut into 7
                              signed 8-bit digits (exact in bf16); digit-pair products
                              accumulated exactly (FP32 sums below 2^24, then 64-bit
                              integers) and combined in FP64; error below 2^-56 of the
                              row and column scales.  `slices` is ignored (7 digits) */
};

/* Look-ahead variant (Section 2.2): 0 = none (the basic right-looking loop), 1 = V1
 * (requires 2b <= w), 2 = V2 (requires 2b > w), -1 = choose from b and w. */
typedef struct bandred_opts {
    int b;                 /* panel width (algorithmic block size), 1 <= b <= w; 0 = default */
    int lookahead;         /* -1 auto, 0 none, 1 V1, 2 V2 */
    int precision;         /* enum bandred_precision */
    int slices;            /* reserved for the digit count of BANDRED_OZAKI; ignored */
    int panel_ctas;        /* CTAs of the panel factorisation (0 = all SMs; with V2
                              look-ahead and BANDRED_OZAKI the next panel takes half the
                              SMs and the rest of the trailing update the others; a value
                              > 0 sets that share).  Batched calls: CTAs (one thread-block
                              cluster, rounded up to a power of two <= 16) per matrix
                              panel; 0 = about 128 rows per CTA */
    int timeout_ms;        /* limit of every device-side wait (0 = 2000 ms) */
    int debug;             /* 0.  Tests only: 1 makes the first device-side wait
                              unsatisfiable, so the call ends through its bounded-wait
                              path and reports BANDRED_DEV_TIMEOUT in dev_status */
    int panel_group;       /* reflectors taken per grid-wide reduction in the FP64 panel
                              factorisation: 0 = default (2), 2 (pairs) or 4 (half the grid
                              barriers, four times the serial scalar work; slower on GB300);
                              1 = pairs, and panels of at most 512 rows on one thread-block
                              cluster, one reflector per cluster barrier (the batched path's
                              panel).  All give the Householder reflectors of Section 2.1 up
                              to rounding */
    int depth;             /* look-ahead depth: 0 = default (1); 2 factors the panel two
                              iterations ahead, only with V1 and 3b <= w (that panel is then
                              reached by one-sided updates alone); otherwise 1 is used */
    int reserved[7];       /* must be zero */
} bandred_opts;

/* Device-side status codes written to dev_status. */
#define BANDRED_DEV_OK 0
#define BANDRED_DEV_TIMEOUT 1      /* a bounded wait ran out; the results are invalid */
#define BANDRED_DEV_INVARIANT 2    /* an internal consistency check failed */
#define BANDRED_DEV_RANGE 3        /* split precision only: an entry outside the range the bf16
                                      slices represent exactly (|x| < 2^-95 or >= 2^127, or
                                      subnormal); results are not valid, use BANDRED_FP64 */

/* Host-side error codes. */
#define BANDRED_ERR_CUDA (-1001)       /* a CUDA runtime call failed */
#define BANDRED_ERR_WORKSPACE (-1002)  /* workspace NULL, misaligned or too small */
#define BANDRED_ERR_UNSUPPORTED (-1003)/* a size beyond what the kernels support */
#define BANDRED_ERR_ALLOC (-1004)      /* the allocating short form could not allocate */
#define BANDRED_ERR_SCRATCH (-1005)    /* bandred_sy2sb_noalloc: the problem needs more than
                                          the fixed scratch (BANDRED_NOALLOC_SCRATCH_BYTES) */

/* Fill *opts with the defaults (b = min(w, 64), auto look-ahead, FP64). */
void bandred_default_opts(bandred_opts* opts);

/* Text for a return value or a device status code. */
const char* bandred_status_string(int code);

/* Description of the last CUDA runtime failure seen by this host thread (the call and
 * the CUDA error), or "" if none.  The string is owned by the library. */
const char* bandred_last_error(void);

/* ---------------------------------------------------------------- sy2sb -------------
 * Symmetric band reduction, Section 2.1: A = Q B Q^T.
 *   n     order of A (n >= 0)
 *   w     bandwidth of B (w >= 1)
 *   A     device, n x n, lda >= max(1, n).  Only the lower triangle is read and written;
 *         the strictly upper triangle is never accessed.  On exit the lower band
 *         0 <= i - j <= w holds B; for reflector c (c = 0 .. n-w-1), A(c+w, c) holds its
 *         beta (the band entry) and A(c+w+1 : n, c) holds v below its implicit unit entry.
 *   tau   device, max(n - w, 0) entries: tau[c] of reflector c (tau[n-w-1] = 0, a length-1
 *         reflector).  Q = H_0 H_1 ... H_{n-w-1}, H_c acting on rows c+w .. n-1.
 * Panels of width b_k = min(b, n - w - 1 - k) start at k = 0, b, 2b, ... while k <= n-w-2.
 */
size_t bandred_sy2sb_workspace(int64_t n, int64_t w, const bandred_opts* opts);

/* Allocating short form: allocates its workspace on `stream` (stream-ordered allocator),
 * runs, synchronises `stream` and returns the device status as a positive code, if any.
 * Not capturable in a CUDA graph.  opts == NULL uses the defaults. */
int bandred_sy2sb(int64_t n, int64_t w, double* A, int64_t lda, double* tau,
                  const bandred_opts* opts, cudaStream_t stream);

/* Non-allocating form.  work: device, 256-byte aligned, at least
 * bandred_sy2sb_workspace(n, w, opts) bytes, not shared with a concurrent call.
 * dev_status: device int (may be NULL) set to 0 at the start and to a BANDRED_DEV_* code
 * on a device-side failure.
 * Every entry point runs on the device that owns A and leaves the caller's current device
 * as it found it.  With look-ahead (the default), the first call of a host thread on a
 * device creates a high-priority stream and four events that the thread's later calls
 * reuse; they live until the process exits. */
int bandred_sy2sb_ex(int64_t n, int64_t w, double* A, int64_t lda, double* tau,
                     const bandred_opts* opts, void* work, size_t work_bytes, int* dev_status,
                     cudaStream_t stream);

/* Non-allocating variant for callers that may not allocate device memory when they
 * call: code inside a stream capture, hosts with a fixed memory budget, plug-ins that
 * do not own the process's allocator.  The paper has no counterpart; this is a
 * deployment convenience.  It computes exactly what bandred_sy2sb_ex computes, with the
 * same arguments minus the workspace: the workspace is a fixed device array of
 * BANDRED_NOALLOC_SCRATCH_BYTES bytes that the library declares at file scope, reserved
 * on every GPU that loads the library until the process exits.  No call allocates or
 * frees memory.
 *   - Limit: the problem must satisfy bandred_sy2sb_workspace(n, w, opts) <=
 *     BANDRED_NOALLOC_SCRATCH_BYTES (about n <= 5500 at w = b = 64 with default options); larger problems
 *     return BANDRED_ERR_SCRATCH before any device work.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before any
 *     stream capture that includes this entry point.  With look-ahead (opts->lookahead
 *     != 0, the default), the first call of a host thread on a device also creates a
 *     high-priority stream and four events that the thread's later calls reuse (as
 *     bandred_sy2sb_ex does); that first call belongs before any capture as well.
 *   - The caller's current device is the same after the call as before it.
 *   - All calls on a device share the one array, and it keeps the previous call's
 *     contents.  Each call zeroes the counters and status word it relies on; everything
 *     else is written before it is read.  Calls that can overlap on the GPU (different
 *     streams without ordering, or different host threads) race on the array: order them.
 * Arguments, layout and return codes are those of bandred_sy2sb_ex. */
#define BANDRED_NOALLOC_SCRATCH_BYTES (16u << 20)
int bandred_sy2sb_noalloc(int64_t n, int64_t w, double* A, int64_t lda, double* tau,
                          const bandred_opts* opts, int* dev_status, cudaStream_t stream);

/* ---------------------------------------------------------------- ge2gb -------------
 * Reduction to upper triangular band form, Section 3.1: A = U B V^T, m >= n.  (m < n: see
 * the end of this comment.)
 *   A     device, m x n, lda >= max(1, m).  On exit the band 0 <= j - i <= w holds B;
 *         left reflector c (c = 0 .. n-1): beta on A(c, c), v below the diagonal in
 *         A(c+1 : m, c); right reflector c (c = 0 .. n-w-1): beta on A(c, c+w), v in row c,
 *         A(c, c+w+1 : n).  Entries below the diagonal and right of superdiagonal w are
 *         reflector storage.
 *   tauq  device, n entries (left reflectors; U = Hq_0 Hq_1 ... Hq_{n-1}, Hq_c acting on
 *         rows c .. m-1).
 *   taup  device, max(n - w, 0) entries (right reflectors; V = Hp_0 Hp_1 ..., Hp_c acting
 *         on columns c+w .. n-1).
 * m < n (Section 3.1 assumes m >= n; the reduction is applied to the tall A^T and
 * written back transposed): A = Q B P^T with B LOWER band, 0 <= i - j <= w.  tauq holds
 * max(m - w, 0) left reflectors: reflector c acts on rows c+w .. m-1, beta on A(c+w, c),
 * v in A(c+w+1 : m, c); Q = Hq_0 Hq_1 ....  taup holds m right reflectors: reflector c
 * acts on columns c .. n-1, beta on A(c, c), v in A(c, c+1 : n); P = Hp_0 Hp_1 ....
 * The workspace then also holds a copy of A^T.
 */
size_t bandred_ge2gb_workspace(int64_t m, int64_t n, int64_t w, const bandred_opts* opts);

int bandred_ge2gb(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq,
                  double* taup, const bandred_opts* opts, cudaStream_t stream);

int bandred_ge2gb_ex(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq,
                     double* taup, const bandred_opts* opts, void* work, size_t work_bytes,
                     int* dev_status, cudaStream_t stream);

/* ---------------------------------------------------------------- ge2bb -------------
 * Reduction to a band with equal lower and upper bandwidth w, Section 3.3 (the SVD band
 * form that admits look-ahead for any b <= w): A = U B V^T, any m, n.
 *   A     device, m x n, lda >= max(1, m).  On exit the band |i - j| <= w holds B; left
 *         reflector c (c = 0 .. min(n, m-w)-1) has beta on A(c+w, c) and v in
 *         A(c+w+1 : m, c); right reflector c (c = 0 .. min(m, n-w)-1) has beta on A(c, c+w)
 *         and v in A(c, c+w+1 : n).
 *   tauq  device, max(min(n, m-w), 0) entries: U = Hq_0 Hq_1 ..., Hq_c on rows c+w .. m-1.
 *   taup  device, max(min(m, n-w), 0) entries: V = Hp_0 Hp_1 ..., Hp_c on columns c+w .. n-1.
 * Per block of b columns and rows: the QR of the column panel and the LQ of the row panel
 * (independent of each other), the one-sided updates of the blocks between the panels and
 * the trailing block, and the trailing block D := Q_L^T D Q_R as one two-sided update
 * D += X Y_R^T + Y_L Z_L^T (Eq. gebrd_2k), with the products in the chosen precision.
 * opts->lookahead: 0 none; otherwise the next iteration's two panels are factored on a
 * second stream, Variant V1 (2b <= w: they lie in B1 and C1, reached by one-sided updates)
 * or V2 (2b > w: after the products of D, the first 2b - w columns and rows of D are
 * updated first, the 2 x 2 partition of D); -1 takes V1 when 2b <= w and none otherwise
 * (V2 measured slower than no look-ahead at b = w), 2 asks for V2.  work, dev_status,
 * return codes: as for bandred_ge2gb_ex.
 */
size_t bandred_ge2bb_workspace(int64_t m, int64_t n, int64_t w, const bandred_opts* opts);
int bandred_ge2bb_ex(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq, double* taup,
                     const bandred_opts* opts, void* work, size_t work_bytes, int* dev_status, cudaStream_t stream);

/* ---------------------------------------------------------------- second stage --------
 * The step after the band form in the paper's eigenvalue experiments (there SBRDT, then
 * DSTERF): band -> tridiagonal by Householder bulge chasing, then the eigenvalues of the
 * tridiagonal.
 *
 * bandred_sb2st: A device, n x n, lda >= max(1, n); its lower band 0 <= i-j <= w holds the
 *   symmetric band B (as bandred_sy2sb leaves it; nothing else of A is read, A is not
 *   written).  Sweep c (c = 0 .. n-3) annihilates B(c+2 : c+w+1, c) by a reflector on the
 *   index range [c+1, c+1+w) applied from both sides, then chases the bulge it creates
 *   below the band down the matrix, one reflector per w rows (larfg convention).  On exit
 *   d (device, n) holds the diagonal and e (device, n - 1) the subdiagonal of T = Q^T B Q.
 *   1 <= w <= 128.  opts: only timeout_ms is used (NULL: defaults).  work: device,
 *   256-byte aligned, >= bandred_sb2st_workspace(n, w) bytes (the band with room for the
 *   bulge, 2 w n doubles, and per-sweep progress counters).  dev_status: as for
 *   bandred_sy2sb_ex (BANDRED_DEV_TIMEOUT when a sweep's bounded wait for the previous
 *   sweep gave up).  Returns 0, -i for an invalid i-th argument, BANDRED_ERR_UNSUPPORTED
 *   for w > 128, or a CUDA error code.
 * bandred_sterf: eigenvalues of the symmetric tridiagonal (d, e) (device, n and n - 1
 *   entries) into lam (device, n, ascending), by trisection on Sturm counts (two lanes per
 *   eigenvalue; a first pass on an FP32 copy of T narrows each bracket, widened well past
 *   its roundoff before the FP64 rounds) to within a few units in the last place of
 *   max |T|.  work: device,
 *   256-byte aligned, >= bandred_sterf_workspace(n) bytes.  Returns 0, -i for an invalid i-th argument.
 */
size_t bandred_sb2st_workspace(int64_t n, int64_t w);
int bandred_sb2st(int64_t n, int64_t w, const double* A, int64_t lda, double* d, double* e,
                  const bandred_opts* opts, void* work, size_t work_bytes, int* dev_status, cudaStream_t stream);
size_t bandred_sterf_workspace(int64_t n);
int bandred_sterf(int64_t n, const double* d, const double* e, double* lam, void* work, size_t work_bytes,
                  cudaStream_t stream);

/* ---------------------------------------------------------------- SVD second stage -----
 * The paper's introduction: for the SVD the compact form is an upper triangular-band
 * matrix with upper bandwidth w (ge2gb's result), which a second stage reduces to
 * bidiagonal form before the singular values are computed.
 *
 * bandred_gb2bd: upper band -> upper bidiagonal by Householder bulge chasing.  A (device,
 *   column-major, lda >= n) holds the band in its upper n x n triangle (entries with
 *   0 <= j - i <= w are read, nothing else: a packed ge2gb result with m >= n goes in
 *   unchanged).  Sweep c (c = 0 .. n-2) alternates a right reflector, which annihilates a
 *   row past its first entry over a column range [a, a+w), and a left reflector, which
 *   annihilates column a below its diagonal, on ranges that move down by w (larfg
 *   convention); the bulges' other rows and columns are taken by the sweeps that follow.
 *   On exit d (device, n) holds the diagonal and e (device, n - 1) the superdiagonal of
 *   B = U^T A V.  1 <= w <= 128.  opts: only timeout_ms is used (NULL: defaults).  work:
 *   device, 256-byte aligned, >= bandred_gb2bd_workspace(n, w) bytes (the band with room
 *   for the bulges, 3 w n doubles, and per-sweep progress counters).  dev_status: as for
 *   bandred_sy2sb_ex (BANDRED_DEV_TIMEOUT when a sweep's bounded wait for the previous
 *   sweep gave up).  Returns 0, -i for an invalid i-th argument, BANDRED_ERR_UNSUPPORTED
 *   for w > 128, or a CUDA error code.
 * bandred_bdsv: singular values of the upper bidiagonal (d, e) (device, n and n - 1
 *   entries) into sigma (device, n, descending): the n largest eigenvalues of its
 *   Golub-Kahan tridiagonal (order 2n, zero diagonal, off-diagonal d_0, e_0, d_1, ..), by
 *   the trisection of bandred_sterf, to within a few units in the last place of max |B|.
 *   work: device, 256-byte aligned, >= bandred_bdsv_workspace(n) bytes.  Returns 0, -i
 *   for an invalid i-th argument, or a CUDA error code.
 */
size_t bandred_gb2bd_workspace(int64_t n, int64_t w);
int bandred_gb2bd(int64_t n, int64_t w, const double* A, int64_t lda, double* d, double* e,
                  const bandred_opts* opts, void* work, size_t work_bytes, int* dev_status, cudaStream_t stream);
size_t bandred_bdsv_workspace(int64_t n);
int bandred_bdsv(int64_t n, const double* d, const double* e, double* sigma, void* work, size_t work_bytes,
                 cudaStream_t stream);

/* ---------------------------------------------------------------- forming Q, U, V ---
 * The orthogonal factors of a finished reduction, formed on the GPU from the packed
 * reflectors (the step that eigenvector and singular-vector solvers take after the band
 * reduction; the paper's introduction).  The reflectors are applied in groups of b
 * (opts->b, 0 = 64, at most 64) in compact-WY form (Section 4.1), last group first; the
 * products run in FP64 for BANDRED_FP64 and as Ozaki-scheme products (FP64-accurate, on the
 * tensor cores) for any other precision.  Q is N x N, column-major, ldq >= max(1, N),
 * device memory owned by the caller and overwritten; A and tau are the outputs of the
 * reduction and are not changed.  work: device, 256-byte aligned, at least
 * bandred_form_workspace(N, opts) bytes.  Stream-ordered; no allocation.  Returns 0, -i
 * for an invalid i-th argument, or a BANDRED_ERR_* code; dev_status as for the reductions.
 *   bandred_sy2sb_form_q: Q of A = Q B Q^T (N = n).
 *   bandred_ge2gb_form:   side 0: U of A = U B V^T (N = m; for m < n the Q of A = Q B P^T);
 *                         side 1: V (N = n; for m < n the P).  tau: tauq for side 0, taup
 *                         for side 1, as the reduction wrote them.
 */
size_t bandred_form_workspace(int64_t N, const bandred_opts* opts);
int bandred_sy2sb_form_q(int64_t n, int64_t w, const double* A, int64_t lda, const double* tau, double* Q,
                         int64_t ldq, const bandred_opts* opts, void* work, size_t work_bytes, int* dev_status,
                         cudaStream_t stream);
int bandred_ge2gb_form(int64_t m, int64_t n, int64_t w, const double* A, int64_t lda, const double* tau, int side,
                       double* Q, int64_t ldq, const bandred_opts* opts, void* work, size_t work_bytes,
                       int* dev_status, cudaStream_t stream);
/*   bandred_ge2bb_form:   side 0: U (N = m), side 1: V (N = n) of a finished ge2bb. */
int bandred_ge2bb_form(int64_t m, int64_t n, int64_t w, const double* A, int64_t lda, const double* tau, int side,
                       double* Q, int64_t ldq, const bandred_opts* opts, void* work, size_t work_bytes,
                       int* dev_status, cudaStream_t stream);

/* ---------------------------------------------------------------- batched -----------
 * Many independent matrices of uneven sizes (Sections 2.1 and 3.1 applied to each).
 * The matrices advance in lockstep: iteration t of every matrix still active runs in the
 * same kernel launches (one thread-block cluster per panel, batched split-precision
 * products), matrices ordered by their number of iterations.  Split precision only
 * (BANDRED_BF16X3 or BANDRED_BF16X6); opts->b is the panel width (0: min(w, 32), clamped
 * to each matrix's w).
 *   count         number of matrices
 *   n, w (m)      host arrays of sizes (ge2gb: m[q] >= n[q])
 *   A, tau(q/p)   host arrays of DEVICE pointers (column-major FP64 matrices, lda[q];
 *                 lda == NULL means lda[q] = n[q] (sy2sb) or m[q] (ge2gb))
 *   work          device, 256-byte aligned, >= the _workspace bytes, one per batch shape
 * _plan builds the launch schedule for these sizes and pointers, writes its parameter
 * tables into `work` (one host-to-device copy) and clears the tau arrays; it is not
 * capturable.  _run issues the schedule's kernel launches and memsets only (no
 * allocation, no synchronisation, no host copy), so it can be captured in a CUDA graph
 * and replayed; call it with the same arguments as the last _plan on this workspace.
 * dev_status (device int, may be NULL) receives the BANDRED_DEV_* code of the run.
 * Outputs per matrix: the packed layouts of bandred_sy2sb / bandred_ge2gb. */
size_t bandred_sy2sb_batched_workspace(int count, const int64_t* n, const int64_t* w, const bandred_opts* opts);
int bandred_sy2sb_batched_plan(int count, const int64_t* n, const int64_t* w, double* const* A,
                               const int64_t* lda, double* const* tau, const bandred_opts* opts,
                               void* work, size_t work_bytes, cudaStream_t stream);
int bandred_sy2sb_batched_run(int count, const int64_t* n, const int64_t* w, double* const* A,
                              const int64_t* lda, double* const* tau, const bandred_opts* opts,
                              void* work, size_t work_bytes, int* dev_status, cudaStream_t stream);
size_t bandred_ge2gb_batched_workspace(int count, const int64_t* m, const int64_t* n, const int64_t* w,
                                       const bandred_opts* opts);
int bandred_ge2gb_batched_plan(int count, const int64_t* m, const int64_t* n, const int64_t* w,
                               double* const* A, const int64_t* lda, double* const* tauq,
                               double* const* taup, const bandred_opts* opts, void* work,
                               size_t work_bytes, cudaStream_t stream);
int bandred_ge2gb_batched_run(int count, const int64_t* m, const int64_t* n, const int64_t* w,
                              double* const* A, const int64_t* lda, double* const* tauq,
                              double* const* taup, const bandred_opts* opts, void* work,
                              size_t work_bytes, int* dev_status, cudaStream_t stream);

/* ---------------------------------------------------------------- split-precision engine
 * The tensor-core products of the trailing updates, usable on their own.  FP64 operands
 * are cut into bf16 slices (x ~ s0 + s1 [+ s2]; s0 keeps the leading 8 bits); the slice
 * products of order < S (precision BANDRED_BF16X3: S = 2, three products; BANDRED_BF16X6:
 * S = 3, six products) run as tcgen05.mma with FP32 accumulation in tensor memory and are
 * recombined in FP64 every 256 reduction steps.  Accuracy is FP32-class (about 1e-5
 * relative for BF16X3 and 1e-6 for BF16X6, relative to sum_k |a_ik||b_kj|).  Entries must
 * be zero or lie in 2^-95 <= |x| < 2^127; otherwise dev_status reports BANDRED_DEV_RANGE.
 * BANDRED_OZAKI takes any finite entries and is accurate to about 2^-56 of
 * max_k |a_ik| max_k |b_kj| per term (FP64-class).
 * Arguments are device pointers (column-major FP64) except sizes; work is a device
 * buffer (256-byte aligned) of at least the queried size.  No allocation, stream-ordered.
 */

/* C (m x n) = op(A) B with op(A) = A (m x k, lda >= m) or A^T (A is k x m, lda >= k when
 * transA != 0); B is k x n (ldb >= k); 1 <= n <= 128.  Used for X1 = A2 W
 * (Eq. updateA2symm) and the products with W of Eqs. updateA1, updateCD and updateD. */
size_t bandred_gemm_split_workspace(int64_t m, int64_t n, int64_t k, int precision);
int bandred_gemm_split(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, int transA,
                       const double* B, int64_t ldb, double* C, int64_t ldc, int precision,
                       void* work, size_t work_bytes, int* dev_status, cudaStream_t stream);

/* Lower triangle of C (n x n) += X Y^T + Y X^T for X, Y (n x kb, 1 <= kb <= 128): the
 * rank-2k update of Eq. updateA2syr2k.  The strictly upper triangle is not accessed. */
size_t bandred_syr2k_split_workspace(int64_t n, int64_t kb, int precision);
int bandred_syr2k_split(int64_t n, int64_t kb, const double* X, int64_t ldx, const double* Y,
                        int64_t ldy, double* C, int64_t ldc, int precision, void* work,
                        size_t work_bytes, int* dev_status, cudaStream_t stream);

/* ---------------------------------------------------------------- tracing -----------
 * Per-kernel-class timing.  Between bandred_profile_begin() and bandred_profile_end()
 * every kernel group the library launches is bracketed by a pair of CUDA events on its
 * stream.  bandred_profile_end synchronises those events and writes one entry per kernel
 * class that ran (at most max_entries): launches, summed event time, and the algorithmic
 * flops and HBM bytes of those launches (the counts of the method, not of the hardware).
 * Returns the number of entries written or a negative code.  Host-side, not thread-safe
 * with concurrent calls on other threads.
 */
typedef struct bandred_kernel_stat {
    char name[32];
    long long launches;
    double ms;
    double flops;
    double bytes;
} bandred_kernel_stat;

int bandred_profile_begin(void);
int bandred_profile_end(bandred_kernel_stat* out, int max_entries);

/* Number of kernel launches the library has issued since it was loaded. */
long long bandred_launch_count(void);

/* Device trace of the look-ahead timeline (Section 2.2's overlap, observed on the GPU).
 * bandred_trace_begin(buf, bytes): buf is a device buffer (256-byte aligned) of 16 bytes
 * per record; it synchronises the device, fills buf and arms the trace.  Until
 * bandred_trace_end, every traced kernel launch of the reductions (the panels, the two
 * halves of the rank-2k update of the Ozaki path, the X1 = A2 W product of the Ozaki
 * path) takes one record, in launch order, and its CTAs store the earliest start and the
 * latest end of the launch, read from the GPU's globaltimer (ns).  bandred_trace_end
 * synchronises the device, copies up to max_records records into out and disarms the
 * trace; it returns the number written, or a negative code.  kind: 0 panel (QR of a
 * column panel), 1 rank-2k update of the next panel's columns (A2^L), 2 rank-2k update
 * of the rest (A2^R, or all of A2 without look-ahead), 3 X1 = A2 W, 4 row panel (LQ),
 * 5 left update (ge2gb), 6 right update (ge2gb), 7 W = -Y T formed after a panel
 * (iteration 0); iteration = the panel's first column.
 * Host-side, one trace at a time per process; a diagnostic, not for the hot path. */
typedef struct bandred_trace_record {
    int kind;
    long long iteration;
    unsigned long long t0_ns, t1_ns;
} bandred_trace_record;
int bandred_trace_begin(void* buf, size_t bytes);
int bandred_trace_end(bandred_trace_record* out, int max_records);

/* Phase timing of one panel (a diagnostic of the panel's latency).  Arms the next panel
 * factorisation that runs as a cooperative grid (every panel of the single-matrix
 * reductions with the default pairs of reflectors): its CTA 0 writes the SM clock (clock64) at 8 points of
 * each step into buf[8 step + q], for steps < max_steps: q = 0 step start, 1 dot products
 * summed, 2 arrival at the grid barrier, 3 barrier passed, 4 reflectors derived, 5 the
 * in-panel update done, 6 step end.  buf: device, 8 * max_steps int64 (slots not written
 * keep their contents).  One panel per call; returns 0 or a negative code. */
int bandred_panel_phase_trace(void* buf, int max_steps);

/* Phase timing of the bulge chase (a diagnostic of bandred_sb2st's step latency).  Arms
 * the next bandred_sb2st with w <= 64: the CTA running sweep (n - 2) / 2 writes the SM
 * clock (clock64) at up to 16 points of each of its steps into buf[16 step + q], for
 * steps < max_steps: q = 0 step start, 1 the wait for the previous sweep passed, 2 the
 * step's blocks in shared memory, 3 the rows below's last column reloaded (thread 32),
 * 5 the reflector's vector formed and the column written, 6 the
 * one-sided blocks and the diagonal matvec done, 7 the bulge written back, K and the
 * next step's reflector formed, 8 the diagonal block's rank-2 update written back, 9 the
 * step released, 10 the first half of the one-sided blocks (the dot products) done, 11 the
 * diagonal block's entries formed (slots 4 and 12-15 are not written).  buf: device,
 * 16 * max_steps int64.  One call; returns 0 or a negative code. */
int bandred_sb2st_phase_trace(void* buf, int max_steps);

/* ---------------------------------------------------------------- diagnostics -------
 * The reciprocal square root and reciprocal that the panel kernels use in place of FP64
 * square root and division when they form a reflector (Section 2.1, Eq. updateA0: beta,
 * tau and 1/(alpha - beta) of the Householder vector): an FP32 hardware estimate refined
 * by two Newton-Raphson steps in FP64.  For i < count: rsqrt[i] = 1/sqrt(x[i]) for x[i] in
 * [2^-1022, 2^1023), and rcp[i] = 1/x[i] for x[i] in [2^-1021, 2^1021] (the panels use
 * [2^-900, 2^1002) and [2^-451, 2^502]); outside those ranges the outputs are undefined.
 * x, rsqrt, rcp: device arrays of count doubles (rsqrt or rcp may be NULL).  Returns 0,
 * -i for an invalid i-th argument, or BANDRED_ERR_CUDA.  Stream-ordered, no allocation.
 */
int bandred_newton_eval(int64_t count, const double* x, double* rsqrt, double* rcp, cudaStream_t stream);

/* FP64 throughput probe: `blocks` CTAs of `threads` threads each run 8 independent chains
 * of `iters` dependent FP64 fused multiply-adds (2 flops each), then write one value per
 * thread to sink (device, blocks * threads doubles) so that no work is dropped.  The flop
 * count is 16 * blocks * threads * iters; time the launch with CUDA events on `stream`
 * to obtain the FP64 rate.  Returns 0, -i for an invalid i-th argument, or
 * BANDRED_ERR_CUDA.  No counterpart in the paper: it measures the FP64 roofline.
 */
int bandred_fp64_probe(int blocks, int threads, int iters, double* sink, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* BANDRED_H */
