// Internal launch interface of the band-reduction kernels (not part of the C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace bandred {

struct GridSync;

// ---------------------------------------------------------------- panel (panel.cu)
struct PanelParams {
  double* A;             // panel element (r, c) at A[r * rs + c * cs]
  int64_t rs, cs;
  int j, bk;             // rows (length of reflector 0) and number of reflectors
  int R, Rp;             // rows per CTA and the shared-memory stride (odd, >= R)
  double* tau;           // bk outputs
  double* Y;             // j x bk, column-major, ld = ldy (unit lower trapezoidal copy of V)
  double* W;             // j x bk, column-major, ld = ldy (W = -Y T)
  int64_t ldy;
  double* acc;           // 3 * panel_acc_entries(bk) * 32 doubles, directly after *gs (zeroed with it)
  double* rowbuf;        // 8 * bk doubles
  GridSync* gs;
  int* status;
  unsigned long long limit_ns;
  unsigned int extra;    // extra awaited arrivals (tests of the timeout path)
  bool w_in_smem;        // this CTA's rows of W kept in shared memory during the panel
  bool w_fp32;           // W formed in FP32 (it only feeds split-precision products)
  unsigned long long* trace;  // device trace record of this launch, or nullptr
  long long* phases;          // grid panel only: clock64 of CTA 0 at 8 points of each step, or nullptr
  int phase_steps;            // steps that fit in phases
  double* G;                  // grid panel, FP64 W: the strict upper triangle of Y^T Y (bk x bk, ld bk)
                              // written instead of W, which w_from_gram then forms (nullptr: W in the panel)
};

// W = -Y T for a factored panel from its Gram coefficients: row r of W solves the forward
// substitution w_r[q] = -tau_q (Y(r, q) + sum_{p<q} w_r[p] G(p, q)) (T^{-1} = strict upper of
// Y^T Y + diag(1 / tau)).  j rows, bk columns, Y and W with leading dimension ldy.
cudaError_t launch_w_from_gram(int j, int bk, const double* Y, const double* tau, const double* G, double* W,
                               int64_t ldy, cudaStream_t s);

// Tn = -T (bk x bk, ld bk, zero below the diagonal) of a factored panel from the same Gram
// coefficients and tau (bk <= 128): W = -Y T = Y Tn is then one product of Y and Tn.
cudaError_t launch_t_from_gram(int bk, const double* tau, const double* G, double* Tn, cudaStream_t s);

size_t panel_smem_bytes(int bk, int Rp, bool w_in_smem);
size_t panel_sync_bytes(int bk);  // bytes from gs to the end of acc
int panel_geometry(int j, int bk, int max_ctas, int min_rows, int* G, int* R, int* Rp, bool* w_in_smem);
cudaError_t launch_panel(const PanelParams& p, int G, cudaStream_t s);
// The same factorisation with up to four reflectors per grid-wide reduction (panel4.cu):
// same parameters, geometry and outputs; its shared memory is panel4_smem_bytes.
size_t panel4_smem_bytes(int bk, int Rp, bool w_in_smem);
cudaError_t launch_panel4(const PanelParams& p, int G, cudaStream_t s);

// One thread-block cluster of C CTAs per panel (panel_cluster.cu).  `single` (host
// struct) or `dev_probs` (device array of nprob structs, inactive when bk == 0) gives the
// problems; each uses rows-per-CTA R = p.R and stride p.Rp <= Rp_max, bk <= bk_max.
size_t panel_cluster_smem_bytes(int bk, int Rp);
int panel_cluster_rows(int j, int bk, int C);
cudaError_t launch_panel_cluster(const PanelParams* single, const PanelParams* dev_probs, int nprob, int C, int Rp_max,
                                 int bk_max, cudaStream_t s);

// ---------------------------------------------------------------- FP64 kernels (gemm_f64.cu)
// A strided matrix view: element (i, k) at p[i * rs + k * cs].
struct MatView {
  const double* p;
  int64_t rs, cs;
};

// C (M x N, column-major, ldc) = alpha * op(A) op(B) + beta * C, where op(A) is the M x K
// view `a` and op(B) the K x N view `b`.  When splits > 1 the K range is cut into
// `splits` pieces whose partial products go to `partial` (splits * M * N doubles) and
// are summed in a fixed order by a second kernel.
cudaError_t gemm_f64(int M, int N, int K, double alpha, MatView a, MatView b, double beta, double* C,
                     int64_t ldc, int splits, double* partial, cudaStream_t s);

// X (n x nb) = S W for symmetric S (n x n) of which only the lower triangle (column-major,
// lds) is read, and W (n x nb, column-major, ldw).
cudaError_t symm_lower_f64(int n, int nb, const double* S, int64_t lds, const double* W, int64_t ldw, double* X,
                           int64_t ldx, cudaStream_t s);

// Lower triangle of S (n x n) += X Y^T + Y X^T for X, Y (n x nb, column-major).  The
// column range [col0, col1) of S is updated (used to split the update around the next
// panel for look-ahead); rows run over the whole lower part of those columns.
cudaError_t syr2k_lower_f64(int n, int nb, double* S, int64_t lds, const double* X, int64_t ldx, const double* Y,
                            int64_t ldy, int col0, int col1, cudaStream_t s);

// D (cols x rows, column-major, ldd) = S^T for S (rows x cols, column-major, lds).
cudaError_t transpose_f64(int rows, int cols, const double* S, int64_t lds, double* D, int64_t ldd, cudaStream_t s);

}  // namespace bandred
