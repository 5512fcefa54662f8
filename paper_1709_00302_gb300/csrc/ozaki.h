// FP64-accurate products on the BF16 tensor cores (the Ozaki scheme): every row of an
// operand is scaled by a power of two bound to its largest entry and cut into S signed
// 8-bit digits held exactly in bf16; digit-pair products are exact in the FP32 tensor
// accumulators (sums of at most 128 reduction steps stay below 2^24), summed per digit
// diagonal into 64-bit integers, and combined into FP64 at the end, so the only errors
// are the dropped digit pairs (below 2^-56 of the row and column scales) and the final
// rounding.  Used by precision BANDRED_OZAKI for every trailing-update product.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace bandred {
namespace ozaki {

constexpr int kDigits = 7;   // S: 56 bits of each row-scaled entry
constexpr int kTileA = 128;  // rows of an A tile (TMEM lanes)
constexpr int kTileB = 64;   // rows of a B tile (columns of C)
constexpr int kDepth = 16;   // reduction depth of one packed block (one pipeline stage)

// An operand op(X) with rows r and reduction index k, possibly two matrices side by side
// along k (k < K1 from M1, then M2).  mode: 0 = M[r + k ld], 1 = M[k + r ld], 2 = symmetric
// with the lower triangle stored (R == K; only for a single source).
// With `sh` set (two sources), the entries of M1 are taken times 2^(-shsign sigma) and those
// of M2 times 2^(+shsign sigma), sigma = floor((sh[0] - sh[1]) / 2) from the largest biased
// exponents sh[0], sh[1] that `balance` writes (sigma = 0 when either source is zero).  A
// product of two such operands with opposite shsign is unchanged, and the two halves of
// every row meet near the same magnitude, so neither is lost below the row's scale.
struct Operand {
  const double* M1;
  int64_t ld1;
  int mode1, K1;
  const double* M2;
  int64_t ld2;
  int mode2, K2;
  int R;
  const int* sh = nullptr;
  int shsign = 0;
};

// sh[0], sh[1] = the largest biased exponents of the two sources of op (0 for a zero source).
cudaError_t balance(const Operand& op, int* sh, cudaStream_t s);

// Largest biased FP64 exponent of every row of op (0 for a zero row) into e[0..R).
cudaError_t row_exponents(const Operand& op, int* e, cudaStream_t s);

// Digits of op, rows scaled by 2^-(e_r - 1021), into blocks of TR rows x kDepth (TR = kTileA
// for the left operand, kTileB for the right one): block (rb, kb) holds the kDigits planes
// stacked along the rows, one (kDigits TR) x kDepth bf16 operand in the canonical K-major
// layout of tcgen05 (plane s = rows s TR .. s TR + TR - 1).
size_t packed_bytes(int R, int K, int TR);
cudaError_t pack(const Operand& op, const int* e, int TR, __nv_bfloat16* out, cudaStream_t s);

struct GemmParams {
  const __nv_bfloat16* A;  // packed left operand, M rows (TR = kTileA)
  const __nv_bfloat16* B;  // packed right operand, N rows (TR = kTileB)
  const int* eA;           // row exponents of A and of B
  const int* eB;
  int M, N, nkb;           // C is M x N; K = nkb * kDepth (zero-padded)
  int kb_per_split;        // reduction blocks per CTA along gridDim.z
  // partial mode (P != nullptr): exact 64-bit digit sums of split z at
  //   Phi[z * sstride + i + j * ldp], Plo[...]
  int64_t* Phi;
  int64_t* Plo;
  int64_t ldp, sstride;
  // direct mode: C(i, j) += alpha * (A B^T)(i, j) for col0 <= j < col1 (and i >= j if lower)
  double* C;
  int64_t ldc;
  int col0, col1, lower;
  double alpha;
  int* status;
  unsigned long long limit_ns;
  unsigned long long* trace;  // device trace record of this launch, or nullptr
};
cudaError_t gemm(const GemmParams& p, int splits, cudaStream_t s);

// C = alpha * sum of the splits' partials + beta * C (M x N, column-major).
cudaError_t reduce(const GemmParams& p, int splits, double alpha, double beta, double* C, int64_t ldc,
                   cudaStream_t s);

// Whole products on top of the kernels above.  Workspace: row exponents, both packed
// operands and the split partials, carved by `carve` from `bytes(M, N, K, splits)`.
struct Bufs {
  int* eA;
  int* eB;
  __nv_bfloat16* Ablob;
  __nv_bfloat16* Bblob;
  int64_t* P;  // 2 * splits * M * N
  // eB and Bblob already hold the right operand's exponents and digits (an earlier product
  // with the same right operand packed them there): not computed again
  bool b_packed = false;
};
int choose_splits(int M, int N, int K, int sms);
size_t bytes(int M, int N, int K, int splits, bool partials = true);
Bufs carve(void* base, int M, int N, int K, int splits);
// The largest split count <= want whose buffers for (M, N, K) fit in cap bytes (>= 1).
int fit_splits(int M, int N, int K, int want, size_t cap);

// C (M x N) = alpha opA opB^T + beta C, K the common reduction length (rows of opB are
// the columns of C).
cudaError_t product(const Operand& A, const Operand& B, int M, int N, int K, double alpha, double beta, double* C,
                    int64_t ldc, const Bufs& b, int splits, int* status, unsigned long long limit_ns,
                    cudaStream_t s);
// Row exponents and digits of both operands into b (for rank_apply; products pack their
// own operands).  When b.eB == b.eA the caller states that every row of B holds the same
// entries as that row of A (in another order), and B's exponents are not computed again.
cudaError_t prepare(const Operand& A, const Operand& B, const Bufs& b, cudaStream_t s);
// C += alpha opA opB^T on columns [col0, col1) (and the lower triangle when `lower`), from
// operands packed by prepare (several calls, on any streams, may share them).  One
// persistent CTA per SM, or at most max_ctas CTAs (> 0), so that another kernel can hold
// the remaining SMs at the same time.
cudaError_t rank_apply(int M, int N, int K, double alpha, double* C, int64_t ldc, int col0, int col1, int lower,
                       const Bufs& b, int* status, unsigned long long limit_ns, cudaStream_t s, int max_ctas = 0);

}  // namespace ozaki
}  // namespace bandred
