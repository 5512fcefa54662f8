// Launch interface of the split-precision tensor-core kernels (split.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>  // CUtensorMap (type only)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace bandred {
namespace split {

// TMA descriptor of an FP64 column-major rows x cols matrix (leading dimension ld) read in
// boxes of box0 (along the rows) x box1, 128-byte swizzled when `swz`; false when the
// driver's encoder is unavailable or rejects the layout (the caller then takes a path
// without TMA).
bool encode_tile_map_f64(CUtensorMap* m, const double* base, int64_t rows, int64_t cols, int64_t ld, uint32_t box0,
                         uint32_t box1, bool swz);

// Streamed operand access modes: element (i, k) of A is
//   kModePlain     A[i + k * lda]
//   kModeTrans     A[k + i * lda]
//   kModeSymLower  i >= k ? A[i + k * lda] : A[k + i * lda]   (lower triangle stored)
enum { kModePlain = 0, kModeTrans = 1, kModeSymLower = 2 };

struct PackParams {
  const double* M1;  // element (r, k) for k < K1: t1 ? M1[k + r*ld1] : M1[r + k*ld1]
  int64_t ld1;
  int K1;
  int t1;
  const double* M2;  // element (r, K1 + k) for k < K2, same convention
  int64_t ld2;
  int K2;
  int t2;
  double scale1, scale2;  // multiply the entries of M1 / M2
  int R;                  // rows of the operand (its M or N dimension)
  int TR, TK;             // tile rows and tile depth (multiples of 8 and 16)
  int nrb, nkb;           // tiles along rows and along K
  int S;                  // slices written (2 or 3)
  __nv_bfloat16* out;
  int* status;
};

struct StreamParams {
  const double* A;
  int64_t lda;
  int mode;
  int M, K, N;                  // C is M x N; reduction length K
  const __nv_bfloat16* Bblob;   // B packed with TR = stream_bn(N), TK = 32
  int nkb;                      // ceil(K / 32)
  int stages_per_split;
  double* P;                    // partial products: P[z * split_stride + i + c * ldp]
  int64_t ldp, split_stride;
  int* status;
  unsigned long long limit_ns;
};

struct RankParams {
  const __nv_bfloat16* Ablob;  // packed with TR = 128, TK = 64, K = Kr
  const __nv_bfloat16* Bblob;
  int Kr;                      // multiple of 64
  double* C;
  int64_t ldc;
  int M, N;
  int col0, col1;              // only columns [col0, col1) change
  int lower;                   // only i >= j changes; tiles above the diagonal are skipped
  int tj0;                     // first column tile of the grid
  double alpha;
  int* status;
  unsigned long long limit_ns;
};

struct ReduceParams {
  int M, N, splits;
  const double* P;
  int64_t ldp, sstride;
  double alpha, beta;
  double* C;
  int64_t ldc;
};

int slices_of(int precision);
int stream_bn(int N);
size_t packed_bytes(int R, int K, int TR, int TK, int S);
cudaError_t pack(const PackParams& p, cudaStream_t s);
cudaError_t stream_gemm(const StreamParams& p, int S, int splits, cudaStream_t s);
cudaError_t reduce(int M, int N, int splits, const double* P, int64_t ldp, int64_t sstride, double alpha, double beta,
                   double* C, int64_t ldc, cudaStream_t s);
cudaError_t rank_update(const RankParams& p, int S, int tiles_i, int tiles_j, cudaStream_t s);

// Batched forms: one launch over nprob problems whose parameters are a device array (an
// entry with an empty size is skipped); grids cover the largest problem.
cudaError_t pack_batched(const PackParams* probs, int nprob, int64_t max_groups, cudaStream_t s);
cudaError_t stream_gemm_batched(const StreamParams* probs, int nprob, int S, int BN, int max_tiles, int max_splits,
                                cudaStream_t s);
cudaError_t reduce_batched(const ReduceParams* probs, int nprob, int64_t max_total, cudaStream_t s);
cudaError_t rank_update_batched(const RankParams* probs, int nprob, int S, int max_ti, int max_tj, cudaStream_t s);

}  // namespace split
}  // namespace bandred
