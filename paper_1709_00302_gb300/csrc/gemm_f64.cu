// FP64 CUDA-core kernels of the trailing updates (the plain FP64 path):
//   gemm_f64        general product with strided operand views and optional split-K
//                   (Eq. updateA1: W^T A1 and A1 + Y Z; Eqs. updateA2gemm1/gemm2: X1^T W
//                   and X1 + Y X2; Eqs. updateCD and updateD of the general case),
//   symm_lower_f64  X1 = A2 W reading only the lower triangle of A2 (Eq. updateA2symm),
//   syr2k_lower_f64 A2 += X3 Y^T + Y X3^T on the lower triangle (Eq. updateA2syr2k).
// GB300 runs FP64 at about 1.2 TFLOP/s (two FP64 FMAs per clock per SM), so these
// kernels are bound by the FP64 pipe; 64 x 64 output tiles with a 4 x 4 register
// micro-tile per thread keep it busy with modest shared-memory traffic.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace bandred {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int PAD = 1;

// Shared tiles: As[k][i] (BK x BM) and Bs[k][j] (BK x BN).
struct Tiles {
  double a[BK][BM + PAD];
  double b[BK][BN + PAD];
};

// ---- operand loaders ------------------------------------------------------------
struct ViewA {  // op(A)(i, k) = p[i * rs + k * cs], M x K
  const double* p;
  int64_t rs, cs;
  int M, K;
  __device__ void load(Tiles& t, int i0, int k0, int tid) const {
    if (rs == 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int ii = tid % BM, kk = tid / BM + 4 * q;
        const int i = i0 + ii, k = k0 + kk;
        t.a[kk][ii] = (i < M && k < K) ? p[i + (int64_t)k * cs] : 0.0;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int kk = tid % BK, ii = tid / BK + 16 * q;
        const int i = i0 + ii, k = k0 + kk;
        t.a[kk][ii] = (i < M && k < K) ? p[(int64_t)i * rs + (int64_t)k * cs] : 0.0;
      }
    }
  }
};

struct ViewB {  // op(B)(k, j) = p[k * rs + j * cs], K x N
  const double* p;
  int64_t rs, cs;
  int K, N;
  __device__ void load(Tiles& t, int k0, int j0, int tid) const {
    if (rs == 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int kk = tid % BK, jj = tid / BK + 16 * q;
        const int k = k0 + kk, j = j0 + jj;
        t.b[kk][jj] = (k < K && j < N) ? p[k + (int64_t)j * cs] : 0.0;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int jj = tid % BN, kk = tid / BN + 4 * q;
        const int k = k0 + kk, j = j0 + jj;
        t.b[kk][jj] = (k < K && j < N) ? p[(int64_t)k * rs + (int64_t)j * cs] : 0.0;
      }
    }
  }
};

// Symmetric n x n matrix from its lower triangle (column-major): S(i, k).
struct SymLowerA {
  const double* p;
  int64_t ld;
  int n;
  __device__ void load(Tiles& t, int i0, int k0, int tid) const {
    if (i0 >= k0 + BK - 1) {  // whole tile in the lower triangle: column-major reads
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int ii = tid % BM, kk = tid / BM + 4 * q;
        const int i = i0 + ii, k = k0 + kk;
        t.a[kk][ii] = (i < n && k < n) ? p[i + (int64_t)k * ld] : 0.0;
      }
    } else if (i0 + BM - 1 < k0) {  // whole tile in the upper triangle: read the mirror
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int kk = tid % BK, ii = tid / BK + 16 * q;
        const int i = i0 + ii, k = k0 + kk;
        t.a[kk][ii] = (i < n && k < n) ? p[k + (int64_t)i * ld] : 0.0;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int ii = tid % BM, kk = tid / BM + 4 * q;
        const int i = i0 + ii, k = k0 + kk;
        double v = 0.0;
        if (i < n && k < n) v = (i >= k) ? p[i + (int64_t)k * ld] : p[k + (int64_t)i * ld];
        t.a[kk][ii] = v;
      }
    }
  }
};

// [X | Y] (n x 2nb) rows, and [Y | X]^T (2nb x n) columns, for the rank-2nb update.
struct ConcatA {
  const double *X, *Y;
  int64_t ldx, ldy;
  int n, nb;
  __device__ void load(Tiles& t, int i0, int k0, int tid) const {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ii = tid % BM, kk = tid / BM + 4 * q;
      const int i = i0 + ii, k = k0 + kk;
      double v = 0.0;
      if (i < n && k < 2 * nb) v = (k < nb) ? X[i + (int64_t)k * ldx] : Y[i + (int64_t)(k - nb) * ldy];
      t.a[kk][ii] = v;
    }
  }
};
struct ConcatBT {
  const double *X, *Y;
  int64_t ldx, ldy;
  int n, nb;
  __device__ void load(Tiles& t, int k0, int j0, int tid) const {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int jj = tid % BN, kk = tid / BN + 4 * q;
      const int j = j0 + jj, k = k0 + kk;
      double v = 0.0;
      if (j < n && k < 2 * nb) v = (k < nb) ? Y[j + (int64_t)k * ldy] : X[j + (int64_t)(k - nb) * ldx];
      t.b[kk][jj] = v;
    }
  }
};

template <class LA, class LB>
__device__ __forceinline__ void tile_product(Tiles& t, const LA& la, const LB& lb, int i0, int j0, int kbeg,
                                             int kend, double (&acc)[4][4]) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    la.load(t, i0, k0, tid);
    lb.load(t, k0, j0, tid);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = t.a[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = t.b[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(NT) gemm_kernel(int M, int N, int K, double alpha, ViewA la, ViewB lb,
                                                  double beta, double* C, int64_t ldc, int kchunk,
                                                  double* partial) {
  __shared__ Tiles t;
  const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  double acc[4][4];
  tile_product(t, la, lb, i0, j0, kbeg, kend, acc);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  if (partial) {
    double* P = partial + (size_t)blockIdx.z * M * N;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = i0 + tx + 16 * a, j = j0 + ty + 16 * b;
        if (i < M && j < N) P[i + (size_t)j * M] = acc[a][b];
      }
    return;
  }
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = i0 + tx + 16 * a, j = j0 + ty + 16 * b;
      if (i < M && j < N) {
        double* c = &C[i + (int64_t)j * ldc];
        *c = (beta == 0.0) ? alpha * acc[a][b] : fma(alpha, acc[a][b], beta * *c);
      }
    }
}

__global__ void splitk_reduce_kernel(int M, int N, int splits, double alpha, const double* partial, double beta,
                                     double* C, int64_t ldc) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += partial[(size_t)z * total + e];
    const int i = (int)(e % M), j = (int)(e / M);
    double* c = &C[i + (int64_t)j * ldc];
    *c = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * *c);
  }
}

__global__ void __launch_bounds__(NT) symm_kernel(int n, int nb, SymLowerA la, ViewB lb, double* X, int64_t ldx) {
  __shared__ Tiles t;
  const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
  double acc[4][4];
  tile_product(t, la, lb, i0, j0, 0, n, acc);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = i0 + tx + 16 * a, j = j0 + ty + 16 * b;
      if (i < n && j < nb) X[i + (int64_t)j * ldx] = acc[a][b];
    }
}

__global__ void __launch_bounds__(NT) syr2k_kernel(int n, int nb, double* S, int64_t lds, ConcatA la, ConcatBT lb,
                                                   int tj0, int col0, int col1) {
  const int I = blockIdx.x, J = tj0 + blockIdx.y;
  if (I < J) return;  // strictly upper tile
  __shared__ Tiles t;
  const int i0 = I * BM, j0 = J * BN;
  double acc[4][4];
  tile_product(t, la, lb, i0, j0, 0, 2 * nb, acc);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = i0 + tx + 16 * a, j = j0 + ty + 16 * b;
      if (i < n && j < col1 && j >= col0 && i >= j) S[i + (int64_t)j * lds] += acc[a][b];
    }
}

}  // namespace

cudaError_t gemm_f64(int M, int N, int K, double alpha, MatView a, MatView b, double beta, double* C,
                     int64_t ldc, int splits, double* partial, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K <= 0) splits = 1;
  if (splits < 1) splits = 1;
  int kchunk = (K + splits - 1) / splits;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  if (kchunk < BK) kchunk = BK;
  splits = (K + kchunk - 1) / kchunk;
  if (splits < 1) splits = 1;
  ViewA la{a.p, a.rs, a.cs, M, K};
  ViewB lb{b.p, b.rs, b.cs, K, N};
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, splits);
  if (splits == 1) {
    gemm_kernel<<<grid, NT, 0, s>>>(M, N, K, alpha, la, lb, beta, C, ldc, kchunk, nullptr);
    prof::count_launch();
    return cudaGetLastError();
  }
  gemm_kernel<<<grid, NT, 0, s>>>(M, N, K, alpha, la, lb, beta, C, ldc, kchunk, partial);
  prof::count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)M * N;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 1184);
  splitk_reduce_kernel<<<blocks, 256, 0, s>>>(M, N, splits, alpha, partial, beta, C, ldc);
  prof::count_launch();
  return cudaGetLastError();
}

cudaError_t symm_lower_f64(int n, int nb, const double* S, int64_t lds, const double* W, int64_t ldw, double* X,
                           int64_t ldx, cudaStream_t s) {
  if (n <= 0 || nb <= 0) return cudaSuccess;
  SymLowerA la{S, lds, n};
  ViewB lb{W, 1, ldw, n, nb};
  dim3 grid((n + BM - 1) / BM, (nb + BN - 1) / BN);
  symm_kernel<<<grid, NT, 0, s>>>(n, nb, la, lb, X, ldx);
  prof::count_launch();
  return cudaGetLastError();
}

cudaError_t syr2k_lower_f64(int n, int nb, double* S, int64_t lds, const double* X, int64_t ldx, const double* Y,
                            int64_t ldy, int col0, int col1, cudaStream_t s) {
  if (col1 > n) col1 = n;
  if (n <= 0 || nb <= 0 || col0 >= col1) return cudaSuccess;
  ConcatA la{X, Y, ldx, ldy, n, nb};
  ConcatBT lb{X, Y, ldx, ldy, n, nb};
  const int T = (n + BM - 1) / BM;
  const int tj0 = col0 / BN, tj1 = (col1 - 1) / BN;
  dim3 grid(T, tj1 - tj0 + 1);
  syr2k_kernel<<<grid, NT, 0, s>>>(n, nb, S, lds, la, lb, tj0, col0, col1);
  prof::count_launch();
  return cudaGetLastError();
}

namespace {

// D (cols x rows) = S^T for S (rows x cols): 32 x 32 tiles through shared memory (one
// padding column against bank conflicts), reads and writes coalesced along columns.
__global__ void transpose_kernel(int rows, int cols, const double* S, int64_t lds, double* D, int64_t ldd) {
  __shared__ double tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int r = r0 + threadIdx.x, c = c0 + q;
    if (r < rows && c < cols) tile[q][threadIdx.x] = S[r + (int64_t)c * lds];
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int c = c0 + threadIdx.x, r = r0 + q;
    if (r < rows && c < cols) D[c + (int64_t)r * ldd] = tile[threadIdx.x][q];
  }
}

}  // namespace

cudaError_t transpose_f64(int rows, int cols, const double* S, int64_t lds, double* D, int64_t ldd, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const dim3 grid((rows + 31) / 32, (cols + 31) / 32);
  prof::count_launch();
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(rows, cols, S, lds, D, ldd);
  return cudaGetLastError();
}

}  // namespace bandred
