// FP64-accurate products on BF16 tensor cores (Ozaki scheme); see ozaki.h.
//
// Digits.  A row r with largest biased exponent E_r is scaled by 2^-(E_r - 1021), so
// every entry x has |x| 2^-(E_r - 1021) < 1/2 and F = round(x 2^(56 - (E_r - 1021))) is an
// integer with |F| < 2^55.  F is written as S = 7 balanced base-256 digits
// d_0 .. d_6 in [-128, 128] (d_0 most significant): x ~= 2^(E_r - 1021) sum_s d_s 2^-8(s+1).
// For C = A B^T the digit pairs (s, t) with s + t <= 6 are multiplied on the tensor cores
// (exact: |d d'| <= 2^14) and accumulated in FP32 per diagonal D = s + t in tensor memory;
// over 128 reduction steps a diagonal's sum stays below 7 * 128 * 2^14 < 2^24, so it is
// exact.  Every 128 steps the diagonals are read out as integers and added into
//   T_hi = P_0 2^16 + P_1 2^8 + P_2,   T_lo = P_3 2^24 + P_4 2^16 + P_5 2^8 + P_6,
// 64-bit integers, and at the end
//   C(i, j) = 2^(E_i - 1021) 2^(E_j - 1021) (T_hi 2^-32 + T_lo 2^-64).
// The dropped pairs (s + t >= 7) weigh at most 2^-72 of the scales per term.
#include <algorithm>
#include <cstring>

#include <cuda.h>  // CUtensorMap (type only)

#include "bandred.h"
#include "common.cuh"
#include "launch.h"
#include "ozaki.h"
#include "prof.h"
#include "split.h"
#include "tc.cuh"

namespace bandred {
namespace ozaki {

namespace {

constexpr int NT = 256;
constexpr int S = kDigits;
constexpr int kChunkBlocks = 128 / kDepth;  // 128 reduction steps per exact FP32 accumulation
constexpr int kSlots = 4;                     // pipeline stages in shared memory

__device__ __forceinline__ int biased_exp(double x) {
  return (int)(((uint32_t)__double2hiint(x) >> 20) & 0x7FFu);
}

__device__ __forceinline__ double elem(const double* M, int64_t ld, int mode, int r, int k) {
  if (mode == 0) return M[r + (int64_t)k * ld];
  if (mode == 1) return M[k + (int64_t)r * ld];
  return k <= r ? M[r + (int64_t)k * ld] : M[k + (int64_t)r * ld];
}

// ---------------------------------------------------------------- row exponents
// sigma of a balanced two-source operand (see Operand in ozaki.h)
__device__ __forceinline__ int balance_sigma(const int* sh) {
  if (!sh) return 0;
  const int a = sh[0], b = sh[1];
  return (a && b) ? (a - b) >> 1 : 0;
}

// biased exponent of x 2^shift for a nonzero x (kept >= 1), 0 for x = 0
__device__ __forceinline__ int shifted_exp(double x, int shift) {
  const int v = biased_exp(x);
  return v ? max(v + shift, 1) : 0;
}

// e[0 .. n) = 0, as a kernel of the launch chain (a memset would end the programmatic
// overlap of the kernels around it); it waits for the previous kernel, which may still
// read the array.
__global__ void zero_kernel(int* e, int n) {
  pdl_wait_and_release();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) e[i] = 0;
}

// e1[0 .. n1) = 0 and e2[0 .. n2) = 0 in one launch (both operands' exponent arrays)
__global__ void zero2_kernel(int* e1, int n1, int* e2, int n2) {
  pdl_wait_and_release();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2; i += gridDim.x * blockDim.x) {
    if (i < n1)
      e1[i] = 0;
    else
      e2[i - n1] = 0;
  }
}

// entries M[r + k ld]: one 32 x 32 tile per block (lanes along rows, eight warps of four
// columns each), row maxima combined across the warps
__global__ void rowexp_cols_kernel(const double* M, int64_t ld, int R, int K, int* e, const int* sh, int dir) {
  __shared__ int rowmax[8][32];
  pdl_wait_and_release();
  const int shift = dir * balance_sigma(sh);
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  int m = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = blockIdx.y * 32 + wy * 4 + q;
    if (i < R && k < K) m = max(m, shifted_exp(M[i + (int64_t)k * ld], shift));
  }
  rowmax[wy][lane] = m;
  __syncthreads();
  if (wy == 0) {
#pragma unroll
    for (int q = 1; q < 8; ++q) m = max(m, rowmax[q][lane]);
    if (m && i < R) atomicMax(&e[i], m);
  }
}

// both sources of a two-source operand in one launch: column blocks [0, t1) of grid.y read
// M1 (shift dir1 sigma), the rest M2 (shift dir2 sigma)
__global__ void rowexp_cols2_kernel(const double* M1, int64_t ld1, int K1, int dir1, const double* M2, int64_t ld2,
                                    int K2, int dir2, int R, int* e, const int* sh) {
  __shared__ int rowmax[8][32];
  pdl_wait_and_release();
  const int t1 = (K1 + 31) / 32;
  const bool first = (int)blockIdx.y < t1;
  const double* M = first ? M1 : M2;
  const int64_t ld = first ? ld1 : ld2;
  const int K = first ? K1 : K2, by = first ? blockIdx.y : blockIdx.y - t1;
  const int shift = (first ? dir1 : dir2) * balance_sigma(sh);
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  int m = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = by * 32 + wy * 4 + q;
    if (i < R && k < K) m = max(m, shifted_exp(M[i + (int64_t)k * ld], shift));
  }
  rowmax[wy][lane] = m;
  __syncthreads();
  if (wy == 0) {
#pragma unroll
    for (int q = 1; q < 8; ++q) m = max(m, rowmax[q][lane]);
    if (m && i < R) atomicMax(&e[i], m);
  }
}

// entries M[k + r ld] (k in [k0, k1), k > r when `upper`): one warp per row
__global__ void rowexp_rows_kernel(const double* M, int64_t ld, int R, int k0, int k1, int upper, int* e,
                                   const int* sh, int dir) {
  pdl_wait_and_release();
  const int shift = dir * balance_sigma(sh);
  const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (r >= R) return;
  const int per = (k1 - k0 + gridDim.y - 1) / gridDim.y;
  int kb = k0 + blockIdx.y * per;
  const int ke = min(k1, kb + per);
  if (upper) kb = max(kb, r + 1);
  int m = 0;
  for (int k = kb + lane; k < ke; k += 32) m = max(m, shifted_exp(M[k + (int64_t)r * ld], shift));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0 && m) atomicMax(&e[r], m);
}

// symmetric, lower triangle stored: one pass over the stored entries; each 32 x 32 tile
// (i >= k) contributes its row maxima to e[i] and its column maxima to e[k] (= row k of
// the symmetric matrix).  Block (tx, ty) = 32 x 8 threads per tile.
__global__ void rowexp_sym_kernel(const double* M, int64_t ld, int R, int* e) {
  const int ti = blockIdx.x, tk = blockIdx.y;
  if (tk > ti) return;
  pdl_wait_and_release();
  __shared__ int colmax[8][32];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int i = ti * 32 + lane;
  int rmax = 0, cm[4] = {0, 0, 0, 0};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = tk * 32 + wy * 4 + q;
    if (i < R && k < R && k <= i) {
      const int v = biased_exp(M[i + (int64_t)k * ld]);
      rmax = max(rmax, v);
      cm[q] = v;
    }
  }
  // row maxima: across the eight warps
  __shared__ int rowmax[8][32];
  rowmax[wy][lane] = rmax;
  // column maxima: across the 32 lanes of each warp, for its four columns
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int v = cm[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) colmax[wy][q] = v;
  }
  __syncthreads();
  if (wy == 0) {
    int m = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) m = max(m, rowmax[q][lane]);
    if (m && i < R) atomicMax(&e[i], m);
  } else if (wy == 1 && lane < 32) {
    const int k = tk * 32 + lane;  // column lane = (warp lane / 4, q = lane % 4)
    const int m = colmax[lane >> 2][lane & 3];
    if (m && k < R) atomicMax(&e[k], m);
  }
}

// largest biased exponent of each source of a two-source operand into sh[0], sh[1]: one
// 32 x 32 tile of source blockIdx.z per block
__global__ void maxexp_kernel(Operand op, int* sh) {
  __shared__ int wmax[8];
  pdl_wait_and_release();
  const int src = blockIdx.z;
  const double* M = src ? op.M2 : op.M1;
  const int64_t ld = src ? op.ld2 : op.ld1;
  const int mode = src ? op.mode2 : op.mode1, K = src ? op.K2 : op.K1;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  int m = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = blockIdx.y * 32 + wy * 4 + q;
    if (M && i < op.R && k < K) m = max(m, biased_exp(elem(M, ld, mode, i, k)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) wmax[wy] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < 8; ++q) m = max(m, wmax[q]);
    if (m) atomicMax(&sh[src], m);
  }
}

// ---------------------------------------------------------------- digits
// x -> its 7 balanced digits (most significant first) as FP32 values, row exponent E.
// F = round(x 2^(56 - (E - 1021))) is a 56-bit integer, |F| < 2^55.  Adding
// C = 0x808080808080 (128 in each of the six low byte positions) leaves bytes g_1 .. g_6
// of G = F + C with d_s = g_s - 128 in [-128, 127] (positions 6 .. 1, least significant
// first) and the top digit d_0 = floor(G / 2^48) in [-128, 128], since
// sum_{s >= 1} d_s 256^(6-s) = (G mod 2^48) - C.  These are the balanced base-256 digits
// (every low digit in [-128, 127]), obtained with one 64-bit add instead of a
// carry loop.  A byte g becomes the float 2^23 + g by a byte permute into the bits of 2^23,
// and one FP32 subtraction of 2^23 + 128 gives g - 128 exactly.
__device__ __forceinline__ void digits(double x, int E, float (&f)[S]) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int ea = (int)((hi >> 20) & 0x7FFu);
  unsigned long long m = ((unsigned long long)(hi & 0xFFFFFu) << 32) | lo;
  if (ea) m |= 1ull << 52;
  const int sh = max(ea, 1) - E + 2;  // F = m 2^sh, sh <= 2
  long long F;
  if (sh >= 0)
    F = (long long)(m << sh);
  else if (sh > -60)
    F = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
  else
    F = 0;
  if (hi & 0x80000000u) F = -F;
  const unsigned long long G = (unsigned long long)F + 0x808080808080ull;
  const uint32_t g0 = (uint32_t)G, g1 = (uint32_t)(G >> 32);
  constexpr float kBias = 8388736.0f;  // 2^23 + 128
  f[6] = __uint_as_float(__byte_perm(g0, 0x4B000000u, 0x7540)) - kBias;
  f[5] = __uint_as_float(__byte_perm(g0, 0x4B000000u, 0x7541)) - kBias;
  f[4] = __uint_as_float(__byte_perm(g0, 0x4B000000u, 0x7542)) - kBias;
  f[3] = __uint_as_float(__byte_perm(g0, 0x4B000000u, 0x7543)) - kBias;
  f[2] = __uint_as_float(__byte_perm(g1, 0x4B000000u, 0x7540)) - kBias;
  f[1] = __uint_as_float(__byte_perm(g1, 0x4B000000u, 0x7541)) - kBias;
  f[0] = __uint_as_float((uint32_t)(((int)g1 >> 16) + (0x4B000000 + 128))) - kBias;  // d_0 + 128 in [0, 256]
}

// two digits -> one 32-bit word of two bf16 (exact: a digit has at most 8 significant bits)
__device__ __forceinline__ uint32_t bf16_pair(float a, float b) {
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

struct PackJob {
  Operand op;
  const int* e;
  int TR, nrb, nkb;
  __nv_bfloat16* out;
};

// group g (TR rows x 8 reduction steps of one packed block) of a packing job
__device__ __forceinline__ void pack_group(const PackJob& jb, int64_t g) {
  const Operand& op = jb.op;
  const int* e = jb.e;
  const int TR = jb.TR, nkb = jb.nkb;
  __nv_bfloat16* out = jb.out;
  const int groups = TR * (kDepth / 8);
  const int K = op.K1 + op.K2;
  const int sigma = op.shsign * balance_sigma(op.sh);  // M1 entries times 2^-sigma, M2 entries times 2^sigma
  {
    const int within = (int)(g % groups);
    const int64_t tile = g / groups;
    const int kb = (int)(tile % nkb), rb = (int)(tile / nkb);
    const int r = within % TR, kg = within / TR;
    const int row = rb * TR + r;
    const int E = row < op.R ? e[row] : 0;
    float d[8][S];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int k = kb * kDepth + kg * 8 + kk;
      double x = 0.0;
      int Es = E;
      if (row < op.R && k < K) {
        x = k < op.K1 ? elem(op.M1, op.ld1, op.mode1, row, k) : elem(op.M2, op.ld2, op.mode2, row, k - op.K1);
        Es = k < op.K1 ? E + sigma : E - sigma;
      }
      digits(x, Es, d[kk]);
    }
    // the block's S planes stacked along the rows: one S TR x kDepth K-major operand, so
    // that consecutive planes form one wider MMA operand
    __nv_bfloat16* base = out + (size_t)tile * S * TR * kDepth;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<char*>(base) + tc::kmajor_offset(s * TR + r, kg * 8, S * TR));
      *dst = make_uint4(bf16_pair(d[0][s], d[1][s]), bf16_pair(d[2][s], d[3][s]), bf16_pair(d[4][s], d[5][s]),
                        bf16_pair(d[6][s], d[7][s]));
    }
  }
}

__device__ __forceinline__ int64_t pack_total(const PackJob& jb) {
  return (int64_t)jb.nrb * jb.nkb * jb.TR * (kDepth / 8);
}

__global__ void pack_kernel(PackJob a) {
  pdl_wait_and_release();
  const int64_t total = pack_total(a);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x)
    pack_group(a, g);
}

// both operands of a product in one launch
__global__ void pack2_kernel(PackJob a, PackJob b) {
  pdl_wait_and_release();
  const int64_t ta = pack_total(a), total = ta + pack_total(b);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    if (g < ta)
      pack_group(a, g);
    else
      pack_group(b, g - ta);
  }
}

// ---------------------------------------------------------------- GEMM
struct Smem {
  static constexpr size_t a_plane = (size_t)kTileA * kDepth * 2;
  static constexpr size_t b_plane = (size_t)kTileB * kDepth * 2;
  static constexpr size_t a_block = S * a_plane;
  static constexpr size_t b_block = S * b_plane;
  static constexpr size_t stage = a_block + b_block;
  static constexpr size_t off_bar = kSlots * stage;
  static constexpr size_t total = off_bar + 128;
};
constexpr int kGemmThreads = NT + 32;  // eight drain/epilogue warps, one control warp
constexpr uint32_t kTmemCols = 512;    // S diagonals x 64 columns = 448, rounded up

__device__ __forceinline__ double pow2(int k) {  // 2^k for -1022 <= k <= 1023
  return __longlong_as_double((long long)(k + 1023) << 52);
}
// v 2^k for any k (two exact power-of-two factors)
__device__ __forceinline__ double scale2(double v, int k) {
  const int k1 = max(-1022, min(1023, k / 2));
  return v * pow2(k1) * pow2(max(-1022, min(1023, k - k1)));
}

// (thi 2^32 + tlo) 2^(k - 64) rounded to nearest even, from integer operations only (a
// 128-bit magnitude normalised to a 64-bit window plus a sticky bit), so that the epilogue
// spends a single FP64 instruction per entry of C on this FP64-poor part.  False when the
// result is not a normal number (the caller then takes the FP64 route).
__device__ __forceinline__ bool fixed_to_f64(long long thi, long long tlo, int k, double& v) {
  const long long h = thi + (tlo >> 32);  // T = h 2^32 + l, 0 <= l < 2^32, |h| < 2^45
  const unsigned long long l = (unsigned long long)tlo & 0xFFFFFFFFull;
  const unsigned long long neg = h < 0 ? 1ull : 0ull;
  unsigned long long H = (unsigned long long)h, L = l;
  if (neg) {  // |T| = (-h - 1) 2^32 + (2^32 - l), or -h 2^32 when l = 0
    H = l ? ~(unsigned long long)h : (unsigned long long)(-h);
    L = l ? (1ull << 32) - l : 0ull;
  }
  if ((H | L) == 0) {
    v = 0.0;
    return true;
  }
  unsigned long long W, sticky = 0;
  int nb;  // bit length of |T|
  if (H >> 32) {
    nb = 96 - __clzll((long long)H);
    const int r = nb - 64;  // 1 .. 13
    W = (H << (32 - r)) | (L >> r);
    sticky = L & ((1ull << r) - 1);
  } else {
    const unsigned long long X = (H << 32) | L;
    nb = 64 - __clzll((long long)X);
    W = X << (64 - nb);
  }
  unsigned long long m = W >> 11;  // 53 bits, leading bit set
  const bool round_bit = (W >> 10) & 1ull, below = (W & 0x3FFull) | sticky;
  if (round_bit && (below || (m & 1ull))) ++m;
  if (m >> 53) {
    m >>= 1;
    ++nb;
  }
  const int e = nb - 1 + k - 64 + 1023;
  if (e < 1 || e > 2046) return false;
  v = __longlong_as_double((long long)((neg << 63) | ((unsigned long long)e << 52) | (m & 0xFFFFFFFFFFFFFull)));
  return true;
}

constexpr int kEpiGroup = 4;
// Pulls the row's entries of C that add_row_products will update into L2 while the
// tile's MMAs are still running.
template <int NC = 32>
__device__ __forceinline__ void prefetch_row(const GemmParams& p, int row, int col0) {
  const double* crow = p.C + row;
#pragma unroll 4
  for (int c = 0; c < NC; ++c) {
    const int col = col0 + c;
    if (col < p.N && col >= p.col0 && col < p.col1 && (!p.lower || row >= col))
      asm volatile("prefetch.global.L2 [%0];" ::"l"(crow + (int64_t)col * p.ldc));
  }
}
// C(row, col) += alpha (thi 2^-32 + tlo 2^-64) 2^(e_row + e_col - 2042) for the NC columns
// col0 .. col0 + NC - 1 of one row held by a thread, restricted to [p.col0, p.col1) (and
// col <= row when p.lower).  Loads of C and of the column exponents go out G columns at a
// time ahead of the stores, so a row pays NC / G memory round trips.
template <int NC = 32, int G = kEpiGroup>
__device__ __forceinline__ void add_row_products(const GemmParams& p, int row, int col0, const long long (&thi)[NC],
                                                 const long long (&tlo)[NC]) {
  const int ei = p.eA[row];
  double* crow = p.C + row;
#pragma unroll
  for (int g = 0; g < NC; g += G) {
    double cv[G];
    int ej[G];
#pragma unroll
    for (int c = 0; c < G; ++c) {
      const int col = col0 + g + c;
      const bool ok = col < p.N && col >= p.col0 && col < p.col1 && (!p.lower || row >= col);
      cv[c] = ok ? crow[(int64_t)col * p.ldc] : 0.0;
      ej[c] = ok ? p.eB[col] : -1;
    }
#pragma unroll
    for (int c = 0; c < G; ++c) {
      if (ej[c] < 0) continue;
      const int k = (ei - 1021) + (ej[c] - 1021);
      double v;
      if (!fixed_to_f64(thi[g + c], tlo[g + c], k, v))
        v = scale2(fma((double)thi[g + c], 0x1p-32, (double)tlo[g + c] * 0x1p-64), k);
      crow[(int64_t)(col0 + g + c) * p.ldc] = fma(p.alpha, v, cv[c]);
    }
  }
}

// All digit products of one stage: A_s times the stacked planes B_t0 .. B_t0+nt-1 (N = nt x
// kTileB <= 256) in one MMA into diagonals s + t0 .., since diagonal D sits at tensor-memory
// columns D kTileB and plane t of B at rows t kTileB of the stacked operand.  10 MMAs
// instead of 28 single-plane ones, each reading its A plane once.  s = 0 covers every
// diagonal first, so `fresh` (0 at a chunk's first stage) there restarts the accumulators.
__device__ __forceinline__ void digit_products(uint32_t tmem, uint64_t ad0, uint64_t bd0, uint32_t fresh) {
  constexpr uint64_t a_step = ((kTileA / 8) * 128) >> 4, b_step = ((kTileB / 8) * 128) >> 4;
#pragma unroll
  for (int s = 0; s < S; ++s) {
#pragma unroll
    for (int t0 = 0; t0 < S - s; t0 += 4) {
      const int nt = (S - s - t0) < 4 ? (S - s - t0) : 4;
      const uint32_t idesc = nt == 4   ? tc::idesc_bf16_f32(kTileA, 4 * kTileB)
                             : nt == 3 ? tc::idesc_bf16_f32(kTileA, 3 * kTileB)
                             : nt == 2 ? tc::idesc_bf16_f32(kTileA, 2 * kTileB)
                                       : tc::idesc_bf16_f32(kTileA, kTileB);
      tc::mma_bf16(tmem + (uint32_t)((s + t0) * kTileB), ad0 + (uint64_t)s * a_step, bd0 + (uint64_t)t0 * b_step,
                   idesc, s == 0 ? fresh : 1u);
    }
  }
}

__global__ void __launch_bounds__(kGemmThreads, 1) gemm_kernel(GemmParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Smem::off_bar);  // [kSlots]
  uint64_t* freed = full + kSlots;                                      // [kSlots] MMAs of a stage done
  uint64_t* acc_ready = freed + kSlots;                                 // chunk's MMAs done
  uint64_t* drained = acc_ready + 1;                                    // tensor memory read
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drained + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int I = blockIdx.x, J = blockIdx.y, z = blockIdx.z;
  const int kb0 = z * p.kb_per_split, kb1 = min(p.nkb, kb0 + p.kb_per_split);
  const int nst = kb1 - kb0;
  if (p.C && p.lower && (I + 1) * kTileA <= J * kTileB) return;  // tile above the diagonal
  if (p.C && (J * kTileB >= p.col1 || (J + 1) * kTileB <= p.col0)) return;
  const unsigned long long deadline = global_ns() + p.limit_ns;
  if (tid == 0) {
    for (int q = 0; q < kSlots; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&freed[q], 1);
    }
    tc::mbar_init(acc_ready, 1);
    tc::mbar_init(drained, NT / 32);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_holder, kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  pdl_wait_and_release();
  trace_start(p.trace);
  int timed_out = 0;
  long long thi[32], tlo[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) thi[c] = tlo[c] = 0;

  if (warp == NT / 32) {
    if (lane == 0 && nst > 0) {
      auto issue = [&](int st) {
        const int kb = kb0 + st, slot = st % kSlots;
        unsigned char* dst = smem + slot * Smem::stage;
        tc::mbar_arrive_expect_tx(&full[slot], (uint32_t)Smem::stage);
        tc::bulk_g2s(dst, reinterpret_cast<const unsigned char*>(p.A) + ((size_t)I * p.nkb + kb) * Smem::a_block,
                     (uint32_t)Smem::a_block, &full[slot]);
        tc::bulk_g2s(dst + Smem::a_block,
                     reinterpret_cast<const unsigned char*>(p.B) + ((size_t)J * p.nkb + kb) * Smem::b_block,
                     (uint32_t)Smem::b_block, &full[slot]);
      };
      for (int q = 0; q < kSlots - 1 && q < nst; ++q) issue(q);
      for (int st = 0; st < nst && !timed_out; ++st) {
        const int slot = st % kSlots, chunk = st / kChunkBlocks;
        if (!tc::mbar_wait(&full[slot], (uint32_t)(st / kSlots) & 1u, deadline)) {
          timed_out = 1;
          break;
        }
        // the chunk's first MMAs overwrite the accumulators: the previous chunk must be read
        if (st % kChunkBlocks == 0 && chunk > 0 &&
            !tc::mbar_wait(drained, (uint32_t)(chunk - 1) & 1u, deadline)) {
          timed_out = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t abase = tc::smem_u32(smem + slot * Smem::stage);
        const uint32_t bbase = abase + (uint32_t)Smem::a_block;
        // descriptors of plane 0 of the stacked operands; plane s starts s (TR / 8) 128 bytes
        // later, which adds that >> 4 to the address field (shared addresses stay below 2^18)
        const uint64_t ad0 = tc::smem_desc(abase, (S * kTileA / 8) * 128, 128);
        const uint64_t bd0 = tc::smem_desc(bbase, (S * kTileB / 8) * 128, 128);
        static_assert(kDepth == 16, "one MMA depth per stage");
        digit_products(tmem, ad0, bd0, (st % kChunkBlocks == 0) ? 0u : 1u);
        tc::mma_commit(&freed[slot]);
        if (st % kChunkBlocks == kChunkBlocks - 1 || st == nst - 1) tc::mma_commit(acc_ready);
        // refill stage st - 1's slot with stage st + kSlots - 1 once its MMAs are done;
        // stage st's MMAs are already queued behind them
        // (slot kSlots - 1 starts empty: stage kSlots - 1 goes there at st = 0)
        if (st + kSlots - 1 < nst) {
          if (st >= 1 &&
              !tc::mbar_wait(&freed[(st - 1) % kSlots], (uint32_t)((st - 1) / kSlots) & 1u, deadline)) {
            timed_out = 1;
            break;
          }
          issue(st + kSlots - 1);
        }
      }
      if (timed_out) {
        const unsigned long long dl = global_ns() + p.limit_ns;
        for (int q = 0; q < kSlots; ++q) {
          tc::mbar_wait(&full[q], 0, dl);
          tc::mbar_wait(&freed[q], 0, dl);
        }
      }
    }
  } else {
    // drain warps: lane quadrant warp & 3, columns 32 (warp >> 2) .. + 31
    const uint32_t q = warp & 3, h = warp >> 2;
    const int nchunks = (nst + kChunkBlocks - 1) / kChunkBlocks;
    if (!p.Phi && I * kTileA + (int)(q * 32) + lane < p.M) prefetch_row(p, I * kTileA + q * 32 + lane, J * kTileB + h * 32);
    for (int c = 0; c < nchunks; ++c) {
      if (!tc::mbar_wait(acc_ready, (uint32_t)c & 1u, deadline)) {
        timed_out = 1;
        break;
      }
      tc::fence_after_sync();
#pragma unroll 1
      for (int D = 0; D < S; ++D) {
        float v[32];
        tc::tmem_ld32(tmem + ((q * 32) << 16) + (uint32_t)(D * kTileB + h * 32), v);
        const int shift = D <= 2 ? 8 * (2 - D) : 8 * (6 - D);
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) {
          const long long iv = (long long)__float2int_rn(v[cc]) << shift;
          if (D <= 2)
            thi[cc] += iv;
          else
            tlo[cc] += iv;
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(drained);
    }
  }

  if (__syncthreads_or(timed_out)) {
    if (tid == 0 && p.status) atomicCAS(p.status, 0, BANDRED_DEV_TIMEOUT);
  } else if (warp < NT / 32) {
    const int q = warp & 3, h = warp >> 2;
    const int row = I * kTileA + q * 32 + lane;
    if (row < p.M) {
      if (p.Phi) {
        int64_t* Ph = p.Phi + (size_t)z * p.sstride;
        int64_t* Pl = p.Plo + (size_t)z * p.sstride;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int col = J * kTileB + h * 32 + c;
          if (col < p.N) {
            Ph[row + (int64_t)col * p.ldp] = thi[c];
            Pl[row + (int64_t)col * p.ldp] = tlo[c];
          }
        }
      } else {
        add_row_products(p, row, J * kTileB + h * 32, thi, tlo);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
  trace_end(p.trace);
}

// Persistent form of the direct mode (C += alpha A B^T, the rank-2k updates): one CTA per
// SM walks its tiles (every gridDim.x-th tile of the lower triangle / column range) with one
// continuous copy and MMA pipeline, so a tile's epilogue (reading and writing C) runs
// while the next tile's MMAs do; only the read-out of tensor memory stalls the MMAs.
// Sixteen drain/epilogue warps of 16 columns each (lane quadrant warp & 3, column group
// warp >> 2): twice the warps of the tile kernel to hide the latency of the C loads and of
// the FP64 adds, with half the 64-bit sums per thread.
constexpr int kMaxTilesPerCta = 1024;
constexpr int kRankWorkers = 16;
constexpr int kRankThreads = kRankWorkers * 32 + 32;
constexpr int kRankCols = kTileB / 4;  // columns per worker thread

__global__ void __launch_bounds__(kRankThreads, 1) rank_kernel(GemmParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Smem::off_bar);
  uint64_t* freed = full + kSlots;
  uint64_t* acc_ready = freed + kSlots;
  uint64_t* drained = acc_ready + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drained + 1);
  int* tiles = reinterpret_cast<int*>(smem + Smem::total);  // this CTA's tiles
  __shared__ int s_nt;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nI = (p.M + kTileA - 1) / kTileA, nJ = (p.N + kTileB - 1) / kTileB;
  const int nkb = p.nkb, cpt = (nkb + kChunkBlocks - 1) / kChunkBlocks;
  const unsigned long long deadline = global_ns() + p.limit_ns;
  if (tid == 0) {
    int n = 0;
    for (int L = blockIdx.x; L < nI * nJ && n < kMaxTilesPerCta; L += gridDim.x) {
      const int I = L % nI, J = L / nI;
      if (p.lower && (I + 1) * kTileA <= J * kTileB) continue;
      if (J * kTileB >= p.col1 || (J + 1) * kTileB <= p.col0) continue;
      tiles[n++] = L;
    }
    s_nt = n;
    for (int q = 0; q < kSlots; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&freed[q], 1);
    }
    tc::mbar_init(acc_ready, 1);
    tc::mbar_init(drained, kRankWorkers);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_holder, kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  pdl_wait_and_release();
  trace_start(p.trace);
  const int nt = s_nt;
  const int total = nt * nkb;
  int timed_out = 0;

  if (warp == kRankWorkers) {
    if (lane == 0 && total > 0) {
      auto issue = [&](int qs) {
        const int L = tiles[qs / nkb], kb = qs % nkb, slot = qs % kSlots;
        const int I = L % nI, J = L / nI;
        unsigned char* dst = smem + slot * Smem::stage;
        tc::mbar_arrive_expect_tx(&full[slot], (uint32_t)Smem::stage);
        tc::bulk_g2s(dst, reinterpret_cast<const unsigned char*>(p.A) + ((size_t)I * nkb + kb) * Smem::a_block,
                     (uint32_t)Smem::a_block, &full[slot]);
        tc::bulk_g2s(dst + Smem::a_block,
                     reinterpret_cast<const unsigned char*>(p.B) + ((size_t)J * nkb + kb) * Smem::b_block,
                     (uint32_t)Smem::b_block, &full[slot]);
      };
      for (int q = 0; q < kSlots - 1 && q < total; ++q) issue(q);
      for (int q = 0; q < total && !timed_out; ++q) {
        const int slot = q % kSlots, kb = q % nkb;
        const int gc = (q / nkb) * cpt + kb / kChunkBlocks;  // chunk index across tiles
        if (!tc::mbar_wait(&full[slot], (uint32_t)(q / kSlots) & 1u, deadline)) {
          timed_out = 1;
          break;
        }
        if (kb % kChunkBlocks == 0 && gc > 0 && !tc::mbar_wait(drained, (uint32_t)(gc - 1) & 1u, deadline)) {
          timed_out = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t abase = tc::smem_u32(smem + slot * Smem::stage);
        const uint64_t ad0 = tc::smem_desc(abase, (S * kTileA / 8) * 128, 128);
        const uint64_t bd0 = tc::smem_desc(abase + (uint32_t)Smem::a_block, (S * kTileB / 8) * 128, 128);
        digit_products(tmem, ad0, bd0, (kb % kChunkBlocks == 0) ? 0u : 1u);
        tc::mma_commit(&freed[slot]);
        if (kb % kChunkBlocks == kChunkBlocks - 1 || kb == nkb - 1) tc::mma_commit(acc_ready);
        if (q + kSlots - 1 < total) {
          if (q >= 1 && !tc::mbar_wait(&freed[(q - 1) % kSlots], (uint32_t)((q - 1) / kSlots) & 1u, deadline)) {
            timed_out = 1;
            break;
          }
          issue(q + kSlots - 1);
        }
      }
      if (timed_out) {
        const unsigned long long dl = global_ns() + p.limit_ns;
        for (int q = 0; q < kSlots; ++q) {
          tc::mbar_wait(&full[q], 0, dl);
          tc::mbar_wait(&freed[q], 0, dl);
        }
      }
    }
  } else {
    const uint32_t qd = warp & 3, h = warp >> 2;
    for (int lt = 0; lt < nt && !timed_out; ++lt) {
      {
        const int L = tiles[lt], row = (L % nI) * kTileA + qd * 32 + lane;
        if (row < p.M) prefetch_row<kRankCols>(p, row, (L / nI) * kTileB + h * kRankCols);
      }
      long long thi[kRankCols], tlo[kRankCols];
#pragma unroll
      for (int c = 0; c < kRankCols; ++c) thi[c] = tlo[c] = 0;
      for (int c = 0; c < cpt; ++c) {
        const int gc = lt * cpt + c;
        if (!tc::mbar_wait(acc_ready, (uint32_t)gc & 1u, deadline)) {
          timed_out = 1;
          break;
        }
        tc::fence_after_sync();
#pragma unroll 1
        for (int D = 0; D < S; ++D) {
          float v[kRankCols];
          tc::tmem_ld16(tmem + ((qd * 32) << 16) + (uint32_t)(D * kTileB + h * kRankCols), v);
          const int shift = D <= 2 ? 8 * (2 - D) : 8 * (6 - D);
#pragma unroll
          for (int cc = 0; cc < kRankCols; ++cc) {
            const long long iv = (long long)__float2int_rn(v[cc]) << shift;
            if (D <= 2)
              thi[cc] += iv;
            else
              tlo[cc] += iv;
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(drained);
      }
      if (timed_out) break;
      // epilogue of this tile while the next tile's MMAs run
      const int L = tiles[lt], I = L % nI, J = L / nI;
      const int row = I * kTileA + qd * 32 + lane;
      if (row < p.M) {
        add_row_products<kRankCols, 8>(p, row, J * kTileB + h * kRankCols, thi, tlo);
      }
    }
  }
  if (__syncthreads_or(timed_out) && tid == 0 && p.status) atomicCAS(p.status, 0, BANDRED_DEV_TIMEOUT);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
  trace_end(p.trace);
}

// ---------------------------------------------------------------- streamed left operand
// C_partial = op(A) B^T with op(A) read as FP64 by the TMA (plain, transposed, or
// symmetric with the lower triangle stored) and cut into digits in shared memory by the
// worker warps, so the left operand is read once and never written back as digits.  A
// stage is one 128 x 16 FP64 box (or, above the diagonal of a symmetric A, one 16 x 128
// box of the mirror, 128-byte swizzled) plus the packed digits of B (N <= kTileB), in a
// ring of four; the digits of A are double-buffered.  Tiles across the diagonal take the
// lower box and fetch their upper entries from the mirror directly.  Sixteen worker warps
// convert and drain (16 columns each), one control warp moves data and issues the MMAs.
struct StreamSmem {
  static constexpr int NS = 4;
  static constexpr size_t tile = (size_t)kTileA * kDepth * 8;
  static constexpr size_t off_b = NS * tile;
  static constexpr size_t off_a = off_b + NS * Smem::b_block;
  static constexpr size_t off_bar = off_a + 2 * Smem::a_block;
  static constexpr size_t total = off_bar + 128 + 1024;  // + alignment of the base to 1024
};
constexpr int kStreamWorkers = 16;
constexpr int kStreamThreads = kStreamWorkers * 32 + 32;

struct StreamParams {
  const double* A;  // op(A)(r, k): mode 0 A[r + k lda], 1 A[k + r lda], 2 symmetric (lower stored)
  int64_t lda;
  int mode;
  int M, K, N;
  const int* eA;           // row exponents of op(A)
  const __nv_bfloat16* B;  // digits of B, packed with TR = kTileB (one row block)
  int nkb, kb_per_split;
  int64_t* Phi;
  int64_t* Plo;
  int64_t ldp, sstride;
  int* status;
  unsigned long long limit_ns;
  unsigned long long* trace;
};

__global__ void __launch_bounds__(kStreamThreads, 1)
    stream_kernel(StreamParams p, const __grid_constant__ CUtensorMap tm_lo, const __grid_constant__ CUtensorMap tm_up) {
  using L = StreamSmem;
  constexpr int NS = L::NS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  double* ring = reinterpret_cast<double*>(smem);
  unsigned char* bring = smem + L::off_b;
  unsigned char* adig = smem + L::off_a;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::off_bar);  // [NS] copies landed
  uint64_t* converted = full + NS;                                    // [2] digits of A written
  uint64_t* mma_done = converted + 2;                                 // [2] MMAs of a stage done
  uint64_t* acc_ready = mma_done + 2;                                 // MMAs of a chunk done
  uint64_t* drained = acc_ready + 1;                                  // tensor memory read
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drained + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * kTileA, z = blockIdx.y;
  const int kb0 = z * p.kb_per_split, kb1 = min(p.nkb, kb0 + p.kb_per_split);
  const int nst = kb1 - kb0;
  const unsigned long long deadline = global_ns() + p.limit_ns;
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) tc::mbar_init(&full[q], 1);
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&converted[q], kStreamWorkers);
      tc::mbar_init(&mma_done[q], 1);
    }
    tc::mbar_init(acc_ready, 1);
    tc::mbar_init(drained, kStreamWorkers);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_holder, kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  pdl_wait_and_release();
  trace_start(p.trace);

  // 0: box read in place; 1: box of the mirror (transposed); 2: symmetric box across the diagonal
  auto kind_of = [&](int kb) -> int {
    if (p.mode != 2) return p.mode;
    const int k0 = kb * kDepth;
    if (k0 + kDepth - 1 <= i0) return 0;
    if (k0 >= i0 + kTileA) return 1;
    return 2;
  };
  int timed_out = 0;
  long long thi[16], tlo[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) thi[c] = tlo[c] = 0;

  if (warp == kStreamWorkers) {
    if (lane == 0 && nst > 0) {
      tc::prefetch_tmap(&tm_lo);
      tc::prefetch_tmap(&tm_up);
      auto issue = [&](int ls) {
        const int kb = kb0 + ls, slot = ls % NS, k0 = kb * kDepth;
        double* dst = ring + (size_t)slot * kTileA * kDepth;
        tc::mbar_arrive_expect_tx(&full[slot], (uint32_t)(L::tile + Smem::b_block));
        if (kind_of(kb) == 1)
          tc::tma_load_2d(dst, &tm_up, k0, i0, &full[slot]);
        else
          tc::tma_load_2d(dst, &tm_lo, i0, k0, &full[slot]);
        tc::bulk_g2s(bring + (size_t)slot * Smem::b_block,
                     reinterpret_cast<const unsigned char*>(p.B) + (size_t)kb * Smem::b_block,
                     (uint32_t)Smem::b_block, &full[slot]);
      };
      int issued = 0;
      for (; issued < NS - 1 && issued < nst; ++issued) issue(issued);
      for (int st = 0; st < nst; ++st) {
        const int sb = st & 1, chunk = st / kChunkBlocks;
        if (!tc::mbar_wait(&converted[sb], (uint32_t)(st >> 1) & 1u, deadline)) {
          timed_out = 1;
          break;
        }
        // the chunk's first MMAs overwrite the accumulators: the previous chunk must be read
        if (st % kChunkBlocks == 0 && chunk > 0 &&
            !tc::mbar_wait(drained, (uint32_t)(chunk - 1) & 1u, deadline)) {
          timed_out = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t abase = tc::smem_u32(adig + (size_t)sb * Smem::a_block);
        const uint32_t bbase = tc::smem_u32(bring + (size_t)(st % NS) * Smem::b_block);
        digit_products(tmem, tc::smem_desc(abase, (S * kTileA / 8) * 128, 128),
                       tc::smem_desc(bbase, (S * kTileB / 8) * 128, 128), (st % kChunkBlocks == 0) ? 0u : 1u);
        tc::mma_commit(&mma_done[sb]);
        if (st % kChunkBlocks == kChunkBlocks - 1 || st == nst - 1) tc::mma_commit(acc_ready);
        // refill the slot of stage st - 1 (its box was converted, its B digits multiplied)
        if (issued < nst) {
          if (st >= 1 &&
              !tc::mbar_wait(&mma_done[(st - 1) & 1], (uint32_t)((st - 1) >> 1) & 1u, deadline)) {
            timed_out = 1;
            break;
          }
          issue(issued++);
        }
      }
      if (timed_out) {  // let copies and MMAs in flight land before the CTA leaves (bounded)
        const unsigned long long dl = global_ns() + p.limit_ns;
        for (int q = 0; q < NS; ++q) tc::mbar_wait(&full[q], 0, dl);
        for (int q = 0; q < 2; ++q) tc::mbar_wait(&mma_done[q], 0, dl);
      }
    }
  } else {
    const int r = tid & (kTileA - 1), kq = tid >> 7;  // row r, k in [4 kq, 4 kq + 4) of a stage
    const int gi = i0 + r;
    const int E = gi < p.M ? p.eA[gi] : 0;
    const uint32_t q = warp & 3, h = warp >> 2;  // tensor-memory lane quadrant, 16-column group
    auto drain = [&](int c) -> bool {
      if (!tc::mbar_wait(acc_ready, (uint32_t)c & 1u, deadline)) return false;
      tc::fence_after_sync();
#pragma unroll 1
      for (int D = 0; D < S; ++D) {
        float v[16];
        tc::tmem_ld16(tmem + ((q * 32) << 16) + (uint32_t)(D * kTileB + h * 16), v);
        const int shift = D <= 2 ? 8 * (2 - D) : 8 * (6 - D);
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) {
          const long long iv = (long long)__float2int_rn(v[cc]) << shift;
          if (D <= 2)
            thi[cc] += iv;
          else
            tlo[cc] += iv;
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(drained);
      return true;
    };
    for (int st = 0; st < nst; ++st) {
      const int sb = st & 1, slot = st % NS, kb = kb0 + st, k0 = kb * kDepth;
      const int kind = kind_of(kb);
      double x[4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) x[kk] = 0.0;
      if (kind == 2) {  // upper entries of a diagonal box, from the stored mirror A(k, r)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const int gk = k0 + 4 * kq + kk;
          if (gi < gk && gk < p.K && gi < p.M) x[kk] = __ldg(p.A + gk + (int64_t)gi * p.lda);
        }
      }
      if (!tc::mbar_wait(&full[slot], (uint32_t)(st / NS) & 1u, deadline) ||
          (st >= 2 && !tc::mbar_wait(&mma_done[sb], (uint32_t)((st - 2) >> 1) & 1u, deadline))) {
        timed_out = 1;
        break;
      }
      const double* tile = ring + (size_t)slot * kTileA * kDepth;
      if (kind == 1) {  // row r holds 16 entries in eight 16-byte chunks, chunk c at c ^ (r & 7)
        const double* row = tile + r * kDepth;
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
          const double2 v = *reinterpret_cast<const double2*>(row + 2 * ((2 * kq + c2) ^ (r & 7)));
          x[2 * c2] = v.x;
          x[2 * c2 + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const double v = tile[(4 * kq + kk) * kTileA + r];
          if (kind == 0 || gi >= k0 + 4 * kq + kk) x[kk] = v;
        }
      }
      float d[4][S];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) digits(x[kk], E, d[kk]);
      unsigned char* dst = adig + (size_t)sb * Smem::a_block;
#pragma unroll
      for (int s = 0; s < S; ++s)
        *reinterpret_cast<uint2*>(dst + tc::kmajor_offset(s * kTileA + r, 4 * kq, S * kTileA)) =
            make_uint2(bf16_pair(d[0][s], d[1][s]), bf16_pair(d[2][s], d[3][s]));
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&converted[sb]);
      if (st % kChunkBlocks == 0 && st > 0 && !drain(st / kChunkBlocks - 1)) {
        timed_out = 1;
        break;
      }
    }
    if (!timed_out && nst > 0 && !drain((nst - 1) / kChunkBlocks)) timed_out = 1;
  }

  if (__syncthreads_or(timed_out)) {
    if (tid == 0 && p.status) atomicCAS(p.status, 0, BANDRED_DEV_TIMEOUT);
  } else if (warp < kStreamWorkers) {
    const int q = warp & 3, h = warp >> 2;
    const int row = i0 + q * 32 + lane;
    if (row < p.M) {
      int64_t* Ph = p.Phi + (size_t)z * p.sstride;
      int64_t* Pl = p.Plo + (size_t)z * p.sstride;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int col = h * 16 + c;
        if (col < p.N) {
          Ph[row + (int64_t)col * p.ldp] = thi[c];
          Pl[row + (int64_t)col * p.ldp] = tlo[c];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
  trace_end(p.trace);
}

__global__ void reduce_kernel(const int64_t* Phi, const int64_t* Plo, int64_t ldp, int64_t sstride, int splits,
                              const int* eA, const int* eB, int M, int N, double alpha, double beta, double* C,
                              int64_t ldc) {
  pdl_wait_and_release();
  const int64_t total = (int64_t)M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % M), j = (int)(idx / M);
    long long h = 0, l = 0;
    for (int z = 0; z < splits; ++z) {
      h += Phi[(size_t)z * sstride + i + (int64_t)j * ldp];
      l += Plo[(size_t)z * sstride + i + (int64_t)j * ldp];
    }
    const double v = scale2(fma((double)h, 0x1p-32, (double)l * 0x1p-64), (eA[i] - 1021) + (eB[j] - 1021));
    double* cp = C + i + (int64_t)j * ldc;
    *cp = beta == 0.0 ? alpha * v : fma(alpha, v, beta * *cp);
  }
}

// The same sums for outputs with many splits (X2 = X1^T W / 2 splits its reduction of
// length j over up to 64 CTAs): 32 consecutive outputs per block, the splits dealt to the
// block's eight warps and their partial sums added in shared memory.  The sums are
// integers, so the result is the one of reduce_kernel bit for bit.
constexpr int kWideSplits = 8;  // splits above which reduce() takes this kernel
__global__ void __launch_bounds__(256)
    reduce_wide_kernel(const int64_t* Phi, const int64_t* Plo, int64_t ldp, int64_t sstride, int splits, const int* eA,
                       const int* eB, int M, int N, double alpha, double beta, double* C, int64_t ldc) {
  __shared__ long long ph[8][32], pl[8][32];
  pdl_wait_and_release();
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int64_t total = (int64_t)M * N;
  const int64_t e = blockIdx.x * 32ll + lane;
  const bool live = e < total;
  const int i = live ? (int)(e % M) : 0, j = live ? (int)(e / M) : 0;
  long long h = 0, l = 0;
  if (live) {
    const size_t off = i + (size_t)j * ldp;
#pragma unroll 4
    for (int z = wy; z < splits; z += 8) {
      h += Phi[(size_t)z * sstride + off];
      l += Plo[(size_t)z * sstride + off];
    }
  }
  ph[wy][lane] = h;
  pl[wy][lane] = l;
  __syncthreads();
  if (wy == 0 && live) {
#pragma unroll
    for (int q = 1; q < 8; ++q) {
      h += ph[q][lane];
      l += pl[q][lane];
    }
    const double v = scale2(fma((double)h, 0x1p-32, (double)l * 0x1p-64), (eA[i] - 1021) + (eB[j] - 1021));
    double* cp = C + i + (int64_t)j * ldc;
    *cp = beta == 0.0 ? alpha * v : fma(alpha, v, beta * *cp);
  }
}

}  // namespace

// ---------------------------------------------------------------- host API
namespace {

// both exponent arrays zeroed by one launch (n2 = 0: the first only)
cudaError_t zero_exponents(int* e1, int n1, int* e2, int n2, cudaStream_t s) {
  n1 = std::max(n1, 0);
  n2 = e2 ? std::max(n2, 0) : 0;
  if (n1 + n2 <= 0) return cudaSuccess;
  prof::count_launch();
  return launch_pdl(zero2_kernel, dim3((unsigned)std::min(1024, (n1 + n2 + 255) / 256)), dim3(256), 0, s, e1, n1, e2,
                    n2);
}

// the row exponents of op into e, which the caller has zeroed
cudaError_t row_exponents_nozero(const Operand& op, int* e, cudaStream_t s) {
  if (op.R <= 0) return cudaSuccess;
  auto one = [&](const double* M, int64_t ld, int mode, int K, int dir) -> cudaError_t {
    if (K <= 0 || !M) return cudaSuccess;
    const int ks = std::max(1, std::min(64, K / 256));
    if (mode == 2) {
      const int T = (op.R + 31) / 32;
      prof::count_launch();
      if (cudaError_t le = launch_pdl(rowexp_sym_kernel, dim3(T, T), dim3(256), 0, s, M, ld, op.R, e)) return le;
    }
    if (mode == 0) {
      prof::count_launch();
      if (cudaError_t le = launch_pdl(rowexp_cols_kernel, dim3((op.R + 31) / 32, (K + 31) / 32), dim3(256), 0, s, M, ld,
                                      op.R, K, e, op.sh, dir))
        return le;
    }
    if (mode == 1) {
      prof::count_launch();
      if (cudaError_t le = launch_pdl(rowexp_rows_kernel, dim3((op.R + 7) / 8, ks), dim3(256), 0, s, M, ld, op.R, 0, K, 0,
                                      e, op.sh, dir))
        return le;
    }
    return cudaGetLastError();
  };
  if (op.M1 && op.M2 && op.mode1 == 0 && op.mode2 == 0 && op.K1 > 0 && op.K2 > 0) {
    const int t = (op.K1 + 31) / 32 + (op.K2 + 31) / 32;
    prof::count_launch();
    if (cudaError_t le = launch_pdl(rowexp_cols2_kernel, dim3((op.R + 31) / 32, t), dim3(256), 0, s, op.M1, op.ld1,
                                    op.K1, op.sh ? -op.shsign : 0, op.M2, op.ld2, op.K2, op.sh ? op.shsign : 0, op.R, e,
                                    op.sh))
      return le;
    return cudaGetLastError();
  }
  cudaError_t err = one(op.M1, op.ld1, op.mode1, op.K1, op.sh ? -op.shsign : 0);
  if (err != cudaSuccess) return err;
  return one(op.M2, op.ld2, op.mode2, op.K2, op.sh ? op.shsign : 0);
}

}  // namespace

cudaError_t row_exponents(const Operand& op, int* e, cudaStream_t s) {
  if (op.R <= 0) return cudaSuccess;
  cudaError_t err = zero_exponents(e, op.R, nullptr, 0, s);
  if (err != cudaSuccess) return err;
  return row_exponents_nozero(op, e, s);
}

cudaError_t balance(const Operand& op, int* sh, cudaStream_t s) {
  prof::count_launch();
  cudaError_t err = launch_pdl(zero_kernel, dim3(1), dim3(32), 0, s, sh, 2);
  if (err != cudaSuccess) return err;
  const int K = std::max(std::max(op.K1, op.K2), 1);
  if (op.R <= 0) return cudaSuccess;
  prof::count_launch();
  return launch_pdl(maxexp_kernel, dim3((op.R + 31) / 32, (K + 31) / 32, 2), dim3(256), 0, s, op, sh);
}

size_t packed_bytes(int R, int K, int TR) {
  const size_t nrb = (R + TR - 1) / TR, nkb = (K + kDepth - 1) / kDepth;
  return nrb * nkb * (size_t)S * TR * kDepth * 2;
}

static PackJob pack_job(const Operand& op, const int* e, int TR, __nv_bfloat16* out) {
  const int K = op.K1 + op.K2;
  PackJob jb{op, e, TR, (op.R + TR - 1) / TR, (K + kDepth - 1) / kDepth, out};
  if (op.R <= 0 || K <= 0) jb.nrb = jb.nkb = 0;
  return jb;
}

cudaError_t pack(const Operand& op, const int* e, int TR, __nv_bfloat16* out, cudaStream_t s) {
  const PackJob jb = pack_job(op, e, TR, out);
  const int64_t total = (int64_t)jb.nrb * jb.nkb * TR * (kDepth / 8);
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
  prof::count_launch();
  return launch_pdl(pack_kernel, dim3(blocks), dim3(256), 0, s, jb);
}

// both operands of a product, one launch
static cudaError_t pack2(const Operand& A, const int* eA, int TRA, __nv_bfloat16* outA, const Operand& B,
                         const int* eB, int TRB, __nv_bfloat16* outB, cudaStream_t s) {
  const PackJob a = pack_job(A, eA, TRA, outA), b = pack_job(B, eB, TRB, outB);
  const int64_t total = (int64_t)a.nrb * a.nkb * TRA * (kDepth / 8) + (int64_t)b.nrb * b.nkb * TRB * (kDepth / 8);
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
  prof::count_launch();
  return launch_pdl(pack2_kernel, dim3(blocks), dim3(256), 0, s, a, b);
}

cudaError_t gemm(const GemmParams& p, int splits, cudaStream_t s) {
  if (p.M <= 0 || p.N <= 0 || p.nkb <= 0) return cudaSuccess;
  static int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Smem::total);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  const dim3 grid((p.M + kTileA - 1) / kTileA, (p.N + kTileB - 1) / kTileB, splits);
  prof::count_launch();
  return launch_pdl(gemm_kernel, grid, dim3(kGemmThreads), Smem::total, s, p);
}

cudaError_t reduce(const GemmParams& p, int splits, double alpha, double beta, double* C, int64_t ldc,
                   cudaStream_t s) {
  const int64_t total = (int64_t)p.M * p.N;
  if (total <= 0) return cudaSuccess;
  if (splits > kWideSplits) {
    prof::count_launch();
    return launch_pdl(reduce_wide_kernel, dim3((unsigned)((total + 31) / 32)), dim3(256), 0, s, p.Phi, p.Plo, p.ldp,
                      p.sstride, splits, p.eA, p.eB, p.M, p.N, alpha, beta, C, ldc);
  }
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  prof::count_launch();
  return launch_pdl(reduce_kernel, dim3(blocks), dim3(256), 0, s, p.Phi, p.Plo, p.ldp, p.sstride, splits, p.eA, p.eB,
                    p.M, p.N, alpha, beta, C, ldc);
}

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

int choose_splits(int M, int N, int K, int sms) {
  const int tiles = ((M + kTileA - 1) / kTileA) * ((N + kTileB - 1) / kTileB);
  const int nkb = (K + kDepth - 1) / kDepth;
  int sp = std::max(1, sms / std::max(tiles, 1));
  sp = std::min(sp, std::max(1, nkb / kChunkBlocks));  // at least one exact chunk per split
  return std::min(sp, 64);
}

size_t bytes(int M, int N, int K, int splits, bool partials) {
  M = std::max(M, 1);
  N = std::max(N, 1);
  K = std::max(K, 1);
  return al256(sizeof(int) * (size_t)M) + al256(sizeof(int) * (size_t)N) + al256(packed_bytes(M, K, kTileA)) +
         al256(packed_bytes(N, K, kTileB)) + (partials ? al256(2 * sizeof(int64_t) * (size_t)splits * M * N) : 0);
}

int fit_splits(int M, int N, int K, int want, size_t cap) {
  int sp = std::max(1, want);
  while (sp > 1 && bytes(M, N, K, sp) > cap) --sp;
  return sp;
}

Bufs carve(void* base, int M, int N, int K, int splits) {
  M = std::max(M, 1);
  N = std::max(N, 1);
  K = std::max(K, 1);
  char* w = static_cast<char*>(base);
  Bufs b;
  b.eA = reinterpret_cast<int*>(w);
  w += al256(sizeof(int) * (size_t)M);
  b.eB = reinterpret_cast<int*>(w);
  w += al256(sizeof(int) * (size_t)N);
  b.Ablob = reinterpret_cast<__nv_bfloat16*>(w);
  w += al256(packed_bytes(M, K, kTileA));
  b.Bblob = reinterpret_cast<__nv_bfloat16*>(w);
  w += al256(packed_bytes(N, K, kTileB));
  b.P = reinterpret_cast<int64_t*>(w);
  return b;
}

cudaError_t prepare(const Operand& A, const Operand& B, const Bufs& b, cudaStream_t s) {
  const bool twoB = b.eB != b.eA && !b.b_packed;
  cudaError_t e = zero_exponents(b.eA, A.R, twoB ? b.eB : nullptr, B.R, s);
  if (e == cudaSuccess) e = row_exponents_nozero(A, b.eA, s);
  if (e == cudaSuccess && twoB) e = row_exponents_nozero(B, b.eB, s);
  if (e == cudaSuccess) {
    if (b.b_packed)
      e = pack(A, b.eA, kTileA, b.Ablob, s);
    else
      e = pack2(A, b.eA, kTileA, b.Ablob, B, b.eB, kTileB, b.Bblob, s);
  }
  return e;
}

namespace {

// The streamed path: a single-source left operand whose base and columns are 16-byte
// aligned (the TMA's rule), N <= kTileB.  False (nothing launched) when it does not apply.
bool stream_product(const Operand& A, const Operand& B, int M, int N, int K, double alpha, double beta, double* C,
                    int64_t ldc, const Bufs& b, int splits, int* status, unsigned long long limit_ns,
                    cudaStream_t s, cudaError_t* err) {
  if (A.M2 || A.K2 != 0 || N > kTileB || A.K1 != K || A.R != M) return false;
  if ((reinterpret_cast<uintptr_t>(A.M1) & 15u) != 0 || (A.ld1 & 1) != 0) return false;
  CUtensorMap lo, up;
  const int mode = A.mode1;
  if (mode == 0 || mode == 2) {
    if (A.ld1 < M || !split::encode_tile_map_f64(&lo, A.M1, M, K, A.ld1, kTileA, kDepth, false)) return false;
  }
  if (mode == 1 || mode == 2) {
    if (A.ld1 < K || !split::encode_tile_map_f64(&up, A.M1, K, M, A.ld1, kDepth, kTileA, true)) return false;
  }
  if (mode == 0) std::memcpy(&up, &lo, sizeof(CUtensorMap));
  if (mode == 1) std::memcpy(&lo, &up, sizeof(CUtensorMap));
  static int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  auto run = [&]() -> cudaError_t {
    if (configured != dev) {
      cudaError_t e = cudaFuncSetAttribute(stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)StreamSmem::total);
      if (e != cudaSuccess) return e;
      configured = dev;
    }
    cudaError_t e = zero_exponents(b.eA, A.R, b.b_packed ? nullptr : b.eB, B.R, s);
    if (e != cudaSuccess) return e;
    if ((e = row_exponents_nozero(A, b.eA, s)) != cudaSuccess) return e;
    if (!b.b_packed) {
      if ((e = row_exponents_nozero(B, b.eB, s)) != cudaSuccess) return e;
      if ((e = pack(B, b.eB, kTileB, b.Bblob, s)) != cudaSuccess) return e;
    }
    StreamParams sp{};
    sp.A = A.M1;
    sp.lda = A.ld1;
    sp.mode = mode;
    sp.M = M;
    sp.K = K;
    sp.N = N;
    sp.eA = b.eA;
    sp.B = b.Bblob;
    sp.nkb = std::max(1, (K + kDepth - 1) / kDepth);
    sp.kb_per_split = (sp.nkb + splits - 1) / splits;
    const int used = (sp.nkb + sp.kb_per_split - 1) / sp.kb_per_split;
    sp.Phi = b.P;
    sp.sstride = (int64_t)M * N;
    sp.Plo = b.P + (size_t)used * sp.sstride;
    sp.ldp = M;
    sp.status = status;
    sp.limit_ns = limit_ns;
    sp.trace = prof::trace_take();
    prof::count_launch();
    if ((e = launch_pdl(stream_kernel, dim3((M + kTileA - 1) / kTileA, used), dim3(kStreamThreads), StreamSmem::total, s,
                        sp, lo, up)) != cudaSuccess)
      return e;
    GemmParams gp{};
    gp.Phi = sp.Phi;
    gp.Plo = sp.Plo;
    gp.ldp = sp.ldp;
    gp.sstride = sp.sstride;
    gp.eA = b.eA;
    gp.eB = b.eB;
    gp.M = M;
    gp.N = N;
    return reduce(gp, used, alpha, beta, C, ldc, s);
  };
  *err = run();
  return true;
}

}  // namespace

cudaError_t product(const Operand& A, const Operand& B, int M, int N, int K, double alpha, double beta, double* C,
                    int64_t ldc, const Bufs& b, int splits, int* status, unsigned long long limit_ns,
                    cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (K > 0 && stream_product(A, B, M, N, K, alpha, beta, C, ldc, b, splits, status, limit_ns, s, &e)) return e;
  e = prepare(A, B, b, s);
  if (e != cudaSuccess) return e;
  GemmParams p{};
  p.A = b.Ablob;
  p.B = b.Bblob;
  p.eA = b.eA;
  p.eB = b.eB;
  p.M = M;
  p.N = N;
  p.nkb = std::max(1, (K + kDepth - 1) / kDepth);
  p.kb_per_split = (p.nkb + splits - 1) / splits;
  const int used = (p.nkb + p.kb_per_split - 1) / p.kb_per_split;
  p.Phi = b.P;
  p.sstride = (int64_t)M * N;
  p.Plo = b.P + (size_t)used * p.sstride;
  p.ldp = M;
  p.status = status;
  p.limit_ns = limit_ns;
  p.trace = prof::trace_take();
  e = gemm(p, used, s);
  if (e != cudaSuccess) return e;
  return reduce(p, used, alpha, beta, C, ldc, s);
}

cudaError_t rank_apply(int M, int N, int K, double alpha, double* C, int64_t ldc, int col0, int col1, int lower,
                       const Bufs& b, int* status, unsigned long long limit_ns, cudaStream_t s, int max_ctas) {
  if (M <= 0 || N <= 0 || col1 <= col0) return cudaSuccess;
  GemmParams p{};
  p.A = b.Ablob;
  p.B = b.Bblob;
  p.eA = b.eA;
  p.eB = b.eB;
  p.M = M;
  p.N = N;
  p.nkb = std::max(1, (K + kDepth - 1) / kDepth);
  p.kb_per_split = p.nkb;
  p.C = C;
  p.ldc = ldc;
  p.col0 = col0;
  p.col1 = col1;
  p.lower = lower;
  p.alpha = alpha;
  p.status = status;
  p.limit_ns = limit_ns;
  p.trace = prof::trace_take();
  static int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  constexpr size_t smem = Smem::total + sizeof(int) * kMaxTilesPerCta;
  if (configured != dev) {
    cudaError_t e = cudaFuncSetAttribute(rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // tiles that hold part of the update: columns in [col0, col1), rows reaching the diagonal
  const int nI = (M + kTileA - 1) / kTileA, nJ = (N + kTileB - 1) / kTileB;
  int64_t valid = 0;
  for (int J = col0 / kTileB; J < nJ && J * kTileB < col1; ++J)
    valid += lower ? std::max(0, nI - (J * kTileB) / kTileA) : nI;
  if (valid == 0) return cudaSuccess;
  const int64_t all = (int64_t)nI * nJ;
  const int cap = max_ctas > 0 ? std::min(max_ctas, sms) : sms;
  const int grid =
      (int)std::max<int64_t>(std::min<int64_t>(cap, valid), (all + kMaxTilesPerCta - 1) / kMaxTilesPerCta);
  prof::count_launch();
  return launch_pdl(rank_kernel, dim3(grid), dim3(kRankThreads), smem, s, p);
}

}  // namespace ozaki
}  // namespace bandred
