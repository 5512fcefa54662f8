// Split-precision tensor-core products for the trailing updates (tcgen05, sm_103a).
//
// Every FP64 operand x is cut into S bf16 slices (x ~ s0 + s1 [+ s2], see tc::split_bf16)
// and a product A B is formed as the sum of the slice products A_s B_t with s + t < S
// (S = 2: three products, "bf16x3"; S = 3: six products, "bf16x6"), accumulated in FP32 in
// tensor memory.  Partial sums are recombined in FP64 every `kChunk` reduction steps, so
// the FP32 accumulation never runs over more than kChunk terms.
//
// Kernels:
//   pack_kernel         FP64 (R x K, optionally two matrices concatenated along K) ->
//                       bf16 slices in the canonical K-major core-matrix layout of
//                       tcgen05 operands, blocked into (TR x TK) tiles.
//   stream_gemm_kernel  C_partial = A B for a large FP64 A streamed from HBM and sliced in
//                       shared memory on the fly (plain, transposed, or symmetric with only
//                       the lower triangle stored), and a pre-packed thin B (N <= 128).
//                       Used for X1 = A2 W (Eq. updateA2symm), W^T E and D W_V.
//   rank_update_kernel  C += alpha A B^T for pre-packed A, B with a short reduction
//                       (Eq. updateA2syr2k on the lower triangle; Eqs. updateCD, updateD).
#include <algorithm>
#include <cstring>

#include <cuda.h>  // CUtensorMap and its enums (types only: the encoder is fetched at run time)

#include "common.cuh"
#include "kernels.h"
#include "launch.h"
#include "prof.h"
#include "split.h"
#include "tc.cuh"

namespace bandred {
namespace split {

namespace {

constexpr int NT = 256;
constexpr int BM = 128;       // rows of a C tile (TMEM lanes)
constexpr int BK = 32;        // reduction depth of one pipeline stage
constexpr int kChunk = 256;   // FP32 accumulation length before FP64 recombination
constexpr int RS = BM + 1;    // k-stride (doubles) of a staged FP64 tile: conflict-free
                              // for both the row-contiguous and the column-contiguous fill
constexpr int CH = kChunk / BK;

__device__ __forceinline__ void report(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ================================================================= pack
__global__ void pack_kernel(PackParams single, const PackParams* probs) {
  const PackParams p = probs ? probs[blockIdx.y] : single;
  if (p.R <= 0) return;
  pdl_wait_and_release();
  const int groups_per_tile = p.TR * (p.TK / 8);
  const int64_t total = (int64_t)p.nrb * p.nkb * groups_per_tile;
  const int K = p.K1 + p.K2;
  bool ok = true;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const int within = (int)(g % groups_per_tile);
    const int64_t tile = g / groups_per_tile;
    const int kb = (int)(tile % p.nkb), rb = (int)(tile / p.nkb);
    const int r = within % p.TR, kg = within / p.TR;
    const int row = rb * p.TR + r;
    uint32_t words[3][4];
#pragma unroll
    for (int kk = 0; kk < 8; kk += 2) {
      __nv_bfloat16 sl0[3], sl1[3];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = kb * p.TK + kg * 8 + kk + h;
        double x = 0.0;
        if (row < p.R && k < K) {
          if (k < p.K1)
            x = p.t1 ? p.M1[k + (int64_t)row * p.ld1] : p.M1[row + (int64_t)k * p.ld1];
          else
            x = p.t2 ? p.M2[(k - p.K1) + (int64_t)row * p.ld2] : p.M2[row + (int64_t)(k - p.K1) * p.ld2];
          x *= (k < p.K1) ? p.scale1 : p.scale2;
        }
        __nv_bfloat16 sl[3];
        ok &= tc::split_bf16<3>(x, sl);
#pragma unroll
        for (int s = 0; s < 3; ++s) (h ? sl1 : sl0)[s] = sl[s];
      }
#pragma unroll
      for (int s = 0; s < 3; ++s)
        words[s][kk / 2] = (uint32_t)__bfloat16_as_ushort(sl0[s]) | ((uint32_t)__bfloat16_as_ushort(sl1[s]) << 16);
    }
    const size_t tile_elems = (size_t)p.TR * p.TK;
    for (int s = 0; s < p.S; ++s) {
      __nv_bfloat16* base = p.out + ((size_t)tile * p.S + s) * tile_elems;
      uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<char*>(base) + tc::kmajor_offset(r, kg * 8, p.TR));
      *dst = make_uint4(words[s][0], words[s][1], words[s][2], words[s][3]);
    }
  }
  if (!ok) report(p.status, BANDRED_DEV_RANGE);
}

// ================================================================= stream GEMM
template <int S>
struct Products;
template <>
struct Products<2> {
  static constexpr int n = 3;
  __device__ static constexpr int s(int q) { return q == 2 ? 1 : 0; }
  __device__ static constexpr int t(int q) { return q == 1 ? 1 : 0; }
};
template <>
struct Products<3> {
  static constexpr int n = 6;
  // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
  __device__ static constexpr int s(int q) { return q == 2 ? 1 : (q == 4 ? 1 : (q == 5 ? 2 : 0)); }
  __device__ static constexpr int t(int q) { return q == 1 ? 1 : (q == 3 ? 2 : (q == 4 ? 1 : 0)); }
};

template <int BN, int S, int NSTAGE>
struct StreamSmem {
  static constexpr int NB = NSTAGE + 1;
  static constexpr size_t fp64_bytes = ((size_t)NSTAGE * BK * RS * 8 + 1023) / 1024 * 1024;
  static constexpr size_t aslice_bytes = (size_t)BM * BK * 2;  // one slice, one stage
  static constexpr size_t bslice_bytes = (size_t)BN * BK * 2;
  static constexpr size_t off_a = fp64_bytes;
  static constexpr size_t off_b = off_a + 2 * S * aslice_bytes;
  static constexpr size_t off_bar = off_b + (size_t)NB * S * bslice_bytes;
  static constexpr size_t total = off_bar + 64;
};

template <int BN, int S, int NSTAGE>
__global__ void __launch_bounds__(NT, 1) stream_gemm_kernel(StreamParams single, const StreamParams* probs) {
  using L = StreamSmem<BN, S, NSTAGE>;
  const StreamParams p = probs ? probs[blockIdx.z] : single;
  if (probs) {  // batched: this CTA's tile or split may lie beyond its problem
    if (p.M <= 0 || p.nkb <= 0 || (int)blockIdx.x * BM >= p.M) return;
    if ((int)blockIdx.y * p.stages_per_split >= p.nkb) return;
  }
  using PR = Products<S>;
  extern __shared__ __align__(1024) unsigned char smem[];
  double* ring = reinterpret_cast<double*>(smem);
  unsigned char* aslices = smem + L::off_a;
  unsigned char* bslices = smem + L::off_b;
  uint64_t* bar_mma = reinterpret_cast<uint64_t*>(smem + L::off_bar);  // [2]
  uint64_t* bar_acc = bar_mma + 2;                                       // [2]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar_acc + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * BM;
  const int z = blockIdx.y;
  const int st_begin = z * p.stages_per_split;
  const int st_end = min(p.nkb, st_begin + p.stages_per_split);
  const int nst = st_end - st_begin;
  constexpr uint32_t kTmemCols = 2 * BN;
  const unsigned long long deadline = global_ns() + p.limit_ns;

  if (tid == 0) {
    tc::mbar_init(&bar_mma[0], 1);
    tc::mbar_init(&bar_mma[1], 1);
    tc::mbar_init(&bar_acc[0], 1);
    tc::mbar_init(&bar_acc[1], 1);
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

  // ---- loads of one stage: the FP64 A tile (BK x BM, [k][i]) and the B slices
  auto issue_loads = [&](int ls) {
    const int kst = st_begin + ls;
    const int k0 = kst * BK;
    double* dst = ring + (size_t)(ls % NSTAGE) * BK * RS;
    const double* A = p.A;
    const int64_t lda = p.lda;
    bool lower_map = true;
    if (p.mode == kModeTrans) lower_map = false;
    if (p.mode == kModeSymLower && k0 >= i0 + BM - 1) lower_map = false;  // whole tile above the diagonal
    const bool mixed = p.mode == kModeSymLower && !(k0 + BK - 1 <= i0) && lower_map;
    if (lower_map) {
#pragma unroll 4
      for (int q = 0; q < (BK * BM) / NT; ++q) {
        const int i = tid & (BM - 1), k = (tid >> 7) + 2 * q;
        const int gi = i0 + i, gk = k0 + k;
        const bool in = gi < p.M && gk < p.K;
        const double* src = A;
        if (in) {
          if (mixed && gi < gk)
            src = A + gk + (int64_t)gi * lda;
          else
            src = A + gi + (int64_t)gk * lda;
        }
        tc::cp_async8(dst + k * RS + i, src, in ? 8u : 0u);
      }
    } else {
#pragma unroll 4
      for (int q = 0; q < (BK * BM) / NT; ++q) {
        const int k = tid & (BK - 1), i = (tid >> 5) + 8 * q;
        const int gi = i0 + i, gk = k0 + k;
        const bool in = gi < p.M && gk < p.K;
        const double* src = in ? A + gk + (int64_t)gi * lda : A;
        tc::cp_async8(dst + k * RS + i, src, in ? 8u : 0u);
      }
    }
    // B slices of this stage: S * BN * BK bf16, contiguous in the packed blob.
    const unsigned char* bsrc =
        reinterpret_cast<const unsigned char*>(p.Bblob) + (size_t)kst * S * L::bslice_bytes;
    unsigned char* bdst = bslices + (size_t)(ls % L::NB) * S * L::bslice_bytes;
    for (int c = tid; c < (int)(S * L::bslice_bytes / 16); c += NT) tc::cp_async16(bdst + 16 * c, bsrc + 16 * c);
  };

  double acc[BN / 2];
#pragma unroll
  for (int c = 0; c < BN / 2; ++c) acc[c] = 0.0;
  int timed_out = 0;
  bool range_ok = true;

  auto drain_chunk = [&](int c) {
    // all threads: wait for the chunk's MMAs, then add its FP32 sums into FP64 registers
    int to = tc::mbar_wait(&bar_acc[c & 1], (c >> 1) & 1, deadline) ? 0 : 1;
    tc::fence_after_sync();
    const uint32_t q = warp & 3, h = warp >> 2;
    const uint32_t taddr = tmem + ((q * 32) << 16) + (uint32_t)((c & 1) * BN + h * (BN / 2));
    if (!to) {
      if constexpr (BN / 2 >= 32) {
#pragma unroll
        for (int part = 0; part < BN / 64; ++part) {
          float v[32];
          tc::tmem_ld32(taddr + part * 32, v);
#pragma unroll
          for (int cc = 0; cc < 32; ++cc) acc[part * 32 + cc] += tc::f32_to_f64(v[cc]);
        }
      } else {
        float v[16];
        tc::tmem_ld16(taddr, v);
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) acc[cc] += tc::f32_to_f64(v[cc]);
      }
    }
    tc::fence_before_sync();
    return to;
  };

  for (int ls = 0; ls < NSTAGE - 1; ++ls) {
    if (ls < nst) issue_loads(ls);
    tc::cp_async_commit();
  }

  for (int st = 0; st < nst && !timed_out; ++st) {
    const int sb = st & 1;
    int to = 0;
    if (st >= 2) to = tc::mbar_wait(&bar_mma[sb], ((st - 2) >> 1) & 1, deadline) ? 0 : 1;
    if (__syncthreads_or(to)) {
      timed_out = 1;
      break;
    }
    const int ls = st + NSTAGE - 1;
    if (ls < nst) issue_loads(ls);
    tc::cp_async_commit();
    tc::cp_async_wait<NSTAGE - 1>();
    __syncthreads();

    // ---- convert the FP64 stage into S bf16 slices (K-major core layout)
    {
      const double* src = ring + (size_t)(st % NSTAGE) * BK * RS;
      unsigned char* adst = aslices + (size_t)sb * S * L::aslice_bytes;
#pragma unroll
      for (int q = 0; q < (BM * (BK / 8)) / NT; ++q) {
        const int i = tid & (BM - 1), kg = (tid >> 7) + 2 * q;
        uint32_t words[S][4];
#pragma unroll
        for (int kk = 0; kk < 8; kk += 2) {
          __nv_bfloat16 a[S], b[S];
          range_ok &= tc::split_bf16<S>(src[(kg * 8 + kk) * RS + i], a);
          range_ok &= tc::split_bf16<S>(src[(kg * 8 + kk + 1) * RS + i], b);
#pragma unroll
          for (int s = 0; s < S; ++s)
            words[s][kk / 2] = (uint32_t)__bfloat16_as_ushort(a[s]) | ((uint32_t)__bfloat16_as_ushort(b[s]) << 16);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
          uint4* d = reinterpret_cast<uint4*>(adst + s * L::aslice_bytes + tc::kmajor_offset(i, kg * 8, BM));
          *d = make_uint4(words[s][0], words[s][1], words[s][2], words[s][3]);
        }
      }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();

    // ---- one thread issues the slice-pair MMAs of this stage
    const int chunk = st / CH;
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t d = tmem + (uint32_t)((chunk & 1) * BN);
      constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
      const uint32_t abase = tc::smem_u32(aslices + (size_t)sb * S * L::aslice_bytes);
      const uint32_t bbase = tc::smem_u32(bslices + (size_t)(st % L::NB) * S * L::bslice_bytes);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
        for (int q = 0; q < PR::n; ++q) {
          const uint64_t ad = tc::smem_desc(abase + PR::s(q) * L::aslice_bytes + kk * 2 * (BM / 8) * 128,
                                            (BM / 8) * 128, 128);
          const uint64_t bd = tc::smem_desc(bbase + PR::t(q) * L::bslice_bytes + kk * 2 * (BN / 8) * 128,
                                            (BN / 8) * 128, 128);
          const uint32_t accum = (st % CH == 0 && kk == 0 && q == 0) ? 0u : 1u;
          tc::mma_bf16(d, ad, bd, idesc, accum);
        }
      }
      tc::mma_commit(&bar_mma[sb]);
      if (st % CH == CH - 1 || st == nst - 1) tc::mma_commit(&bar_acc[chunk & 1]);
    }

    // ---- FP64 recombination of the previous chunk, one stage into the next one
    if (st % CH == 0 && st > 0) {
      to = drain_chunk(chunk - 1);
      if (__syncthreads_or(to)) timed_out = 1;
    }
  }
  if (!timed_out && nst > 0) {
    const int last = (nst - 1) / CH;
    const int to = drain_chunk(last);
    if (__syncthreads_or(to)) timed_out = 1;
  }
  tc::cp_async_wait_all();

  if (timed_out) {
    report(p.status, BANDRED_DEV_TIMEOUT);
  } else {
    const int q = warp & 3, h = warp >> 2;
    const int row = i0 + q * 32 + lane;
    double* P = p.P + (size_t)z * p.split_stride;
    if (row < p.M) {
#pragma unroll
      for (int c = 0; c < BN / 2; ++c) {
        const int col = h * (BN / 2) + c;
        if (col < p.N) P[row + (int64_t)col * p.ldp] = acc[c];
      }
    }
  }
  if (!__syncthreads_and(range_ok ? 1 : 0) && tid == 0) report(p.status, BANDRED_DEV_RANGE);
  // Let any MMA still in flight finish before TMEM is released (bounded).
  if (timed_out && tid == 0) {
    const unsigned long long dl = global_ns() + p.limit_ns;
    for (int b = 0; b < 2; ++b) tc::mbar_wait(&bar_mma[b], 0, dl);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// ================================================================= stream GEMM, TMA
// The same product as stream_gemm_kernel with the FP64 tiles moved by the tensor-memory
// accelerator: a stage is one 2-D box of the tensor map (128 rows x 32 k, or for tiles
// read transposed two 16 x 128 boxes in the 128-byte swizzled layout, whose rows a warp
// reads without bank conflicts) plus one bulk copy of the packed B slices, both
// completing on the stage's mbarrier, loaded two stages ahead into a ring of four.  Tiles
// that cross the diagonal of a symmetric A take the lower box and fetch their upper
// entries from the mirror position directly.  Slicing works on pairs of entries with
// integer and FP32 operations (tc::split_pair), and the FP32 chunk sums are accumulated
// as double-float pairs, so the streamed elements cost no FP64 instruction.
template <int BN, int S>
struct TmaSmem {
  static constexpr int NS = 4;
  static constexpr size_t tile_bytes = (size_t)BM * BK * 8;
  static constexpr size_t aslice_bytes = (size_t)BM * BK * 2;
  static constexpr size_t bslice_bytes = (size_t)BN * BK * 2;
  static constexpr size_t bstage_bytes = (size_t)S * bslice_bytes;
  static constexpr size_t off_b = (size_t)NS * tile_bytes;
  static constexpr size_t off_a = off_b + (size_t)NS * bstage_bytes;
  static constexpr size_t off_bar = off_a + 2 * (size_t)S * aslice_bytes;
  static constexpr size_t total = off_bar + 128 + 1024;  // + alignment of the base to 1024
};

constexpr int kTmaThreads = NT + 32;  // eight converter warps and one control warp

template <int BN, int S>
__global__ void __launch_bounds__(kTmaThreads, 1)
    stream_tma_kernel(StreamParams p, const __grid_constant__ CUtensorMap tm_lower,
                      const __grid_constant__ CUtensorMap tm_upper) {
  using L = TmaSmem<BN, S>;
  constexpr int NS = L::NS;
  using PR = Products<S>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  double* ring = reinterpret_cast<double*>(smem);
  unsigned char* bring = smem + L::off_b;
  unsigned char* aslices = smem + L::off_a;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::off_bar);  // [NS] copies landed
  uint64_t* sliced = full + NS;                                       // [2] slices written
  uint64_t* bar_mma = sliced + 2;                                     // [2] MMAs of a stage done
  uint64_t* bar_acc = bar_mma + 2;                                    // [2] MMAs of a chunk done
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar_acc + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * BM;
  const int z = blockIdx.y;
  const int st_begin = z * p.stages_per_split;
  const int st_end = min(p.nkb, st_begin + p.stages_per_split);
  const int nst = st_end - st_begin;
  constexpr uint32_t kTmemCols = 2 * BN;
  constexpr int kConvWarps = NT / 32;
  const unsigned long long deadline = global_ns() + p.limit_ns;

  if (tid == 0) {
    for (int q = 0; q < NS; ++q) tc::mbar_init(&full[q], 1);
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&sliced[q], kConvWarps);
      tc::mbar_init(&bar_mma[q], 1);
      tc::mbar_init(&bar_acc[q], 1);
    }
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

  // 0: every entry of the tile read in place (A(i, k) at A[i + k lda]); 1: every entry read
  // transposed (A[k + i lda]); 2: a symmetric tile across the diagonal
  auto kind_of = [&](int kst) -> int {
    if (p.mode == kModePlain) return 0;
    if (p.mode == kModeTrans) return 1;
    const int k0 = kst * BK;
    if (k0 + BK - 1 <= i0) return 0;
    if (k0 >= i0 + BM - 1) return 1;
    return 2;
  };

  int timed_out = 0;
  bool range_ok = true;
  float acc_hi[BN / 2], acc_lo[BN / 2];
#pragma unroll
  for (int c = 0; c < BN / 2; ++c) acc_hi[c] = acc_lo[c] = 0.0f;

  if (warp == kConvWarps) {
    // ---------------- control warp, one lane: TMA copies three stages ahead, MMAs
    if (lane == 0 && nst > 0) {
      tc::prefetch_tmap(&tm_lower);
      tc::prefetch_tmap(&tm_upper);
      auto issue = [&](int ls) {
        const int kst = st_begin + ls, slot = ls % NS, k0 = kst * BK;
        double* dst = ring + (size_t)slot * BM * BK;
        tc::mbar_arrive_expect_tx(&full[slot], (uint32_t)(L::tile_bytes + L::bstage_bytes));
        if (kind_of(kst) == 1) {
          tc::tma_load_2d(dst, &tm_upper, k0, i0, &full[slot]);
          tc::tma_load_2d(dst + BM * 16, &tm_upper, k0 + 16, i0, &full[slot]);
        } else {
          tc::tma_load_2d(dst, &tm_lower, i0, k0, &full[slot]);
        }
        tc::bulk_g2s(bring + (size_t)slot * L::bstage_bytes,
                     reinterpret_cast<const unsigned char*>(p.Bblob) + (size_t)kst * L::bstage_bytes,
                     (uint32_t)L::bstage_bytes, &full[slot]);
      };
      int issued = 0;
      for (; issued < NS - 1 && issued < nst; ++issued) issue(issued);
      for (int st = 0; st < nst; ++st) {
        if (!tc::mbar_wait(&sliced[st & 1], (uint32_t)(st >> 1) & 1u, deadline)) {
          timed_out = 1;
          break;
        }
        tc::fence_after_sync();
        const int chunk = st / CH;
        const uint32_t d = tmem + (uint32_t)((chunk & 1) * BN);
        constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
        const uint32_t abase = tc::smem_u32(aslices + (size_t)(st & 1) * S * L::aslice_bytes);
        const uint32_t bbase = tc::smem_u32(bring + (size_t)(st % NS) * L::bstage_bytes);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
          for (int q = 0; q < PR::n; ++q) {
            const uint64_t ad = tc::smem_desc(abase + PR::s(q) * L::aslice_bytes + kk * 2 * (BM / 8) * 128,
                                              (BM / 8) * 128, 128);
            const uint64_t bd = tc::smem_desc(bbase + PR::t(q) * L::bslice_bytes + kk * 2 * (BN / 8) * 128,
                                              (BN / 8) * 128, 128);
            const uint32_t accum = (st % CH == 0 && kk == 0 && q == 0) ? 0u : 1u;
            tc::mma_bf16(d, ad, bd, idesc, accum);
          }
        }
        tc::mma_commit(&bar_mma[st & 1]);
        if (st % CH == CH - 1 || st == nst - 1) tc::mma_commit(&bar_acc[chunk & 1]);
        // refill the slot of stage st - 1 once its MMAs (readers of its B slices) are done
        if (issued < nst) {
          if (st >= 1 && !tc::mbar_wait(&bar_mma[(st - 1) & 1], (uint32_t)((st - 1) >> 1) & 1u, deadline)) {
            timed_out = 1;
            break;
          }
          issue(issued++);
        }
      }
      if (timed_out) {  // let copies and MMAs in flight land before the CTA leaves (bounded)
        const unsigned long long dl = global_ns() + p.limit_ns;
        for (int q = 0; q < NS; ++q) tc::mbar_wait(&full[q], 0, dl);
        for (int q = 0; q < 2; ++q) tc::mbar_wait(&bar_mma[q], 0, dl);
      }
    }
  } else {
    // ---------------- converter warps: FP64 stage -> bf16 slices; chunk sums -> (hi, lo)
    const int ti = tid & (BM - 1), half = tid >> 7;  // row ti, k in [16 half, 16 half + 16)
    auto drain_chunk = [&](int c) -> bool {
      if (!tc::mbar_wait(&bar_acc[c & 1], (c >> 1) & 1, deadline)) return false;
      tc::fence_after_sync();
      const uint32_t q = warp & 3, h = warp >> 2;
      const uint32_t taddr = tmem + ((q * 32) << 16) + (uint32_t)((c & 1) * BN + h * (BN / 2));
      auto add = [&](int cc, float v) {  // (hi, lo) += v, error-free (Knuth's two-sum)
        const float s2 = acc_hi[cc] + v;
        const float bb = s2 - acc_hi[cc];
        const float err = (acc_hi[cc] - (s2 - bb)) + (v - bb);
        acc_hi[cc] = s2;
        acc_lo[cc] += err;
      };
      if constexpr (BN / 2 >= 32) {
#pragma unroll
        for (int part = 0; part < BN / 64; ++part) {
          float v[32];
          tc::tmem_ld32(taddr + part * 32, v);
#pragma unroll
          for (int cc = 0; cc < 32; ++cc) add(part * 32 + cc, v[cc]);
        }
      } else {
        float v[16];
        tc::tmem_ld16(taddr, v);
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) add(cc, v[cc]);
      }
      tc::fence_before_sync();
      return true;
    };
    for (int st = 0; st < nst; ++st) {
      const int sb = st & 1, slot = st % NS;
      const int kst = st_begin + st, k0 = kst * BK;
      const int kind = kind_of(kst);
      double x[16];
      const int gi = i0 + ti;
      if (kind == 2) {  // upper entries of a diagonal tile, from the stored mirror A(k, i)
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          const int gk = k0 + 16 * half + kk;
          x[kk] = (gi < gk && gk < p.K && gi < p.M) ? __ldg(p.A + gk + (int64_t)gi * p.lda) : 0.0;
        }
      }
      if (!tc::mbar_wait(&full[slot], (uint32_t)(st / NS) & 1u, deadline) ||
          (st >= 2 && !tc::mbar_wait(&bar_mma[sb], (uint32_t)((st - 2) >> 1) & 1u, deadline))) {
        timed_out = 1;
        break;
      }
      const double* tile = ring + (size_t)slot * BM * BK;
      if (kind == 1) {
        const double* box = tile + half * (BM * 16) + ti * 16;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const double2 v = *reinterpret_cast<const double2*>(box + 2 * (c ^ (ti & 7)));
          x[2 * c] = v.x;
          x[2 * c + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          const double v = tile[(16 * half + kk) * BM + ti];
          if (kind == 0 || gi >= k0 + 16 * half + kk) x[kk] = v;
        }
      }
      unsigned char* adst = aslices + (size_t)sb * S * L::aslice_bytes;
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        uint32_t w[4][S];
#pragma unroll
        for (int c = 0; c < 4; ++c) range_ok &= tc::split_pair<S>(x[8 * g + 2 * c], x[8 * g + 2 * c + 1], w[c]);
        const uint32_t off = tc::kmajor_offset(ti, (2 * half + g) * 8, BM);
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
          *reinterpret_cast<uint4*>(adst + sl * L::aslice_bytes + off) =
              make_uint4(w[0][sl], w[1][sl], w[2][sl], w[3][sl]);
      }
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&sliced[sb]);
      if (st % CH == 0 && st > 0 && !drain_chunk(st / CH - 1)) {
        timed_out = 1;
        break;
      }
    }
    if (!timed_out && nst > 0 && !drain_chunk((nst - 1) / CH)) timed_out = 1;
  }

  if (__syncthreads_or(timed_out)) {
    if (tid == 0) report(p.status, BANDRED_DEV_TIMEOUT);
  } else if (warp < kConvWarps) {
    const int q = warp & 3, h = warp >> 2;
    const int row = i0 + q * 32 + lane;
    double* P = p.P + (size_t)z * p.split_stride;
    if (row < p.M) {
#pragma unroll
      for (int c = 0; c < BN / 2; ++c) {
        const int col = h * (BN / 2) + c;
        if (col < p.N) P[row + (int64_t)col * p.ldp] = tc::f32_to_f64(acc_hi[c]) + tc::f32_to_f64(acc_lo[c]);
      }
    }
  }
  if (!__syncthreads_and(range_ok ? 1 : 0) && tid == 0) report(p.status, BANDRED_DEV_RANGE);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// ================================================================= rank update
constexpr int RK = 64;  // reduction depth per smem load

template <int S>
struct RankSmem {
  static constexpr size_t slice_bytes = (size_t)BM * RK * 2;
  static constexpr size_t off_b = (size_t)S * slice_bytes;
  static constexpr size_t off_bar = off_b + (size_t)S * slice_bytes;
  static constexpr size_t total = off_bar + 64;
};

template <int S>
__global__ void __launch_bounds__(NT, 2) rank_update_kernel(RankParams single, const RankParams* probs) {
  using L = RankSmem<S>;
  using PR = Products<S>;
  const RankParams p = probs ? probs[blockIdx.z] : single;
  const int I = blockIdx.x, J = p.tj0 + blockIdx.y;
  if (p.M <= 0 || p.N <= 0 || p.col1 <= p.col0) return;
  if (I * BM >= p.M || J * BM >= min(p.N, p.col1)) return;
  if (p.lower && I < J) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* as = smem;
  unsigned char* bs = smem + L::off_b;
  uint64_t* bar_ld = reinterpret_cast<uint64_t*>(smem + L::off_bar);
  uint64_t* bar_mma = bar_ld + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar_mma + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned long long deadline = global_ns() + p.limit_ns;
  if (tid == 0) {
    tc::mbar_init(bar_ld, 1);
    tc::mbar_init(bar_mma, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_holder, BM);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  pdl_wait_and_release();
  const int nkb = p.Kr / RK;
  const size_t blk = (size_t)S * L::slice_bytes;  // one (row block, K block) of a blob
  // Start fetching this CTA's C tile into L2 now, so the epilogue's reads overlap the
  // slice copies and the MMAs instead of following them: one 128-byte line per
  // (column, 16-row group), columns this CTA will update.
  {
    const int row0 = I * BM;
    for (int q = tid; q < BM * (BM / 16); q += NT) {
      const int col = J * BM + q / (BM / 16), r = row0 + (q % (BM / 16)) * 16;
      if (r < p.M && col < p.N && col >= p.col0 && col < p.col1 && (!p.lower || r + 15 >= col))
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p.C + r + (int64_t)col * p.ldc));
    }
  }
  int to = 0;
  for (int kb = 0; kb < nkb && !to; ++kb) {
    if (tid == 0) {
      tc::mbar_arrive_expect_tx(bar_ld, (uint32_t)(2 * blk));
      tc::bulk_g2s(as, reinterpret_cast<const unsigned char*>(p.Ablob) + ((size_t)I * nkb + kb) * blk,
                   (uint32_t)blk, bar_ld);
      tc::bulk_g2s(bs, reinterpret_cast<const unsigned char*>(p.Bblob) + ((size_t)J * nkb + kb) * blk,
                   (uint32_t)blk, bar_ld);
      int t = tc::mbar_wait(bar_ld, kb & 1, deadline) ? 0 : 1;
      if (!t) {
        tc::fence_after_sync();
        constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BM);
        const uint32_t ab = tc::smem_u32(as), bb = tc::smem_u32(bs);
#pragma unroll
        for (int kk = 0; kk < RK / 16; ++kk)
#pragma unroll
          for (int q = 0; q < PR::n; ++q) {
            const uint64_t ad = tc::smem_desc(ab + PR::s(q) * L::slice_bytes + kk * 2 * (BM / 8) * 128, (BM / 8) * 128, 128);
            const uint64_t bd = tc::smem_desc(bb + PR::t(q) * L::slice_bytes + kk * 2 * (BM / 8) * 128, (BM / 8) * 128, 128);
            tc::mma_bf16(tmem, ad, bd, idesc, (kb == 0 && kk == 0 && q == 0) ? 0u : 1u);
          }
        tc::mma_commit(bar_mma);
        t = tc::mbar_wait(bar_mma, kb & 1, deadline) ? 0 : 1;
      }
      to = t;
    }
    to = __syncthreads_or(to);
  }
  if (!to) {
    tc::fence_after_sync();
    const int q = warp & 3, h = warp >> 2;
    const int row = I * BM + q * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 64);
    const bool unit_alpha = p.alpha == 1.0;
    // 16 columns at a time (two CTAs fit an SM: one's epilogue overlaps the other's
    // copies and MMAs); all loads of a part are issued before its stores.
#pragma unroll 1
    for (int part = 0; part < 4; ++part) {
      float v[16];
      tc::tmem_ld16(taddr + part * 16, v);
      const int colb = J * BM + h * 64 + part * 16;
      double old[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int col = colb + c;
        const bool in = row < p.M && col < p.N && col >= p.col0 && col < p.col1 && (!p.lower || row >= col);
        old[c] = in ? p.C[row + (int64_t)col * p.ldc] : 0.0;
      }
      // one FP64 instruction per entry (the FP64 pipe bounds this epilogue): alpha = 1
      // adds, other values take the FMA in a separate, uniform branch
      if (unit_alpha) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int col = colb + c;
          const bool in = row < p.M && col < p.N && col >= p.col0 && col < p.col1 && (!p.lower || row >= col);
          if (in) p.C[row + (int64_t)col * p.ldc] = old[c] + tc::f32_to_f64(v[c]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int col = colb + c;
          const bool in = row < p.M && col < p.N && col >= p.col0 && col < p.col1 && (!p.lower || row >= col);
          if (in) p.C[row + (int64_t)col * p.ldc] = fma(p.alpha, tc::f32_to_f64(v[c]), old[c]);
        }
      }
    }
  } else if (tid == 0) {
    report(p.status, BANDRED_DEV_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, BM);
  }
}

// ================================================================= split-K reduce
__global__ void reduce_kernel(ReduceParams single, const ReduceParams* probs) {
  const ReduceParams r = probs ? probs[blockIdx.y] : single;
  pdl_wait_and_release();
  const int64_t total = (int64_t)r.M * r.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % r.M), c = (int)(e / r.M);
    double s = 0.0;
    for (int z = 0; z < r.splits; ++z) s += r.P[(size_t)z * r.sstride + i + (int64_t)c * r.ldp];
    double* cp = &r.C[i + (int64_t)c * r.ldc];
    *cp = (r.beta == 0.0) ? r.alpha * s : fma(r.alpha, s, r.beta * *cp);
  }
}

// The same sums for outputs with many splits (the b x b product X1^T W splits its long
// reduction over up to 256 CTAs): 32 consecutive outputs per block, the splits dealt to the
// block's eight warps (z = warp, warp + 8, ...) and the eight partial sums added in warp
// order, so a thread waits on about splits / 8 loads instead of all of them.  The order
// is fixed, so results repeat bit for bit.
constexpr int kWideSplits = 8;  // splits above which reduce() takes this kernel
__global__ void __launch_bounds__(256) reduce_wide_kernel(ReduceParams r) {
  __shared__ double part[8][32];
  pdl_wait_and_release();
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
  const int64_t total = (int64_t)r.M * r.N;
  const int64_t e = blockIdx.x * 32ll + lane;
  const bool live = e < total;
  const int i = live ? (int)(e % r.M) : 0, c = live ? (int)(e / r.M) : 0;
  double s0 = 0.0, s1 = 0.0;
  if (live) {
    const double* src = r.P + i + (int64_t)c * r.ldp;
    int z = wy;
#pragma unroll 4
    for (; z + 8 < r.splits; z += 16) {
      s0 += src[(size_t)z * r.sstride];
      s1 += src[(size_t)(z + 8) * r.sstride];
    }
    if (z < r.splits) s0 += src[(size_t)z * r.sstride];
  }
  part[wy][lane] = s0 + s1;
  __syncthreads();
  if (wy == 0 && live) {
    double v = part[0][lane];
#pragma unroll
    for (int q = 1; q < 8; ++q) v += part[q][lane];
    double* cp = &r.C[i + (int64_t)c * r.ldc];
    *cp = (r.beta == 0.0) ? r.alpha * v : fma(r.alpha, v, r.beta * *cp);
  }
}

template <int BN, int S, int NSTAGE>
cudaError_t launch_stream(const StreamParams& p, const StreamParams* probs, dim3 grid, cudaStream_t s) {
  using L = StreamSmem<BN, S, NSTAGE>;
  static_assert(L::total <= 227 * 1024, "stream GEMM shared memory");
  static int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    cudaError_t e = cudaFuncSetAttribute(stream_gemm_kernel<BN, S, NSTAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L::total);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  prof::count_launch();
  if (probs) {
    stream_gemm_kernel<BN, S, NSTAGE><<<grid, NT, L::total, s>>>(p, probs);
    return cudaGetLastError();
  }
  return launch_pdl(stream_gemm_kernel<BN, S, NSTAGE>, grid, dim3(NT), L::total, s, p, probs);
}

template <int BN, int S>
cudaError_t launch_stream_tma(const StreamParams& p, const CUtensorMap& lo, const CUtensorMap& up, dim3 grid,
                              cudaStream_t s) {
  using L = TmaSmem<BN, S>;
  static_assert(L::total <= 227 * 1024, "TMA stream GEMM shared memory");
  static int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    cudaError_t e =
        cudaFuncSetAttribute(stream_tma_kernel<BN, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::total);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  prof::count_launch();
  return launch_pdl(stream_tma_kernel<BN, S>, grid, dim3(kTmaThreads), L::total, s, p, lo, up);
}

// cuTensorMapEncodeTiled, fetched from the driver once (the library links no libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  return fn;
}

// FP64 column-major rows x cols matrix with leading dimension ld, boxes of box0 (along
// the rows) x box1; `swz` selects the 128-byte swizzle.
bool encode_f64(CUtensorMap* m, const double* base, int64_t rows, int64_t cols, int64_t ld, uint32_t box0,
                uint32_t box1, bool swz) {
  EncodeTiledFn fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  const cuuint32_t box[2] = {box0, box1};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of the streamed operand when the TMA kernel can take it: 16-byte aligned
// base, even leading dimension (16-byte row stride), N <= 64.
bool stream_maps(const StreamParams& p, CUtensorMap* lo, CUtensorMap* up) {
  if (stream_bn(p.N) > 64 || p.M <= 0 || p.K <= 0) return false;
  if ((reinterpret_cast<uintptr_t>(p.A) & 15u) != 0 || (p.lda & 1) != 0) return false;
  bool ok = true;
  if (p.mode == kModePlain || p.mode == kModeSymLower) {
    if (p.lda < p.M) return false;
    ok = ok && encode_f64(lo, p.A, p.M, p.K, p.lda, BM, BK, false);
  }
  if (p.mode == kModeTrans || p.mode == kModeSymLower) {
    if (p.lda < p.K) return false;
    ok = ok && encode_f64(up, p.A, p.K, p.M, p.lda, 16, BM, true);
  }
  if (!ok) return false;
  if (p.mode == kModePlain) std::memcpy(up, lo, sizeof(CUtensorMap));
  if (p.mode == kModeTrans) std::memcpy(lo, up, sizeof(CUtensorMap));
  return true;
}

template <int S>
cudaError_t launch_rank(const RankParams& p, const RankParams* probs, dim3 grid, cudaStream_t s) {
  using L = RankSmem<S>;
  static int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    cudaError_t e =
        cudaFuncSetAttribute(rank_update_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::total);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  prof::count_launch();
  if (probs) {
    rank_update_kernel<S><<<grid, NT, L::total, s>>>(p, probs);
    return cudaGetLastError();
  }
  return launch_pdl(rank_update_kernel<S>, grid, dim3(NT), L::total, s, p, probs);
}

}  // namespace

// ================================================================= host API
bool encode_tile_map_f64(CUtensorMap* m, const double* base, int64_t rows, int64_t cols, int64_t ld, uint32_t box0,
                         uint32_t box1, bool swz) {
  return encode_f64(m, base, rows, cols, ld, box0, box1, swz);
}

int slices_of(int precision) { return precision == BANDRED_BF16X3 ? 2 : 3; }

size_t packed_bytes(int R, int K, int TR, int TK, int S) {
  const size_t nrb = (R + TR - 1) / TR, nkb = (K + TK - 1) / TK;
  return nrb * nkb * (size_t)S * TR * TK * 2;
}

cudaError_t pack(const PackParams& pp, cudaStream_t s) {
  const int64_t total = (int64_t)pp.nrb * pp.nkb * pp.TR * (pp.TK / 8);
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  prof::count_launch();
  return launch_pdl(pack_kernel, dim3(blocks), dim3(256), 0, s, pp, (const PackParams*)nullptr);
}

cudaError_t pack_batched(const PackParams* probs, int nprob, int64_t max_groups, cudaStream_t s) {
  if (nprob <= 0 || max_groups <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((max_groups + 255) / 256, 1024);
  pack_kernel<<<dim3(blocks, nprob), 256, 0, s>>>(PackParams{}, probs);
  prof::count_launch();
  return cudaGetLastError();
}

int stream_bn(int N) { return N <= 32 ? 32 : (N <= 64 ? 64 : 128); }

template <int S>
static cudaError_t stream_dispatch(int BN, const StreamParams& p, const StreamParams* probs, dim3 grid,
                                   cudaStream_t s) {
  if (BN == 32) return launch_stream<32, S, 3>(p, probs, grid, s);
  if (BN == 64) return launch_stream<64, S, 3>(p, probs, grid, s);
  return launch_stream<128, S, 2>(p, probs, grid, s);
}

cudaError_t stream_gemm(const StreamParams& p, int S, int splits, cudaStream_t s) {
  const int BN = stream_bn(p.N);
  const dim3 grid((p.M + BM - 1) / BM, splits);
  alignas(64) CUtensorMap lo, up;
  if (stream_maps(p, &lo, &up)) {
    if (S == 2) return BN == 32 ? launch_stream_tma<32, 2>(p, lo, up, grid, s) : launch_stream_tma<64, 2>(p, lo, up, grid, s);
    return BN == 32 ? launch_stream_tma<32, 3>(p, lo, up, grid, s) : launch_stream_tma<64, 3>(p, lo, up, grid, s);
  }
  return S == 2 ? stream_dispatch<2>(BN, p, nullptr, grid, s) : stream_dispatch<3>(BN, p, nullptr, grid, s);
}

cudaError_t stream_gemm_batched(const StreamParams* probs, int nprob, int S, int BN, int max_tiles, int max_splits,
                                cudaStream_t s) {
  if (nprob <= 0 || max_tiles <= 0 || max_splits <= 0) return cudaSuccess;
  const dim3 grid(max_tiles, max_splits, nprob);
  return S == 2 ? stream_dispatch<2>(BN, StreamParams{}, probs, grid, s)
                : stream_dispatch<3>(BN, StreamParams{}, probs, grid, s);
}

cudaError_t reduce(int M, int N, int splits, const double* P, int64_t ldp, int64_t sstride, double alpha, double beta,
                   double* C, int64_t ldc, cudaStream_t s) {
  const int64_t total = (int64_t)M * N;
  if (total <= 0) return cudaSuccess;
  ReduceParams r{M, N, splits, P, ldp, sstride, alpha, beta, C, ldc};
  if (splits > kWideSplits) {
    prof::count_launch();
    return launch_pdl(reduce_wide_kernel, dim3((unsigned)((total + 31) / 32)), dim3(256), 0, s, r);
  }
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 2048);
  prof::count_launch();
  return launch_pdl(reduce_kernel, dim3(blocks), dim3(256), 0, s, r, (const ReduceParams*)nullptr);
}

cudaError_t reduce_batched(const ReduceParams* probs, int nprob, int64_t max_total, cudaStream_t s) {
  if (nprob <= 0 || max_total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((max_total + 255) / 256, 256);
  reduce_kernel<<<dim3(blocks, nprob), 256, 0, s>>>(ReduceParams{}, probs);
  prof::count_launch();
  return cudaGetLastError();
}

cudaError_t rank_update(const RankParams& p, int S, int tiles_i, int tiles_j, cudaStream_t s) {
  if (tiles_i <= 0 || tiles_j <= 0) return cudaSuccess;
  const dim3 grid(tiles_i, tiles_j);
  return S == 2 ? launch_rank<2>(p, nullptr, grid, s) : launch_rank<3>(p, nullptr, grid, s);
}

cudaError_t rank_update_batched(const RankParams* probs, int nprob, int S, int max_ti, int max_tj, cudaStream_t s) {
  if (nprob <= 0 || max_ti <= 0 || max_tj <= 0) return cudaSuccess;
  const dim3 grid(max_ti, max_tj, nprob);
  return S == 2 ? launch_rank<2>(RankParams{}, probs, grid, s) : launch_rank<3>(RankParams{}, probs, grid, s);
}

}  // namespace split
}  // namespace bandred
