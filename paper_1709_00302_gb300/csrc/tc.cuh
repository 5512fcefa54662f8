// Inline-PTX wrappers for the Blackwell (sm_103a) tensor-core path: mbarriers, bulk and
// asynchronous copies into shared memory, TMEM allocation, tcgen05.mma/commit/ld, and the
// shared-memory matrix and instruction descriptors of tcgen05.mma.kind::f16.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>

#include "common.cuh"

namespace bandred {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity to complete; false when the deadline passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long deadline) {
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() > deadline) return false;
  }
  return true;
}

// ---------------------------------------------------------------- copies
// Bulk copy global -> shared (TMA engine, untiled); bytes and both addresses 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Tiled 2-D tensor copy global -> shared (TMA): the box of the tensor map at element
// coordinates (x, y), x along the contiguous dimension; x * 8 bytes must be a multiple of
// 16 for FP64 maps.  Completes on *bar with the box's byte count (out-of-range elements
// are written as zeros and counted).
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

// 8-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp_async8(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Generic-proxy shared-memory writes -> visible to the async proxy (tcgen05.mma operands).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Orders this thread's view of global memory (including writes by other CTAs that an
// acquire has made visible) before its later bulk copies, which read through the async
// proxy.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// ---------------------------------------------------------------- TMEM
// Whole warp: allocates ncols (power of two, >= 32) columns; the address lands in *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---------------------------------------------------------------- MMA
// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (bf16 inputs, FP32 accumulation), one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives once on *bar when every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Instruction descriptor: BF16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle.  K-major canonical layout: 8 x 16-byte
// core matrices; lbo = byte distance between core matrices adjacent along K, sbo = byte
// distance between core matrices adjacent along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;
}

// Byte offset of element (r, k) of an R x K bf16 operand tile in the K-major canonical
// layout used here: core matrix (r/8, k/8) at (k/8) * (R/8) * 128 + (r/8) * 128.
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int r, int k, int R) {
  return (uint32_t)((k >> 3) * (R >> 3) * 128 + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// ---------------------------------------------------------------- TMEM -> registers
// 32 lanes x 32 consecutive FP32 columns: thread t of the warp gets lane (base lane + t).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// FP32 -> FP64 by bit manipulation: the conversion instruction runs on the FP64 pipe,
// which GB300 issues at two operations per clock per SM.  Branch-free (a predicated
// conversion would still occupy the FP64 pipe): Inf and NaN keep their class, FP32
// subnormals become zero of the same sign.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint32_t m = e == 0u ? 0u : (u & 0x7FFFFFu);
  const uint32_t e64 = e == 0u ? 0u : (e == 0xFFu ? 0x7FFu : e + 896u);
  return __hiloint2double((int)((u & 0x80000000u) | (e64 << 20) | (m >> 3)), (int)(m << 29));
}

// ---------------------------------------------------------------- FP64 -> bf16 slices
// x ~= s0 + s1 (+ s2): s0 is x truncated to bf16 (8 significant bits, exponent kept),
// s1 = bf16_rn(x - s0), s2 = bf16_rn(x - s0 - s1).  Integer and FP32 operations only (the
// FP64 pipe of GB300 is ~60x slower than FP32).  The remainder x - s0 is carried with its
// leading 24 bits, so s0 + s1 + s2 agrees with x to about 2^-24 relative.
// Exact for 2^-95 <= |x| < 2^127; returns false (and zero slices) outside that range
// unless x == 0.
template <int S>
__device__ __forceinline__ bool split_bf16(double x, __nv_bfloat16 (&out)[S]) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(u >> 63);
  const int e = (int)((u >> 52) & 0x7FF);
  const __nv_bfloat16 z = __ushort_as_bfloat16((unsigned short)0);
#pragma unroll
  for (int s = 0; s < S; ++s) out[s] = z;
  if (e == 0) return ((u << 1) == 0ull);  // zero: fine; subnormal: out of range
  if (e < 928 || e > 1149) return false;  // keeps s0 and the scaled remainder normal
  const uint32_t hi = (sign << 15) | ((uint32_t)(e - 896) << 7) | (uint32_t)((u >> 45) & 0x7F);
  out[0] = __ushort_as_bfloat16((unsigned short)hi);
  if (S > 1) {
    const uint32_t r24 = (uint32_t)((u >> 21) & 0xFFFFFFull);  // next 24 mantissa bits
    // value of the remainder: r24 * 2^(e - 1023 - 52 + 21) = r24 * 2^(e - 1054)
    const float scale = __uint_as_float((uint32_t)(e - 1054 + 127) << 23);
    float r = __uint2float_rz(r24) * scale;
    if (sign) r = -r;
    const __nv_bfloat16 s1 = __float2bfloat16_rn(r);
    out[1] = s1;
    if (S > 2) out[2] = __float2bfloat16_rn(r - __bfloat162float(s1));
  }
  return true;
}


// FP64 -> FP32 rounded to 24 significant bits (ties away from zero) with integer
// operations only; false when x is outside 2^-95 <= |x| < 2^127 and not zero (the range
// in which the slices below stay normal).  Zero gives +0.
__device__ __forceinline__ bool f64_to_f32_int(double x, float& f) {
  const uint32_t lo = (uint32_t)__double2loint(x), hi = (uint32_t)__double2hiint(x);
  const uint32_t mag = hi & 0x7FFFFFFFu;
  const uint32_t t = mag - (896u << 20);           // FP32 biased exponent in bits 20..27
  uint32_t m = __funnelshift_l(lo, t, 3);           // (t << 3) | (lo >> 29): 23 mantissa bits
  m += (lo >> 28) & 1u;                             // round on the first dropped bit
  const bool zero = (mag | lo) == 0u;
  f = zero ? 0.0f : __uint_as_float(m | (hi & 0x80000000u));
  return zero || ((mag >> 20) - 928u <= 221u);
}

// The S bf16 slices of a pair (a, b) as packed words (low half a, high half b):
// f = fp32(x); s0 = f truncated to bf16 (its upper half), s1 = bf16_rn(f - s0),
// s2 = bf16_rn(f - s0 - s1).  The differences are exact in FP32, so s0 + s1 + s2 agrees
// with x to about 2^-24 relative (2^-17 for S = 2).
template <int S>
__device__ __forceinline__ bool split_pair(double a, double b, uint32_t (&w)[S]) {
  float fa, fb;
  const bool ok = f64_to_f32_int(a, fa) & f64_to_f32_int(b, fb);
  const uint32_t ua = __float_as_uint(fa), ub = __float_as_uint(fb);
  w[0] = __byte_perm(ua, ub, 0x7632);
  if constexpr (S > 1) {
    const float da = fa - __uint_as_float(ua & 0xFFFF0000u);
    const float db = fb - __uint_as_float(ub & 0xFFFF0000u);
    const __nv_bfloat162 p1 = __floats2bfloat162_rn(da, db);
    w[1] = *reinterpret_cast<const uint32_t*>(&p1);
    if constexpr (S > 2) {
      const float ea = da - __uint_as_float(w[1] << 16);
      const float eb = db - __uint_as_float(w[1] & 0xFFFF0000u);
      const __nv_bfloat162 p2 = __floats2bfloat162_rn(ea, eb);
      w[2] = *reinterpret_cast<const uint32_t*>(&p2);
    }
  }
  return ok;
}

}  // namespace tc
}  // namespace bandred
