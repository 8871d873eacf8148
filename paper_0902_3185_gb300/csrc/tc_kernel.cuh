// tcgen05 building blocks (sm_100a / sm_103a): mbarriers with bounded waits,
// bulk global->shared copies, TMEM allocation, UMMA descriptors, MMA issue,
// commit, and TMEM loads.  Inline PTX only; no library code.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dmrg {
namespace tc {

// Every device-side wait gives up after this long and reports DMRG_ETIMEOUT.
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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

// Wait for the phase with the given parity to complete.  Returns false if the
// wait ran out of time or another role raised *abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (globaltimer() - t0 > WAIT_LIMIT_NS) {
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Contiguous global -> shared copy completed on an mbarrier (16-byte aligned,
// size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ------------------------------------------------------------------ TMEM
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ----------------------------------------------------------- descriptors
// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle.  Rows
// are 64 B (one K chunk), 8-row atoms of 512 B are stacked along M/N, so the
// stride between atoms (SBO) is 512 B; the leading offset is unused for this
// layout.  Version bits 46-47 = 1; layout type (bits 61-63) 4 = SW64.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t smem_addr) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Instruction descriptor of kind::f16 / kind::tf32 with an F32 accumulator,
// both operands K-major: bits 4-5 D format (1 = F32), 7-9 A format, 10-12 B
// format (BF16 = 1, TF32 = 2), 17-22 N >> 3, 24-28 M >> 4.
__host__ __device__ constexpr uint32_t idesc_f32acc(uint32_t ab_format, uint32_t M, uint32_t N) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
constexpr uint32_t FMT_BF16 = 1, FMT_TF32 = 2;

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Arrive on an mbarrier once every MMA issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns (one row per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// float64 <-> float32 conversions with integer instructions.  GB300 issues
// float64 work (conversions included) at 1/64 of the float32 rate, so the
// staging and epilogue paths, which convert every element, do it on the
// integer pipes instead.
//
// double -> float, round to nearest even; results below the float normal
// range are rounded into float subnormals, overflow gives +-inf.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ff);
  const unsigned long long m = u & 0xfffffffffffffull;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  if (e == 0) return __uint_as_float(sign);  // float64 subnormals are far below float range
  int e32 = e - 1023 + 127;
  unsigned long long sig = m | (1ull << 52);  // 53-bit significand
  int shift = 29;                              // keep 24 bits
  if (e32 <= 0) {                              // float subnormal: shift further
    shift += 1 - e32;
    e32 = 0;
    if (shift > 63) return __uint_as_float(sign);
  }
  unsigned long long kept = sig >> shift;
  const unsigned long long rem = sig & ((1ull << shift) - 1);
  const unsigned long long half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (kept & 1ull))) ++kept;
  uint32_t bits;
  if (e32 == 0) {
    bits = (uint32_t)kept;  // subnormal (a carry into bit 23 makes it the smallest normal)
  } else {
    if (kept >> 24) {  // rounding carried out of the significand
      kept >>= 1;
      ++e32;
    }
    if (e32 >= 255) return __uint_as_float(sign | 0x7f800000u);
    bits = ((uint32_t)e32 << 23) | ((uint32_t)kept & 0x7fffffu);
  }
  return __uint_as_float(sign | bits);
}

// double -> float, round to nearest even, with 32-bit integer instructions
// when the result is a normal float (the common case: one exponent test, the
// 23 kept mantissa bits and a round-half-even increment whose carry moves
// into the exponent); zeros, subnormal results, overflow, inf and NaN take
// d2f_rn.
__device__ __forceinline__ float d2f_rn32(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 254u) {  // float exponent e - 896 in 1..254
    const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rem = lo & 0x1fffffffu;
    const uint32_t up = (uint32_t)(rem > 0x10000000u) | ((uint32_t)(rem == 0x10000000u) & m);
    return __uint_as_float((hi & 0x80000000u) | (((e - 896u) << 23) + m + (up & 1u)));
  }
  return d2f_rn(x);
}

// float -> double, exact
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ef = (u >> 23) & 0xffu;
  if (ef - 1u < 254u) {  // normal float: rebias the exponent, shift the mantissa into place (32-bit halves)
    const uint32_t m = u & 0x7fffffu;
    return __hiloint2double((int)((u & 0x80000000u) | ((ef + 896u) << 20) | (m >> 3)), (int)(m << 29));
  }
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const uint32_t e = (u >> 23) & 0xff;
  uint32_t m = u & 0x7fffffu;
  if (e == 0xff) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | ((unsigned long long)m << 29)));
  if (e == 0) {
    if (m == 0) return __longlong_as_double((long long)sign);
    const int lz = __clz(m) - 8;  // leading bit at 23 - lz: normalise, value = 2^(p - 149)
    m = (m << lz) & 0x7fffffu;
    const unsigned long long ed = (unsigned long long)(1023 - 126 - lz);
    return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)m << 29)));
  }
  const unsigned long long ed = (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)m << 29)));
}

// two floats -> packed bfloat16 pair (x0 in the low half), round to nearest even
__device__ __forceinline__ uint32_t bf16x2_rn(float x0, float x1) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
  return r;
}

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tc
}  // namespace dmrg
