// tw_bulk.cuh -- bulk (TMA engine) copies between global and shared memory on
// sm_103a: cp.async.bulk with mbarrier completion for global -> shared, bulk
// groups for shared -> global.  Every address handed to a bulk copy is 16-byte
// aligned and every size a multiple of 16 bytes (callers round their ranges
// out to 16 bytes inside padded tables).
#pragma once
#include <cstdint>

namespace tw {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// mbarrier with one arrival per phase (the thread that issues the copies)
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// waits for the phase `parity` of the barrier with an iteration limit; false
// when the limit ran out (the caller records it and abandons the work)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  for (int k = 0; k < (1 << 22); k++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// global -> shared, completion counted on `bar` in bytes
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// shared -> global in the thread's current bulk group
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// the shared memory read by this thread's committed bulk stores may be reused
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// generic-proxy writes to shared memory become visible to the bulk (async) proxy
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// A float widened to double exactly on the integer pipes: a normal float's
// bits map to the double's by moving the sign, re-biasing the exponent
// (127 -> 1023) and shifting the mantissa; a subnormal float m * 2^-149 is
// normalised by its leading bit; zeros keep their sign, infinities and NaNs
// their class.  (The split-precision output hi + lo then costs one FP64
// addition instead of two conversions and an addition on the FP64 pipe.)
__device__ __forceinline__ double widen_f32(float x) {
  const uint32_t f = __float_as_uint(x);
  const uint32_t e = (f >> 23) & 0xffu;
  const uint64_t s = (uint64_t)(f >> 31) << 63;
  if (e == 0u) {
    const uint32_t mf = f & 0x7fffffu;
    if (mf == 0u) return __longlong_as_double((long long)s);
    const int top = 31 - __clz((int)mf);  // value = 1.x * 2^(top - 149)
    const uint64_t mant = ((uint64_t)mf << (52 - top)) & ((1ull << 52) - 1ull);
    const uint64_t ed = (uint64_t)(top - 149 + 1023);
    return __longlong_as_double((long long)(s | (ed << 52) | mant));
  }
  const uint64_t m = (uint64_t)(f & 0x7fffffu) << 29;
  const uint64_t ed = e == 0xffu ? 0x7ffull : (uint64_t)(e + (1023u - 127u));
  return __longlong_as_double((long long)(s | (ed << 52) | m));
}

}  // namespace tw
