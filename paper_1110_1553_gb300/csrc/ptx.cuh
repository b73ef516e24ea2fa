// Inline-PTX helpers for sm_103a: mbarriers, bulk (TMA engine) copies,
// proxy fences, acquire/release accesses and the global timer.
#pragma once

#include <cstdint>

namespace hqr {
namespace ptx {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Exact widening of a stored element to FP64. FP32 values are widened with
// integer operations: on this GPU the conversion instruction occupies the
// FP64 pipe for as long as a DFMA (measured: 0.60 T conversions/s against
// 2.8 T/s for the integer form), which would halve the rate of an FP64
// product with FP32 data. Normal numbers: the 8-bit exponent is rebiased by
// 1023 - 127 = 896 and the 23-bit fraction moves up by 29 bits (both in one
// shift and add of the magnitude's bits); zeros keep their sign; subnormals
// m 2^-149 are normalized from the position p of their leading one
// (exponent p - 149); infinities and NaNs keep their fraction under the
// all-ones exponent. Bit-exact with the conversion instruction except that
// a signalling NaN stays signalling.
__host__ __device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float f) {
  const uint32_t b = __float_as_uint(f), mag = b & 0x7fffffffu;
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  uint64_t w = ((uint64_t)mag << 29) + (896ull << 52);  // normal
  if (mag >= 0x7f800000u) w = ((uint64_t)mag << 29) | (0x7ffull << 52);  // infinity, NaN
  if (mag < 0x00800000u) {  // zero, subnormal
    const int p = 31 - __clz(mag | 1u);
    w = mag ? (((uint64_t)(p + 874) << 52) | (((uint64_t)mag << (52 - p)) & 0xfffffffffffffull)) : 0ull;
  }
  return __longlong_as_double((long long)(sign | w));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bulk copy global -> shared through the TMA engine, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Dynamic shared memory of the running launch, in bytes.
__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
  uint32_t v;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}

// Orders this thread's generic-proxy accesses with its later async-proxy
// (bulk copy) accesses, in global and shared memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

}  // namespace ptx
}  // namespace hqr
