// Small inline-PTX helpers shared by the kernels that use mbarriers and bulk copies.
#pragma once

#include <cstdint>

namespace sparc {
namespace ptx {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with parity `parity` of barrier b; gives up after about
// 2^32 SM clocks (about two seconds) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(b, parity))
    if (clock64() - t0 > (1LL << 32)) return false;
  return true;
}
// The same with a limit of `limit` SM clocks.
__device__ __forceinline__ bool mbar_wait_lim(uint64_t* b, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_test(b, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
// One arrival on b that also raises its expected transaction count by `bytes`.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
// Bulk copy global -> shared of `bytes` (multiple of 16; both addresses 16-byte
// aligned), completing as a transaction on barrier b.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(b))
      : "memory");
}

}  // namespace ptx
}  // namespace sparc
