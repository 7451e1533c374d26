// Device helpers shared by the tcgen05 kernels (k_ozaki.cu, k_qslice.cu):
// shared-memory addresses, shared-memory matrix descriptors for the
// no-swizzle K-major operand layout, bounded mbarrier waits and the exact
// conversion of an integer-valued FP32 accumulator to FP64.
#pragma once

#include <stdint.h>

namespace spk {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Descriptor of a K-major operand without swizzle: core matrices of 8 rows x
// 16 bytes (8 BF16 along K), `lbo` bytes between core matrices adjacent in K,
// `sbo` bytes between groups of 8 rows; bit 46 is the descriptor version of
// tcgen05.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both
// operands K-major, an M x N tile.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// x 2^sh for the FP32 bit pattern f of an integer with |x| < 2^24, built on
// the integer pipe: FP32 exponent rebiased to FP64 (+896) and shifted by sh,
// mantissa moved to the top of the FP64 fraction.  Exact.
__device__ __forceinline__ double f32_int_to_f64(uint32_t f, int sh) {
  if ((f & 0x7fffffffu) == 0u) return 0.0;
  const uint32_t e = ((f >> 23) & 0xffu) + 896u + (uint32_t)sh;
  const uint32_t mant = f & 0x7fffffu;
  const uint32_t hi = (f & 0x80000000u) | (e << 20) | (mant >> 3);
  return __hiloint2double((int)hi, (int)(mant << 29));
}

// Wait for the phase with the given parity of an mbarrier, at most `spin`
// polls; false if the phase did not complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long spin) {
  uint32_t done = 0;
  for (long it = 0; it < spin && !done; ++it) {
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  }
  return done != 0;
}

}  // namespace tc
}  // namespace spk
