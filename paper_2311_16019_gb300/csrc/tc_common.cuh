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

// Balanced base-2^7 digits of N = rint(x 2^(56-e)) for |x| < 2^e, from the
// FP64 bit pattern on the integer pipe: n[0] is the leading digit (|n[0]| <=
// 128, <= 64 when |x| < 2^(e-1)), n[1..7] lie in [-64, 63];
// x = 2^e sum_p n[p] 2^(-7 (p+1)) + rest with |rest| <= 2^(e-57).
__device__ __forceinline__ void digits8(double x, int e, int (&n)[8]) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FF);
  long long N = 0;
  if (E != 0) {
    const unsigned long long M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - 1023 - e + 4;     // x 2^(56-e) = M 2^sh, sh <= 3 as |x| < 2^e
    if (sh >= 0)
      N = (long long)(M << sh);
    else if (sh > -54)
      N = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
    if (u >> 63) N = -N;
  }
#pragma unroll
  for (int p = 7; p >= 1; --p) {
    const int d = (int)((N + 64) & 127) - 64;
    n[p] = d;
    N = (N - d) >> 7;
  }
  n[0] = (int)N;
}

// BF16 bit pattern of an integer with |n| <= 255 (exact; the digits passed
// here have |n| <= 128).
__device__ __forceinline__ uint32_t bf16_int(int n) {
  if (n == 0) return 0u;
  const uint32_t a = (uint32_t)(n < 0 ? -n : n);
  const int pos = 31 - __clz(a);
  return (n < 0 ? 0x8000u : 0u) | ((uint32_t)(127 + pos) << 7) | ((a << (7 - pos)) & 0x7Fu);
}

// Integer value of an FP32 bit pattern holding an integer of magnitude < 2^24.
__device__ __forceinline__ int f32_int(uint32_t f) {
  const int e = (int)((f >> 23) & 0xFFu);
  if (e < 127) return 0;
  const int v = (int)(((f & 0x7FFFFFu) | 0x800000u) >> (150 - e));
  return (f >> 31) ? -v : v;
}

// x 2^sh as FP64 for an integer |x| < 2^53, built on the integer pipe (exact;
// ldexp when the result leaves the normal range).
__device__ __forceinline__ double i64_f64(long long x, int sh) {
  if (x == 0) return 0.0;
  const unsigned long long a = (unsigned long long)(x < 0 ? -x : x);
  const int pos = 63 - __clzll((long long)a);
  const int ex = 1023 + pos + sh;
  if (ex <= 0 || ex >= 2047) return ldexp((double)x, sh);
  const unsigned long long mant = (a << (52 - pos)) & 0xFFFFFFFFFFFFFull;
  return __longlong_as_double((long long)((x < 0 ? (1ull << 63) : 0ull) |
                                          ((unsigned long long)ex << 52) | mant));
}

// Exponent e with 2^e > |x| for the magnitude bits a of an FP64 value (0 for 0).
__device__ __forceinline__ int exp_above(unsigned long long a) {
  return a ? (int)((a >> 52) & 0x7FF) - 1022 : 0;
}

}  // namespace tc
}  // namespace spk
