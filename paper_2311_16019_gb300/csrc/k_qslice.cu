// Whitening products on the tcgen05 tensor cores (Proposition 2.1: block CGS
// of the sketched block against Q_d).
//
//   t = Q_d^T w   (m x r, from the s x m basis and the s x r block)
//   w' = w - Q_d t
//
// Both read all of Q_d (s x m, FP64) for r = 1..4 columns: on the FP64 pipe
// (2 FMA per clock per SM on this GPU) they do 2r flops per 8-byte element
// of Q and are bound by the FP64 rate.  Here each product is an error-free
// splitting into BF16 products (Ozaki, Ogita, Oishi and Rump, Numer.
// Algorithms 59 (2012)), with the splitting and the recombination done on
// the integer pipe so that no FP64 arithmetic is left but a few operations
// per output:
//
// Digits.  A value x with |x| < 2^e is rounded to the integer
// N = rint(x 2^(56-e)) (|N| < 2^56, built from the FP64 bit pattern) and
// written in balanced base 2^7 from the bottom: N = sum_{p=1..8} n_p 2^(56-7p)
// with n_2 .. n_8 in [-64, 63] and |n_1| <= 128.  The representation holds x
// to 2^(e-57) absolute, and the digits are exact in BF16.
//
// Q slices.  The columns of Q are orthonormal, so |q| < 2 and e = 1 (|n_1|
// <= 64): every entry of Q is held to 2^-56, which bounds the error of a dot
// product with w by 2^-56 sum |w_i| <= 2^-56 sqrt(s) ||w||, below the
// rounding error of an FP64 dot product of length s.  Q grows by r columns
// per iteration, and the new columns are split once (k_qs_append) into two
// copies laid out for the two products:
//   QA: rows = columns j of Q, K = rows i of Q   (A operand of Q^T w)
//   QB: rows = rows i of Q,    K = columns j     (A operand of Q t)
// The digits are stored as biased bytes (n + 128), one byte per digit, so a
// copy is as large as Q itself.  Each copy is a sequence of 16 KB stages:
// for a tile of 128 rows and 16 K positions, the 8 slice tiles of 2 KB in
// the byte order of the tensor cores' K-major core-matrix layout at half
// width; loader warps read a stage with 16-byte loads (the next stage in
// flight) and widen it to BF16 in shared memory, where byte offset o lands
// at 2 o, the layout the MMAs read.
//
// Right-hand side.  Each CTA handles 256 K positions; it splits its part of
// the r columns of w (or t) with e_c from the largest magnitude of column c
// in that part, and all 8 digit planes of all r columns form one B operand
// of N = 8 r rows (padded to 16 or 32), so one MMA per Q slice p and K step
// of 16 gives the products of slice p with every digit plane q of every
// column.  Each product n_p n_q is at most 2^13 in magnitude; over 256 K
// positions every accumulator is an integer of magnitude at most 2^21 and
// exact in FP32.
// Pairs with p + q > 9 (weights below 2^-70) are dropped; the epilogue turns
// the other 36 per column into integers, adds those of one weight level
// 2^(-7 (p+q)) exactly, combines the levels exactly into two 64-bit integers
// and converts those to FP64.  The CTAs of one product write partial sums
// per K range, reduced in a fixed order by the FP64 path's finishing
// kernels, so the result is deterministic.
#include "spk_internal.cuh"
#include "tc_common.cuh"

#include <algorithm>

namespace spk {

namespace {

constexpr int kQsS = 8;                                   // slices
constexpr int kQsBits = 7;                                // bits per slice
constexpr int kQsTM = 128;                                // tile rows (M of the MMA)
constexpr int kQsKC = 16;                                 // K per stage (one MMA per slice)
constexpr int kQsStages = 3;                              // stages in flight per CTA
constexpr int kQsKper = 256;                              // K positions per CTA
constexpr int kQsSliceTile = kQsTM * kQsKC * 2;           // 4 KB (BF16, shared memory)
constexpr int kQsStage = kQsS * kQsSliceTile;             // 32 KB
constexpr int kQsSliceTile8 = kQsTM * kQsKC;              // 2 KB (biased int8 digits, global)
constexpr int kQsStage8 = kQsS * kQsSliceTile8;           // 16 KB
constexpr int kQsLoaders = 256;                           // warps 0..7 widen the stages
constexpr int kQsLoads = kQsStage8 / 16 / kQsLoaders;     // 16-byte loads per loader and stage
constexpr int kQsNmax = 32;                               // B rows (8 r, padded)
constexpr int kQsBBytes = kQsNmax * kQsKper * 2;          // 16 KB
constexpr int kQsSmem = kQsStages * kQsStage + kQsBBytes; // 112 KB: two CTAs per SM
constexpr uint32_t kQsLbo = 128;                          // next 8-element K group
constexpr uint32_t kQsSboA = (kQsKC / 8) * 128;           // next 8-row group, A tiles
constexpr uint32_t kQsSboB = (kQsKper / 8) * 128;         // next 8-row group, B
constexpr long kQsSpin = 1l << 26;                        // bounded mbarrier waits
constexpr int kQsThreads = kQsLoaders + 32;              // + warp 8: the MMA issuer

static_assert(kQsKper % kQsKC == 0, "stages tile the K range of a CTA");
static_assert(kQsKper * (1 << 13) < (1 << 24), "accumulators stay exact in FP32");

// Byte offset of (row i, K position k) inside a tile of `sbo`-spaced row groups.
__host__ __device__ __forceinline__ uint32_t qs_offset(int i, int k, uint32_t sbo) {
  return (uint32_t)((i >> 3) * sbo + (k >> 3) * kQsLbo + (i & 7) * 16 + (k & 7) * 2);
}

// Byte offset of (row i, K position k) inside an int8 slice tile: the BF16
// core-matrix layout at half the bytes, so that the widened copy of byte
// offset o lies at 2 o.
__host__ __device__ __forceinline__ uint32_t qs_offset8(int i, int k) {
  return (uint32_t)((i >> 3) * (kQsSboA / 2) + (k >> 3) * (kQsLbo / 2) + (i & 7) * 8 + (k & 7));
}

// 8 values (8 consecutive K positions of one row) -> one 8-byte core-matrix
// row of biased digits (n + 128) per slice at base + p * kQsSliceTile8.
__device__ __forceinline__ void qs_store_row8(const double (&x)[8], int e, uint8_t* base) {
  int n[8][kQsS];
#pragma unroll
  for (int u = 0; u < 8; ++u) tc::digits8(x[u], e, n[u]);
#pragma unroll
  for (int p = 0; p < kQsS; ++p) {
    uint32_t w[2] = {0u, 0u};
#pragma unroll
    for (int u = 0; u < 8; ++u) w[u >> 2] |= (uint32_t)(n[u][p] + 128) << (8 * (u & 3));
    *reinterpret_cast<uint2*>(base + (int64_t)p * kQsSliceTile8) = make_uint2(w[0], w[1]);
  }
}

// The new columns j = m .. m + r - 1 of Q (ld s) into both copies (e = 1).
//   QA: one thread per (new column, group of 8 rows of Q): the K padding
//       i >= s up to the last tile is written as zeros (it meets zero B rows
//       and must not be NaN).
//   QB: one thread per (row i, group of 8 columns) for the column groups
//       g0 .. g1 - 1 that hold the new columns: columns below m are written
//       again (the same digits), columns from m + r on are written as zeros
//       (a K tile that this append opens is zeroed to its end, so that its
//       unwritten columns are finite when an MMA reads them).
__global__ void k_qs_append(const double* __restrict__ Q, int64_t s, int m, int r, int g0, int g1,
                            uint8_t* __restrict__ QA, int KTA, uint8_t* __restrict__ QB,
                            int KTB) {
  const int64_t ga = 2 * (int64_t)KTA;
  const int64_t na = (int64_t)r * ga;
  const int64_t nb = s * (int64_t)(g1 - g0);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < na + nb;
       t += (int64_t)gridDim.x * blockDim.x) {
    double x[8];
    if (t < na) {
      const int c = (int)(t / ga);
      const int64_t i0 = (t - (int64_t)c * ga) * 8;
      const int j = m + c;
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = i0 + u < s ? Q[i0 + u + (int64_t)j * s] : 0.0;
      const int64_t tile = ((int64_t)(j / kQsTM) * KTA + i0 / kQsKC) * kQsS;
      qs_store_row8(x, 1, QA + tile * kQsSliceTile8 + qs_offset8(j % kQsTM, (int)(i0 % kQsKC)));
    } else {
      const int64_t e = t - na;
      const int G = g0 + (int)(e / s);
      const int64_t i = e - (int64_t)(G - g0) * s;
      const int j0 = 8 * G;
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = j0 + u < m + r ? Q[i + (int64_t)(j0 + u) * s] : 0.0;
      const int64_t tile = ((i / kQsTM) * KTB + j0 / kQsKC) * kQsS;
      qs_store_row8(x, 1, QB + tile * kQsSliceTile8 + qs_offset8((int)(i % kQsTM), j0 % kQsKC));
    }
  }
}

// 16 biased int8 digits -> 16 BF16 values (two 16-byte stores): 2^23 + u is
// exact in FP32, minus 2^23 + 128 gives the digit, and the upper half of an
// FP32 holding an integer of at most 8 bits is its BF16 pattern.
__device__ __forceinline__ void qs_widen16(const uint4 v, uint8_t* dst) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint32_t o[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float f[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      f[j] = __uint_as_float(__byte_perm(w[q], 0x4B00u, 0x5440u | (uint32_t)j)) - 8388736.0f;
    o[2 * q] = __byte_perm(__float_as_uint(f[0]), __float_as_uint(f[1]), 0x7632u);
    o[2 * q + 1] = __byte_perm(__float_as_uint(f[2]), __float_as_uint(f[3]), 0x7632u);
  }
  reinterpret_cast<uint4*>(dst)[0] = make_uint4(o[0], o[1], o[2], o[3]);
  reinterpret_cast<uint4*>(dst)[1] = make_uint4(o[4], o[5], o[6], o[7]);
}

// Integer value of an FP32 accumulator holding an integer of magnitude < 2^22.
__device__ __forceinline__ int qs_f32_int(uint32_t f) {
  return __float_as_int(__uint_as_float(f) + 12582912.0f) - 0x4B400000;
}

// Level sums of one half of the Q slices (p = P0 .. P0 + 3) for one tile row:
// lev[L][c] = sum over kept pairs p + q = L of D_p(row, q R + c), exact in
// int32; then hi[c] = sum_{L<4} lev[L][c] 2^(7 (3-L)), lo[c] = sum_{L>=4}
// lev[L][c] 2^(7 (7-L)), exact in int64.
template <int R, int N, int P0>
__device__ __forceinline__ void qs_epilogue_half(uint32_t trow, long long (&hi)[R],
                                                 long long (&lo)[R]) {
  int lev[kQsS][R];
#pragma unroll
  for (int L = 0; L < kQsS; ++L)
#pragma unroll
    for (int c = 0; c < R; ++c) lev[L][c] = 0;
#pragma unroll
  for (int pp = 0; pp < 4; ++pp) {
    const int p = P0 + pp;
    // the slice's column chunks with a kept pair, loaded together and waited
    // for once (each wait is a round trip to tensor memory)
    uint32_t v[N / 16][16];
#pragma unroll
    for (int ch = 0; ch < N / 16; ++ch) {
      if ((16 * ch) / R > kQsS - 1 - p) continue;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(v[ch][0]), "=r"(v[ch][1]), "=r"(v[ch][2]), "=r"(v[ch][3]), "=r"(v[ch][4]),
                     "=r"(v[ch][5]), "=r"(v[ch][6]), "=r"(v[ch][7]), "=r"(v[ch][8]), "=r"(v[ch][9]),
                     "=r"(v[ch][10]), "=r"(v[ch][11]), "=r"(v[ch][12]), "=r"(v[ch][13]),
                     "=r"(v[ch][14]), "=r"(v[ch][15])
                   : "r"(trow + (uint32_t)(p * N + 16 * ch)));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int ch = 0; ch < N / 16; ++ch) {
      if ((16 * ch) / R > kQsS - 1 - p) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = 16 * ch + j;
        const int q = n / R, c = n % R;
        if (n < 8 * R && p + q <= kQsS - 1) lev[p + q][c] += qs_f32_int(v[ch][j]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < R; ++c) {
    long long h = 0, l = 0;
#pragma unroll
    for (int L = 0; L < 4; ++L) h += (long long)lev[L][c] << (kQsBits * (3 - L));
#pragma unroll
    for (int L = 4; L < kQsS; ++L) l += (long long)lev[L][c] << (kQsBits * (7 - L));
    hi[c] = h;
    lo[c] = l;
  }
}

// One CTA per (128-row tile mt, K range ks of kQsKper positions):
//   partial[(ks M + row) R + c] = sum_{k in range} Q-copy(row, k) B(k, c).
// Warps 0..7 load the 16 KB int8 stages of the A copy (the first before B is
// split, each next one while the current one is widened) and widen them into
// a ring of 32 KB BF16 stages; warp 8 lane 0 issues the MMAs (8 per stage,
// one per Q slice); all warps split B into shared memory, warps 0..7 run the
// epilogue.
template <int R>
__global__ void __launch_bounds__(kQsThreads, 2) k_qs_mma(const uint8_t* __restrict__ As, int M,
                                                          int KT, int K,
                                                          const double* __restrict__ B,
                                                          int64_t bks, int64_t bcs, int eA,
                                                          double* __restrict__ partial,
                                                          uint32_t* __restrict__ flags) {
  constexpr int N = (8 * R + 15) / 16 * 16;
  constexpr int kVals = (kQsKper * R + kQsThreads - 1) / kQsThreads;   // B values per thread
  // no-swizzle operands and bulk copies need 16-byte alignment only; a
  // smaller alignment keeps the static part small (two CTAs per SM)
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + kQsStages * kQsStage;
  __shared__ __align__(8) uint64_t full[kQsStages], empty[kQsStages], done;
  __shared__ unsigned long long cmax[4];
  __shared__ int s_e[4];
  __shared__ uint32_t tmem_base;
  __shared__ int failed_s;
  volatile int& failed = failed_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, ks = blockIdx.y;
  const int k0 = ks * kQsKper;
  const int kn = min(kQsKper, K - k0);
  const int ns = (kn + kQsKC - 1) / kQsKC;
  const int kt0 = k0 / kQsKC;
  if (tid == 0) failed = 0;
  if (tid < 4) cmax[tid] = 0ull;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(tc::smem_u32(&tmem_base)), "r"(kQsS * N) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int q = 0; q < kQsStages; ++q) {
      // full: one arrive per loader warp; empty: the MMA commit
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                   :: "r"(tc::smem_u32(&full[q])), "r"(kQsLoaders / 32) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc::smem_u32(&empty[q])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc::smem_u32(&done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  {
    uint4* z = reinterpret_cast<uint4*>(sB);
    for (int e = tid; e < N * kQsKper * 2 / 16; e += kQsThreads) z[e] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  // loaders: the int8 digits of stage st, 16 bytes per load, kQsLoads per thread
  const bool loader = tid < kQsLoaders;
  auto load_stage = [&](int st, uint4 (&v)[kQsLoads]) {
    const uint4* src = reinterpret_cast<const uint4*>(As + ((int64_t)mt * KT + kt0 + st) * kQsStage8);
#pragma unroll
    for (int u = 0; u < kQsLoads; ++u) v[u] = __ldcs(src + tid + u * kQsLoaders);
  };
  uint4 cur[kQsLoads], nxt[kQsLoads];
  if (loader && ns > 0) load_stage(0, cur);
  // B digits: rows q R + c (q = digit plane, c = column) of this K range,
  // with the exponent of each column's largest magnitude in the range
  double bv[kVals];
  unsigned long long mx[R];
#pragma unroll
  for (int c = 0; c < R; ++c) mx[c] = 0ull;
#pragma unroll
  for (int u = 0; u < kVals; ++u) {
    const int e = tid + u * kQsThreads;
    bv[u] = 0.0;
    if (e < kn * R) {
      const int c = e / kn, k = e - c * kn;
      bv[u] = B[(int64_t)(k0 + k) * bks + (int64_t)c * bcs];
      const unsigned long long a = (unsigned long long)__double_as_longlong(bv[u]) & ~(1ull << 63);
#pragma unroll
      for (int cc = 0; cc < R; ++cc)
        if (c == cc && a > mx[cc]) mx[cc] = a;
    }
  }
#pragma unroll
  for (int c = 0; c < R; ++c)
    if (mx[c]) atomicMax(&cmax[c], mx[c]);
  __syncthreads();
  if (tid < R) {
    const unsigned long long a = cmax[tid];
    s_e[tid] = tc::exp_above(a);     // 2^e > max |B(:, c)|
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kVals; ++u) {
    const int e = tid + u * kQsThreads;
    if (e < kn * R) {
      const int c = e / kn, k = e - c * kn;
      int n[kQsS];
      tc::digits8(bv[u], s_e[c], n);
#pragma unroll
      for (int q = 0; q < kQsS; ++q)
        *reinterpret_cast<uint16_t*>(sB + qs_offset(q * R + c, k, kQsSboB)) = (uint16_t)tc::bf16_int(n[q]);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (loader) {
    // stage st into slot st % kQsStages once the MMAs of stage st - kQsStages
    // have released it; the next stage's loads are in flight meanwhile
    for (int st = 0; st < ns; ++st) {
      if (st + 1 < ns) load_stage(st + 1, nxt);
      const int slot = st % kQsStages;
      if (st >= kQsStages &&
          !tc::mbar_wait(tc::smem_u32(&empty[slot]), (uint32_t)((st / kQsStages - 1) & 1), kQsSpin)) {
        failed = 1;
        break;
      }
      if (failed) break;
      uint8_t* dst = sA + slot * kQsStage;
#pragma unroll
      for (int u = 0; u < kQsLoads; ++u) qs_widen16(cur[u], dst + 32 * (tid + u * kQsLoaders));
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_u32(&full[slot])) : "memory");
#pragma unroll
      for (int u = 0; u < kQsLoads; ++u) cur[u] = nxt[u];
    }
  } else if (tid == kQsLoaders) {
    // MMA issuer
    constexpr uint32_t idesc = tc::idesc_bf16(kQsTM, N);
    bool ok = true;
    for (int st = 0; st < ns; ++st) {
      const int slot = st % kQsStages;
      if (!tc::mbar_wait(tc::smem_u32(&full[slot]), (uint32_t)((st / kQsStages) & 1), kQsSpin) ||
          failed) {
        failed = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t db = tc::desc_kmajor(tc::smem_u32(sB) + (uint32_t)st * 2 * kQsLbo, kQsLbo, kQsSboB);
#pragma unroll
      for (int p = 0; p < kQsS; ++p) {
        const uint64_t da = tc::desc_kmajor(tc::smem_u32(sA + slot * kQsStage + p * kQsSliceTile),
                                            kQsLbo, kQsSboA);
        const uint32_t d = tmem + (uint32_t)(p * N);
        const uint32_t accum = st > 0 ? 1u : 0u;
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(d), "l"(da), "l"(db), "r"(idesc), "r"(accum) : "memory");
      }
      // release the slot only to a later stage of this CTA (an arrive after
      // the CTA's end must not be left pending)
      if (st + kQsStages < ns)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(tc::smem_u32(&empty[slot])) : "memory");
    }
    if (ok)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(tc::smem_u32(&done)) : "memory");
  }
  __syncwarp();
  bool got = !failed && tc::mbar_wait(tc::smem_u32(&done), 0u, kQsSpin);
  got = __syncthreads_and(got) != 0;    // uniform: the tensor-memory loads are .aligned
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warps w and w + 4 share lane quadrant w (tile rows 32 w ..
  // 32 w + 31); warp half h takes the Q slices p = 4 h .. 4 h + 3
  const int quad = warp & 3, half = warp >> 2;
  const uint32_t trow = tmem + ((uint32_t)(32 * quad) << 16);
  long long hi[R], lo[R];
  if (got && loader) {
    if (half == 0)
      qs_epilogue_half<R, N, 0>(trow, hi, lo);
    else
      qs_epilogue_half<R, N, 4>(trow, hi, lo);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();    // every MMA is complete: sB is free for the half sums
  long long* red = reinterpret_cast<long long*>(sB);
  const int rt = 32 * quad + lane;
  if (half == 1 && got && loader) {
#pragma unroll
    for (int c = 0; c < R; ++c) {
      red[(2 * rt) * R + c] = hi[c];
      red[(2 * rt + 1) * R + c] = lo[c];
    }
  }
  __syncthreads();
  if (half == 0 && got) {
    const int row = mt * kQsTM + rt;
    if (row < M) {
#pragma unroll
      for (int c = 0; c < R; ++c) {
        const long long h = hi[c] + red[(2 * rt) * R + c];
        const long long l = lo[c] + red[(2 * rt + 1) * R + c];
        const int sc = eA + s_e[c];
        partial[((int64_t)ks * M + row) * R + c] =
            tc::i64_f64(h, sc - 5 * kQsBits) + tc::i64_f64(l, sc - 9 * kQsBits);
      }
    }
  }
  if (tid == 0 && !got) atomicOr(flags, kFlagTimeout);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kQsS * N) : "memory");
}

template <int R>
void qs_mma_launch(const uint8_t* As, int M, int KT, int K, const double* B, int64_t bks,
                   int64_t bcs, double* partial, uint32_t* flags, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_qs_mma<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kQsSmem);
    attr = true;
  }
  const dim3 grid((unsigned)((M + kQsTM - 1) / kQsTM), (unsigned)((K + kQsKper - 1) / kQsKper));
  count_launches(1);
  k_qs_mma<R><<<grid, kQsThreads, kQsSmem, st>>>(As, M, KT, K, B, bks, bcs, 1, partial, flags);
}

void qs_product(const uint8_t* As, int M, int KT, int K, const double* B, int64_t bks, int64_t bcs,
                int r, double* partial, uint32_t* flags, cudaStream_t st) {
  switch (r) {
    case 1: qs_mma_launch<1>(As, M, KT, K, B, bks, bcs, partial, flags, st); break;
    case 2: qs_mma_launch<2>(As, M, KT, K, B, bks, bcs, partial, flags, st); break;
    case 3: qs_mma_launch<3>(As, M, KT, K, B, bks, bcs, partial, flags, st); break;
    default: qs_mma_launch<4>(As, M, KT, K, B, bks, bcs, partial, flags, st); break;
  }
}

}  // namespace

QsGeom qs_geometry(int64_t s, int mmax) {
  QsGeom g;
  g.s = s;
  g.mmax = mmax;
  g.MTA = (mmax + kQsTM - 1) / kQsTM;
  g.KTA = (int)((s + kQsKC - 1) / kQsKC);
  g.MTB = (int)((s + kQsTM - 1) / kQsTM);
  g.KTB = (mmax + kQsKC - 1) / kQsKC;
  g.bytesA = (size_t)g.MTA * g.KTA * kQsStage8;
  g.bytesB = (size_t)g.MTB * g.KTB * kQsStage8;
  return g;
}

int qs_chunks(int64_t K) { return (int)((K + kQsKper - 1) / kQsKper); }

bool qs_enabled(int64_t s, int m) { return m >= 256 && s >= 1024; }

void qs_append_launch(const double* Q, const QsGeom& g, int m, int r, uint8_t* QA, uint8_t* QB,
                      cudaStream_t st) {
  // a K tile of QB opened by this append is zeroed to its end
  const int last = m + r - 1;
  const bool opens = m == 0 || last / kQsKC != (m - 1) / kQsKC;
  const int je = opens ? std::min(g.KTB * kQsKC, (last / kQsKC + 1) * kQsKC) : m + r;
  const int g0 = m / 8, g1 = (je + 7) / 8;
  const int64_t work = (int64_t)r * 2 * g.KTA + g.s * (int64_t)(g1 - g0);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 8));
  count_launches(1);
  k_qs_append<<<blocks, 256, 0, st>>>(Q, g.s, m, r, g0, g1, QA, g.KTA, QB, g.KTB);
}

void qs_qt_launch(const QsGeom& g, const uint8_t* QA, int m, const double* w, int r, double* t,
                  double* tpart, uint32_t* flags, cudaStream_t st) {
  // t (m x r, row-major) = Q^T w, w column-major (ld s)
  qs_product(QA, m, g.KTA, (int)g.s, w, 1, g.s, r, tpart, flags, st);
  qt_finish_launch(tpart, (int64_t)m * r, qs_chunks(g.s), t, st);
}

void qs_update_launch(const QsGeom& g, const uint8_t* QB, int m, const double* t, int r,
                      const double* w_in, double* w_out, double* partial, uint32_t* flags,
                      cudaStream_t st) {
  // w_out = w_in - Q t, t row-major (m x r)
  qs_product(QB, (int)g.s, g.KTB, m, t, r, 1, r, partial, flags, st);
  q_update_finish_launch(w_in, w_out, partial, g.s, r, qs_chunks(m), st);
}

}  // namespace spk
