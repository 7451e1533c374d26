// Whitening products on the tcgen05 tensor cores (Proposition 2.1: block CGS
// of the sketched block against Q_d).
//
//   t = Q_d^T w   (m x r, from the s x m basis and the s x r block)
//   w' = w - Q_d t
//
// Both read all of Q_d (s x m, FP64) for r = 1..4 columns: on the FP64 pipe
// they do 2r flops per 8-byte element of Q and are bound by the FP64 rate.
// Here each product is an error-free splitting into BF16 products (Ozaki,
// Ogita, Oishi and Rump, Numer. Algorithms 59 (2012)):
//
// Q slices.  The columns of Q are orthonormal, so |q| <= 1 and x = q/2 has
// |x| <= 1/2 (up to rounding).  x = sum_{p=1..8} n_p 2^(-7p) + rest with
// integer digits n_p = rint(2^7 x_p), x_{p+1} = 2^7 x_p - n_p, so |n_p| <= 64
// and |rest| <= 2^-57: every entry of Q is held to 2^-56 absolute, which
// bounds the error of a dot product with w by 2^-56 sum |w_i| <= 2^-56
// sqrt(s) ||w||, below the rounding error of an FP64 dot product of length s.
// The digits are exact in BF16.  Q grows by r columns per iteration, and the
// new columns are split once (k_qs_append) into two copies laid out for the
// two products:
//   QA: rows = columns j of Q, K = rows i of Q   (A operand of Q^T w)
//   QB: rows = rows i of Q,    K = columns j     (A operand of Q t)
// Each copy is a sequence of 32 KB stages: for a tile of 128 rows and 16 K
// positions, the 8 slice tiles of 4 KB in the tensor cores' K-major core
// matrix layout (8 rows x 16 bytes), so one bulk copy moves a whole stage.
//
// Right-hand side.  The r columns of w (or t) are scaled by 2^-e_c (2^e_c >
// max |column c|) and split the same way (|n_1| <= 128, |n_q| <= 64 after);
// all 8 digit planes of all r columns form one B operand of N = 8 r rows
// (padded to 16 or 32), so one MMA per Q slice p and K step of 16 gives the
// products of slice p with every digit plane q of every column.  Each
// product n_p n_q is at most 2^13 in magnitude; over the at most 256 K
// positions a CTA handles, every accumulator is an integer below 2^21 and
// exact in FP32.  Pairs with p + q > 9 (weights below 2^-70) are dropped in
// the epilogue, which converts the other 36 per column exactly to FP64 and
// adds them with their weights 2^(-7 (p+q)), then scales by 2^(1 + e_c).
// The CTAs of one product write partial sums per K range, reduced in a fixed
// order by the FP64 path's finishing kernels, so the result is deterministic.
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
constexpr int kQsSliceTile = kQsTM * kQsKC * 2;           // 4 KB
constexpr int kQsStage = kQsS * kQsSliceTile;             // 32 KB
constexpr int kQsNmax = 32;                               // B rows (8 r, padded)
constexpr int kQsBBytes = kQsNmax * kQsKper * 2;          // 16 KB
constexpr int kQsSmem = kQsStages * kQsStage + kQsBBytes; // 112 KB: two CTAs per SM
constexpr uint32_t kQsLbo = 128;                          // next 8-element K group
constexpr uint32_t kQsSboA = (kQsKC / 8) * 128;           // next 8-row group, A tiles
constexpr uint32_t kQsSboB = (kQsKper / 8) * 128;         // next 8-row group, B
constexpr long kQsSpin = 1l << 26;                        // bounded mbarrier waits
constexpr int kQsThreads = 256;

static_assert(kQsKper % kQsKC == 0, "stages tile the K range of a CTA");
static_assert(kQsKper * (1 << 13) < (1 << 24), "accumulators stay exact in FP32");

// Byte offset of (row i, K position k) inside a tile of `sbo`-spaced row groups.
__host__ __device__ __forceinline__ uint32_t qs_offset(int i, int k, uint32_t sbo) {
  return (uint32_t)((i >> 3) * sbo + (k >> 3) * kQsLbo + (i & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint16_t bf16_bits(float v) {
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  return *reinterpret_cast<const uint16_t*>(&b);
}

// The new columns j = m .. m + r - 1 of Q (ld s) into both copies.
//   QA: one thread per (new column, group of 8 rows of Q): 8 digits of 8
//       consecutive K positions -> one 16-byte store per slice; the K
//       padding i >= s up to the last tile is written as zeros (it meets
//       zero B rows and must not be NaN).
//   QB: one thread per (row i, column j) for j in [m, je): the new columns,
//       and the rest of a K tile that this append opens (zeros, so that the
//       tile's unwritten columns are finite when an MMA reads them).
__global__ void k_qs_append(const double* __restrict__ Q, int64_t s, int m, int r, int je,
                            uint8_t* __restrict__ QA, int KTA, uint8_t* __restrict__ QB,
                            int KTB) {
  const int64_t groups = 2 * (int64_t)KTA;   // every K group of the row, padding included
  const int64_t na = (int64_t)r * groups;
  const int64_t nb = s * (int64_t)(je - m);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < na + nb;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < na) {
      const int c = (int)(t / groups);
      const int64_t g = t - (int64_t)c * groups;
      const int j = m + c;
      const int64_t i0 = g * 8;
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t i = i0 + u;
        x[u] = i < s ? 0.5 * Q[i + (int64_t)j * s] : 0.0;
      }
      const int64_t tile = ((int64_t)(j / kQsTM) * KTA + i0 / kQsKC) * kQsS;
      uint8_t* base = QA + tile * kQsSliceTile + qs_offset(j % kQsTM, (int)(i0 % kQsKC), kQsSboA);
#pragma unroll
      for (int p = 0; p < kQsS; ++p) {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          const double t0 = x[u] * 128.0, t1 = x[u + 1] * 128.0;
          const double n0 = rint(t0), n1 = rint(t1);
          x[u] = t0 - n0;
          x[u + 1] = t1 - n1;
          w[u / 2] = (uint32_t)bf16_bits((float)n0) | ((uint32_t)bf16_bits((float)n1) << 16);
        }
        *reinterpret_cast<uint4*>(base + (int64_t)p * kQsSliceTile) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    } else {
      const int64_t e = t - na;
      const int j = m + (int)(e / s);
      const int64_t i = e - (int64_t)(j - m) * s;
      double x = j < m + r ? 0.5 * Q[i + (int64_t)j * s] : 0.0;
      const int64_t tile = ((i / kQsTM) * KTB + j / kQsKC) * kQsS;
      uint8_t* base = QB + tile * kQsSliceTile + qs_offset((int)(i % kQsTM), j % kQsKC, kQsSboA);
#pragma unroll
      for (int p = 0; p < kQsS; ++p) {
        const double t0 = x * 128.0;
        const double n0 = rint(t0);
        x = t0 - n0;
        *reinterpret_cast<uint16_t*>(base + (int64_t)p * kQsSliceTile) = bf16_bits((float)n0);
      }
    }
  }
}

// e[c] with 2^e[c] > max_k |B(k, c)| (0 for a zero column); one CTA per column.
__global__ void k_qs_colexp(const double* __restrict__ B, int64_t bks, int64_t bcs, int K,
                            int* __restrict__ e) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double mx = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) mx = fmax(mx, fabs(B[k * bks + c * bcs]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) {
      int ex = 0;
      if (mx > 0.0) frexp(mx, &ex);
      e[c] = ex;
    }
  }
}

// One CTA per (128-row tile mt, K range ks of kQsKper positions):
//   partial[(ks M + row) R + c] = sum_{k in range} Q-copy(row, k) B(k, c).
// Warp 0 lane 0 streams the 32 KB stages of the A copy with bulk copies;
// warp 1 lane 0 issues the MMAs (8 per stage, one per Q slice); all warps
// split B into shared memory first and run the FP64 epilogue last.
template <int R>
__global__ void __launch_bounds__(kQsThreads, 2) k_qs_mma(const uint8_t* __restrict__ As, int M,
                                                          int KT, int K,
                                                          const double* __restrict__ B,
                                                          int64_t bks, int64_t bcs,
                                                          const int* __restrict__ eB, int eA,
                                                          double* __restrict__ partial,
                                                          uint32_t* __restrict__ flags) {
  constexpr int N = (8 * R + 15) / 16 * 16;
  // no-swizzle operands and bulk copies need 16-byte alignment only; a
  // smaller alignment keeps the static part small (two CTAs per SM)
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + kQsStages * kQsStage;
  __shared__ __align__(8) uint64_t full[kQsStages], empty[kQsStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ int failed_s;
  volatile int& failed = failed_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, ks = blockIdx.y;
  const int k0 = ks * kQsKper;
  const int kn = min(kQsKper, K - k0);
  const int ns = (kn + kQsKC - 1) / kQsKC;
  if (tid == 0) failed = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(tc::smem_u32(&tmem_base)), "r"(kQsS * N) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int q = 0; q < kQsStages; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc::smem_u32(&full[q])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc::smem_u32(&empty[q])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc::smem_u32(&done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B digits: rows q R + c (q = digit plane, c = column), K positions of this range
  {
    uint4* z = reinterpret_cast<uint4*>(sB);
    for (int e = tid; e < N * kQsKper * 2 / 16; e += kQsThreads) z[e] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  for (int e = tid; e < kn * R; e += kQsThreads) {
    const int c = e / kn, k = e - c * kn;
    double x = ldexp(B[(int64_t)(k0 + k) * bks + (int64_t)c * bcs], -eB[c]);
#pragma unroll
    for (int q = 0; q < kQsS; ++q) {
      const double t0 = x * 128.0;
      const double n0 = rint(t0);
      x = t0 - n0;
      *reinterpret_cast<uint16_t*>(sB + qs_offset(q * R + c, k, kQsSboB)) = bf16_bits((float)n0);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int kt0 = k0 / kQsKC;
  if (tid == 0) {
    // producer: stage st into slot st % kQsStages once the MMAs of stage
    // st - kQsStages have released it
    for (int st = 0; st < ns; ++st) {
      const int slot = st % kQsStages;
      if (st >= kQsStages &&
          !tc::mbar_wait(tc::smem_u32(&empty[slot]), (uint32_t)((st / kQsStages - 1) & 1), kQsSpin)) {
        failed = 1;
        break;
      }
      if (failed) break;
      const uint8_t* src = As + ((int64_t)mt * KT + kt0 + st) * kQsStage;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(tc::smem_u32(&full[slot])), "r"((uint32_t)kQsStage) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   :: "r"(tc::smem_u32(sA + slot * kQsStage)), "l"(src), "r"((uint32_t)kQsStage),
                      "r"(tc::smem_u32(&full[slot])) : "memory");
    }
  } else if (tid == 32) {
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
  double acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = 0.0;
  if (got) {
#pragma unroll
    for (int pp = 0; pp < 4; ++pp) {
      const int p = 4 * half + pp;
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t v[16];
        const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(p * N + c0);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                       "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                       "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                     : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = c0 + j;
          const int q = n / R, c = n - (n / R) * R;
          if (n < 8 * R && p + q <= kQsS - 1)
            acc[c] += tc::f32_int_to_f64(v[j], -kQsBits * (p + q + 2));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();    // every MMA is complete: sB is free for the half sums
  double* red = reinterpret_cast<double*>(sB);
  const int rt = 32 * quad + lane;
  if (half == 1 && got) {
#pragma unroll
    for (int c = 0; c < R; ++c) red[rt * R + c] = acc[c];
  }
  __syncthreads();
  if (half == 0 && got) {
    const int row = mt * kQsTM + rt;
    if (row < M) {
#pragma unroll
      for (int c = 0; c < R; ++c)
        partial[((int64_t)ks * M + row) * R + c] = ldexp(acc[c] + red[rt * R + c], eA + eB[c]);
    }
  }
  if (tid == 0 && !got) atomicOr(flags, kFlagTimeout);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kQsS * N) : "memory");
}

template <int R>
void qs_mma_launch(const uint8_t* As, int M, int KT, int K, const double* B, int64_t bks,
                   int64_t bcs, const int* eB, double* partial, uint32_t* flags, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_qs_mma<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, kQsSmem);
    attr = true;
  }
  const dim3 grid((unsigned)((M + kQsTM - 1) / kQsTM), (unsigned)((K + kQsKper - 1) / kQsKper));
  count_launches(1);
  k_qs_mma<R><<<grid, kQsThreads, kQsSmem, st>>>(As, M, KT, K, B, bks, bcs, eB, 1, partial, flags);
}

void qs_product(const uint8_t* As, int M, int KT, int K, const double* B, int64_t bks, int64_t bcs,
                int r, int* eB, double* partial, uint32_t* flags, cudaStream_t st) {
  count_launches(1);
  k_qs_colexp<<<r, 512, 0, st>>>(B, bks, bcs, K, eB);
  switch (r) {
    case 1: qs_mma_launch<1>(As, M, KT, K, B, bks, bcs, eB, partial, flags, st); break;
    case 2: qs_mma_launch<2>(As, M, KT, K, B, bks, bcs, eB, partial, flags, st); break;
    case 3: qs_mma_launch<3>(As, M, KT, K, B, bks, bcs, eB, partial, flags, st); break;
    default: qs_mma_launch<4>(As, M, KT, K, B, bks, bcs, eB, partial, flags, st); break;
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
  g.bytesA = (size_t)g.MTA * g.KTA * kQsStage;
  g.bytesB = (size_t)g.MTB * g.KTB * kQsStage;
  return g;
}

int qs_chunks(int64_t K) { return (int)((K + kQsKper - 1) / kQsKper); }

bool qs_enabled(int64_t s, int m) { return m >= 256 && s >= 1024; }

void qs_append_launch(const double* Q, const QsGeom& g, int m, int r, uint8_t* QA, uint8_t* QB,
                      cudaStream_t st) {
  // a K tile of QB opened by this append gets its remaining columns zeroed
  const int last = m + r - 1;
  const bool opens = m == 0 || last / kQsKC != (m - 1) / kQsKC;
  const int je = opens ? std::min(g.KTB * kQsKC, (last / kQsKC + 1) * kQsKC) : m + r;
  const int64_t work = (int64_t)r * 2 * g.KTA + g.s * (int64_t)(je - m);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 8));
  count_launches(1);
  k_qs_append<<<blocks, 256, 0, st>>>(Q, g.s, m, r, je, QA, g.KTA, QB, g.KTB);
}

void qs_qt_launch(const QsGeom& g, const uint8_t* QA, int m, const double* w, int r, double* t,
                  double* tpart, int* eB, uint32_t* flags, cudaStream_t st) {
  // t (m x r, row-major) = Q^T w, w column-major (ld s)
  qs_product(QA, m, g.KTA, (int)g.s, w, 1, g.s, r, eB, tpart, flags, st);
  qt_finish_launch(tpart, (int64_t)m * r, qs_chunks(g.s), t, st);
}

void qs_update_launch(const QsGeom& g, const uint8_t* QB, int m, const double* t, int r,
                      const double* w_in, double* w_out, double* partial, int* eB,
                      uint32_t* flags, cudaStream_t st) {
  // w_out = w_in - Q t, t row-major (m x r)
  qs_product(QB, (int)g.s, g.KTB, m, t, r, 1, r, eB, partial, flags, st);
  q_update_finish_launch(w_in, w_out, partial, g.s, r, qs_chunks(m), st);
}

}  // namespace spk
