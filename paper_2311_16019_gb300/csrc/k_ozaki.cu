// FP64 matrix product on the tcgen05 tensor cores by error-free splitting
// (Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012); here with BF16 slices and the
// FP32 accumulators of the tensor cores).
//
//   C = alpha op(A) op(B) + beta C,   op(A): M x K,  op(B): K x N,  FP64.
//
// Splitting.  Row i of op(A) is rounded to 56 bits relative to 2^eA_i (eA_i:
// 2^eA_i above its largest magnitude) and written as a sum of kOzS slices,
// v = 2^eA_i sum_p n_p 2^(-7 p), balanced base-2^7 digits taken from the
// FP64 bit pattern on the integer pipe (|n_1| <= 128, n_p in [-64, 63] for
// p >= 2); likewise column j of op(B) with eB_j.  The integers are exact in
// BF16, and the remainder is below 2^-57 of the row's scale: the splitting
// is exact to more than FP64's 53 bits.
//
// Products.  The (at most 8) slice pairs of one level L = p + q share one
// FP32 accumulator in tensor memory over K-ranges of 256 (four chunks of 64
// staged through shared memory): a level sum is at most
// 256 (2 2^13 + 6 2^12) < 2^24 in magnitude (2^22 for L = 2), so every
// level sum is EXACT in FP32.  Levels 2 .. 9 (the 36 pairs with p + q <= 9;
// the pairs left out are below 2^-58 of |row| |col| per product) live side
// by side in the 512 columns of tensor memory.  The epilogue reads each
// level sum as an integer and adds it, shifted by its weight, to one of two
// exact 64-bit integer accumulators per element (levels 2..5 and 6..9),
// range after range, all on the integer pipe; at the end the two are
// converted to FP64 (exact below 2^53) and scaled by alpha 2^(eA_i + eB_j).
// GB300's FP64 pipe retires 2 FMAs per clock per SM, so FP64 arithmetic is
// kept to three operations per element of C.
//
// Kernels: k_oz_rowexp (the exponents), k_oz_split (slices, written in the
// tensor cores' shared-memory operand layout: 8-row x 16-byte core matrices,
// K-major, no swizzle), k_oz_mma (one CTA per 128 x 64 tile of C; one thread
// issues the bulk copies of the chunk's slices and the tcgen05.mma
// instructions, all eight warps read tensor memory for the epilogue).
#include "spk_internal.cuh"
#include "tc_common.cuh"

#include <algorithm>

namespace spk {

namespace {

constexpr int kOzS = 8;          // slices per operand
constexpr int kOzBits = 7;       // bits per slice
constexpr int kOzTM = 128;       // tile rows (M of the MMA)
constexpr int kOzTN = 64;        // tile columns (N of the MMA)
constexpr int kOzKC = 64;        // K per chunk (4 MMAs of K = 16)
constexpr int kOzEpi = 4;        // chunks accumulated in tensor memory between epilogues
constexpr int kOzLevels = 8;     // levels L = 2 .. 9
constexpr int kOzATile = kOzTM * kOzKC * 2;   // bytes of one A slice tile (16 KB)
constexpr int kOzBTile = kOzTN * kOzKC * 2;   // bytes of one B slice tile (8 KB)
constexpr int kOzSmem = kOzS * (kOzATile + kOzBTile);   // 192 KB
constexpr uint32_t kOzSbo = (kOzKC / 8) * 128;          // next 8-row group of core matrices
constexpr uint32_t kOzLbo = 128;                        // next 8-element K group
constexpr long kOzSpin = 1l << 26;                      // bounded mbarrier waits
constexpr int kOzThreads = 256;                         // 8 warps: two per TMEM lane quadrant

// Byte offset of element (i, k) inside a slice tile (K-major core matrices).
__host__ __device__ __forceinline__ uint32_t oz_offset(int i, int k) {
  return (uint32_t)((i >> 3) * kOzSbo + (k >> 3) * kOzLbo + (i & 7) * 16 + (k & 7) * 2);
}

// Element (i, k) of a strided view: P[i * rs + k * ks].
struct View {
  const double* p;
  int64_t rs, ks;
};

// Exponent of the largest magnitude of each row of the view (rows x K):
// 2^e > max |row|, e = 0 for a zero row.  One thread per row (rs == 1) or
// one warp per row (ks == 1).
__global__ void k_oz_rowexp(View v, int rows, int K, int rows_pad, int* __restrict__ e) {
  // magnitudes compared as FP64 bit patterns with the sign cleared (the
  // order of non-negative doubles), on the integer pipe
  const unsigned long long kMag = ~(1ull << 63);
  if (v.rs == 1) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows_pad; i += gridDim.x * blockDim.x) {
      unsigned long long mx = 0ull;
      if (i < rows)
        for (int k = 0; k < K; ++k) {
          const unsigned long long a = (unsigned long long)__double_as_longlong(v.p[i + k * v.ks]) & kMag;
          mx = a > mx ? a : mx;
        }
      e[i] = tc::exp_above(mx);
    }
  } else {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows_pad; i += warps) {
      unsigned long long mx = 0ull;
      if (i < rows)
        for (int k = lane; k < K; k += 32) {
          const unsigned long long a =
              (unsigned long long)__double_as_longlong(v.p[i * v.rs + (int64_t)k * v.ks]) & kMag;
          mx = a > mx ? a : mx;
        }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
      }
      if (lane == 0) e[i] = tc::exp_above(mx);
    }
  }
}

// Slices of the view: out[(((rt * KT + kt) * kOzS + p) * tile + oz_offset(i % TR, k % KC)]
// (the 8 slice tiles of one tile and K chunk are contiguous: one bulk copy)
// = n_p(i, k) for the tiles of TR rows and kOzKC columns; padding is zero.
// One thread per row and group of 8 consecutive k (one 16-byte row of a
// core matrix): 8 loads, and one 16-byte store per slice.
template <int TR>
__global__ void k_oz_split(View v, int rows, int K, const int* __restrict__ e, int RT, int KT,
                           __nv_bfloat16* __restrict__ out) {
  const int64_t rows_pad = (int64_t)RT * TR, groups = (int64_t)KT * (kOzKC / 8);
  const int64_t total = rows_pad * groups;
  const int64_t tile = (int64_t)TR * kOzKC;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    // consecutive threads take consecutive rows (coalesced when the view's
    // rows are unit-stride) or consecutive groups of a row (when k is)
    int64_t i, g;
    if (v.ks == 1) {
      i = t / groups;
      g = t - i * groups;
    } else {
      g = t / rows_pad;
      i = t - g * rows_pad;
    }
    const int64_t k0 = g * 8;
    const int ei = i < rows ? e[i] : 0;
    int n[8][kOzS];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t k = k0 + u;
      tc::digits8((i < rows && k < K) ? v.p[i * v.rs + k * v.ks] : 0.0, ei, n[u]);
    }
    const int rt = (int)(i / TR), kt = (int)(k0 / kOzKC);
    uint4* o = reinterpret_cast<uint4*>(out + ((int64_t)rt * KT + kt) * kOzS * tile +
                                        oz_offset((int)(i % TR), (int)(k0 % kOzKC)) / 2);
#pragma unroll
    for (int p = 0; p < kOzS; ++p) {
      uint32_t w[4];
#pragma unroll
      for (int u = 0; u < 8; u += 2) w[u / 2] = tc::bf16_int(n[u][p]) | (tc::bf16_int(n[u + 1][p]) << 16);
      o[p * (tile / 8)] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

using tc::smem_u32;

__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
  return tc::desc_kmajor(saddr, kOzLbo, kOzSbo);
}

__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity) {
  return tc::mbar_wait(bar, parity, kOzSpin);
}

// One CTA per 128 x 64 tile of C; 256 threads.
__global__ void __launch_bounds__(kOzThreads, 1) k_oz_mma(const uint8_t* __restrict__ As,
                                                   const uint8_t* __restrict__ Bs,
                                                   const int* __restrict__ eA,
                                                   const int* __restrict__ eB, int M, int N,
                                                   int MT, int NT, int KT, double alpha,
                                                   double beta, double* __restrict__ C,
                                                   int64_t ldc, uint32_t* __restrict__ flags) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + kOzS * kOzATile;
  __shared__ __align__(8) uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, nt = blockIdx.y;
  if (tid == 0) failed = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(kOzLevels * kOzTN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_load)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_mma)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = tc::idesc_bf16(kOzTM, kOzTN);
  // warps w and w + 4 share the lane quadrant w of tensor memory (rows
  // 32 w .. 32 w + 31 of the tile) and take one half of the columns each
  const int quad = warp & 3, half = warp >> 2;
  constexpr int kCols = kOzTN / 2;
  // exact integer accumulators: hi = sum over levels L = 0..3 of the level
  // sums 2^(7 (3-L)), lo likewise over L = 4..7 (weights 2^-35 and 2^-63)
  long long hi[kCols], lo[kCols];
#pragma unroll
  for (int j = 0; j < kCols; ++j) hi[j] = lo[j] = 0;
  for (int kt = 0; kt < KT; ++kt) {
    const uint32_t parity = kt & 1;
    if (tid == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(smem_u32(&bar_load)), "r"((uint32_t)kOzSmem) : "memory");
      // the chunk's 8 A slice tiles and 8 B slice tiles are contiguous: two
      // bulk copies (many small copies are processed one after another)
      {
        const uint8_t* src = As + ((int64_t)mt * KT + kt) * kOzS * kOzATile;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(smem_u32(sA)), "l"(src), "r"((uint32_t)(kOzS * kOzATile)),
                        "r"(smem_u32(&bar_load)) : "memory");
      }
      {
        const uint8_t* src = Bs + ((int64_t)nt * KT + kt) * kOzS * kOzBTile;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(smem_u32(sB)), "l"(src), "r"((uint32_t)(kOzS * kOzBTile)),
                        "r"(smem_u32(&bar_load)) : "memory");
      }
      if (!oz_wait(smem_u32(&bar_load), parity)) {
        failed = 1;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const bool range_start = (kt % kOzEpi) == 0;
        for (int p = 0; p < kOzS; ++p) {
          for (int q = 0; p + q < kOzLevels; ++q) {
            const uint32_t d = tmem + (uint32_t)((p + q) * kOzTN);
#pragma unroll
            for (int ks = 0; ks < kOzKC / 16; ++ks) {
              const uint64_t da = oz_desc(smem_u32(sA + p * kOzATile) + ks * 2 * kOzLbo);
              const uint64_t db = oz_desc(smem_u32(sB + q * kOzBTile) + ks * 2 * kOzLbo);
              const uint32_t accum = (p > 0 || ks > 0 || !range_start) ? 1u : 0u;
              asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                           "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                           :: "r"(d), "l"(da), "l"(db), "r"(idesc), "r"(accum) : "memory");
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&bar_mma)) : "memory");
      }
    }
    __syncthreads();
    if (failed) break;
    if (!oz_wait(smem_u32(&bar_mma), parity)) {
      if (lane == 0) failed = 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (failed) break;
    // the level sums stay in tensor memory until the end of a 256-wide range
    if ((kt % kOzEpi) != kOzEpi - 1 && kt != KT - 1) continue;
    // FP64 epilogue: row 32 warp + lane of the tile, 64 columns per level
    // levels lv0 .. lv0 + 3 into acc, level lv weighted 2^(7 (lv0 + 3 - lv))
    // levels lv0 .. lv0 + 3 into acc, level lv weighted 2^(7 (lv0 + 3 - lv))
    auto levels = [&](long long (&acc)[kCols], int lv0) {
#pragma unroll 1
      for (int lv = lv0; lv < lv0 + 4; ++lv) {
        const int sh = kOzBits * (lv0 + 3 - lv);
#pragma unroll
        for (int c0 = 0; c0 < kCols; c0 += 16) {
          uint32_t r[16];
          const uint32_t ta = tmem + ((uint32_t)(32 * quad) << 16) +
                              (uint32_t)(lv * kOzTN + half * kCols + c0);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                       : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                         "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                         "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                       : "r"(ta));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[c0 + j] += (long long)tc::f32_int(r[j]) << sh;
        }
      }
    };
    levels(hi, 0);
    levels(lo, 4);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (failed) {
    if (tid == 0) atomicOr(flags, kFlagTimeout);
  } else {
    const int row = mt * kOzTM + 32 * quad + lane;
    if (row < M) {
      const int ea = eA[row];
#pragma unroll
      for (int j = 0; j < kCols; ++j) {
        const int col = nt * kOzTN + half * kCols + j;
        if (col < N) {
          double* c = C + (int64_t)col * ldc + row;
          const int sc = ea + eB[col];
          const double v = alpha * (tc::i64_f64(hi[j], sc - 5 * kOzBits) +
                                    tc::i64_f64(lo[j], sc - 9 * kOzBits));
          *c = beta == 0.0 ? v : fma(beta, *c, v);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kOzLevels * kOzTN) : "memory");
}

int oz_grid(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

}  // namespace

size_t ozaki_work_bytes(int M, int N, int K) {
  const int64_t MT = (M + kOzTM - 1) / kOzTM, NT = (N + kOzTN - 1) / kOzTN;
  const int64_t KT = (K + kOzKC - 1) / kOzKC;
  return (size_t)(kOzS * MT * KT * kOzATile + kOzS * NT * KT * kOzBTile) +
         sizeof(int) * (size_t)(MT * kOzTM + NT * kOzTN) + 1024;
}

bool ozaki_enabled(int M, int N, int K) {
  // below these sizes the FP64 GEMM's few CTAs finish sooner than the splitting
  return M >= 256 && N >= 256 && K >= 64;
}

void ozaki_gemm(char ta, char tb, int M, int N, int K, double alpha, const double* A, int64_t lda,
                const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* work,
                uint32_t* flags, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_oz_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
    attr = true;
  }
  const int MT = (M + kOzTM - 1) / kOzTM, NT = (N + kOzTN - 1) / kOzTN;
  const int KT = (K + kOzKC - 1) / kOzKC;
  uint8_t* base = static_cast<uint8_t*>(work);
  uint8_t* As = base;
  uint8_t* Bs = As + (size_t)kOzS * MT * KT * kOzATile;
  int* eA = reinterpret_cast<int*>(Bs + (size_t)kOzS * NT * KT * kOzBTile);
  int* eB = eA + (size_t)MT * kOzTM;
  // op(A)(i, k) and B^T(j, k) = op(B)(k, j) as strided views
  const View va = ta == 'N' ? View{A, 1, lda} : View{A, lda, 1};
  const View vb = tb == 'N' ? View{B, ldb, 1} : View{B, 1, ldb};
  count_launches(5);
  k_oz_rowexp<<<oz_grid((int64_t)MT * kOzTM * (va.rs == 1 ? 1 : 32), 256), 256, 0, st>>>(
      va, M, K, MT * kOzTM, eA);
  k_oz_rowexp<<<oz_grid((int64_t)NT * kOzTN * (vb.rs == 1 ? 1 : 32), 256), 256, 0, st>>>(
      vb, N, K, NT * kOzTN, eB);
  k_oz_split<kOzTM><<<oz_grid((int64_t)MT * kOzTM * KT * kOzKC, 256), 256, 0, st>>>(
      va, M, K, eA, MT, KT, reinterpret_cast<__nv_bfloat16*>(As));
  k_oz_split<kOzTN><<<oz_grid((int64_t)NT * kOzTN * KT * kOzKC, 256), 256, 0, st>>>(
      vb, N, K, eB, NT, KT, reinterpret_cast<__nv_bfloat16*>(Bs));
  k_oz_mma<<<dim3((unsigned)MT, (unsigned)NT), kOzThreads, kOzSmem, st>>>(As, Bs, eA, eB, M, N, MT, NT,
                                                                    KT, alpha, beta, C, ldc, flags);
}

}  // namespace spk
