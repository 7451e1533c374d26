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
// FP32 accumulator in tensor memory over K-ranges of 256 (16 stages of 16
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
// K-major, no swizzle, the 8 slices of a tile and 16-wide K stage stored
// together), k_oz_gemm (persistent, one CTA per SM over 128 x 32 tiles of C:
// a copy lane, an MMA lane and four epilogue warps, with a 4-stage ring of
// shared-memory buffers and two accumulator sets in tensor memory, so that
// copies, MMAs and the epilogue of the previous K range overlap).
#include "spk_internal.cuh"
#include "tc_common.cuh"

#include <algorithm>

namespace spk {

namespace {

constexpr int kOzS = 8;          // slices per operand
constexpr int kOzBits = 7;       // bits per slice
constexpr int kOzTM = 128;       // tile rows (M of the MMA)
constexpr int kOzTN = 32;        // tile columns (N of the MMA)
constexpr int kOzKS = 16;        // K per pipeline stage (one MMA per slice pair)
constexpr int kOzStages = 4;     // stages in flight
constexpr int kOzRange = 256;    // K accumulated exactly in tensor memory between epilogues
constexpr int kOzLevels = 8;     // levels L = 2 .. 9
constexpr int kOzATile = kOzTM * kOzKS * 2;   // bytes of one A slice tile (4 KB)
constexpr int kOzBTile = kOzTN * kOzKS * 2;   // bytes of one B slice tile (1 KB)
constexpr int kOzAStage = kOzS * kOzATile;    // 32 KB
constexpr int kOzBStage = kOzS * kOzBTile;    // 8 KB
constexpr int kOzStage = kOzAStage + kOzBStage;
constexpr int kOzSmem = kOzStages * kOzStage; // 160 KB
constexpr int kOzSetCols = kOzLevels * kOzTN; // tensor-memory columns of one accumulator set
constexpr uint32_t kOzSbo = (kOzKS / 8) * 128;          // next 8-row group of core matrices
constexpr uint32_t kOzLbo = 128;                        // next 8-element K group
constexpr long kOzSpin = 1l << 26;                      // bounded mbarrier waits
constexpr int kOzThreads = 192;  // warp 0 copies, warp 1 MMAs, warps 2..5 epilogue

static_assert(kOzRange % kOzKS == 0, "stages tile an exact range");
static_assert(2 * kOzSetCols <= 512, "two accumulator sets fit in tensor memory");

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

// Slices of the view: out[(((rt * KT + kt) * kOzS + p) * tile + oz_offset(i % TR, k % kOzKS)]
// for tiles of TR rows and kOzKS columns (the 8 slice tiles of one tile and
// stage are contiguous: one bulk copy); padding is zero.  One thread per row
// and group of 8 consecutive k (one 16-byte row of a core matrix): 8 loads,
// and one 16-byte store per slice.
template <int TR>
__global__ void k_oz_split(View v, int rows, int K, const int* __restrict__ e, int RT, int KT,
                           __nv_bfloat16* __restrict__ out) {
  const int64_t rows_pad = (int64_t)RT * TR, groups = (int64_t)KT * (kOzKS / 8);
  const int64_t total = rows_pad * groups;
  const int64_t tile = (int64_t)TR * kOzKS;
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
    const int rt = (int)(i / TR), kt = (int)(k0 / kOzKS);
    uint4* o = reinterpret_cast<uint4*>(out + ((int64_t)rt * KT + kt) * kOzS * tile +
                                        oz_offset((int)(i % TR), (int)(k0 % kOzKS)) / 2);
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

// Persistent, one CTA per SM; tiles of 128 x 32 of C taken round robin,
// each in units of kOzRange K positions.
//   warp 0, lane 0:  bulk copies of the stages (A slices 32 KB, B slices 8 KB)
//                    into a ring of kOzStages buffers;
//   warp 1, lane 0:  36 MMAs per stage into accumulator set u & 1 of unit u
//                    (8 levels x 32 columns), commits releasing the stage
//                    and, at the end of the unit, the set;
//   warps 2..5:      epilogue of unit u while the MMAs of unit u + 1 run:
//                    level sums as integers into exact 64-bit accumulators,
//                    then, after the tile's last unit, C = alpha (.) + beta C.
// Every wait is bounded; on expiry the kernel sets the timeout flag, stops
// issuing, and returns after the others have stopped too.
__global__ void __launch_bounds__(kOzThreads, 1) k_oz_gemm(const uint8_t* __restrict__ As,
                                                    const uint8_t* __restrict__ Bs,
                                                    const int* __restrict__ eA,
                                                    const int* __restrict__ eB, int M, int N,
                                                    int MT, int NT, int KT, int S, int ups,
                                                    double alpha, double beta,
                                                    double* __restrict__ C, int64_t ldc,
                                                    double* __restrict__ partial,
                                                    uint32_t* __restrict__ flags) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[kOzStages], empty[kOzStages], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed_s;
  volatile int& failed = failed_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // work items: (tile, K split), the tile's column block fastest so that the
  // CTAs sharing a block of A rows run together; item w covers the units
  // (kOzRange K positions each) ups w_s .. ups (w_s + 1) - 1 of its tile
  const int nitems = MT * NT * S;
  constexpr int kPerRange = kOzRange / kOzKS;
  const int nr = (KT + kPerRange - 1) / kPerRange;     // units per tile
  auto item = [&](int w, int& mt, int& nt, int& r0, int& r1) {
    nt = w % NT;
    const int rest = w / NT;
    const int sk = rest % S;
    mt = rest / S;
    r0 = sk * ups;
    r1 = min(nr, r0 + ups);
  };
  int64_t total = 0;                                    // stages of this CTA
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    int mt, nt, r0, r1;
    item(w, mt, nt, r0, r1);
    total += min(KT, r1 * kPerRange) - r0 * kPerRange;
  }
  if (tid == 0) failed = 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(2 * kOzSetCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int q = 0; q < kOzStages; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[q])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[q])) : "memory");
    }
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&tfull[q])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" :: "r"(smem_u32(&tempty[q])) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;
      for (int w = blockIdx.x; w < nitems && !failed; w += gridDim.x) {
        int mt, nt, r0, r1;
        item(w, mt, nt, r0, r1);
        for (int kt = r0 * kPerRange; kt < min(KT, r1 * kPerRange); ++kt, ++g) {
          const int slot = (int)(g % kOzStages);
          const int64_t use = g / kOzStages;
          if (use > 0 && !oz_wait(smem_u32(&empty[slot]), (uint32_t)((use - 1) & 1))) {
            failed = 1;
            break;
          }
          if (failed) break;
          uint8_t* sA = smem + slot * kOzStage;
          uint8_t* sB = sA + kOzAStage;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                       :: "r"(smem_u32(&full[slot])), "r"((uint32_t)kOzStage) : "memory");
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                       :: "r"(smem_u32(sA)), "l"(As + ((int64_t)mt * KT + kt) * kOzAStage),
                          "r"((uint32_t)kOzAStage), "r"(smem_u32(&full[slot])) : "memory");
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                       :: "r"(smem_u32(sB)), "l"(Bs + ((int64_t)nt * KT + kt) * kOzBStage),
                          "r"((uint32_t)kOzBStage), "r"(smem_u32(&full[slot])) : "memory");
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16(kOzTM, kOzTN);
      int64_t g = 0, u = 0;
      for (int w = blockIdx.x; w < nitems && !failed; w += gridDim.x) {
        int mt, nt, r0, r1;
        item(w, mt, nt, r0, r1);
        for (int r = r0; r < r1 && !failed; ++r, ++u) {
          const int set = (int)(u & 1);
          const int64_t uses = u >> 1;
          if (uses > 0 && !oz_wait(smem_u32(&tempty[set]), (uint32_t)((uses - 1) & 1))) {
            failed = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int k0 = r * kPerRange, k1 = min(KT, k0 + kPerRange);
          bool ok = true;
          for (int kt = k0; kt < k1; ++kt, ++g) {
            const int slot = (int)(g % kOzStages);
            if (!oz_wait(smem_u32(&full[slot]), (uint32_t)((g / kOzStages) & 1)) || failed) {
              failed = 1;
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sA = smem_u32(smem + slot * kOzStage);
            const uint32_t sB = sA + kOzAStage;
#pragma unroll
            for (int p = 0; p < kOzS; ++p) {
              const uint64_t da = oz_desc(sA + p * kOzATile);
#pragma unroll
              for (int q = 0; p + q < kOzLevels; ++q) {
                const uint64_t db = oz_desc(sB + q * kOzBTile);
                const uint32_t d = tmem + (uint32_t)(set * kOzSetCols + (p + q) * kOzTN);
                const uint32_t accum = (p > 0 || kt > k0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                             :: "r"(d), "l"(da), "l"(db), "r"(idesc), "r"(accum) : "memory");
              }
            }
            // release the stage buffer to a later copy of this CTA only (an
            // arrive nobody waits for must not be left pending)
            if (g + kOzStages < total)
              asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                           :: "r"(smem_u32(&empty[slot])) : "memory");
          }
          if (!ok) break;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(smem_u32(&tfull[set])) : "memory");
        }
      }
    }
  } else {
    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (tile rows)
    const int quad = warp & 3;
    const int rt = 32 * quad + lane;
    const uint32_t trow = tmem + ((uint32_t)(32 * quad) << 16);
    long long hi[kOzTN], lo[kOzTN];
#pragma unroll
    for (int j = 0; j < kOzTN; ++j) hi[j] = lo[j] = 0;
    int64_t u = 0;
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
      int mt, nt, r0, r1;
      item(w, mt, nt, r0, r1);
      bool stop = false;
      for (int r = r0; r < r1; ++r, ++u) {
        const int set = (int)(u & 1);
        bool got = !failed && oz_wait(smem_u32(&tfull[set]), (uint32_t)((u >> 1) & 1));
        got = __all_sync(0xffffffffu, got);        // the loads below are .aligned
        if (!got) {
          if (lane == 0) failed = 1;
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // two levels per round: both loads issued, then one wait (each
        // wait is a round trip to tensor memory)
        auto two_levels = [&](long long (&acc)[kOzTN], int lv, int sh0) {
          uint32_t v[2][kOzTN];
#pragma unroll
          for (int h = 0; h < 2; ++h)
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(v[h][0]), "=r"(v[h][1]), "=r"(v[h][2]), "=r"(v[h][3]), "=r"(v[h][4]),
                           "=r"(v[h][5]), "=r"(v[h][6]), "=r"(v[h][7]), "=r"(v[h][8]), "=r"(v[h][9]),
                           "=r"(v[h][10]), "=r"(v[h][11]), "=r"(v[h][12]), "=r"(v[h][13]),
                           "=r"(v[h][14]), "=r"(v[h][15]), "=r"(v[h][16]), "=r"(v[h][17]),
                           "=r"(v[h][18]), "=r"(v[h][19]), "=r"(v[h][20]), "=r"(v[h][21]),
                           "=r"(v[h][22]), "=r"(v[h][23]), "=r"(v[h][24]), "=r"(v[h][25]),
                           "=r"(v[h][26]), "=r"(v[h][27]), "=r"(v[h][28]), "=r"(v[h][29]),
                           "=r"(v[h][30]), "=r"(v[h][31])
                         : "r"(trow + (uint32_t)(set * kOzSetCols + (lv + h) * kOzTN)));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < kOzTN; ++j)
            acc[j] += ((long long)tc::f32_int(v[0][j]) << sh0) +
                      ((long long)tc::f32_int(v[1][j]) << (sh0 - kOzBits));
        };
        // level lv of hi (lv < 4) weighs 2^(7 (3 - lv)), of lo 2^(7 (7 - lv))
        two_levels(hi, 0, 3 * kOzBits);
        two_levels(hi, 2, 1 * kOzBits);
        two_levels(lo, 4, 3 * kOzBits);
        two_levels(lo, 6, 1 * kOzBits);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&tempty[set])) : "memory");
      }
      if (stop) break;
      const int row = mt * kOzTM + rt;
      if (row < M) {
        const int ea = eA[row];
#pragma unroll
        for (int j = 0; j < kOzTN; ++j) {
          const int col = nt * kOzTN + j;
          if (col < N) {
            const int sc = ea + eB[col];
            const double v = alpha * (tc::i64_f64(hi[j], sc - 5 * kOzBits) +
                                      tc::i64_f64(lo[j], sc - 9 * kOzBits));
            if (S == 1) {
              double* c = C + (int64_t)col * ldc + row;
              *c = beta == 0.0 ? v : fma(beta, *c, v);
            } else {
              // K split: partial sums (column-major M x N per split), added
              // in split order by k_oz_reduce
              partial[((int64_t)(r0 / ups) * N + col) * M + row] = v;
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kOzTN; ++j) hi[j] = lo[j] = 0;
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && failed) atomicOr(flags, kFlagTimeout);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(2 * kOzSetCols) : "memory");
}

// C = beta C + sum over the S splits (in order) of the partial products.
__global__ void k_oz_reduce(const double* __restrict__ partial, int M, int N, int S, double beta,
                            double* __restrict__ C, int64_t ldc) {
  const int64_t count = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = partial[e];
    for (int k = 1; k < S; ++k) s += partial[(int64_t)k * count + e];
    const int64_t col = e / M, row = e - col * M;
    double* c = C + col * ldc + row;
    *c = beta == 0.0 ? s : fma(beta, *c, s);
  }
}

int oz_grid(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

int oz_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;
  }
  return n;
}

// K splits: enough work items for about two per SM when the tiles alone are
// fewer, each split at least one exact range of K.
void oz_splits(int M, int N, int K, int* S, int* ups) {
  const int64_t tiles = (int64_t)((M + kOzTM - 1) / kOzTM) * ((N + kOzTN - 1) / kOzTN);
  const int nr = (K + kOzRange - 1) / kOzRange;
  int want = tiles >= 2 * 152 ? 1 : (int)std::min<int64_t>(nr, (2 * 152 + tiles - 1) / tiles);
  want = std::max(1, want);
  *ups = (nr + want - 1) / want;
  *S = (nr + *ups - 1) / *ups;
}

}  // namespace

// Work of every product with M' <= M, N' <= N, K' <= K: the slices, the
// exponents and the K-split partial sums, S' M' N' <= M N + 2 152 kOzTM kOzTN
// doubles (a split happens only when the tiles, each kOzTM x kOzTN, number
// fewer than 2 x 152).
size_t ozaki_work_bytes(int M, int N, int K) {
  const int64_t MT = (M + kOzTM - 1) / kOzTM, NT = (N + kOzTN - 1) / kOzTN;
  const int64_t KT = (K + kOzKS - 1) / kOzKS;
  return (size_t)(MT * KT * kOzAStage + NT * KT * kOzBStage) +
         sizeof(int) * (size_t)(MT * kOzTM + NT * kOzTN) + 1024 +
         sizeof(double) * ((size_t)M * N + 2 * 152 * (size_t)kOzTM * kOzTN) + 256;
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
    cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
    attr = true;
  }
  const int MT = (M + kOzTM - 1) / kOzTM, NT = (N + kOzTN - 1) / kOzTN;
  const int KT = (K + kOzKS - 1) / kOzKS;
  uint8_t* base = static_cast<uint8_t*>(work);
  uint8_t* As = base;
  uint8_t* Bs = As + (size_t)MT * KT * kOzAStage;
  int* eA = reinterpret_cast<int*>(Bs + (size_t)NT * KT * kOzBStage);
  int* eB = eA + (size_t)MT * kOzTM;
  int S = 1, ups = 1;
  oz_splits(M, N, K, &S, &ups);
  double* partial = nullptr;
  if (S > 1) {
    const uintptr_t p = reinterpret_cast<uintptr_t>(eB + (size_t)NT * kOzTN);
    partial = reinterpret_cast<double*>((p + 255) & ~(uintptr_t)255);
  }
  // op(A)(i, k) and B^T(j, k) = op(B)(k, j) as strided views
  const View va = ta == 'N' ? View{A, 1, lda} : View{A, lda, 1};
  const View vb = tb == 'N' ? View{B, ldb, 1} : View{B, 1, ldb};
  count_launches(5);
  k_oz_rowexp<<<oz_grid((int64_t)MT * kOzTM * (va.rs == 1 ? 1 : 32), 256), 256, 0, st>>>(
      va, M, K, MT * kOzTM, eA);
  k_oz_rowexp<<<oz_grid((int64_t)NT * kOzTN * (vb.rs == 1 ? 1 : 32), 256), 256, 0, st>>>(
      vb, N, K, NT * kOzTN, eB);
  k_oz_split<kOzTM><<<oz_grid((int64_t)MT * kOzTM * KT * (kOzKS / 8), 256), 256, 0, st>>>(
      va, M, K, eA, MT, KT, reinterpret_cast<__nv_bfloat16*>(As));
  k_oz_split<kOzTN><<<oz_grid((int64_t)NT * kOzTN * KT * (kOzKS / 8), 256), 256, 0, st>>>(
      vb, N, K, eB, NT, KT, reinterpret_cast<__nv_bfloat16*>(Bs));
  const int grid = std::min(MT * NT * S, oz_sm_count());
  k_oz_gemm<<<grid, kOzThreads, kOzSmem, st>>>(As, Bs, eA, eB, M, N, MT, NT, KT, S, ups, alpha,
                                               beta, C, ldc, partial, flags);
  if (S > 1) {
    count_launches(1);
    k_oz_reduce<<<oz_grid((int64_t)M * N, 256), 256, 0, st>>>(partial, M, N, S, beta, C, ldc);
  }
}

}  // namespace spk
