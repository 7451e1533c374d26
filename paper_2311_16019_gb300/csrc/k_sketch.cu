// Subsampled randomized Hadamard sketch (Section 2.2 of the paper) on sm_103a.
//
// S = (1/sqrt(s)) D H_{n'} E P: E = diag(e_i) Rademacher signs, P zero-pads
// length n to n' = 2^ceil(log2 n), H_{n'} the unnormalised Walsh-Hadamard
// transform, D selects s rows rho_0 < ... < rho_{s-1}.  Entry-wise
//     S[j, i] = e_i (-1)^popcount(rho_j & i) / sqrt(s).
//
// Random draws: SplitMix64 (Steele, Lea, Flood 2014; Vigna's reference
// definition), i-th output of a stream started at x0 is
//     z = x0 + (i+1)*0x9E3779B97F4A7C15; z = (z^(z>>30))*0xBF58476D1CE4E5B9;
//     z = (z^(z>>27))*0x94D049BB133111EB; out = z^(z>>31).
// x0 = seed + (1 + 2*sketch_id + sub)*0x632BE59BD9B4E019, sub 0 = row keys,
// sub 1 = signs.  e_i = 1 - 2*(out_i >> 63); the rows are the s indices of
// [0, n') with the smallest keys (distinct: the map i -> key is injective).
//
// Application, two levels (n' = n1 * n2, i = c*n2 + t):
//   (-1)^popcount(rho & i) = (-1)^popcount(rho_hi & c) * (-1)^popcount(rho_lo & t)
// pass 1: per chunk c, load e_i x_i into shared memory and run the length-n2
//         butterfly transform; store y[t][c][col];
// pass 2: per selected row j, sum over the n1 chunks with the +-1 pattern of
//         rho_hi; one warp per row, fixed summation order (deterministic).
#include "spk_internal.cuh"

#include <atomic>

#include <cmath>
#include <cstdio>
#include <vector>

namespace spk {

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStream = 0x632BE59BD9B4E019ull;

__host__ __device__ __forceinline__ uint64_t splitmix_at(uint64_t x0, uint64_t i) {
  uint64_t z = x0 + (i + 1ull) * kGamma;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_sign_draws(int64_t n, uint64_t x0, int8_t* signs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    signs[i] = (splitmix_at(x0, (uint64_t)i) >> 63) ? (int8_t)-1 : (int8_t)1;
  }
}

__global__ void k_candidates(int64_t npad, uint64_t x0, uint64_t thr, int32_t cap,
                             int32_t* cnt, int32_t* cidx, uint64_t* ckey) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npad;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = splitmix_at(x0, (uint64_t)i);
    if (k <= thr) {
      int pos = atomicAdd(cnt, 1);
      if (pos < cap) {
        cidx[pos] = (int32_t)i;
        ckey[pos] = k;
      }
    }
  }
}

// selected[c] = (number of candidate keys smaller than key c) < s
__global__ void k_rank_keys(const int32_t* cnt_p, const uint64_t* ckey, int32_t s, int8_t* sel) {
  const int cnt = *cnt_p;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cnt; c += gridDim.x * blockDim.x) {
    const uint64_t kc = ckey[c];
    int rank = 0;
    for (int o = 0; o < cnt; ++o) rank += (ckey[o] < kc);
    sel[c] = rank < s;
  }
}

// rows[pos] = index, pos = number of selected candidates with a smaller index
__global__ void k_place_rows(const int32_t* cnt_p, const int32_t* cidx, const int8_t* sel,
                             int32_t* rows) {
  const int cnt = *cnt_p;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cnt; c += gridDim.x * blockDim.x) {
    if (!sel[c]) continue;
    const int ic = cidx[c];
    int pos = 0;
    for (int o = 0; o < cnt; ++o) pos += (sel[o] && cidx[o] < ic);
    rows[pos] = ic;
  }
}

// First level of the transform: for chunk q (blockIdx.x) and column c
// (blockIdx.y), the length-n2 Walsh-Hadamard transform of the signed rows
// q*n2 .. q*n2+n2-1 of column c, written to Y[(t*n1 + q)*r + c].  The stages
// (butterflies a+b, a-b at distance h = 1, 2, 4, ...) are taken three at a
// time on eight values held in registers, one shared-memory round trip per
// three stages; the operations and their order are those of the radix-2
// sweep.
template <typename TC>
__device__ __forceinline__ void bfly(TC& a, TC& b) {
  const TC x = a, y = b;
  a = x + y;
  b = x - y;
}

template <typename TB, typename TC>
__global__ void __launch_bounds__(512) k_fwht_chunks(const TB* __restrict__ X, int64_t n, int r,
                                                     const int8_t* __restrict__ signs, int n2,
                                                     int log2n2, int64_t n1, TC* __restrict__ Y) {
  extern __shared__ unsigned char smem_raw[];
  TC* buf = reinterpret_cast<TC*>(smem_raw);
  const int64_t chunk = blockIdx.x;
  const int c = blockIdx.y;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const int64_t row = chunk * n2 + t;
    TC v = TC(0);
    if (row < n) {
      v = TC(Store<TB>::ld(X + row * r + c));
      if (signs[row] < 0) v = -v;
    }
    buf[t] = v;
  }
  __syncthreads();
  int lg = 0;
  for (; lg + 3 <= log2n2; lg += 3) {
    const int h = 1 << lg;
    for (int b = threadIdx.x; b < (n2 >> 3); b += blockDim.x) {
      const int base = ((b >> lg) << (lg + 3)) + (b & (h - 1));
      TC v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = buf[base + k * h];
#pragma unroll
      for (int k = 0; k < 8; k += 2) bfly(v[k], v[k + 1]);       // distance h
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (!(k & 2)) bfly(v[k], v[k + 2]);                       // distance 2h
#pragma unroll
      for (int k = 0; k < 4; ++k) bfly(v[k], v[k + 4]);           // distance 4h
#pragma unroll
      for (int k = 0; k < 8; ++k) buf[base + k * h] = v[k];
    }
    __syncthreads();
  }
  for (; lg < log2n2; ++lg) {
    const int h = 1 << lg;
    for (int b = threadIdx.x; b < (n2 >> 1); b += blockDim.x) {
      const int i = ((b >> lg) << (lg + 1)) + (b & (h - 1));
      TC a = buf[i], bb = buf[i + h];
      bfly(a, bb);
      buf[i] = a;
      buf[i + h] = bb;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n2; t += blockDim.x) Y[((int64_t)t * n1 + chunk) * r + c] = buf[t];
}

// One warp per selected row; the r column sums end in a reduce-scatter
// warp sum (6 additions per lane for r = 4 instead of 20).
template <typename TC, int R>
__global__ void k_gather_rows(const TC* __restrict__ Y, int64_t n1, int n2, int log2n2,
                              const int32_t* __restrict__ rows, int32_t s, double scale,
                              double* __restrict__ SX) {
  __shared__ double out[8][R];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int wl = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= s) return;
  const int32_t rho = rows[warp];
  const int64_t lo = rho & (n2 - 1);
  const int64_t hi = (int64_t)rho >> log2n2;
  double acc[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = 0.0;
  for (int64_t c = lane; c < n1; c += 32) {
    const bool neg = __popcll((unsigned long long)(hi & c)) & 1;
    const TC* y = Y + (lo * n1 + c) * R;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const double v = (double)y[k];
      acc[k] += neg ? -v : v;
    }
  }
  warp_sum_store<R>(acc, out[wl]);
  __syncwarp();
  if (lane < R) SX[warp + (int64_t)lane * s] = out[wl][lane] * scale;
}

template <typename TB>
__global__ void k_identity_sketch(const TB* __restrict__ X, int64_t n, int r, double scale,
                                  double* __restrict__ SX) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r;
    const int c = (int)(e - i * r);
    SX[i + (int64_t)c * n] = (double)Store<TB>::ld(X + e) * scale;
  }
}

int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

static int64_t next_pow2(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

static size_t cand_cap(int64_t npad, int32_t s) {
  double expect = s + 6.0 * std::sqrt((double)s) + 64.0;
  size_t cap = (size_t)(2.0 * expect) + 1024;
  if ((int64_t)cap > npad) cap = (size_t)npad;
  return cap;
}

size_t sketch_draws_scratch_bytes(int64_t n, int32_t s, int64_t range) {
  const int64_t npad = range > 0 ? range : next_pow2(n);
  const size_t cap = cand_cap(npad, s);
  return 256 + cap * (sizeof(int32_t) + sizeof(uint64_t) + sizeof(int8_t)) + 3 * 256;
}

int sketch_draws_launch(int64_t n, int32_t s, uint64_t seed, int32_t sketch_id, int32_t* rows,
                        int8_t* signs, void* scratch, size_t scratch_bytes, cudaStream_t st,
                        char* err, size_t errlen, int64_t range) {
  // rows are drawn over [0, range): the padded length n' for the SRHT, n for
  // the DCT sketch
  const int64_t npad = range > 0 ? range : next_pow2(n);
  if (s < 1 || s > npad) {
    snprintf(err, errlen, "sketch rows s=%d must lie in [1, %lld]", s, (long long)npad);
    return SPK_ERR_ARG;
  }
  const uint64_t x0r = seed + (uint64_t)(1 + 2 * sketch_id + 0) * kStream;
  const uint64_t x0s = seed + (uint64_t)(1 + 2 * sketch_id + 1) * kStream;
  count_launches(1);
  k_sign_draws<<<grid_for(n, 256), 256, 0, st>>>(n, x0s, signs);
  const size_t cap = cand_cap(npad, s);
  if (scratch_bytes < sketch_draws_scratch_bytes(n, s, range)) {
    snprintf(err, errlen, "sketch scratch too small");
    return SPK_ERR_ARG;
  }
  char* base = static_cast<char*>(scratch);
  int32_t* cnt = reinterpret_cast<int32_t*>(base);
  uint64_t* ckey = reinterpret_cast<uint64_t*>(base + 256);
  int32_t* cidx = reinterpret_cast<int32_t*>(base + 256 + cap * sizeof(uint64_t));
  int8_t* sel = reinterpret_cast<int8_t*>(base + 256 + cap * (sizeof(uint64_t) + sizeof(int32_t)));
  // threshold on the uniform keys: expected count ~ s + 6 sqrt(s) + 64
  double frac = (s + 6.0 * std::sqrt((double)s) + 64.0) / (double)npad;
  for (int attempt = 0; attempt < 12; ++attempt) {
    uint64_t thr;
    if (frac >= 1.0) thr = ~0ull;
    else thr = (uint64_t)(frac * 18446744073709551616.0);
    if (cudaMemsetAsync(cnt, 0, sizeof(int32_t), st) != cudaSuccess) return SPK_ERR_CUDA;
    count_launches(1);
    k_candidates<<<grid_for(npad, 256), 256, 0, st>>>(npad, x0r, thr, (int32_t)cap, cnt, cidx, ckey);
    // a copy into pageable host memory blocks until the stream's earlier
    // work is done, without a limit: drain the stream by a bounded wait
    // first, so that the copy starts at once, then wait for the copy
    int32_t hcnt = 0;
    int w = bounded_stream_wait(st, kHostWaitSeconds);
    if (w == 0) {
      if (cudaMemcpyAsync(&hcnt, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SPK_ERR_CUDA;
      w = bounded_stream_wait(st, kHostWaitSeconds);
    }
    if (w == 1) {
      snprintf(err, errlen, "sketch row selection: device work did not finish");
      return SPK_ERR_TIMEOUT;
    }
    if (w != 0) return SPK_ERR_CUDA;
    if (hcnt < s) { frac = frac * 1.5 + 1e-12; continue; }
    if ((size_t)hcnt > cap) { frac = frac * 0.8; continue; }
    const int g = grid_for(hcnt, 256);
    count_launches(1);
    k_rank_keys<<<g, 256, 0, st>>>(cnt, ckey, s, sel);
    count_launches(1);
    k_place_rows<<<g, 256, 0, st>>>(cnt, cidx, sel, rows);
    return cudaGetLastError() == cudaSuccess ? SPK_OK : SPK_ERR_CUDA;
  }
  snprintf(err, errlen, "sketch row selection did not settle");
  return SPK_ERR_ARG;
}

void sketch_geometry(SketchDev& sk, int64_t n, int32_t s, int identity, int elem_bytes, int r) {
  sk.n = n;
  sk.identity = identity;
  if (identity) {
    sk.s = (int32_t)n;
    sk.npad = n;
    sk.n2 = 1;
    sk.log2n2 = 0;
    sk.n1 = n;
    sk.scale = 1.0;
    return;
  }
  sk.s = s;
  sk.npad = next_pow2(n);
  // largest power of two chunk that fits 128 KB of shared memory
  int64_t n2 = 4096;
  while (n2 > 1 && n2 * r * elem_bytes > 128 * 1024) n2 >>= 1;
  if (n2 > sk.npad) n2 = sk.npad;
  sk.n2 = (int32_t)n2;
  int l = 0;
  while ((1ll << l) < n2) ++l;
  sk.log2n2 = l;
  sk.n1 = sk.npad / n2;
  sk.scale = 1.0 / std::sqrt((double)s);
}

size_t sketch_apply_scratch_bytes(const SketchDev& sk, int r) {
  if (sk.identity) return 0;
  return (size_t)sk.npad * r * sizeof(double);
}

template <typename TB, typename TC>
void sketch_apply_launch(const SketchDev& sk, const TB* X, int r, double* SX, TC* scratch,
                         cudaStream_t st) {
  if (sk.identity) {
    count_launches(1);
    k_identity_sketch<TB><<<grid_for(sk.n * r, 256), 256, 0, st>>>(X, sk.n, r, sk.scale, SX);
    return;
  }
  if (sk.is_dct) {
    dct_apply_launch<TB>(sk, X, r, SX, sk.cwork, st);
    return;
  }
  const size_t smem = (size_t)sk.n2 * sizeof(TC);
  const int threads = (int)std::min<int64_t>(512, std::max<int64_t>(32, (int64_t)sk.n2 >> 3));
  count_launches(1);
  k_fwht_chunks<TB, TC><<<dim3((unsigned)sk.n1, (unsigned)r), threads, smem, st>>>(
      X, sk.n, r, sk.signs, sk.n2, sk.log2n2, sk.n1, scratch);
  const int warps_per_block = 8;
  const int blocks = (sk.s + warps_per_block - 1) / warps_per_block;
  count_launches(1);
  switch (r) {
    case 1:
      k_gather_rows<TC, 1><<<blocks, warps_per_block * 32, 0, st>>>(
          scratch, sk.n1, sk.n2, sk.log2n2, sk.rows, sk.s, sk.scale, SX);
      break;
    case 2:
      k_gather_rows<TC, 2><<<blocks, warps_per_block * 32, 0, st>>>(
          scratch, sk.n1, sk.n2, sk.log2n2, sk.rows, sk.s, sk.scale, SX);
      break;
    case 3:
      k_gather_rows<TC, 3><<<blocks, warps_per_block * 32, 0, st>>>(
          scratch, sk.n1, sk.n2, sk.log2n2, sk.rows, sk.s, sk.scale, SX);
      break;
    default:
      k_gather_rows<TC, 4><<<blocks, warps_per_block * 32, 0, st>>>(
          scratch, sk.n1, sk.n2, sk.log2n2, sk.rows, sk.s, sk.scale, SX);
      break;
  }
}

template void sketch_apply_launch<double, double>(const SketchDev&, const double*, int, double*,
                                                  double*, cudaStream_t);
template void sketch_apply_launch<float, float>(const SketchDev&, const float*, int, double*,
                                                float*, cudaStream_t);
template void sketch_apply_launch<__nv_bfloat16, float>(const SketchDev&, const __nv_bfloat16*,
                                                        int, double*, float*, cudaStream_t);

}  // namespace spk
