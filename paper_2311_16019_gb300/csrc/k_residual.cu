// True residual of a factored solution (no counterpart step in Algorithm 1,
// whose stopping test is the sketched estimate of Eq. (3.5)):
//
//     R = A X + X B - C1 C2^T,  X = X1 X2^T,
//     R = L M^T,  L = [A X1, X1, -C1],  M = [X2, B^T X2, C2]   (n1 x w, n2 x w)
//
// since X B = X1 (B^T X2)^T.  ||R||_F^2 = trace(L^T L M^T M) = sum_ij G_ij H_ij
// with G = L^T L and H = M^T M (w x w, w = 2 ell + r).  X is never formed.
//
// The terms of R cancel: at a relative residual of 1e-8 the result is about
// 1e-16 of sum |G_ij H_ij|.  Gram matrices accumulated in FP64 carry errors
// of u |L_i|^T |L_j| per entry (u = 2^-53), which would swamp that; here every
// Gram entry and the final trace are accumulated in double-double arithmetic
// (an unevaluated sum hi + lo, with Knuth's TwoSum for the additions and the
// FMA-based TwoProduct for the products: Ogita, Rump and Oishi, "Accurate sum
// and dot product", SIAM J. Sci. Comput. 26 (2005), Algorithm Dot2).  The
// error of each entry is then of order n u^2 |L_i|^T |L_j|, and ||R||_F is
// resolved down to roughly sqrt(n) u (||L|| ||M||) instead of sqrt(u).
//
// Every operation below that must stay exact is written with the _rn
// intrinsics, which the compiler never contracts into an FMA.
#include "spk_internal.cuh"

#include <algorithm>

namespace spk {

namespace {

constexpr int kGT = 32;        // Gram tile (kGT x kGT entries per CTA)
constexpr int kGRows = 32;     // rows staged in shared memory per step
constexpr int kGThreads = 256; // 8 warps: warp y owns rows y, y+8, y+16, y+24 of the tile

// hi + lo += a * b (TwoProduct of a b, TwoSum into hi, errors into lo)
__device__ __forceinline__ void dd_acc(double& hi, double& lo, double a, double b) {
  const double p = __dmul_rn(a, b);
  const double pe = __fma_rn(a, b, -p);
  const double s = __dadd_rn(hi, p);
  const double bb = __dsub_rn(s, hi);
  const double e = __dadd_rn(__dsub_rn(hi, __dsub_rn(s, bb)), __dsub_rn(p, bb));
  hi = s;
  lo = __dadd_rn(lo, __dadd_rn(e, pe));
}

// (hi, lo) += (bh, bl), renormalised so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ void dd_add(double& hi, double& lo, double bh, double bl) {
  const double s = __dadd_rn(hi, bh);
  const double bb = __dsub_rn(s, hi);
  double e = __dadd_rn(__dsub_rn(hi, __dsub_rn(s, bb)), __dsub_rn(bh, bb));
  e = __dadd_rn(e, __dadd_rn(lo, bl));
  const double nh = __dadd_rn(s, e);
  lo = __dsub_rn(e, __dsub_rn(nh, s));
  hi = nh;
}

__device__ __forceinline__ double part_elem(const GramParts& P, int64_t i, int col) {
  int c = col;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (c < P.w[q]) return P.sgn[q] * P.p[q][i * P.w[q] + c];
    c -= P.w[q];
  }
  return 0.0;
}

// Partial Gram tiles: CTA (tile, chunk) accumulates, over rows
// [chunk * rows_per_chunk, ...), the kGT x kGT tile (ti, tj) of P^T P in
// double-double; out[((chunk * ntiles + tile) * kGT * kGT + e) * 2 + {0, 1}].
__global__ void __launch_bounds__(kGThreads) k_gram_dd(GramParts P, const int2* __restrict__ tiles,
                                                       int ntiles, int64_t rows_per_chunk,
                                                       double* __restrict__ out) {
  __shared__ double si[kGRows][kGT + 1];
  __shared__ double sj[kGRows][kGT + 1];
  const int tile = blockIdx.x;
  const int chunk = blockIdx.y;
  const int ti = tiles[tile].x, tj = tiles[tile].y;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)chunk * rows_per_chunk;
  const int64_t r1 = min(P.n, r0 + rows_per_chunk);
  double hi[4] = {0.0, 0.0, 0.0, 0.0}, lo[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t rb = r0; rb < r1; rb += kGRows) {
    for (int e = threadIdx.x; e < kGRows * kGT; e += kGThreads) {
      const int rr = e / kGT, cc = e - rr * kGT;
      const int64_t row = rb + rr;
      const int ci = ti * kGT + cc, cj = tj * kGT + cc;
      const bool ok = row < r1;
      si[rr][cc] = (ok && ci < P.wtot) ? part_elem(P, row, ci) : 0.0;
      sj[rr][cc] = (ok && cj < P.wtot) ? part_elem(P, row, cj) : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < kGRows; ++rr) {
      const double b = sj[rr][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) dd_acc(hi[q], lo[q], si[rr][ty + 8 * q], b);
    }
    __syncthreads();
  }
  double* o = out + ((int64_t)chunk * ntiles + tile) * kGT * kGT * 2;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = (ty + 8 * q) * kGT + tx;
    o[2 * e] = hi[q];
    o[2 * e + 1] = lo[q];
  }
}

// Sum the chunk partials of each tile in a fixed order (double-double) and
// write the symmetric w x w Gram matrix G (hi and lo parts, column-major).
__global__ void k_gram_reduce(const double* __restrict__ part, const int2* __restrict__ tiles,
                              int ntiles, int nchunks, int w, double* __restrict__ Ghi,
                              double* __restrict__ Glo) {
  const int tile = blockIdx.x;
  const int ti = tiles[tile].x, tj = tiles[tile].y;
  for (int e = threadIdx.x; e < kGT * kGT; e += blockDim.x) {
    double hi = 0.0, lo = 0.0;
    for (int c = 0; c < nchunks; ++c) {
      const double* p = part + (((int64_t)c * ntiles + tile) * kGT * kGT + e) * 2;
      dd_add(hi, lo, p[0], p[1]);
    }
    const int i = ti * kGT + e / kGT, j = tj * kGT + (e % kGT);
    if (i < w && j < w) {
      Ghi[(int64_t)j * w + i] = hi;
      Glo[(int64_t)j * w + i] = lo;
      Ghi[(int64_t)i * w + j] = hi;
      Glo[(int64_t)i * w + j] = lo;
    }
  }
}

// out[0], out[1] = hi, lo of sum_e (Ghi + Glo)_e (Hhi + Hlo)_e over count
// entries (one CTA; the lo * lo terms are below the double-double rounding).
__global__ void __launch_bounds__(1024) k_trace_dd(const double* __restrict__ Ghi,
                                                   const double* __restrict__ Glo,
                                                   const double* __restrict__ Hhi,
                                                   const double* __restrict__ Hlo, int64_t count,
                                                   double* __restrict__ out) {
  __shared__ double shi[1024], slo[1024];
  double hi = 0.0, lo = 0.0;
  for (int64_t e = threadIdx.x; e < count; e += blockDim.x) {
    const double a = Ghi[e], al = Glo[e], b = Hhi[e], bl = Hlo[e];
    dd_acc(hi, lo, a, b);
    lo = __dadd_rn(lo, __dadd_rn(__dmul_rn(a, bl), __dmul_rn(al, b)));
  }
  shi[threadIdx.x] = hi;
  slo[threadIdx.x] = lo;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      double a = shi[threadIdx.x], al = slo[threadIdx.x];
      dd_add(a, al, shi[threadIdx.x + h], slo[threadIdx.x + h]);
      shi[threadIdx.x] = a;
      slo[threadIdx.x] = al;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // renormalise once more before the split is read as two doubles
    double a = shi[0], al = slo[0];
    dd_add(a, al, 0.0, 0.0);
    out[0] = a;
    out[1] = al;
  }
}

// out3 = {||R||_F, ||C1 C2^T||_F, ratio} from the double-double squares
// num = (num[0] + num[1]) and den = (den[0] + den[1]).
__global__ void k_residual_finish(const double* __restrict__ num, const double* __restrict__ den,
                                  double* __restrict__ out3) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double n2 = num[0] + num[1];
  const double d2 = den[0] + den[1];
  const double nr = sqrt(n2 > 0.0 ? n2 : 0.0);
  const double dr = sqrt(d2 > 0.0 ? d2 : 0.0);
  out3[0] = nr;
  out3[1] = dr;
  out3[2] = dr > 0.0 ? nr / dr : (nr > 0.0 ? INFINITY : 0.0);
}

}  // namespace

int gram_dd_tiles(int w) {
  const int T = (w + kGT - 1) / kGT;
  return T * (T + 1) / 2;
}

int gram_dd_chunks(int64_t n, int w, int sm_count) {
  const int nt = gram_dd_tiles(w);
  int64_t want = std::max<int64_t>(1, ((int64_t)sm_count * 8 + nt - 1) / nt);
  const int64_t max_by_rows = std::max<int64_t>(1, (n + kGRows * 4 - 1) / (kGRows * 4));
  return (int)std::min<int64_t>(std::min<int64_t>(want, max_by_rows), 4096);
}

size_t gram_dd_work_doubles(int64_t n, int w, int sm_count) {
  return (size_t)gram_dd_chunks(n, w, sm_count) * gram_dd_tiles(w) * kGT * kGT * 2;
}

void gram_dd_tile_list(int w, int2* host_tiles) {
  const int T = (w + kGT - 1) / kGT;
  int q = 0;
  for (int i = 0; i < T; ++i)
    for (int j = i; j < T; ++j) host_tiles[q++] = make_int2(i, j);
}

void gram_dd_launch(const GramParts& P, const int2* tiles_dev, int sm_count, double* work,
                    double* Ghi, double* Glo, cudaStream_t st) {
  const int w = P.wtot;
  const int nt = gram_dd_tiles(w);
  const int nch = gram_dd_chunks(P.n, w, sm_count);
  int64_t rpc = (P.n + nch - 1) / nch;
  rpc = ((rpc + kGRows - 1) / kGRows) * kGRows;
  count_launches(2);
  k_gram_dd<<<dim3((unsigned)nt, (unsigned)nch), kGThreads, 0, st>>>(P, tiles_dev, nt, rpc, work);
  k_gram_reduce<<<nt, 256, 0, st>>>(work, tiles_dev, nt, nch, w, Ghi, Glo);
}

void trace_dd_launch(const double* Ghi, const double* Glo, const double* Hhi, const double* Hlo,
                     int64_t count, double* out2, cudaStream_t st) {
  count_launches(1);
  k_trace_dd<<<1, 1024, 0, st>>>(Ghi, Glo, Hhi, Hlo, count, out2);
}

void residual_finish_launch(const double* num2, const double* den2, double* out3,
                            cudaStream_t st) {
  count_launches(1);
  k_residual_finish<<<1, 32, 0, st>>>(num2, den2, out3);
}

}  // namespace spk
