// Truncated block Arnoldi kernels (Algorithm 1's basis loop; Eq. (2.4)).
//
// Per iteration d and operator (A, U) or (B^T, V):
//   spmm_dots   : U~ = A U_d (thread per CSR row; the r-wide row of U is one
//                 or two 16-byte loads) fused with the window inner products
//                 h_{i,d} = U_i^T U~ for up to four window blocks; per-CTA
//                 partial sums, reduced in a fixed order (deterministic).
//   update_gram : U~ -= sum_i U_i h_{i,d} (classical Gram-Schmidt on the
//                 locally orthonormal window -- equal to Algorithm 1's
//                 modified Gram-Schmidt in exact arithmetic) and G = U~^T U~.
//   chol_small  : Cholesky G = R^T R (R upper, positive diagonal), R^{-1}.
//   scale_gram / scale_store : Cholesky QR applied twice (CholQR2):
//                 U_{d+1} = (U~ R1^{-1}) R2^{-1}, h_{d+1,d} = R2 R1.
// The second (two-pass) sweep re-runs spmm (no dots), update and the two
// scalings with the stored coefficients, which reproduces U_j bit for bit.
#include "spk_internal.cuh"
#include "small_mat.cuh"

#include <algorithm>

namespace spk {

namespace {

constexpr int kFuse = 4;  // window blocks handled per dots pass

template <int R, typename TB, typename TC>
__device__ __forceinline__ void load_row(const TB* p, TC (&v)[R]) {
#pragma unroll
  for (int a = 0; a < R; ++a) v[a] = (TC)Store<TB>::ld(p + a);
}

template <typename TB, typename TC, typename TV, int R, bool DOTS>
__global__ void __launch_bounds__(256) k_spmm_dots(const int32_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col,
                                                   const TV* __restrict__ val, int64_t n,
                                                   const TB* __restrict__ U, TC* __restrict__ W,
                                                   WindowPtrs win, double* __restrict__ partial) {
  // per-thread partial sums in the compute type (FP32 in the mixed forms,
  // over a few rows only), cross-thread sums in FP64
  TC acc[DOTS ? kFuse * R * R : 1];
  if constexpr (DOTS) {
#pragma unroll
    for (int e = 0; e < kFuse * R * R; ++e) acc[e] = TC(0);
  }
  const int nwin = DOTS ? win.nwin : 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    TC w[R];
#pragma unroll
    for (int a = 0; a < R; ++a) w[a] = TC(0);
    const int e0 = rowptr[i], e1 = rowptr[i + 1];
    for (int e = e0; e < e1; ++e) {
      const TC v = (TC)val[e];
      TC u[R];
      load_row<R>(U + (int64_t)col[e] * R, u);
#pragma unroll
      for (int a = 0; a < R; ++a) w[a] = fma(v, u[a], w[a]);
    }
#pragma unroll
    for (int a = 0; a < R; ++a) W[i * R + a] = w[a];
    if constexpr (DOTS) {
#pragma unroll
      for (int q = 0; q < kFuse; ++q) {
        if (q < nwin) {
          TC u[R];
          load_row<R>(static_cast<const TB*>(win.blk[q]) + i * R, u);
#pragma unroll
          for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < R; ++b)
              acc[(q * R + a) * R + b] = fma(u[a], w[b], acc[(q * R + a) * R + b]);
        }
      }
    }
  }
  if constexpr (DOTS) {
    double accd[kFuse * R * R];
#pragma unroll
    for (int e = 0; e < kFuse * R * R; ++e) accd[e] = (double)acc[e];
    block_sum_store<kFuse * R * R>(accd, partial + (int64_t)blockIdx.x * kFuse * R * R);
  }
}

// Dots of an already computed U~ against up to four more window blocks.
template <typename TB, typename TC, int R>
__global__ void __launch_bounds__(256) k_dots(const TC* __restrict__ W, int64_t n, WindowPtrs win,
                                              double* __restrict__ partial) {
  TC acc[kFuse * R * R];
#pragma unroll
  for (int e = 0; e < kFuse * R * R; ++e) acc[e] = TC(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    TC w[R];
#pragma unroll
    for (int a = 0; a < R; ++a) w[a] = W[i * R + a];
#pragma unroll
    for (int q = 0; q < kFuse; ++q) {
      if (q < win.nwin) {
        TC u[R];
        load_row<R>(static_cast<const TB*>(win.blk[q]) + i * R, u);
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
          for (int b = 0; b < R; ++b)
            acc[(q * R + a) * R + b] = fma(u[a], w[b], acc[(q * R + a) * R + b]);
      }
    }
  }
  double accd[kFuse * R * R];
#pragma unroll
  for (int e = 0; e < kFuse * R * R; ++e) accd[e] = (double)acc[e];
  block_sum_store<kFuse * R * R>(accd, partial + (int64_t)blockIdx.x * kFuse * R * R);
}

// out[e] = sum_p partial[p*stride + e] for e < count: warp w of the block
// takes e = w, w + 8, ...; its lanes load the partials p = lane, lane + 32,
// ... (independent loads in flight) and finish with a shuffle sum, so the
// order of the additions is fixed.
__device__ __forceinline__ void sum_partials(const double* __restrict__ partial, int nparts,
                                             int stride, int count, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = wid; e < count; e += nw) {
    double s = 0.0;
    for (int p = lane; p < nparts; p += 32) s += partial[(int64_t)p * stride + e];
    s = warp_sum(s);
    if (lane == 0) out[e] = s;
  }
}

__global__ void __launch_bounds__(256) k_reduce_partials(const double* __restrict__ partial,
                                                         int nparts, int stride, int count,
                                                         double* __restrict__ out) {
  sum_partials(partial, nparts, stride, count, out);
}

template <typename TB, typename TC, int R>
__global__ void __launch_bounds__(256) k_update_gram(TC* __restrict__ W, int64_t n, WindowPtrs win,
                                                     const double* __restrict__ h,
                                                     double* __restrict__ partial, int want_gram) {
  __shared__ TC hs[kMaxWin * R * R];
  for (int e = threadIdx.x; e < win.nwin * R * R; e += blockDim.x) hs[e] = (TC)h[e];
  __syncthreads();
  TC acc[R * R];
#pragma unroll
  for (int e = 0; e < R * R; ++e) acc[e] = TC(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    TC w[R];
#pragma unroll
    for (int a = 0; a < R; ++a) w[a] = W[i * R + a];
    for (int q = 0; q < win.nwin; ++q) {
      TC u[R];
      load_row<R>(static_cast<const TB*>(win.blk[q]) + i * R, u);
      const TC* hq = hs + q * R * R;
#pragma unroll
      for (int b = 0; b < R; ++b) {
        TC s = w[b];
#pragma unroll
        for (int a = 0; a < R; ++a) s = fma(-u[a], hq[a * R + b], s);
        w[b] = s;
      }
    }
#pragma unroll
    for (int a = 0; a < R; ++a) W[i * R + a] = w[a];
    if (want_gram) {
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) acc[a * R + b] = fma(w[a], w[b], acc[a * R + b]);
    }
  }
  if (want_gram) {
    double accd[R * R];
#pragma unroll
    for (int e = 0; e < R * R; ++e) accd[e] = (double)acc[e];
    block_sum_store<R * R>(accd, partial + (int64_t)blockIdx.x * R * R);
  }
}

// G = sum of partial Grams; R upper with R^T R = G; Rinv = R^{-1}.
// Gram matrix from the partial sums, then its Cholesky factor (upper,
// positive diagonal) and the factor's inverse, in registers.
template <int R>
__global__ void k_chol_small(const double* __restrict__ partial, int nparts,
                             double* __restrict__ Rout, double* __restrict__ Rinv,
                             uint32_t* flags, double rel_floor) {
  __shared__ double G[R * R];
  sum_partials(partial, nparts, R * R, R * R, G);
  __syncthreads();
  if (threadIdx.x != 0) return;
  double U[R][R];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) U[a][b] = 0.0;
  double tr = 0.0;
#pragma unroll
  for (int a = 0; a < R; ++a) tr += G[a * R + a];
  const bool bad = !isfinite(tr);
  if (!bad) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      double s = G[j * R + j];
#pragma unroll
      for (int l = 0; l < j; ++l) s -= U[l][j] * U[l][j];
      if (!(s > rel_floor * tr) || !(tr > 0.0)) {
        atomicOr(flags, kFlagBreakdown);
        s = (tr > 0.0 && isfinite(tr)) ? fmax(s, rel_floor * tr) : 1.0;
        if (!(s > 0.0)) s = 1.0;
      }
      U[j][j] = sqrt(s);
      const double dj = 1.0 / U[j][j];
#pragma unroll
      for (int i = j + 1; i < R; ++i) {
        double t = G[j * R + i];
#pragma unroll
        for (int l = 0; l < j; ++l) t -= U[l][j] * U[l][i];
        U[j][i] = t * dj;
      }
    }
  } else {
    atomicOr(flags, kFlagNonfinite);
#pragma unroll
    for (int a = 0; a < R; ++a) U[a][a] = 1.0;
  }
  double Ui[R][R];
  sm::upper_inv<R>(U, Ui);
  if (Rout) sm::store_rm<R>(U, Rout);
  if (Rinv) sm::store_rm<R>(Ui, Rinv);
}

template <typename TC, int R>
__global__ void __launch_bounds__(256) k_scale_gram(TC* __restrict__ W, int64_t n,
                                                    const double* __restrict__ Rinv,
                                                    double* __restrict__ partial) {
  __shared__ TC ri[R * R];
  if (threadIdx.x < R * R) ri[threadIdx.x] = (TC)Rinv[threadIdx.x];
  __syncthreads();
  TC acc[R * R];
#pragma unroll
  for (int e = 0; e < R * R; ++e) acc[e] = TC(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    TC w[R], o[R];
#pragma unroll
    for (int a = 0; a < R; ++a) w[a] = W[i * R + a];
#pragma unroll
    for (int b = 0; b < R; ++b) {
      TC s = TC(0);
#pragma unroll
      for (int a = 0; a <= b; ++a) s = fma(w[a], ri[a * R + b], s);
      o[b] = s;
    }
#pragma unroll
    for (int a = 0; a < R; ++a) W[i * R + a] = o[a];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) acc[a * R + b] = fma(o[a], o[b], acc[a * R + b]);
  }
  double accd[R * R];
#pragma unroll
  for (int e = 0; e < R * R; ++e) accd[e] = (double)acc[e];
  block_sum_store<R * R>(accd, partial + (int64_t)blockIdx.x * R * R);
}

template <typename TB, typename TC, int R>
__global__ void __launch_bounds__(256) k_scale_store(const TC* __restrict__ W, int64_t n,
                                                     const double* __restrict__ Rinv,
                                                     TB* __restrict__ dst) {
  __shared__ TC ri[R * R];
  if (threadIdx.x < R * R) ri[threadIdx.x] = (TC)Rinv[threadIdx.x];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    TC w[R];
#pragma unroll
    for (int a = 0; a < R; ++a) w[a] = W[i * R + a];
#pragma unroll
    for (int b = 0; b < R; ++b) {
      TC s = TC(0);
#pragma unroll
      for (int a = 0; a <= b; ++a) s = fma(w[a], ri[a * R + b], s);
      Store<TB>::st(dst + i * R + b, s);
    }
  }
}

// X (n x ell, row-major FP64) += sum_q U_q Wrows[q r .. q r + r-1, :]
// (Wrows column-major with leading dimension ldw).  CTA tile: 64 columns of
// X by kXRows rows; the W chunk and the U rows are staged in shared memory,
// X is read and written once, coalesced along its columns.
constexpr int kXCols = 64, kXRows = 32;
template <typename TB>
__global__ void __launch_bounds__(256) k_x_accumulate(double* __restrict__ X, int64_t n, int ell, int r,
                                                      WindowPtrs blocks,
                                                      const double* __restrict__ Wrows, int64_t ldw) {
  __shared__ double Ws[kXMaxBlocks * kMaxR][kXCols];
  __shared__ double Us[kXRows][kXMaxBlocks * kMaxR + 1];
  const int kr = blocks.nwin * r;
  const int c0 = blockIdx.y * kXCols;
  const int64_t i0 = (int64_t)blockIdx.x * kXRows;
  const int tx = threadIdx.x & (kXCols - 1), ty = threadIdx.x / kXCols;  // 64 x 4
  for (int e = threadIdx.x; e < kr * kXCols; e += blockDim.x) {
    const int qa = e / kXCols, c = e - qa * kXCols;
    Ws[qa][c] = (c0 + c < ell) ? Wrows[qa + (int64_t)(c0 + c) * ldw] : 0.0;
  }
  for (int e = threadIdx.x; e < kXRows * kr; e += blockDim.x) {
    const int ri = e / kr, qa = e - ri * kr;
    const int q = qa / r, a = qa - q * r;
    const int64_t i = i0 + ri;
    Us[ri][qa] = (i < n) ? (double)Store<TB>::ld(static_cast<const TB*>(blocks.blk[q]) + i * r + a) : 0.0;
  }
  __syncthreads();
  const int c = c0 + tx;
  if (c >= ell) return;
  for (int ri = ty; ri < kXRows; ri += 4) {
    const int64_t i = i0 + ri;
    if (i >= n) break;
    double s = X[i * ell + c];
    for (int qa = 0; qa < kr; ++qa) s = fma(Us[ri][qa], Ws[qa][tx], s);
    X[i * ell + c] = s;
  }
}

__global__ void k_spmm_wide(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, int64_t n, int w,
                            const double* __restrict__ X, double* __restrict__ Y) {
  const int64_t total = n * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / w;
    const int c = (int)(e - i * w);
    double s = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s = fma(val[k], X[(int64_t)col[k] * w + c], s);
    Y[e] = s;
  }
}

template <typename TD>
__global__ void k_convert(const double* __restrict__ src, TD* __restrict__ dst, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    Store<TD>::st(dst + e, (decltype(Store<TD>::ld(dst)))src[e]);
}

// mode 0: C = A B;  mode 1: C = A B^T  (r x r row-major); one thread per entry
template <int R>
__global__ void k_combine_small(const double* A, const double* B, double* C, int mode) {
  const int e = threadIdx.x;
  double s = 0.0;
  if (e < R * R) {
    const int a = e / R, b = e - a * R;
#pragma unroll
    for (int l = 0; l < R; ++l) s += A[a * R + l] * (mode == 0 ? B[l * R + b] : B[b * R + l]);
  }
  __syncthreads();    // C may alias A or B
  if (e < R * R) C[e] = s;
}

int default_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 4));
}

// Row-major n x r block <-> columns of a column-major matrix (ld ldv).
__global__ void k_block_to_cols(const double* __restrict__ B, int64_t n, int r,
                                double* __restrict__ V, int64_t ldv) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r;
    const int c = (int)(e - i * r);
    V[i + c * ldv] = B[e];
  }
}

__global__ void k_cols_to_block(const double* __restrict__ V, int64_t ldv, int64_t n, int r,
                                double* __restrict__ B) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / r;
    const int c = (int)(e - i * r);
    B[e] = V[i + c * ldv];
  }
}

}  // namespace

// P[i + (c0 + a) * ldp] = U[i * r + a]: block columns into an FP64 panel
template <typename TB>
__global__ void k_block_to_panel(const TB* __restrict__ U, int64_t n, int r,
                                 double* __restrict__ P, int64_t ldp) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / n, i = e - a * n;
    P[i + a * ldp] = (double)Store<TB>::ld(U + i * r + a);
  }
}

template <typename TB>
void block_to_panel_launch(const TB* U, int64_t n, int r, double* P, int64_t ldp, cudaStream_t st) {
  count_launches(1);
  k_block_to_panel<TB><<<default_grid(n * r), 256, 0, st>>>(U, n, r, P, ldp);
}

// X (n x ell row-major) = Xcm (n x ell column-major), through 32 x 32 tiles
__global__ void k_cols_to_rows(const double* __restrict__ Xcm, int64_t n, int ell,
                               double* __restrict__ X) {
  __shared__ double tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int cc = ty; cc < 32; cc += 8) {
    const int c = c0 + cc;
    const int64_t i = i0 + tx;
    tile[cc][tx] = (c < ell && i < n) ? Xcm[(int64_t)c * n + i] : 0.0;
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int64_t i = i0 + ii;
    const int c = c0 + tx;
    if (i < n && c < ell) X[i * ell + c] = tile[tx][ii];
  }
}

void cols_to_rows_launch(const double* Xcm, int64_t n, int ell, double* X, cudaStream_t st) {
  count_launches(1);
  k_cols_to_rows<<<dim3((unsigned)((n + 31) / 32), (unsigned)((ell + 31) / 32)), 256, 0, st>>>(
      Xcm, n, ell, X);
}

void block_to_cols_launch(const double* B, int64_t n, int r, double* V, int64_t ldv,
                          cudaStream_t st) {
  count_launches(1);
  k_block_to_cols<<<default_grid(n * r), 256, 0, st>>>(B, n, r, V, ldv);
}

void cols_to_block_launch(const double* V, int64_t ldv, int64_t n, int r, double* B,
                          cudaStream_t st) {
  count_launches(1);
  k_cols_to_block<<<default_grid(n * r), 256, 0, st>>>(V, ldv, n, r, B);
}

template <typename TB, typename TC, typename TV>
void spmm_dots_launch(const int32_t* rowptr, const int32_t* col, const TV* val, int64_t n, int r,
                      const TB* U, TC* W, WindowPtrs win, double* partial, int grid,
                      cudaStream_t st) {
  // first group fused with the product, further groups as separate passes
  WindowPtrs g0 = win;
  g0.nwin = std::min(win.nwin, kFuse);
  const bool dots = win.nwin > 0;
#define SPK_SPMM(RR)                                                                           \
  count_launches(1);                                                                           \
  if (dots)                                                                                    \
    k_spmm_dots<TB, TC, TV, RR, true><<<grid, 256, 0, st>>>(rowptr, col, val, n, U, W, g0, partial); \
  else                                                                                         \
    k_spmm_dots<TB, TC, TV, RR, false><<<grid, 256, 0, st>>>(rowptr, col, val, n, U, W, g0, partial);
  switch (r) {
    case 1: SPK_SPMM(1) break;
    case 2: SPK_SPMM(2) break;
    case 3: SPK_SPMM(3) break;
    default: SPK_SPMM(4) break;
  }
#undef SPK_SPMM
  for (int g = kFuse; g < win.nwin; g += kFuse) {
    WindowPtrs gw;
    gw.nwin = std::min(kFuse, win.nwin - g);
    for (int q = 0; q < gw.nwin; ++q) gw.blk[q] = win.blk[g + q];
    double* part = partial + (int64_t)(g / kFuse) * grid * kFuse * r * r;
    switch (r) {
      case 1: count_launches(1); k_dots<TB, TC, 1><<<grid, 256, 0, st>>>(W, n, gw, part); break;
      case 2: count_launches(1); k_dots<TB, TC, 2><<<grid, 256, 0, st>>>(W, n, gw, part); break;
      case 3: count_launches(1); k_dots<TB, TC, 3><<<grid, 256, 0, st>>>(W, n, gw, part); break;
      default: count_launches(1); k_dots<TB, TC, 4><<<grid, 256, 0, st>>>(W, n, gw, part); break;
    }
  }
}

void reduce_partials_launch(const double* partial, int nparts, int stride, int count,
                            double* out, cudaStream_t st) {
  count_launches(1);
  k_reduce_partials<<<1, 256, 0, st>>>(partial, nparts, stride, count, out);
}

template <typename TB, typename TC>
void update_gram_launch(TC* W, int64_t n, int r, WindowPtrs win, const double* h, double* partial,
                        int grid, int want_gram, cudaStream_t st) {
  switch (r) {
    case 1: count_launches(1); k_update_gram<TB, TC, 1><<<grid, 256, 0, st>>>(W, n, win, h, partial, want_gram); break;
    case 2: count_launches(1); k_update_gram<TB, TC, 2><<<grid, 256, 0, st>>>(W, n, win, h, partial, want_gram); break;
    case 3: count_launches(1); k_update_gram<TB, TC, 3><<<grid, 256, 0, st>>>(W, n, win, h, partial, want_gram); break;
    default: count_launches(1); k_update_gram<TB, TC, 4><<<grid, 256, 0, st>>>(W, n, win, h, partial, want_gram); break;
  }
}

void chol_small_launch(const double* partial, int nparts, int r, double* R, double* Rinv,
                       uint32_t* flags, double rel_floor, cudaStream_t st) {
  count_launches(1);
  switch (r) {
    case 1: k_chol_small<1><<<1, 256, 0, st>>>(partial, nparts, R, Rinv, flags, rel_floor); break;
    case 2: k_chol_small<2><<<1, 256, 0, st>>>(partial, nparts, R, Rinv, flags, rel_floor); break;
    case 3: k_chol_small<3><<<1, 256, 0, st>>>(partial, nparts, R, Rinv, flags, rel_floor); break;
    default: k_chol_small<4><<<1, 256, 0, st>>>(partial, nparts, R, Rinv, flags, rel_floor); break;
  }
}

template <typename TC>
void scale_gram_launch(TC* W, int64_t n, int r, const double* Rinv, double* partial, int grid,
                       cudaStream_t st) {
  switch (r) {
    case 1: count_launches(1); k_scale_gram<TC, 1><<<grid, 256, 0, st>>>(W, n, Rinv, partial); break;
    case 2: count_launches(1); k_scale_gram<TC, 2><<<grid, 256, 0, st>>>(W, n, Rinv, partial); break;
    case 3: count_launches(1); k_scale_gram<TC, 3><<<grid, 256, 0, st>>>(W, n, Rinv, partial); break;
    default: count_launches(1); k_scale_gram<TC, 4><<<grid, 256, 0, st>>>(W, n, Rinv, partial); break;
  }
}

template <typename TB, typename TC>
void scale_store_launch(const TC* W, int64_t n, int r, const double* Rinv, TB* dst,
                        cudaStream_t st) {
  const int grid = default_grid(n);
  switch (r) {
    case 1: count_launches(1); k_scale_store<TB, TC, 1><<<grid, 256, 0, st>>>(W, n, Rinv, dst); break;
    case 2: count_launches(1); k_scale_store<TB, TC, 2><<<grid, 256, 0, st>>>(W, n, Rinv, dst); break;
    case 3: count_launches(1); k_scale_store<TB, TC, 3><<<grid, 256, 0, st>>>(W, n, Rinv, dst); break;
    default: count_launches(1); k_scale_store<TB, TC, 4><<<grid, 256, 0, st>>>(W, n, Rinv, dst); break;
  }
}

template <typename TB>
void x_accumulate_launch(double* X, int64_t n, int ell, int r, WindowPtrs blocks,
                         const double* Wrows, int64_t ldw, cudaStream_t st) {
  if (ell <= 0 || blocks.nwin <= 0) return;
  dim3 grid((unsigned)((n + kXRows - 1) / kXRows), (unsigned)((ell + kXCols - 1) / kXCols));
  count_launches(1);
  k_x_accumulate<TB><<<grid, 256, 0, st>>>(X, n, ell, r, blocks, Wrows, ldw);
}

void spmm_wide_launch(const int32_t* rowptr, const int32_t* col, const double* val, int64_t n,
                      int w, const double* X, double* Y, cudaStream_t st) {
  if (w <= 0 || n <= 0) return;
  count_launches(1);
  k_spmm_wide<<<default_grid(n * w), 256, 0, st>>>(rowptr, col, val, n, w, X, Y);
}

template <typename TV>
void convert_values_launch(const double* src, TV* dst, int64_t count, cudaStream_t st) {
  count_launches(1);
  k_convert<TV><<<default_grid(count), 256, 0, st>>>(src, dst, count);
}
template <typename TB>
void convert_block_launch(const double* src, TB* dst, int64_t count, cudaStream_t st) {
  count_launches(1);
  k_convert<TB><<<default_grid(count), 256, 0, st>>>(src, dst, count);
}

void combine_small_launch(const double* A, const double* B, double* C, int r, int mode,
                          cudaStream_t st) {
  count_launches(1);
  switch (r) {
    case 1: k_combine_small<1><<<1, 32, 0, st>>>(A, B, C, mode); break;
    case 2: k_combine_small<2><<<1, 32, 0, st>>>(A, B, C, mode); break;
    case 3: k_combine_small<3><<<1, 32, 0, st>>>(A, B, C, mode); break;
    default: k_combine_small<4><<<1, 32, 0, st>>>(A, B, C, mode); break;
  }
}

// ---- explicit instantiations: FP64, mixed FP32, mixed BF16-basis
#define SPK_INST(TB, TC, TV)                                                                     \
  template void spmm_dots_launch<TB, TC, TV>(const int32_t*, const int32_t*, const TV*, int64_t, \
                                             int, const TB*, TC*, WindowPtrs, double*, int,     \
                                             cudaStream_t);                                     \
  template void update_gram_launch<TB, TC>(TC*, int64_t, int, WindowPtrs, const double*,         \
                                           double*, int, int, cudaStream_t);                    \
  template void scale_store_launch<TB, TC>(const TC*, int64_t, int, const double*, TB*,          \
                                           cudaStream_t);                                       \
  template void x_accumulate_launch<TB>(double*, int64_t, int, int, WindowPtrs, const double*,  \
                                        int64_t, cudaStream_t);                                 \
  template void convert_block_launch<TB>(const double*, TB*, int64_t, cudaStream_t);         \
  template void block_to_panel_launch<TB>(const TB*, int64_t, int, double*, int64_t, cudaStream_t);
SPK_INST(double, double, double)
SPK_INST(float, float, float)
SPK_INST(__nv_bfloat16, float, float)
#undef SPK_INST
template void scale_gram_launch<double>(double*, int64_t, int, const double*, double*, int,
                                        cudaStream_t);
template void scale_gram_launch<float>(float*, int64_t, int, const double*, double*, int,
                                       cudaStream_t);
template void convert_values_launch<float>(const double*, float*, int64_t, cudaStream_t);

}  // namespace spk
