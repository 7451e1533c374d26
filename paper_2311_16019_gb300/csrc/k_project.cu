// Projected matrices and the residual estimate (Eqs. (2.9)-(2.10), Section 5, Eq. (3.5)).
//
// H~_d = Hhat_d + Hhat E_d^T with Hhat_d = T_d H_d T_d^{-1} and
// Hhat = T_H h_{d+1,d} tau_d^{-1} is kept up to date by the bordering update of
// Section 5: from H~_{d-1} and the new columns of T and H,
//   (1,2) block = (-H~_{d-1} T_H + T_{d-1} H_col + T_H h_{d,d}) tau_d^{-1}
//   (2,1) block = tau_d h_{d,d-1} tau_{d-1}^{-1}            (last block column)
//   (2,2) block = tau_d (h_{d,d} - h_{d,d-1} tau_{d-1}^{-1} E^T T_H) tau_d^{-1}
// (T_H = T[0:(d-1)r, (d-1)r:dr], tau_d its diagonal block; the last term of
// the (1,2) block carries tau_d^{-1} -- direct expansion of T H T^{-1}), then
// the correction H~_d = Hhat_d + T_H' h_{d+1,d} tau_d^{-1} E_d^T is added with
// the newest column T_H' of T_{d+1}.
// rho (Eq. (3.5)) uses the whitened subdiagonals
//   hhat = tau_{d+1} h_{d+1,d} tau_d^{-1},  ghat = theta_{d+1} g_{d+1,d} theta_d^{-1}.
#include "spk_internal.cuh"
#include "small_mat.cuh"

#include <algorithm>

namespace spk {

namespace {

__host__ __device__ void upper_inv(const double* T, int64_t ldT, int off, int r, double* Ri) {
  // Ri (r x r row-major) = inverse of the upper-triangular block T[off.., off..]
  for (int e = 0; e < r * r; ++e) Ri[e] = 0.0;
  for (int j = 0; j < r; ++j) {
    Ri[j * r + j] = 1.0 / T[off + j + (int64_t)(off + j) * ldT];
    for (int i = j - 1; i >= 0; --i) {
      double t = 0.0;
      for (int l = i + 1; l <= j; ++l) t += T[off + i + (int64_t)(off + l) * ldT] * Ri[l * r + j];
      Ri[i * r + j] = -t / T[off + i + (int64_t)(off + i) * ldT];
    }
  }
}

__host__ __device__ void tblock(const double* T, int64_t ldT, int off, int r, double* B) {
  for (int a = 0; a < r; ++a)
    for (int c = 0; c < r; ++c) B[a * r + c] = T[off + a + (int64_t)(off + c) * ldT];
}

__host__ __device__ void mm(const double* A, const double* B, double* C, int r) {
  double o[kMaxR * kMaxR];
  for (int a = 0; a < r; ++a)
    for (int c = 0; c < r; ++c) {
      double s = 0.0;
      for (int l = 0; l < r; ++l) s += A[a * r + l] * B[l * r + c];
      o[a * r + c] = s;
    }
  for (int e = 0; e < r * r; ++e) C[e] = o[e];
}

constexpr int kBRows = 32;     // rows per CTA of the bordering GEMV (one per lane)
constexpr int kBWarps = 8;     // warps per CTA, each on kBWarpCols columns
constexpr int kBWarpCols = 32;
constexpr int kBCols = kBWarps * kBWarpCols;   // columns of H~ per CTA

// partial[(chunk*mp + i)*r + c] = sum_{l in chunk} H~[i, l] T_H[l, c]: lane =
// row (coalesced column reads of H~), warp = 32-column slice of the chunk,
// slices summed in shared memory in a fixed order.
__global__ void __launch_bounds__(kBWarps * 32) k_border_gemv(const double* __restrict__ Ht,
                                                             int64_t ldH, int mp, int r,
                                                             const double* __restrict__ T,
                                                             int64_t ldT,
                                                             double* __restrict__ partial) {
  __shared__ double th[kBCols * kMaxR];
  __shared__ double red[kBWarps][kBRows * kMaxR];
  const int l0 = blockIdx.y * kBCols;
  const int l1 = min(mp, l0 + kBCols);
  for (int e = threadIdx.x; e < (l1 - l0) * r; e += blockDim.x) {
    const int l = e / r, c = e - l * r;
    th[e] = T[l0 + l + (int64_t)(mp + c) * ldT];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i = blockIdx.x * kBRows + lane;
  double v[kMaxR] = {0, 0, 0, 0};
  const int la = l0 + wid * kBWarpCols;
  const int lb = min(l1, la + kBWarpCols);
  if (i < mp) {
    const double* hrow = Ht + i;
#pragma unroll 8
    for (int l = la; l < lb; ++l) {
      const double hv = hrow[(int64_t)l * ldH];
      const double* t = th + (l - l0) * r;
#pragma unroll
      for (int c = 0; c < kMaxR; ++c)
        if (c < r) v[c] = fma(hv, t[c], v[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < kMaxR; ++c) red[wid][lane * kMaxR + c] = v[c];
  __syncthreads();
  if (wid == 0 && i < mp) {
    for (int c = 0; c < r; ++c) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kBWarps; ++w) s += red[w][lane * kMaxR + c];
      partial[((int64_t)blockIdx.y * mp + i) * r + c] = s;
    }
  }
}

// Rows i < mp of the new block column of H~:
// (-sum of GEMV partials + T_{d-1} H_col + T_H h_{d,d}) tau_d^{-1}.
template <int R>
__global__ void k_border_col(double* __restrict__ Ht, int64_t ldH, int mp,
                             const double* __restrict__ T, int64_t ldT,
                             const double* __restrict__ hslots, int first_block, int nslots,
                             const double* __restrict__ h_dd, const double* __restrict__ partial,
                             int nchunk) {
  __shared__ double tinv[R * R];
  __shared__ double hdd[R * R];
  if (threadIdx.x == 0) {
    double U[R][R], Ui[R][R];
    sm::load_tblock<R>(T, ldT, mp, U);
    sm::upper_inv<R>(U, Ui);
    sm::store_rm<R>(Ui, tinv);
  }
  if (threadIdx.x < R * R) hdd[threadIdx.x] = h_dd[threadIdx.x];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= mp) return;
  double v[R];
#pragma unroll
  for (int c = 0; c < R; ++c) v[c] = 0.0;
#pragma unroll 4
  for (int ch = 0; ch < nchunk; ++ch) {
    const double* pp = partial + ((int64_t)ch * mp + i) * R;
#pragma unroll
    for (int c = 0; c < R; ++c) v[c] -= pp[c];
  }
  for (int q = 0; q < nslots; ++q) {
    const int b = first_block + q;  // 1-based block index
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const int l = (b - 1) * R + a;
      const double t = T[i + (int64_t)l * ldT];
#pragma unroll
      for (int c = 0; c < R; ++c) v[c] += t * hslots[(q * R + a) * R + c];
    }
  }
#pragma unroll
  for (int a = 0; a < R; ++a) {
    const double t = T[i + (int64_t)(mp + a) * ldT];
#pragma unroll
    for (int c = 0; c < R; ++c) v[c] += t * hdd[a * R + c];
  }
#pragma unroll
  for (int c = 0; c < R; ++c) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a <= c; ++a) s += v[a] * tinv[a * R + c];
    Ht[i + (int64_t)(mp + c) * ldH] = s;
  }
}

}  // namespace

namespace {

// Rows mp..mp+r of H~ (the (2,1) and (2,2) blocks of the bordering update).
template <int R>
__global__ void k_border_small(double* __restrict__ Ht, int64_t ldH, int mp,
                               const double* __restrict__ T, int64_t ldT,
                               const double* __restrict__ h_sub, const double* __restrict__ h_dd) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double tau[R][R], tinv[R][R], X[R][R], Y[R][R], H[R][R];
  sm::load_tblock<R>(T, ldT, mp, tau);
  sm::upper_inv<R>(tau, tinv);
  sm::load_rm<R>(h_dd, H);
  if (mp == 0) {
    sm::mul<R>(tau, H, X);
    sm::mul<R>(X, tinv, Y);
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int c = 0; c < R; ++c) Ht[a + (int64_t)c * ldH] = Y[a][c];
    return;
  }
  double tp[R][R], tpinv[R][R], hs[R][R], hs_tp[R][R], ET[R][R];
  sm::load_tblock<R>(T, ldT, mp - R, tp);
  sm::upper_inv<R>(tp, tpinv);
  // (2,1): tau_d h_{d,d-1} tau_{d-1}^{-1}
  sm::load_rm<R>(h_sub, hs);
  sm::mul<R>(hs, tpinv, hs_tp);
  sm::mul<R>(tau, hs_tp, X);
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) Ht[mp + a + (int64_t)(mp - R + c) * ldH] = X[a][c];
  // (2,2): tau_d (h_{d,d} - h_{d,d-1} tau_{d-1}^{-1} E^T T_H) tau_d^{-1}
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) ET[a][c] = T[mp - R + a + (int64_t)(mp + c) * ldT];
  sm::mul<R>(hs_tp, ET, X);
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) X[a][c] = H[a][c] - X[a][c];
  sm::mul<R>(tau, X, Y);
  sm::mul<R>(Y, tinv, X);
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) Ht[mp + a + (int64_t)(mp + c) * ldH] = X[a][c];
}

// H~[:, m-r:m] += T[:, m:m+r] h_{d+1,d} tau_d^{-1}  (rows < m)
template <int R>
__global__ void k_border_correct(double* __restrict__ Ht, int64_t ldH, int m,
                                 const double* __restrict__ T, int64_t ldT,
                                 const double* __restrict__ h_next) {
  __shared__ double K[R * R];
  if (threadIdx.x == 0) {
    double U[R][R], Ui[R][R], Hn[R][R], Kk[R][R];
    sm::load_tblock<R>(T, ldT, m - R, U);
    sm::upper_inv<R>(U, Ui);
    sm::load_rm<R>(h_next, Hn);
    sm::mul<R>(Hn, Ui, Kk);
    sm::store_rm<R>(Kk, K);
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double v[R];
#pragma unroll
  for (int a = 0; a < R; ++a) v[a] = T[i + (int64_t)(m + a) * ldT];
#pragma unroll
  for (int c = 0; c < R; ++c) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < R; ++a) s += v[a] * K[a * R + c];
    Ht[i + (int64_t)(m - R + c) * ldH] += s;
  }
}

// out3 = {rho, rho/||beta_U beta_V^T||_F, ||beta_U beta_V^T||_F}
// Residual estimate at a check (Y m x m column-major, ld ldY).
// Sketched method (TU, TV given), Eq. (3.5) with the whitened subdiagonal
// blocks hhat = tau_{d+1} h_{d+1,d} tau_d^{-1} (and ghat likewise):
//   rho = sqrt(||hhat E_d^T Y||_F^2 + ||Y E_d ghat^T||_F^2).
// Truncated method (TU == nullptr, bound != 0), the bound of Proposition 3.1
// (Eq. (3.2)):  rho = sqrt(m) (||h E_d^T Y||_F + ||Y E_d g^T||_F),  h = h_{d+1,d}.
// Full Arnoldi (TU == nullptr, bound == 0), the exact residual norm of the
// Galerkin solution:  rho = sqrt(||h E_d^T Y||_F^2 + ||Y E_d g^T||_F^2).
// out3 = {rho, rho / ||beta1 beta2^T||_F, ||beta1 beta2^T||_F}.
__global__ void k_rho(const double* __restrict__ Y, int64_t ldY, int m, int r,
                      const double* __restrict__ TU, int64_t ldTU, const double* __restrict__ TV,
                      int64_t ldTV, const double* __restrict__ hU, const double* __restrict__ hV,
                      const double* __restrict__ bU, const double* __restrict__ bV,
                      int bound, double* __restrict__ out3) {
  __shared__ double hh[kMaxR * kMaxR], gh[kMaxR * kMaxR];
  __shared__ double red[2][32];
  __shared__ double nb;
  const bool sketched = TU != nullptr;
  if (threadIdx.x == 0) {
    if (sketched) {
      double tau[kMaxR * kMaxR], tinv[kMaxR * kMaxR], X[kMaxR * kMaxR];
      tblock(TU, ldTU, m, r, tau);
      upper_inv(TU, ldTU, m - r, r, tinv);
      mm(tau, hU, X, r);
      mm(X, tinv, hh, r);
      tblock(TV, ldTV, m, r, tau);
      upper_inv(TV, ldTV, m - r, r, tinv);
      mm(tau, hV, X, r);
      mm(X, tinv, gh, r);
    } else {
      for (int e = 0; e < r * r; ++e) {
        hh[e] = hU[e];
        gh[e] = hV[e];
      }
    }
    double s = 0.0;
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) {
        double f = 0.0;
        for (int l = 0; l < r; ++l) f += bU[a * r + l] * bV[b * r + l];
        s += f * f;
      }
    nb = sqrt(s);
  }
  __syncthreads();
  double accH = 0.0, accG = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    // row block: (hhat Y[m-r:m, j])_a
    for (int a = 0; a < r; ++a) {
      double s = 0.0;
      for (int b = 0; b < r; ++b) s += hh[a * r + b] * Y[m - r + b + (int64_t)j * ldY];
      accH += s * s;
    }
    // column block: (Y[j, m-r:m] ghat^T)_a
    for (int a = 0; a < r; ++a) {
      double s = 0.0;
      for (int b = 0; b < r; ++b) s += Y[j + (int64_t)(m - r + b) * ldY] * gh[a * r + b];
      accG += s * s;
    }
  }
  accH = warp_sum(accH);
  accG = warp_sum(accG);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = accH;
    red[1][threadIdx.x >> 5] = accG;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sH = 0.0, sG = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sH += red[0][w];
      sG += red[1][w];
    }
    const double rho = (sketched || !bound) ? sqrt(sH + sG)
                                            : sqrt((double)m) * (sqrt(sH) + sqrt(sG));
    out3[0] = rho;
    out3[1] = rho / nb;
    out3[2] = nb;
  }
}

// Dense H_d (m x m column-major, zeroed beforehand) from the stored Arnoldi
// coefficients: block column j (1..d) holds h_{i,j} for the window rows
// i = j-k+1 .. j and h_{j+1,j} (slot q <-> i = j-k+1+q), rows i in [1, d].
__global__ void k_band_to_dense(const double* __restrict__ hband, int k, int r, int d,
                                double* __restrict__ H, int64_t ldH) {
  const int64_t per_col = (int64_t)(k + 1) * r * r;
  const int64_t total = (int64_t)d * per_col;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / per_col) + 1;
    const int64_t rem = e - (int64_t)(j - 1) * per_col;
    const int q = (int)(rem / (r * r));
    const int ac = (int)(rem - (int64_t)q * r * r);
    const int a = ac / r, c = ac - a * r;
    const int i = j - k + 1 + q;
    if (i < 1 || i > d) continue;
    H[(int64_t)(i - 1) * r + a + ((int64_t)(j - 1) * r + c) * ldH] =
        hband[(int64_t)j * per_col + (int64_t)q * r * r + a * r + c];
  }
}

// L[a + l*ldL] = beta[a*r + l]: the r x r row-major beta into the top of a
// column-major factor.
__global__ void k_fill_factor(double* L, int64_t ldL, int r, const double* beta) {
  const int e = threadIdx.x;
  if (e >= r * r) return;
  const int a = e / r, l = e - a * r;
  L[a + (int64_t)l * ldL] = beta[a * r + l];
}

// out[a*r + c] = A[row0 + a + (col0 + c)*ld]  (an r x r block, row-major)
__global__ void k_sub_block(const double* __restrict__ A, int64_t ld, int row0, int col0, int r,
                            double* __restrict__ out) {
  const int e = threadIdx.x;
  if (e >= r * r) return;
  const int a = e / r, c = e - a * r;
  out[e] = A[row0 + a + (int64_t)(col0 + c) * ld];
}

}  // namespace

void sub_block_launch(const double* A, int64_t ld, int row0, int col0, int r, double* out,
                      cudaStream_t st) {
  count_launches(1);
  k_sub_block<<<1, 32, 0, st>>>(A, ld, row0, col0, r, out);
}

int border_chunks(int mp) { return std::max(1, (mp + kBCols - 1) / kBCols); }

void border_col_launch(double* Ht, int64_t ldH, int mp, int r, const double* T, int64_t ldT,
                       const double* hslots, int first_block, int nslots, const double* h_dd,
                       double* partial, cudaStream_t st) {
  if (mp <= 0) return;
  const int nch = border_chunks(mp);
  dim3 grid((mp + kBRows - 1) / kBRows, nch);
  count_launches(1);
  k_border_gemv<<<grid, kBWarps * 32, 0, st>>>(Ht, ldH, mp, r, T, ldT, partial);
  count_launches(1);
  const unsigned g = (unsigned)((mp + 31) / 32);
#define SPK_BCOL(R) k_border_col<R><<<g, 32, 0, st>>>(Ht, ldH, mp, T, ldT, hslots, first_block, nslots, h_dd, partial, nch)
  switch (r) {
    case 1: SPK_BCOL(1); break;
    case 2: SPK_BCOL(2); break;
    case 3: SPK_BCOL(3); break;
    default: SPK_BCOL(4); break;
  }
#undef SPK_BCOL
}

void border_small_launch(double* Ht, int64_t ldH, int mp, int r, const double* T, int64_t ldT,
                         const double* h_sub, const double* h_dd, cudaStream_t st) {
  count_launches(1);
  switch (r) {
    case 1: k_border_small<1><<<1, 32, 0, st>>>(Ht, ldH, mp, T, ldT, h_sub, h_dd); break;
    case 2: k_border_small<2><<<1, 32, 0, st>>>(Ht, ldH, mp, T, ldT, h_sub, h_dd); break;
    case 3: k_border_small<3><<<1, 32, 0, st>>>(Ht, ldH, mp, T, ldT, h_sub, h_dd); break;
    default: k_border_small<4><<<1, 32, 0, st>>>(Ht, ldH, mp, T, ldT, h_sub, h_dd); break;
  }
}

void border_correct_launch(double* Ht, int64_t ldH, int m, int r, const double* T, int64_t ldT,
                           const double* h_next, cudaStream_t st) {
  count_launches(1);
  const unsigned g = (unsigned)((m + 127) / 128);
  switch (r) {
    case 1: k_border_correct<1><<<g, 128, 0, st>>>(Ht, ldH, m, T, ldT, h_next); break;
    case 2: k_border_correct<2><<<g, 128, 0, st>>>(Ht, ldH, m, T, ldT, h_next); break;
    case 3: k_border_correct<3><<<g, 128, 0, st>>>(Ht, ldH, m, T, ldT, h_next); break;
    default: k_border_correct<4><<<g, 128, 0, st>>>(Ht, ldH, m, T, ldT, h_next); break;
  }
}

void rho_launch(const double* Y, int64_t ldY, int m, int r, const double* TU, int64_t ldTU,
                const double* TV, int64_t ldTV, const double* hU, const double* hV,
                const double* betaU, const double* betaV, int bound, double* out3,
                cudaStream_t st) {
  count_launches(1);
  k_rho<<<1, 256, 0, st>>>(Y, ldY, m, r, TU, ldTU, TV, ldTV, hU, hV, betaU, betaV, bound, out3);
}

void band_to_dense_launch(const double* hband, int k, int r, int d, double* H, int64_t ldH,
                          cudaStream_t st) {
  const int64_t total = (int64_t)d * (k + 1) * r * r;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 4));
  count_launches(1);
  k_band_to_dense<<<g, 256, 0, st>>>(hband, k, r, d, H, ldH);
}

void fill_factor_launch(double* L, int64_t ldL, int r, const double* beta, cudaStream_t st) {
  count_launches(1);
  k_fill_factor<<<1, 32, 0, st>>>(L, ldL, r, beta);
}

}  // namespace spk
