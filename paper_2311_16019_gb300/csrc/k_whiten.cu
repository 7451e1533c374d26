// Whitening QR update (Proposition 2.1; Algorithm 1's sketched-basis QR).
//
// Given Q_d (s x dr, orthonormal columns, FP64 column-major) and the sketch
// w = S U_{d+1} (s x r), block classical Gram-Schmidt with one
// reorthogonalisation:
//     t1 = Q_d^T w,  w1 = w - Q_d t1,  t2 = Q_d^T w1,  w2 = w1 - Q_d t2,
//     Q_new tau_{d+1} = w2  (Cholesky QR applied twice),
//     T_{d+1} = [[T_d, t1 + t2], [0, tau_{d+1}]].
// All FP64 (also in the mixed forms).  Every reduction has a fixed order.
#include "spk_internal.cuh"

#include <algorithm>

namespace spk {

namespace {

// Partial dot products of the columns of Q with w over one chunk of rows:
//   tpart[(ch*m + j)*R + c] = sum_{i in chunk ch} Q[i + j*ldq] * w[i + c*s],
// one warp per (column j, row chunk ch).  Splitting the rows gives enough
// equal work items to keep every SM's FP64 pipe busy to the end (one warp
// per column alone leaves a partial last wave on 152 SMs).
template <int R>
__global__ void __launch_bounds__(256) k_qt_dot(const double* __restrict__ Q, int64_t ldq, int64_t s,
                                                int m, int64_t rows_per_chunk, int nchunk,
                                                const double* __restrict__ w,
                                                double* __restrict__ tpart) {
  // warps stride over the items (a grid of a few CTAs per SM): every SM gets
  // the same share of FP64 work and no partial last wave is left
  const int lane = threadIdx.x & 31;
  const int64_t nitems = (int64_t)m * nchunk;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < nitems;
       item += nwarps) {
    const int j = (int)(item % m);
    const int ch = (int)(item / m);
    const int64_t i0 = (int64_t)ch * rows_per_chunk;
    const int64_t i1 = min(s, i0 + rows_per_chunk);
    const double* q = Q + (int64_t)j * ldq;
    double acc[R];
#pragma unroll
    for (int c = 0; c < R; ++c) acc[c] = 0.0;
    for (int64_t i = i0 + lane; i < i1; i += 32) {
      const double qi = q[i];
#pragma unroll
      for (int c = 0; c < R; ++c) acc[c] = fma(qi, w[i + c * s], acc[c]);
    }
    warp_sum_store<R>(acc, tpart + ((int64_t)ch * m + j) * R);
  }
}

// t[e] = sum_ch tpart[ch*m*R + e], chunks in ascending order.
__global__ void k_qt_finish(const double* __restrict__ tpart, int64_t count, int nchunk,
                            double* __restrict__ t) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) acc += tpart[(int64_t)ch * count + e];
    t[e] = acc;
  }
}

constexpr int kRowTile = 128;
constexpr int kColChunk = 256;
constexpr int kQtMaxChunks = 32;

// partial[(chunk*s + i)*r + c] = sum_{j in chunk} Q[i + j*ldq] * t[j*r + c],
// chunks of cw <= kColChunk columns
template <int R>
__global__ void __launch_bounds__(kRowTile) k_q_times_t(const double* __restrict__ Q, int64_t ldq,
                                                        int64_t s, int m, int cw,
                                                        const double* __restrict__ t,
                                                        double* __restrict__ partial) {
  __shared__ double ts[kColChunk * R];
  const int chunk = blockIdx.y;
  const int j0 = chunk * cw;
  const int j1 = min(m, j0 + cw);
  for (int e = threadIdx.x; e < (j1 - j0) * R; e += blockDim.x) ts[e] = t[(int64_t)j0 * R + e];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kRowTile + threadIdx.x;
  if (i >= s) return;
  double acc[R];
#pragma unroll
  for (int c = 0; c < R; ++c) acc[c] = 0.0;
  const double* q = Q + i + (int64_t)j0 * ldq;
  for (int j = 0; j < j1 - j0; ++j) {
    const double qi = q[(int64_t)j * ldq];
#pragma unroll
    for (int c = 0; c < R; ++c) acc[c] = fma(qi, ts[j * R + c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < R; ++c) partial[((int64_t)chunk * s + i) * R + c] = acc[c];
}

// w_out[i + c*s] = w_in[i + c*s] - sum_chunk partial[chunk][i][c]
template <int R>
__global__ void k_q_update_finish(const double* __restrict__ w_in, double* __restrict__ w_out,
                                  const double* __restrict__ partial, int64_t s, int nchunk) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < R; ++c) {
      double acc = 0.0;
      for (int ch = 0; ch < nchunk; ++ch) acc += partial[((int64_t)ch * s + i) * R + c];
      w_out[i + c * s] = w_in[i + c * s] - acc;
    }
  }
}

template <int R>
__global__ void __launch_bounds__(256) k_ts_gram(const double* __restrict__ w, int64_t s,
                                                 double* __restrict__ partial) {
  double acc[R * R];
#pragma unroll
  for (int e = 0; e < R * R; ++e) acc[e] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v[R];
#pragma unroll
    for (int c = 0; c < R; ++c) v[c] = w[i + c * s];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) acc[a * R + b] = fma(v[a], v[b], acc[a * R + b]);
  }
  block_sum_store<R * R>(acc, partial + (int64_t)blockIdx.x * R * R);
}

// out[i + c*ldo] = sum_{a<=c} w[i + a*s] Rinv[a][c]   (w may alias out when ldo == s)
template <int R>
__global__ void k_ts_scale(const double* w, int64_t s, const double* __restrict__ Rinv,
                           double* out, int64_t ldo) {
  __shared__ double ri[R * R];
  if (threadIdx.x < R * R) ri[threadIdx.x] = Rinv[threadIdx.x];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v[R], o[R];
#pragma unroll
    for (int c = 0; c < R; ++c) v[c] = w[i + c * s];
#pragma unroll
    for (int c = 0; c < R; ++c) {
      double acc = 0.0;
#pragma unroll
      for (int a = 0; a <= c; ++a) acc = fma(v[a], ri[a * R + c], acc);
      o[c] = acc;
    }
#pragma unroll
    for (int c = 0; c < R; ++c) out[i + c * ldo] = o[c];
  }
}

__global__ void k_t_write(double* __restrict__ T, int64_t ldT, int m, int r,
                          const double* __restrict__ t1, const double* __restrict__ t2,
                          const double* __restrict__ tau) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (m + r) * r; e += gridDim.x * blockDim.x) {
    const int j = e / r, c = e - j * r;
    double v;
    if (j < m) {
      v = t1 ? t1[(int64_t)j * r + c] : 0.0;
      if (t2) v += t2[(int64_t)j * r + c];
    } else {
      const int a = j - m;
      v = (a <= c) ? tau[a * r + c] : 0.0;
    }
    T[j + (int64_t)(m + c) * ldT] = v;
  }
}

int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 4));
}

}  // namespace

int qt_dot_chunks(int64_t s, int m) {
  // about two warps' worth of items per resident warp slot (152 SMs x 64),
  // at least 256 rows per chunk
  const int64_t target = 2LL * 152 * 64;
  int64_t nc = (target + m - 1) / std::max(1, m);
  nc = std::min<int64_t>(nc, std::max<int64_t>(1, s / 256));
  return (int)std::max<int64_t>(1, std::min<int64_t>(nc, kQtMaxChunks));
}

void qt_dot_launch(const double* Q, int64_t ldq, int64_t s, int m, const double* w, int r,
                   double* t, double* tpart, cudaStream_t st) {
  if (m <= 0) return;
  const int nc = qt_dot_chunks(s, m);
  const int64_t rows = ((s + nc - 1) / nc + 31) / 32 * 32;
  double* out = nc == 1 ? t : tpart;
  const unsigned blocks = (unsigned)std::min<int64_t>(((int64_t)m * nc + 7) / 8, 152 * 8);
  count_launches(1);
  switch (r) {
    case 1: k_qt_dot<1><<<blocks, 256, 0, st>>>(Q, ldq, s, m, rows, nc, w, out); break;
    case 2: k_qt_dot<2><<<blocks, 256, 0, st>>>(Q, ldq, s, m, rows, nc, w, out); break;
    case 3: k_qt_dot<3><<<blocks, 256, 0, st>>>(Q, ldq, s, m, rows, nc, w, out); break;
    default: k_qt_dot<4><<<blocks, 256, 0, st>>>(Q, ldq, s, m, rows, nc, w, out); break;
  }
  if (nc > 1) {
    count_launches(1);
    k_qt_finish<<<grid_for((int64_t)m * r, 256), 256, 0, st>>>(tpart, (int64_t)m * r, nc, t);
  }
}

int qt_dot_partial_doubles(int mmax, int r) { return kQtMaxChunks * mmax * r; }

void qt_finish_launch(const double* tpart, int64_t count, int nchunk, double* t, cudaStream_t st) {
  count_launches(1);
  k_qt_finish<<<grid_for(count, 256), 256, 0, st>>>(tpart, count, nchunk, t);
}

void q_update_finish_launch(const double* w_in, double* w_out, const double* partial, int64_t s,
                            int r, int nchunk, cudaStream_t st) {
  const int g = grid_for(s, 256);
  count_launches(1);
  switch (r) {
    case 1: k_q_update_finish<1><<<g, 256, 0, st>>>(w_in, w_out, partial, s, nchunk); break;
    case 2: k_q_update_finish<2><<<g, 256, 0, st>>>(w_in, w_out, partial, s, nchunk); break;
    case 3: k_q_update_finish<3><<<g, 256, 0, st>>>(w_in, w_out, partial, s, nchunk); break;
    default: k_q_update_finish<4><<<g, 256, 0, st>>>(w_in, w_out, partial, s, nchunk); break;
  }
}

void q_update_launch(const double* Q, int64_t ldq, int64_t s, int m, const double* t, int r,
                     const double* w_in, double* w_out, double* partial, int nchunk,
                     cudaStream_t st) {
  if (m <= 0) {
    cudaMemcpyAsync(w_out, w_in, sizeof(double) * s * r, cudaMemcpyDeviceToDevice, st);
    return;
  }
  const int cw = (m + nchunk - 1) / nchunk;    // <= kColChunk (q_update_chunks)
  dim3 grid((unsigned)((s + kRowTile - 1) / kRowTile), (unsigned)nchunk);
  const int g2 = grid_for(s, 256);
  switch (r) {
    case 1:
      count_launches(1);
      k_q_times_t<1><<<grid, kRowTile, 0, st>>>(Q, ldq, s, m, cw, t, partial);
      count_launches(1);
      k_q_update_finish<1><<<g2, 256, 0, st>>>(w_in, w_out, partial, s, nchunk);
      break;
    case 2:
      count_launches(1);
      k_q_times_t<2><<<grid, kRowTile, 0, st>>>(Q, ldq, s, m, cw, t, partial);
      count_launches(1);
      k_q_update_finish<2><<<g2, 256, 0, st>>>(w_in, w_out, partial, s, nchunk);
      break;
    case 3:
      count_launches(1);
      k_q_times_t<3><<<grid, kRowTile, 0, st>>>(Q, ldq, s, m, cw, t, partial);
      count_launches(1);
      k_q_update_finish<3><<<g2, 256, 0, st>>>(w_in, w_out, partial, s, nchunk);
      break;
    default:
      count_launches(1);
      k_q_times_t<4><<<grid, kRowTile, 0, st>>>(Q, ldq, s, m, cw, t, partial);
      count_launches(1);
      k_q_update_finish<4><<<g2, 256, 0, st>>>(w_in, w_out, partial, s, nchunk);
      break;
  }
}

// Column chunks of Q t: at least ceil(m / kColChunk), and more (down to 32
// columns each) while the row tiles alone would leave the GPU short of about
// four CTAs per SM.  Non-decreasing in m, so the count at the largest m
// sizes the partial buffer.
int q_update_chunks(int m, int64_t s) {
  const int base = std::max(1, (m + kColChunk - 1) / kColChunk);
  const int64_t tiles = std::max<int64_t>(1, (s + kRowTile - 1) / kRowTile);
  const int want = (int)std::min<int64_t>(64, (4 * 152 + tiles - 1) / tiles);
  const int fine = std::max(1, std::min(want, (m + 31) / 32));
  return std::max(base, fine);
}

void ts_gram_launch(const double* w, int64_t s, int r, double* partial, int grid, cudaStream_t st) {
  switch (r) {
    case 1: count_launches(1); k_ts_gram<1><<<grid, 256, 0, st>>>(w, s, partial); break;
    case 2: count_launches(1); k_ts_gram<2><<<grid, 256, 0, st>>>(w, s, partial); break;
    case 3: count_launches(1); k_ts_gram<3><<<grid, 256, 0, st>>>(w, s, partial); break;
    default: count_launches(1); k_ts_gram<4><<<grid, 256, 0, st>>>(w, s, partial); break;
  }
}

void ts_scale_launch(double* w, int64_t s, int r, const double* Rinv, double* out, int64_t ldo,
                     cudaStream_t st) {
  const int g = grid_for(s, 256);
  switch (r) {
    case 1: count_launches(1); k_ts_scale<1><<<g, 256, 0, st>>>(w, s, Rinv, out, ldo); break;
    case 2: count_launches(1); k_ts_scale<2><<<g, 256, 0, st>>>(w, s, Rinv, out, ldo); break;
    case 3: count_launches(1); k_ts_scale<3><<<g, 256, 0, st>>>(w, s, Rinv, out, ldo); break;
    default: count_launches(1); k_ts_scale<4><<<g, 256, 0, st>>>(w, s, Rinv, out, ldo); break;
  }
}

void t_write_launch(double* T, int64_t ldT, int m, int r, const double* t1, const double* t2,
                    const double* tau, cudaStream_t st) {
  count_launches(1);
  k_t_write<<<grid_for((int64_t)(m + r) * r, 256), 256, 0, st>>>(T, ldT, m, r, t1, t2, tau);
}

}  // namespace spk
