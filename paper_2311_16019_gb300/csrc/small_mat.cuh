// r x r (r <= 4) matrix helpers with the size a template parameter, so that
// the matrices live in registers: the single-thread parts of the Cholesky
// QR, the T-block inverses and the bordering update run as straight-line
// code.  Divisions are one reciprocal per diagonal entry.
#pragma once

#include <stdint.h>

namespace spk {
namespace sm {

// B[a][c] = T[off + a, off + c] (T column-major, leading dimension ldT)
template <int R>
__device__ __forceinline__ void load_tblock(const double* T, int64_t ldT, int off, double (&B)[R][R]) {
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) B[a][c] = T[off + a + (int64_t)(off + c) * ldT];
}

// A[a][c] = p[a R + c] (row-major)
template <int R>
__device__ __forceinline__ void load_rm(const double* p, double (&A)[R][R]) {
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) A[a][c] = p[a * R + c];
}

template <int R>
__device__ __forceinline__ void store_rm(const double (&A)[R][R], double* p) {
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) p[a * R + c] = A[a][c];
}

// C = A B
template <int R>
__device__ __forceinline__ void mul(const double (&A)[R][R], const double (&B)[R][R], double (&C)[R][R]) {
  double o[R][R];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < R; ++l) s = fma(A[a][l], B[l][c], s);
      o[a][c] = s;
    }
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) C[a][c] = o[a][c];
}

// Ri = U^{-1} for upper-triangular U (back substitution, column by column)
template <int R>
__device__ __forceinline__ void upper_inv(const double (&U)[R][R], double (&Ri)[R][R]) {
  double d[R];
#pragma unroll
  for (int j = 0; j < R; ++j) d[j] = 1.0 / U[j][j];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int c = 0; c < R; ++c) Ri[a][c] = 0.0;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    Ri[j][j] = d[j];
#pragma unroll
    for (int i = j - 1; i >= 0; --i) {
      double t = 0.0;
#pragma unroll
      for (int l = i + 1; l <= j; ++l) t = fma(U[i][l], Ri[l][j], t);
      Ri[i][j] = -t * d[i];
    }
  }
}

}  // namespace sm
}  // namespace spk
