// Kernels of the split solve of the projected Sylvester equation (Eq. (3.4))
// when H~ or G~ has eigenvalues off the open right half plane, where the sign
// iteration alone does not apply (see the driver in spk_api.cu):
//   - affine combinations of a matrix and its sign function (the spectral
//     projectors P+- = (I +- S)/2 and the shifted matrices H + c P-);
//   - the complex Schur form of a small k x k matrix (k <= kSplitMaxK):
//     Householder reduction to Hessenberg form, then the single-shift QR
//     algorithm with Wilkinson shifts and Givens rotations (Golub and Van
//     Loan, Matrix Computations, Sections 7.4-7.5, in complex arithmetic);
//   - the pieces of the back substitution T Zt + Zt G^T = Rt row by row,
//     each row a shifted system (G + t_ii I) z^T = rhs^T in its real 2m x 2m
//     form [[G + a I, -b I], [b I, G + a I]] for t_ii = a + i b.
#include "spk_internal.cuh"

#include <cmath>

namespace spk {

namespace {

int grid_for_n(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  return (int)g;
}

// out = alpha A + beta (I + gamma S)     (m x m, column-major)
__global__ void k_sign_affine(const double* __restrict__ A, int64_t lda, double alpha,
                              const double* __restrict__ S, int64_t lds, double beta, double gamma,
                              int m, double* __restrict__ out, int64_t ldo) {
  const int64_t total = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    double v = beta * gamma * S[j * lds + i];
    if (i == j) v += beta;
    if (A) v += alpha * A[j * lda + i];
    out[j * ldo + i] = v;
  }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {   // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 csqrt(double2 z) {
  const double r = cabs2(z);
  if (r == 0.0) return make_double2(0.0, 0.0);
  double re = sqrt(0.5 * (r + fabs(z.x)));
  double im = 0.5 * z.y / re;
  if (z.x < 0.0) {
    const double t = fabs(im);
    im = copysign(re, z.y);
    re = t;
  }
  return make_double2(re, im);
}

// Complex Schur form A = U T U^H of a real k x k matrix A (column-major, ld
// lda), one thread: T (k x k, upper triangular) and U (unitary), both
// column-major with leading dimension k.  flags |= kFlagZeroPivot when the
// QR iteration does not converge in 60 k steps.
__global__ void k_small_schur(const double* __restrict__ A, int64_t lda, int k,
                              double2* __restrict__ U, double2* __restrict__ T,
                              uint32_t* __restrict__ flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
#define TT(i, j) T[(j) * k + (i)]
#define UU(i, j) U[(j) * k + (i)]
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) {
      TT(i, j) = make_double2(A[j * lda + i], 0.0);
      UU(i, j) = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
  // Householder reduction to upper Hessenberg form: T <- P T P, U <- U P with
  // P = I - 2 v v^H acting on rows/columns j+1 .. k-1
  double2 v[kSplitMaxK];
  for (int j = 0; j + 2 < k; ++j) {
    double nx = 0.0;
    for (int i = j + 1; i < k; ++i) nx = hypot(nx, cabs2(TT(i, j)));
    if (nx == 0.0) continue;
    const double2 x0 = TT(j + 1, j);
    const double a0 = cabs2(x0);
    const double2 ph = a0 > 0.0 ? cscale(x0, 1.0 / a0) : make_double2(1.0, 0.0);
    // v = x + ph ||x|| e1  (alpha = -ph ||x||), normalised
    for (int i = j + 1; i < k; ++i) v[i] = TT(i, j);
    v[j + 1] = cadd(v[j + 1], cscale(ph, nx));
    double nv = 0.0;
    for (int i = j + 1; i < k; ++i) nv = hypot(nv, cabs2(v[i]));
    for (int i = j + 1; i < k; ++i) v[i] = cscale(v[i], 1.0 / nv);
    // left: T[j+1:, :] -= 2 v (v^H T[j+1:, :])
    for (int c = 0; c < k; ++c) {
      double2 s = make_double2(0.0, 0.0);
      for (int i = j + 1; i < k; ++i) s = cadd(s, cconjmul(v[i], TT(i, c)));
      for (int i = j + 1; i < k; ++i) TT(i, c) = csub(TT(i, c), cscale(cmul(v[i], s), 2.0));
    }
    // right: T[:, j+1:] -= 2 (T[:, j+1:] v) v^H; same for U
    for (int rr = 0; rr < k; ++rr) {
      double2 s = make_double2(0.0, 0.0), su = make_double2(0.0, 0.0);
      for (int i = j + 1; i < k; ++i) {
        s = cadd(s, cmul(TT(rr, i), v[i]));
        su = cadd(su, cmul(UU(rr, i), v[i]));
      }
      for (int i = j + 1; i < k; ++i) {
        TT(rr, i) = csub(TT(rr, i), cscale(cmul(s, cconj(v[i])), 2.0));
        UU(rr, i) = csub(UU(rr, i), cscale(cmul(su, cconj(v[i])), 2.0));
      }
    }
    for (int i = j + 2; i < k; ++i) TT(i, j) = make_double2(0.0, 0.0);
  }
  // shifted QR iteration on the active block [lo, hi]
  const double eps = 2.220446049250313e-16;
  int hi = k - 1, iter = 0, since = 0;
  double cs[kSplitMaxK];
  double2 sn[kSplitMaxK];
  while (hi > 0) {
    int lo = hi;
    while (lo > 0) {
      const double sub = cabs2(TT(lo, lo - 1));
      if (sub <= eps * (cabs2(TT(lo - 1, lo - 1)) + cabs2(TT(lo, lo)))) {
        TT(lo, lo - 1) = make_double2(0.0, 0.0);
        break;
      }
      --lo;
    }
    if (lo == hi) {
      --hi;
      since = 0;
      continue;
    }
    if (++iter > 60 * k) {
      atomicOr(flags, kFlagZeroPivot);
      break;
    }
    ++since;
    // Wilkinson shift: eigenvalue of the trailing 2 x 2 block closest to T[hi, hi]
    const double2 a = TT(hi - 1, hi - 1), b = TT(hi - 1, hi), c = TT(hi, hi - 1), d = TT(hi, hi);
    const double2 tr2 = cscale(cadd(a, d), 0.5);
    const double2 disc = csqrt(cadd(cmul(cscale(csub(a, d), 0.5), cscale(csub(a, d), 0.5)), cmul(b, c)));
    const double2 l1 = cadd(tr2, disc), l2 = csub(tr2, disc);
    double2 mu = cabs2(csub(l1, d)) < cabs2(csub(l2, d)) ? l1 : l2;
    if (since % 11 == 10) mu = cadd(d, make_double2(cabs2(c), 0.0));   // exceptional shift
    for (int i = lo; i <= hi; ++i) TT(i, i) = csub(TT(i, i), mu);
    // T - mu I = Q R by Givens rotations on rows p, p+1
    for (int p = lo; p < hi; ++p) {
      const double2 x = TT(p, p), y = TT(p + 1, p);
      const double ax = cabs2(x), r = hypot(ax, cabs2(y));
      double cc;
      double2 ss;
      if (r == 0.0) {
        cc = 1.0;
        ss = make_double2(0.0, 0.0);
      } else if (ax == 0.0) {
        cc = 0.0;
        ss = make_double2(1.0, 0.0);
      } else {
        cc = ax / r;
        ss = cscale(cmul(cscale(x, 1.0 / ax), cconj(y)), 1.0 / r);
      }
      cs[p] = cc;
      sn[p] = ss;
      for (int col = p; col < k; ++col) {
        const double2 u0 = TT(p, col), u1 = TT(p + 1, col);
        TT(p, col) = cadd(cscale(u0, cc), cmul(ss, u1));
        TT(p + 1, col) = csub(cscale(u1, cc), cmul(cconj(ss), u0));
      }
    }
    // R Q^H (+ mu I): rotations on columns p, p+1 of T (rows 0..p+1) and of U
    for (int p = lo; p < hi; ++p) {
      const double cc = cs[p];
      const double2 ss = sn[p];
      for (int rr = 0; rr <= p + 1; ++rr) {
        const double2 u0 = TT(rr, p), u1 = TT(rr, p + 1);
        TT(rr, p) = cadd(cscale(u0, cc), cmul(u1, cconj(ss)));
        TT(rr, p + 1) = csub(cscale(u1, cc), cmul(u0, ss));
      }
      for (int rr = 0; rr < k; ++rr) {
        const double2 u0 = UU(rr, p), u1 = UU(rr, p + 1);
        UU(rr, p) = cadd(cscale(u0, cc), cmul(u1, cconj(ss)));
        UU(rr, p + 1) = csub(cscale(u1, cc), cmul(u0, ss));
      }
    }
    for (int i = lo; i <= hi; ++i) TT(i, i) = cadd(TT(i, i), mu);
  }
  for (int j = 0; j < k; ++j)
    for (int i = j + 1; i < k; ++i) TT(i, j) = make_double2(0.0, 0.0);
#undef TT
#undef UU
}

// Rt (k x n complex, column-major ld k) = U^H R, R real k x n (ld ldr)
__global__ void k_uh_times(const double2* __restrict__ U, int k, const double* __restrict__ R,
                           int64_t ldr, int64_t n, double2* __restrict__ Rt) {
  const int64_t total = (int64_t)k * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / k;
    const int i = (int)(e - col * k);
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < k; ++j) s = cadd(s, cconjmul(U[i * k + j], make_double2(R[col * ldr + j], 0.0)));
    Rt[col * k + i] = s;
  }
}

// rhs (2n: real parts then imaginary parts) = Rt[i, :] - sum_{j > i} T[i, j] Zt[j, :]
__global__ void k_row_rhs(const double2* __restrict__ Rt, const double2* __restrict__ T, int k, int i,
                          const double2* __restrict__ Zt, int64_t n, double* __restrict__ rhs) {
  for (int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; col < n;
       col += (int64_t)gridDim.x * blockDim.x) {
    double2 s = Rt[col * k + i];
    for (int j = i + 1; j < k; ++j) s = csub(s, cmul(T[j * k + i], Zt[col * k + j]));
    rhs[col] = s.x;
    rhs[n + col] = s.y;
  }
}

// M (2n x 2n, column-major) = [[G + a I, -b I], [b I, G + a I]], t = a + i b = T[i, i]
__global__ void k_realify_shift(const double* __restrict__ G, int64_t ldg, int n,
                                const double2* __restrict__ T, int k, int i,
                                double* __restrict__ M) {
  const double2 t = T[i * k + i];
  const int64_t n2 = 2 * (int64_t)n;
  const int64_t total = n2 * n2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n2, rr = e - c * n2;
    const int64_t bi = rr / n, bj = c / n, li = rr - bi * n, lj = c - bj * n;
    double v;
    if (bi == bj) {
      v = G[lj * ldg + li] + (li == lj ? t.x : 0.0);
    } else {
      v = li == lj ? (bi == 0 ? -t.y : t.y) : 0.0;
    }
    M[c * n2 + rr] = v;
  }
}

// Zt[i, :] = x[0:n] + i x[n:2n]
__global__ void k_store_row(const double* __restrict__ x, int64_t n, int k, int i,
                            double2* __restrict__ Zt) {
  for (int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; col < n;
       col += (int64_t)gridDim.x * blockDim.x)
    Zt[col * k + i] = make_double2(x[col], x[n + col]);
}

// Z (k x n real, ld k) = Re(U Zt)
__global__ void k_u_times_real(const double2* __restrict__ U, int k, const double2* __restrict__ Zt,
                               int64_t n, double* __restrict__ Z) {
  const int64_t total = (int64_t)k * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / k;
    const int i = (int)(e - col * k);
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += cmul(U[j * k + i], Zt[col * k + j]).x;
    Z[col * k + i] = s;
  }
}

}  // namespace

void sign_affine_launch(const double* A, int64_t lda, double alpha, const double* S, int64_t lds,
                        double beta, double gamma, int m, double* out, int64_t ldo,
                        cudaStream_t st) {
  count_launches(1);
  k_sign_affine<<<grid_for_n((int64_t)m * m, 256), 256, 0, st>>>(A, lda, alpha, S, lds, beta,
                                                                  gamma, m, out, ldo);
}

void small_schur_launch(const double* A, int64_t lda, int k, double2* U, double2* T,
                        uint32_t* flags, cudaStream_t st) {
  count_launches(1);
  k_small_schur<<<1, 32, 0, st>>>(A, lda, k, U, T, flags);
}

void uh_times_launch(const double2* U, int k, const double* R, int64_t ldr, int64_t n,
                     double2* Rt, cudaStream_t st) {
  count_launches(1);
  k_uh_times<<<grid_for_n((int64_t)k * n, 256), 256, 0, st>>>(U, k, R, ldr, n, Rt);
}

void row_rhs_launch(const double2* Rt, const double2* T, int k, int i, const double2* Zt,
                    int64_t n, double* rhs, cudaStream_t st) {
  count_launches(1);
  k_row_rhs<<<grid_for_n(n, 256), 256, 0, st>>>(Rt, T, k, i, Zt, n, rhs);
}

void realify_shift_launch(const double* G, int64_t ldg, int n, const double2* T, int k, int i,
                          double* M, cudaStream_t st) {
  count_launches(1);
  k_realify_shift<<<grid_for_n(4 * (int64_t)n * n, 256), 256, 0, st>>>(G, ldg, n, T, k, i, M);
}

void store_row_launch(const double* x, int64_t n, int k, int i, double2* Zt, cudaStream_t st) {
  count_launches(1);
  k_store_row<<<grid_for_n(n, 256), 256, 0, st>>>(x, n, k, i, Zt);
}

void u_times_real_launch(const double2* U, int k, const double2* Zt, int64_t n, double* Z,
                         cudaStream_t st) {
  count_launches(1);
  k_u_times_real<<<grid_for_n((int64_t)k * n, 256), 256, 0, st>>>(U, k, Zt, n, Z);
}

}  // namespace spk
