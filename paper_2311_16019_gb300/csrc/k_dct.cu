// DCT sketch: S X = sqrt(n/s) (N E X)[rows, :] with N the orthonormal DCT-II,
// the trigonometric transform the paper's experiments use (Section 6).
//
// DCT-II by Makhoul's reordering: v_j = x_{2j} for j < ceil(n/2) and
// v_{n-1-j} = x_{2j+1}, V = FFT_n(v), X_k = a_k Re(exp(-i pi k / (2n)) V_k),
// a_0 = sqrt(1/n), a_k = sqrt(2/n).  The complex FFT of length n = f1 f2 is
// done by the four-step method (j = j1 + f1 j2, k = k2 + f2 k1):
//   pass A (CTA per j1, column): length-f2 transforms over j2, times
//          exp(-2 pi i j1 k2 / n);
//   pass B (CTA per k2, column): length-f1 transforms over j1, then the DCT
//          post-twiddle and scale, writing only the s selected outputs.
// Each sub-transform is a mixed-radix (4, 2, 3, 5) Stockham FFT in shared
// memory; twiddle tables are computed once per sketch.  FP64 throughout,
// also in the mixed forms (the sketch output is FP64).
#include "spk_internal.cuh"

#include <cmath>
#include <vector>

namespace spk {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double t) { return make_double2(a.x * t, a.y * t); }
// -i * a
__device__ __forceinline__ double2 mul_mi(double2 a) { return make_double2(a.y, -a.x); }

// Radix-R DFTs, V_p = sum_q v_q w^{p q}, w = exp(-2 pi i / R), with the
// roots of unity written from their closed forms.
__device__ __forceinline__ void dft2(double2& v0, double2& v1) {
  const double2 a = cadd(v0, v1), b = csub(v0, v1);
  v0 = a;
  v1 = b;
}

__device__ __forceinline__ void dft4(double2 (&v)[4]) {
  const double2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  const double2 t2 = cadd(v[1], v[3]), t3 = mul_mi(csub(v[1], v[3]));
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

__device__ __forceinline__ void dft3(double2 (&v)[3]) {
  constexpr double c = -0.5;                    // cos(2 pi / 3)
  constexpr double sn = 0.86602540378443865;    // sin(2 pi / 3) = sqrt(3)/2
  const double2 s = cadd(v[1], v[2]);
  const double2 d = cscale(mul_mi(csub(v[1], v[2])), sn);
  const double2 base = cadd(v[0], cscale(s, c));
  v[0] = cadd(v[0], s);
  v[1] = cadd(base, d);
  v[2] = csub(base, d);
}

__device__ __forceinline__ void dft5(double2 (&v)[5]) {
  constexpr double c1 = 0.30901699437494742;    // cos(2 pi/5) = (sqrt5 - 1)/4
  constexpr double s1 = 0.95105651629515357;    // sin(2 pi/5)
  constexpr double c2 = -0.80901699437494742;   // cos(4 pi/5) = -(sqrt5 + 1)/4
  constexpr double s2 = 0.58778525229247313;    // sin(4 pi/5)
  const double2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
  const double2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
  const double2 r1 = cadd(v[0], cadd(cscale(a1, c1), cscale(a2, c2)));
  const double2 r2 = cadd(v[0], cadd(cscale(a1, c2), cscale(a2, c1)));
  const double2 i1 = mul_mi(cadd(cscale(b1, s1), cscale(b2, s2)));
  const double2 i2 = mul_mi(csub(cscale(b1, s2), cscale(b2, s1)));
  v[0] = cadd(v[0], cadd(a1, a2));
  v[1] = cadd(r1, i1);
  v[4] = csub(r1, i1);
  v[2] = cadd(r2, i2);
  v[3] = csub(r2, i2);
}

// One Stockham stage of radix R on a length-L sequence: a -> b.  Ns is the
// product of the earlier radices; tw[t] = exp(-2 pi i t / L).
template <int R>
__device__ void stockham_stage(const double2* a, double2* b, int L, int Ns,
                               const double2* __restrict__ tw) {
  const int m = L / R;
  const int step = L / (Ns * R);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const int k = j % Ns;
    double2 v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = a[j + q * m];
    if (Ns > 1) {
#pragma unroll
      for (int q = 1; q < R; ++q) v[q] = cmul(v[q], tw[(q * k * step) % L]);
    }
    if constexpr (R == 2) dft2(v[0], v[1]);
    if constexpr (R == 3) dft3(v);
    if constexpr (R == 4) dft4(v);
    if constexpr (R == 5) dft5(v);
    const int idx = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) b[idx + q * Ns] = v[q];
  }
}

// Full transform of buf[0] (length L) in shared memory; returns the buffer
// that holds the result.
__device__ double2* stockham_fft(double2* buf0, double2* buf1, const FftPlan& pl,
                                 const double2* __restrict__ tw) {
  double2* a = buf0;
  double2* b = buf1;
  int Ns = 1;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = pl.radix[st];
    if (R == 4) stockham_stage<4>(a, b, pl.len, Ns, tw);
    else if (R == 2) stockham_stage<2>(a, b, pl.len, Ns, tw);
    else if (R == 3) stockham_stage<3>(a, b, pl.len, Ns, tw);
    else stockham_stage<5>(a, b, pl.len, Ns, tw);
    __syncthreads();
    Ns *= R;
    double2* t = a;
    a = b;
    b = t;
  }
  return a;
}

// Pass A: CTA (j1, c).  v_j for j = j1 + f1 j2 (Makhoul reordering of the
// signed column c), length-f2 FFT over j2, times exp(-2 pi i j1 k2 / n);
// Y[c n + k2 f1 + j1].
template <typename TB>
__global__ void __launch_bounds__(256) k_dct_pass_a(const TB* __restrict__ X, int64_t n, int r,
                                                    const int8_t* __restrict__ signs, DctDev dd,
                                                    double2* __restrict__ Y) {
  __shared__ double2 buf[2][kFftMax];
  const int j1 = blockIdx.x, c = blockIdx.y;
  const int f1 = dd.p1.len, f2 = dd.p2.len;
  const int64_t half = (n + 1) / 2;
  for (int j2 = threadIdx.x; j2 < f2; j2 += blockDim.x) {
    const int64_t j = j1 + (int64_t)f1 * j2;
    const int64_t src = j < half ? 2 * j : 2 * (n - 1 - j) + 1;
    double v = (double)Store<TB>::ld(X + src * r + c);
    if (signs[src] < 0) v = -v;
    buf[0][j2] = make_double2(v, 0.0);
  }
  __syncthreads();
  const double2* res = stockham_fft(buf[0], buf[1], dd.p2, dd.tw2);
  for (int k2 = threadIdx.x; k2 < f2; k2 += blockDim.x)
    Y[(int64_t)c * n + (int64_t)k2 * f1 + j1] = cmul(res[k2], dd.twn[(int64_t)j1 * k2]);
}

// Pass B: CTA (k2, c).  Length-f1 FFT over j1 of Y[c n + k2 f1 + j1]; output
// k1 is V_k for k = k2 + f2 k1; selected k go to SX[pos + c s].
__global__ void __launch_bounds__(256) k_dct_pass_b(const double2* __restrict__ Y, int64_t n,
                                                    DctDev dd, const int32_t* __restrict__ selpos,
                                                    int32_t s, double scale,
                                                    double* __restrict__ SX) {
  __shared__ double2 buf[2][kFftMax];
  const int k2 = blockIdx.x, c = blockIdx.y;
  const int f1 = dd.p1.len, f2 = dd.p2.len;
  for (int j1 = threadIdx.x; j1 < f1; j1 += blockDim.x)
    buf[0][j1] = Y[(int64_t)c * n + (int64_t)k2 * f1 + j1];
  __syncthreads();
  const double2* res = stockham_fft(buf[0], buf[1], dd.p1, dd.tw1);
  const double a0 = sqrt(1.0 / (double)n), ak = sqrt(2.0 / (double)n);
  for (int k1 = threadIdx.x; k1 < f1; k1 += blockDim.x) {
    const int64_t k = k2 + (int64_t)f2 * k1;
    const int32_t pos = selpos[k];
    if (pos < 0) continue;
    const double2 w = cmul(dd.post[k], res[k1]);
    SX[pos + (int64_t)c * s] = w.x * (k == 0 ? a0 : ak) * scale;
  }
}

// tab[t] = exp(-2 pi i t num / den) for t < count.
__global__ void k_twiddles(double2* tab, int64_t count, int64_t num, int64_t den) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    // angle -2 t num / den in units of pi, reduced to [0, 2) exactly in integers
    const int64_t q = (t * num) % den;
    double sv, cv;
    sincospi(-2.0 * (double)q / (double)den, &sv, &cv);
    tab[t] = make_double2(cv, sv);
  }
}

__global__ void k_selpos(const int32_t* __restrict__ rows, int32_t s, int32_t* __restrict__ selpos) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < s; j += gridDim.x * blockDim.x)
    selpos[rows[j]] = j;
}

bool plan_for(int L, FftPlan& pl) {
  pl.len = L;
  pl.nst = 0;
  int m = L;
  while (m > 1) {
    int R = 0;
    if (m % 4 == 0) R = 4;
    else if (m % 2 == 0) R = 2;
    else if (m % 3 == 0) R = 3;
    else if (m % 5 == 0) R = 5;
    else return false;
    if (pl.nst >= kFftMaxStages) return false;
    pl.radix[pl.nst++] = (int8_t)R;
    m /= R;
  }
  return true;
}

int grid_of(int64_t work) {
  int64_t g = (work + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

}  // namespace

bool dct_geometry(int64_t n, DctDev& dd) {
  // n = f1 f2 with both lengths <= kFftMax, f1 as close to sqrt(n) as allowed
  int best = -1;
  for (int f1 = 1; f1 <= kFftMax && f1 <= n; ++f1) {
    if (n % f1) continue;
    const int64_t f2 = n / f1;
    if (f2 > kFftMax) continue;
    FftPlan a, b;
    if (!plan_for(f1, a) || !plan_for((int)f2, b)) continue;
    if (best < 0 || std::llabs((int64_t)f1 * f1 - n) < std::llabs((int64_t)best * best - n)) best = f1;
  }
  if (best < 0) return false;
  plan_for(best, dd.p1);
  plan_for((int)(n / best), dd.p2);
  return true;
}

size_t dct_table_doubles(int64_t n, const DctDev& dd) {
  return 2 * ((size_t)dd.p1.len + dd.p2.len + 2 * (size_t)n);
}

void dct_tables_launch(int64_t n, DctDev& dd, double* tables, cudaStream_t st) {
  double2* t = reinterpret_cast<double2*>(tables);
  double2* tw1 = t;
  double2* tw2 = t + dd.p1.len;
  double2* twn = t + dd.p1.len + dd.p2.len;
  double2* post = t + dd.p1.len + dd.p2.len + n;
  count_launches(4);
  k_twiddles<<<grid_of(dd.p1.len), 256, 0, st>>>(tw1, dd.p1.len, 1, dd.p1.len);
  k_twiddles<<<grid_of(dd.p2.len), 256, 0, st>>>(tw2, dd.p2.len, 1, dd.p2.len);
  k_twiddles<<<grid_of(n), 256, 0, st>>>(twn, n, 1, n);
  // exp(-i pi k / (2n)) = exp(-2 pi i k / (4n))
  k_twiddles<<<grid_of(n), 256, 0, st>>>(post, n, 1, 4 * n);
  dd.tw1 = tw1;
  dd.tw2 = tw2;
  dd.twn = twn;
  dd.post = post;
}

void dct_selpos_launch(const int32_t* rows, int32_t s, int64_t n, int32_t* selpos, cudaStream_t st) {
  cudaMemsetAsync(selpos, 0xff, sizeof(int32_t) * (size_t)n, st);
  count_launches(1);
  k_selpos<<<grid_of(s), 256, 0, st>>>(rows, s, selpos);
}

template <typename TB>
void dct_apply_launch(const SketchDev& sk, const TB* X, int r, double* SX, double* cwork,
                      cudaStream_t st) {
  double2* Y = reinterpret_cast<double2*>(cwork);
  count_launches(1);
  k_dct_pass_a<TB><<<dim3((unsigned)sk.dct.p1.len, (unsigned)r), 256, 0, st>>>(
      X, sk.n, r, sk.signs, sk.dct, Y);
  count_launches(1);
  k_dct_pass_b<<<dim3((unsigned)sk.dct.p2.len, (unsigned)r), 256, 0, st>>>(
      Y, sk.n, sk.dct, sk.selpos, sk.s, sk.scale, SX);
}

template void dct_apply_launch<double>(const SketchDev&, const double*, int, double*, double*,
                                       cudaStream_t);
template void dct_apply_launch<float>(const SketchDev&, const float*, int, double*, double*,
                                      cudaStream_t);
template void dct_apply_launch<__nv_bfloat16>(const SketchDev&, const __nv_bfloat16*, int, double*,
                                              double*, cudaStream_t);

}  // namespace spk
