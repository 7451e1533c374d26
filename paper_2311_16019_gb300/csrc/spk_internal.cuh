// Internal declarations of libspk (not part of the C ABI).
//
// Layout conventions used by every kernel:
//   block vectors  n x r   row-major, element (i, c) at [i * r + c]
//   dense matrices m x m   column-major with an explicit leading dimension
//   T (whitening factor), Q (sketched basis), H~ (projected matrix): FP64
//   column-major; the window of basis blocks is a ring of k+1 blocks.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/spk.h"

namespace spk {

constexpr int kMaxR = 4;      // block width r supported by the fused kernels
constexpr int kMaxWin = 16;   // largest truncation window k
constexpr int kXMaxBlocks = 8; // blocks per factor-accumulation launch
constexpr int kXPanelCols = 64; // basis columns per tensor-core accumulation

// Device-side status word bits (written by kernels, read by the host).
enum : uint32_t {
  kFlagBreakdown = 1u << 0,
  kFlagNonfinite = 1u << 1,
  kFlagZeroPivot = 1u << 2,
  kFlagTimeout = 1u << 3,     // a bounded device-side wait gave up
};

// Number of kernel launches issued by the library since it was loaded.
void count_launches(int64_t n);
int64_t launch_count();
// Bounded host waits: poll until the stream (event) completes, an error
// appears, or budget_s seconds pass.  0 = done, 1 = timed out, 2 = error.
int bounded_stream_wait(cudaStream_t st, double budget_s);
int bounded_event_wait(cudaEvent_t ev, double budget_s);
constexpr double kHostWaitSeconds = 600.0;

// ---------------------------------------------------------------- storage
template <typename T> struct Store;
template <> struct Store<double> {
  __device__ __forceinline__ static double ld(const double* p) { return *p; }
  __device__ __forceinline__ static void st(double* p, double v) { *p = v; }
};
template <> struct Store<float> {
  __device__ __forceinline__ static float ld(const float* p) { return *p; }
  __device__ __forceinline__ static void st(float* p, float v) { *p = v; }
};
template <> struct Store<__nv_bfloat16> {
  __device__ __forceinline__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ __forceinline__ static void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of R <= 4 per-lane values, written to out[c] (c < R) by the lane
// that ends up holding sum c.  The first one or two shuffle levels are a
// reduce-scatter (each lane keeps half of its values), so R = 4 costs 6
// additions per lane instead of 20.  Fixed order (deterministic).
template <int R>
__device__ __forceinline__ void warp_sum_store(const double (&acc)[R], double* out) {
  const int lane = threadIdx.x & 31;
  if constexpr (R == 1) {
    const double v = warp_sum(acc[0]);
    if (lane == 0) out[0] = v;
  } else {
    constexpr int RP = R <= 2 ? 2 : 4;
    double v[RP];
#pragma unroll
    for (int e = 0; e < RP; ++e) v[e] = e < R ? acc[e] : 0.0;
    {
      const bool up = (lane & 16) != 0;
#pragma unroll
      for (int e = 0; e < RP / 2; ++e) {
        const double give = up ? v[e] : v[e + RP / 2];
        const double keep = up ? v[e + RP / 2] : v[e];
        v[e] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
      }
    }
    int idx = (lane >> 4) & 1;
    int first = 8;
    if constexpr (RP == 4) {
      const bool up = (lane & 8) != 0;
      const double give = up ? v[0] : v[1];
      const double keep = up ? v[1] : v[0];
      v[0] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
      idx = 2 * idx + ((lane >> 3) & 1);
      first = 4;
    }
    for (int o = first; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    if ((lane & (2 * first - 1)) == 0 && idx < R) out[idx] = v[0];
  }
}

// Block-wide sums of NV per-thread values: out[e] = sum over the block's
// threads of acc[e], for e < NV (fixed order, so deterministic).  Within a
// warp, NV > 8 values are reduce-scattered: at each of the five shuffle
// levels a lane keeps one half of its values and adds its partner's copy of
// that half, ending with NV/32 complete warp sums for about NV additions
// (5 NV with one shuffle tree per value).  acc may be clobbered.  Ends
// with a barrier, so the caller may reuse shared memory afterwards.
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&acc)[NV], double* out) {
  constexpr int NVP = NV <= 8 ? NV : ((NV + 31) / 32) * 32;
  __shared__ double red[32][NVP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  if constexpr (NV <= 8) {
#pragma unroll
    for (int e = 0; e < NV; ++e) {
      const double v = warp_sum(acc[e]);
      if (lane == 0) red[wid][e] = v;
    }
  } else {
    // in place when NV is a multiple of 32 (acc is clobbered), else padded
    double pad[NV == NVP ? 1 : NVP];
    double* v;
    if constexpr (NV == NVP) {
      v = acc;
    } else {
#pragma unroll
      for (int e = 0; e < NVP; ++e) pad[e] = e < NV ? acc[e] : 0.0;
      v = pad;
    }
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
      const int o = 16 >> lv;
      const int half = NVP >> (lv + 1);
      const bool upper = (lane & o) != 0;
#pragma unroll
      for (int e = 0; e < half; ++e) {
        const double give = upper ? v[e] : v[e + half];
        const double keep = upper ? v[e + half] : v[e];
        v[e] = keep + __shfl_xor_sync(0xffffffffu, give, o);
      }
    }
    // lane holds the sums of entries lane*PER .. lane*PER + PER - 1
    constexpr int PER = NVP / 32;
#pragma unroll
    for (int e = 0; e < PER; ++e) red[wid][lane * PER + e] = v[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NV; e += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w][e];
    out[e] = t;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- sketch
// Mixed-radix plan of one DCT sub-transform length (radices 4, 2, 3, 5).
constexpr int kFftMax = 1024;
constexpr int kFftMaxStages = 10;
struct FftPlan {
  int32_t len = 1;
  int32_t nst = 0;
  int8_t radix[kFftMaxStages] = {};
};
// DCT sketch geometry: n = p1.len * p2.len and device twiddle tables.
struct DctDev {
  FftPlan p1, p2;
  const double2* tw1 = nullptr;   // exp(-2 pi i t / f1)
  const double2* tw2 = nullptr;   // exp(-2 pi i t / f2)
  const double2* twn = nullptr;   // exp(-2 pi i t / n)
  const double2* post = nullptr;  // exp(-i pi k / (2 n))
};

struct SketchDev {
  int64_t n = 0;        // rows of the sketched blocks
  int64_t npad = 0;     // n' = 2^ceil(log2 n)
  int32_t s = 0;        // sketch rows
  int32_t n2 = 1;       // first-level transform length (power of two)
  int32_t log2n2 = 0;
  int64_t n1 = 1;       // number of first-level chunks, npad / n2
  int32_t identity = 0; // S = I (s = n)
  double scale = 1.0;   // 1/sqrt(s) (SRHT) or 1 (identity)
  int32_t* rows = nullptr;   // s selected rows, ascending
  int8_t* signs = nullptr;   // n Rademacher signs
  // DCT sketch (is_dct): rows drawn over [0, n), selpos[k] = position of row
  // k in rows or -1, cwork = 2 n r doubles of complex work
  int32_t is_dct = 0;
  DctDev dct;
  int32_t* selpos = nullptr;
  double* cwork = nullptr;
};

// Launchers (k_sketch.cu)
// DCT sketch: geometry (false if n is not a product of two lengths <= 1024
// built from the radices 2, 3, 5), twiddle tables (dct_table_doubles
// doubles, kept alive by the caller), row positions, and the application.
bool dct_geometry(int64_t n, DctDev& dd);
size_t dct_table_doubles(int64_t n, const DctDev& dd);
void dct_tables_launch(int64_t n, DctDev& dd, double* tables, cudaStream_t st);
void dct_selpos_launch(const int32_t* rows, int32_t s, int64_t n, int32_t* selpos, cudaStream_t st);
template <typename TB>
void dct_apply_launch(const SketchDev& sk, const TB* X, int r, double* SX, double* cwork,
                      cudaStream_t st);

int sketch_draws_launch(int64_t n, int32_t s, uint64_t seed, int32_t sketch_id,
                        int32_t* rows, int8_t* signs, void* scratch, size_t scratch_bytes,
                        cudaStream_t st, char* err, size_t errlen,
                        int64_t range = 0);
size_t sketch_draws_scratch_bytes(int64_t n, int32_t s, int64_t range = 0);
void sketch_geometry(SketchDev& sk, int64_t n, int32_t s, int identity, int elem_bytes, int r);
size_t sketch_apply_scratch_bytes(const SketchDev& sk, int r);
// SX (s x r column-major, FP64) = S X, X row-major n x r of type TB.
template <typename TB, typename TC>
void sketch_apply_launch(const SketchDev& sk, const TB* X, int r, double* SX, TC* scratch,
                         cudaStream_t st);

// ---------------------------------------------------------------- Arnoldi
struct WindowPtrs {
  const void* blk[kMaxWin];   // U_i for the k window blocks, oldest first
  int nwin;
};

template <typename TB, typename TC, typename TV>
void spmm_dots_launch(const int32_t* rowptr, const int32_t* col, const TV* val, int64_t n, int r,
                      const TB* U, TC* W, WindowPtrs win, double* partial, int grid, cudaStream_t st);
void reduce_partials_launch(const double* partial, int nparts, int stride, int count,
                            double* out, cudaStream_t st);
template <typename TB, typename TC>
void update_gram_launch(TC* W, int64_t n, int r, WindowPtrs win, const double* h, double* partial,
                        int grid, int want_gram, cudaStream_t st);
void chol_small_launch(const double* partial, int nparts, int r, double* R, double* Rinv,
                       uint32_t* flags, double rel_floor, cudaStream_t st);
template <typename TC>
void scale_gram_launch(TC* W, int64_t n, int r, const double* Rinv, double* partial, int grid,
                       cudaStream_t st);
template <typename TB, typename TC>
void scale_store_launch(const TC* W, int64_t n, int r, const double* Rinv, TB* dst,
                        cudaStream_t st);
template <typename TB>
void x_accumulate_launch(double* X, int64_t n, int ell, int r, WindowPtrs blocks,
                         const double* Wrows, int64_t ldw, cudaStream_t st);
void spmm_wide_launch(const int32_t* rowptr, const int32_t* col, const double* val, int64_t n,
                      int w, const double* X, double* Y, cudaStream_t st);
template <typename TV>
void convert_values_launch(const double* src, TV* dst, int64_t count, cudaStream_t st);
// r columns of a row-major n x r block into an FP64 column-major panel (ld ldp)
template <typename TB>
void block_to_panel_launch(const TB* U, int64_t n, int r, double* P, int64_t ldp, cudaStream_t st);
// X (n x ell, row-major) from Xcm (n x ell, column-major)
void cols_to_rows_launch(const double* Xcm, int64_t n, int ell, double* X, cudaStream_t st);
template <typename TB>
void convert_block_launch(const double* src, TB* dst, int64_t count, cudaStream_t st);
void combine_small_launch(const double* A, const double* B, double* C, int r, int mode,
                          cudaStream_t st);

// ---------------------------------------------------------------- whitening
// t (m x r, row-major) = Q^T w for Q s x m (ld ldq) and w s x r (column-major);
// tpart: qt_dot_partial_doubles(mmax, r) doubles of scratch.
void qt_dot_launch(const double* Q, int64_t ldq, int64_t s, int m, const double* w, int r,
                   double* t, double* tpart, cudaStream_t st);
int qt_dot_partial_doubles(int mmax, int r);
void q_update_launch(const double* Q, int64_t ldq, int64_t s, int m, const double* t, int r,
                     const double* w_in, double* w_out, double* partial, int nchunk,
                     cudaStream_t st);
void ts_gram_launch(const double* w, int64_t s, int r, double* partial, int grid, cudaStream_t st);
void ts_scale_launch(double* w, int64_t s, int r, const double* Rinv, double* out,
                     int64_t ldo, cudaStream_t st);
int q_update_chunks(int m, int64_t s);
void t_write_launch(double* T, int64_t ldT, int m, int r, const double* t1, const double* t2,
                    const double* tau, cudaStream_t st);
// t[e] = sum over nchunk chunks of tpart[ch * count + e], chunks in order
void qt_finish_launch(const double* tpart, int64_t count, int nchunk, double* t, cudaStream_t st);
// w_out[i + c s] = w_in[i + c s] - sum_ch partial[(ch s + i) r + c]
void q_update_finish_launch(const double* w_in, double* w_out, const double* partial, int64_t s,
                            int r, int nchunk, cudaStream_t st);

// Whitening products on the tensor cores (k_qslice.cu): two int8 digit
// copies of Q (one byte per BF16 digit), appended as Q grows, and the two
// products from them.
struct QsGeom {
  int64_t s = 0;
  int mmax = 0;
  int MTA = 0, KTA = 0, MTB = 0, KTB = 0;   // tiles of the two copies
  size_t bytesA = 0, bytesB = 0;
};
QsGeom qs_geometry(int64_t s, int mmax);
int qs_chunks(int64_t K);                  // K ranges (partial sums) of a product
bool qs_enabled(int64_t s, int m);         // the tensor-core products pay off
void qs_append_launch(const double* Q, const QsGeom& g, int m, int r, uint8_t* QA, uint8_t* QB,
                      cudaStream_t st);
// t (m x r, row-major) = Q^T w; tpart: qs_chunks(s) * m * r doubles
void qs_qt_launch(const QsGeom& g, const uint8_t* QA, int m, const double* w, int r, double* t,
                  double* tpart, uint32_t* flags, cudaStream_t st);
// w_out = w_in - Q t; partial: qs_chunks(m) * s * r doubles
void qs_update_launch(const QsGeom& g, const uint8_t* QB, int m, const double* t, int r,
                      const double* w_in, double* w_out, double* partial, uint32_t* flags,
                      cudaStream_t st);

// ---------------------------------------------------------------- projected
// partial: border_chunks(mp) * mp * r doubles of scratch
int border_chunks(int mp);
void border_col_launch(double* Ht, int64_t ldH, int mp, int r, const double* T, int64_t ldT,
                       const double* hslots, int first_block, int nslots, const double* h_dd,
                       double* partial, cudaStream_t st);
void border_small_launch(double* Ht, int64_t ldH, int mp, int r, const double* T, int64_t ldT,
                         const double* h_sub, const double* h_dd, cudaStream_t st);
void border_correct_launch(double* Ht, int64_t ldH, int m, int r, const double* T, int64_t ldT,
                           const double* h_next, cudaStream_t st);
void rho_launch(const double* Y, int64_t ldY, int m, int r, const double* TU, int64_t ldTU,
                const double* TV, int64_t ldTV, const double* hU, const double* hV,
                const double* betaU, const double* betaV, int bound, double* out3,
                cudaStream_t st);
// Dense block Hessenberg H_d (m = d r, column-major, zeroed beforehand) from
// the stored coefficients hband ((k+1) r x r row-major slots per column).
void band_to_dense_launch(const double* hband, int k, int r, int d, double* H, int64_t ldH,
                          cudaStream_t st);
// out (r x r row-major) = A[row0 .. row0+r-1, col0 .. col0+r-1] (column-major A).
void sub_block_launch(const double* A, int64_t ld, int row0, int col0, int r, double* out,
                      cudaStream_t st);
// Row-major n x r FP64 block <-> r columns of a column-major matrix.
void block_to_cols_launch(const double* B, int64_t n, int r, double* V, int64_t ldv,
                          cudaStream_t st);
void cols_to_block_launch(const double* V, int64_t ldv, int64_t n, int r, double* B,
                          cudaStream_t st);
// Top r x r block of a column-major m x q factor from a row-major r x r beta.
void fill_factor_launch(double* L, int64_t ldL, int r, const double* beta, cudaStream_t st);

// ---------------------------------------------------------------- dense FP64
void gemm_f64(char ta, char tb, int M, int N, int K, double alpha, const double* A, int64_t lda,
              const double* B, int64_t ldb, double beta, double* C, int64_t ldc, cudaStream_t st,
              size_t reserve_smem = 0);
void copy_matrix_launch(const double* A, int64_t lda, double* B, int64_t ldb, int M, int N,
                        cudaStream_t st);
void set_zero_launch(double* A, int64_t count, cudaStream_t st);
struct GjeState {
  int32_t* ipiv;   // m
  double* cvec;    // 2 m
  double* scal;    // [0] log|det|, [2], [3] pivots (ping-pong)
  uint32_t* flags;
  double* panel = nullptr;   // m x 64 scratch (blocked path)
  double* bsave = nullptr;   // 64 x m scratch (blocked path)
  void* oz_work = nullptr;   // ozaki_work_bytes(m, m, nb): trailing updates on the tensor cores
  // one launch per panel (gje_persistent_ok): the published pivot columns
  // (nb x m), per-step records (4 nb: pivot row, pivot value, raw column at
  // the step's row, and in the fourth word the generation that releases the
  // record; zeroed per solve); `ready` (nb words, zeroed per solve) is not
  // read by the kernel any more, its presence selects the one-launch path
  double* cstore = nullptr;
  double* pstore = nullptr;
  uint32_t* ready = nullptr;
  // the panel's row exchanges as one gather: 4 nb + 1 ints (destination rows,
  // source rows, count)
  int32_t* perm = nullptr;
};
bool gje_persistent_ok(int m);
void gje_invert(double* A, int64_t lda, int m, GjeState gs, cudaStream_t st);
// The blocked inversion's pieces (m > 256 with panel/bsave scratch): for
// k0 = 0, nb, 2 nb, ...: gje_panel_launch (pivot sweeps of columns
// [k0, k0+nb)) then gje_update_launch (row exchanges and GEMM update of all
// other columns); finally gje_finish_launch (column permutation).
bool gje_blocked(int m, const GjeState& gs);
int gje_panel_width();
void gje_panel_launch(double* A, int64_t lda, int m, int k0, int nb, GjeState gs, cudaStream_t st);
void gje_update_launch(double* A, int64_t lda, int m, int k0, int nb, GjeState gs, cudaStream_t st);
void gje_finish_launch(double* A, int64_t lda, int m, GjeState gs, cudaStream_t st);
int sign_combine_grid(int m);
void sign_combine_launch(double* Hk, const double* Hinv, int64_t ld, int m, double c,
                         double* partial, int grid, cudaStream_t st);
void scale_matrix_launch(double* A, int64_t ld, int M, int N, double a, cudaStream_t st);
void trsm_upper_left_launch(const double* T, int64_t ldT, int m, double* X, int64_t ldX, int ncol,
                            cudaStream_t st);
void gaussian_fill_launch(double* A, int64_t count, uint64_t seed, cudaStream_t st);
// one-sided Jacobi on the columns of A (M x N, column-major), accumulating V (N x N)
void jacobi_round_launch(double* A, int64_t lda, int M, int N, double* V, int64_t ldv,
                         const int* pairs, int npairs, double* offmax, cudaStream_t st);
void col_norms_launch(const double* A, int64_t lda, int M, int N, double* out, cudaStream_t st);
// singular value selection: idx[0..ell) = columns by decreasing sigma with
// sigma > tol * sigma_max; f1 = sigma^{1/2}, f2 = sigma^{-1/2}; ell to *ell_out
void select_sv_launch(const double* sigma, int N, double tol, int* idx, double* f1, double* f2,
                      int* ell_out, cudaStream_t st);
// out[:, t] = A[:, idx[t]] * f[t]
void gather_cols_launch(const double* A, int64_t lda, int M, const int* idx, const double* f,
                        int ncols, double* out, int64_t ldo, cudaStream_t st);
// out[j] = column absolute sums of A (M x N, column-major)
void col_abs_sums_launch(const double* A, int64_t lda, int M, int N, double* out, cudaStream_t st);
// Spectral-radius estimates of nmat <= 4 matrices (m x m, column-major,
// leading dimension ld) by `steps` >= 2 power-iteration steps from a fixed
// start vector: out[q] (device) = ||M_q x|| with x the normalised iterate
// after steps - 1 products.  work: power_work_doubles(m) doubles.
size_t power_work_doubles(int m);
void power_radius_launch(const double* const* M, int nmat, int m, int64_t ld, int steps,
                         double* work, double* out, cudaStream_t st);
// out2_dev = {trace(A), trace(B)}, A and B m x m column-major.
void diag_sums_launch(const double* A, int64_t lda, const double* B, int64_t ldb, int m,
                      double* out2_dev, cudaStream_t st);
// ---------------------------------------------------------------- true residual
// Columns of a virtual n x wtot matrix P = [sgn0 P0, sgn1 P1, sgn2 P2], each
// part row-major n x w[q] (w[q] may be 0).
struct GramParts {
  const double* p[3] = {nullptr, nullptr, nullptr};
  int w[3] = {0, 0, 0};
  double sgn[3] = {1.0, 1.0, 1.0};
  int64_t n = 0;
  int wtot = 0;
};
// G = P^T P (wtot x wtot, column-major, both triangles) in double-double:
// G = Ghi + Glo.  tiles_dev: gram_dd_tiles(w) int2 from gram_dd_tile_list;
// work: gram_dd_work_doubles(n, w, sm_count) doubles.
int gram_dd_tiles(int w);
size_t gram_dd_work_doubles(int64_t n, int w, int sm_count);
void gram_dd_tile_list(int w, int2* host_tiles);
void gram_dd_launch(const GramParts& P, const int2* tiles_dev, int sm_count, double* work,
                    double* Ghi, double* Glo, cudaStream_t st);
// out2 = double-double sum_e (Ghi + Glo)_e (Hhi + Hlo)_e over count entries.
void trace_dd_launch(const double* Ghi, const double* Glo, const double* Hhi, const double* Hlo,
                     int64_t count, double* out2, cudaStream_t st);
// out3 = {sqrt(num), sqrt(den), sqrt(num / den)} of double-double squares.
void residual_finish_launch(const double* num2, const double* den2, double* out3,
                            cudaStream_t st);

// ---------------------------------------------------------------- tensor-core FP64 GEMM
// C = alpha op(A) op(B) + beta C (column-major FP64) on the tcgen05 tensor
// cores by error-free splitting into BF16 slices (k_ozaki.cu).  work:
// ozaki_work_bytes(M, N, K) bytes (16-byte aligned); a failed bounded wait
// sets kFlagTimeout in flags.  ozaki_enabled: sizes where it pays.
size_t ozaki_work_bytes(int M, int N, int K);
bool ozaki_enabled(int M, int N, int K);
void ozaki_gemm(char ta, char tb, int M, int N, int K, double alpha, const double* A, int64_t lda,
                const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* work,
                uint32_t* flags, cudaStream_t st);

// ---------------------------------------------------------------- split solve
// Largest number of eigenvalues off the open right half plane that the split
// solve of the projected equation handles (k_split.cu).
constexpr int kSplitMaxK = 16;
// out = alpha A + beta (I + gamma S) for m x m column-major A (may be null), S
void sign_affine_launch(const double* A, int64_t lda, double alpha, const double* S, int64_t lds,
                        double beta, double gamma, int m, double* out, int64_t ldo,
                        cudaStream_t st);
// complex Schur form A = U T U^H of a real k x k matrix (k <= kSplitMaxK)
void small_schur_launch(const double* A, int64_t lda, int k, double2* U, double2* T,
                        uint32_t* flags, cudaStream_t st);
void uh_times_launch(const double2* U, int k, const double* R, int64_t ldr, int64_t n,
                     double2* Rt, cudaStream_t st);
void row_rhs_launch(const double2* Rt, const double2* T, int k, int i, const double2* Zt,
                    int64_t n, double* rhs, cudaStream_t st);
void realify_shift_launch(const double* G, int64_t ldg, int n, const double2* T, int k, int i,
                          double* M, cudaStream_t st);
void store_row_launch(const double* x, int64_t n, int k, int i, double2* Zt, cudaStream_t st);
void u_times_real_launch(const double2* U, int k, const double2* Zt, int64_t n, double* Z,
                         cudaStream_t st);

// Measured FP64 FMA rate of the device in TFLOP/s (dependent-chain probe).
double fp64_fma_probe(int sm_count, double* scratch, cudaStream_t st);
// out_dev[0] = trace(A B), A p x q and B q x p column-major (ld p and q).
void trace_product_launch(const double* A, const double* B, int p, int q, double* out_dev,
                          cudaStream_t st);

}  // namespace spk
