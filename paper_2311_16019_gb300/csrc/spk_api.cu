// libspk C ABI: handle, workspace and the device-side driver of Algorithm 1
// (s-PKSM) of the paper.  Every arithmetic step runs in this library's
// kernels; the host only sequences launches, reads back the residual
// estimate at check iterations, and sizes buffers.
//
// One iteration d, for each side (A, U) and (B^T, V):
//   spmm + window dots -> reduce -> GS update + Gram -> Cholesky (R1)
//   -> scale + Gram -> Cholesky (R2) -> h_{d+1,d} = R2 R1 -> U_{d+1}
//   -> sketch S U_{d+1} -> whitening CGS2 against Q -> Cholesky QR (tau)
//   -> T column block -> bordering update of H~ (Section 5).
// At a check: sign-function solve of H~ Y + Y G~^T = E1 b1 b2^T E1^T (Eq. (3.4)),
// rho (Eq. (3.5)).  After the loop: SVD truncation of Y, W = T^{-1} Y_i,
// second Arnoldi sweep accumulating X1 = U_d W1, X2 = V_d W2.
#include "spk_internal.cuh"

#include <algorithm>
#include <thread>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <ctime>
#include <map>
#include <string>
#include <vector>

using namespace spk;

#include <atomic>
namespace spk {
static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {
template <typename Q>
int bounded_poll(Q query, double budget_s) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = query();
    if (e == cudaSuccess) return 0;
    if (e != cudaErrorNotReady) return 2;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el >= budget_s) return 1;
    if (el > 1e-3) {
      struct timespec ts{0, 50000};
      nanosleep(&ts, nullptr);
    }
  }
}
}  // namespace

int bounded_stream_wait(cudaStream_t st, double budget_s) {
  return bounded_poll([st]() { return cudaStreamQuery(st); }, budget_s);
}
int bounded_event_wait(cudaEvent_t ev, double budget_s) {
  return bounded_poll([ev]() { return cudaEventQuery(ev); }, budget_s);
}
}  // namespace spk

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Kernel families timed by the optional profiler (CUDA events recorded on
// the launching stream around each group of launches).
enum ProfFam {
  F_SPMM, F_UPDATE, F_SCALE, F_SKETCH, F_QTDOT, F_QUPDATE, F_TSQR, F_BORDER,
  F_GJE, F_GEMM, F_SIGNCOMB, F_RHO, F_TRUNC, F_TRSM, F_XACC, F_GJE_PANEL, F_GJE_UPDATE,
  F_SIGNSCALE, F_COUNT
};
static const char* kFamNames[F_COUNT] = {
  "spmm_dots", "gs_update", "cholqr_scale", "sketch_srht", "whiten_qt_dot", "whiten_q_update",
  "whiten_cholqr", "border_update", "gje_invert", "gemm_f64", "sign_combine", "rho", "truncate_svd",
  "trsm", "x_accumulate", "gje_panel_H", "gje_update_H", "sign_scaling"};

struct ProfAcc {
  double ms = 0, bytes = 0, flops = 0;
  int64_t launches = 0, groups = 0;
};

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> free_ev;
  struct Pending { int f; cudaEvent_t a, b; int64_t launches; double bytes, flops; };
  std::vector<Pending> pend;
  ProfAcc acc[F_COUNT];
  cudaEvent_t get() {
    if (free_ev.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      return e;
    }
    cudaEvent_t e = free_ev.back();
    free_ev.pop_back();
    return e;
  }
  void resolve() {
    for (auto& p : pend) {
      bounded_event_wait(p.b, kHostWaitSeconds);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, p.a, p.b);
      auto& a = acc[p.f];
      a.ms += ms;
      a.bytes += p.bytes;
      a.flops += p.flops;
      a.launches += p.launches;
      a.groups += 1;
      free_ev.push_back(p.a);
      free_ev.push_back(p.b);
    }
    pend.clear();
  }
  ~Profiler() {
    for (auto e : free_ev) cudaEventDestroy(e);
    for (auto& p : pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  }
};

struct spk_handle {
  int device = 0;
  int sm_count = 152;
  std::string err;
  std::map<std::string, Buf> bufs;
  uint32_t* flags = nullptr;
  double host_wait_s = 600.0;
  Profiler prof;
  // second stream and fork/join events: the two inversions of a sign step
  // run concurrently (each one's latency-bound panel sweeps overlap the
  // other's GEMM updates)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // set by the sign iteration when it fails because of the spectrum (an
  // eigenvalue off the open right half plane, or no convergence)
  bool spectrum_bad = false;
  // set with spectrum_bad when the iteration converged and the traces of
  // sign(H), sign(G) counted neg_h, neg_g eigenvalues with negative real
  // part (the iterates then hold sign(H) and sign(G))
  bool trace_fail = false;
  int neg_h = 0, neg_g = 0;
  // dense products of the projected solve on the tensor cores (error-free
  // BF16 splitting) where the sizes pay; off: the FP64 CUDA-core GEMM
  bool tensor_gemm = true;
  // batched form: worker handles, each with its own stream and workspace
  struct Worker {
    spk_handle* h = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
  };
  std::vector<Worker> workers;
};

namespace {
// RAII timing of one group of launches of one family.  `bytes` and `flops`
// are the group's algorithmic traffic and work; the launch count is taken
// from the library's launch counter over the scope.
struct ProfScope {
  spk_handle* h;
  int f;
  cudaStream_t st;
  int64_t l0;
  double bytes, flops;
  cudaEvent_t a = nullptr;
  ProfScope(spk_handle* h_, int f_, cudaStream_t st_, double by, double fl)
      : h(h_), f(f_), st(st_), l0(launch_count()), bytes(by), flops(fl) {
    if (h->prof.on) {
      a = h->prof.get();
      cudaEventRecord(a, st);
    }
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = h->prof.get();
    cudaEventRecord(b, st);
    h->prof.pend.push_back({f, a, b, launch_count() - l0, bytes, flops});
    if (h->prof.pend.size() > 8192) h->prof.resolve();
  }
};
}  // namespace

namespace {

int fail(spk_handle* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(h, SPK_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                    \
  } while (0)

#define TRY(expr)            \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != SPK_OK) return rc_; \
  } while (0)

void* ws_get(spk_handle* h, const std::string& name, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  Buf& b = h->bufs[name];
  if (b.bytes >= bytes) return b.p;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return nullptr;
  }
  b.bytes = bytes;
  return b.p;
}

#define WS(var, type, name, count)                                                           \
  type* var = static_cast<type*>(ws_get(h, name, sizeof(type) * (size_t)(count)));           \
  if (!var) return fail(h, SPK_ERR_ALLOC, "cannot allocate %s (%zu bytes)", name,            \
                        sizeof(type) * (size_t)(count));

// Bounded wait on a stream: poll with a wall-clock budget (never blocks forever).
int wait_stream(spk_handle* h, cudaStream_t st, double budget_s) {
  if (budget_s <= 0.0) {
    // zero budget (fault injection): report the expired wait; queued work
    // completes in stream order and the context stays usable
    (void)cudaStreamQuery(st);
    return fail(h, SPK_ERR_TIMEOUT, "bounded wait with a zero budget expired");
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) return SPK_OK;
    if (e != cudaErrorNotReady)
      return fail(h, SPK_ERR_CUDA, "stream error: %s", cudaGetErrorString(e));
    const double el =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el >= budget_s) return fail(h, SPK_ERR_TIMEOUT, "device work did not finish in %.1f s", budget_s);
    if (el > 1e-3) {
      struct timespec ts{0, 50000};
      nanosleep(&ts, nullptr);
    }
  }
}

// Device-to-host read into pageable host memory.  Such a copy blocks the
// calling thread until the work queued before it on the stream has finished,
// with no limit, so the stream is first drained by the bounded wait; the
// copy then starts at once, and a second bounded wait covers the copy.
int d2h(spk_handle* h, void* dst, const void* src, size_t bytes, cudaStream_t st,
        double budget_s) {
  TRY(wait_stream(h, st, budget_s));
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
  return wait_stream(h, st, budget_s);
}
int d2h(spk_handle* h, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  return d2h(h, dst, src, bytes, st, h->host_wait_s);
}

int read_flags(spk_handle* h, cudaStream_t st, uint32_t* out) {
  return d2h(h, out, h->flags, sizeof(uint32_t), st);
}

int flags_to_status(spk_handle* h, uint32_t f) {
  if (f & kFlagTimeout)
    return fail(h, SPK_ERR_TIMEOUT, "a bounded device-side wait expired (a kernel gave up)");
  if (f & kFlagNonfinite) return fail(h, SPK_ERR_NONFINITE, "non-finite value in a reduction");
  if (f & kFlagBreakdown)
    return fail(h, SPK_ERR_BREAKDOWN, "rank-deficient block in a Cholesky QR (Gram pivot <= 1e-14 trace)");
  if (f & kFlagZeroPivot)
    return fail(h, SPK_ERR_SINGULAR_PROJECTED, "zero pivot in the projected-matrix inversion");
  return SPK_OK;
}

// A new block whose Gram matrix has a Cholesky pivot below 1e-14 of its
// trace (condition number above ~1e7) is reported as a breakdown.
constexpr double kBreakdownFloor = 1e-14;

// Row kernels with per-CTA partial sums: two CTAs of 256 threads per SM, so
// that each thread covers several rows before its block reduction (the
// reduction's FP64 additions, per row, shrink in proportion).
int grid_rows(spk_handle* h, int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)h->sm_count * 2));
}

// Double-double Gram matrix of the virtual matrix P (see k_residual.cu) into
// the named workspace buffers <tag>hi, <tag>lo (w x w each).
int gram_dd(spk_handle* h, const GramParts& P, const std::string& tag, double** hi, double** lo,
            cudaStream_t st) {
  const int w = P.wtot;
  const int nt = gram_dd_tiles(w);
  WS(tiles, int2, (tag + "tiles").c_str(), nt);
  WS(work, double, "rs_work", gram_dd_work_doubles(P.n, w, h->sm_count));
  WS(Ghi, double, (tag + "hi").c_str(), (size_t)w * w);
  WS(Glo, double, (tag + "lo").c_str(), (size_t)w * w);
  std::vector<int2> ht(nt);
  gram_dd_tile_list(w, ht.data());
  CK(cudaMemcpyAsync(tiles, ht.data(), sizeof(int2) * nt, cudaMemcpyHostToDevice, st));
  gram_dd_launch(P, tiles, h->sm_count, work, Ghi, Glo, st);
  // the host tile list must outlive the copy
  TRY(wait_stream(h, st, h->host_wait_s));
  *hi = Ghi;
  *lo = Glo;
  return SPK_OK;
}

// ||A X + X B - C1 C2^T||_F and ||C1 C2^T||_F for X = X1 X2^T (ell columns;
// BT = B^T generates the right space), in the factored form
// [A X1, X1, -C1] [X2, B^T X2, C2]^T with double-double Gram matrices
// (k_residual.cu).  out3 (host) = {||R||_F, ||C1 C2^T||_F, ratio}.
int true_residual(spk_handle* h, const spk_csr* A, const spk_csr* BT, const double* C1,
                  const double* C2, int r, const double* X1, const double* X2, int ell,
                  cudaStream_t st, double out3[3]) {
  const int64_t n1 = A->nrows, n2 = BT->nrows;
  WS(AX1, double, "rs_AX1", (size_t)n1 * std::max(ell, 1));
  WS(BX2, double, "rs_BX2", (size_t)n2 * std::max(ell, 1));
  WS(sc, double, "rs_scalars", 8);
  if (ell > 0) {
    spmm_wide_launch(A->rowptr_dev, A->col_dev, A->val_dev, n1, ell, X1, AX1, st);
    spmm_wide_launch(BT->rowptr_dev, BT->col_dev, BT->val_dev, n2, ell, X2, BX2, st);
  }
  GramParts L, M, c1, c2;
  L.n = n1;
  L.p[0] = AX1; L.w[0] = ell;
  L.p[1] = X1; L.w[1] = ell;
  L.p[2] = C1; L.w[2] = r; L.sgn[2] = -1.0;
  L.wtot = 2 * ell + r;
  M.n = n2;
  M.p[0] = X2; M.w[0] = ell;
  M.p[1] = BX2; M.w[1] = ell;
  M.p[2] = C2; M.w[2] = r;
  M.wtot = 2 * ell + r;
  c1.n = n1; c1.p[0] = C1; c1.w[0] = r; c1.wtot = r;
  c2.n = n2; c2.p[0] = C2; c2.w[0] = r; c2.wtot = r;
  double *Lh, *Ll, *Mh, *Ml, *c1h, *c1l, *c2h, *c2l;
  TRY(gram_dd(h, L, "rs_GL", &Lh, &Ll, st));
  TRY(gram_dd(h, M, "rs_GM", &Mh, &Ml, st));
  TRY(gram_dd(h, c1, "rs_GC1", &c1h, &c1l, st));
  TRY(gram_dd(h, c2, "rs_GC2", &c2h, &c2l, st));
  const int64_t w = L.wtot;
  trace_dd_launch(Lh, Ll, Mh, Ml, w * w, sc, st);
  trace_dd_launch(c1h, c1l, c2h, c2l, (int64_t)r * r, sc + 2, st);
  residual_finish_launch(sc, sc + 2, sc + 4, st);
  CK(cudaGetLastError());
  TRY(d2h(h, out3, sc + 4, 3 * sizeof(double), st));
  return SPK_OK;
}

// --------------------------------------------------------------------------
// Small dense Sylvester solve H Y + Y G^T = F by the scaled Newton iteration
// for the matrix sign function of Z = [[H, -F], [0, -G^T]] (Roberts):
//   H <- (c H + H^{-1}/c)/2,  G <- (c G + G^{-1}/c)/2,
//   F <- (c F + H^{-1} F G^{-T} / c)/2,    Y = F_inf / 2,
// with one scalar c for the whole of Z while the iterates still change by
// more than 1e-2, c = 1 afterwards.  c is the spectral scaling of Kenney and
// Laub, c = (|lambda|_min |lambda|_max)^{-1/2} over the eigenvalues of H and
// G together, with the two moduli estimated by power iteration on H, G,
// H^{-1} and G^{-1} (kPowerSteps products each; an error of a few percent
// in c costs nothing measurable); if an estimate is not finite and positive,
// the 1-norm scaling c = (||H^{-1}||_1 ||G^{-1}||_1 / (||H||_1 ||G||_1))^{1/4}.
// Quadratic convergence: once an update changes H and G by less than 1e-8
// (relative Frobenius), the next error is below 1e-16 and the loop stops.
// Requires the spectra of H and G in the open right half plane (true for
// the convection-diffusion operators here); a zero pivot is reported.
// In: Hk, Gk, F (m x m, ld m, overwritten); out: F holds Y.
//
// Low-rank right-hand side (Lf != nullptr): F_0 = L_0 R_0^T with q0 columns
// (the projected equation's right-hand side E_1 beta_1 beta_2^T E_1^T has
// rank r), and the input F is not read.  The F update then keeps factors,
//   L <- [sqrt(c/2) L, H^{-1} L / sqrt(2c)],  R <- [sqrt(c/2) R, G^{-1} R / sqrt(2c)],
// which doubles the column count per step at 4 m^2 q flops instead of the
// 8 m^3 of the two dense products; once 2q would pass qcap (the factors'
// capacity) the product is formed and the iteration continues densely.
constexpr int kPowerSteps = 10;

// Adaptive check schedule.  Doubling warm-up (checks at p, 2p, 4p, ...)
// until log(rho) has decreased over two checks.  Then the step to the next
// check is kCheckStepFraction times the iterations that the straight line
// through the last two log(rho) values needs to reach tol (+5%), rounded up
// to a multiple of p.  log(rho) steepens as d grows (the convergence is
// superlinear), so the line through two checks overestimates what is left;
// a check costs a chain of O(d r) dependent launches plus O((d r)^3) flops,
// so it pays to check a little early rather than add more checks.
// hd[0..count): the checked iterations, hrel: their relative estimates.
constexpr double kCheckStepFraction = 0.7;

int next_check_adaptive(const int32_t* hd, const double* hrel, int count, double tol, int p,
                        int dmax) {
  const int d = hd[count - 1];
  int64_t nxt = 2 * (int64_t)d;
  if (count >= 3 && hrel[count - 1] < hrel[count - 2] && hrel[count - 2] < hrel[count - 3] &&
      hrel[count - 1] > 0 && hd[count - 1] > hd[count - 2]) {
    const double slope = (std::log(hrel[count - 1]) - std::log(hrel[count - 2])) /
                         (double)(hd[count - 1] - hd[count - 2]);
    if (slope < 0) {
      const double need = (std::log(tol) - std::log(hrel[count - 1])) / slope * 1.05;
      double step = std::min(kCheckStepFraction * need, 1e9);
      if (!(step >= 0.0)) step = 0.0;
      int64_t pred = d + (int64_t)std::ceil(step);
      pred = ((pred + p - 1) / p) * p;
      nxt = std::max<int64_t>(pred, (int64_t)d + p);
    }
  }
  return (int)std::max<int64_t>((int64_t)d + 1, std::min<int64_t>(nxt, dmax));
}

int sign_solve(spk_handle* h, int m, double* Hk, double* Gk, double* F, int max_newton,
               cudaStream_t st, int* iters_out, double* Lf = nullptr, double* Rf = nullptr,
               int q0 = 0, int qcap = 0) {
  bool fact = Lf != nullptr && Rf != nullptr && q0 > 0;
  int q = q0;
  WS(Hinv, double, "sg_Hinv", (size_t)m * m);
  WS(Ginv, double, "sg_Ginv", (size_t)m * m);
  WS(P, double, "sg_P", (size_t)m * m);
  WS(ipiv, int32_t, "sg_ipiv", m);
  WS(cvec, double, "sg_cvec", 2 * (size_t)m);
  WS(ipivG, int32_t, "sg_ipivG", m);
  WS(cvecG, double, "sg_cvecG", 2 * (size_t)m);
  WS(scalH, double, "sg_scalH", 8);
  WS(scalG, double, "sg_scalG", 8);
  WS(cs, double, "sg_colsums", 4 * (size_t)m + 4);
  WS(pwork, double, "sg_power", power_work_doubles(m));
  WS(gpanel, double, "sg_panel", (size_t)m * gje_panel_width());
  WS(gbsave, double, "sg_bsave", (size_t)m * gje_panel_width());
  WS(gpanelG, double, "sg_panelG", (size_t)m * gje_panel_width());
  WS(gbsaveG, double, "sg_bsaveG", (size_t)m * gje_panel_width());
  const int sgrid = sign_combine_grid(m);
  WS(part, double, "sg_part", 4 * (size_t)sgrid);
  // tensor-core products (error-free BF16 splitting): the two inversions'
  // trailing updates and the right-hand side updates
  const bool oz = h->tensor_gemm && ozaki_enabled(m, m, gje_panel_width());
  void *ozH = nullptr, *ozG = nullptr, *ozF = nullptr;
  if (oz) {
    ozH = ws_get(h, "sg_ozH", ozaki_work_bytes(m, m, gje_panel_width()));
    ozG = ws_get(h, "sg_ozG", ozaki_work_bytes(m, m, gje_panel_width()));
    ozF = ws_get(h, "sg_ozF", ozaki_work_bytes(m, m, m));
    if (!ozH || !ozG || !ozF) return fail(h, SPK_ERR_ALLOC, "cannot allocate tensor-core GEMM work");
  }
  // one launch per Gauss-Jordan panel: published pivot columns, pivot values
  // and ready flags for each of the two concurrent inversions
  const int nbw = gje_panel_width();
  double *cstH = nullptr, *cstG = nullptr, *pstH = nullptr, *pstG = nullptr;
  uint32_t *rdyH = nullptr, *rdyG = nullptr;
  if (gje_persistent_ok(m)) {
    cstH = static_cast<double*>(ws_get(h, "sg_cstH", sizeof(double) * (size_t)m * nbw));
    cstG = static_cast<double*>(ws_get(h, "sg_cstG", sizeof(double) * (size_t)m * nbw));
    pstH = static_cast<double*>(ws_get(h, "sg_pstH", sizeof(double) * 4 * nbw));
    pstG = static_cast<double*>(ws_get(h, "sg_pstG", sizeof(double) * 4 * nbw));
    rdyH = static_cast<uint32_t*>(ws_get(h, "sg_rdyH", sizeof(uint32_t) * nbw));
    rdyG = static_cast<uint32_t*>(ws_get(h, "sg_rdyG", sizeof(uint32_t) * nbw));
    if (!cstH || !cstG || !pstH || !pstG || !rdyH || !rdyG)
      return fail(h, SPK_ERR_ALLOC, "cannot allocate Gauss-Jordan panel work");
    CK(cudaMemsetAsync(rdyH, 0, sizeof(uint32_t) * nbw, st));
    CK(cudaMemsetAsync(rdyG, 0, sizeof(uint32_t) * nbw, st));
    CK(cudaMemsetAsync(pstH, 0, sizeof(double) * 4 * nbw, st));
    CK(cudaMemsetAsync(pstG, 0, sizeof(double) * 4 * nbw, st));
  }
  WS(permH, int32_t, "sg_permH", 4 * (size_t)nbw + 1);
  WS(permG, int32_t, "sg_permG", 4 * (size_t)nbw + 1);
  auto gemm = [&](char ta, char tb, int M, int N, int K, double alpha, const double* A, int64_t lda,
                  const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                  cudaStream_t s_) {
    if (oz && ozaki_enabled(M, N, K))
      ozaki_gemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ozF, h->flags, s_);
    else
      gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s_);
  };
  std::vector<double> hpart(4 * (size_t)sgrid), hcs(4 * (size_t)m + 4);
  double delta_prev = 1e300;
  bool converged = false;
  int it = 0;
  for (it = 0; it < max_newton; ++it) {
    CK(cudaMemcpyAsync(Hinv, Hk, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(Ginv, Gk, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, st));
    {
      const double mm2 = (double)m * m;
      ProfScope ps(h, F_GJE, st, 2 * 16.0 * mm2, 2 * 2.0 * mm2 * m);
      GjeState gh{ipiv, cvec, scalH, h->flags, gpanel, gbsave, ozH, cstH, pstH, rdyH, permH};
      GjeState gg{ipivG, cvecG, scalG, h->flags, gpanelG, gbsaveG, ozG, cstG, pstG, rdyG, permG};
      CK(cudaEventRecord(h->ev_fork, st));
      CK(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
      if (gje_blocked(m, gh)) {
        // the two blocked inversions interleaved panel by panel; the
        // sub-families time the H inversion's own stream
        const int nbw = gje_panel_width();
        for (int k0 = 0; k0 < m; k0 += nbw) {
          const int nb = std::min(nbw, m - k0);
          {
            ProfScope pp(h, F_GJE_PANEL, st, 16.0 * m * nb, 2.0 * m * nb * nb);
            gje_panel_launch(Hinv, m, m, k0, nb, gh, st);
          }
          gje_panel_launch(Ginv, m, m, k0, nb, gg, h->aux);
          {
            ProfScope pu(h, F_GJE_UPDATE, st, 8.0 * (2.0 * m * m + 2.0 * m * nb),
                         2.0 * m * m * nb);
            gje_update_launch(Hinv, m, m, k0, nb, gh, st);
          }
          gje_update_launch(Ginv, m, m, k0, nb, gg, h->aux);
        }
        gje_finish_launch(Hinv, m, m, gh, st);
        gje_finish_launch(Ginv, m, m, gg, h->aux);
      } else {
        gje_invert(Hinv, m, m, gh, st);
        gje_invert(Ginv, m, m, gg, h->aux);
      }
      CK(cudaEventRecord(h->ev_join, h->aux));
      CK(cudaStreamWaitEvent(st, h->ev_join, 0));
    }
    double c = 1.0;
    const bool scale = delta_prev > 1e-2;
    if (scale) {
      col_abs_sums_launch(Hk, m, m, m, cs, st);
      col_abs_sums_launch(Hinv, m, m, m, cs + m, st);
      col_abs_sums_launch(Gk, m, m, m, cs + 2 * m, st);
      col_abs_sums_launch(Ginv, m, m, m, cs + 3 * m, st);
      {
        const double mm2 = (double)m * m;
        ProfScope ps(h, F_SIGNSCALE, st, kPowerSteps * 4 * 8.0 * mm2, kPowerSteps * 4 * 2.0 * mm2);
        const double* mats[4] = {Hk, Gk, Hinv, Ginv};
        power_radius_launch(mats, 4, m, m, kPowerSteps, pwork, cs + 4 * m, st);
      }
      TRY(d2h(h, hcs.data(), cs, sizeof(double) * (4 * m + 4), st));
    }
    TRY(wait_stream(h, st, h->host_wait_s));
    CK(cudaGetLastError());
    uint32_t f = 0;
    TRY(read_flags(h, st, &f));
    if (f & kFlagTimeout) {
      *iters_out = it;
      return fail(h, SPK_ERR_TIMEOUT, "a bounded device-side wait expired in sign iteration %d "
                  "(m=%d)", it, m);
    }
    if (f & kFlagZeroPivot) {
      *iters_out = it;
      return fail(h, SPK_ERR_SINGULAR_PROJECTED, "zero pivot in sign iteration %d (m=%d)", it, m);
    }
    if (scale) {
      // rad: estimates of rho(H), rho(G), rho(H^{-1}), rho(G^{-1})
      const double* rad = hcs.data() + 4 * (size_t)m;
      c = std::sqrt(std::max(rad[2], rad[3]) / std::max(rad[0], rad[1]));
      if (!std::isfinite(c) || c <= 0.0) {
        double n1[4] = {0, 0, 0, 0};
        for (int q = 0; q < 4; ++q)
          for (int j = 0; j < m; ++j) n1[q] = std::max(n1[q], hcs[(size_t)q * m + j]);
        c = std::pow((n1[1] * n1[3]) / (n1[0] * n1[2]), 0.25);
      }
      if (!std::isfinite(c) || c <= 0.0) c = 1.0;
    }
    if (fact && 2 * q > qcap) {
      // the factors would outgrow their capacity: F = L R^T from here on
      const double mm2 = (double)m * m;
      ProfScope ps(h, F_GEMM, st, 8.0 * (mm2 + 2.0 * m * q), 2.0 * mm2 * q);
      gemm('N', 'T', m, m, q, 1.0, Lf, m, Rf, m, 0.0, F, m, st);
      fact = false;
    }
    if (fact) {
      const double mm2 = (double)m * m;
      ProfScope ps(h, F_GEMM, st, 2 * 8.0 * (mm2 + 3.0 * m * q), 2 * 2.0 * mm2 * q);
      const double a_new = 1.0 / std::sqrt(2.0 * c), a_old = std::sqrt(0.5 * c);
      gemm('N', 'N', m, q, m, a_new, Hinv, m, Lf, m, 0.0, Lf + (size_t)q * m, m, st);
      gemm('N', 'N', m, q, m, a_new, Ginv, m, Rf, m, 0.0, Rf + (size_t)q * m, m, st);
      scale_matrix_launch(Lf, m, m, q, a_old, st);
      scale_matrix_launch(Rf, m, m, q, a_old, st);
      q *= 2;
    } else {
      // F <- (c/2) F + (1/(2c)) (H^{-1} F) G^{-T}
      const double mm2 = (double)m * m;
      ProfScope ps(h, F_GEMM, st, 7 * 8.0 * mm2, 4.0 * mm2 * m);
      gemm('N', 'N', m, m, m, 1.0, Hinv, m, F, m, 0.0, P, m, st);
      gemm('N', 'T', m, m, m, 0.5 / c, P, m, Ginv, m, 0.5 * c, F, m, st);
    }
    {
      const double mm2 = (double)m * m;
      ProfScope ps(h, F_SIGNCOMB, st, 2 * 3 * 8.0 * mm2, 2 * 3.0 * mm2);
      sign_combine_launch(Hk, Hinv, m, m, c, part, sgrid, st);
      sign_combine_launch(Gk, Ginv, m, m, c, part + 2 * sgrid, sgrid, st);
    }
    TRY(d2h(h, hpart.data(), part, sizeof(double) * 4 * sgrid, st));
    double dH = 0, nH = 0, dG = 0, nG = 0;
    for (int b = 0; b < sgrid; ++b) {
      dH += hpart[2 * b];
      nH += hpart[2 * b + 1];
      dG += hpart[2 * sgrid + 2 * b];
      nG += hpart[2 * sgrid + 2 * b + 1];
    }
    const double delta = std::sqrt(dH / std::max(nH, 1e-300)) + std::sqrt(dG / std::max(nG, 1e-300));
    if (!std::isfinite(delta)) {
      *iters_out = it + 1;
      return fail(h, SPK_ERR_NONFINITE, "non-finite sign iteration (m=%d)", m);
    }
    if (delta < 1e-8) {
      ++it;
      converged = true;
      break;
    }
    delta_prev = delta;
  }
  *iters_out = it;
  if (!converged) {
    h->spectrum_bad = true;
    return fail(h, SPK_ERR_SINGULAR_PROJECTED,
                "sign iteration did not converge in %d steps (m=%d)", max_newton, m);
  }
  // The iterates converge to sign(H) and sign(G), which are the identity
  // only if every eigenvalue lies in the open right half plane; otherwise
  // the limit of F is not 2Y.  trace(sign(H)) = m - 2 (#eigenvalues with
  // negative real part).
  {
    double tr[2] = {0.0, 0.0};
    diag_sums_launch(Hk, m, Gk, m, m, part, st);
    TRY(d2h(h, tr, part, sizeof tr, st));
    const int negH = (int)std::lround((m - tr[0]) / 2.0), negG = (int)std::lround((m - tr[1]) / 2.0);
    if (negH != 0 || negG != 0) {
      h->spectrum_bad = true;
      h->trace_fail = true;
      h->neg_h = negH;
      h->neg_g = negG;
      return fail(h, SPK_ERR_SINGULAR_PROJECTED,
                  "projected matrices have %d and %d eigenvalues off the open right half plane "
                  "(m=%d): the sign iteration does not apply",
                  negH, negG, m);
    }
  }
  if (fact) {
    const double mm2 = (double)m * m;
    ProfScope ps(h, F_GEMM, st, 8.0 * (mm2 + 2.0 * m * q), 2.0 * mm2 * q);
    gemm('N', 'T', m, m, q, 0.5, Lf, m, Rf, m, 0.0, F, m, st);
  } else {
    scale_matrix_launch(F, m, m, m, 0.5, st);
  }
  return SPK_OK;
}

int jacobi_svd(spk_handle* h, double* A, int64_t lda, int M, int N, double* V, cudaStream_t st);

int max_col_abs_sum(spk_handle* h, const double* A, int64_t lda, int m, cudaStream_t st,
                    double* out) {
  WS(cs, double, "sp_colsum", m);
  col_abs_sums_launch(A, lda, m, m, cs, st);
  std::vector<double> hc(m);
  TRY(d2h(h, hc.data(), cs, sizeof(double) * m, st));
  double mx = 0.0;
  for (double v : hc) mx = std::max(mx, v);
  *out = mx;
  return SPK_OK;
}

// The part of the solution of A X + X B^T = R0 that lies in the invariant
// subspace of A's kA eigenvalues with negative real part: X = P_A- X with
// A X + X B^T = P_A- R0, P_A- = (I - S_A)/2 the spectral projector from
// S_A = sign(A).  With W an orthonormal basis of range(P_A-) (range finder
// on P_A- and one-sided Jacobi), A W = W L with L = W^T A W (kA x kA), and
// X = W Z where L Z + Z B^T = V^T R0, V^T = W^T P_A-.  The small equation is
// solved through the complex Schur form L = U T U^H: row i of Zt = U^H Z
// (from the last) solves (B + t_ii I) z^T = (Rt_i - sum_{j>i} t_ij Zt_j)^T,
// a real 2m x 2m system inverted by Gauss-Jordan; Z = Re(U Zt).  Adds X (or
// X^T when transpose) to out (m x m, column-major).
int minus_block(spk_handle* h, int m, const double* A, int64_t lda, const double* B, int64_t ldb,
                const double* SA, int64_t lds, int kA, const double* R0, bool transpose,
                double* out, uint64_t seed, cudaStream_t st) {
  const int q = std::min(m, kA + 4);
  WS(Om, double, "sp_Om", (size_t)m * q);
  WS(Z0, double, "sp_Z0", (size_t)m * q);
  WS(nrm, double, "sp_nrm", q);
  WS(idx, int, "sp_idx", q);
  WS(fac, double, "sp_fac", q);
  WS(W, double, "sp_W", (size_t)m * kA);
  WS(AW, double, "sp_AW", (size_t)m * kA);
  WS(L, double, "sp_L", (size_t)kA * kA);
  WS(Vt, double, "sp_Vt", (size_t)m * kA);
  WS(R, double, "sp_R", (size_t)kA * m);
  WS(U, double2, "sp_U", (size_t)kA * kA);
  WS(T, double2, "sp_T", (size_t)kA * kA);
  WS(Rt, double2, "sp_Rt", (size_t)kA * m);
  WS(Zt, double2, "sp_Zt", (size_t)kA * m);
  WS(Z, double, "sp_Zr", (size_t)kA * m);
  WS(rhs, double, "sp_rhs", 2 * (size_t)m);
  WS(x, double, "sp_x", 2 * (size_t)m);
  const int m2 = 2 * m;
  WS(M, double, "sp_M", (size_t)m2 * m2);
  WS(ipiv, int32_t, "sp_ipiv", m2);
  WS(cvec, double, "sp_cvec", 2 * (size_t)m2);
  WS(scal, double, "sp_scal", 8);
  WS(gpanel, double, "sp_panel", (size_t)m2 * gje_panel_width());
  WS(gbsave, double, "sp_bsave", (size_t)m2 * gje_panel_width());
  // range of P_A-: Z0 = (Om - S_A Om) / 2, orthogonal columns by Jacobi
  gaussian_fill_launch(Om, (int64_t)m * q, seed, st);
  copy_matrix_launch(Om, m, Z0, m, m, q, st);
  gemm_f64('N', 'N', m, q, m, -0.5, SA, lds, Om, m, 0.5, Z0, m, st);
  TRY(jacobi_svd(h, Z0, m, m, q, nullptr, st));
  col_norms_launch(Z0, m, m, q, nrm, st);
  std::vector<double> hn(q);
  TRY(d2h(h, hn.data(), nrm, sizeof(double) * q, st));
  std::vector<int> order(q);
  for (int j = 0; j < q; ++j) order[j] = j;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return hn[a] > hn[b]; });
  // the projector has rank kA: a clear gap after the kA-th singular value
  if (!(hn[order[kA - 1]] > 0.0) || (q > kA && hn[order[kA]] > 1e-6 * hn[order[kA - 1]]))
    return fail(h, SPK_ERR_SINGULAR_PROJECTED,
                "split solve: the spectral projector's numerical rank is not %d", kA);
  std::vector<int> hidx(kA);
  std::vector<double> hf(kA);
  for (int t = 0; t < kA; ++t) {
    hidx[t] = order[t];
    hf[t] = 1.0 / hn[order[t]];
  }
  CK(cudaMemcpyAsync(idx, hidx.data(), sizeof(int) * kA, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(fac, hf.data(), sizeof(double) * kA, cudaMemcpyHostToDevice, st));
  gather_cols_launch(Z0, m, m, idx, fac, kA, W, m, st);
  // L = W^T A W, V = P_A-^T W = (W - S_A^T W) / 2, R = V^T R0
  gemm_f64('N', 'N', m, kA, m, 1.0, A, lda, W, m, 0.0, AW, m, st);
  gemm_f64('T', 'N', kA, kA, m, 1.0, W, m, AW, m, 0.0, L, kA, st);
  copy_matrix_launch(W, m, Vt, m, m, kA, st);
  gemm_f64('T', 'N', m, kA, m, -0.5, SA, lds, W, m, 0.5, Vt, m, st);
  gemm_f64('T', 'N', kA, m, m, 1.0, Vt, m, R0, m, 0.0, R, kA, st);
  small_schur_launch(L, kA, kA, U, T, h->flags, st);
  uh_times_launch(U, kA, R, kA, m, Rt, st);
  // host copies kept alive until the stream is drained below
  TRY(wait_stream(h, st, h->host_wait_s));
  // the shifts t_ii: a real one (the usual case: a real eigenvalue off the
  // half plane) needs only the m x m inverse of B + t I, applied to the real
  // and imaginary parts of the right-hand side alike
  std::vector<double2> tdiag(kA);
  for (int i = 0; i < kA; ++i)
    TRY(d2h(h, &tdiag[i], T + (size_t)i * kA + i, sizeof(double2), st));
  // the inversions' trailing updates on the tensor cores, one launch per panel
  const int nbw = gje_panel_width();
  GjeState gs{ipiv, cvec, scal, h->flags, gpanel, gbsave};
  if (h->tensor_gemm && ozaki_enabled(m, m, nbw)) {
    gs.oz_work = ws_get(h, "sp_oz", ozaki_work_bytes(m2, m2, nbw));
    if (!gs.oz_work) return fail(h, SPK_ERR_ALLOC, "cannot allocate split-solve GEMM work");
  }
  if (gje_persistent_ok(m2)) {
    gs.cstore = static_cast<double*>(ws_get(h, "sp_cst", sizeof(double) * (size_t)m2 * nbw));
    gs.pstore = static_cast<double*>(ws_get(h, "sp_pst", sizeof(double) * 4 * nbw));
    gs.ready = static_cast<uint32_t*>(ws_get(h, "sp_rdy", sizeof(uint32_t) * nbw));
    gs.perm = static_cast<int32_t*>(ws_get(h, "sp_perm", sizeof(int32_t) * (4 * nbw + 1)));
    if (!gs.cstore || !gs.pstore || !gs.ready || !gs.perm)
      return fail(h, SPK_ERR_ALLOC, "cannot allocate split-solve panel work");
    CK(cudaMemsetAsync(gs.ready, 0, sizeof(uint32_t) * nbw, st));
    CK(cudaMemsetAsync(gs.pstore, 0, sizeof(double) * 4 * nbw, st));
  }
  for (int i = kA - 1; i >= 0; --i) {
    row_rhs_launch(Rt, T, kA, i, Zt, m, rhs, st);
    const double2 t = tdiag[i];
    if (std::fabs(t.y) <= 1e-13 * std::max(1.0, std::hypot(t.x, t.y))) {
      // M = B + Re(t) I (m x m); x = M^{-1} [rhs_re, rhs_im]
      sign_affine_launch(B, ldb, 1.0, B, ldb, t.x, 0.0, m, M, m, st);
      gje_invert(M, m, m, gs, st);
      gemm_f64('N', 'N', m, 2, m, 1.0, M, m, rhs, m, 0.0, x, m, st);
    } else {
      realify_shift_launch(B, ldb, m, T, kA, i, M, st);
      gje_invert(M, m2, m2, gs, st);
      gemm_f64('N', 'N', m2, 1, m2, 1.0, M, m2, rhs, m2, 0.0, x, m2, st);
    }
    store_row_launch(x, m, kA, i, Zt, st);
  }
  u_times_real_launch(U, kA, Zt, m, Z, st);
  if (!transpose)
    gemm_f64('N', 'N', m, m, kA, 1.0, W, m, Z, kA, 1.0, out, m, st);
  else
    gemm_f64('T', 'T', m, m, kA, 1.0, Z, kA, W, m, 1.0, out, m, st);
  uint32_t f = 0;
  TRY(read_flags(h, st, &f));
  if (f & kFlagZeroPivot)
    return fail(h, SPK_ERR_SINGULAR_PROJECTED,
                "split solve: a shifted system is singular or the small Schur form did not converge");
  return SPK_OK;
}

// H Y + Y G^T = F (m x m, column-major, ld m) when H and/or G have eigenvalues
// off the open right half plane (Eq. (3.4) with a sketched projection whose
// field of values left the half plane): the sign iteration alone does not
// apply, but its iterates converged to S_H = sign(H), S_G = sign(G) with
// kH, kG eigenvalues of negative real part (kH, kG <= kSplitMaxK).  With the
// spectral projectors P_H+- = (I +- S_H)/2 and P_G+- likewise,
//   Y = P_H+ Y P_G+^T + P_H+ Y P_G-^T + P_H- Y.
// The first part solves H' Y + Y G'^T = P_H+ F P_G+^T with H' = H + c_H P_H-,
// G' = G + c_G P_G- (c = twice the largest column sum, so that every
// eigenvalue is moved into the right half plane; H' and H agree on the range
// of P_H+), by the sign iteration.  The last part is minus_block on (H, G),
// the middle one minus_block on the transposed equation (G, H).  Y to Yout.
int split_solve(spk_handle* h, int m, const double* H, const double* G, const double* SH,
                const double* SG, int kH, int kG, const double* F, double* Yout, int max_newton,
                uint64_t seed, cudaStream_t st, int* iters_out) {
  if (kH > kSplitMaxK || kG > kSplitMaxK || kH < 0 || kG < 0 || kH + kG == 0)
    return fail(h, SPK_ERR_SINGULAR_PROJECTED,
                "projected matrices have %d and %d eigenvalues off the open right half plane "
                "(m=%d): more than the split solve handles (%d)", kH, kG, m, kSplitMaxK);
  WS(H1, double, "sp_H1", (size_t)m * m);
  WS(G1, double, "sp_G1", (size_t)m * m);
  WS(P, double, "sp_P", (size_t)m * m);
  WS(F1, double, "sp_F1", (size_t)m * m);
  WS(T1, double, "sp_T1", (size_t)m * m);
  double cH = 0.0, cG = 0.0;
  TRY(max_col_abs_sum(h, H, m, m, st, &cH));
  TRY(max_col_abs_sum(h, G, m, m, st, &cG));
  cH *= 2.0;
  cG *= 2.0;
  // F1 = P_H+ F P_G+^T; T1 = P_H+ F (kept for the middle part)
  sign_affine_launch(nullptr, m, 0.0, SH, m, 0.5, 1.0, m, P, m, st);
  gemm_f64('N', 'N', m, m, m, 1.0, P, m, F, m, 0.0, T1, m, st);
  sign_affine_launch(nullptr, m, 0.0, SG, m, 0.5, 1.0, m, P, m, st);
  gemm_f64('N', 'T', m, m, m, 1.0, T1, m, P, m, 0.0, F1, m, st);
  // H' = H + c_H (I - S_H)/2, G' = G + c_G (I - S_G)/2
  sign_affine_launch(H, m, 1.0, SH, m, 0.5 * cH, -1.0, m, H1, m, st);
  sign_affine_launch(G, m, 1.0, SG, m, 0.5 * cG, -1.0, m, G1, m, st);
  copy_matrix_launch(F1, m, Yout, m, m, m, st);
  h->trace_fail = false;
  TRY(sign_solve(h, m, H1, G1, Yout, max_newton, st, iters_out));
  if (kH > 0) TRY(minus_block(h, m, H, m, G, m, SH, m, kH, F, false, Yout, seed + 17, st));
  if (kG > 0) {
    // the transposed equation G X + X H^T = (P_H+ F)^T for X = (P_H+ Y P_G-^T)^T
    WS(T1t, double, "sp_T1t", (size_t)m * m);
    sign_affine_launch(nullptr, m, 0.0, SH, m, 0.5, 1.0, m, P, m, st);
    gemm_f64('T', 'T', m, m, m, 1.0, F, m, P, m, 0.0, T1t, m, st);
    TRY(minus_block(h, m, G, m, H, m, SG, m, kG, T1t, true, Yout, seed + 29, st));
  }
  TRY(wait_stream(h, st, h->host_wait_s));
  CK(cudaGetLastError());
  return SPK_OK;
}

// Round-robin pairing of N (even) columns for one Jacobi sweep: rounds x pairs.
void jacobi_schedule(int N, std::vector<int>& pairs, int& rounds, int& npairs) {
  const int Ne = N + (N & 1);
  rounds = Ne - 1;
  npairs = Ne / 2;
  pairs.assign((size_t)rounds * npairs * 2, 0);
  std::vector<int> ring(Ne);
  for (int i = 0; i < Ne; ++i) ring[i] = i;
  for (int rd = 0; rd < rounds; ++rd) {
    for (int k = 0; k < npairs; ++k) {
      int a = ring[k], b = ring[Ne - 1 - k];
      if (a > b) std::swap(a, b);
      pairs[((size_t)rd * npairs + k) * 2] = a;
      pairs[((size_t)rd * npairs + k) * 2 + 1] = b;  // b == N (odd N) marks a dummy
    }
    // rotate all but the first
    int last = ring[Ne - 1];
    for (int i = Ne - 1; i > 1; --i) ring[i] = ring[i - 1];
    ring[1] = last;
  }
}

// One-sided Jacobi on the columns of A (M x N, ld lda); V (N x N) accumulated
// when non-null (set to I first).  Stops when every pair is orthogonal to 1e-15.
int jacobi_svd(spk_handle* h, double* A, int64_t lda, int M, int N, double* V, cudaStream_t st) {
  std::vector<int> pairs;
  int rounds = 0, npairs = 0;
  jacobi_schedule(N, pairs, rounds, npairs);
  WS(dpairs, int, "jac_pairs", pairs.size());
  WS(offs, double, "jac_offs", (size_t)rounds * npairs);
  CK(cudaMemcpyAsync(dpairs, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice, st));
  if (V) {
    set_zero_launch(V, (int64_t)N * N, st);
    std::vector<double> eye((size_t)N * N, 0.0);
    for (int i = 0; i < N; ++i) eye[(size_t)i * N + i] = 1.0;
    CK(cudaMemcpyAsync(V, eye.data(), sizeof(double) * N * N, cudaMemcpyHostToDevice, st));
    TRY(wait_stream(h, st, h->host_wait_s));
  }
  std::vector<double> hoffs((size_t)rounds * npairs);
  for (int sweep = 0; sweep < 30; ++sweep) {
    for (int rd = 0; rd < rounds; ++rd)
      jacobi_round_launch(A, lda, M, N, V, N, dpairs + (size_t)rd * npairs * 2, npairs,
                          offs + (size_t)rd * npairs, st);
    TRY(d2h(h, hoffs.data(), offs, sizeof(double) * hoffs.size(), st));
    CK(cudaGetLastError());
    double mx = 0.0;
    for (double v : hoffs) mx = std::max(mx, v);
    if (mx < 1e-14) break;
  }
  return SPK_OK;
}

// Low-rank factors of Y (m x m): Y ~= Y1 Y2^T, keeping singular values above
// trunc_tol * sigma_1 (Algorithm 1 after the loop).  An adaptive blocked
// randomized range finder (Gaussian blocks of 64 columns, each projected twice
// against the basis found so far and orthogonalised by one-sided Jacobi) runs
// until a fresh block's projected norms fall below 0.01 * trunc_tol * ||Y||;
// then B = Q^T Y is factored by one-sided Jacobi: Y ~= (Q V) Sigma U_b^T.
// Y1 = (Q V) Sigma^{1/2}, Y2 = U_b Sigma^{1/2} (m x ell, column-major, ld m),
// returned as workspace buffers.
int truncate_Y(spk_handle* h, const double* Y, int m, double trunc_tol, uint64_t seed,
               cudaStream_t st, double** Y1p, double** Y2p, int* ell_out) {
  const int kcap = std::min(m, 2048);
  const int bsz = std::min(m, 64);
  WS(Q, double, "tr_Q", (size_t)m * kcap);
  WS(Z, double, "tr_Z", (size_t)m * bsz);
  WS(C, double, "tr_C", (size_t)kcap * bsz);
  WS(nrm, double, "tr_nrm", bsz);
  WS(idx, int, "tr_idx", std::max(bsz, kcap));
  WS(f1, double, "tr_f1", std::max(bsz, kcap));
  WS(f2, double, "tr_f2", std::max(bsz, kcap));
  WS(dcount, int, "tr_cnt", 1);
  std::vector<double> hn(bsz);
  int k = 0;
  double scale = 0.0;
  for (int blk = 0; k < kcap; ++blk) {
    const int b = std::min(bsz, kcap - k);
    WS(Om, double, "tr_Om", (size_t)m * bsz);
    gaussian_fill_launch(Om, (int64_t)m * b, seed + 7919ull * (blk + 1), st);
    gemm_f64('N', 'N', m, b, m, 1.0, Y, m, Om, m, 0.0, Z, m, st);
    for (int pass = 0; pass < 2 && k > 0; ++pass) {   // Z -= Q (Q^T Z), twice
      gemm_f64('T', 'N', k, b, m, 1.0, Q, m, Z, m, 0.0, C, k, st);
      gemm_f64('N', 'N', m, b, k, -1.0, Q, m, C, k, 1.0, Z, m, st);
    }
    col_norms_launch(Z, m, m, b, nrm, st);
    TRY(d2h(h, hn.data(), nrm, sizeof(double) * b, st));
    double mx = 0.0;
    for (int j = 0; j < b; ++j) mx = std::max(mx, hn[j]);
    if (blk == 0) scale = mx;
    if (!(scale > 0.0) || !std::isfinite(mx)) break;
    if (blk > 0 && mx <= 1e-2 * trunc_tol * scale) break;
    TRY(jacobi_svd(h, Z, m, m, b, nullptr, st));
    col_norms_launch(Z, m, m, b, nrm, st);
    // keep directions above 1e-3 * trunc_tol of the scale, normalised
    select_sv_launch(nrm, b, 1e-3 * trunc_tol * scale / std::max(mx, 1e-300), idx, f1, f2, dcount, st);
    int kb = 0;
    TRY(d2h(h, &kb, dcount, sizeof(int), st));
    TRY(d2h(h, hn.data(), nrm, sizeof(double) * b, st));
    if (kb <= 0) break;
    // 1/sigma factors (f2 holds sigma^{-1/2}: square it on the device side of the gather)
    std::vector<double> hf(kb);
    std::vector<int> hidx(kb);
    TRY(d2h(h, hidx.data(), idx, sizeof(int) * kb, st));
    for (int t = 0; t < kb; ++t) hf[t] = 1.0 / hn[hidx[t]];
    CK(cudaMemcpyAsync(f1, hf.data(), sizeof(double) * kb, cudaMemcpyHostToDevice, st));
    WS(Zn, double, "tr_Zn", (size_t)m * bsz);
    gather_cols_launch(Z, m, m, idx, f1, kb, Zn, m, st);
    // the normalised block is projected against Q twice more and
    // re-orthogonalised: its pre-normalisation remainder can be ~1e-12 of the
    // sample, so projections before normalising leave O(u / 1e-12) overlap
    for (int pass = 0; pass < 2 && k > 0; ++pass) {
      gemm_f64('T', 'N', k, kb, m, 1.0, Q, m, Zn, m, 0.0, C, k, st);
      gemm_f64('N', 'N', m, kb, k, -1.0, Q, m, C, k, 1.0, Zn, m, st);
    }
    TRY(jacobi_svd(h, Zn, m, m, kb, nullptr, st));
    col_norms_launch(Zn, m, m, kb, nrm, st);
    TRY(d2h(h, hn.data(), nrm, sizeof(double) * kb, st));
    for (int t = 0; t < kb; ++t) {
      hidx[t] = t;
      hf[t] = hn[t] > 0.0 ? 1.0 / hn[t] : 0.0;
    }
    CK(cudaMemcpyAsync(idx, hidx.data(), sizeof(int) * kb, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(f1, hf.data(), sizeof(double) * kb, cudaMemcpyHostToDevice, st));
    gather_cols_launch(Zn, m, m, idx, f1, kb, Q + (size_t)k * m, m, st);
    TRY(wait_stream(h, st, h->host_wait_s));
    k += kb;
    if (kb < b) break;   // the sample did not fill: the range is exhausted
  }
  if (k == 0) {
    *ell_out = 0;
    return SPK_OK;
  }
  // B^T = Y^T Q (m x k); one-sided Jacobi with V accumulation
  WS(Bt, double, "tr_Bt", (size_t)m * k);
  WS(Vb, double, "tr_Vb", (size_t)k * k);
  gemm_f64('T', 'N', m, k, m, 1.0, Y, m, Q, m, 0.0, Bt, m, st);
  TRY(jacobi_svd(h, Bt, m, m, k, Vb, st));
  WS(sg, double, "tr_sg", k);
  WS(idx2, int, "tr_idx2", k);
  WS(g1, double, "tr_g1", k);
  WS(g2, double, "tr_g2", k);
  WS(dell2, int, "tr_ell2", 1);
  col_norms_launch(Bt, m, m, k, sg, st);
  select_sv_launch(sg, k, trunc_tol, idx2, g1, g2, dell2, st);
  int ell = 0;
  TRY(d2h(h, &ell, dell2, sizeof(int), st));
  WS(Y1, double, "tr_Y1", (size_t)m * std::max(ell, 1));
  WS(Y2, double, "tr_Y2", (size_t)m * std::max(ell, 1));
  WS(QV, double, "tr_QV", (size_t)m * k);
  gemm_f64('N', 'N', m, k, k, 1.0, Q, m, Vb, k, 0.0, QV, m, st);
  gather_cols_launch(QV, m, m, idx2, g1, ell, Y1, m, st);
  gather_cols_launch(Bt, m, m, idx2, g2, ell, Y2, m, st);
  *Y1p = Y1;
  *Y2p = Y2;
  *ell_out = ell;
  return SPK_OK;
}

// ---------------------------------------------------------------------------
template <typename TB, typename TC, typename TV>
struct Side {
  const spk_csr* op = nullptr;
  int64_t n = 0;
  int k = 1, r = 1, maxit = 1;
  const TV* vals = nullptr;
  TB* win = nullptr;
  TC* W = nullptr;
  double* hband = nullptr;   // (maxit+1) x (k+1) x r x r
  double* r1inv = nullptr;   // (maxit+1) x r x r
  double* r2inv = nullptr;
  double* T = nullptr;
  int64_t ldT = 0;
  double* Q = nullptr;       // s x ldT
  // int8 digit copies of Q for the tensor-core whitening products
  QsGeom qs;
  uint8_t *QA = nullptr, *QB = nullptr;
  bool qs_on = false;
  double* Ht = nullptr;
  int64_t ldH = 0;
  SketchDev sk;
  TC* sk_scratch = nullptr;
  double *w = nullptr, *w1 = nullptr, *t1 = nullptr, *t2 = nullptr;
  double *ell = nullptr, *beta = nullptr, *R1 = nullptr, *R2 = nullptr, *Rinv = nullptr, *tau = nullptr;
  double* partial = nullptr;
  double* qpartial = nullptr;
  double* cwork = nullptr;   // DCT sketch: 2 n r doubles of complex work
  double* V = nullptr;       // full method: n x (maxit+1) r column-major basis
  double *wn = nullptr, *wn1 = nullptr;   // full method: n x r column-major work
  // mixed forms with an FP64 start (spk_opts.fp64_until > 0): FP64 ring and
  // work block of the iterations before the switch, FP64 sketch scratch
  double* win64 = nullptr;
  double* W64 = nullptr;
  double* sk_scratch64 = nullptr;
  int grid = 1;

  TB* block(int j) const { return win + (size_t)(j % (k + 1)) * n * r; }
  double* block64(int j) const { return win64 + (size_t)(j % (k + 1)) * n * r; }
  double* hcol(int d) const { return hband + (size_t)d * (k + 1) * r * r; }
  double* hslot(int d, int q) const { return hcol(d) + (size_t)q * r * r; }
  double* R1inv(int d) const { return r1inv + (size_t)d * r * r; }
  double* R2inv(int d) const { return r2inv + (size_t)d * r * r; }
};

template <typename TB, typename TC, typename TV>
struct Solver {
  spk_handle* h;
  cudaStream_t st;
  spk_opts o;
  int r = 1;
  Side<TB, TC, TV> S[2];
  // Precision schedule of the mixed forms: Arnoldi step d (d = 0: the
  // initial QR of C) runs in FP64 while d < switch_d and in the form's
  // precision from switch_d on; block U_j is FP64 iff j <= switch_d.
  // switch_d = 0: the form's precision throughout (also the FP64 form);
  // kNever: no switch yet (fp64_until > 0 until a check falls below it).
  static constexpr int kNever = 0x7fffffff;
  int switch_d = 0;
  bool two_prec() const { return !std::is_same<TB, double>::value && o.fp64_until > 0.0; }
  bool hi_step(int d) const { return d < switch_d; }

  int alloc_side(int idx, const spk_csr* op, int k, int s_rows, int sketch_id) {
    auto& sd = S[idx];
    const std::string p = idx == 0 ? "U_" : "V_";
    sd.op = op;
    sd.n = op->nrows;
    sd.k = k;
    sd.r = r;
    sd.maxit = o.maxit;
    sd.grid = grid_rows(h, sd.n);
    const int64_t mmax = (int64_t)(o.maxit + 1) * r;
    sd.ldT = mmax;
    sd.ldH = mmax;
    if (std::is_same<TV, double>::value) {
      sd.vals = reinterpret_cast<const TV*>(op->val_dev);
    } else {
      TV* v = static_cast<TV*>(ws_get(h, p + "vals", sizeof(TV) * (size_t)std::max<int64_t>(op->nnz, 1)));
      if (!v) return fail(h, SPK_ERR_ALLOC, "cannot allocate converted values");
      convert_values_launch<TV>(op->val_dev, v, op->nnz, st);
      sd.vals = v;
    }
#define SWS(field, type, name, count)                                                     \
  sd.field = static_cast<type*>(ws_get(h, p + name, sizeof(type) * (size_t)(count)));     \
  if (!sd.field) return fail(h, SPK_ERR_ALLOC, "cannot allocate %s%s", p.c_str(), name);
    SWS(win, TB, "win", (size_t)(k + 1) * sd.n * r);
    SWS(W, TC, "W", (size_t)sd.n * r);
    if (two_prec()) {
      SWS(win64, double, "win64", (size_t)(k + 1) * sd.n * r);
      SWS(W64, double, "W64", (size_t)sd.n * r);
    }
    SWS(hband, double, "hband", (size_t)(o.maxit + 2) * (k + 1) * r * r);
    SWS(r1inv, double, "r1inv", (size_t)(o.maxit + 2) * r * r);
    SWS(r2inv, double, "r2inv", (size_t)(o.maxit + 2) * r * r);
    const bool sketched = o.method == SPK_METHOD_SKETCHED;
    if (o.method == SPK_METHOD_FULL) {
      // the whole basis, the Hessenberg matrix, CGS2 and Cholesky QR work
      SWS(V, double, "V", (size_t)sd.n * mmax);
      SWS(wn, double, "wn", (size_t)sd.n * r);
      SWS(wn1, double, "wn1", (size_t)sd.n * r);
      SWS(Ht, double, "Ht", (size_t)sd.ldH * sd.ldH);
      SWS(t1, double, "t1", (size_t)mmax * r);
      SWS(t2, double, "t2", (size_t)mmax * r);
      SWS(qpartial, double, "qpartial",
          std::max((size_t)q_update_chunks((int)mmax, sd.n) * sd.n * r,
                   (size_t)qt_dot_partial_doubles((int)mmax, r)));
      CK(cudaMemsetAsync(sd.Ht, 0, sizeof(double) * sd.ldH * sd.ldH, st));
    }
    const bool dct = sketched && o.sketch_kind == SPK_SKETCH_DCT;
    if (sketched) {
      SWS(T, double, "T", (size_t)sd.ldT * sd.ldT);
      SWS(Ht, double, "Ht", (size_t)sd.ldH * sd.ldH);
      sketch_geometry(sd.sk, sd.n, s_rows, o.sketch_kind == SPK_SKETCH_IDENTITY, (int)sizeof(TC), r);
      if (dct) {
        // the DCT sketch of the paper's experiments: rows over [0, n), scale sqrt(n/s)
        sd.sk.is_dct = 1;
        sd.sk.npad = sd.n;
        sd.sk.scale = std::sqrt((double)sd.n / (double)s_rows);
        if (!dct_geometry(sd.n, sd.sk.dct))
          return fail(h, SPK_ERR_UNSUPPORTED,
                      "DCT sketch needs n = f1 f2 with f1, f2 <= 1024 built from 2, 3, 5 (n=%lld)",
                      (long long)sd.n);
        SWS(cwork, double, "dct_work", 2 * (size_t)sd.n * r);
        sd.sk.cwork = sd.cwork;
        double* tabs = static_cast<double*>(ws_get(h, p + "dct_tables",
                                                   sizeof(double) * dct_table_doubles(sd.n, sd.sk.dct)));
        if (!tabs) return fail(h, SPK_ERR_ALLOC, "cannot allocate DCT tables");
        dct_tables_launch(sd.n, sd.sk.dct, tabs, st);
      }
    } else {
      sketch_geometry(sd.sk, sd.n, 1, 1, (int)sizeof(TC), r);
    }
    const int64_t s = sketched ? sd.sk.s : 1;
    if (sketched) {
      SWS(Q, double, "Q", (size_t)s * sd.ldT);
      SWS(w, double, "w", (size_t)s * r);
      SWS(w1, double, "w1", (size_t)s * r);
      SWS(t1, double, "t1", (size_t)mmax * r);
      SWS(t2, double, "t2", (size_t)mmax * r);
    }
    SWS(ell, double, "ell", r * r);
    SWS(beta, double, "beta", r * r);
    SWS(R1, double, "R1", r * r);
    SWS(R2, double, "R2", r * r);
    SWS(Rinv, double, "Rinv", r * r);
    SWS(tau, double, "tau", r * r);
    const int groups = (k + 3) / 4;
    SWS(partial, double, "partial",
        (size_t)std::max(std::max(sd.grid, 2 * h->sm_count), 64) * 4 * r * r * std::max(groups, 1));
    if (sketched) {
      sd.qs_on = h->tensor_gemm && qs_enabled(s, (int)mmax);
      size_t qpd = std::max({(size_t)q_update_chunks((int)mmax, s) * s * r,
                             (size_t)border_chunks((int)mmax) * mmax * r,
                             (size_t)qt_dot_partial_doubles((int)mmax, r)});
      if (sd.qs_on) {
        sd.qs = qs_geometry(s, (int)mmax);
        SWS(QA, uint8_t, "QA", sd.qs.bytesA);
        SWS(QB, uint8_t, "QB", sd.qs.bytesB);
        qpd = std::max({qpd, (size_t)qs_chunks(s) * mmax * r, (size_t)qs_chunks(mmax) * s * r});
      }
      SWS(qpartial, double, "qpartial", qpd);
      SWS(sk_scratch, TC, "skscratch", std::max<int64_t>(1, sd.sk.npad * r));
      if (two_prec()) {
        SWS(sk_scratch64, double, "skscratch64", std::max<int64_t>(1, sd.sk.npad * r));
      }
    }
#undef SWS
    if (sketched && !sd.sk.identity) {
      int32_t* rows = static_cast<int32_t*>(ws_get(h, p + "rows", sizeof(int32_t) * s));
      int8_t* signs = static_cast<int8_t*>(ws_get(h, p + "signs", (size_t)sd.n));
      const int64_t range = dct ? sd.n : 0;
      const size_t sb = sketch_draws_scratch_bytes(sd.n, s, range);
      void* scratch = ws_get(h, "sk_draw_scratch", sb);
      if (!rows || !signs || !scratch) return fail(h, SPK_ERR_ALLOC, "cannot allocate sketch draws");
      char e[256] = {0};
      int rc = sketch_draws_launch(sd.n, (int32_t)s, o.seed, sketch_id, rows, signs, scratch, sb, st,
                                   e, sizeof e, range);
      if (rc != SPK_OK) return fail(h, rc, "%s", e);
      sd.sk.rows = rows;
      sd.sk.signs = signs;
      if (dct) {
        int32_t* selpos = static_cast<int32_t*>(ws_get(h, p + "selpos", sizeof(int32_t) * (size_t)sd.n));
        if (!selpos) return fail(h, SPK_ERR_ALLOC, "cannot allocate DCT row positions");
        dct_selpos_launch(rows, (int32_t)s, sd.n, selpos, st);
        sd.sk.selpos = selpos;
      }
    }
    if (sketched) {
      CK(cudaMemsetAsync(sd.T, 0, sizeof(double) * sd.ldT * sd.ldT, st));
      CK(cudaMemsetAsync(sd.Ht, 0, sizeof(double) * sd.ldH * sd.ldH, st));
    }
    CK(cudaMemsetAsync(sd.hband, 0, sizeof(double) * (o.maxit + 2) * (k + 1) * r * r, st));
    return SPK_OK;
  }

  // CholQR2 of the s x r sketch block w: Q[:, m:m+r] tau = w.
  void sketch_qr(Side<TB, TC, TV>& sd, int m) {
    const int64_t s = sd.sk.s;
    const int g = std::max(1, std::min<int>((int)((s + 255) / 256), h->sm_count * 2));
    ts_gram_launch(sd.w, s, r, sd.partial, g, st);
    chol_small_launch(sd.partial, g, r, sd.R1, sd.Rinv, h->flags, 1e-28, st);
    ts_scale_launch(sd.w, s, r, sd.Rinv, sd.w, s, st);
    ts_gram_launch(sd.w, s, r, sd.partial, g, st);
    chol_small_launch(sd.partial, g, r, sd.R2, sd.Rinv, h->flags, 1e-28, st);
    ts_scale_launch(sd.w, s, r, sd.Rinv, sd.Q + (int64_t)m * s, s, st);
    combine_small_launch(sd.R2, sd.R1, sd.tau, r, 0, st);
    if (sd.qs_on) qs_append_launch(sd.Q, sd.qs, m, r, sd.QA, sd.QB, st);
  }

  int init_side(Side<TB, TC, TV>& sd, const double* C) {
    if (hi_step(0)) return init_side_t<double, double>(sd, C, sd.win64, sd.W64, sd.sk_scratch64);
    return init_side_t<TB, TC>(sd, C, sd.win, sd.W, sd.sk_scratch);
  }

  template <typename XB, typename XC>
  int init_side_t(Side<TB, TC, TV>& sd, const double* C, XB* ring, XC* W, XC* skscr) {
    XB* U1 = ring + (size_t)(1 % (sd.k + 1)) * sd.n * r;
    // U_1 = C ell^{-1} by Cholesky QR twice (Algorithm 1, first step)
    convert_block_launch<XC>(C, W, sd.n * r, st);
    WindowPtrs none{};
    none.nwin = 0;
    update_gram_launch<XB, XC>(W, sd.n, r, none, sd.hband, sd.partial, sd.grid, 1, st);
    chol_small_launch(sd.partial, sd.grid, r, sd.R1, sd.R1inv(0), h->flags, kBreakdownFloor, st);
    scale_gram_launch<XC>(W, sd.n, r, sd.R1inv(0), sd.partial, sd.grid, st);
    chol_small_launch(sd.partial, sd.grid, r, sd.R2, sd.R2inv(0), h->flags, 1e-28, st);
    combine_small_launch(sd.R2, sd.R1, sd.ell, r, 0, st);
    scale_store_launch<XB, XC>(W, sd.n, r, sd.R2inv(0), U1, st);
    if (o.method != SPK_METHOD_SKETCHED) {
      // Algorithm 2 and full Arnoldi: C = U_1 beta with beta = ell
      CK(cudaMemcpyAsync(sd.beta, sd.ell, sizeof(double) * r * r, cudaMemcpyDeviceToDevice, st));
      if (o.method == SPK_METHOD_FULL)
        block_to_cols_launch(reinterpret_cast<const double*>(U1), sd.n, r, sd.V, sd.n, st);
      return SPK_OK;
    }
    // T_1 = R factor of S U_1 (reading of Algorithm 1's first step), beta = T_1 ell
    sketch_apply_launch<XB, XC>(sd.sk, U1, r, sd.w, skscr, st);
    sketch_qr(sd, 0);
    t_write_launch(sd.T, sd.ldT, 0, r, nullptr, nullptr, sd.tau, st);
    combine_small_launch(sd.tau, sd.ell, sd.beta, r, 0, st);
    return SPK_OK;
  }

  template <typename XB>
  WindowPtrs window_in(const Side<TB, TC, TV>& sd, XB* ring, int d, int* first) const {
    const int i0 = std::max(1, d - sd.k + 1);
    WindowPtrs w{};
    w.nwin = d - i0 + 1;
    for (int q = 0; q < w.nwin; ++q) w.blk[q] = ring + (size_t)((i0 + q) % (sd.k + 1)) * sd.n * r;
    *first = i0;
    return w;
  }
  WindowPtrs window(const Side<TB, TC, TV>& sd, int d, int* first) const {
    return window_in(sd, sd.win, d, first);
  }

  // First step in the form's precision after FP64 steps: the window blocks
  // it reads (U_{d-k+1} .. U_d, all FP64) are rounded into the mixed ring.
  void convert_window(Side<TB, TC, TV>& sd, int d) {
    for (int j = std::max(1, d - sd.k + 1); j <= d; ++j)
      convert_block_launch<TB>(sd.block64(j), sd.block(j), sd.n * r, st);
  }

  // Arnoldi step d for one side, up to and including U_{d+1} (no sketch).
  void arnoldi_basis(Side<TB, TC, TV>& sd, int d, bool replay) {
    if (hi_step(d)) {
      arnoldi_basis_t<double, double, double>(sd, d, replay, sd.win64, sd.W64, sd.op->val_dev);
      return;
    }
    if (d == switch_d && switch_d > 0) convert_window(sd, d);
    arnoldi_basis_t<TB, TC, TV>(sd, d, replay, sd.win, sd.W, sd.vals);
  }

  template <typename XB, typename XC, typename XV>
  void arnoldi_basis_t(Side<TB, TC, TV>& sd, int d, bool replay, XB* ring, XC* W,
                       const XV* vals) {
    auto blk = [&](int j) { return ring + (size_t)(j % (sd.k + 1)) * sd.n * r; };
    int i0 = 0;
    WindowPtrs win = window_in(sd, ring, d, &i0);
    const int slot0 = i0 - (d - sd.k + 1);
    double* hs = sd.hslot(d, slot0);
    const spk_csr* op = sd.op;
    const double nr = (double)sd.n * r, bB = sizeof(XB), bC = sizeof(XC), bV = sizeof(XV);
    const double csr_bytes = (double)op->nnz * (bV + 4) + (double)(sd.n + 1) * 4;
    if (!replay) {
      {
        ProfScope ps(h, F_SPMM, st,
                     csr_bytes + nr * (bB + bC) + win.nwin * nr * bB,
                     2.0 * op->nnz * r + 2.0 * win.nwin * nr * r);
        spmm_dots_launch<XB, XC, XV>(op->rowptr_dev, op->col_dev, vals, sd.n, r, blk(d), W,
                                     win, sd.partial, sd.grid, st);
        for (int g = 0; g < win.nwin; g += 4) {
          const int nq = std::min(4, win.nwin - g);
          reduce_partials_launch(sd.partial + (size_t)(g / 4) * sd.grid * 4 * r * r, sd.grid,
                                 4 * r * r, nq * r * r, hs + (size_t)g * r * r, st);
        }
      }
      {
        ProfScope ps(h, F_UPDATE, st, 2 * nr * bC + win.nwin * nr * bB,
                     2.0 * win.nwin * nr * r + 2.0 * nr * r);
        update_gram_launch<XB, XC>(W, sd.n, r, win, hs, sd.partial, sd.grid, 1, st);
        chol_small_launch(sd.partial, sd.grid, r, sd.R1, sd.R1inv(d), h->flags, kBreakdownFloor, st);
      }
      ProfScope ps(h, F_SCALE, st, 3 * nr * bC + nr * bB, 4.0 * nr * r);
      scale_gram_launch<XC>(W, sd.n, r, sd.R1inv(d), sd.partial, sd.grid, st);
      chol_small_launch(sd.partial, sd.grid, r, sd.R2, sd.R2inv(d), h->flags, 1e-28, st);
      combine_small_launch(sd.R2, sd.R1, sd.hslot(d, sd.k), r, 0, st);
      scale_store_launch<XB, XC>(W, sd.n, r, sd.R2inv(d), blk(d + 1), st);
    } else {
      WindowPtrs none{};
      none.nwin = 0;
      {
        ProfScope ps(h, F_SPMM, st, csr_bytes + nr * (bB + bC), 2.0 * op->nnz * r);
        spmm_dots_launch<XB, XC, XV>(op->rowptr_dev, op->col_dev, vals, sd.n, r, blk(d), W, none,
                                     sd.partial, sd.grid, st);
      }
      {
        ProfScope ps(h, F_UPDATE, st, 2 * nr * bC + win.nwin * nr * bB, 2.0 * win.nwin * nr * r);
        update_gram_launch<XB, XC>(W, sd.n, r, win, hs, sd.partial, sd.grid, 0, st);
      }
      ProfScope ps(h, F_SCALE, st, 3 * nr * bC + nr * bB, 2.0 * nr * r);
      scale_gram_launch<XC>(W, sd.n, r, sd.R1inv(d), sd.partial, sd.grid, st);
      scale_store_launch<XB, XC>(W, sd.n, r, sd.R2inv(d), blk(d + 1), st);
    }
  }

  // Full block Arnoldi step d (Section 2.1): U~ = A U_d against all previous
  // blocks by block CGS2 (the whitening kernels with n rows), Cholesky QR
  // twice for U_{d+1} and h_{d+1,d}; block column d of the Hessenberg H_d.
  void arnoldi_full(Side<TB, TC, TV>& sd, int d) {
    const int m = d * r;
    const int64_t n = sd.n;
    WindowPtrs none{};
    none.nwin = 0;
    const double nr = (double)n * r;
    {
      ProfScope ps(h, F_SPMM, st, (double)sd.op->nnz * 12 + 2.0 * nr * 8, 2.0 * sd.op->nnz * r);
      spmm_dots_launch<TB, TC, TV>(sd.op->rowptr_dev, sd.op->col_dev, sd.vals, n, r, sd.block(d),
                                   sd.W, none, sd.partial, sd.grid, st);
    }
    block_to_cols_launch(reinterpret_cast<const double*>(sd.W), n, r, sd.wn, n, st);
    const int nch = q_update_chunks(m, n);
    const double nm8 = 8.0 * n * m, nr8 = 8.0 * nr;
    {
      ProfScope ps(h, F_QTDOT, st, nm8 + nr8, 2.0 * n * m * r);
      qt_dot_launch(sd.V, n, n, m, sd.wn, r, sd.t1, sd.qpartial, st);
    }
    {
      ProfScope ps(h, F_QUPDATE, st, nm8 + 2 * nr8, 2.0 * n * m * r);
      q_update_launch(sd.V, n, n, m, sd.t1, r, sd.wn, sd.wn1, sd.qpartial, nch, st);
    }
    {
      ProfScope ps(h, F_QTDOT, st, nm8 + nr8, 2.0 * n * m * r);
      qt_dot_launch(sd.V, n, n, m, sd.wn1, r, sd.t2, sd.qpartial, st);
    }
    {
      ProfScope ps(h, F_QUPDATE, st, nm8 + 2 * nr8, 2.0 * n * m * r);
      q_update_launch(sd.V, n, n, m, sd.t2, r, sd.wn1, sd.wn, sd.qpartial, nch, st);
    }
    {
      ProfScope ps(h, F_TSQR, st, 6 * nr8, 6.0 * nr * r);
      tall_qr(sd.wn, n, sd.V + (int64_t)m * n, n);
      // block column d of H_d: h_{i,d} = t1 + t2 (rows < m), h_{d+1,d} = tau
      t_write_launch(sd.Ht - (int64_t)r * sd.ldH, sd.ldH, m, r, sd.t1, sd.t2, sd.tau, st);
      cols_to_block_launch(sd.V + (int64_t)m * n, n, n, r,
                           reinterpret_cast<double*>(sd.block(d + 1)), st);
    }
  }

  // Cholesky QR twice of an n x r column-major block w (ld n): out tau = w,
  // out written with leading dimension ldo; tau (r x r, row-major) in sd.tau
  // of the side being processed (set by the caller through `cur`).
  Side<TB, TC, TV>* cur = nullptr;
  void tall_qr(double* w, int64_t n, double* out, int64_t ldo) {
    auto& sd = *cur;
    const int g = std::max(1, std::min<int>((int)((n + 255) / 256), h->sm_count * 2));
    ts_gram_launch(w, n, r, sd.partial, g, st);
    chol_small_launch(sd.partial, g, r, sd.R1, sd.Rinv, h->flags, kBreakdownFloor, st);
    ts_scale_launch(w, n, r, sd.Rinv, w, n, st);
    ts_gram_launch(w, n, r, sd.partial, g, st);
    chol_small_launch(sd.partial, g, r, sd.R2, sd.Rinv, h->flags, 1e-28, st);
    ts_scale_launch(w, n, r, sd.Rinv, out, ldo, st);
    combine_small_launch(sd.R2, sd.R1, sd.tau, r, 0, st);
  }

  // Sketch of U_{d+1}, QR update of S U_{d+1}, T column, bordering update of H~.
  void whiten_and_border(Side<TB, TC, TV>& sd, int d) {
    const int m = d * r;
    const int64_t s = sd.sk.s;
    const double sr8 = 8.0 * s * r, sm8 = 8.0 * s * m;
    {
      ProfScope ps(h, F_SKETCH, st,
                   (double)sd.n * r * sizeof(TB) + (double)sd.n + sr8,
                   sd.sk.identity ? 0.0 : (double)sd.sk.npad * r * sd.sk.log2n2 + (double)s * sd.sk.n1 * r);
      if (hi_step(d))
        sketch_apply_launch<double, double>(sd.sk, sd.block64(d + 1), r, sd.w, sd.sk_scratch64, st);
      else
        sketch_apply_launch<TB, TC>(sd.sk, sd.block(d + 1), r, sd.w, sd.sk_scratch, st);
    }
    const int nch = q_update_chunks(m, s);
    // CGS2 against Q: on the tensor cores from the sliced copies of Q (the
    // algorithmic bytes are those of the FP64 Q, so the two paths compare)
    const bool tq = sd.qs_on && qs_enabled(s, m);
    auto qt = [&](const double* w, double* t) {
      ProfScope ps(h, F_QTDOT, st, sm8 + sr8 + 8.0 * m * r, 2.0 * s * m * r);
      if (tq)
        qs_qt_launch(sd.qs, sd.QA, m, w, r, t, sd.qpartial, h->flags, st);
      else
        qt_dot_launch(sd.Q, s, s, m, w, r, t, sd.qpartial, st);
    };
    auto qupd = [&](const double* t, const double* w_in, double* w_out) {
      ProfScope ps(h, F_QUPDATE, st, sm8 + 2 * sr8 + 8.0 * m * r, 2.0 * s * m * r);
      if (tq)
        qs_update_launch(sd.qs, sd.QB, m, t, r, w_in, w_out, sd.qpartial, h->flags, st);
      else
        q_update_launch(sd.Q, s, s, m, t, r, w_in, w_out, sd.qpartial, nch, st);
    };
    qt(sd.w, sd.t1);
    qupd(sd.t1, sd.w, sd.w1);
    qt(sd.w1, sd.t2);
    qupd(sd.t2, sd.w1, sd.w);
    {
      ProfScope ps(h, F_TSQR, st, 6 * sr8, 6.0 * s * r * r);
      sketch_qr(sd, m);
      t_write_launch(sd.T, sd.ldT, m, r, sd.t1, sd.t2, sd.tau, st);
    }
    ProfScope psb(h, F_BORDER, st, 8.0 * (double)(m - r) * (m - r) + 16.0 * m * r,
                  2.0 * (double)(m - r) * (m - r) * r);
    // bordering (Section 5): Hhat_d from H~_{d-1}, then the correction -> H~_d
    const int mp = m - r;
    int i0 = 0;
    (void)window(sd, d, &i0);
    const int slot0 = i0 - (d - sd.k + 1);
    if (d == 1) {
      border_small_launch(sd.Ht, sd.ldH, 0, r, sd.T, sd.ldT, nullptr, sd.hslot(1, slot0), st);
    } else {
      const int nslots = d - i0;  // blocks i0 .. d-1
      border_col_launch(sd.Ht, sd.ldH, mp, r, sd.T, sd.ldT, sd.hslot(d, slot0), i0, nslots,
                        sd.hslot(d, slot0 + nslots), sd.qpartial, st);
      border_small_launch(sd.Ht, sd.ldH, mp, r, sd.T, sd.ldT, sd.hslot(d - 1, sd.k),
                          sd.hslot(d, slot0 + nslots), st);
    }
    border_correct_launch(sd.Ht, sd.ldH, m, r, sd.T, sd.ldT, sd.hslot(d, sd.k), st);
  }

  int check(int d, double* rho3, int* newton_iters) {
    const int m = d * r;
    WS(Hk, double, "pj_Hk", (size_t)m * m);
    WS(Gk, double, "pj_Gk", (size_t)m * m);
    WS(F, double, "pj_F", (size_t)m * m);
    WS(out3, double, "pj_out3", 4);
    const bool sketched = o.method == SPK_METHOD_SKETCHED;
    const bool full = o.method == SPK_METHOD_FULL;
    if (sketched || full) {
      copy_matrix_launch(S[0].Ht, S[0].ldH, Hk, m, m, m, st);
      copy_matrix_launch(S[1].Ht, S[1].ldH, Gk, m, m, m, st);
    } else {
      // Algorithm 2: the projected matrices are the banded H_d, G_d themselves
      set_zero_launch(Hk, (int64_t)m * m, st);
      set_zero_launch(Gk, (int64_t)m * m, st);
      band_to_dense_launch(S[0].hband, S[0].k, r, d, Hk, m, st);
      band_to_dense_launch(S[1].hband, S[1].k, r, d, Gk, m, st);
    }
    // right-hand side E_1 beta_1 beta_2^T E_1^T in factored form, L_0 = E_1 beta_1,
    // R_0 = E_1 beta_2 (the sign iteration forms F once the factors pass m/2 columns)
    const int qcap = std::max(r, m / 2);
    WS(Lf, double, "pj_L", (size_t)m * qcap);
    WS(Rf, double, "pj_R", (size_t)m * qcap);
    set_zero_launch(Lf, (int64_t)m * r, st);
    set_zero_launch(Rf, (int64_t)m * r, st);
    fill_factor_launch(Lf, m, r, S[0].beta, st);
    fill_factor_launch(Rf, m, r, S[1].beta, st);
    if (o.inject & SPK_INJECT_SINGULAR)
      return fail(h, SPK_ERR_SINGULAR_PROJECTED, "injected: singular projected equation");
    h->trace_fail = false;
    int src = sign_solve(h, m, Hk, Gk, F, o.max_newton, st, newton_iters, Lf, Rf, r, qcap);
    if (src == SPK_ERR_SINGULAR_PROJECTED && h->trace_fail) {
      // eigenvalues off the open right half plane: Hk and Gk now hold sign(H~)
      // and sign(G~); solve by spectral splitting on the original matrices
      const int kH = h->neg_h, kG = h->neg_g;
      WS(H0, double, "pj_H0", (size_t)m * m);
      WS(G0, double, "pj_G0", (size_t)m * m);
      WS(Fd, double, "pj_Fd", (size_t)m * m);
      if (sketched || full) {
        copy_matrix_launch(S[0].Ht, S[0].ldH, H0, m, m, m, st);
        copy_matrix_launch(S[1].Ht, S[1].ldH, G0, m, m, m, st);
      } else {
        set_zero_launch(H0, (int64_t)m * m, st);
        set_zero_launch(G0, (int64_t)m * m, st);
        band_to_dense_launch(S[0].hband, S[0].k, r, d, H0, m, st);
        band_to_dense_launch(S[1].hband, S[1].k, r, d, G0, m, st);
      }
      set_zero_launch(Lf, (int64_t)m * r, st);
      set_zero_launch(Rf, (int64_t)m * r, st);
      fill_factor_launch(Lf, m, r, S[0].beta, st);
      fill_factor_launch(Rf, m, r, S[1].beta, st);
      gemm_f64('N', 'T', m, m, r, 1.0, Lf, m, Rf, m, 0.0, Fd, m, st);
      h->spectrum_bad = false;
      src = split_solve(h, m, H0, G0, Hk, Gk, kH, kG, Fd, F, o.max_newton, o.seed, st,
                        newton_iters);
      // unsolved: let the caller fall back to an earlier check
      if (src != SPK_OK) h->spectrum_bad = true;
    }
    TRY(src);
    {
      ProfScope ps(h, F_RHO, st, 16.0 * m * r, 8.0 * m * r * r);
      // the newest subdiagonal blocks: h_{d+1,d} (hband slot, or the Cholesky
      // factor of the full method, read from block column d of H)
      const double* hU = S[0].hslot(d, S[0].k);
      const double* hV = S[1].hslot(d, S[1].k);
      if (full) {
        WS(hsub, double, "pj_hsub", 2 * (size_t)r * r);
        sub_block_launch(S[0].Ht, S[0].ldH, m, m - r, r, hsub, st);
        sub_block_launch(S[1].Ht, S[1].ldH, m, m - r, r, hsub + r * r, st);
        hU = hsub;
        hV = hsub + r * r;
      }
      rho_launch(F, m, m, r, sketched ? S[0].T : nullptr, S[0].ldT, sketched ? S[1].T : nullptr,
                 S[1].ldT, hU, hV, S[0].beta, S[1].beta, o.method == SPK_METHOD_TRUNCATED, out3,
                 st);
    }
    TRY(d2h(h, rho3, out3, 3 * sizeof(double), st,
            (o.inject & SPK_INJECT_TIMEOUT) ? 0.0 : h->host_wait_s));
    CK(cudaGetLastError());
    return SPK_OK;
  }

  int recover(int d, const double* Y, spk_result* out) {
    const int m = d * r;
    double *Y1 = nullptr, *Y2 = nullptr;
    int ell = 0;
    {
      ProfScope ps(h, F_TRUNC, st, 8.0 * m * m, 0.0);
      TRY(truncate_Y(h, Y, m, o.trunc_tol, o.seed, st, &Y1, &Y2, &ell));
    }
    out->rank = ell;
    out->mem_solution_vectors = 2 * (int64_t)ell;
    if (ell == 0) return SPK_OK;
    // W_i = T_i^{-1} Y_i  (T_U, T_V leading m x m)
    {
      ProfScope ps(h, F_TRSM, st, 2 * 8.0 * ((double)m * m / 2 + 2.0 * m * ell), 2.0 * m * m * ell);
      if (o.method == SPK_METHOD_SKETCHED) {
        trsm_upper_left_launch(S[0].T, S[0].ldT, m, Y1, m, ell, st);
        trsm_upper_left_launch(S[1].T, S[1].ldT, m, Y2, m, ell, st);
      }
    }
    double* Wf[2] = {Y1, Y2};
    for (int side = 0; side < 2; ++side) {
      auto& sd = S[side];
      double* X = nullptr;
      if (cudaMalloc(&X, sizeof(double) * sd.n * ell) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, SPK_ERR_ALLOC, "cannot allocate factor X%d", side + 1);
      }
      if (side == 0) out->X1_dev = X; else out->X2_dev = X;
      if (o.method == SPK_METHOD_FULL) {
        // the basis is kept: X (n x ell, row-major) = (V_d W)^T in column-major terms
        ProfScope ps(h, F_XACC, st, (double)sd.n * (8.0 * m + 8.0 * ell), 2.0 * sd.n * m * ell);
        gemm_f64('T', 'T', ell, (int)sd.n, m, 1.0, Wf[side], m, sd.V, sd.n, 0.0, X, ell, st);
        continue;
      }
      if (h->tensor_gemm && sd.n >= 4096 && ell >= 8) {
        // second sweep on the tensor cores: the regenerated blocks fill a
        // panel of kXPanelCols FP64 columns; each full panel adds
        // P W[rows] to a column-major accumulator (tcgen05, error-free
        // splitting), transposed into X at the end
        const int bpp = std::max(1, kXPanelCols / r);
        const int pc = bpp * r;
        WS(Pn, double, "x_panel", (size_t)sd.n * pc);
        WS(Xcm, double, "x_colmajor", (size_t)sd.n * ell);
        WS(ozw, uint8_t, "x_ozaki", ozaki_work_bytes((int)sd.n, ell, pc));
        CK(cudaMemsetAsync(Xcm, 0, sizeof(double) * sd.n * ell, st));
        int j0 = 1;
        for (int j = 1; j <= d; ++j) {
          const int slot = j - j0;
          if (j <= switch_d)
            block_to_panel_launch<double>(sd.block64(j), sd.n, r, Pn + (size_t)slot * r * sd.n,
                                          sd.n, st);
          else
            block_to_panel_launch<TB>(sd.block(j), sd.n, r, Pn + (size_t)slot * r * sd.n, sd.n, st);
          if (slot + 1 == bpp || j == d) {
            const int cols = (slot + 1) * r;
            ProfScope ps(h, F_XACC, st, (double)sd.n * (2.0 * 8 * ell + 8.0 * cols),
                         2.0 * sd.n * ell * cols);
            ozaki_gemm('N', 'N', (int)sd.n, ell, cols, 1.0, Pn, sd.n,
                       Wf[side] + (size_t)(j0 - 1) * r, m, 1.0, Xcm, sd.n, ozw, h->flags, st);
            j0 = j + 1;
          }
          if (j == d) break;
          arnoldi_basis(sd, j, true);
        }
        cols_to_rows_launch(Xcm, sd.n, ell, X, st);
        continue;
      }
      CK(cudaMemsetAsync(X, 0, sizeof(double) * sd.n * ell, st));
      // second sweep: U_1 from C, then U_{j+1} from the stored coefficients
      int last = 0;
      for (int j = 1; j <= d; ++j) {
        // chunks never straddle the precision switch: U_j is FP64 iff j <= switch_d
        if (j - last == std::min(sd.k, kXMaxBlocks) || j == d || j == switch_d) {
          WindowPtrs blocks{};
          blocks.nwin = j - last;
          const bool hi = last + 1 <= switch_d;
          for (int q = 0; q < blocks.nwin; ++q)
            blocks.blk[q] = hi ? static_cast<const void*>(sd.block64(last + 1 + q))
                               : static_cast<const void*>(sd.block(last + 1 + q));
          ProfScope ps(h, F_XACC, st,
                       (double)sd.n * (2.0 * 8 * ell + blocks.nwin * r * (hi ? 8 : sizeof(TB))),
                       2.0 * sd.n * ell * r * blocks.nwin);
          if (hi)
            x_accumulate_launch<double>(X, sd.n, ell, r, blocks, Wf[side] + (size_t)last * r, m, st);
          else
            x_accumulate_launch<TB>(X, sd.n, ell, r, blocks, Wf[side] + (size_t)last * r, m, st);
          last = j;
        }
        if (j == d) break;
        arnoldi_basis(sd, j, true);
      }
    }
    return SPK_OK;
  }

  int replay_start(Side<TB, TC, TV>& sd, const double* C) {
    if (hi_step(0)) {
      convert_block_launch<double>(C, sd.W64, sd.n * r, st);
      scale_gram_launch<double>(sd.W64, sd.n, r, sd.R1inv(0), sd.partial, sd.grid, st);
      scale_store_launch<double, double>(sd.W64, sd.n, r, sd.R2inv(0), sd.block64(1), st);
      return SPK_OK;
    }
    convert_block_launch<TC>(C, sd.W, sd.n * r, st);
    scale_gram_launch<TC>(sd.W, sd.n, r, sd.R1inv(0), sd.partial, sd.grid, st);
    scale_store_launch<TB, TC>(sd.W, sd.n, r, sd.R2inv(0), sd.block(1), st);
    return SPK_OK;
  }

  int run(const spk_csr* A, const spk_csr* BT, const double* C1, const double* C2,
          spk_result* out) {
    cudaEvent_t e0, e1, ec0, ec1, er0, er1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&ec0);
    cudaEventCreate(&ec1);
    cudaEventCreate(&er0);
    cudaEventCreate(&er1);
    int rc = run_inner(A, BT, C1, C2, out, e0, e1, ec0, ec1, er0, er1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(ec0);
    cudaEventDestroy(ec1);
    cudaEventDestroy(er0);
    cudaEventDestroy(er1);
    return rc;
  }

  int run_inner(const spk_csr* A, const spk_csr* BT, const double* C1, const double* C2,
                spk_result* out, cudaEvent_t e0, cudaEvent_t e1, cudaEvent_t ec0, cudaEvent_t ec1,
                cudaEvent_t er0, cudaEvent_t er1) {
    CK(cudaMemsetAsync(h->flags, 0, sizeof(uint32_t), st));
    // optional host-side fault injection on a private copy of C1
    const double* C1use = C1;
    if (o.inject & (SPK_INJECT_NAN_C1 | SPK_INJECT_RANK_DEFICIENT)) {
      WS(c1c, double, "inj_C1", (size_t)A->nrows * r);
      CK(cudaMemcpyAsync(c1c, C1, sizeof(double) * A->nrows * r, cudaMemcpyDeviceToDevice, st));
      if (o.inject & SPK_INJECT_NAN_C1) {
        const double nanv = std::nan("");
        CK(cudaMemcpyAsync(c1c, &nanv, sizeof(double), cudaMemcpyHostToDevice, st));
      }
      if ((o.inject & SPK_INJECT_RANK_DEFICIENT) && r > 1) {
        // column 1 := column 0 (row-major, strided copy)
        CK(cudaMemcpy2DAsync(c1c + 1, sizeof(double) * r, C1, sizeof(double) * r, sizeof(double),
                             A->nrows, cudaMemcpyDeviceToDevice, st));
      }
      TRY(wait_stream(h, st, h->host_wait_s));
      C1use = c1c;
    }
    switch_d = two_prec() ? kNever : 0;
    const int s_req = o.s;
    TRY(alloc_side(0, A, o.k_left, s_req, 0));
    TRY(alloc_side(1, BT, o.k_right, s_req, o.same_sketch ? 0 : 1));
    cudaEventRecord(e0, st);
    TRY(init_side(S[0], C1use));
    TRY(init_side(S[1], C2));
    uint32_t f = 0;
    TRY(read_flags(h, st, &f));
    TRY(flags_to_status(h, f));

    std::vector<int32_t> hd;
    std::vector<double> hrel;
    double rho3[3] = {0, 0, 0};
    int newton = 0;
    int d = 0;
    bool converged = false;
    int last_good = 0;
    double ms_proj = 0.0, ms_loop = 0.0, ms_rec = 0.0;
    int next_check = o.fixed_d > 0 ? o.fixed_d : o.p;
    const int dmax = o.fixed_d > 0 ? std::min(o.fixed_d, o.maxit) : o.maxit;
    // The sketched estimate rho (Eq. (3.5)) measures the projected problem;
    // with a basis recurrence in reduced precision the Arnoldi relation
    // (Eq. (2.4)) holds only to that precision, which rho cannot see.  The
    // mixed forms therefore check the returned factors' true residual; when
    // it is above tol while rho is below, the iteration resumes (the replay
    // leaves the window as the first pass left it) with a lower target for
    // rho, at most kVerifyResumes times.
    const bool verify = o.verify > 0 || (o.verify == 0 && o.precision != SPK_PREC_FP64);
    constexpr int kVerifyResumes = 3;
    double target = o.tol;
    double true_rel = -1.0;
    int d_start = 1;
    for (int attempt = 0;; ++attempt) {
      for (d = d_start; d <= dmax; ++d) {
        for (int side = 0; side < 2; ++side) {
          if (o.method == SPK_METHOD_FULL) {
            cur = &S[side];
            arnoldi_full(S[side], d);
            continue;
          }
          arnoldi_basis(S[side], d, false);
          if (o.method == SPK_METHOD_SKETCHED) whiten_and_border(S[side], d);
        }
        const bool last = d == dmax;
        bool do_check = last;
        if (o.fixed_d <= 0) {
          if (o.check_schedule == SPK_CHECK_EVERY_P) do_check = do_check || (d % o.p == 0);
          else do_check = do_check || d >= next_check;
        }
        if (!do_check) continue;
        TRY(read_flags(h, st, &f));
        CK(cudaGetLastError());
        TRY(flags_to_status(h, f));
        cudaEventRecord(ec0, st);
        h->spectrum_bad = false;
        int crc = check(d, rho3, &newton);
        if (crc == SPK_ERR_SINGULAR_PROJECTED && h->spectrum_bad && o.fixed_d <= 0) {
          // Eigenvalues of H~ or G~ off the open right half plane.  Past
          // convergence the truncated basis degrades and such eigenvalues
          // appear; the leading block of H~_d is H~_d' for every d' < d, so
          // bisect between the last good check and d for a check that solves.
          int lo = last_good, hi = d, found = -1;
          while (hi - lo > 1) {
            const int mid = lo + (hi - lo) / 2;
            double r3[3] = {0, 0, 0};
            h->spectrum_bad = false;
            const int rc2 = check(mid, r3, &newton);
            if (rc2 == SPK_OK) {
              hd.push_back(mid);
              hrel.push_back(r3[1]);
              if (!std::isfinite(r3[1])) return fail(h, SPK_ERR_NONFINITE, "non-finite residual estimate at d=%d", mid);
              if (r3[1] < target) {
                found = mid;
                for (int e = 0; e < 3; ++e) rho3[e] = r3[e];
                break;
              }
              lo = mid;
            } else if (rc2 == SPK_ERR_SINGULAR_PROJECTED && h->spectrum_bad) {
              hi = mid;
            } else {
              return rc2;
            }
          }
          if (found < 0 && lo == 0) return crc;  // no solvable check at all (message kept)
          if (found < 0) {
            // not converged: the factors of the last solvable check
            TRY(check(lo, rho3, &newton));
            d = lo;
          } else {
            d = found;
            converged = true;
          }
          cudaEventRecord(ec1, st);
          TRY(wait_stream(h, st, h->host_wait_s));
          float msb = 0.f;
          cudaEventElapsedTime(&msb, ec0, ec1);
          ms_proj += msb;
          // no resumption after a backtrack: the window is past d
          attempt = kVerifyResumes;
          break;
        }
        TRY(crc);
        cudaEventRecord(ec1, st);
        TRY(wait_stream(h, st, h->host_wait_s));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ec0, ec1);
        ms_proj += ms;
        hd.push_back(d);
        hrel.push_back(rho3[1]);
        if (!std::isfinite(rho3[1])) return fail(h, SPK_ERR_NONFINITE, "non-finite residual estimate at d=%d", d);
        if (o.fixed_d <= 0 && rho3[1] < target) {
          converged = true;
          break;
        }
        last_good = d;
        // mixed forms with an FP64 start: the basis recurrence turns to the
        // form's precision once the estimate is below fp64_until
        if (two_prec() && switch_d == kNever && rho3[1] < o.fp64_until) switch_d = d + 1;
        if (o.check_schedule == SPK_CHECK_ADAPTIVE && o.fixed_d <= 0)
          next_check = next_check_adaptive(hd.data(), hrel.data(), (int)hd.size(), target, o.p, dmax);
      }
      if (d > dmax) d = dmax;
      cudaEventRecord(e1, st);
      TRY(read_flags(h, st, &f));
      TRY(flags_to_status(h, f));
      {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_loop += ms;
      }
      // Y of the last check is in pj_F
      double* Y = static_cast<double*>(h->bufs["pj_F"].p);
      cudaEventRecord(er0, st);
      if (o.method != SPK_METHOD_FULL) {
        TRY(replay_start(S[0], C1use));
        TRY(replay_start(S[1], C2));
      }
      TRY(recover(d, Y, out));
      cudaEventRecord(er1, st);
      TRY(wait_stream(h, st, h->host_wait_s));
      CK(cudaGetLastError());
      TRY(read_flags(h, st, &f));
      TRY(flags_to_status(h, f));
      {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, er0, er1);
        ms_rec += ms;
      }
      if (!verify) break;
      double t3[3] = {0.0, 0.0, 0.0};
      TRY(true_residual(h, A, BT, C1use, C2, r, out->X1_dev, out->X2_dev, out->rank, st, t3));
      true_rel = t3[2];
      if (o.fixed_d > 0 || true_rel < o.tol) break;
      const bool can_resume = converged && d < dmax && attempt < kVerifyResumes;
      converged = false;
      if (!can_resume) break;
      // resume: drop these factors, regenerate U_{d+1} and V_{d+1} (the
      // replay stops at U_d) from the stored coefficients, and aim rho lower
      cudaFree(out->X1_dev);
      cudaFree(out->X2_dev);
      out->X1_dev = out->X2_dev = nullptr;
      out->rank = 0;
      if (o.method != SPK_METHOD_FULL)
        for (int side = 0; side < 2; ++side) arnoldi_basis(S[side], d, true);
      target = std::min(target, rho3[1]) * std::max(0.1, 0.5 * o.tol / true_rel);
      d_start = d + 1;
      last_good = d;
      next_check = o.check_schedule == SPK_CHECK_ADAPTIVE
                       ? next_check_adaptive(hd.data(), hrel.data(), (int)hd.size(), target, o.p, dmax)
                       : d + 1;
      cudaEventRecord(e0, st);
    }
    h->prof.resolve();
    out->iters = d;
    out->converged = converged ? 1 : 0;
    out->rel_rho = rho3[1];
    out->rho = rho3[0];
    out->newton_iters = newton;
    out->n_hist = (int)hd.size();
    out->hist_d_host = (int32_t*)malloc(sizeof(int32_t) * std::max<size_t>(1, hd.size()));
    out->hist_rel_host = (double*)malloc(sizeof(double) * std::max<size_t>(1, hrel.size()));
    for (size_t i = 0; i < hd.size(); ++i) {
      out->hist_d_host[i] = hd[i];
      out->hist_rel_host[i] = hrel[i];
    }
    out->mem_basis_vectors = o.method == SPK_METHOD_FULL
                                 ? (int64_t)2 * (d + 1) * r
                                 : (int64_t)(o.k_left + 1 + o.k_right + 1) * r;
    out->ms_project = ms_proj;
    out->ms_arnoldi = std::max(0.0, ms_loop - ms_proj);
    out->ms_recover = ms_rec;
    out->true_rel_res = true_rel;
    out->switch_d = two_prec() ? (switch_d == kNever ? -1 : switch_d) : 0;
    out->status = (converged || o.fixed_d > 0) ? SPK_OK : SPK_ERR_NOT_CONVERGED;
    return out->status;
  }
};

int validate(spk_handle* h, const spk_csr* A, const spk_csr* BT, const double* C1, const double* C2,
             int r, const spk_opts* o) {
  if (!h) return SPK_ERR_ARG;
  if (!A || !BT || !C1 || !C2 || !o) return fail(h, SPK_ERR_ARG, "null argument");
  if (r < 1 || r > kMaxR) return fail(h, SPK_ERR_ARG, "block width r=%d outside [1, %d]", r, kMaxR);
  if (A->nrows != A->ncols || BT->nrows != BT->ncols || A->nrows < 1 || BT->nrows < 1)
    return fail(h, SPK_ERR_ARG, "operators must be square and non-empty");
  if (!A->rowptr_dev || !A->col_dev || !A->val_dev || !BT->rowptr_dev || !BT->col_dev || !BT->val_dev)
    return fail(h, SPK_ERR_ARG, "null CSR array");
  if (o->k_left < 1 || o->k_right < 1 || o->k_left > kMaxWin || o->k_right > kMaxWin)
    return fail(h, SPK_ERR_ARG, "truncation k must lie in [1, %d]", kMaxWin);
  if (o->maxit < 1 || o->p < 1) return fail(h, SPK_ERR_ARG, "maxit and p must be >= 1");
  if (o->max_newton < 1) return fail(h, SPK_ERR_ARG, "max_newton must be >= 1");
  if (o->same_sketch && A->nrows != BT->nrows)
    return fail(h, SPK_ERR_ARG, "same_sketch needs n1 == n2");
  const int64_t mmax = (int64_t)(o->maxit + 1) * r;
  if (o->method != SPK_METHOD_SKETCHED && o->method != SPK_METHOD_TRUNCATED &&
      o->method != SPK_METHOD_FULL)
    return fail(h, SPK_ERR_ARG, "unknown method");
  if (o->method == SPK_METHOD_FULL && o->precision != SPK_PREC_FP64)
    return fail(h, SPK_ERR_UNSUPPORTED, "the full Arnoldi method is FP64 only");
  if (o->method != SPK_METHOD_SKETCHED) {
    // no sketch
  } else if (o->sketch_kind == SPK_SKETCH_IDENTITY) {
    if (A->nrows < mmax || BT->nrows < mmax)
      return fail(h, SPK_ERR_ARG, "identity sketch needs n >= (maxit+1) r");
  } else if (o->sketch_kind == SPK_SKETCH_SRHT || o->sketch_kind == SPK_SKETCH_DCT) {
    if (o->s < mmax)
      return fail(h, SPK_ERR_ARG, "sketch rows s=%d must be >= (maxit+1) r = %lld", o->s, (long long)mmax);
    if (o->sketch_kind == SPK_SKETCH_DCT && (o->s > A->nrows || o->s > BT->nrows))
      return fail(h, SPK_ERR_ARG, "DCT sketch rows s=%d must be <= n", o->s);
  } else {
    return fail(h, SPK_ERR_ARG, "unknown sketch kind");
  }
  if (o->precision < SPK_PREC_FP64 || o->precision > SPK_PREC_MIXED_BF16)
    return fail(h, SPK_ERR_ARG, "unknown precision");
  return SPK_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

int spk_version(void) { return 100; }

void spk_opts_default(spk_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->k_left = 2;
  o->k_right = 2;
  o->s = 600;
  o->maxit = 300;
  o->p = 1;
  o->sketch_kind = SPK_SKETCH_SRHT;
  o->precision = SPK_PREC_FP64;
  o->check_schedule = SPK_CHECK_EVERY_P;
  o->max_newton = 100;
  o->tol = 1e-8;
  o->trunc_tol = 1e-12;
  o->seed = 0;
}

const char* spk_status_string(int s) {
  switch (s) {
    case SPK_OK: return "ok";
    case SPK_ERR_ARG: return "invalid argument";
    case SPK_ERR_CUDA: return "CUDA error";
    case SPK_ERR_ALLOC: return "device allocation failed";
    case SPK_ERR_BREAKDOWN: return "rank-deficient block (Cholesky breakdown)";
    case SPK_ERR_SINGULAR_PROJECTED: return "projected equation not solvable";
    case SPK_ERR_NONFINITE: return "non-finite value";
    case SPK_ERR_NOT_CONVERGED: return "not converged within maxit";
    case SPK_ERR_TIMEOUT: return "bounded wait expired";
    case SPK_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

int spk_create(spk_handle** out, int device) {
  if (!out) return SPK_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return SPK_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return SPK_ERR_CUDA;
  spk_handle* h = new spk_handle();
  h->device = device;
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&h->flags, sizeof(uint32_t)) != cudaSuccess) {
    delete h;
    return SPK_ERR_ALLOC;
  }
  if (cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    spk_destroy(h);
    return SPK_ERR_CUDA;
  }
  *out = h;
  return SPK_OK;
}

void spk_destroy(spk_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  for (auto& w : h->workers) {
    if (w.st) cudaStreamDestroy(w.st);
    if (w.done) cudaEventDestroy(w.done);
    spk_destroy(w.h);
  }
  h->workers.clear();
  for (auto& kv : h->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  if (h->flags) cudaFree(h->flags);
  if (h->aux) cudaStreamDestroy(h->aux);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  delete h;
}

const char* spk_last_error(spk_handle* h) { return h ? h->err.c_str() : "null handle"; }

void spk_result_free(spk_result* res) {
  if (!res) return;
  if (res->X1_dev) cudaFree(res->X1_dev);
  if (res->X2_dev) cudaFree(res->X2_dev);
  free(res->hist_d_host);
  free(res->hist_rel_host);
  res->X1_dev = res->X2_dev = nullptr;
  res->hist_d_host = nullptr;
  res->hist_rel_host = nullptr;
}

int spk_solve(spk_handle* h, const spk_csr* A, const spk_csr* BT, const double* C1,
              const double* C2, int r, const spk_opts* opts, void* stream, spk_result* out) {
  if (!out) return SPK_ERR_ARG;
  memset(out, 0, sizeof *out);
  out->n1 = A ? A->nrows : 0;
  out->n2 = BT ? BT->nrows : 0;
  int rc = validate(h, A, BT, C1, C2, r, opts);
  if (rc != SPK_OK) {
    out->status = rc;
    return rc;
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPK_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (opts->precision) {
    case SPK_PREC_FP64: {
      Solver<double, double, double> s{h, st, *opts, r};
      rc = s.run(A, BT, C1, C2, out);
      break;
    }
    case SPK_PREC_MIXED_FP32: {
      Solver<float, float, float> s{h, st, *opts, r};
      rc = s.run(A, BT, C1, C2, out);
      break;
    }
    default: {
      Solver<__nv_bfloat16, float, float> s{h, st, *opts, r};
      rc = s.run(A, BT, C1, C2, out);
      break;
    }
  }
  if (rc != SPK_OK && rc != SPK_ERR_NOT_CONVERGED) {
    spk_result_free(out);
    out->rank = 0;
  }
  out->status = rc;
  return rc;
}

int spk_solve_batched(spk_handle* h, int32_t count, const spk_problem* probs,
                      int32_t concurrency, void* stream, spk_result* outs) {
  if (!h || count < 0 || (count > 0 && (!probs || !outs)) || concurrency < 1 || concurrency > 64)
    return SPK_ERR_ARG;
  if (count == 0) return SPK_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPK_ERR_CUDA, "cudaSetDevice failed");
  const int nw = std::min<int>(concurrency, count);
  while ((int)h->workers.size() < nw) {
    spk_handle::Worker w;
    int rc = spk_create(&w.h, h->device);
    if (rc != SPK_OK) return fail(h, rc, "cannot create batched worker");
    if (cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (w.st) cudaStreamDestroy(w.st);
      spk_destroy(w.h);
      return fail(h, SPK_ERR_CUDA, "cannot create batched worker stream");
    }
    w.h->host_wait_s = h->host_wait_s;
    w.h->tensor_gemm = h->tensor_gemm;
    h->workers.push_back(w);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaEventRecord(h->ev_fork, st));
  for (int t = 0; t < nw; ++t) CK(cudaStreamWaitEvent(h->workers[t].st, h->ev_fork, 0));
  std::atomic<int> next{0};
  std::vector<int> status(count, SPK_OK);
  std::vector<std::string> msgs(count);
  std::vector<std::thread> threads;
  threads.reserve(nw);
  for (int t = 0; t < nw; ++t) {
    threads.emplace_back([&, t]() {
      spk_handle::Worker& w = h->workers[t];
      cudaSetDevice(h->device);
      for (;;) {
        const int i = next.fetch_add(1);
        if (i >= count) break;
        const spk_problem& pb = probs[i];
        status[i] = spk_solve(w.h, &pb.A, &pb.BT, pb.C1_dev, pb.C2_dev, pb.r, &pb.opts, w.st,
                              &outs[i]);
        if (status[i] != SPK_OK && status[i] != SPK_ERR_NOT_CONVERGED) msgs[i] = w.h->err;
      }
      cudaEventRecord(w.done, w.st);
    });
  }
  for (auto& th : threads) th.join();
  for (int t = 0; t < nw; ++t) CK(cudaStreamWaitEvent(st, h->workers[t].done, 0));
  for (int i = 0; i < count; ++i)
    if (status[i] != SPK_OK && status[i] != SPK_ERR_NOT_CONVERGED)
      return fail(h, status[i], "instance %d: %s", i, msgs[i].c_str());
  return SPK_OK;
}

int spk_solve_adjoint(spk_handle* h, const spk_csr* AT, const spk_csr* B, const double* G1,
                      const double* G2, int q, const spk_opts* opts, void* stream,
                      spk_result* out) {
  // A^T L + L B^T = G1 G2^T is Eq. (1.1) with coefficients (A^T, B^T): its
  // right Krylov space is K((B^T)^T, G2) = K(B, G2).
  return spk_solve(h, AT, B, G1, G2, q, opts, stream, out);
}

int spk_adjoint_gradients(spk_handle* h, const spk_result* X, const spk_result* L,
                          const double* C1, const double* C2, int r, const spk_csr* A_theta,
                          const spk_csr* B_theta, double* dC1, double* dC2, double* dtheta,
                          void* stream) {
  if (!h || !X || !L || !C1 || !C2 || !dC1 || !dC2) return SPK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int lx = X->rank, ll = L->rank;
  const int n1 = X->n1, n2 = X->n2;
  if (L->n1 != n1 || L->n2 != n2) return fail(h, SPK_ERR_ARG, "solution and adjoint sizes differ");
  if (ll == 0 || lx == 0) {
    CK(cudaMemsetAsync(dC1, 0, sizeof(double) * n1 * r, st));
    CK(cudaMemsetAsync(dC2, 0, sizeof(double) * n2 * r, st));
    if (dtheta) *dtheta = 0.0;
    return wait_stream(h, st, h->host_wait_s);
  }
  // Row-major n x c  ==  column-major c x n with leading dimension c.
  WS(t1, double, "ag_t1", (size_t)ll * r);
  // dC1 = L1 (L2^T C2)
  gemm_f64('N', 'T', ll, r, n2, 1.0, L->X2_dev, ll, C2, r, 0.0, t1, ll, st);
  gemm_f64('T', 'N', r, n1, ll, 1.0, t1, ll, L->X1_dev, ll, 0.0, dC1, r, st);
  // dC2 = L2 (L1^T C1)
  gemm_f64('N', 'T', ll, r, n1, 1.0, L->X1_dev, ll, C1, r, 0.0, t1, ll, st);
  gemm_f64('T', 'N', r, n2, ll, 1.0, t1, ll, L->X2_dev, ll, 0.0, dC2, r, st);
  if (dtheta) {
    // dtheta = -<L, A_theta X + X B_theta>_F
    //        = -trace((L1^T A_theta X1)(X2^T L2)) - trace((L1^T X1)(X2^T B_theta L2))
    WS(M1, double, "ag_M1", (size_t)ll * lx);
    WS(M2, double, "ag_M2", (size_t)lx * ll);
    WS(sc, double, "ag_sc", 2);
    CK(cudaMemsetAsync(sc, 0, 2 * sizeof(double), st));
    if (A_theta) {
      WS(AX, double, "ag_AX", (size_t)n1 * lx);
      spmm_wide_launch(A_theta->rowptr_dev, A_theta->col_dev, A_theta->val_dev, n1, lx, X->X1_dev,
                       AX, st);
      // M1 = L1^T (A_theta X1)  (ll x lx);  M2 = X2^T L2  (lx x ll)
      gemm_f64('N', 'T', ll, lx, n1, 1.0, L->X1_dev, ll, AX, lx, 0.0, M1, ll, st);
      gemm_f64('N', 'T', lx, ll, n2, 1.0, X->X2_dev, lx, L->X2_dev, ll, 0.0, M2, lx, st);
      trace_product_launch(M1, M2, ll, lx, sc, st);
    }
    if (B_theta) {
      WS(BL, double, "ag_BL", (size_t)n2 * ll);
      spmm_wide_launch(B_theta->rowptr_dev, B_theta->col_dev, B_theta->val_dev, n2, ll,
                       L->X2_dev, BL, st);
      // M1 = L1^T X1  (ll x lx);  M2 = X2^T (B_theta L2)  (lx x ll)
      gemm_f64('N', 'T', ll, lx, n1, 1.0, L->X1_dev, ll, X->X1_dev, lx, 0.0, M1, ll, st);
      gemm_f64('N', 'T', lx, ll, n2, 1.0, X->X2_dev, lx, BL, ll, 0.0, M2, lx, st);
      trace_product_launch(M1, M2, ll, lx, sc + 1, st);
    }
    double hv[2] = {0.0, 0.0};
    TRY(d2h(h, hv, sc, sizeof hv, st));
    *dtheta = -(hv[0] + hv[1]);
  }
  TRY(wait_stream(h, st, h->host_wait_s));
  CK(cudaGetLastError());
  return SPK_OK;
}

int spk_true_residual(spk_handle* h, const spk_csr* A, const spk_csr* BT, const double* C1,
                      const double* C2, int r, const spk_result* res, double* out3,
                      void* stream) {
  if (!h) return SPK_ERR_ARG;
  if (!A || !BT || !C1 || !C2 || !res || !out3 || r < 1)
    return fail(h, SPK_ERR_ARG, "spk_true_residual: null argument or r < 1");
  if (A->nrows != res->n1 || BT->nrows != res->n2 || A->nrows != A->ncols ||
      BT->nrows != BT->ncols)
    return fail(h, SPK_ERR_ARG, "spk_true_residual: operator sizes differ from the result's");
  if (res->rank < 0 || (res->rank > 0 && (!res->X1_dev || !res->X2_dev)))
    return fail(h, SPK_ERR_ARG, "spk_true_residual: result holds no factors");
  if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPK_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TRY(true_residual(h, A, BT, C1, C2, r, res->X1_dev, res->X2_dev, res->rank, st, out3));
  CK(cudaGetLastError());
  return SPK_OK;
}

int spk_sketch_draws(spk_handle* h, int64_t n, int32_t s, uint64_t seed, int32_t sketch_id,
                     int32_t* rows, int8_t* signs, void* stream) {
  if (!h || !rows || !signs || n < 1) return SPK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t sb = sketch_draws_scratch_bytes(n, s);
  void* scratch = ws_get(h, "sk_draw_scratch", sb);
  if (!scratch) return fail(h, SPK_ERR_ALLOC, "cannot allocate sketch scratch");
  char e[256] = {0};
  int rc = sketch_draws_launch(n, s, seed, sketch_id, rows, signs, scratch, sb, st, e, sizeof e);
  if (rc != SPK_OK) return fail(h, rc, "%s", e);
  return wait_stream(h, st, h->host_wait_s);
}

int spk_sketch_apply(spk_handle* h, int64_t n, int32_t s, uint64_t seed, int32_t sketch_id,
                     const double* X, int32_t r, double* SX, void* stream) {
  if (!h || !X || !SX || n < 1 || r < 1 || r > kMaxR) return SPK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SketchDev sk;
  sketch_geometry(sk, n, s, 0, (int)sizeof(double), r);
  int32_t* rows = static_cast<int32_t*>(ws_get(h, "sa_rows", sizeof(int32_t) * s));
  int8_t* signs = static_cast<int8_t*>(ws_get(h, "sa_signs", (size_t)n));
  double* scratch = static_cast<double*>(ws_get(h, "sa_scratch", sketch_apply_scratch_bytes(sk, r)));
  if (!rows || !signs || !scratch) return fail(h, SPK_ERR_ALLOC, "cannot allocate sketch buffers");
  int rc = spk_sketch_draws(h, n, s, seed, sketch_id, rows, signs, stream);
  if (rc != SPK_OK) return rc;
  sk.rows = rows;
  sk.signs = signs;
  sketch_apply_launch<double, double>(sk, X, r, SX, scratch, st);
  TRY(wait_stream(h, st, h->host_wait_s));
  CK(cudaGetLastError());
  return SPK_OK;
}

int spk_dct_sketch_draws(spk_handle* h, int64_t n, int32_t s, uint64_t seed, int32_t sketch_id,
                         int32_t* rows, int8_t* signs, void* stream) {
  if (!h || !rows || !signs || n < 1) return SPK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t sb = sketch_draws_scratch_bytes(n, s, n);
  void* scratch = ws_get(h, "sk_draw_scratch", sb);
  if (!scratch) return fail(h, SPK_ERR_ALLOC, "cannot allocate sketch scratch");
  char e[256] = {0};
  int rc = sketch_draws_launch(n, s, seed, sketch_id, rows, signs, scratch, sb, st, e, sizeof e, n);
  if (rc != SPK_OK) return fail(h, rc, "%s", e);
  return wait_stream(h, st, h->host_wait_s);
}

int spk_dct_sketch_apply(spk_handle* h, int64_t n, int32_t s, uint64_t seed, int32_t sketch_id,
                         const double* X, int32_t r, double* SX, void* stream) {
  if (!h || !X || !SX || n < 1 || r < 1 || r > kMaxR || s < 1 || s > n) return SPK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SketchDev sk;
  sk.n = n;
  sk.npad = n;
  sk.s = s;
  sk.is_dct = 1;
  sk.scale = std::sqrt((double)n / (double)s);
  if (!dct_geometry(n, sk.dct))
    return fail(h, SPK_ERR_UNSUPPORTED, "DCT sketch: n=%lld is not f1 f2 with f1, f2 <= 1024 "
                "built from 2, 3, 5", (long long)n);
  int32_t* rows = static_cast<int32_t*>(ws_get(h, "sa_rows", sizeof(int32_t) * s));
  int8_t* signs = static_cast<int8_t*>(ws_get(h, "sa_signs", (size_t)n));
  int32_t* selpos = static_cast<int32_t*>(ws_get(h, "sa_selpos", sizeof(int32_t) * (size_t)n));
  double* cwork = static_cast<double*>(ws_get(h, "sa_dct_work", sizeof(double) * 2 * (size_t)n * r));
  double* tabs = static_cast<double*>(ws_get(h, "sa_dct_tables",
                                             sizeof(double) * dct_table_doubles(n, sk.dct)));
  if (!rows || !signs || !selpos || !cwork || !tabs)
    return fail(h, SPK_ERR_ALLOC, "cannot allocate sketch buffers");
  int rc = spk_dct_sketch_draws(h, n, s, seed, sketch_id, rows, signs, stream);
  if (rc != SPK_OK) return rc;
  dct_tables_launch(n, sk.dct, tabs, st);
  dct_selpos_launch(rows, s, n, selpos, st);
  sk.rows = rows;
  sk.signs = signs;
  sk.selpos = selpos;
  sk.cwork = cwork;
  dct_apply_launch<double>(sk, X, r, SX, cwork, st);
  TRY(wait_stream(h, st, h->host_wait_s));
  CK(cudaGetLastError());
  return SPK_OK;
}

int spk_spmm(spk_handle* h, const spk_csr* A, const double* X, int32_t r, double* Y, void* stream) {
  if (!h || !A || !X || !Y || r < 1) return SPK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (r <= kMaxR) {
    WindowPtrs none{};
    none.nwin = 0;
    spmm_dots_launch<double, double, double>(A->rowptr_dev, A->col_dev, A->val_dev, A->nrows, r, X,
                                             Y, none, nullptr, grid_rows(h, A->nrows), st);
  } else {
    spmm_wide_launch(A->rowptr_dev, A->col_dev, A->val_dev, A->nrows, r, X, Y, st);
  }
  TRY(wait_stream(h, st, h->host_wait_s));
  CK(cudaGetLastError());
  return SPK_OK;
}

int spk_set_tensor_gemm(spk_handle* h, int32_t on) {
  if (!h) return SPK_ERR_ARG;
  h->tensor_gemm = on != 0;
  for (auto& w : h->workers) w.h->tensor_gemm = h->tensor_gemm;
  return SPK_OK;
}

int spk_dense_gemm(spk_handle* h, int32_t engine, char ta, char tb, int32_t M, int32_t N,
                   int32_t K, double alpha, const double* A, int64_t lda, const double* B,
                   int64_t ldb, double beta, double* C, int64_t ldc, void* stream) {
  if (!h) return SPK_ERR_ARG;
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || (ta != 'N' && ta != 'T') ||
      (tb != 'N' && tb != 'T') || (engine != 0 && engine != 1))
    return fail(h, SPK_ERR_ARG, "spk_dense_gemm: bad argument");
  if (lda < (ta == 'N' ? M : K) || ldb < (tb == 'N' ? K : N) || ldc < M)
    return fail(h, SPK_ERR_ARG, "spk_dense_gemm: leading dimension too small");
  if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPK_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(h->flags, 0, sizeof(uint32_t), st));
  if (engine == 0) {
    gemm_f64(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
  } else {
    WS(work, uint8_t, "oz_work", ozaki_work_bytes(M, N, K));
    ozaki_gemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, work, h->flags, st);
  }
  TRY(wait_stream(h, st, h->host_wait_s));
  CK(cudaGetLastError());
  uint32_t f = 0;
  TRY(read_flags(h, st, &f));
  if (f) return fail(h, SPK_ERR_TIMEOUT, "spk_dense_gemm: a bounded wait in the tensor-core GEMM expired");
  return SPK_OK;
}

int spk_sylvester_dense(spk_handle* h, int32_t m, const double* H, const double* G,
                        const double* F, double* Y, int32_t* newton_iters, void* stream) {
  if (!h || m < 1 || !H || !G || !F || !Y) return SPK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WS(Hk, double, "sd_Hk", (size_t)m * m);
  WS(Gk, double, "sd_Gk", (size_t)m * m);
  CK(cudaMemcpyAsync(Hk, H, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(Gk, G, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(Y, F, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(h->flags, 0, sizeof(uint32_t), st));
  int it = 0;
  h->trace_fail = false;
  int rc = sign_solve(h, m, Hk, Gk, Y, 100, st, &it);
  if (rc == SPK_ERR_SINGULAR_PROJECTED && h->trace_fail) {
    // eigenvalues off the open right half plane: spectral splitting (Hk, Gk
    // hold sign(H), sign(G); the right-hand side is copied again)
    CK(cudaMemcpyAsync(Y, F, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, st));
    WS(Fd, double, "sd_F", (size_t)m * m);
    CK(cudaMemcpyAsync(Fd, F, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, st));
    rc = split_solve(h, m, H, G, Hk, Gk, h->neg_h, h->neg_g, Fd, Y, 100, 12345, st, &it);
  }
  if (newton_iters) *newton_iters = it;
  if (rc != SPK_OK) return rc;
  TRY(wait_stream(h, st, h->host_wait_s));
  CK(cudaGetLastError());
  return SPK_OK;
}

int64_t spk_launch_count(void) { return launch_count(); }

int32_t spk_next_check(const int32_t* hist_d, const double* hist_rel, int32_t count, double tol,
                       int32_t p, int32_t dmax) {
  if (!hist_d || !hist_rel || count < 1 || p < 1 || !(tol > 0.0) || dmax < 1) return SPK_ERR_ARG;
  return next_check_adaptive(hist_d, hist_rel, count, tol, p, dmax);
}

int spk_profile_enable(spk_handle* h, int on) {
  if (!h) return SPK_ERR_ARG;
  h->prof.resolve();
  h->prof.on = on != 0;
  for (auto& a : h->prof.acc) a = ProfAcc();
  return SPK_OK;
}

int spk_profile_read(spk_handle* h, int family, const char** name, double* ms, int64_t* launches,
                     int64_t* groups, double* bytes, double* flops) {
  if (!h || family < 0 || family >= F_COUNT) return SPK_ERR_ARG;
  h->prof.resolve();
  const ProfAcc& a = h->prof.acc[family];
  if (name) *name = kFamNames[family];
  if (ms) *ms = a.ms;
  if (launches) *launches = a.launches;
  if (groups) *groups = a.groups;
  if (bytes) *bytes = a.bytes;
  if (flops) *flops = a.flops;
  return SPK_OK;
}

int spk_fp64_peak(spk_handle* h, double* tflops, void* stream) {
  if (!h || !tflops) return SPK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WS(scr, double, "fp64_probe", 4);
  *tflops = fp64_fma_probe(h->sm_count, scr, st);
  CK(cudaGetLastError());
  return SPK_OK;
}

int spk_inspect(spk_handle* h, const char* name, double* dst, int64_t count, int64_t* avail) {
  if (!h || !name) return SPK_ERR_ARG;
  static const char* allowed[] = {"U_T", "V_T", "U_Ht", "V_Ht", "U_hband", "V_hband", "U_beta",
                                  "V_beta", "pj_F", "tr_Y1", "tr_Y2"};
  bool ok = false;
  for (const char* a : allowed) ok = ok || strcmp(a, name) == 0;
  auto it = h->bufs.find(name);
  if (!ok || it == h->bufs.end() || !it->second.p) return fail(h, SPK_ERR_ARG, "no buffer %s", name);
  const int64_t n = (int64_t)(it->second.bytes / sizeof(double));
  if (avail) *avail = n;
  if (dst && count > 0) {
    if (bounded_stream_wait(0, h->host_wait_s) != 0)
      return fail(h, SPK_ERR_TIMEOUT, "inspect: device work did not finish");
    CK(cudaMemcpy(dst, it->second.p, sizeof(double) * std::min(n, count), cudaMemcpyDeviceToHost));
  }
  return SPK_OK;
}

}  // extern "C"
