/*
 * spk.h -- C ABI of libspk, a GB300 (sm_103a) implementation of the
 * sketched-and-truncated polynomial Krylov method (s-PKSM) of Palitta,
 * Schweitzer and Simoncini, "Sketched and truncated polynomial Krylov
 * subspace methods: matrix Sylvester equations" (arXiv 2311.16019), for
 *
 *     A X + X B = C1 C2^T,   A: n1 x n1, B: n2 x n2 sparse, C1: n1 x r,
 *     C2: n2 x r,  r << n                                  (Eq. (1.1)).
 *
 * Conventions for every entry point
 *  - Pointers named *_dev are DEVICE pointers on the handle's device; the
 *    caller owns them and keeps them alive until the call returns.  Pointers
 *    named *_host are host pointers.  Nothing is retained after a call except
 *    the library-owned buffers inside spk_result (see spk_result_free).
 *  - Block vectors (n x r) are ROW-MAJOR: element (i, c) at [i * r + c].
 *  - CSR matrices are 0-based, int32 row pointers and column indices,
 *    float64 values, columns sorted within each row.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls that return scalars or host
 *    data synchronise that stream before returning.
 *  - Return value: SPK_OK (0) or a negative SPK_ERR_* code.  A human-readable
 *    reason is kept per handle (spk_last_error).  No call aborts, traps or
 *    falls back to the CPU: every arithmetic step of the method runs in this
 *    library's CUDA kernels.
 */
#ifndef SPK_H
#define SPK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
    SPK_OK = 0,
    SPK_ERR_ARG = -1,                 /* invalid argument / shape / size       */
    SPK_ERR_CUDA = -2,                /* a CUDA runtime call failed            */
    SPK_ERR_ALLOC = -3,               /* device allocation failed              */
    SPK_ERR_BREAKDOWN = -4,           /* rank-deficient new block (Cholesky)   */
    SPK_ERR_SINGULAR_PROJECTED = -5,  /* projected equation (Eq. (3.4)) not solvable
                                         by the sign iteration (zero pivot or an
                                         eigenvalue off the open right half plane) */
    SPK_ERR_NONFINITE = -6,           /* NaN/Inf met in a reduction            */
    SPK_ERR_NOT_CONVERGED = -7,       /* maxit reached; factors still returned */
    SPK_ERR_TIMEOUT = -8,             /* bounded device/host wait expired      */
    SPK_ERR_UNSUPPORTED = -9          /* option combination not built          */
};

/* ---- option enums ------------------------------------------------------ */
/* SPK_SKETCH_SRHT: subsampled randomized Walsh-Hadamard transform on n'
 * (Section 2.2, N = Hadamard, zero padding); SPK_SKETCH_DCT: the orthonormal
 * DCT-II on n rows as in the paper's experiments (Section 6; n must be
 * f1 f2 with f1, f2 <= 1024 built from 2, 3, 5; s <= n);
 * SPK_SKETCH_IDENTITY: S = I (tests).                                     */
enum { SPK_SKETCH_SRHT = 0, SPK_SKETCH_IDENTITY = 1, SPK_SKETCH_DCT = 2 };
enum { SPK_PREC_FP64 = 0, SPK_PREC_MIXED_FP32 = 1, SPK_PREC_MIXED_BF16 = 2 };
enum { SPK_CHECK_EVERY_P = 0, SPK_CHECK_ADAPTIVE = 1 };
/* SPK_METHOD_SKETCHED: Algorithm 1 (s-PKSM, whitened by the sketch).
 * SPK_METHOD_TRUNCATED: Algorithm 2 (t-PKSM): the same truncated Arnoldi
 * without sketch or whitening; projected equation with the banded H_d, G_d
 * and the residual bound of Proposition 3.1 (Eq. (3.2)); s is ignored.    */
/* SPK_METHOD_FULL: full block Arnoldi (Section 2.1) with the Galerkin
 * projected equation and the exact residual norm; the basis of both spaces
 * is kept ((maxit+1) r length-n vectors each, FP64 only), s is ignored.
 * The comparator of the paper's experiments.                               */
enum { SPK_METHOD_SKETCHED = 0, SPK_METHOD_TRUNCATED = 1, SPK_METHOD_FULL = 2 };
/* host-side fault injection bits for spk_opts.inject (tests only) */
enum {
    SPK_INJECT_NAN_C1 = 1u << 0,      /* treat C1 as containing a NaN          */
    SPK_INJECT_RANK_DEFICIENT = 1u << 1, /* duplicate column 0 of C1 into 1    */
    SPK_INJECT_TIMEOUT = 1u << 2,     /* bounded waits get a zero budget       */
    SPK_INJECT_SINGULAR = 1u << 3     /* make the projected solve report a zero pivot */
};

typedef struct spk_handle spk_handle;

/* CSR operator on the device (caller-owned). */
typedef struct spk_csr {
    int32_t nrows, ncols;
    int64_t nnz;
    const int32_t* rowptr_dev;   /* nrows + 1 */
    const int32_t* col_dev;      /* nnz */
    const double*  val_dev;      /* nnz */
} spk_csr;

/* Options of Algorithm 1 (inputs k, maxit, tol, p, S_U, S_V) plus the
 * implementation's choices.  spk_opts_default fills every field. */
typedef struct spk_opts {
    int32_t k_left;          /* truncation k for K(A, C1): orthogonalise the new
                                block against the last k blocks (Eq. (2.4))    */
    int32_t k_right;         /* truncation k for K(B^T, C2)                    */
    int32_t s;               /* sketch rows (SRHT); ignored for IDENTITY       */
    int32_t maxit;           /* maximum number of iterations d                 */
    int32_t p;               /* check period of Algorithm 1                    */
    int32_t sketch_kind;     /* SPK_SKETCH_*                                   */
    int32_t precision;       /* SPK_PREC_*                                     */
    int32_t check_schedule;  /* SPK_CHECK_EVERY_P or SPK_CHECK_ADAPTIVE        */
    int32_t same_sketch;     /* nonzero: S_V = S_U (needs n1 == n2)            */
    int32_t fixed_d;         /* >0: run exactly this many iterations, one check
                                at the end, tol ignored                         */
    int32_t max_newton;      /* cap on sign-function iterations (a9)           */
    uint32_t inject;         /* SPK_INJECT_* (host-side), 0 in production      */
    double tol;              /* stop when rho / ||beta1 beta2^T||_F < tol      */
    double trunc_tol;        /* keep singular values of Y above trunc_tol*s_1  */
    uint64_t seed;           /* sketch draws (SplitMix64 streams)              */
    int32_t method;          /* SPK_METHOD_*                                   */
    int32_t verify;          /* true-residual check of the returned factors
                                (spk_true_residual) after the solve: 0 = for
                                the mixed forms only (default), 1 = always,
                                -1 = never.  When it runs and the relative
                                true residual exceeds tol, the status is
                                SPK_ERR_NOT_CONVERGED (factors still returned) */
    double fp64_until;       /* mixed forms: the basis recurrence runs in FP64
                                until a check's rho / ||beta1 beta2^T||_F is
                                below this value, in the mixed precision after
                                (the replay switches at the same iteration);
                                0 = mixed precision from the first iteration   */
    int32_t reserved[4];
} spk_opts;

/* Result of a solve.  X1/X2 and the history arrays are library-owned and
 * released by spk_result_free. */
typedef struct spk_result {
    int32_t status;          /* SPK_OK, SPK_ERR_NOT_CONVERGED or an error      */
    int32_t iters;           /* final d                                        */
    int32_t rank;            /* ell: columns of X1 and X2                      */
    int32_t n1, n2;
    int32_t n_hist;          /* number of residual checks                      */
    int32_t converged;
    int32_t newton_iters;    /* sign-function iterations of the last check     */
    double rel_rho;          /* last rho / ||beta1 beta2^T||_F                 */
    double rho;              /* last sketched residual norm (Eq. (3.5))        */
    double* X1_dev;          /* n1 x rank row-major, device                    */
    double* X2_dev;          /* n2 x rank row-major, device                    */
    int32_t* hist_d_host;    /* iteration of each check                        */
    double* hist_rel_host;   /* rho / ||beta1 beta2^T|| at each check          */
    int64_t mem_basis_vectors;    /* length-n vectors of the two windows       */
    int64_t mem_solution_vectors; /* 2 * rank                                  */
    double ms_arnoldi, ms_project, ms_recover;  /* GPU time per phase          */
    double true_rel_res;     /* ||A X + X B - C1 C2^T||_F / ||C1 C2^T||_F of the
                                returned factors when the verification ran
                                (spk_opts.verify), else -1                     */
    int32_t switch_d;        /* mixed forms with fp64_until > 0: first
                                iteration in the mixed precision (0 = from the
                                start, -1 = the whole run stayed FP64)         */
    int32_t reserved[5];
} spk_result;

/* ---- lifetime ---------------------------------------------------------- */
int  spk_create(spk_handle** h, int device);
void spk_destroy(spk_handle* h);
const char* spk_last_error(spk_handle* h);
const char* spk_status_string(int status);
int  spk_version(void);
void spk_opts_default(spk_opts* o);

/* ---- the solver (Algorithm 1) -------------------------------------------
 * spk_solve: the whole s-PKSM path of Algorithm 1 on the device.  A is the
 * left operator (n1 x n1), BT = B^T (n2 x n2) generates K(B^T, C2)
 * (Eq. (1.2)).  C1_dev (n1 x r), C2_dev (n2 x r) row-major device.
 * 1 <= r <= 4.  Returns SPK_OK, SPK_ERR_NOT_CONVERGED (factors of the last
 * check still returned) or an error (out->X1_dev == NULL).               */
int spk_solve(spk_handle* h, const spk_csr* A, const spk_csr* BT,
              const double* C1_dev, const double* C2_dev, int r,
              const spk_opts* opts, void* stream, spk_result* out);

/* spk_solve_adjoint: the transposed equation A^T L + L B^T = G1 G2^T with the
 * same solver (operators A^T and B; L = X1 X2^T on return).  Used for the
 * gradient of a loss of X (differentiate Eq. (1.1)).                      */
int spk_solve_adjoint(spk_handle* h, const spk_csr* AT, const spk_csr* B,
                      const double* G1_dev, const double* G2_dev, int q,
                      const spk_opts* opts, void* stream, spk_result* out);

/* spk_adjoint_gradients: given X = X1 X2^T (solution), L = L1 L2^T (adjoint),
 * C1, C2 and the derivative operators A_theta = dA/dtheta, B_theta = dB/dtheta
 * (CSR, device), writes dC1 = L C2 (n1 x r), dC2 = L^T C1 (n2 x r) row-major
 * device, and *dtheta_host = -<L, A_theta X + X B_theta>_F.               */
int spk_adjoint_gradients(spk_handle* h, const spk_result* X, const spk_result* L,
                          const double* C1_dev, const double* C2_dev, int r,
                          const spk_csr* A_theta, const spk_csr* B_theta,
                          double* dC1_dev, double* dC2_dev, double* dtheta_host,
                          void* stream);

void spk_result_free(spk_result* res);

/* ---- batched form -------------------------------------------------------
 * One instance of Eq. (1.1) for spk_solve_batched: device CSR operators and
 * factors (caller-owned, as for spk_solve), its own r and options.        */
typedef struct spk_problem {
    spk_csr A;               /* left operator, n1 x n1                         */
    spk_csr BT;              /* B^T, n2 x n2                                   */
    const double* C1_dev;    /* n1 x r row-major                               */
    const double* C2_dev;    /* n2 x r row-major                               */
    int32_t r;
    int32_t reserved0;
    spk_opts opts;
} spk_problem;

/* spk_solve_batched: Algorithm 1 for `count` independent instances of
 * uneven sizes.  Up to `concurrency` workers (1..64), each with its own
 * stream and workspace kept in the handle between calls, take the
 * instances in index order, so that small instances share the SMs.  All
 * workers start after the work already queued on `stream`, and `stream`
 * waits for all of them.  outs[i] is filled as by spk_solve (free each with
 * spk_result_free) and outs[i].status is that instance's status.  Returns
 * SPK_OK when every instance ended with SPK_OK or SPK_ERR_NOT_CONVERGED,
 * else the status of the lowest-index instance that did not (its message
 * in spk_last_error(h)).  A worker's results are bitwise those of spk_solve
 * on the same instance.                                                   */
int spk_solve_batched(spk_handle* h, int32_t count, const spk_problem* probs,
                      int32_t concurrency, void* stream, spk_result* outs);

/* spk_true_residual: the true residual of factors X = X1 X2^T (res->X1_dev,
 * res->X2_dev, res->rank columns, as spk_solve returns them) of Eq. (1.1):
 *     out3_host[0] = ||A X + X B - C1 C2^T||_F,
 *     out3_host[1] = ||C1 C2^T||_F,   out3_host[2] = their ratio,
 * computed on the device in the factored form
 * [A X1, X1, -C1] [X2, B^T X2, C2]^T without forming X: the two factors'
 * Gram matrices and the trace of their product are accumulated in
 * double-double arithmetic, so that the cancellation between the three
 * terms does not limit the result (a plain FP64 Gram would resolve it only
 * to ~1e-8 of the terms).  Not a step of Algorithm 1, which stops on the
 * sketched estimate of Eq. (3.5); this is the check that estimate stands
 * for.  A, BT (= B^T), C1, C2 as for spk_solve.  SPK_ERR_ARG for null
 * pointers or sizes that differ from the result's.  Synchronises `stream`. */
int spk_true_residual(spk_handle* h, const spk_csr* A, const spk_csr* BT,
                      const double* C1_dev, const double* C2_dev, int r,
                      const spk_result* res, double* out3_host, void* stream);

/* ---- single steps, for parity tests ----------------------------------- */
/* Sketch draws (Section 2.2; SplitMix64 streams as documented in the
 * library): rows_dev[s] ascending in [0, n'), n' = 2^ceil(log2 n), and
 * signs_dev[n] in {-1, +1}.                                               */
int spk_sketch_draws(spk_handle* h, int64_t n, int32_t s, uint64_t seed,
                     int32_t sketch_id, int32_t* rows_dev, int8_t* signs_dev,
                     void* stream);
/* SX = S X with S[j,i] = e_i (-1)^popcount(rho_j & i) / sqrt(s);
 * X_dev n x r row-major, SX_dev s x r column-major.                       */
int spk_sketch_apply(spk_handle* h, int64_t n, int32_t s, uint64_t seed,
                     int32_t sketch_id, const double* X_dev, int32_t r,
                     double* SX_dev, void* stream);
/* The DCT sketch of the paper's experiments (Section 6):
 * SX = sqrt(n/s) (N E X)[rows, :], N the orthonormal DCT-II on the n rows,
 * rows drawn over [0, n) (same SplitMix64 streams as the SRHT), signs as for
 * the SRHT.  X_dev n x r row-major, SX_dev s x r column-major; n must be
 * f1 f2 with f1, f2 <= 1024 built from the factors 2, 3, 5
 * (SPK_ERR_UNSUPPORTED otherwise), 1 <= s <= n.                           */
int spk_dct_sketch_draws(spk_handle* h, int64_t n, int32_t s, uint64_t seed,
                         int32_t sketch_id, int32_t* rows_dev, int8_t* signs_dev,
                         void* stream);
int spk_dct_sketch_apply(spk_handle* h, int64_t n, int32_t s, uint64_t seed,
                         int32_t sketch_id, const double* X_dev, int32_t r, double* SX_dev,
                         void* stream);
/* Y = A X for CSR A and X_dev (ncols x r row-major), Y_dev (nrows x r):
 * the product A U_d that starts each step of Algorithm 1 (Eq. (2.4)), any
 * r >= 1.  SPK_ERR_ARG for null pointers or r < 1.                        */
int spk_spmm(spk_handle* h, const spk_csr* A, const double* X_dev, int32_t r,
             double* Y_dev, void* stream);
/* Small dense Sylvester solve H Y + Y G^T = F (column-major m x m, device)
 * by the scaled Newton sign iteration: the projected equation of Eq. (3.4)
 * with H = H~_d, G = G~_d.  Y_dev m x m column-major; *newton_iters_host
 * receives the Newton steps taken.  SPK_ERR_SINGULAR_PROJECTED when a pivot
 * vanishes or the spectra are not in the open right half plane.          */
int spk_sylvester_dense(spk_handle* h, int32_t m, const double* H_dev,
                        const double* G_dev, const double* F_dev, double* Y_dev,
                        int32_t* newton_iters_host, void* stream);

/* Dense FP64 product C = alpha op(A) op(B) + beta C (column-major, op = 'N'
 * or 'T', device pointers), by one of the library's two engines: engine 0,
 * the FP64 CUDA-core GEMM; engine 1, the tcgen05 tensor cores by
 * error-free splitting of the FP64 operands into BF16 slices (Ozaki et al.,
 * 2012): eight balanced base-2^7 digits per entry, scaled per row of op(A)
 * and column of op(B), level sums exact in the FP32 accumulators, combined
 * exactly in 64-bit integers and converted to FP64 once.  These are the
 * products of the projected solve (Eq. (3.4)) and of the factor recovery;
 * exposed for parity tests and for small device-side products of the
 * binding.  SPK_ERR_ARG for bad sizes or pointers.  Synchronises `stream`. */
int spk_dense_gemm(spk_handle* h, int32_t engine, char ta, char tb, int32_t M, int32_t N,
                   int32_t K, double alpha, const double* A_dev, int64_t lda,
                   const double* B_dev, int64_t ldb, double beta, double* C_dev, int64_t ldc,
                   void* stream);

/* spk_set_tensor_gemm: whether the handle's solves run their large dense
 * FP64 products on the tensor cores (on = 1, the default) or on the FP64
 * CUDA cores (on = 0): the whitening products against Q (Proposition 2.1,
 * from 256 columns of Q and 1024 sketch rows), the Gauss-Jordan trailing
 * updates and right-hand-side products of the projected solve (Eq. (3.4))
 * and the factor recovery.  Both are FP64-accurate; the switch exists for
 * comparison.  Applies to the handle's batched workers too.               */
int spk_set_tensor_gemm(spk_handle* h, int32_t on);

/* ---- allocation-free variant ----------------------------------------------
 * spk_sketch_apply_static: the same S X as spk_sketch_apply (same kernels,
 * same output layout), without a handle and without allocating device
 * memory, for callers that cannot let a library call cudaMalloc (a process
 * that reserved the device heap for its own pool, a framework whose
 * allocator must remain the only owner of device memory, a service with a
 * fixed, pre-proven memory budget).  No counterpart in the paper: it is an
 * interface variant of the sketch step.  Working memory is one file-scope
 * device array of 10.1 MiB per device, held until the process exits.
 * Limits: n <= 2^20, 1 <= r <= 4, n' r <= 2^20 (n' = 2^ceil(log2 n)),
 * 1 <= s <= min(n', 32768); beyond them SPK_ERR_ARG and a message in err
 * (errlen bytes, may be NULL).  The first call on a device (that device
 * current) looks up the array's device address and creates one event.
 * Every call waits on the host for `stream` (SPK_ERR_TIMEOUT after 600 s),
 * so it must not be called while `stream` is being captured into a CUDA
 * graph.  All calls on a device share the array and leave their data in
 * it; calls whose device work overlaps race and must be ordered by the
 * caller.  After a SPK_ERR_TIMEOUT the array stays in use until that call's
 * kernels finish: the next call on the device waits for them (bounded, else
 * SPK_ERR_TIMEOUT again).                                                 */
int spk_sketch_apply_static(int64_t n, int32_t s, uint64_t seed, int32_t sketch_id,
                            const double* X_dev, int32_t r, double* SX_dev, void* stream,
                            char* err, size_t errlen);

/* ---- measurement --------------------------------------------------------
 * spk_launch_count: number of CUDA kernel launches issued by the library
 * since it was loaded (all handles).                                      */
int64_t spk_launch_count(void);

/* spk_next_check: the adaptive check schedule (SPK_CHECK_ADAPTIVE), as the
 * solver applies it, exposed as a host-only function (no device, no handle).
 * hist_d[0..count) are the iterations at which the residual estimate was
 * computed (increasing) and hist_rel their relative estimates
 * rho / ||beta_1 beta_2^T||_F (Eq. (3.5)).  With d = hist_d[count - 1]:
 * while count < 3 or the last three estimates do not strictly decrease, the
 * next check is 2 d; otherwise the line through the last two (d, log rho)
 * points reaches log tol after `need` more iterations, and the next check is
 * d + ceil(0.7 * 1.05 * need) rounded up to a multiple of p, and at least
 * d + p.  The result is then min(result, dmax), raised to d + 1 if that
 * is smaller (the solver's last check is at dmax).  Returns SPK_ERR_ARG
 * for null pointers, count < 1, p < 1, tol <= 0 or dmax < 1.  Not in the
 * paper, which checks every p iterations.                                 */
int32_t spk_next_check(const int32_t* hist_d, const double* hist_rel, int32_t count,
                       double tol, int32_t p, int32_t dmax);
/* spk_profile_enable: turn per-family timing on/off for this handle and reset
 * the counters.  When on, CUDA events are recorded on the launching stream
 * around every group of launches of a kernel family; spk_profile_read
 * returns, for family index 0, 1, ... (18 families, indices 0..17, in
 * this version; SPK_ERR_ARG past the last), its name, total GPU
 * milliseconds, kernel launches, timed groups, and the ALGORITHMIC bytes and
 * flops of those launches (the minimum the step must move/compute).      */
int spk_profile_enable(spk_handle* h, int on);
int spk_profile_read(spk_handle* h, int family, const char** name, double* ms,
                     int64_t* launches, int64_t* groups, double* bytes, double* flops);
/* spk_fp64_peak: measured FP64 FMA rate of the handle's device (TFLOP/s),
 * from a kernel of independent FMA chains on every SM (no paper counterpart;
 * the denominator of the FP64-ALU roofline).                              */
int spk_fp64_peak(spk_handle* h, double* tflops, void* stream);

/* Copy an internal FP64 buffer of the handle's last solve to the host, for
 * element-wise parity tests of single steps: "U_T"/"V_T" (whitening factors
 * T_U, T_V, (maxit+1) r square, column-major), "U_Ht"/"V_Ht" (projected
 * matrices H~, G~, same layout), "U_hband"/"V_hband" (Hessenberg blocks:
 * per iteration d, k+1 blocks r x r row-major; block q is h_{d-k+1+q, d},
 * block k is h_{d+1,d}), "U_beta"/"V_beta" (r x r), "pj_F" (the projected
 * solution Y of the last check, m x m column-major), "tr_Y1"/"tr_Y2" (the
 * recovery coefficients W1 = T_U^{-1} Y1, W2 = T_V^{-1} Y2, m x rank
 * column-major).  count = doubles wanted;
 * *avail_out receives the buffer's size in doubles.  SPK_ERR_ARG if the
 * name is unknown.                                                        */
int spk_inspect(spk_handle* h, const char* name, double* dst_host, int64_t count,
                int64_t* avail_out);

#ifdef __cplusplus
}
#endif
#endif /* SPK_H */
