"""ctypes binding of libspk (include/spk.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module
moves tensors to the device, fills the C structs, calls the C ABI and wraps
library-owned device buffers as torch tensors (copied before release).
There is no CPU fallback: if the library or a GPU is missing the calls raise.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspk.so")

SPK_OK = 0
SPK_ERR_ARG = -1
SPK_ERR_CUDA = -2
SPK_ERR_ALLOC = -3
SPK_ERR_BREAKDOWN = -4
SPK_ERR_SINGULAR_PROJECTED = -5
SPK_ERR_NONFINITE = -6
SPK_ERR_NOT_CONVERGED = -7
SPK_ERR_TIMEOUT = -8
SPK_ERR_UNSUPPORTED = -9

SKETCH = {"srht": 0, "identity": 1, "dct": 2}
PRECISION = {"fp64": 0, "mixed_fp32": 1, "mixed_bf16": 2}
METHOD = {"sketched": 0, "truncated": 1, "full": 2}
CHECK = {"every_p": 0, "adaptive": 1}
INJECT_NAN_C1, INJECT_RANK_DEFICIENT, INJECT_TIMEOUT, INJECT_SINGULAR = 1, 2, 4, 8


class Csr(C.Structure):
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr_dev", C.c_void_p), ("col_dev", C.c_void_p), ("val_dev", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("k_left", C.c_int32), ("k_right", C.c_int32), ("s", C.c_int32),
                ("maxit", C.c_int32), ("p", C.c_int32), ("sketch_kind", C.c_int32),
                ("precision", C.c_int32), ("check_schedule", C.c_int32),
                ("same_sketch", C.c_int32), ("fixed_d", C.c_int32), ("max_newton", C.c_int32),
                ("inject", C.c_uint32), ("tol", C.c_double), ("trunc_tol", C.c_double),
                ("seed", C.c_uint64), ("method", C.c_int32), ("verify", C.c_int32),
                ("fp64_until", C.c_double), ("reserved", C.c_int32 * 4)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("rank", C.c_int32),
                ("n1", C.c_int32), ("n2", C.c_int32), ("n_hist", C.c_int32),
                ("converged", C.c_int32), ("newton_iters", C.c_int32),
                ("rel_rho", C.c_double), ("rho", C.c_double),
                ("X1_dev", C.c_void_p), ("X2_dev", C.c_void_p),
                ("hist_d_host", C.POINTER(C.c_int32)), ("hist_rel_host", C.POINTER(C.c_double)),
                ("mem_basis_vectors", C.c_int64), ("mem_solution_vectors", C.c_int64),
                ("ms_arnoldi", C.c_double), ("ms_project", C.c_double), ("ms_recover", C.c_double),
                ("true_rel_res", C.c_double), ("switch_d", C.c_int32), ("reserved", C.c_int32 * 5)]


class Problem(C.Structure):
    _fields_ = [("A", Csr), ("BT", Csr), ("C1_dev", C.c_void_p), ("C2_dev", C.c_void_p),
                ("r", C.c_int32), ("reserved0", C.c_int32), ("opts", Opts)]


_lib = None


def load() -> C.CDLL:
    """Load libspk.so (built in-tree by paper_2311_16019_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2311_16019_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    P = C.POINTER
    sig = {
        "spk_create": (i32, [P(vp), C.c_int]),
        "spk_destroy": (None, [vp]),
        "spk_last_error": (C.c_char_p, [vp]),
        "spk_status_string": (C.c_char_p, [C.c_int]),
        "spk_version": (C.c_int, []),
        "spk_opts_default": (None, [P(Opts)]),
        "spk_solve": (i32, [vp, P(Csr), P(Csr), vp, vp, C.c_int, P(Opts), vp, P(Result)]),
        "spk_solve_adjoint": (i32, [vp, P(Csr), P(Csr), vp, vp, C.c_int, P(Opts), vp, P(Result)]),
        "spk_adjoint_gradients": (i32, [vp, P(Result), P(Result), vp, vp, C.c_int, P(Csr), P(Csr),
                                        vp, vp, P(dbl), vp]),
        "spk_result_free": (None, [P(Result)]),
        "spk_true_residual": (i32, [vp, P(Csr), P(Csr), vp, vp, C.c_int, P(Result), P(dbl), vp]),
        "spk_set_tensor_gemm": (i32, [vp, i32]),
        "spk_dense_gemm": (i32, [vp, i32, C.c_char, C.c_char, i32, i32, i32, dbl, vp, i64, vp,
                                 i64, dbl, vp, i64, vp]),
        "spk_sketch_draws": (i32, [vp, i64, i32, u64, i32, vp, vp, vp]),
        "spk_sketch_apply": (i32, [vp, i64, i32, u64, i32, vp, i32, vp, vp]),
        "spk_spmm": (i32, [vp, P(Csr), vp, i32, vp, vp]),
        "spk_sylvester_dense": (i32, [vp, i32, vp, vp, vp, vp, P(i32), vp]),
        "spk_inspect": (i32, [vp, C.c_char_p, vp, i64, P(i64)]),
        "spk_launch_count": (i64, []),
        "spk_next_check": (i32, [P(i32), P(dbl), i32, dbl, i32, i32]),
        "spk_profile_enable": (i32, [vp, C.c_int]),
        "spk_profile_read": (i32, [vp, C.c_int, P(C.c_char_p), P(dbl), P(i64), P(i64), P(dbl), P(dbl)]),
        "spk_fp64_peak": (i32, [vp, P(dbl), vp]),
        "spk_solve_batched": (i32, [vp, i32, P(Problem), i32, vp, P(Result)]),
        "spk_dct_sketch_draws": (i32, [vp, i64, i32, u64, i32, vp, vp, vp]),
        "spk_dct_sketch_apply": (i32, [vp, i64, i32, u64, i32, vp, i32, vp, vp]),
        "spk_sketch_apply_static": (i32, [i64, i32, u64, i32, vp, i32, vp, vp, C.c_char_p,
                                          C.c_size_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class SpkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libspk needs a CUDA GPU; none is visible")
    return torch


class DeviceCSR:
    """A CSR matrix held in device memory (int32 indices, float64 values)."""

    def __init__(self, M, device="cuda"):
        torch = _torch()
        M = M.tocsr()
        M.sort_indices()
        self.shape = M.shape
        self.rowptr = torch.as_tensor(M.indptr.astype(np.int32), device=device)
        self.col = torch.as_tensor(M.indices.astype(np.int32), device=device)
        self.val = torch.as_tensor(M.data.astype(np.float64), device=device)
        self.c = Csr(M.shape[0], M.shape[1], M.nnz, self.rowptr.data_ptr(), self.col.data_ptr(),
                     self.val.data_ptr())

    @classmethod
    def from_device(cls, shape, rowptr, col, val) -> "DeviceCSR":
        """Wrap device tensors (int32 rowptr and col, float64 values) that the
        caller keeps alive."""
        self = cls.__new__(cls)
        self.shape = tuple(shape)
        self.rowptr, self.col, self.val = rowptr, col, val
        self.c = Csr(self.shape[0], self.shape[1], int(val.numel()), rowptr.data_ptr(),
                     col.data_ptr(), val.data_ptr())
        return self


class _CAI:
    def __init__(self, ptr: int, shape, typestr="<f8"):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Handle:
    def __init__(self, device: int = 0):
        self.lib = load()
        h = C.c_void_p()
        rc = self.lib.spk_create(C.byref(h), device)
        if rc != SPK_OK:
            raise SpkError(rc, "spk_create failed")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.spk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self) -> str:
        return self.lib.spk_last_error(self.h).decode()


_handles: dict = {}


def handle(device: int = 0) -> Handle:
    if device not in _handles:
        _handles[device] = Handle(device)
    return _handles[device]


@dataclasses.dataclass
class SolveResult:
    status: int
    iters: int
    rank: int
    converged: bool
    rel_rho: float
    rho: float
    X1: object          # torch (n1 x rank) float64 on the device
    X2: object
    hist_d: list
    hist_rel: list
    newton_iters: int
    mem_basis_vectors: int
    mem_solution_vectors: int
    ms_arnoldi: float
    ms_project: float
    ms_recover: float
    true_rel_res: float = -1.0   # relative true residual when verified, else -1
    switch_d: int = 0            # mixed forms: first iteration in mixed precision


def make_opts(*, k=2, k_right=None, s=600, maxit=300, p=1, tol=1e-8, trunc_tol=1e-12, seed=0,
              sketch="srht", precision="fp64", check="every_p", same_sketch=False, fixed_d=0,
              max_newton=100, inject=0, method="sketched", verify=0,
              fp64_until=0.0) -> Opts:
    """The spk_opts struct of include/spk.h from keyword options.

    k, k_right: truncation (window) of the left and right Krylov spaces
        (Eq. (2.4)); k_right defaults to k.
    s: sketch rows (s >= (maxit + 1) r for the sketched method).
    maxit, p, tol: Algorithm 1's iteration cap, check period and stopping
        tolerance on rho / ||beta_1 beta_2^T||_F (Eq. (3.5)).
    trunc_tol: keep the singular values of Y above trunc_tol * sigma_1.
    seed: seed of the sketch draws (SplitMix64 streams).
    sketch: "srht" (Walsh-Hadamard, Section 2.2), "dct" (the paper's
        experiments, Section 6) or "identity".
    precision: "fp64", "mixed_fp32" or "mixed_bf16" (basis storage and
        SpMM; the sketch side stays FP64).
    check: "every_p" (Algorithm 1) or "adaptive" (spk_next_check).
    same_sketch: S_V = S_U (square problems only).
    fixed_d: > 0 runs exactly that many iterations with one check.
    max_newton: cap on sign-function iterations of the projected solve.
    inject: SPK_INJECT_* bits (host-side fault injection, tests only).
    method: "sketched" (Algorithm 1), "truncated" (Algorithm 2) or "full"
        (full block Arnoldi, Section 2.1).
    verify: true-residual check of the returned factors: 0 for the mixed
        forms only, 1 always, -1 never (status NOT_CONVERGED above tol).
    fp64_until: mixed forms: FP64 basis recurrence until a check's relative
        estimate is below this value, the mixed precision after (0: mixed
        from the start).
    """
    o = Opts()
    load().spk_opts_default(C.byref(o))
    o.k_left = k
    o.k_right = k if k_right is None else k_right
    o.s = s
    o.maxit = maxit
    o.p = p
    o.tol = tol
    o.trunc_tol = trunc_tol
    o.seed = seed
    o.sketch_kind = SKETCH[sketch]
    o.precision = PRECISION[precision]
    o.check_schedule = CHECK[check]
    o.same_sketch = int(bool(same_sketch))
    o.fixed_d = fixed_d
    o.max_newton = max_newton
    o.inject = inject
    o.method = METHOD[method]
    o.verify = int(verify)
    o.fp64_until = float(fp64_until)
    return o


def _result_to_py(lib, res: Result, keep_status=(SPK_OK, SPK_ERR_NOT_CONVERGED)) -> SolveResult:
    torch = _torch()
    X1 = X2 = None
    if res.rank > 0 and res.X1_dev:
        X1 = torch.as_tensor(_CAI(res.X1_dev, (res.n1, res.rank)), device="cuda").clone()
        X2 = torch.as_tensor(_CAI(res.X2_dev, (res.n2, res.rank)), device="cuda").clone()
    hd = [res.hist_d_host[i] for i in range(res.n_hist)] if res.hist_d_host else []
    hr = [res.hist_rel_host[i] for i in range(res.n_hist)] if res.hist_rel_host else []
    return SolveResult(res.status, res.iters, res.rank, bool(res.converged), res.rel_rho, res.rho,
                       X1, X2, hd, hr, res.newton_iters, res.mem_basis_vectors,
                       res.mem_solution_vectors, res.ms_arnoldi, res.ms_project, res.ms_recover,
                       res.true_rel_res, res.switch_d)


def _block(C_, device="cuda"):
    torch = _torch()
    t = torch.as_tensor(np.ascontiguousarray(C_), dtype=torch.float64, device=device) \
        if not hasattr(C_, "is_cuda") else C_.to(device=device, dtype=torch.float64)
    if t.dim() == 1:
        t = t[:, None]
    return t.contiguous()


def solve(A, BT, C1, C2, *, device: int = 0, stream=None, raise_on_error: bool = True,
          keep_raw: bool = False, **opts):
    """s-PKSM solve of A X + X B = C1 C2^T; BT = B^T (CSR, scipy or DeviceCSR).

    C1 (n1 x r) and C2 (n2 x r), 1 <= r <= 4, are numpy arrays or torch
    tensors (moved to the device as float64).  `opts` are the keywords of
    make_opts.  Runs on `device` and the current torch stream unless
    `stream` is given.  Returns SolveResult with X = X1 X2^T (device
    tensors; SPK_ERR_NOT_CONVERGED returns the last check's factors with
    converged False); any other error status raises SpkError unless
    raise_on_error is False.  With keep_raw the library-owned Result struct is returned as
    well (the caller then frees it with free_raw); used by the adjoint
    gradients.
    """
    return _solve_entry("spk_solve", A, BT, C1, C2, device, stream, raise_on_error, keep_raw,
                        opts)


def solve_adjoint(AT, B, G1, G2, *, device: int = 0, stream=None, raise_on_error: bool = True,
                  keep_raw: bool = False, **opts):
    """The transposed equation A^T L + L B^T = G1 G2^T by the same solver:
    pass AT = A^T and B itself (the right Krylov space is K(B, G2))."""
    return _solve_entry("spk_solve_adjoint", AT, B, G1, G2, device, stream, raise_on_error,
                        keep_raw, opts)


def adjoint_gradients(xraw: Result, lraw: Result, C1, C2, A_theta=None, B_theta=None,
                      device: int = 0):
    """dC1 = L C2, dC2 = L^T C1 (device tensors) and dtheta =
    -<L, A_theta X + X B_theta>_F (None without derivative operators), from the
    raw results of a solve (X) and of its adjoint solve (L)."""
    torch = _torch()
    h = handle(device)
    c1, c2 = _block(C1), _block(C2)
    dC1 = torch.empty_like(c1)
    dC2 = torch.empty_like(c2)
    dA = None if A_theta is None else (A_theta if isinstance(A_theta, DeviceCSR) else DeviceCSR(A_theta))
    dB = None if B_theta is None else (B_theta if isinstance(B_theta, DeviceCSR) else DeviceCSR(B_theta))
    dth = C.c_double(0.0)
    want = dA is not None or dB is not None
    rc = h.lib.spk_adjoint_gradients(
        h.h, C.byref(xraw), C.byref(lraw), C.c_void_p(c1.data_ptr()), C.c_void_p(c2.data_ptr()),
        c1.shape[1], C.byref(dA.c) if dA is not None else None,
        C.byref(dB.c) if dB is not None else None, C.c_void_p(dC1.data_ptr()),
        C.c_void_p(dC2.data_ptr()), C.byref(dth) if want else None, _stream_ptr())
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return dC1, dC2, (dth.value if want else None)


def _solve_entry(fn, A, BT, C1, C2, device, stream, raise_on_error, keep_raw, opts):
    torch = _torch()
    h = handle(device)
    dA = A if isinstance(A, DeviceCSR) else DeviceCSR(A)
    dB = BT if isinstance(BT, DeviceCSR) else DeviceCSR(BT)
    c1 = _block(C1)
    c2 = _block(C2)
    o = make_opts(**opts)
    res = Result()
    torch.cuda.synchronize()
    rc = getattr(h.lib, fn)(h.h, C.byref(dA.c), C.byref(dB.c), C.c_void_p(c1.data_ptr()),
                            C.c_void_p(c2.data_ptr()), c1.shape[1], C.byref(o),
                            _stream_ptr(stream), C.byref(res))
    if rc not in (SPK_OK, SPK_ERR_NOT_CONVERGED):
        msg = h.error()
        h.lib.spk_result_free(C.byref(res))
        if raise_on_error:
            raise SpkError(rc, msg)
        return SolveResult(rc, 0, 0, False, float("nan"), float("nan"), None, None, [], [], 0,
                           0, 0, 0.0, 0.0, 0.0)
    out = _result_to_py(h.lib, res)
    if keep_raw:
        return out, res
    h.lib.spk_result_free(C.byref(res))
    return out


def solve_batched(problems, *, concurrency: int = 8, device: int = 0, stream=None,
                  raise_on_error: bool = True, opts_list=None, **opts):
    """The batched form: solve independent instances (objects with A, BT, C1,
    C2 as scipy CSR / arrays) by concurrent workers on the device.

    Options are common (**opts) unless opts_list gives one dict per
    instance.  Returns (status, [SolveResult per instance]); an instance that
    failed has X1 = X2 = None and its own status."""
    torch = _torch()
    h = handle(device)
    keep = []
    arr = (Problem * max(1, len(problems)))()
    for i, P in enumerate(problems):
        dA = P.A if isinstance(P.A, DeviceCSR) else DeviceCSR(P.A)
        dB = P.BT if isinstance(P.BT, DeviceCSR) else DeviceCSR(P.BT)
        c1, c2 = _block(P.C1), _block(P.C2)
        keep += [dA, dB, c1, c2]
        o = make_opts(**(opts_list[i] if opts_list is not None else opts))
        arr[i] = Problem(dA.c, dB.c, c1.data_ptr(), c2.data_ptr(), c1.shape[1], 0, o)
    outs = (Result * max(1, len(problems)))()
    torch.cuda.synchronize()
    rc = h.lib.spk_solve_batched(h.h, len(problems), arr, concurrency, _stream_ptr(stream), outs)
    torch.cuda.synchronize()
    results = []
    for i in range(len(problems)):
        if outs[i].status in (SPK_OK, SPK_ERR_NOT_CONVERGED):
            results.append(_result_to_py(h.lib, outs[i]))
        else:
            results.append(SolveResult(outs[i].status, 0, 0, False, float("nan"), float("nan"),
                                       None, None, [], [], 0, 0, 0, 0.0, 0.0, 0.0))
        h.lib.spk_result_free(C.byref(outs[i]))
    msg = h.error() if rc != SPK_OK else ""
    if rc != SPK_OK and raise_on_error:
        raise SpkError(rc, msg)
    return rc, results


def autotune_concurrency(problems, *, candidates=(2, 4, 8, 16), probe_iters: int = 40,
                         device: int = 0, opts_list=None, **opts) -> int:
    """Pick the batched form's worker count by measurement: every candidate
    runs the whole batch for a fixed, short number of iterations (one check
    at the end) and the fastest is returned.  The probe shortens only the
    iteration count; instance sizes, ranks and options stay as given."""
    import time
    torch = _torch()
    base = opts_list if opts_list is not None else [opts] * len(problems)
    probe = []
    for o in base:
        d = max(1, min(probe_iters, o.get("maxit", 300)))
        probe.append(dict(o, fixed_d=d, maxit=d, tol=0.0))
    best, best_t = candidates[0], float("inf")
    for c in candidates:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solve_batched(problems, concurrency=c, device=device, opts_list=probe,
                      raise_on_error=False)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        if t < best_t:
            best, best_t = c, t
    return best


def result_view(sol: "SolveResult") -> Result:
    """A Result struct whose factor pointers view sol.X1, sol.X2 (tensors the
    caller keeps alive), for spk_adjoint_gradients."""
    res = Result()
    res.status, res.iters, res.rank = sol.status, sol.iters, sol.rank
    res.n1 = sol.X1.shape[0] if sol.X1 is not None else 0
    res.n2 = sol.X2.shape[0] if sol.X2 is not None else 0
    res.X1_dev = sol.X1.data_ptr() if sol.X1 is not None else None
    res.X2_dev = sol.X2.data_ptr() if sol.X2 is not None else None
    return res


def true_residual(A, BT, C1, C2, sol: "SolveResult", device: int = 0):
    """(||A X + X B - C1 C2^T||_F, ||C1 C2^T||_F, ratio) for X = sol.X1 sol.X2^T,
    computed on the device by spk_true_residual (BT = B^T)."""
    h = handle(device)
    dA = A if isinstance(A, DeviceCSR) else DeviceCSR(A)
    dB = BT if isinstance(BT, DeviceCSR) else DeviceCSR(BT)
    c1, c2 = _block(C1), _block(C2)
    res = result_view(sol)
    out = (C.c_double * 3)()
    rc = h.lib.spk_true_residual(h.h, C.byref(dA.c), C.byref(dB.c), C.c_void_p(c1.data_ptr()),
                                 C.c_void_p(c2.data_ptr()), c1.shape[1], C.byref(res), out,
                                 _stream_ptr())
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return out[0], out[1], out[2]


def free_raw(res: Result, device: int = 0):
    handle(device).lib.spk_result_free(C.byref(res))


def sketch_draws(n: int, s: int, seed: int, sketch_id: int, device: int = 0):
    torch = _torch()
    h = handle(device)
    rows = torch.empty(s, dtype=torch.int32, device="cuda")
    signs = torch.empty(n, dtype=torch.int8, device="cuda")
    rc = h.lib.spk_sketch_draws(h.h, n, s, seed, sketch_id, C.c_void_p(rows.data_ptr()),
                                C.c_void_p(signs.data_ptr()), _stream_ptr())
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return rows, signs


def sketch_apply(X, s: int, seed: int, sketch_id: int, device: int = 0):
    torch = _torch()
    h = handle(device)
    x = _block(X)
    n, r = x.shape
    SX = torch.empty((r, s), dtype=torch.float64, device="cuda")  # column-major s x r
    rc = h.lib.spk_sketch_apply(h.h, n, s, seed, sketch_id, C.c_void_p(x.data_ptr()), r,
                                C.c_void_p(SX.data_ptr()), _stream_ptr())
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return SX.t()


def dct_sketch_draws(n: int, s: int, seed: int, sketch_id: int, device: int = 0):
    torch = _torch()
    h = handle(device)
    rows = torch.empty(s, dtype=torch.int32, device="cuda")
    signs = torch.empty(n, dtype=torch.int8, device="cuda")
    rc = h.lib.spk_dct_sketch_draws(h.h, n, s, seed, sketch_id, C.c_void_p(rows.data_ptr()),
                                    C.c_void_p(signs.data_ptr()), _stream_ptr())
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return rows, signs


def dct_sketch_apply(X, s: int, seed: int, sketch_id: int, device: int = 0):
    torch = _torch()
    h = handle(device)
    x = _block(X)
    n, r = x.shape
    SX = torch.empty((r, s), dtype=torch.float64, device="cuda")  # column-major s x r
    rc = h.lib.spk_dct_sketch_apply(h.h, n, s, seed, sketch_id, C.c_void_p(x.data_ptr()), r,
                                    C.c_void_p(SX.data_ptr()), _stream_ptr())
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return SX.t()


def spmm(A, X, device: int = 0):
    torch = _torch()
    h = handle(device)
    dA = A if isinstance(A, DeviceCSR) else DeviceCSR(A)
    x = _block(X)
    Y = torch.empty((dA.shape[0], x.shape[1]), dtype=torch.float64, device="cuda")
    rc = h.lib.spk_spmm(h.h, C.byref(dA.c), C.c_void_p(x.data_ptr()), x.shape[1],
                        C.c_void_p(Y.data_ptr()), _stream_ptr())
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return Y


def sylvester_dense(H, G, F, device: int = 0):
    """Y with H Y + Y G^T = F (m x m), by the library's sign-function solver."""
    torch = _torch()
    h = handle(device)
    # column-major buffers: pass transposed contiguous copies
    cm = lambda M: torch.as_tensor(np.asarray(M, dtype=np.float64).T.copy(), device="cuda")
    Hd, Gd, Fd = cm(H), cm(G), cm(F)
    m = Hd.shape[0]
    Y = torch.empty_like(Fd)
    it = C.c_int32(0)
    rc = h.lib.spk_sylvester_dense(h.h, m, C.c_void_p(Hd.data_ptr()), C.c_void_p(Gd.data_ptr()),
                                   C.c_void_p(Fd.data_ptr()), C.c_void_p(Y.data_ptr()),
                                   C.byref(it), _stream_ptr())
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return Y.t().cpu().numpy(), it.value


def set_tensor_gemm(on: bool, device: int = 0):
    """Projected-solve products on the tensor cores (True) or FP64 CUDA cores."""
    h = handle(device)
    rc = h.lib.spk_set_tensor_gemm(h.h, 1 if on else 0)
    if rc != SPK_OK:
        raise SpkError(rc, h.error())


def dense_gemm(A, B, *, ta="N", tb="N", alpha=1.0, beta=0.0, Cin=None, engine="tensor",
               device: int = 0):
    """C = alpha op(A) op(B) + beta Cin in FP64 on the device (spk_dense_gemm):
    engine "fp64" (CUDA cores) or "tensor" (tcgen05, error-free BF16 splitting).
    A, B, Cin are numpy arrays (copied in column-major order); returns C."""
    torch = _torch()
    h = handle(device)
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    M, K = (A.shape if ta == "N" else A.shape[::-1])
    K2, N = (B.shape if tb == "N" else B.shape[::-1])
    if K != K2:
        raise ValueError("inner dimensions differ")
    cm = lambda X: torch.as_tensor(np.asarray(X, dtype=np.float64).T.copy(), device="cuda")
    Ad, Bd = cm(A), cm(B)
    Cd = cm(Cin) if Cin is not None else torch.zeros((N, M), dtype=torch.float64, device="cuda")
    rc = h.lib.spk_dense_gemm(h.h, 0 if engine == "fp64" else 1, ta.encode(), tb.encode(), M, N,
                              K, alpha, C.c_void_p(Ad.data_ptr()), A.shape[0],
                              C.c_void_p(Bd.data_ptr()), B.shape[0], beta,
                              C.c_void_p(Cd.data_ptr()), M, _stream_ptr())
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return Cd.t().cpu().numpy()


def dense_gemm_device(M: int, N: int, K: int, A, lda: int, B, ldb: int, Cm, ldc: int, *,
                      ta="N", tb="N", alpha=1.0, beta=0.0, engine="fp64", device: int = 0,
                      stream=None):
    """Cm = alpha op(A) op(B) + beta Cm on device tensors (column-major views
    given by the leading dimensions), through spk_dense_gemm."""
    h = handle(device)
    rc = h.lib.spk_dense_gemm(h.h, 0 if engine == "fp64" else 1, ta.encode(), tb.encode(), M, N,
                              K, alpha, _ptr(A), lda, _ptr(B), ldb, beta, _ptr(Cm), ldc,
                              _stream_ptr(stream))
    if rc != SPK_OK:
        raise SpkError(rc, h.error())


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def inspect(name: str, device: int = 0) -> np.ndarray:
    """Copy of an internal FP64 buffer of the last solve (see spk_inspect)."""
    h = handle(device)
    avail = C.c_int64(0)
    rc = h.lib.spk_inspect(h.h, name.encode(), None, 0, C.byref(avail))
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    out = np.empty(avail.value, dtype=np.float64)
    rc = h.lib.spk_inspect(h.h, name.encode(), out.ctypes.data_as(C.c_void_p), avail.value,
                           C.byref(avail))
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return out


def launch_count() -> int:
    return int(load().spk_launch_count())


def next_check(hist_d, hist_rel, tol: float, p: int, dmax: int) -> int:
    """The adaptive schedule's next check iteration (spk_next_check; host only)."""
    d = np.ascontiguousarray(hist_d, dtype=np.int32)
    r = np.ascontiguousarray(hist_rel, dtype=np.float64)
    if d.shape != r.shape:
        raise ValueError("hist_d and hist_rel differ in length")
    rc = load().spk_next_check(d.ctypes.data_as(C.POINTER(C.c_int32)),
                               r.ctypes.data_as(C.POINTER(C.c_double)), int(d.size), float(tol),
                               int(p), int(dmax))
    if rc < 0:
        raise SpkError(rc, "spk_next_check: invalid argument")
    return int(rc)


def profile_enable(on: bool = True, device: int = 0):
    h = handle(device)
    h.lib.spk_profile_enable(h.h, int(on))


def profile_read(device: int = 0) -> dict:
    """{family: dict(ms, launches, groups, bytes, flops)} of the enabled profiler."""
    h = handle(device)
    out = {}
    f = 0
    while True:
        name = C.c_char_p()
        ms, by, fl = C.c_double(), C.c_double(), C.c_double()
        la, gr = C.c_int64(), C.c_int64()
        rc = h.lib.spk_profile_read(h.h, f, C.byref(name), C.byref(ms), C.byref(la), C.byref(gr),
                                    C.byref(by), C.byref(fl))
        if rc != SPK_OK:
            break
        out[name.value.decode()] = dict(ms=ms.value, launches=la.value, groups=gr.value,
                                        bytes=by.value, flops=fl.value)
        f += 1
    return out


def fp64_peak(device: int = 0) -> float:
    h = handle(device)
    v = C.c_double()
    rc = h.lib.spk_fp64_peak(h.h, C.byref(v), _stream_ptr())
    if rc != SPK_OK:
        raise SpkError(rc, h.error())
    return v.value


def sketch_apply_static(X, s: int, seed: int, sketch_id: int):
    """S X through the allocation-free entry point (no handle, static scratch)."""
    torch = _torch()
    lib = load()
    x = _block(X)
    n, r = x.shape
    SX = torch.empty((r, s), dtype=torch.float64, device="cuda")
    err = C.create_string_buffer(256)
    rc = lib.spk_sketch_apply_static(n, s, seed, sketch_id, C.c_void_p(x.data_ptr()), r,
                                     C.c_void_p(SX.data_ptr()), _stream_ptr(), err, 256)
    if rc != SPK_OK:
        raise SpkError(rc, err.value.decode())
    return SX.t()
