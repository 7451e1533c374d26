#!/usr/bin/env python
"""Benchmark of the s-PKSM solver (libspk) on GB300.

Metric: solves per second to relative residual 1e-8 (rho / ||beta1 beta2^T||
< 1e-8, the stopping test of Algorithm 1) on the 2-D convection-diffusion
workload: A = -Lap + 10 (x, y).grad, B = -Lap + 10 (y, -x).grad, upwind
5-point stencil on a 512 x 512 grid (n = 262144, CSR), r = 4, k = 4, C1, C2
i.i.d. N(0,1) (seed 1), sketch s = 12000 rows (2 x the maximal basis size
r * maxit), maxit = 1500, checks every p = 20 iterations on the adaptive
schedule.  Both the FP64 form (the JSON `value`) and the mixed form (FP32
basis and SpMM, FP64 whitening / projected solve / residual) are timed.

One step = one whole solve (every step of the hot path: basis, sketch,
whitening, projected solves, truncation, two-pass recovery) from
device-resident inputs.  `e2e` repeats the measurement through the public
API with pinned host buffers: the host->device copy of the CSR operators and
C1, C2 and the device->host copy of X1, X2 are inside the timed region.

N > 1 (torchrun): every rank solves its own replica (the method has no
data-parallel exchange; replicas only) and `value` = all ranks' solves / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "cd2d_512_r4"
def metric_name(tol: float) -> str:
    m, e = f"{tol:.0e}".split("e")
    return f"solves/s to rel. residual {m}e{int(e)} (FP64 form)"
SOLVER = dict(k=4, s=12000, maxit=1500, p=20, tol=1e-8, seed=0, check="adaptive",
              trunc_tol=1e-12)


def workload_config(P, opts, world):
    mmax = (opts["maxit"] + 1) * P.r
    ws = 2 * 8 * (opts["s"] * mmax + 2 * mmax * mmax)     # Q, T, H~ of both sides
    l2 = (f"sketch-side working set (Q, T, H~) {ws / 1e9:.2f} GB, larger than L2; no flush"
          if ws > 129e6 else
          f"sketch-side working set {ws / 1e6:.0f} MB fits L2; no flush")
    return {"workload": P.name, "n": P.n1, "nnz": int(P.A.nnz), "r": P.r, **opts,
            "parallelism": "replicas" if world > 1 else "single", "l2": l2}


def solver_opts(args):
    o = dict(SOLVER, s=args.s, maxit=args.maxit, p=args.p, k=args.k, tol=args.tol,
             check=args.check)
    if args.method != "sketched":
        o["method"] = args.method
    if args.sketch != "srht":
        o["sketch"] = args.sketch
    if args.fixed_d > 0:
        o.update(fixed_d=args.fixed_d, tol=0.0)
    return o


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="spk", choices=["spk", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--maxit", type=int, default=SOLVER["maxit"])
    ap.add_argument("--s", type=int, default=SOLVER["s"])
    ap.add_argument("--p", type=int, default=SOLVER["p"])
    ap.add_argument("--k", type=int, default=SOLVER["k"])
    ap.add_argument("--tol", type=float, default=SOLVER["tol"])
    ap.add_argument("--method", default="sketched", choices=["sketched", "truncated", "full"])
    ap.add_argument("--sketch", default="srht", choices=["srht", "dct"])
    ap.add_argument("--check", default=SOLVER["check"], choices=["adaptive", "every_p"])
    ap.add_argument("--fixed-d", type=int, default=0,
                    help="run exactly this many iterations (small profiling cases)")
    ap.add_argument("--forms", default="fp64,mixed_fp32")
    ap.add_argument("--engine", default="tensor", choices=["tensor", "fp64"],
                    help="dense products of the projected solve: tensor cores (error-free "
                         "splitting) or FP64 CUDA cores")
    ap.add_argument("--fp64-until", type=float, default=1e-4,
                    help="mixed forms: FP64 basis until the relative estimate is below this")
    ap.add_argument("--oracle-sample", default=None,
                    help=argparse.SUPPRESS)   # internal: one oracle sample in a fresh process
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-iters", type=int, default=40)
    ap.add_argument("--kernel-case", default=None, choices=["gje"],
                    help="run one small isolated case of a kernel family (for ncu captures)")
    ap.add_argument("--m", type=int, default=4200, help="size of the dense case")
    ap.add_argument("--engines", default="fp64,tensor",
                    help="dense case: engines to run (fp64, tensor)")
    ap.add_argument("--batched", action="store_true",
                    help="time the batched form on the 64-instance workload instead")
    ap.add_argument("--concurrency", type=int, default=0,
                    help="batched-form workers (0: chosen by the autotuner)")
    return ap.parse_args()


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return (d.get("hbm_gbs"), d.get("bf16_tflops"), "measured",
                d.get("bf16_tflops_sustained") or d.get("bf16_tflops"))
    return 6800.0, 1900.0, "fallback", 1700.0


def fp64_alu_peak(sm_count: int):
    """FP64 ALU peak in TFLOP/s from unit counts and clocks: each SM retires
    2 FP64 FMAs per clock (4 flop), at the maximum SM clock."""
    mhz = 2070.0
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return sm_count * 4 * mhz * 1e6 / 1e12, mhz


def dist_setup(n_gpus, backend: str = "nccl"):
    """One process per GPU (torchrun environment); replicas of the solve,
    no data-path collective.  The backend is NCCL on GPUs (gloo in the CPU
    tests of this helper)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, value: float) -> float:
    if pg is None:
        return value
    import torch
    dev = "cpu" if pg.get_backend() == "gloo" else "cuda"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, steps: int, ms_max: float) -> float:
    """Whole-job solves/s of `world` replicas, each timing `steps` solves,
    over the slowest rank's time."""
    return world * steps / (ms_max * 1e-3)


# families that time a composite of several kernels (the wall time of the
# two concurrent inversions of a sign step, whose trailing products run on
# the tensor cores): reported in the table, not chosen for the roofline
COMPOSITE_FAMILIES = ("gje_invert",)
# with the tensor-core engine: FP64 products emulated on the tensor cores
# (36 BF16 slice products per FP64 product), and the whitening products,
# which read BF16-sliced copies of Q and are bound by HBM
TENSOR_FAMILIES = ("gje_update_H", "gemm_f64", "x_accumulate")
SLICED_FAMILIES = ("whiten_qt_dot", "whiten_q_update")
OZAKI_PAIRS = 36


def family_bound(fam: str, p: dict, engine: str, balance: float) -> str:
    if engine == "tensor" and fam in TENSOR_FAMILIES:
        return "tensor"
    if engine == "tensor" and fam in SLICED_FAMILIES:
        return "hbm"
    return "alu" if p["flops"] / max(p["bytes"], 1.0) > balance else "hbm"


def pick_roofline(prof: dict, hbm_gbs: float, fp64_tflops: float, tensor_fp64_tflops: float = 0.0,
                  engine: str = "fp64"):
    """Dominant single-kernel family by GPU time, against the peak of the unit
    that bounds it: the FP64 pipe (derived), HBM (measured copy), or the
    tensor cores' FP64-equivalent rate (measured sustained BF16 rate / 36)."""
    if not prof:
        return None, {}
    cands = [k for k in prof if k not in COMPOSITE_FAMILIES] or list(prof)
    fam = max(cands, key=lambda k: prof[k]["ms"])
    p = prof[fam]
    ms_per_launch_group = p["ms"] / max(1, p["groups"])
    secs = p["ms"] * 1e-3
    balance = fp64_tflops * 1e12 / (hbm_gbs * 1e9)   # flop per byte
    bound = family_bound(fam, p, engine, balance)
    if bound == "alu":
        achieved = p["flops"] / secs / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_tflops, "unit": "TFLOP/s",
                "frac": achieved / fp64_tflops}
    elif bound == "tensor":
        achieved = p["flops"] / secs / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": tensor_fp64_tflops,
                "unit": "TFLOP/s", "frac": achieved / tensor_fp64_tflops}
    else:
        achieved = p["bytes"] / secs / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s",
                "frac": achieved / hbm_gbs}
    roof.update({"kernel": fam, "traffic": None, "launches": p["launches"],
                 "avg_launch_ms": p["ms"] / max(1, p["launches"]),
                 "avg_group_ms": ms_per_launch_group,
                 "algorithmic_bytes_per_launch": p["bytes"] / max(1, p["launches"]),
                 "algorithmic_flops_per_launch": p["flops"] / max(1, p["launches"])})
    table = {k: {"ms": round(v["ms"], 3), "share": round(v["ms"] / max(1e-9, sum(x["ms"] for x in prof.values())), 4),
                 "launches": v["launches"],
                 "GBps": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1),
                 "TFLOPs": round(v["flops"] / max(v["ms"], 1e-9) / 1e9, 4),
                 "bound": family_bound(k, v, engine, fp64_tflops * 1e3 / hbm_gbs)}
             for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]) if v["ms"] > 0}
    return roof, table


# --------------------------------------------------------------------- accuracy of a result
def _lowrank_fro(L, R):
    """||L R^T||_F from the triangular factors of L and R (X is never formed)."""
    _, Ra = np.linalg.qr(L, mode="reduced")
    _, Rb = np.linalg.qr(R, mode="reduced")
    return float(np.linalg.norm(Ra @ Rb.T))


# --------------------------------------------------------------------- CPU oracle sample
def oracle_sample(P, opts, iters: int, hist_d, r: int):
    """Time the oracle (FP64 NumPy/SciPy, as it stands) on a bounded sample of
    the workload and extrapolate to one full solve with the GPU's schedule.

    Sample: `iters` Arnoldi + sketch + whitening iterations of the oracle
    (per-iteration times fitted by a + b d with a, b >= 0, since the
    whitening cost grows with d), one projected Sylvester solve at
    d = iters, and the oracle's Bartels-Stewart routine on a dense pair of
    order m1 = 1200 (its cost, scaled by (m / m1)^3, is the cost of a check
    at order m).  Full solve = sum over d <= D of (a + b d) + sum over the
    GPU run's check iterations of the scaled projected-solve time.
    """
    import numpy as np
    import scipy.linalg as sl
    from oracle import spkms as SP

    U = SP._init_side(P.A, P.C1, opts["k"], SP.Sketch(P.n1, opts["s"], opts["seed"], 0), False)
    V = SP._init_side(P.BT, P.C2, opts["k"], SP.Sketch(P.n2, opts["s"], opts["seed"], 1), False)
    ts = []
    t_all = time.perf_counter()
    for d in range(1, iters + 1):
        t0 = time.perf_counter()
        SP._arnoldi_step(U, d)
        SP._arnoldi_step(V, d)
        ts.append(time.perf_counter() - t0)
    m0 = iters * r
    Ht, _ = SP.projected_matrix(U, iters)
    Gt, _ = SP.projected_matrix(V, iters)
    F = np.zeros((m0, m0))
    F[:r, :r] = U.beta @ V.beta.T
    t0 = time.perf_counter()
    sl.solve_sylvester(Ht, Gt.T, F)
    tproj = time.perf_counter() - t0
    m1 = 1200
    rng = np.random.default_rng(5)
    H1 = rng.standard_normal((m1, m1)) / np.sqrt(m1) + 4.0 * np.eye(m1)
    G1 = rng.standard_normal((m1, m1)) / np.sqrt(m1) + 4.0 * np.eye(m1)
    F1 = np.zeros((m1, m1))
    F1[:r, :r] = 1.0
    t0 = time.perf_counter()
    sl.solve_sylvester(H1, G1.T, F1)
    tproj1 = time.perf_counter() - t0
    sample_s = time.perf_counter() - t_all
    dd = np.arange(1, iters + 1, dtype=np.float64)
    b, a = np.polyfit(dd, np.array(ts), 1)
    if b < 0.0:
        b, a = 0.0, float(np.mean(ts))
    a = max(a, 0.0)
    D = max(hist_d) if hist_d else iters
    t_iters = a * D + b * D * (D + 1) / 2.0
    t_checks = sum(tproj1 * ((c * r) / m1) ** 3 for c in (hist_d or [D]))
    total = t_iters + t_checks
    return {"solves_per_s": 1.0 / total, "seconds_per_solve": total, "sample_seconds": sample_s,
            "iters_sampled": iters, "extrapolated_to_d": int(D), "checks": len(hist_d or [D]),
            "t_iter_first_last": [float(ts[0]), float(ts[-1])], "t_proj_m0": tproj, "m0": m0,
            "t_proj_m1": tproj1, "m1": m1, "fit_a_b": [float(a), float(b)]}


def oracle_sample_fresh(workload: str, opts: dict, iters: int, hist_d, r: int) -> dict:
    """oracle_sample in a fresh Python process with the BLAS thread count
    pinned to the host's cores, so that the reference arm and the
    cpu_baseline leg time the same program under the same conditions (in
    the GPU arm's process, the CUDA runtime and torch's own thread pool
    share the cores with OpenBLAS)."""
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[var] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    spec = json.dumps({"workload": workload, "opts": opts, "iters": iters,
                       "hist": list(hist_d), "r": r})
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", spec],
                         capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1]
    res = json.loads(line)
    res["cores"] = cores
    return res


def run_oracle_sample(spec_json: str):
    from paper_2311_16019_gb300 import inputs as I
    spec = json.loads(spec_json)
    P = I.workload(spec["workload"])
    res = oracle_sample(P, spec["opts"], spec["iters"], spec["hist"], spec["r"])
    print(json.dumps(res), flush=True)


# --------------------------------------------------------------------- main arms
def run_reference(args, rank, world, pg):
    if rank != 0:
        return
    from paper_2311_16019_gb300 import inputs as I
    P = I.workload(args.workload)
    opts = solver_opts(args)
    # schedule to extrapolate to: the checks the adaptive schedule makes on
    # this workload (the oracle's residual history is the GPU's, so it would
    # check at the same iterations: 20, 40, 80, 400, 900 on 512^2 with r = 4);
    # other workloads: a doubling schedule up to 300.
    hist = {"cd2d_512_r4": [20, 40, 80, 400, 900]}.get(args.workload, [20, 40, 80, 160, 300])
    D = hist[-1]
    times = []
    for step in range(args.warmup + args.steps):
        res = oracle_sample_fresh(args.workload, opts, args.cpu_sample_iters, hist, P.r)
        if step >= args.warmup:
            times.append(res["solves_per_s"])
    value = statistics.median(times)
    line = {"impl": "reference", "metric": metric_name(opts["tol"]),
            "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": workload_config(P, opts, 1),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": res["cores"],
                             "kind": "oracle", "sample": f"{args.cpu_sample_iters} oracle "
                             f"iterations + projected solves at m={res['m0']} and m={res['m1']} "
                             f"per step, extrapolated to d={D} (fresh process, BLAS threads "
                             f"= {res['cores']})"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_spk(args, rank, world, local, pg):
    import numpy as np
    import torch
    from paper_2311_16019_gb300 import build, inputs as I, spk

    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    barrier(pg)
    spk.load()
    spk.set_tensor_gemm(args.engine == "tensor", local)
    P = I.workload(args.workload)
    opts = solver_opts(args)
    dA, dB = spk.DeviceCSR(P.A), spk.DeviceCSR(P.BT)
    c1 = torch.as_tensor(P.C1, device="cuda")
    c2 = torch.as_tensor(P.C2, device="cuda")
    hbm, bf16, peak_src, bf16_sus = measured_peaks()
    fp64 = spk.fp64_peak(local)
    forms = [f for f in args.forms.split(",") if f]
    per_form = {}
    sampler = ClockSampler(local)
    first = None
    for form in forms:
        fopts = dict(opts)
        if form != "fp64":
            fopts["fp64_until"] = args.fp64_until
        for _ in range(args.warmup):
            spk.solve(dA, dB, c1, c2, precision=form, device=local,
                      raise_on_error=form == forms[0], **fopts)
        torch.cuda.synchronize()
        barrier(pg)
        # timed with the library's per-family profiler off (its events would
        # add to the time); the family table comes from an untimed repeat
        spk.profile_enable(False, local)
        launches0 = spk.launch_count()
        if form == forms[0]:
            sampler.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(pg)
        ev0.record()
        results = []
        for _ in range(args.steps):
            results.append(spk.solve(dA, dB, c1, c2, precision=form, device=local,
                                     raise_on_error=form == forms[0], **fopts))
        ev1.record()
        torch.cuda.synchronize()
        barrier(pg)
        ms = ev0.elapsed_time(ev1)
        launches = spk.launch_count() - launches0
        clocks = sampler.stop() if form == forms[0] else None
        ms_max = max_over_ranks(pg, ms)
        g = results[-1]
        if g.X1 is None:
            # a later form that stopped with an error (reported, not timed as a solve)
            per_form[form] = dict(status=g.status, ms_per_step=ms_max / args.steps)
            continue
        prof = None
        if form == forms[0]:
            spk.profile_enable(True, local)
            spk.solve(dA, dB, c1, c2, precision=form, device=local, **fopts)
            torch.cuda.synchronize()
            prof = spk.profile_read(local)
            spk.profile_enable(False, local)
        tres = g.true_rel_res if g.true_rel_res >= 0 else \
            spk.true_residual(dA, dB, c1, c2, g, device=local)[2]
        X1, X2 = g.X1.cpu().numpy(), g.X2.cpu().numpy()
        per_form[form] = dict(ms_per_step=ms_max / args.steps,
                              solves_per_s=replica_throughput(world, args.steps, ms_max),
                              iters=g.iters, rank=g.rank, converged=g.converged,
                              rel_rho=g.rel_rho, true_rel_residual=tres, checks=g.hist_d,
                              ms_phases=dict(arnoldi=g.ms_arnoldi, project=g.ms_project,
                                             recover=g.ms_recover),
                              gpu_launches=launches, clocks=clocks, prof=prof, X=(X1, X2),
                              status=g.status)
        if form != "fp64":
            per_form[form]["fp64_until"] = args.fp64_until
            per_form[form]["switch_d"] = g.switch_d
        if first is None:
            first = form
    base = per_form[first]
    # error of the mixed form against the FP64 GPU form
    for f, v in per_form.items():
        if f != first and "X" in v:
            v["rel_err_vs_fp64"] = (_lowrank_fro(np.hstack([v["X"][0], -base["X"][0]]),
                                                 np.hstack([v["X"][1], base["X"][1]]))
                                    / _lowrank_fro(*base["X"]))
    # end-to-end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hostA = [torch.as_tensor(a).pin_memory() for a in
                 (P.A.indptr, P.A.indices, P.A.data, P.BT.indptr, P.BT.indices, P.BT.data)]
        hostC = [torch.as_tensor(P.C1).pin_memory(), torch.as_tensor(P.C2).pin_memory()]
        h2d = sum(t.numel() * t.element_size() for t in hostA + hostC)
        d2h = 0
        torch.cuda.synchronize()
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            dev = [t.to("cuda", non_blocking=True) for t in hostA + hostC]
            A_ = spk.DeviceCSR.__new__(spk.DeviceCSR)
            A_.shape, A_.rowptr, A_.col, A_.val = P.A.shape, dev[0], dev[1], dev[2]
            A_.c = spk.Csr(P.n1, P.n1, P.A.nnz, dev[0].data_ptr(), dev[1].data_ptr(), dev[2].data_ptr())
            B_ = spk.DeviceCSR.__new__(spk.DeviceCSR)
            B_.shape, B_.rowptr, B_.col, B_.val = P.BT.shape, dev[3], dev[4], dev[5]
            B_.c = spk.Csr(P.n2, P.n2, P.BT.nnz, dev[3].data_ptr(), dev[4].data_ptr(), dev[5].data_ptr())
            g = spk.solve(A_, B_, dev[6], dev[7], precision=first, device=local, **opts)
            o1 = torch.empty(g.X1.shape, dtype=torch.float64).pin_memory()
            o2 = torch.empty(g.X2.shape, dtype=torch.float64).pin_memory()
            o1.copy_(g.X1, non_blocking=True)
            o2.copy_(g.X2, non_blocking=True)
            d2h = o1.numel() * 8 + o2.numel() * 8
        torch.cuda.synchronize()
        barrier(pg)
        secs = max_over_ranks(pg, time.perf_counter() - t0)
        e2e = {"value": world * args.steps / secs, "unit": "solves/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp64_peak, mhz = fp64_alu_peak(sms)
    tensor_fp64 = bf16_sus / OZAKI_PAIRS
    roof, table = pick_roofline(base["prof"] or {}, hbm, fp64_peak, tensor_fp64, args.engine)
    if roof is not None:
        roof["peak_source"] = (f"HBM: {peak_src} copy GB/s (MEASURED_PEAKS.json); FP64 ALU: derived, "
                               f"{sms} SMs x 2 FMA/clk x 2 flop x {mhz:.0f} MHz = {fp64_peak:.4f} "
                               f"TFLOP/s (live FMA probe {fp64:.4f}); tensor: FP64-equivalent = "
                               f"{peak_src} sustained BF16 {bf16_sus:.1f} TFLOP/s / {OZAKI_PAIRS} "
                               f"slice products = {tensor_fp64:.2f} TFLOP/s")
    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        s = oracle_sample_fresh(args.workload, opts, args.cpu_sample_iters, base["checks"], P.r)
        cpu = {"value": s["solves_per_s"], "unit": "solves/s", "cores": s["cores"],
               "kind": "oracle",
               "sample": (f"{s['iters_sampled']} oracle iterations + one projected solve at "
                          f"m={s['m0']} + Bartels-Stewart at m={s['m1']} "
                          f"({s['sample_seconds']:.1f} s, fresh process, BLAS threads = "
                          f"{s['cores']}), extrapolated to d={s['extrapolated_to_d']} "
                          f"with the GPU run's {s['checks']} checks (a + b d per iteration, "
                          f"m^3 per check)")}
    if rank == 0:
        forms_out = {f: {k: v for k, v in d.items() if k not in ("X", "prof", "clocks")}
                     for f, d in per_form.items()}
        line = {
            "metric": metric_name(opts["tol"]),
            "value": base["solves_per_s"], "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": base["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if first == "fp64" else "f32+f64", "data": "synthetic",
            "config": workload_config(P, opts, world),
            "forms": forms_out,
            "clocks": base["clocks"], "gpu_launches": base["gpu_launches"],
            "e2e": e2e, "roofline": roof, "kernels": table, "fp64_tflops_measured": fp64,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def run_kernel_case(args):
    """Dense sign-function solve of H Y + Y G^T = F, m x m (default 4200: the
    matrices exceed L2), as a small isolated case of the inversion kernels."""
    import numpy as np
    import torch
    from paper_2311_16019_gb300 import build, spk
    build.build()
    rng = np.random.default_rng(11)
    m = args.m
    def rhp():
        A = rng.standard_normal((m, m)) * (0.3 / np.sqrt(m))
        A[np.diag_indices(m)] += rng.uniform(1.0, 100.0, m)
        return A
    H, G = rhp(), rhp()
    F = np.zeros((m, m))
    F[:4, :4] = rng.standard_normal((4, 4))
    out = {"kernel_case": args.kernel_case, "m": m}
    Ys = {}
    for engine in args.engines.split(","):
        spk.set_tensor_gemm(engine == "tensor")
        spk.sylvester_dense(H, G, F)        # warm-up (workspace, first launches)
        torch.cuda.synchronize()
        spk.profile_enable(True)
        t0 = time.perf_counter()
        Y, it = spk.sylvester_dense(H, G, F)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        prof = spk.profile_read()
        spk.profile_enable(False)
        Ys[engine] = Y
        fams = {k: {"ms": round(v["ms"], 2), "launches": v["launches"],
                    "TFLOPs": round(v["flops"] / max(v["ms"], 1e-9) / 1e9, 4)}
                for k, v in prof.items() if v["ms"] > 0}
        out[engine] = {"newton_iters": it, "seconds": secs, "families": fams}
    if "tensor" in Ys and "fp64" in Ys:
        out["tensor_vs_fp64_rel_diff"] = float(np.linalg.norm(Ys["tensor"] - Ys["fp64"]) /
                                               np.linalg.norm(Ys["fp64"]))
    spk.set_tensor_gemm(args.engine == "tensor")
    print(json.dumps(out), flush=True)


def batched_opts(P, form, maxit=2000):
    """Per-instance options of the batched workload: k = 4, tol 1e-8, p = 20,
    s = min(n', 2 r maxit) and maxit clamped so that s >= (maxit + 1) r."""
    npad = 1 << (P.n1 - 1).bit_length()
    s = min(npad, 2 * P.r * maxit)
    return dict(k=4, s=s, maxit=min(maxit, s // P.r - 1), p=20, tol=1e-8, seed=4,
                check="adaptive", trunc_tol=1e-12, precision=form)


def run_batched(args):
    """The batched form on 64 uneven conv-diff instances (N uniform in
    [64, 384], theta in [1, 50], r in {1, 2, 4}), solved by concurrent
    workers; one step = the whole batch."""
    import torch
    from paper_2311_16019_gb300 import build, inputs as I, spk
    build.build()
    spk.load()
    form = args.forms.split(",")[0]
    probs = I.batched_instances(count=64, seed=4)
    opts = [batched_opts(P, form) for P in probs]
    dev = [(spk.DeviceCSR(P.A), spk.DeviceCSR(P.BT)) for P in probs]

    class Inst:
        pass
    insts = []
    for P, (dA, dB) in zip(probs, dev):
        o = Inst()
        o.A, o.BT = dA, dB
        o.C1 = torch.as_tensor(P.C1, device="cuda")
        o.C2 = torch.as_tensor(P.C2, device="cuda")
        insts.append(o)
    conc = args.concurrency
    if conc <= 0:
        # worker count by measurement on a short probe of the same batch
        conc = spk.autotune_concurrency(insts, opts_list=opts)
    args.concurrency = conc
    for _ in range(args.warmup):
        spk.solve_batched(insts, concurrency=args.concurrency, opts_list=opts, raise_on_error=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs = None
    for _ in range(args.steps):
        rc, outs = spk.solve_batched(insts, concurrency=args.concurrency, opts_list=opts,
                                     raise_on_error=False)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    conv = sum(1 for g in outs if g.converged)
    not_conv = [i for i, g in enumerate(outs) if not g.converged]
    failed = {}
    for g in outs:
        if g.X1 is None:
            failed[str(g.status)] = failed.get(str(g.status), 0) + 1
    line = {"metric": "solves/s, batched form (64 uneven instances)",
            "value": len(insts) * args.steps / secs, "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f32+f64" if form != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": "batch64: N~U{64..384}, theta~U[1,50], r~U{1,2,4}, k=4, "
                                   "tol=1e-8, p=20 adaptive", "form": form,
                       "concurrency": args.concurrency},
            "seconds_per_batch": secs / args.steps, "converged": conv, "failed": failed,
            "not_converged": not_conv,
            "iters": [g.iters if g.X1 is not None else g.status for g in outs],
            "first_error": spk.handle().error() if failed else ""}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.oracle_sample:
        run_oracle_sample(args.oracle_sample)
        return
    if args.kernel_case:
        run_kernel_case(args)
        return
    if args.batched:
        run_batched(args)
        return
    rank, world, local, pg = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world, pg)
    else:
        run_spk(args, rank, world, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
