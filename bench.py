"""Benchmark of the accuracy-controlled H^2 direct solver on one GB300.

Workload (default): 32^3 = 32,768-point regular grid, cube side 2 wavelengths
(k = 2 pi, h = 1/16), uniform contrast chi = 3 (eps_r = 4), leaf 64,
admissibility 1.0, eps_build = eps_fill = 1e-6, 16 complex Gaussian RHS
(seed 1).  A "step" is one pass of the hot path on resident inputs:
h2_factorize (mixed precision: complex64 bulk, FP64 rank decisions) followed
by h2_solve of the 16 RHS with FP64-matvec iterative refinement to a relative
residual of 1e-6.  value = N / (step time) unknowns/s; the FP64 factorization
is timed beside it.  The H^2 construction (h2_build) is not timed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (plain FP64 numpy) on a bounded sample
of the same workload: the 16^3 sub-grid with the same h, chi and eps.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

K = 2.0 * math.pi
H = 1.0 / 16.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=32)
    p.add_argument("--eps", type=float, default=1e-6)
    p.add_argument("--chi", type=float, default=3.0)
    p.add_argument("--nrhs", type=int, default=16)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--tol", type=float, default=1e-6)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--rod-lengths", default="25,50,100,200,400",
                   help="rod workload: lengths in wavelengths (cross-section 0.4 x 0.4, h = 0.1)")
    p.add_argument("--workload", default="grid", choices=["grid", "batch", "grad", "rod"],
                   help="grid: one instance (default); batch: many independent instances in shared launches")
    p.add_argument("--instances", type=int, default=64, help="batch workload: number of instances")
    p.add_argument("--batch-reserve-gb", type=float, default=24.0,
                   help="batch workload: stop adding instances when less device memory than this is free")
    p.add_argument("--solve-graph-check", action="store_true",
                   help="also time repeated solves with CUDA-graph replay (builds a second context)")
    p.add_argument("--profile-levels", action="store_true", help="kernel classes kept apart per tree level")
    p.add_argument("--apply-path", type=int, default=0, choices=[0, 1, 2],
                   help="Step 2 / panel applications: 0 auto, 1 in-place kernel, 2 GEMM + copy")
    p.add_argument("--tensor-cores", type=int, default=None, choices=[0, 1, 2],
                   help="complex64 GEMM tiles: 2 tcgen05, 1 warp-level TF32 MMA, 0 FP32 FMA (default: library's)")
    p.add_argument("--eig-solver", type=int, default=None, choices=[0, 1, 2],
                   help="Step-0 eigen-decomposition: 0 cyclic Jacobi, 1 tridiagonal + QL, "
                        "2 one-sided Jacobi SVD of the Cholesky factor (default: library's)")
    p.add_argument("--ldlt", type=int, default=None, choices=[0, 1, 2],
                   help="elimination form: 0 block LU, 1 block LDL^T of the symmetric matrix, 2 LDL^T for FP64 "
                        "factorizations only (default: library's)")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison factorization (large grids)")
    p.add_argument("--proxy", type=int, default=0,
                   help="construction with proxy points (h2_opts.proxy_min; 0 = exact far-field sample)")
    p.add_argument("--arena-cap-gb", type=float, default=0.0,
                   help="cap on the library's device memory (h2_opts.arena_cap_bytes; 0 = none)")
    p.add_argument("--json-extra", action="store_true", help="print per-level stats")
    p.add_argument("--profile-step", action="store_true",
                   help="build, then exactly one factorize + refined solve (for profiler captures)")
    p.add_argument("--cpu-baseline-only", action="store_true", help=argparse.SUPPRESS)
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self):
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=" + q, "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout.strip()
                f = [x.strip() for x in out.split(",")]
                if len(f) >= 7:
                    self.samples.append(f)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def workload_name(args):
    """The grid workload's name (both arms)."""
    n = args.grid
    return "grid%d (N=%d), chi=%g, eps=%g, nrhs=%d, leaf 64, eta 1" % (n, n ** 3, args.chi, args.eps, args.nrhs)


def tc_opts(args):
    o = {} if args.tensor_cores is None else {"tensor_cores": args.tensor_cores}
    if args.eig_solver is not None:
        o["eig_solver"] = args.eig_solver
    if args.ldlt is not None:
        o["ldlt"] = args.ldlt
    return o


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


MEASURED = {}  # FP64 / FP32 / DMMA rates measured by the peak probes in this run


def probe_peaks():
    """FP64 FMA, FP32 FMA and FP64 tensor-core (DMMA) throughput measured on
    this GPU with the probe kernels of libh2peaks.so (CUDA events)."""
    import ctypes
    path = os.path.join(ROOT, "paper_1703_06155_gb300", "libh2peaks.so")
    if not os.path.exists(path):
        return {}
    lib = ctypes.CDLL(path)
    lib.h2_peak_probe.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = {}
    for kind, name in ((0, "fp64"), (1, "fp32"), (2, "dmma_fp64")):
        v = ctypes.c_double()
        if lib.h2_peak_probe(kind, ctypes.byref(v)) == 0:
            out[name] = v.value
    return out


def fp_peaks(clocks):
    """Peak FP64 / FP32 (non-tensor) rates: measured by the probes of this run
    when they ran, else derived from unit counts and the SM clock (152 SMs, 2
    FP64 FMA and 128 FP32 FMA per SM per clock)."""
    f = (clocks or {}).get("sm_max_mhz") or 2070.0
    out = {"fp64": 152 * 2 * 2 * f * 1e6 / 1e12, "fp32": 152 * 128 * 2 * f * 1e6 / 1e12, "mhz": f,
           "source": "derived"}
    if MEASURED.get("fp64") and MEASURED.get("fp32"):
        out.update(fp64=MEASURED["fp64"], fp32=MEASURED["fp32"], source="measured")
    return out


def roofline(st, clocks, kernel=None, workload=None):
    """Roofline entry of one kernel class (default: the class with the most
    device time among the classes with an algorithmic flop or byte count),
    from the per-launch CUDA events of the instrumented pass."""
    kern = st.get("kernels", {})
    cands = [(k, v) for k, v in kern.items() if (v.get("flops", 0) > 0 or v.get("bytes", 0) > 0) and v["ms"] > 0]
    if kernel is not None:
        cands = [(k, v) for k, v in cands if k == kernel]
    if not cands:
        return None
    k, v = max(cands, key=lambda kv: kv[1]["ms"])
    pk = fp_peaks(clocks)
    if v.get("flops", 0) <= 0:
        # memory-bound class (copies, traces): algorithmic bytes over time
        pv, src = peaks()
        achieved = v["bytes"] / (v["ms"] * 1e-3) / 1e9
        return {"kernel": k, "pipe": "hbm", "achieved": achieved, "unit": "GB/s", "bound": "hbm",
                "peak": pv["hbm_gbs"], "peak_source": "%s HBM copy bandwidth" % src, "frac": achieved / pv["hbm_gbs"],
                "traffic": None, "launches": v["launches"], "avg_launch_ms": v["ms"] / v["launches"],
                "bytes_per_launch": v["bytes"] / v["launches"]}
    achieved = v["flops"] / (v["ms"] * 1e-3) / 1e12
    out = {"kernel": k, "pipe": v.get("pipe"), "achieved": achieved, "unit": "TFLOP/s",
           "traffic": measured_traffic(k, workload), "launches": v["launches"],
           "avg_launch_ms": v["ms"] / v["launches"], "flops_per_launch": v["flops"] / v["launches"]}
    pipe = v.get("pipe") or ("fp64" if st.get("prec") == "fp64" else "fp32")
    if pipe.endswith("tf32x3"):
        # complex64 products as three TF32 tensor-core products each: the
        # FP32-accurate rate is a third of the TF32 rate, taken as the
        # measured bf16 GEMM rate x the nominal TF32 / bf16 ratio (1.1 / 2.25)
        # (sustained figure: the kernel runs inside a seconds-long step)
        pv, src = peaks()
        bf16 = pv.get("bf16_tflops_sustained", pv["bf16_tflops"])
        peak = bf16 * (1.1 / 2.25) / 3.0
        out.update(bound="tensor", peak=peak, peak_source="%s sustained bf16 %.0f TF/s x 1.1/2.25 (TF32) / 3 "
                   "(hi/lo split)" % (src, bf16))
    elif pipe == "fp32_df":
        # FP64-accurate products of complex64 operands on the FP32 pipe: 4
        # exact real products summed in double-float per complex
        # multiply-add, 9 FP32 operations each (36 per 8 algorithmic flops)
        peak = pk["fp32"] / 2.0 * 8.0 / 36.0
        out.update(bound="alu", peak=peak, peak_source="%s FP32 lane rate x 8 flops / 36 FP32 operations per "
                   "complex multiply-add (double-float, FP32 pipe)" % pk["source"])
    elif pipe == "fp64_dd":
        # complex128 products in double-float on the FP32 pipe: per real
        # product a split multiply (4 FP32 operations) and a TwoSum
        # accumulation (8), 48 per complex multiply-add of 8 algorithmic flops
        peak = pk["fp32"] / 2.0 * 8.0 / 48.0
        out.update(bound="alu", peak=peak, peak_source="%s FP32 lane rate x 8 flops / 48 FP32 operations per "
                   "complex multiply-add (double-float products of FP64 operands, FP32 pipe)" % pk["source"])
    elif pipe == "fp32_dfr":
        # one-sided Jacobi rotations in double-float on the FP32 pipe: per
        # entry of a rotated column pair, the complex dot product (4
        # double-float multiply-adds of 15 FP32 operations) and the rotation
        # of the entry pair of W and of J (2 double-float multiplies of 7 and
        # 8 multiply-adds of 15 operations each, twice): 328 FP32 operations
        # for 48 algorithmic flops
        peak = pk["fp32"] / 2.0 * 48.0 / 328.0
        out.update(bound="alu", peak=peak, peak_source="%s FP32 lane rate x 48 flops / 328 FP32 operations per "
                   "rotated entry pair (double-float, FP32 pipe)" % pk["source"])
    else:
        fp64 = pipe == "fp64"
        peak = pk["fp64"] if fp64 else pk["fp32"]
        if pk["source"] == "measured":
            src = "measured in this run by the %s FMA probe (libh2peaks)" % ("FP64" if fp64 else "FP32")
        else:
            src = "derived: 152 SM x %s FMA/clk x 2 flops x %.0f MHz (%s)" % (
                "2 FP64" if fp64 else "128 FP32", pk["mhz"], "FP64 pipe" if fp64 else "FP32 pipe")
        out.update(bound="alu", peak=peak, peak_source=src)
    out["frac"] = achieved / out["peak"]
    return out


def roofline_table(st, clocks, top=14):
    """One roofline row per kernel class with an algorithmic count, by device time."""
    rows = []
    kern = st.get("kernels", {})
    for k in sorted(kern, key=lambda k: -kern[k]["ms"]):
        r = roofline(st, clocks, kernel=k)
        if r is None:
            continue
        rows.append({"kernel": k, "ms": round(kern[k]["ms"], 3), "launches": kern[k]["launches"],
                     "pipe": r["pipe"], "bound": r["bound"], "achieved": round(r["achieved"], 4),
                     "unit": r["unit"], "peak": round(r["peak"], 3), "frac": round(r["frac"], 4)})
        if len(rows) >= top:
            break
    return rows


def measured_traffic(kernel_class, workload=None):
    """DRAM bytes per launch of a kernel class from the committed ncu summary,
    if it was taken for this class, on this workload, with the kernel's
    current source (else None: the counters do not describe this run)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            d = json.load(f)
        with open(os.path.join(ROOT, d["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except Exception:
        return None
    if d.get("kernel_class") != kernel_class.split("@")[0] or d.get("source_sha256") != sha:
        return None
    if workload is not None and d.get("workload") != workload:
        return None
    return d.get("dram_bytes_per_launch")


# --------------------------------------------------------------- oracle ---

def oracle_sample(args, repeat=1):
    """Oracle (CPU, FP64) build + factorize + solve on the 16^3 sub-grid."""
    from oracle import factor, h2
    from paper_1703_06155_gb300 import inputs
    n = min(args.grid, 16)
    pts = inputs.grid_points(n, H)
    N = len(pts)
    chi = inputs.chi_uniform(N, args.chi)
    Hm = h2.build(pts, chi, K, H, leafsize=64, eps=args.eps)
    b = inputs.rhs_gaussian(N, args.nrhs, args.seed)
    bt = b[Hm.tree.perm]
    times = []
    for _ in range(repeat):
        t0 = time.perf_counter()
        Fz = factor.factorize(Hm, args.eps, "colored", bulk=np.complex64 if args.prec == "mixed" else np.complex128)
        x, hist = factor.refine(Fz, bt, tol=args.tol, max_iter=20)
        times.append(time.perf_counter() - t0)
    return N, times, hist[-1]


def oracle_precision(args):
    """What the oracle computes in the sample (numpy complex128 arithmetic)."""
    if args.prec == "mixed":
        return "mixed-precision emulation: complex128 arithmetic with the bulk rounded to complex64, FP64 rank " \
               "decisions and refinement"
    return "complex128 throughout"


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        return max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    N, times, res = oracle_sample(args, repeat=args.warmup + args.steps)
    t = times[args.warmup:] if len(times) > args.warmup else times
    step = float(np.mean(t))
    v = N / step
    line = {
        "impl": "reference", "metric": "H2 factorize+solve unknowns/s (rel. residual 1e-6)", "value": v,
        "unit": "unknowns/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128 (bulk rounded to c64)" if args.prec == "mixed" else "c128", "data": "synthetic",
        "config": {"workload": workload_name(args), "precision": "oracle, " + oracle_precision(args),
                   "sample": "16^3 sub-grid of the workload, same h, chi, eps (N=%d), build untimed" % N},
        "cpu_baseline": {"value": v, "unit": "unknowns/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": "oracle factorize + refined solve of the 16^3 sub-grid (N=%d), %s" % (
                             N, oracle_precision(args))},
        "e2e": {"value": v, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "final_residual": res,
    }
    print(json.dumps(line))


# ------------------------------------------------------- multi-rank ----

def max_over_ranks(ms, dist, device):
    """Step time of the whole job: the slowest rank's (replicas run
    independent instances; there is no data-path collective)."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, n_per_rank, ms):
    """Unknowns per second of all ranks together (weak scaling)."""
    return world * n_per_rank / (ms / 1e3)


# ------------------------------------------------------------------ GPU ---

def run_grad(args):
    """Contrast gradient of a scattered-field objective: n^3 cells (default
    48^3, cube side 3 wavelengths), chi_i = 1.5 + 0.5 U(0,1) (seed 4), plane
    wave b = exp(-jkz), L = sum over 64 Fibonacci-sphere probes (radius twice
    the cube's half-diagonal) of |E|^2 with E = G_E D_chi x.  Timed: the
    autograd step (refined forward solve, refined adjoint solve on the same
    factors, h2_grad_chi).  Checked: central differences (step 1e-6) on 8
    random cells, each perturbed system solved by refinement with the
    unperturbed factors against A' x = A x + (d / chi_i)(A e_i - e_i) x_i."""
    import torch
    from paper_1703_06155_gb300 import H2, autograd, inputs

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    n = args.grid if args.grid != 32 else 48
    pts = inputs.grid_points(n, H)
    N = len(pts)
    chi = inputs.chi_random_cells(N, 4)
    t0 = time.perf_counter()
    A = H2.build(pts, K, H, chi, args.eps, stream=stream, **tc_opts(args))
    t_build = time.perf_counter() - t0
    f0 = time.perf_counter()
    A.factorize(args.eps, args.prec)
    t_fac = time.perf_counter() - f0
    dev = torch.device("cuda")
    b = torch.from_numpy(inputs.rhs_plane_wave(pts, K)).to(dev)
    radius = 2.0 * (math.sqrt(3.0) / 2.0) * n * H
    probes = torch.from_numpy(inputs.fibonacci_sphere(64, pts.mean(axis=0), radius)).to(dev)
    P = torch.from_numpy(pts).to(dev)
    r = torch.cdist(probes, P)
    G = (K * K * H ** 3) * torch.exp(-1j * K * r) / (4 * math.pi * r)
    chi_t = torch.from_numpy(chi).to(dev)
    tol = 1e-12

    def grad_step():
        c = chi_t.clone().requires_grad_(True)
        x = autograd.solve(A, c, b, refine=True, tol=tol)
        L = torch.sum(torch.abs(G @ (c * x)) ** 2)
        L.backward()
        return float(L.detach()), c.grad

    for _ in range(max(1, args.warmup)):
        grad_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        L0, g = grad_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # central differences on 8 cells
    cells = np.random.default_rng(4).choice(N, 8, replace=False)
    nb = float(torch.linalg.norm(b))

    def objective(i, d):
        e = torch.zeros(N, dtype=torch.complex128, device=dev)
        e[i] = 1.0
        col = A.matvec(e) - e
        x = A.solve(b, refine=True, tol=tol, max_iter=30)
        for _ in range(60):
            res = b - A.matvec(x) - (d / chi[i]) * col * x[i]
            if float(torch.linalg.norm(res)) <= 1e-13 * nb:
                break
            x = x + A.solve(res)
        c = chi_t.clone()
        c[i] += d
        return float(torch.sum(torch.abs(G @ (c * x)) ** 2))

    delta = 1e-6
    fd = np.array([(objective(int(i), delta) - objective(int(i), -delta)) / (2 * delta) for i in cells])
    gc = g.detach().cpu().numpy()[cells]
    err = float(np.max(np.abs(fd - gc)) / np.max(np.abs(g.detach().cpu().numpy())))
    print(json.dumps({
        "metric": "contrast gradient (autograd: refined solve + adjoint solve + grad kernel)",
        "value": ms, "unit": "ms per gradient", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "dtype": "c64 bulk + c128 rank/refine" if args.prec == "mixed" else "c128",
        "data": "synthetic",
        "config": {"workload": "grad%d (N=%d), chi_i=1.5+0.5U(0,1), plane wave, 64 probes, eps=%g, refine tol %g" % (
            n, N, args.eps, tol)},
        "objective": L0, "fd_max_rel_err_8_cells": err, "factorize_s": t_fac, "build_s": t_build,
        "dev_peak_gb": A.stats()["dev_peak"] / 1e9,
    }))


def run_rod(args):
    """The rod workload of Sec. VI-B on a regular grid: cross-section 0.4 x 0.4
    wavelengths, cells of 0.1 wavelength (4 x 4 per layer), eps_r = 2.54
    (chi = 1.54), eps = 1e-4, length growing (--rod-lengths, wavelengths).
    A 1-D configuration: the ranks stay bounded as it grows, so factorization,
    solve and memory should grow linearly in N (eq. 44, Fig. 5).  Per length:
    h2_build untimed, factorization and refined solve timed with CUDA events
    (one warm-up, median of 3), peak device memory; the log-log slope of the
    times against N is reported."""
    import torch
    from paper_1703_06155_gb300 import H2, inputs

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    h, chi, eps = 0.1, 1.54, args.eps if args.eps != 1e-6 else 1e-4
    rows = []
    for length in [float(v) for v in args.rod_lengths.split(",")]:
        pts = inputs.rod_points(length, h)
        N = len(pts)
        A = H2.build(pts, K, h, chi, eps, stream=stream, **tc_opts(args))
        b = torch.from_numpy(inputs.rhs_gaussian(N, args.nrhs, args.seed)).to("cuda")
        A.factorize(eps, args.prec)
        A.solve(b, refine=True, tol=args.tol, max_iter=30)
        fac, sol = [], []
        for _ in range(3):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            torch.cuda.synchronize()
            e0.record(stream)
            A.factorize(eps, args.prec)
            e1.record(stream)
            x = A.solve(b, refine=True, tol=args.tol, max_iter=30)
            e2.record(stream)
            torch.cuda.synchronize()
            fac.append(e0.elapsed_time(e1))
            sol.append(e1.elapsed_time(e2))
        st = A.stats()
        res = float(torch.linalg.norm(A.matvec(x) - b) / torch.linalg.norm(b))
        rows.append({"length_wavelengths": length, "N": N, "factorize_ms": float(np.median(fac)),
                     "refined_solve_ms": float(np.median(sol)), "dev_peak_gb": st["dev_peak"] / 1e9,
                     "kt_max": max(lv["kt_max"] for lv in st["levels"]), "final_residual": res,
                     "refine_iters": A.last_solve["iters"]})
        A.close()
    Ns = np.array([r["N"] for r in rows], dtype=float)

    def slope(key):
        return float(np.polyfit(np.log(Ns), np.log([r[key] for r in rows]), 1)[0]) if len(rows) > 1 else None

    print(json.dumps({
        "metric": "H2 factorize unknowns/s on the rod workload (1-D, constant rank)",
        "value": rows[-1]["N"] / (rows[-1]["factorize_ms"] / 1e3), "unit": "unknowns/s", "higher_is_better": True,
        "n_gpus": 1, "dtype": "c64 bulk + c128 rank/refine" if args.prec == "mixed" else "c128", "data": "synthetic",
        "config": {"workload": "rod 0.4 x 0.4 x L wavelengths, h = 0.1, eps_r = 2.54, eps = %g, nrhs = %d, leaf 64"
                   % (eps, args.nrhs), "precision": args.prec},
        "rows": rows, "loglog_slope": {"factorize": slope("factorize_ms"), "solve": slope("refined_solve_ms"),
                                       "memory": slope("dev_peak_gb")},
    }))


def run_batch(args):
    """Independent instances: grids drawn from {12..32}^3 (cube sides 0.75-2
    wavelengths at h = 1/16), eps_r ~ U[2, 6] per instance (chi = eps_r - 1),
    mixed factorization + FP64-refined solve of nrhs Gaussian right-hand sides
    each.  Timed: one batched step (h2_factorize_batch + h2_solve_batch) and
    the same instances one by one (h2_factorize + h2_solve each)."""
    import torch
    from paper_1703_06155_gb300 import H2, factorize_batch, inputs, solve_batch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(args.seed)
    sizes = rng.choice([12, 16, 20, 24, 28, 32], args.instances)
    chis = rng.uniform(2.0, 6.0, args.instances) - 1.0
    ctxs, bs, Ns = [], [], []
    t0 = time.perf_counter()
    reserve = int(args.batch_reserve_gb * (1 << 30))  # keep this much device memory free
    for i, (n, chi) in enumerate(zip(sizes, chis)):
        pts = inputs.grid_points(int(n), H)
        A = H2.build(pts, K, H, float(chi), args.eps, stream=stream, **tc_opts(args))
        b = torch.from_numpy(inputs.rhs_gaussian(len(pts), args.nrhs, args.seed + i)).to("cuda")
        A.factorize(args.eps, args.prec)  # sizes the instance's arenas
        A.solve(b, refine=True, tol=args.tol, max_iter=30)
        ctxs.append(A)
        bs.append(b)
        Ns.append(len(pts))
        if torch.cuda.mem_get_info()[0] < reserve:
            break
    t_build = time.perf_counter() - t0
    Ntot = int(sum(Ns))

    def batched():
        factorize_batch(ctxs, args.eps, args.prec)
        return solve_batch(ctxs, bs, refine=True, tol=args.tol, max_iter=30)

    def one_by_one():
        out = []
        for A, b in zip(ctxs, bs):
            A.factorize(args.eps, args.prec)
            out.append(A.solve(b, refine=True, tol=args.tol, max_iter=30))
        return out

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, r

    with ClockSampler() as cs:
        ms_b, (xs, info) = timed(batched)
        ms_1, xs1 = timed(one_by_one)
    res = max(float(torch.linalg.norm(A.matvec(x) - b) / torch.linalg.norm(b)) for A, x, b in zip(ctxs, xs, bs))
    diff = max(float(torch.linalg.norm(x - y) / torch.linalg.norm(y)) for x, y in zip(xs, xs1))
    line = {
        "metric": "H2 factorize+solve unknowns/s (rel. residual 1e-6)", "value": Ntot / (ms_b / 1e3),
        "unit": "unknowns/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 bulk + c128 rank/refine" if args.prec == "mixed" else "c128", "data": "synthetic",
        "config": {"workload": "batch of %d independent instances (grids %s^3, chi in [1, 5], eps=%g, nrhs=%d)" % (
            len(ctxs), ",".join(str(int(n)) for n in sizes[:len(ctxs)]), args.eps, args.nrhs),
            "unknowns": Ntot, "requested_instances": args.instances, "l2": "inputs larger than L2"},
        "one_by_one": {"ms_per_step": ms_1, "value": Ntot / (ms_1 / 1e3)},
        "batched_speedup": ms_1 / ms_b, "final_residual_max": res, "batched_vs_single_max_rel_diff": diff,
        "refine_iters": info["iters"], "build_s": t_build, "clocks": cs.summary(),
    }
    print(json.dumps(line))



def run_ours(args):
    import torch
    from paper_1703_06155_gb300 import H2, inputs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    MEASURED.update(probe_peaks())
    pts = inputs.grid_points(args.grid, H)
    N = len(pts)
    tun = dict(apply_path=args.apply_path, **tc_opts(args))
    prof = 2 if args.profile_levels else 1
    t0 = time.perf_counter()
    # the timed steps run without per-launch events (profile = 0); the kernel
    # table comes from a separate instrumented pass afterwards
    A = H2.build(pts, K, H, args.chi, args.eps, stream=stream, profile=0,
                 arena_cap_bytes=int(args.arena_cap_gb * 1e9), proxy_min=args.proxy, **tun)
    t_build = time.perf_counter() - t0
    b_host = inputs.rhs_gaussian(N, args.nrhs, args.seed + rank)  # independent instance per rank
    b = torch.from_numpy(b_host).to("cuda")
    if args.profile_step:
        A.factorize(args.eps, args.prec)
        A.solve(b, refine=True, tol=args.tol, max_iter=30)
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": True, "stats": A.stats()}))
        return

    for _ in range(args.warmup):
        A.factorize(args.eps, args.prec)
        A.solve(b, refine=True, tol=args.tol, max_iter=30)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches = 0
    with ClockSampler() as cs:
        ev0.record(stream)
        fac_ms = []
        for _ in range(args.steps):
            f0 = time.perf_counter()
            A.factorize(args.eps, args.prec)
            fac_ms.append((time.perf_counter() - f0) * 1e3)
            x = A.solve(b, refine=True, tol=args.tol, max_iter=30)
            st = A.stats()
            launches += int(st["launches_factor"] + st["launches_solve"])
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, "cuda")
    clocks = cs.summary()
    solve_info = dict(A.last_solve)
    # residual of the result against the H^2 matrix (FP64 matvec), and the
    # matvec's own time (CUDA events, mean of 3)
    r = A.matvec(x) - b
    res = float(torch.linalg.norm(r) / torch.linalg.norm(b))
    torch.cuda.synchronize()
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(3):
        A.matvec(x, stream=stream)
    m1.record(stream)
    torch.cuda.synchronize()
    matvec_ms = m0.elapsed_time(m1) / 3

    def timed_step(prec):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record(stream)
        A.factorize(args.eps, prec)
        e1.record(stream)
        A.solve(b, refine=True, tol=args.tol, max_iter=30)
        e2.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), A.last_solve["iters"], A.last_solve["resid"]

    # FP64 comparison arm (not part of the metric): one warm-up, median of 3
    fp64 = None
    if not args.no_fp64:
        timed_step("fp64")
        runs = [timed_step("fp64") for _ in range(3)]
        fm = float(np.median([u[0] for u in runs]))
        fp64 = {"factorize_ms": fm, "factorize_ms_runs": [round(u[0], 2) for u in runs],
                "refined_solve_ms": float(np.median([u[1] for u in runs])), "solve_iters": runs[-1][2],
                "final_residual": runs[-1][3], "factorize_unknowns_per_s": N / (fm / 1e3),
                "timing": "CUDA events, 1 warm-up, median of 3"}
    # instrumented pass: per-launch CUDA events of one factorize + refined
    # solve in the same configuration (kernel table, roofline; not timed)
    A.set_opts(profile=prof, **tun)
    A.factorize(args.eps, args.prec)
    A.solve(b, refine=True, tol=args.tol, max_iter=30)
    torch.cuda.synchronize()
    st = A.stats()
    A.set_opts(profile=0, **tun)
    roof = roofline(st, clocks, workload=workload_name(args))
    table = roofline_table(st, clocks)
    # repeated solves with the same factors: plain launches vs CUDA-graph replay
    # of the sweeps (h2_opts.solve_graph; not part of the metric)
    A.factorize(args.eps, args.prec)
    G = (H2.build(pts, K, H, args.chi, args.eps, stream=stream, solve_graph=1, **tc_opts(args))
         if args.solve_graph_check else None)

    def solves(ctx, n):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            ctx.solve(b, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    solve_graph = None
    if G is not None:
        G.factorize(args.eps, args.prec)
        solves(G, 2)  # sizing run + capture
        solve_graph = {"ms_per_solve_plain": solves(A, 10), "ms_per_solve_graph": solves(G, 10)}
        G.close()
    # e2e: same step through the public API with HOST buffers (H2D of b and
    # D2H of x inside the timed region, every step)
    A.factorize(args.eps, args.prec)
    e0 = time.perf_counter()
    ne = max(1, args.steps // 2)
    for _ in range(ne):
        A.factorize(args.eps, args.prec)
        xh = A.solve(b_host, refine=True, tol=args.tol, max_iter=30)
    e_ms = (time.perf_counter() - e0) * 1e3 / ne
    value = whole_job_value(world, N, ms)
    line = {
        "metric": "H2 factorize+solve unknowns/s (rel. residual 1e-6)", "value": value, "unit": "unknowns/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 bulk + c128 rank/refine" if args.prec == "mixed" else "c128",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "precision": args.prec,
                   "construction": "proxy points (min %d per sphere)" % args.proxy if args.proxy else "exact far field",
                   "l2": "inputs larger than L2 (near-field arena %.0f MB)" % (st.get("dev_bytes", 0) / 1e6),
                   "timed_steps": "no per-launch events (kernel table from a separate instrumented pass)"},
        "factorize_ms": float(np.mean(fac_ms)), "solve_iters": solve_info.get("iters"),
        "final_residual": res, "fp64": fp64,
        "refined_solve_ms": ms - float(np.mean(fac_ms)), "matvec_ms": matvec_ms,
        "dev_peak_gb": st.get("dev_peak", 0) / 1e9,
        "dev_bytes_by_kind_gb": {k: round(v / 1e9, 3) for k, v in st.get("mem", {}).items()},
        "factorize_unknowns_per_s": N / (float(np.mean(fac_ms)) / 1e3),
        "mixed_over_fp64_factorize": (fp64["factorize_ms"] / float(np.mean(fac_ms))) if fp64 else None,
        "build_s": t_build, "build_phases_ms": st.get("t_build_phases_ms"), "gpu_launches": launches,
        "e2e": {"value": world * N / (e_ms / 1e3), "unit": "unknowns/s",
                "h2d_bytes_per_step": int(b_host.nbytes), "d2h_bytes_per_step": int(b_host.nbytes)},
        "clocks": clocks,
        "roofline": roof,
        "roofline_table": table,
        "measured_peaks_tflops": {k: round(v, 3) for k, v in MEASURED.items()},
        "solve_graph": solve_graph,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3)} for k, v in
                    sorted(st.get("kernels", {}).items(), key=lambda kv: -kv[1]["ms"])[:40 if args.profile_levels else 14]},
    }
    if args.json_extra:
        line["stats"] = st
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_subprocess(args)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def cpu_baseline_subprocess(args):
    """The oracle's factorize + refined solve of the 16^3 sub-grid on ONE host
    core (the paper's single-core setting): a child process with the BLAS
    thread pools limited to one thread before numpy loads; build untimed."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-only", "--grid", str(args.grid),
           "--eps", str(args.eps), "--chi", str(args.chi), "--nrhs", str(args.nrhs), "--seed", str(args.seed),
           "--prec", args.prec, "--tol", str(args.tol)]
    try:
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal to the GPU line
        return {"value": None, "unit": "unknowns/s", "cores": 1, "kind": "oracle", "error": str(e)[:200]}


def cpu_baseline_only(args):
    Nc, times, res = oracle_sample(args, repeat=1)
    print(json.dumps({"value": Nc / times[0], "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                      "sample": "oracle factorize + refined solve (to %g) of the 16^3 sub-grid (N=%d), %s, one "
                                "host core, build untimed" % (args.tol, Nc, oracle_precision(args)),
                      "final_residual": res}))


def main():
    args = parse()
    if args.cpu_baseline_only:
        return cpu_baseline_only(args)
    if args.impl == "ours" and args.workload == "batch":
        return run_batch(args)
    if args.impl == "ours" and args.workload == "grad":
        return run_grad(args)
    if args.impl == "ours" and args.workload == "rod":
        return run_rod(args)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
