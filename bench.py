"""Benchmark of the exact-GP hot path on one GB300 (or N replicas).

Workload (default): N = 32768 training and M = 8192 test points of the seeded
mass-spring-damper generator, 8 lagged-input regressors, (l, nu, sigma^2) =
(1, 1, 0.1); mixed precision (128 x 128 tiles of 256) by default, with one
FP64 run (same tiles) on the same inputs for the speed-ups and the
per-output relative errors, and the same workload with 128 regressors;
--precision fp64 benchmarks the FP64 path.  Inputs are resident in HBM
before the timed region; the factor alone (4.3 GB of tiles) is far larger
than L2.

One step = one pass of the whole hot path, three calls on the handle:
  set_hyper(theta0) ; gp_predict(Xs -> mean, var)   predict+variance (assembly, Cholesky,
                                                    alpha, cross-covariance, multi-RHS solve,
                                                    mean, variance and its correction)
  gp_predict(Xs -> full covariance)                 on the same factor
  set_hyper(theta0) ; gp_optimize(1 step)           NLML+grad (assembly, Cholesky, alpha,
                                                    NLML, K^{-1}, adjoint gradient, Adam)
Headline value: predict+variance ms, plus NLML+grad steps/s, each the mean
over the timed steps of one CUDA-event interval around its call sequence.
--impl reference times the plain FP64 CPU oracle on a bounded sample of the
same workload and scales each phase by its own operation count.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "predict+variance ms & NLML+grad steps/s @n=32768; mixed vs FP64 at 1e-8 rel"
# Exact digit-pair products of k_ozaki_tc: x~0 in 2 digits, K in 6, pairs (s, u) with s + u <= 7.
OZAKI_PAIRS = 11
# DRAM bytes (read + write) of one k_ozaki_tc launch at N = 32768, M = 8192: the ncu
# capture of the current kernel at N = 8192, M = 2048 (1.647 GB) scaled by the operand
# stream M N^2 (x 64); None for any other size.
OZAKI_TRAFFIC_FULL = 1.647e9 * 64
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
NOMINAL_BF16_TFLOPS = 2250.0      # dense, per GPU
NOMINAL_FP64_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "fp64_ozaki"], default="mixed")
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--m", type=int, default=8192)
    ap.add_argument("--d", type=int, default=8)
    ap.add_argument("--tiles", type=int, default=None, help="tiles per dimension (default 128: tiles of 256)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=2048)
    ap.add_argument("--cpu-sample-m", type=int, default=512)
    ap.add_argument("--no-compare", action="store_true", help="mixed: skip the FP64 comparison run")
    ap.add_argument("--fp64-tiles", type=int, default=128)
    ap.add_argument("--no-d128", action="store_true", help="mixed: skip the 128-regressor line")
    ap.add_argument("--no-learned-init", action="store_true",
                    help="skip the learned-initialiser measurement (small corpus, untimed for value)")
    args = ap.parse_args()
    if args.tiles is None:
        args.tiles = 128
    return args


HYP0 = (1.0, 1.0, 0.1)


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except OSError:
        return None


_FP64_PEAK = None


def fp64_peak():
    """FP64 tensor peak: mma.sync.m8n8k4.f64 throughput measured on this GPU in this
    run (gp_measure_fp64_peaks), else the fallback (nominal FP64/BF16 ratio x 1.9 PF)."""
    global _FP64_PEAK
    if _FP64_PEAK is None:
        try:
            from paper_2505_00136_gb300 import gprat
            dmma, _ = gprat.measure_fp64_peaks()
            _FP64_PEAK = (dmma, "of measured (mma.sync f64 throughput loop, this run)")
        except Exception:   # no device: fallback figure
            _FP64_PEAK = (1900.0 * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS,
                          "of fallback (1.9 PF bf16 x nominal fp64/bf16)")
    return _FP64_PEAK


# ---------------------------------------------------------------- CPU oracle baseline
def _oracle_sample(n, m, d, seed):
    """One bounded oracle run: assembly, Cholesky and prediction with variance at
    (n, m); returns the phase times in seconds."""
    import oracle
    from paper_2505_00136_gb300 import datagen as dg
    orc = oracle.Oracle()
    X, y, Xs, _ = dg.msd_dataset(n, m, d, seed)
    t0 = time.perf_counter()
    K = orc.cov_train(X, HYP0)
    t1 = time.perf_counter()
    orc.cholesky(K)
    t2 = time.perf_counter()
    orc.predict(X, y, Xs, HYP0)           # assembly + Cholesky + solves + cross-covariance + mean/var
    t3 = time.perf_counter()
    return {"assemble": t1 - t0, "cholesky": t2 - t1, "predict": t3 - t2}


def cpu_baseline(args, d, seed):
    """The plain FP64 CPU oracle, as it stands (single-threaded C), on a bounded
    sample of the workload: one run on one core, and one independent run per
    core at once (processes started with spawn; ms per problem = wall time /
    cores).  Each phase is scaled to N, M by its own operation count:
    assembly N^2 d, Cholesky N^3, solves and cross-covariance N^2 M."""
    import multiprocessing as mp
    ns, ms = args.cpu_sample_n, args.cpu_sample_m
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    ph = _oracle_sample(ns, ms, d, seed)
    rest = max(ph["predict"] - ph["assemble"] - ph["cholesky"], 0.0)
    fa, fc, fp = (args.n / ns) ** 2, (args.n / ns) ** 3, (args.n / ns) ** 2 * (args.m / ms)

    def scaled(p, rest_):
        return (p["assemble"] * fa + p["cholesky"] * fc + rest_ * fp) * 1e3

    one_core_ms = scaled(ph, rest)
    all_ms = None
    if cores > 1:
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(cores) as pool:
            res = pool.starmap(_oracle_sample, [(ns, ms, d, seed)] * cores)
        wall = time.perf_counter() - t0
        sample_wall = sum(r["predict"] for r in res) / cores          # mean per-process predict time
        per = {k: sum(r[k] for r in res) / cores for k in res[0]}
        rest_c = max(per["predict"] - per["assemble"] - per["cholesky"], 0.0)
        # one problem per core at once: the job's time per problem is its wall time / cores
        all_ms = scaled(per, rest_c) / cores
        all_note = (f"{cores} independent oracle runs at once (spawned processes, {wall:.1f} s wall, "
                    f"{sample_wall:.2f} s mean predict each)")
    out = {"value": all_ms if all_ms is not None else one_core_ms, "unit": "ms",
           "cores": cores if all_ms is not None else 1, "kind": "oracle",
           "one_core_ms": one_core_ms, "all_cores_ms": all_ms,
           "sample": (f"oracle (single-threaded FP64 C) at N={ns}, M={ms}, D={d}: assembly {ph['assemble']:.2f} s, "
                      f"Cholesky {ph['cholesky']:.2f} s, predict with variance {ph['predict']:.2f} s on one core; "
                      f"phases scaled to N={args.n}, M={args.m} by N^2 (assembly), N^3 (Cholesky) and N^2 M "
                      f"(solves, cross-covariance)" +
                      ("; value = all cores: " + all_note if all_ms is not None else ""))}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    seed = 1002
    samples = []
    cb = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(args, args.d, seed)
        if i >= args.warmup:
            samples.append(cb["value"])
    value = float(np.mean(samples))
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic mass-spring-damper (seeded)",
            "config": workload_config(args),
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": f"exact GP regression, SE kernel, N={args.n} train, M={args.m} test, "
                        f"D={args.d} lagged regressors, {args.tiles} tiles/dim",
            "n_train": args.n, "n_test": args.m, "regressors": args.d, "tiles_per_dim": args.tiles,
            "hyper": list(HYP0), "precision": args.precision,
            "l2": "inputs larger than L2 (factor tiles 4.3 GB at N=32768)"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: GPRAT_CLOCKS_DIR if set, else the system temporary directory
        cdir = os.environ.get("GPRAT_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(cdir, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm
def update_flops(T, b):
    """Algorithmic flops of all trailing SYRK/GEMM launches: sum_k sum over trailing tiles."""
    tot = 0.0
    for tt in range(1, T):
        tot += (tt * (tt - 1)) * b ** 3 + tt * float(b) ** 3   # GEMM: 2b^3 each (tt(tt-1)/2 of them); SYRK: b^3
    return tot


def replica_seed(rank):
    """Every rank of a multi-GPU launch solves its own problem (replicas, no
    data-path exchange): seed 1002 + rank."""
    return 1002 + rank


def max_over_ranks(values, device):
    """Element-wise maximum over the ranks of the initialised process group
    (the slowest replica sets the job's time); the values themselves when
    there is no group or it has one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def profiled_step(gprat, gp, Xs):
    """timed_step's three calls with per-launch events: phase ms and launch
    counts of each call (predict+variance, full covariance, NLML+grad)."""
    gp.profile(True)
    gp.profile_read()
    gp.set_hyper(HYP0)
    gp.predict(Xs, mean=True, var=True)
    p_pv = gp.profile_read()
    gp.predict(Xs, mean=False, var=False, cov=True)
    p_cv = gp.profile_read()
    gp.set_hyper(HYP0)
    st = gprat._lib.gp_optimize(gp.h, 1, 0.1, None)
    if st != gprat.GP_OK:
        raise gprat.GPError(st, -1, "gp_optimize")
    p_ng = gp.profile_read()
    gp.profile(False)
    return p_pv, p_cv, p_ng


def timed_step(gprat, gp, Xs, stream, torch):
    """One pass of the whole hot path, with CUDA events on the handle's stream
    around its two timed calls:
      predict+variance: set_hyper(theta0) ; gp_predict(Xs -> mean, var)
        (assembly, Cholesky, alpha, cross-covariance, multi-RHS solve, mean,
        variance; on the mixed path also the variance correction);
      full covariance: gp_predict(Xs -> cov) on the same factor;
      NLML+grad step: set_hyper(theta0) ; gp_optimize(1 step)
        (assembly, Cholesky, alpha, NLML, K^{-1}, adjoint gradient, Adam).
    Returns the three intervals in ms."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    gp.set_hyper(HYP0)
    ev[0].record(stream)
    gp.predict(Xs, mean=True, var=True)
    ev[1].record(stream)
    ev[2].record(stream)
    gp.predict(Xs, mean=False, var=False, cov=True)
    ev[3].record(stream)
    gp.set_hyper(HYP0)
    ev[4].record(stream)
    st = gprat._lib.gp_optimize(gp.h, 1, 0.1, None)
    ev[5].record(stream)
    if st != gprat.GP_OK:
        raise gprat.GPError(st, -1, "gp_optimize")
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3]), ev[4].elapsed_time(ev[5])


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2505_00136_gb300 import datagen as dg
    from paper_2505_00136_gb300 import gprat

    seed = replica_seed(rank)
    Xh, yh, Xsh, _ = dg.msd_dataset(args.n, args.m, args.d, seed)
    X = torch.from_numpy(Xh).to(dev)
    y = torch.from_numpy(yh).to(dev)
    Xs = torch.from_numpy(Xsh).to(dev)
    stream = torch.cuda.current_stream(dev)
    gp = gprat.GP(X, y, HYP0, n_tiles=args.tiles, precision=args.precision)
    info = gp.info()
    T, b = info["n_tiles"], info["tile"]

    for _ in range(args.warmup):
        timed_step(gprat, gp, Xs, stream, torch)
    torch.cuda.synchronize(dev)
    l0 = gp.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    pv, cv, ng = [], [], []
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            a, c, g = timed_step(gprat, gp, Xs, stream, torch)
            pv.append(a)
            cv.append(c)
            ng.append(g)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    total_ms = e0.elapsed_time(e1)
    launches = gp.launch_count() - l0
    K = args.steps
    predict_var_ms, cov_ms, grad_ms = float(np.mean(pv)), float(np.mean(cv)), float(np.mean(ng))
    ms_per_step = total_ms / K
    predict_var_ms, cov_ms, grad_ms, ms_per_step = max_over_ranks([predict_var_ms, cov_ms, grad_ms, ms_per_step],
                                                                  dev)

    # one more step with per-launch events (outside the timed region) for the phase
    # breakdown and the dominant kernel's launch time
    p_pv, p_cv, p_ng = profiled_step(gprat, gp, Xs)
    roof = roofline(args, p_pv, T, b)
    chol_ms = p_pv["potrf"][0] + p_pv["trsm"][0] + p_pv["update"][0]

    def phases(p):
        return {k: round(v[0], 3) for k, v in p.items() if v[1]}

    line = {"metric": METRIC, "value": predict_var_ms, "unit": "ms", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "mixed" if args.precision == "mixed" else "f64",
            "data": "synthetic mass-spring-damper (seeded), inputs resident in HBM",
            "config": workload_config(args),
            "nlml_grad_steps_per_s": 1e3 / grad_ms, "nlml_grad_ms": grad_ms, "full_cov_ms": cov_ms,
            "timing": "predict+variance and NLML+grad are each one timed call sequence (CUDA events on the "
                      "handle's stream around set_hyper+gp_predict and set_hyper+gp_optimize(1)); "
                      "phases_ms comes from one extra profiled step",
            "phases_ms": {"predict_var": phases(p_pv), "full_cov": phases(p_cv), "nlml_grad": phases(p_ng)},
            "roofline": roof, "gpu_launches": launches, "clocks": clk.summary()}
    if args.precision != "mixed":
        peak64 = fp64_peak()
        line["cholesky_tflops_fp64"] = (args.n ** 3 / 3.0) / (chol_ms * 1e-3) / 1e12
        line["cholesky_frac_of_fp64_peak"] = line["cholesky_tflops_fp64"] / peak64[0]
        line["fp64_peak_note"] = peak64[1]
    else:
        line["refine_iters"] = gp.info()["refine_iters"]
        line["refine_residual"] = gp.info()["refine_residual"]
        line["accuracy_note"] = ("mixed path: alpha, mean and variances FP64-level (refinement, exact "
                                 "variance correction); NLML, gradient and full covariance FP32-factor level "
                                 "(see mixed_vs_fp64.rel_err); the NLML+grad figure at FP64 accuracy is "
                                 "nlml_grad_fp64_accurate (the GP_FP64_OZAKI path)")
    if args.precision == "mixed" and not args.no_compare:
        line["mixed_vs_fp64"] = cmp = compare_fp64(args, gprat, torch, dev, gp, X, y, Xs, predict_var_ms, grad_ms)
        # NLML+grad at FP64 accuracy (the mixed path's NLML and gradient are FP32-factor level)
        line["nlml_grad_fp64_accurate"] = {"steps_per_s": cmp["fp64_ozaki"]["nlml_grad_steps_per_s"],
                                           "ms": cmp["fp64_ozaki"]["nlml_grad_ms"], "path": "fp64_ozaki",
                                           "rel_err_vs_fp64": cmp["fp64_ozaki"]["rel_err_vs_fp64"]}
    if args.precision == "mixed" and not args.no_d128:
        line["d128"] = d128_block(args, gprat, torch, dev, dg)
    if rank == 0 and world == 1 and not args.no_e2e:
        line["e2e"] = e2e(args, gprat, torch, dev, Xh, yh, Xsh)
    if rank == 0 and world == 1 and not args.no_learned_init:
        line["learned_init"] = learned_init_block(args, gprat, torch, dev, X, y)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, args.d, seed)
    gp.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def roofline(args, prof, T, b):
    """Roofline of the dominant kernel from one profiled step (per-launch CUDA
    events on the launching stream)."""
    upd_launch_ms = prof["update"][0] / max(prof["update"][1], 1)
    upd_flops_per_launch = update_flops(T, b) / max(T - 1, 1)
    if args.precision == "mixed":
        pk = peaks() or {}
        # kernels timed inside a seconds-long step: the sustained BF16 figure
        peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))
        peak_note = ("of measured bf16 sustained" if "bf16_tflops_sustained" in pk else
                     "of measured bf16 burst" if "bf16_tflops" in pk else "of fallback bf16")
        # k_ozaki_tc computes C = K x~0 for every test point (2 M N^2 flops of the method's own
        # work) as OZAKI_PAIRS exact BF16 digit-pair products, each 2 M N^2 tensor flops
        method_flops = 2.0 * args.m * args.n * args.n
        tensor_flops = OZAKI_PAIRS * method_flops
        oz_ms = prof["ozaki"][0] / max(prof["ozaki"][1], 1)
        achieved = method_flops / (oz_ms * 1e-3) / 1e12
        tensor_achieved = tensor_flops / (oz_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": "k_ozaki_tc (K x~0 for the exact variance correction, "
                                             f"{OZAKI_PAIRS} BF16 digit-pair products on tcgen05)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_note": peak_note,
                "traffic": OZAKI_TRAFFIC_FULL if (args.n, args.m) == (32768, 8192) else None,
                "traffic_note": "ncu DRAM bytes at N=8192, M=2048 scaled by M N^2 to N=32768, M=8192",
                "algorithmic_flops_per_launch": method_flops,
                "work_note": "achieved/frac count the method's own work, 2 M N^2 (K x~0); the emulation "
                             f"executes {OZAKI_PAIRS}x that on the BF16 tensor pipe (tensor_op_frac)",
                "tensor_flops_per_launch": tensor_flops, "tensor_achieved": tensor_achieved,
                "tensor_op_frac": tensor_achieved / peak,
                "avg_launch_ms": oz_ms, "launches": prof["ozaki"][1]}
        tensor_upd = 6.0 * upd_flops_per_launch      # six BF16 plane products per FP32-accurate product
        roof["second"] = {"kernel": "k_tgemm<OpUpdate> (trailing SYRK/GEMM, split-BF16 x6, tcgen05)",
                          "achieved": upd_flops_per_launch / (upd_launch_ms * 1e-3) / 1e12, "peak": peak,
                          "unit": "TFLOP/s",
                          "frac": upd_flops_per_launch / (upd_launch_ms * 1e-3) / 1e12 / peak,
                          "tensor_op_frac": tensor_upd / (upd_launch_ms * 1e-3) / 1e12 / peak,
                          "algorithmic_flops_per_launch": upd_flops_per_launch,
                          "avg_launch_ms": upd_launch_ms, "launches": prof["update"][1]}
        return roof
    if args.precision == "fp64_ozaki":
        # per factorisation step: one panel slicing and one k_ozgemm<OgChol> launch; 28 digit-pair
        # products (7 + 7 slices, levels 2..8) of the step's trailing SYRK/GEMM on the BF16 pipe
        pk = peaks() or {}
        peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))
        steps = max(T - 1, 1)
        step_ms = prof["update"][0] / steps
        achieved = upd_flops_per_launch / (step_ms * 1e-3) / 1e12
        return {"bound": "tensor", "kernel": "k_ozgemm<OgChol> (trailing SYRK/GEMM as 28 exact BF16 digit-pair "
                                              "products, FP64-accurate)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_note": "of measured bf16 sustained", "traffic": None,
                "work_note": "achieved/frac count the FP64 algorithmic flops of the update; the emulation executes "
                             "28x that on the BF16 tensor pipe (tensor_op_frac)",
                "tensor_op_frac": 28.0 * achieved / peak, "fp64_equivalent_frac_of_fp64_peak": achieved / fp64_peak()[0],
                "algorithmic_flops_per_launch": upd_flops_per_launch, "avg_launch_ms": step_ms,
                "launches": prof["update"][1]}
    peak, peak_note = fp64_peak()
    achieved = upd_flops_per_launch / (upd_launch_ms * 1e-3) / 1e12
    return {"bound": "tensor", "kernel": "k_update (trailing SYRK/GEMM, mma.sync f64)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_note": peak_note, "traffic": None,
            "algorithmic_flops_per_launch": upd_flops_per_launch,
            "avg_launch_ms": upd_launch_ms, "launches": prof["update"][1]}


def compare_fp64(args, gprat, torch, dev, gp_mixed, X, y, Xs, mixed_ms, mixed_grad_ms):
    """The FP64 path on the same inputs: its predict+variance and NLML+grad step
    times (each one timed call sequence, as the mixed path's) and the mixed
    path's relative errors against it, output by output."""
    def rel(a, b):
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))

    def worst(a, b, floor):
        return float(torch.max(torch.abs(a - b) / torch.clamp(torch.abs(b), min=floor)))

    gp_mixed.set_hyper(HYP0)
    mu_m, va_m, _ = gp_mixed.predict(Xs, mean=True, var=True)
    f_m, g_m = gp_mixed.nlml_grad()
    stream = torch.cuda.current_stream(dev)
    with gprat.GP(X, y, HYP0, n_tiles=args.fp64_tiles) as g64:
        pv, _, ng = timed_step_no_cov(gprat, g64, Xs, stream, torch)
        g64.set_hyper(HYP0)
        mu_d, va_d, _ = g64.predict(Xs, mean=True, var=True)
        f_d, g_d = g64.nlml_grad()
    # the FP64-accurate path on the tensor cores (GP_FP64_OZAKI): one warm-up, then one timed step
    with gprat.GP(X, y, HYP0, n_tiles=args.fp64_tiles, precision="fp64_ozaki") as go:
        timed_step_no_cov(gprat, go, Xs, stream, torch)
        pv_o, _, ng_o = timed_step_no_cov(gprat, go, Xs, stream, torch)
        go.set_hyper(HYP0)
        mu_o, va_o, _ = go.predict(Xs, mean=True, var=True)
        f_o, g_o = go.nlml_grad()
    oz = {"predict_var_ms": pv_o, "nlml_grad_ms": ng_o, "nlml_grad_steps_per_s": 1e3 / ng_o,
          "rel_err_vs_fp64": {"mean": rel(mu_o, mu_d), "var": rel(va_o, va_d), "nlml": abs(f_o - f_d) / abs(f_d),
                              "grad": float(np.linalg.norm(g_o - g_d) / np.linalg.norm(g_d))},
          "note": "GP_FP64_OZAKI: the FP64 path with every O(n^3) and O(n^2 m) product as exact BF16 digit "
                  "products on the tensor cores; FP64-level outputs"}
    return {"fp64_predict_var_ms": pv, "fp64_nlml_grad_ms": ng, "fp64_nlml_grad_steps_per_s": 1e3 / ng,
            "fp64_ozaki": oz,
            "speedup_predict_var": pv / mixed_ms, "speedup_nlml_grad": ng / mixed_grad_ms,
            "rel_err": {"mean": rel(mu_m, mu_d), "var": rel(va_m, va_d),
                        "mean_worst": worst(mu_m, mu_d, 1e-3 * float(torch.abs(mu_d).max())),
                        "var_worst": worst(va_m, va_d, 1e-12),
                        "nlml": abs(f_m - f_d) / abs(f_d),
                        "grad": float(np.linalg.norm(g_m - g_d) / np.linalg.norm(g_d)),
                        "grad_worst": float(np.max(np.abs(g_m - g_d) / np.abs(g_d)))},
            "note": "relative errors of the mixed outputs against the FP64 GPU path on the same inputs "
                    "(norm-wise, and worst element); the FP64 times are one cold call each"}


def timed_step_no_cov(gprat, gp, Xs, stream, torch):
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    gp.set_hyper(HYP0)
    ev[0].record(stream)
    gp.predict(Xs, mean=True, var=True)
    ev[1].record(stream)
    gp.set_hyper(HYP0)
    ev[2].record(stream)
    st = gprat._lib.gp_optimize(gp.h, 1, 0.1, None)
    ev[3].record(stream)
    if st != gprat.GP_OK:
        raise gprat.GPError(st, -1, "gp_optimize")
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]), None, ev[2].elapsed_time(ev[3])


def d128_block(args, gprat, torch, dev, dg):
    """The same workload with 128 lagged-input regressors (l = sqrt(128), the
    non-degenerate length scale at that width): mixed predict+variance and
    NLML+grad, 2 warm-up and 3 timed steps."""
    d = 128
    Xh, yh, Xsh, _ = dg.msd_dataset(args.n, args.m, d, 1002)
    X = torch.from_numpy(Xh).to(dev)
    y = torch.from_numpy(yh).to(dev)
    Xs = torch.from_numpy(Xsh).to(dev)
    hyp = (d ** 0.5, 1.0, 0.1)
    stream = torch.cuda.current_stream(dev)
    with gprat.GP(X, y, hyp, n_tiles=args.tiles, precision=args.precision) as gp:
        pv, ng = [], []
        for i in range(5):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            gp.set_hyper(hyp)
            ev[0].record(stream)
            gp.predict(Xs, mean=True, var=True)
            ev[1].record(stream)
            gp.set_hyper(hyp)
            ev[2].record(stream)
            st = gprat._lib.gp_optimize(gp.h, 1, 0.1, None)
            ev[3].record(stream)
            if st != gprat.GP_OK:
                raise gprat.GPError(st, -1, "gp_optimize")
            torch.cuda.synchronize()
            if i >= 2:
                pv.append(ev[0].elapsed_time(ev[1]))
                ng.append(ev[2].elapsed_time(ev[3]))
        gp.profile(True)
        gp.profile_read()
        gp.set_hyper(hyp)
        gp.predict(Xs, mean=True, var=True)
        prof = gp.profile_read()
        gp.profile(False)
    return {"regressors": d, "lengthscale": hyp[0], "predict_var_ms": float(np.mean(pv)),
            "nlml_grad_ms": float(np.mean(ng)), "nlml_grad_steps_per_s": 1e3 / float(np.mean(ng)),
            "predict_phases_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]}}


def learned_init_block(args, gprat, torch, dev, X, y):
    """Learned initialiser: a bounded corpus run (labels from the library's own
    Adam, GPU training, held-out steps to the default optimum) and the timed
    inference (summary + network) on the benchmark's training set."""
    from paper_2505_00136_gb300 import datagen as dg
    from paper_2505_00136_gb300 import learned_init as li
    res = li.run(n_train_sys=192, n_eval_sys=24, n=256, n_eval=256, d=32, label_steps=600, eval_steps=2000,
                 epochs=600)
    omega = torch.from_numpy(dg.rff_frequencies()).to(dev)
    model = li.new_model()
    scratch = torch.empty(gprat.GP_LEARNED_INIT_SCRATCH, dtype=torch.float64, device=dev)
    hp = gprat.gp_hyper()
    stream = torch.cuda.current_stream(dev)
    import ctypes
    times = []
    for _ in range(4):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = gprat.gp_learned_init(X.data_ptr(), y.data_ptr(), X.shape[0], X.shape[1], model.data_ptr(),
                                   omega.data_ptr(), scratch.data_ptr(), ctypes.byref(hp), stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
    return {"median_steps_default": res["median_steps_default"],
            "median_steps_learned": res["median_steps_learned"], "cap": res["cap"],
            "learned_capped": res["learned_capped"],
            "default_last100_rel_change_median": res["default_last100_rel_change_median"],
            "scale_note": "config 5 asks 2000 label systems at n=4096 (32 regressors) and 200 held-out at "
                          "n=16384; this bounded run uses the sizes in 'corpus'",
            "label_s": res["label_s"], "train_s": res["train_s"], "corpus": res["corpus"],
            "inference_ms_n32768": float(np.median(times[1:])), "inference_status": int(st)}


def e2e(args, gprat, torch, dev, Xh, yh, Xsh):
    """predict+variance through the public API from pinned host buffers:
    H2D of X, y, Xs and D2H of mean and var inside the timed region."""
    Xp = torch.from_numpy(Xh).pin_memory()
    yp = torch.from_numpy(yh).pin_memory()
    Xsp = torch.from_numpy(Xsh).pin_memory()
    mean = torch.empty(args.m, dtype=torch.float64).pin_memory()
    var = torch.empty(args.m, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with gprat.GP(Xp, yp, HYP0, n_tiles=args.tiles, precision=args.precision,
                  stream=stream.cuda_stream) as g2:
        st = gprat._lib.gp_predict_var(g2.h, Xsp.data_ptr(), args.m, mean.data_ptr(), var.data_ptr())
        if st != 0:
            raise gprat.GPError(st, -1, "gp_predict_var")
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return {"value": e0.elapsed_time(e1), "unit": "ms",
            "h2d_bytes_per_step": int(Xh.nbytes + yh.nbytes + Xsh.nbytes),
            "d2h_bytes_per_step": int(mean.numel() * 8 + var.numel() * 8),
            "note": "gp_create + gp_predict_var + gp_destroy from pinned host buffers, 1 step"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
