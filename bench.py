"""Benchmark of polynomial evaluation and differentiation at power series.

Workload (one step): value and full gradient of a p2-like polynomial (n=128
variables, 128 monomials of 64 distinct variables each, every coefficient and
input a random series truncated at degree d=152, deca double k=10), through
the library's C-ABI (pes_eval_grad), inputs resident in device memory.

Headline `value`: double-precision-equivalent TFLOP/s, counting the
algorithmic work of the method (Sec. 6.2 convention with the triangular
convolution): per convolution (d+1)(d+2)/2 multiplications and d(d+1)/2
additions of deca doubles at 3089 and 397 double operations, plus d+1 deca
double additions per addition job.

Also reported: `e2e` (same metric through the Python API with pinned host
buffers, copies inside the timed region), `roofline` of the convolution kernel
against the unit-count peak of the integer multiply-add pipe (and the measured
microbenchmark peak), the oracle as `cpu_baseline`, launch count and SM clocks
sampled during the timed region; beside the headline: p1 at d=8 in double
double (`config0`), two cells of the 64 x 64 system sweep (`config4`), the
whole batched recipe at k=2 and its first 512 instances at k=8 against plain
calls (`batched`, `batched_k8`, with the ceiling any batched launch has),
autograd, powers, complex series, large degrees and the system plan.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run, one rank per GPU) every rank
evaluates its own polynomial of the same shape (weak scaling, no collective on
the data path); rank 0 prints one JSON line.  --shard also times the headline
polynomial split over the ranks by monomials (strong scaling, exact integer
all-reduces).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "eval+grad DP-equiv TFLOP/s, k=10 d=152; batched vs plain ms/instance at tol"
UNIT = "TFLOP/s"
L2_FLUSH_BYTES = 256 << 20


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--arith", choices=["auto", "fp64", "int"], default="auto",
                    help="multiply-accumulate pipe of the headline run (auto: integer when the degree allows)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default CTA shape instead of timing the candidates on the first call")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the extra kernel-only timing of the FP64 variant")
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0: one lane per coefficient)")
    ap.add_argument("--staging", type=int, default=0, choices=[0, 1, 2],
                    help="staging depth of the convolution kernel (0: automatic / autotuned)")
    ap.add_argument("--split", type=int, default=0, choices=[0, 1, 2, 4, 8, 16],
                    help="parts per convolution job (0: automatic / autotuned)")
    ap.add_argument("--tile", type=int, default=0,
                    help="coefficients per output tile of the tiled kernel (0: whole series where they fit)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["p2", "p1", "p3", "sweep", "batch", "batch-small"], default="p2",
                    help="p2: the headline workload; p1 / p3: the paper's other test polynomials (analysis); "
                         "sweep: the 64x64 system over k x d (one JSON line per cell); "
                         "batch: the full batched recipe (2048 instances) batched vs plain")
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--d", type=int, default=152)
    ap.add_argument("--monomials", type=int, default=0,
                    help="use only the first M monomials of the workload (smaller case for profiling)")
    ap.add_argument("--batch-count", type=int, default=None,
                    help="instances of the batched comparison (default 2048: the whole recipe at k=2, and its "
                         "first 512 instances at k=8; 0 skips it in the default run)")
    ap.add_argument("--batch-k", type=int, default=2)
    ap.add_argument("--no-autograd", action="store_true")
    ap.add_argument("--no-complex", action="store_true",
                    help="skip the measurement of the workload with complex series")
    ap.add_argument("--no-large-degree", action="store_true",
                    help="skip the measurement of the tiled kernel (p2-like at d=1023, and d=471 with both kernels)")
    ap.add_argument("--no-system", action="store_true",
                    help="skip the measurement of the 64 x 64 system (values and Jacobian in one plan)")
    ap.add_argument("--no-powers", action="store_true",
                    help="skip the measurement of the workload with powers (monomials with exponents 1-3)")
    ap.add_argument("--no-config0", action="store_true",
                    help="skip the p1 d=8 k=2 measurement (config0)")
    ap.add_argument("--no-config4", action="store_true",
                    help="skip the two cells of the 64 x 64 system sweep (config4)")
    ap.add_argument("--shard", action="store_true",
                    help="with N > 1: also time one polynomial of the workload split over the N ranks by "
                         "monomials (strong scaling; exact integer all-reduces of grids and digit sums)")
    ap.add_argument("--cpu-sample-vars", type=int, default=12,
                    help="variables of the monomial the oracle evaluates as the CPU sample")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# operation counts
# ---------------------------------------------------------------------------

# Double-operation cost of one k-double multiplication and addition.  k = 10:
# the paper's counts (Sec. 6.2: 3089 and 397).  Other k: project-defined, the
# FP64 operation counts of the library's md_mul / md_add (the values
# pes_md_costs returns; a test keeps the two equal).  Kept here as a table so
# that the oracle arm loads nothing of the CUDA library.
MD_COSTS = {1: (1.0, 1.0), 2: (56.0, 27.0), 3: (129.0, 45.0), 4: (248.0, 63.0), 5: (425.0, 81.0),
            8: (1424.0, 135.0), 10: (3089.0, 397.0)}


def md_costs(k):
    return MD_COSTS[k]


def dp_equiv_ops(conv_jobs, add_jobs, d, k):
    """Double-operation equivalent of the algorithmic work (triangular products)."""
    cm, ca = md_costs(k)
    per_conv = (d + 1) * (d + 2) // 2 * cm + d * (d + 1) // 2 * ca
    return conv_jobs * per_conv + add_jobs * (d + 1) * ca


def paper_convention_ops(conv_jobs, add_jobs, d, k):
    """Double-operation equivalent in the paper's own count (Sec. 6.2): every
    convolution as (d+1)^2 k-double multiplications and d(d+1) additions (the
    zero-padded loop), every series addition as d+1 additions."""
    cm, ca = md_costs(k)
    return conv_jobs * ((d + 1) ** 2 * cm + d * (d + 1) * ca) + add_jobs * (d + 1) * ca


def digit_fma_flops(conv_jobs, d, digits):
    """Flops (2 per multiply-add) of the exact digit products the convolution
    kernel executes: L(L+1)/2 per term, (d+1)(d+2)/2 terms per convolution."""
    L = digits
    return conv_jobs * (d + 1) * (d + 2) // 2 * (L * (L + 1) // 2) * 2


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu_index), "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------

def dist_setup(args, backend=None):
    """World, rank and local rank from the torchrun environment; for N > 1 one
    process group (NCCL, one GPU per rank; gloo when asked for or without CUDA,
    for the host-side logic)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    elif backend == "nccl":
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(world, ops_per_step, steps, max_ms):
    """Whole-job throughput under weak scaling: every rank ran `steps` steps of
    its own workload of `ops_per_step` operations; the slowest rank's time."""
    return world * ops_per_step * steps / (max_ms * 1e-3) / 1e12


# ---------------------------------------------------------------------------
# CPU sample of the same workload (the oracle)
# ---------------------------------------------------------------------------

def cpu_sample(prob, nvars):
    """The oracle on one monomial of the workload restricted to its first
    `nvars` variables (value and gradient at the full degree and precision)."""
    from paper_2101_10881_gb300 import synth
    supp = [prob.supports[0][:nvars]]
    used = sorted(set(supp[0]))
    remap = {v: i for i, v in enumerate(used)}
    s2 = [[remap[v] for v in supp[0]]]
    coeff = prob.coeff[:, :2].copy()
    inputs = prob.inputs[:, used].copy()
    sub = synth.Problem("cpu sample", len(used), prob.d, prob.k, s2, coeff, inputs)
    return sub


def run_oracle(sub):
    from oracle import oracle
    t0 = time.perf_counter()
    oracle.eval_grad(sub.supports, sub.n, sub.coeff, sub.inputs)
    return time.perf_counter() - t0, oracle.threads()


def sample_ops(sub):
    m = len(sub.supports[0])
    conv = 3 * m - 3 if m >= 2 else 1
    add_jobs = 1  # a_0 + f_{1,m}; every partial has a single term
    return dp_equiv_ops(conv, add_jobs, sub.d, sub.k)


def sample_convolutions(sub):
    """Convolutions of the sample: credited (the reverse mode's 3m - 3, the count
    the metric charges) and executed by the oracle (naive: m for the value,
    m - 1 for each of the m partials)."""
    m = len(sub.supports[0])
    return {"credited_reverse_mode": 3 * m - 3 if m >= 2 else 1, "executed_by_oracle": m * m}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def reference_arm(args, world, rank):
    """The oracle as it stands, on the machine's host cores, on a bounded sample."""
    if rank != 0:
        return 0
    prob = make_workload(args, 0)
    sub = cpu_sample(prob, args.cpu_sample_vars)
    for _ in range(args.warmup):
        run_oracle(sub)
    times, cores = [], 1
    for _ in range(args.steps):
        t, cores = run_oracle(sub)
        times.append(t)
    total = sum(times)
    ops = sample_ops(sub) * args.steps
    value = ops / total / 1e12
    sample = (f"oracle value+gradient of monomial 1 of the workload restricted to its first "
              f"{len(sub.supports[0])} variables, d={sub.d}, k={sub.k}, per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(prob, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "convolutions_per_step": sample_convolutions(sub)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def make_workload(args, rank):
    from paper_2101_10881_gb300 import synth
    seed = args.seed + 1000 * rank
    if args.workload == "p1":
        return synth.make_problem("p1", synth.supports_p1(), 16, args.d, args.k, seed)
    if args.workload == "p3":
        return synth.make_problem("p3", synth.supports_p3(), 128, args.d, args.k, seed)
    return synth.config1(seed=seed, d=args.d, k=args.k)


def workload_config(prob, args):
    sizes = sorted({len(s) for s in prob.supports})
    shape = {"p2": "p2-like", "p1": "p1", "p3": "p3"}[args.workload]
    vars_ = sizes[0] if len(sizes) == 1 else sizes
    return {"workload": f"{shape} polynomial n={prob.n} N={prob.N} monomials of {vars_} "
                        f"variables, d={prob.d}, k={prob.k}, value + full gradient per step",
            "autotune": not args.no_autotune and args.threads == 0,
            "global_batch": 1, "seq_len": prob.d + 1, "parallelism": f"replicas x{args.gpus}",
            "arith": args.arith, "threads_per_cta": args.threads or "auto",
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write); workspace > L2"}


def kernel_source_hash():
    """Hash of the convolution kernel's sources with comments and white space
    removed: the DRAM counters of a capture stay valid while the code is the
    same."""
    import re
    h = hashlib.sha256()
    for f in ("kernels.cu", "digits.cuh", "kernels.hpp"):
        with open(os.path.join(ROOT, "paper_2101_10881_gb300", "csrc", f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(re.sub(r"\s+", "", text).encode())
    return h.hexdigest()[:16]


def traffic_per_launch(conv_jobs_full, arith):
    """DRAM bytes of one convolution launch from the committed ncu summary, if
    it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"dag_kernel_{arith}_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if "=" in line and not line.lstrip().startswith("#"):
            k_, v_ = line.split("=", 1)
            vals[k_.strip()] = v_.split("#")[0].strip()
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        per_job = float(vals["dram_bytes_per_launch"]) / float(vals["conv_jobs"])
    except (KeyError, ValueError, ZeroDivisionError):
        return None
    return per_job * conv_jobs_full


def ours_arm(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2101_10881_gb300 import pes, synth

    pes.build()
    dev = torch.device("cuda", local)
    prob = make_workload(args, rank)
    if args.monomials:
        prob = synth.Problem(prob.name, prob.n, prob.d, prob.k, prob.supports[: args.monomials],
                             prob.coeff[:, : args.monomials + 1].copy(), prob.inputs)
    plan = pes.Plan(prob.supports, prob.n, prob.d, prob.k, arith=args.arith, threads=args.threads,
                    with_vjp=False, profile=True, autotune=not args.no_autotune and args.threads == 0,
                    staging=args.staging, split=args.split, tile=args.tile)
    info = plan.info()
    C = torch.from_numpy(prob.coeff).to(dev)
    Z = torch.from_numpy(prob.inputs).to(dev)
    V = torch.empty(plan.shapes()["value"], dtype=torch.float64, device=dev)
    G = torch.empty(plan.shapes()["grad"], dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    fp64_peak = pes.fp64_peak(repeats=7)
    int_peak = pes.int_peak(repeats=7)

    ops_step = dp_equiv_ops(info["conv_jobs"], info["add_jobs"], prob.d, prob.k)
    digit_flops = digit_fma_flops(info["conv_jobs"], prob.d, info["digits"])

    def timed(p, steps, min_warm_s=0.0):
        """Device-resident steps with an L2 flush between them; per-step and
        convolution-kernel milliseconds from CUDA events on the launching stream.
        The untimed warm-up runs at least `warmup` steps and at least
        min_warm_s seconds (so that the clock sampler, started before it, has
        samples under load before the timed steps begin)."""
        t0 = time.perf_counter()
        done = 0
        while done < max(args.warmup, 3) or time.perf_counter() - t0 < min_warm_s:
            p.eval_grad(C, Z, V, G)
            torch.cuda.synchronize(dev)
            done += 1
        torch.cuda.synchronize(dev)
        p.check()
        barrier(world)
        torch.cuda.synchronize(dev)
        wall_box[0] = time.perf_counter()
        sms, cms, nl = [], [], 0
        for _ in range(steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.eval_grad(C, Z, V, G)
            e1.record(stream)
            e1.synchronize()
            sms.append(e0.elapsed_time(e1))
            t = p.last_timing()
            cms.append(t["conv_ms"])
            nl += t["launches"]
        torch.cuda.synchronize(dev)
        barrier(world)
        wall_box[1] = time.perf_counter()
        p.check()
        return sms, cms, nl

    wall_box = [0.0, 0.0]  # wall clock around the timed steps of the last timed() call
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, conv_ms, launches = timed(plan, args.steps, min_warm_s=0.5)
    wall = wall_box[1] - wall_box[0]
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(step_ms), world)

    # ---- end to end through the public API: pinned host buffers, copies timed ----
    hC = torch.from_numpy(prob.coeff).pin_memory()
    hZ = torch.from_numpy(prob.inputs).pin_memory()
    hV = torch.empty(V.shape, dtype=torch.float64).pin_memory()
    hG = torch.empty(G.shape, dtype=torch.float64).pin_memory()
    h2d = hC.numel() * 8 + hZ.numel() * 8
    d2h = hV.numel() * 8 + hG.numel() * 8
    e2e_ms = []
    barrier(world)
    torch.cuda.synchronize(dev)
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        C.copy_(hC, non_blocking=True)
        Z.copy_(hZ, non_blocking=True)
        plan.eval_grad(C, Z, V, G)
        hV.copy_(V, non_blocking=True)
        hG.copy_(G, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    barrier(world)
    e2e_total = max_over_ranks(sum(e2e_ms), world)

    value = whole_job_tflops(world, ops_step, args.steps, total_ms)
    e2e_value = whole_job_tflops(world, ops_step, args.steps, e2e_total)
    mean_conv = statistics.mean(conv_ms)
    work = (f"{info['conv_jobs']} convolutions x {(prob.d + 1) * (prob.d + 2) // 2} terms x "
            f"{info['digits'] * (info['digits'] + 1) // 2} digit products")
    arith = info["arith_name"]
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_max_mhz = clk.get("sm_max_mhz")
    if arith == "fp64":
        achieved = digit_flops / (mean_conv * 1e-3) / 1e12
        roofline = {"bound": "alu", "pipe": "fp64 (DFMA)", "achieved": achieved, "peak": fp64_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                    "peak_source": "measured: pes_fp64_peak DFMA microbenchmark (burst, all SMs), this run"}
    else:
        achieved = digit_flops / 2 / (mean_conv * 1e-3) / 1e12
        derived = 8 * 4 * nsm * clk_max_mhz * 1e6 / 1e12 if clk_max_mhz else None
        peak = derived if derived else int_peak
        roofline = {"bound": "alu", "pipe": "int (IMAD.WIDE 32x32+64)", "achieved": achieved, "peak": peak,
                    "unit": "Tops/s", "frac": achieved / peak,
                    "peak_source": ("derived: 8 lanes/clock per SM sub-partition (a 32x32+64 multiply-add "
                                    "occupies the heavy FMA pipe 4 clocks per warp, ncu) x 4 x SMs x max SM clock"
                                    if derived else "measured: pes_int_peak (no clock reading)"),
                    "peak_measured": {"value": int_peak, "frac": achieved / int_peak,
                                      "source": "pes_int_peak: 8x8 outer products of shared-memory digit rows "
                                                "(burst, all SMs), this run"}}
    roofline.update({"traffic": traffic_per_launch(info["conv_jobs"], arith), "work": work, "kernel_ms": mean_conv})

    # ---- the other multiply-accumulate pipe, kernel-only, same workload ----
    variants = {arith: {"ms_per_step": total_ms / args.steps, "value": value, "roofline_frac": roofline["frac"],
                        "pipe": roofline["pipe"], "digits": info["digits"]}}
    if not args.no_variants and arith == "int":
        p64 = pes.Plan(prob.supports, prob.n, prob.d, prob.k, arith="fp64", with_vjp=False, profile=True)
        i64 = p64.info()
        sms, cms, _ = timed(p64, max(2, min(args.steps, 3)))
        f64 = digit_fma_flops(i64["conv_jobs"], prob.d, i64["digits"])
        ms64 = max_over_ranks(sum(sms), world) / len(sms)
        variants["fp64"] = {"ms_per_step": ms64, "value": world * ops_step / (ms64 * 1e-3) / 1e12,
                            "roofline_frac": f64 / (statistics.mean(cms) * 1e-3) / 1e12 / fp64_peak,
                            "pipe": "fp64 (DFMA)", "digits": i64["digits"],
                            "dp_equiv_over_fp64_peak": ops_step / (ms64 * 1e-3) / 1e12 / fp64_peak}
        del p64
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64" if arith == "int" else "f64",
        "data": "synthetic", "config": dict(workload_config(prob, args), arith_used=arith,
                                            values="k-double series (k float64 limbs per coefficient)"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_total / args.steps},
        "roofline": roofline,
        "gpu_launches": launches,
        "clocks": clk,
        "dp_equiv_over_fp64_peak": value / world / fp64_peak,
        "variants": variants,
        "peaks": {"fp64_tflops": fp64_peak, "int_mad_wide_tops": int_peak},
        "ops_per_step": ops_step,
        "paper_convention": {
            "value": whole_job_tflops(world, paper_convention_ops(info["conv_jobs"], info["add_jobs"], prob.d,
                                                                  prob.k), args.steps, total_ms),
            "unit": UNIT,
            "rule": "the paper's count: (d+1)^2 k-double multiplications and d(d+1) additions per convolution"},
        "wall_s_timed_region": wall,
        "step_ms_spread": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms),
                           "steps": len(step_ms)},
        "plan": {"conv_jobs": info["conv_jobs"], "layers": info["layers"], "add_jobs": info["add_jobs"],
                 "grid": plan.info()["grid"], "threads_per_cta": plan.info()["threads"],
                 "staging_depth": plan.info()["staging"], "split": plan.info()["split"],
                 "smem_bytes": plan.info()["smem_bytes"], "digits": info["digits"], "tile": plan.info()["tile"]},
    }
    if not args.no_autograd:
        out["autograd"] = autograd_measure(args, dev, flush)
    if args.workload == "p2" and not args.no_powers:
        out["powers"] = powers_measure(args, dev, flush, roofline["peak"] if arith == "int" else None)
    if args.workload == "p2" and not args.no_complex:
        out["complex"] = complex_measure(args, dev, flush, roofline["peak"] if arith == "int" else None)
    if args.workload == "p2" and not args.no_large_degree:
        out["large_degree"] = large_degree_measure(args, dev, flush, roofline["peak"] if arith == "int" else None)
    if args.workload == "p2" and not args.no_system:
        out["system"] = system_measure(args, dev, flush, roofline["peak"] if arith == "int" else None)
    if world > 1 and args.shard:
        out["shard"] = shard_measure(args, dev, world, rank, prob, ops_step, flush)
    int_peak_unit = roofline["peak"] if arith == "int" else None
    if args.workload == "p2" and not args.no_config0:
        out["config0"] = config0_measure(args, dev, flush)
    if args.workload == "p2" and not args.no_config4:
        out["config4"] = config4_measure(args, dev)
    count = 2048 if args.batch_count is None else args.batch_count
    if count > 0:
        out["batched"] = batch_measure(args, dev, count, k=2, peak=int_peak_unit)
        out["batched_k8"] = batch_measure(args, dev, min(count, 512), k=8, peak=int_peak_unit)
        out["batched_small"] = batch_measure(args, dev, 2048, small=True)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sub = cpu_sample(prob, args.cpu_sample_vars)
        t, cores = run_oracle(sub)
        out["cpu_baseline"] = {"value": sample_ops(sub) / t / 1e12, "unit": UNIT, "cores": cores,
                               "kind": "oracle", "seconds": t, "convolutions": sample_convolutions(sub),
                               "sample": f"value+gradient of monomial 1 restricted to its first "
                                         f"{len(sub.supports[0])} variables, d={sub.d}, k={sub.k}"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def config0_measure(args, dev, flush):
    """The paper's p1 at the smallest size of its tables: n=16, all 1820 products
    of 4 distinct variables, d=8, double double (random series, seed 0).
    Latency-bound: a few microseconds of digit work in 16,380 convolutions over
    4 layers.  ms per eval+grad step (CUDA events, L2 flushed between steps),
    kernels launched per step; the paper's V100 time for this shape (0.18 ms,
    sum of its kernels) is context only."""
    import torch
    from paper_2101_10881_gb300 import pes, synth
    prob = synth.config0(seed=args.seed)
    plan = pes.Plan(prob.supports, prob.n, prob.d, prob.k, with_vjp=False, profile=True, autotune=not args.no_autotune)
    C = torch.from_numpy(prob.coeff).to(dev)
    Z = torch.from_numpy(prob.inputs).to(dev)
    V = torch.empty(plan.shapes()["value"], dtype=torch.float64, device=dev)
    G = torch.empty(plan.shapes()["grad"], dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        plan.eval_grad(C, Z, V, G)
    torch.cuda.synchronize(dev)
    times, launches = [], 0
    for _ in range(max(args.steps, 5)):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.eval_grad(C, Z, V, G)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        launches = plan.last_timing()["launches"]
    plan.check()
    info = plan.info()
    ms = statistics.median(times)
    return {"workload": "p1 n=16 N=1820 monomials of 4 variables, d=8, k=2 (random series)",
            "ms_per_step": ms, "ms_min": min(times), "launches_per_step": launches,
            "value": dp_equiv_ops(info["conv_jobs"], info["add_jobs"], prob.d, prob.k) / (ms * 1e-3) / 1e12,
            "unit": UNIT, "conv_jobs": info["conv_jobs"], "threads_per_cta": info["threads"],
            "paper_v100_ms": 0.18, "paper_v100_note": "sum of the paper's kernel times on a V100 (context)"}


def config4_measure(args, dev):
    """64 polynomials in 64 variables, 512 monomials of 4-16 variables each,
    degree-0 random coefficients, inputs z_i = exp(a_i t): two cells of the
    k x d sweep (k=10 and k=2 at d=152), the 64 polynomials as one system plan:
    forward (values) and the autograd backward of L = sum_p sum_j v_pj^2, with
    the normwise error of two polynomials' values against the exact closed form.
    The whole 7 x 7 sweep: bench.py --workload sweep."""
    import numpy as np
    import torch
    from paper_2101_10881_gb300 import pes, synth
    from paper_2101_10881_gb300.autograd import poly_eval
    stream = torch.cuda.current_stream(dev)
    tol = {1: 1e-13, 2: 1e-29, 3: 1e-44, 4: 1e-60, 5: 1e-76, 8: 1e-123, 10: 1e-150}
    cells = {}
    for k, d in ((10, 152), (2, 152)):
        sysc = synth.config4(d, k, seed=args.seed)
        sysp = pes.System([supp for supp, _ in sysc.polys], sysc.n, d, k)
        C = torch.from_numpy(np.concatenate([c for _, c in sysc.polys], axis=1)).to(dev)
        Z = torch.from_numpy(sysc.inputs).to(dev)
        fb = []
        for it in range(3):
            Cg, Zg = C.clone().requires_grad_(True), Z.clone().requires_grad_(True)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            v = poly_eval(Cg, Zg, sysp)
            e1.record(stream)
            v.backward(2 * v.detach())
            e2.record(stream)
            e2.synchronize()
            if it >= 1:
                fb.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
        sysp.check()
        vals = v.detach().cpu().numpy()
        errs = [closed_form_err(supp, c, sysc.avals, vals[:, q], 53 * k + 64)
                for q, (supp, c) in enumerate(sysc.polys[:2])]
        info = sysp.info()
        f = statistics.mean(t[0] for t in fb)
        b = statistics.mean(t[1] for t in fb)
        cells[f"k{k}_d{d}"] = {"k": k, "d": d, "forward_ms": f, "backward_ms": b, "backward_over_forward": b / f,
                               "forward_value": dp_equiv_ops(info["conv_jobs"], info["add_jobs"], d, k) / (f * 1e-3)
                               / 1e12, "unit": UNIT, "conv_jobs": info["conv_jobs"],
                               "closed_form_err": max(errs), "tol": tol[k], "within_tol": max(errs) <= tol[k]}
        del sysp, C, Z, Cg, Zg, v
    return {"workload": "system of 64 polynomials in 64 variables, 512 monomials of 4-16 variables, inputs "
                        "exp(a_i t), one system plan, forward + autograd backward of sum_p sum_j v_pj^2",
            "cells": cells}


def shard_measure(args, dev, world, rank, prob, ops_step, flush):
    """The workload's polynomial split over the ranks by monomials (contiguous
    ranges balanced by convolution jobs): per step every rank runs its
    convolutions, the ranks all-reduce the grids (maximum) and the exact digit
    sums (sum) over NCCL, and every rank rounds the whole value and gradient
    once.  Strong scaling: the whole polynomial per step, time of the slowest
    rank."""
    import torch
    from paper_2101_10881_gb300.shard import ShardPlan
    sp = ShardPlan(prob.supports, prob.n, prob.d, prob.k, world, rank, arith=args.arith)
    C = sp.coeff_of(torch.from_numpy(prob.coeff).to(dev))
    Z = torch.from_numpy(prob.inputs).to(dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        sp.eval_grad(C, Z)
    torch.cuda.synchronize(dev)
    times = []
    for _ in range(args.steps):
        flush.fill_(1)
        barrier(world)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sp.eval_grad(C, Z)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    sp.plan.check()
    ms = max_over_ranks(statistics.mean(times), world)
    return {"workload": "the headline polynomial split over the ranks by monomials", "ranks": world,
            "monomials_this_rank": sp.m_end - sp.m_begin, "ms_per_step": ms,
            "value": ops_step / (ms * 1e-3) / 1e12, "unit": UNIT, "scaling": "strong",
            "exchange": "all-reduce max of int32 grids, all-reduce sum of int64 digit sums"}


def autograd_measure(args, dev, flush):
    """Config 2 shape (p3: n=128, all 8128 pairs, d=152, k=4): forward through
    the autograd Function, then the backward (the VJP kernels) of
    L = sum_j v_j^2, both timed with CUDA events; backward / forward ratio."""
    import torch
    from paper_2101_10881_gb300 import pes, synth
    from paper_2101_10881_gb300.autograd import poly_eval
    prob = synth.config2(seed=args.seed)
    plan = pes.Plan(prob.supports, prob.n, prob.d, prob.k)
    C = torch.from_numpy(prob.coeff).to(dev)
    Z = torch.from_numpy(prob.inputs).to(dev)
    stream = torch.cuda.current_stream(dev)
    fwd, bwd = [], []
    for it in range(max(args.warmup, 3) + args.steps):
        Cg = C.clone().requires_grad_(True)
        Zg = Z.clone().requires_grad_(True)
        flush.fill_(1)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        v = poly_eval(Cg, Zg, plan)
        e1.record(stream)
        v.backward(2 * v.detach())
        e2.record(stream)
        e2.synchronize()
        if it >= max(args.warmup, 3):
            fwd.append(e0.elapsed_time(e1))
            bwd.append(e1.elapsed_time(e2))
    plan.check()
    f, b = statistics.mean(fwd), statistics.mean(bwd)
    info = plan.info()
    return {"workload": f"p3 n=128 N=8128 d={prob.d} k={prob.k}: value forward, VJP backward of sum_j v_j^2",
            "forward_ms": f, "backward_ms": b, "backward_over_forward": b / f,
            "backward_reuses_forward_products": True,
            "vjp_jobs": {"monomial_products": info["vjp_conv_jobs"], "correlations": info["vjp_corr_jobs"]}}


def powers_measure(args, dev, flush, peak):
    """Monomials with powers (Sec. 3): the p2-like workload (n=128, 128 monomials
    of 64 variables, d=152, k=10) with every exponent drawn uniformly from 1-3.
    Every convolution counts, the power table and the common factors included;
    ms per eval+grad step with CUDA events and an L2 flush between steps."""
    import numpy as np
    import torch
    from paper_2101_10881_gb300 import pes, synth
    prob = synth.config1(seed=args.seed)
    rng = np.random.default_rng(args.seed + 31)
    ex = [[int(e) for e in rng.integers(1, 4, size=len(s_))] for s_ in prob.supports]
    plan = pes.Plan(prob.supports, prob.n, prob.d, prob.k, exponents=ex, with_vjp=False, profile=True,
                    autotune=not args.no_autotune)
    C = torch.from_numpy(prob.coeff).to(dev)
    Z = torch.from_numpy(prob.inputs).to(dev)
    stream = torch.cuda.current_stream(dev)
    times, conv = [], []
    for it in range(max(args.warmup, 3) + args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.eval_grad(C, Z)
        e1.record(stream)
        e1.synchronize()
        if it >= max(args.warmup, 3):
            times.append(e0.elapsed_time(e1))
            conv.append(plan.last_timing()["conv_ms"])
    plan.check()
    info = plan.info()
    ms, cms = statistics.mean(times), statistics.mean(conv)
    ops = dp_equiv_ops(info["conv_jobs"], info["add_jobs"], prob.d, prob.k)
    macs = digit_fma_flops(info["conv_jobs"], prob.d, info["digits"]) / 2
    plain = pes.jobc_stats(prob.supports, prob.n)["conv_jobs"]
    return {"workload": "p2-like, n=128, 128 monomials of 64 variables, exponents uniform in 1-3, d=152, k=10",
            "ms_per_step": ms, "value": ops / (ms * 1e-3) / 1e12, "unit": UNIT,
            "conv_jobs": info["conv_jobs"], "power_and_factor_jobs": info["conv_jobs"] - plain,
            "roofline_frac": (macs / (cms * 1e-3) / 1e12) / peak if peak else None,
            "kernel_ms": cms, "threads_per_cta": info["threads"], "arith": info["arith_name"]}


def complex_measure(args, dev, flush, peak):
    """Complex coefficient and input series: the p2-like workload (n=128, 128
    monomials of 64 variables, d=152, k=10) with random complex series.  Every
    complex product is 4 real convolutions and 2 series additions (the paper's
    count for a complex multiplication: 4 multiplications and 2 additions);
    ms per eval+grad step with CUDA events and an L2 flush between steps; and
    the VJP (gradients with respect to real and imaginary parts) after it."""
    import numpy as np
    import torch
    from paper_2101_10881_gb300 import pes, synth
    prob = synth.config1(seed=args.seed)
    rng = np.random.default_rng(args.seed + 41)
    coeff = np.stack([prob.coeff, synth.random_md(rng, prob.k, prob.coeff.shape[1:])])
    inputs = np.stack([prob.inputs, synth.random_md(rng, prob.k, prob.inputs.shape[1:])])
    plan = pes.Plan(prob.supports, prob.n, prob.d, prob.k, complex_series=True, profile=True,
                    autotune=not args.no_autotune)
    C = torch.from_numpy(coeff).to(dev)
    Z = torch.from_numpy(inputs).to(dev)
    stream = torch.cuda.current_stream(dev)
    times, conv = [], []
    for it in range(max(args.warmup, 3) + args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.eval_grad(C, Z)
        e1.record(stream)
        e1.synchronize()
        if it >= max(args.warmup, 3):
            times.append(e0.elapsed_time(e1))
            conv.append(plan.last_timing()["conv_ms"])
    # the VJP of the real loss sum Re u Re v + Im u Im v, reusing the forward
    # products (the backward of the autograd Function)
    U = torch.from_numpy(np.stack([synth.random_md(rng, prob.k, (prob.d + 1,)) for _ in range(2)])).to(dev)
    vjp_ms = []
    for it in range(3):
        plan.eval_grad(C, Z)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.vjp(C, Z, U, reuse_forward=True)
        e1.record(stream)
        e1.synchronize()
        if it >= 1:
            vjp_ms.append(e0.elapsed_time(e1))
    plan.check()
    info = plan.info()
    ms, cms = statistics.mean(times), statistics.mean(conv)
    jobs = info["conv_jobs"]               # 6 per complex product: 4 convolutions, 2 additions
    products, series_adds = jobs * 4 // 6, jobs * 2 // 6
    cm, ca = md_costs(prob.k)
    ops = dp_equiv_ops(products, info["add_jobs"], prob.d, prob.k) + series_adds * (prob.d + 1) * ca
    macs = digit_fma_flops(products, prob.d, info["digits"]) / 2
    return {"workload": "p2-like, n=128, 128 monomials of 64 variables, complex series, d=152, k=10",
            "ms_per_step": ms, "value": ops / (ms * 1e-3) / 1e12, "unit": UNIT,
            "real_convolutions": products, "series_additions": series_adds,
            "roofline_frac": (macs / (cms * 1e-3) / 1e12) / peak if peak else None,
            "kernel_ms": cms, "threads_per_cta": info["threads"], "arith": info["arith_name"],
            "workspace_bytes": info["workspace_bytes"],
            "vjp_ms": statistics.mean(vjp_ms), "vjp_over_forward": statistics.mean(vjp_ms) / ms}


def system_measure(args, dev, flush, peak):
    """A system of 64 polynomials in 64 variables, each 512 monomials of 4-16
    variables, inputs exp(a_i t), d=152, k=10: the 64 values and the 64 x 64
    Jacobian matrix series in one plan (pes_plan_system, one P x n matrix per
    power of t) against one plan per polynomial (64 eval+grad calls), both
    without autotuning; ms per step with CUDA events and an L2 flush between
    steps; the two results compared bit for bit."""
    import numpy as np
    import torch
    from paper_2101_10881_gb300 import pes, synth
    sysc = synth.config4(152, 10, seed=args.seed)
    polys = [s_ for s_, _ in sysc.polys]
    sysp = pes.System(polys, sysc.n, sysc.d, sysc.k, profile=True)
    C = torch.from_numpy(np.concatenate([c for _, c in sysc.polys], axis=1)).to(dev)
    Z = torch.from_numpy(sysc.inputs).to(dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        out = []
        for it in range(2 + reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if it >= 2:
                out.append(e0.elapsed_time(e1))
        return statistics.mean(out)

    res = {}
    res["system"] = timed(lambda: res.__setitem__("sys_out", sysp.eval_system(C, Z, "matrix")), 3)
    conv_ms = sysp.last_timing()["conv_ms"]
    sysp.check()
    info = sysp.info()
    v, J = res.pop("sys_out")
    # autograd through the system plan: forward (values) and backward of
    # L = sum_p sum_j v_pj^2 (one VJP, one upstream series per polynomial)
    from paper_2101_10881_gb300.autograd import poly_eval
    fb = []
    for it in range(3):
        Cg, Zg = C.clone().requires_grad_(True), Z.clone().requires_grad_(True)
        flush.fill_(1)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        vv = poly_eval(Cg, Zg, sysp)
        e1.record(stream)
        vv.backward(2 * vv.detach())
        e2.record(stream)
        e2.synchronize()
        if it >= 1:
            fb.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
    sysp.check()
    del Cg, Zg, vv
    plans = [pes.Plan(s_, sysc.n, sysc.d, sysc.k, with_vjp=False) for s_ in polys]
    Cs = [torch.from_numpy(c).to(dev) for _, c in sysc.polys]
    outs = [None] * len(plans)

    def separate():
        for q, (pl, c) in enumerate(zip(plans, Cs)):
            outs[q] = pl.eval_grad(c, Z)

    res["plans"] = timed(separate, 3)
    for pl in plans:
        pl.check()
    same = all(torch.equal(v[:, :, q], outs[q][0]) and torch.equal(J[:, :, q], outs[q][1].permute(0, 2, 1))
               for q in range(len(plans)))
    ops = dp_equiv_ops(info["conv_jobs"], info["add_jobs"], sysc.d, sysc.k)
    macs = digit_fma_flops(info["conv_jobs"], sysc.d, info["digits"]) / 2
    return {"workload": "system of 64 polynomials in 64 variables, 512 monomials of 4-16 variables each, "
                        "inputs exp(a_i t), d=152, k=10: values + 64 x 64 Jacobian series",
            "ms_per_step": res["system"], "value": ops / (res["system"] * 1e-3) / 1e12, "unit": UNIT,
            "plans_ms_per_step": res["plans"], "plans_over_system": res["plans"] / res["system"],
            "conv_jobs": info["conv_jobs"], "jacobian_layout": "matrix [k][d+1][P][n]",
            "roofline_frac": (macs / (conv_ms * 1e-3) / 1e12) / peak if peak else None,
            "kernel_ms": conv_ms, "workspace_bytes": info["workspace_bytes"],
            "system_equals_plans_bitwise": bool(same), "launches_system": 4, "launches_plans": 4 * len(plans),
            "autograd": {"forward_ms": statistics.mean(t[0] for t in fb),
                         "backward_ms": statistics.mean(t[1] for t in fb),
                         "backward_over_forward": statistics.mean(t[1] for t in fb) / statistics.mean(t[0] for t in fb),
                         "loss": "sum_p sum_j v_pj^2, one VJP through the system plan"}}


def large_degree_measure(args, dev, flush, peak):
    """Degrees beyond the whole-series staging: the p2-like polynomial (n=128,
    128 monomials of 64 variables, k=10) at d=1023, where the tiled kernel
    runs (tiles of 128 coefficients), and at d=471, the largest degree the
    whole-series kernel takes, once with each kernel; ms per eval+grad step
    with CUDA events and an L2 flush between steps."""
    import numpy as np
    import torch
    from paper_2101_10881_gb300 import pes, synth
    base = synth.config1(seed=args.seed)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, d, tile in (("d1023_tiled", 1023, 0), ("d471_whole", 471, 0), ("d471_tiled", 471, 128)):
        rng = np.random.default_rng(args.seed + d)
        coeff = synth.random_md(rng, base.k, (base.N + 1, d + 1))
        inputs = synth.random_md(rng, base.k, (base.n, d + 1))
        plan = pes.Plan(base.supports, base.n, d, base.k, with_vjp=False, profile=True, tile=tile)
        C = torch.from_numpy(coeff).to(dev)
        Z = torch.from_numpy(inputs).to(dev)
        times, conv = [], []
        for it in range(2 + max(2, min(args.steps, 3))):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.eval_grad(C, Z)
            e1.record(stream)
            e1.synchronize()
            if it >= 2:
                times.append(e0.elapsed_time(e1))
                conv.append(plan.last_timing()["conv_ms"])
        plan.check()
        info = plan.info()
        ms, cms = statistics.mean(times), statistics.mean(conv)
        ops = dp_equiv_ops(info["conv_jobs"], info["add_jobs"], d, base.k)
        macs = digit_fma_flops(info["conv_jobs"], d, info["digits"]) / 2
        out[name] = {"d": d, "tile": info["tile"], "ms_per_step": ms, "value": ops / (ms * 1e-3) / 1e12,
                     "unit": UNIT, "kernel_ms": cms,
                     "roofline_frac": (macs / (cms * 1e-3) / 1e12) / peak if peak else None,
                     "threads_per_cta": info["threads"], "grid": info["grid"],
                     "workspace_bytes": info["workspace_bytes"]}
        del plan, C, Z
    out["workload"] = "p2-like, n=128, 128 monomials of 64 variables, k=10, random series"
    out["tiled_over_whole_at_d471"] = out["d471_tiled"]["ms_per_step"] / out["d471_whole"]["ms_per_step"]
    return out


def batch_measure(args, dev, count, small=False, k=None, peak=None):
    """Config 3 recipe (random sparse polynomials: n 8-128, m 16-2048 monomials of
    2-8 variables, d in {15,31,63,127,152}), first `count` instances, k=2 (or,
    with `small`, the small instances of synth.small_batch_shapes): one
    graph-captured batched call vs the same instances one plain pes_eval_grad
    call after another on one stream (plans built beforehand), ms per instance;
    the batched results must equal the plain ones."""
    import numpy as np
    import torch
    from paper_2101_10881_gb300 import pes, synth
    k = args.batch_k if k is None else k
    shapes = (synth.small_batch_shapes if small else synth.config3_shapes)(seed=args.seed, count=count)
    rng = np.random.default_rng(args.seed + 7)
    probs = []
    for b, (n, supp, d) in enumerate(shapes):
        N = len(supp)
        probs.append(synth.Problem(f"b{b}", n, d, k, supp, synth.random_md(rng, k, (N + 1, d + 1)),
                                   synth.random_md(rng, k, (n, d + 1))))
    B = pes.Batch([(p.supports, p.n, p.d) for p in probs], k, autotune=True, profile=True)
    C = torch.from_numpy(np.concatenate([p.coeff.ravel() for p in probs])).to(dev)
    Z = torch.from_numpy(np.concatenate([p.inputs.ravel() for p in probs])).to(dev)
    ln = B.lengths()
    V = torch.empty(ln["value"], dtype=torch.float64, device=dev)
    G = torch.empty(ln["grad"], dtype=torch.float64, device=dev)
    plans = [pes.Plan(p.supports, p.n, p.d, k, with_vjp=False) for p in probs]
    Vp = torch.empty_like(V)
    Gp = torch.empty_like(G)
    views = []
    for b, p in enumerate(probs):
        views.append((C[B.coeff_off[b]:B.coeff_off[b + 1]].view(k, p.N + 1, p.d + 1),
                      Z[B.input_off[b]:B.input_off[b + 1]].view(k, p.n, p.d + 1),
                      Vp[B.value_off[b]:B.value_off[b + 1]].view(k, p.d + 1),
                      Gp[B.grad_off[b]:B.grad_off[b + 1]].view(k, p.n, p.d + 1)))
    stream = torch.cuda.current_stream(dev)

    def batched():
        B.eval_grad(C, Z, V, G)

    def plain():
        for pl, (c, z, v, g) in zip(plans, views):
            pl.eval_grad(c, z, v, g)

    res = {}
    for name, fn in (("batched", batched), ("plain", plain)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        times = []
        for _ in range(max(2, min(args.steps, 3))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        res[name] = statistics.mean(times)
    B.check()
    same = bool(torch.equal(V, Vp) and torch.equal(G, Gp))
    info = B.info()
    what = ("small instances (n 4-16, 4-32 monomials of 2-4 variables, d in {7,15,31})" if small
            else "instances of the batched recipe")
    # digit multiply-adds of the whole batch, and what the unit-count peak of
    # the integer pipe would make of them: the ceiling of any batched launch
    L = info["digits"]
    macs = sum(pl.info()["conv_jobs"] * (p.d + 1) * (p.d + 2) // 2 for pl, p in zip(plans, probs)) * (L * (L + 1) // 2)
    out = {"workload": f"first {count} {what} (seed {args.seed}), k={k}",
           "instances": count, "k": k, "conv_jobs": info["conv_jobs"], "groups": info["grid"],
           "batched_ms_per_instance": res["batched"] / count, "plain_ms_per_instance": res["plain"] / count,
           "plain_over_batched": res["plain"] / res["batched"],
           "batched_equals_plain_bitwise": same, "launches_plain_per_call": 4 * count,
           "digit_mads": macs,
           "graph": "one CUDA graph: per group pack + persistent convolution + addition, groups on forked streams"}
    if peak:
        at_peak_ms = macs / (peak * 1e12) * 1e3
        out.update({"batched_frac_of_int_peak": at_peak_ms / res["batched"],
                    "plain_frac_of_int_peak": at_peak_ms / res["plain"],
                    "ceiling_plain_over_batched": res["plain"] / at_peak_ms,
                    "ceiling_rule": "plain time over the time of the batch's digit multiply-adds at the integer "
                                    "pipe's unit-count peak (no batched launch can be faster)"})
    return out


def limbs_to_fraction(limbs):
    from fractions import Fraction
    return sum((Fraction(float(x)) for x in limbs), Fraction(0))


def closed_form_err(supports, coeff, avals, value, prec_bits):
    """Normwise error of one value series (k, d+1) against the exact closed form
    c_0 + sum_m c_m exp((sum_{i in S_m} a_i) t) (degree-0 coefficients c_m, exact
    inputs a_i): every coefficient evaluated in integers scaled by 2^prec_bits,
    each term rounded once (an error far below every tolerance)."""
    from fractions import Fraction
    d = value.shape[1] - 1
    scale = 1 << prec_bits
    fact = [1]
    for j in range(1, d + 1):
        fact.append(fact[-1] * j)
    cs = [limbs_to_fraction(coeff[:, m, 0]) for m in range(coeff.shape[1])]
    ref = [0] * (d + 1)
    c0 = cs[0]
    ref[0] += (c0.numerator * scale) // c0.denominator
    for m, supp in enumerate(supports):
        sm = sum((Fraction(avals[i]) for i in supp), Fraction(0))
        c = cs[m + 1]
        num, den = c.numerator, c.denominator
        pn, pd = 1, 1
        for j in range(d + 1):
            ref[j] += (num * pn * scale) // (den * pd * fact[j])
            pn *= sm.numerator
            pd *= sm.denominator
    got = [limbs_to_fraction(value[:, j]) for j in range(d + 1)]
    num = max(abs(g * scale - r) for g, r in zip(got, ref))
    den = max(abs(r) for r in ref)
    return float(num / den) if den else 0.0


def sweep_arm(args, world, rank):
    """64 polynomials in 64 variables, each 512 monomials of 4-16 variables with
    degree-0 random coefficients, inputs z_i = exp(a_i t): for every k x d cell,
    forward (64 value series) and autograd backward of L = sum_p sum_j v_pj^2
    with respect to the shared inputs and all coefficients; closed-form check of
    the values of two polynomials per cell; and the 64 polynomials as one
    system plan (values and the 64 x 64 Jacobian in one launch), timed and
    compared bit for bit with the per-polynomial values, and the same forward
    and backward through the system plan."""
    import torch
    from paper_2101_10881_gb300 import pes, synth
    from paper_2101_10881_gb300.autograd import poly_eval
    if rank != 0:
        return 0
    pes.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    tol = {1: 1e-13, 2: 1e-29, 3: 1e-44, 4: 1e-60, 5: 1e-76, 8: 1e-123, 10: 1e-150}
    rows = []
    for k in synth.KS:
        for d in (0, 7, 15, 31, 63, 127, 152):
            sysc = synth.config4(d, k, seed=args.seed)
            plans = [pes.Plan(supp, sysc.n, d, k) for supp, _ in sysc.polys]
            coeffs = [torch.from_numpy(c).to(dev) for _, c in sysc.polys]
            Zb = torch.from_numpy(sysc.inputs).to(dev)
            info = [p.info() for p in plans]
            conv_jobs = sum(i["conv_jobs"] for i in info)
            add_jobs = sum(i["add_jobs"] for i in info)
            times = []
            for it in range(3):
                Z = Zb.clone().requires_grad_(True)
                Cs = [c.clone().requires_grad_(True) for c in coeffs]
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                vs = [poly_eval(c, Z, p) for c, p in zip(Cs, plans)]
                e1.record(stream)
                torch.autograd.backward(vs, [2 * v.detach() for v in vs])
                e2.record(stream)
                e2.synchronize()
                times.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
            for p in plans:
                p.check()
            fwd = min(t[0] for t in times)
            bwd = min(t[1] for t in times)
            errs = []
            for q in (0, 1):
                supp, c = sysc.polys[q]
                errs.append(closed_form_err(supp, c, sysc.avals, vs[q].detach().cpu().numpy(), 53 * k + 64))
            # the same 64 polynomials as one system plan: values and the 64 x 64
            # Jacobian in one launch, bit for bit the per-polynomial results
            sysp = pes.System([supp for supp, _ in sysc.polys], sysc.n, d, k)
            Csys = torch.cat(coeffs, dim=1)
            st, sfb = [], []
            for it in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sv, sj = sysp.eval_system(Csys, Zb)
                e1.record(stream)
                e1.synchronize()
                st.append(e0.elapsed_time(e1))
            sys_same = all(torch.equal(sv[:, q], vs[q].detach()) for q in range(len(vs)))
            # forward and backward of the same loss through the system plan: one
            # VJP with one upstream series per polynomial, the input gradient
            # summed over the polynomials exactly (autograd through 64 plans
            # adds the 64 input gradients limb by limb instead)
            for it in range(3):
                Zs = Zb.clone().requires_grad_(True)
                Cq = Csys.clone().requires_grad_(True)
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                v_sys = poly_eval(Cq, Zs, sysp)
                e1.record(stream)
                v_sys.backward(2 * v_sys.detach())
                e2.record(stream)
                e2.synchronize()
                sfb.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
            sysp.check()
            del sysp, Csys, sv, sj, v_sys, Zs, Cq
            ops = dp_equiv_ops(conv_jobs, add_jobs, d, k)
            row = {"cell": f"k={k} d={d}", "k": k, "d": d, "forward_ms": fwd, "backward_ms": bwd,
                   "backward_over_forward": bwd / fwd if fwd > 0 else None,
                   "forward_dp_equiv_tflops": ops / (fwd * 1e-3) / 1e12, "conv_jobs": conv_jobs,
                   "closed_form_err": max(errs), "tol": tol[k], "within_tol": max(errs) <= tol[k],
                   "arith": info[0]["arith_name"], "system_values_and_jacobian_ms": min(st),
                   "system_values_equal_plans_bitwise": bool(sys_same),
                   "system_forward_ms": min(t[0] for t in sfb), "system_backward_ms": min(t[1] for t in sfb)}
            rows.append(row)
            print(json.dumps(row), flush=True)
            del plans, vs, Cs, Z
            torch.cuda.empty_cache()
    print(json.dumps({"metric": METRIC, "sweep": "64x64 system, k x d", "cells": len(rows),
                      "all_within_tol": all(r["within_tol"] for r in rows),
                      "system_plan_bitwise_in_every_cell": all(r["system_values_equal_plans_bitwise"] for r in rows),
                      "max_backward_over_forward": max(r["backward_over_forward"] or 0 for r in rows)}), flush=True)
    return 0


def main():
    args = parse_args()
    world, rank, local = dist_setup(args) if args.impl == "ours" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        return reference_arm(args, world, rank)
    if args.workload == "sweep":
        return sweep_arm(args, world, rank)
    if args.workload in ("batch", "batch-small"):
        import torch
        from paper_2101_10881_gb300 import pes
        pes.build()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "batched": batch_measure(args, torch.device("cuda", local),
                                                                          args.batch_count or 2048,
                                                                          small=args.workload == "batch-small")}),
                  flush=True)
        return 0
    rc = ours_arm(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
