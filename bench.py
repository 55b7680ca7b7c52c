#!/usr/bin/env python
"""Benchmark of the Gauss-Newton hot path on GB300.

Workload: the plain Gauss-Newton system at scale (n = N = 256 variables and
equations, 256 terms of 16 distinct variables per polynomial, exponents
uniform in 1..5, unit-modulus coefficients, exact root built in), complex
double double.  A step is one whole Gauss-Newton step from the perturbed
start point x* + 1e-6: evaluate f and J (Section 2), MGS least squares on
[J, -f] (Section 3), x += dx (Section 4), through the C ABI call gn_newton.

The JSON line reports Newton steps/s as ``value`` (device-timed, inputs
resident), the same through host buffers as ``e2e``, per-precision
evaluation/differentiation throughput (monomials/s) and least-squares
times, the roofline of the dominant kernel group, and the CPU oracle timed
on this machine's host cores.

Under torchrun each rank solves its own independent system (weak scaling,
no collective on the data path).  ``--impl reference`` times the CPU oracle
on the same workload and metric.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "complex DD/QD monomial eval+diff/s; Newton steps/s; % of FP64 peak vs plain"
UNIT = "Newton steps/s"
WORKLOAD = "gn256"
L2_BYTES = 129 * 2 ** 20
# Issue rates per SM per clock of the pipes the kernels use: 2 FP64 lanes
# (GB300's nominal 1.25 TFLOP/s FMA rate over 152 SMs at 2070 MHz) and 64
# 32-bit IMAD lanes (half the 128 FP32 lanes).  Peaks are these times the
# device's SM count and maximum SM clock (device_peaks); the probes in
# probe/rates.cu measure the same pipes (measured_rates).
FP64_LANES_PER_SM = 2
IMAD_LANES_PER_SM = 64
PRECS = {"d": 1, "dd": 2, "qd": 4}
# DRAM bytes (read + write) of one k_mgs_int launch at 256 x 257, by limbs,
# from a one-kernel ncu capture of the current kernel with the L2 kept
# between kernels (--only mgs under ncu); null for a precision without a
# capture of the current kernel
MGS_TRAFFIC = {1: 132864 + 559360, 2: 202240 + 2200064, 4: 436480 + 3690496}
# untimed steps run just before the timed region while the clocks are sampled
SOAK_S = 1.0
# kernels one Gauss-Newton step launches at n = 256 (integer arithmetic):
# k_powers_cf, k_monomials_cf, k_sum_jacobian_cf, k_sum_f_cf, k_mgs_int,
# k_bs_inv and k_backsub_cl (the blocked back substitution), k_update
LAUNCHES_PER_STEP = 8

# FP64 instructions (DADD, DMUL, DFMA each one) per complex operation of the
# device arithmetic in csrc/mw.cuh, counted from the source.
FP64_COST = {
    1: dict(mul=4, add=2, scale=2, mul_real=2, abs2=2),
    2: dict(mul=38, add=22, scale=12, mul_real=14, abs2=19),
    4: dict(mul=456, add=152, scale=128, mul_real=232, abs2=228),
}


def algorithmic_fp64(system, L):
    """FP64 instructions of one evaluation (Section 2) and one MGS least-squares
    solve (Section 3) of ``system``, from the operation counts of the method
    and the per-operation costs above."""
    import numpy as np

    c = FP64_COST[L]
    k = np.diff(system.mono_ptr)
    cs = np.concatenate([[0], np.cumsum(system.exp >= 2)])
    ell = cs[system.mono_ptr[1:]] - cs[system.mono_ptr[:-1]]
    mults = np.where(k >= 2, 3 * k - 3, np.where(k == 1, 1, 0)) + ell
    pmax = max(int(system.exp.max()) - 1, 1)
    eval_ops = int(mults.sum()) * c["mul"] + int(k.sum()) * c["scale"]
    eval_ops += system.n * (pmax - 1) * c["mul"]
    # term sums: about one complex addition per contribution (J) and per term (f)
    eval_ops += (system.nnz + system.T) * c["add"]
    m, n = system.N, system.n
    pairs = m * n * (n + 1) // 2
    mgs_ops = pairs * 2 * (c["mul"] + c["add"]) + (n + 1) * m * (c["abs2"] + c["add"] + c["mul_real"])
    back_ops = n * (n - 1) // 2 * (c["mul"] + c["add"]) + n * c["mul_real"]
    return eval_ops, mgs_ops + back_ops


def algorithmic_imad_mgs(m, ncols, L):
    """32-bit partial products (IMAD lane-instructions) of the MGS factorisation
    (Section 3) of an m x ncols complex matrix with L-limb integer mantissas:
    every column's norm (2 real squares per entry) and normalisation (2 real
    products per entry), and per column pair one dot and one axpy (4 real
    products per entry each); a real product of two L-limb mantissas is
    L^2 64 x 64-bit products of 4 partial products each."""
    pairs = ncols * (ncols - 1) // 2
    real_products = ncols * 4 * m + pairs * 8 * m
    return real_products * 4 * L * L


def device_peaks(dev):
    """FP64 and IMAD issue peaks (G lane-instructions/s) of the device: lanes
    per SM per clock x SMs (read from the device) x maximum SM clock (from
    nvidia-smi, else the GB300's 2070 MHz)."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz, src = 2070.0, "GB300 maximum (nvidia-smi unavailable)"
    try:
        out = subprocess.run(["nvidia-smi", f"--id={torch.cuda.current_device()}",
                              "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        mhz, src = float(out.splitlines()[0]), "nvidia-smi clocks.max.sm"
    except Exception:
        pass
    ghz = mhz / 1e3
    return {"sms": sms, "sm_max_mhz": mhz, "clock_source": src,
            "fp64_ginstr": FP64_LANES_PER_SM * sms * ghz, "imad_ginstr": IMAD_LANES_PER_SM * sms * ghz,
            "derivation": f"lanes/clk/SM x {sms} SMs x {mhz:.0f} MHz "
                          f"(FP64 {FP64_LANES_PER_SM}, IMAD {IMAD_LANES_PER_SM})"}


def measured_hbm_gbs() -> float:
    """The machine's measured copy bandwidth (GB/s) when the driver wrote it,
    else the fallback figure of one earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def measured_rates():
    """Issue rates of the FP64 FMA, FP64 tensor (DMMA), IMAD and FP32 FMA pipes
    measured by the probes of probe/rates.cu on this device (one launch each
    of about 20-60 ms, after one warm-up launch)."""
    import ctypes as C

    from paper_1402_2626_gb300 import build

    lib = C.CDLL(build.PROBE_LIB)
    lib.gn_probe_rate.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]
    out = {}
    for which, name, iters, unit in ((0, "fp64_fma", 20000, "G lane-op/s"),
                                     (1, "dmma_fp64", 5000, "GFLOP/s"),
                                     (2, "imad", 400000, "G lane-op/s"),
                                     (3, "fp32_fma", 600000, "G lane-op/s")):
        rate, ms = C.c_double(), C.c_double()
        st = lib.gn_probe_rate(which, 4, iters, C.byref(rate), C.byref(ms))
        out[name] = {"rate": rate.value, "unit": unit, "ms": ms.value} if st == 0 else {"error": st}
    return out


def rank_system(rank: int):
    """The independent system rank ``rank`` solves (weak scaling: one seeded
    system per rank, no exchange on the data path)."""
    from paper_1402_2626_gb300 import inputs

    return inputs.workload(WORKLOAD, rank)


def max_over_ranks(value: float, dist, device) -> float:
    """The largest ``value`` over all ranks (the job's time is its slowest rank)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, t_max: float) -> float:
    """Whole-job Newton steps/s: every rank takes ``steps`` steps of its own system."""
    return world * steps / t_max


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms; each sample
    is stamped on arrival, and only those inside the marked region count (the
    timed steps and the untimed run of the same steps just before them)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line))

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except Exception:
            self.proc = None
            return
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()

    def region(self, t0: float, t1: float):
        """The timed region, in time.perf_counter() seconds."""
        self.t0, self.t1 = t0, t1

    def stop(self):
        if self.proc is None:
            return summarize_clocks([], None, None)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.reader.join(timeout=5)
        return summarize_clocks(list(self.lines), self.t0, self.t1)


def summarize_clocks(lines, t0, t1):
    """Median SM clock, maximum clock and throttle reasons of the stamped
    nvidia-smi lines (FIELDS order) that fall in [t0, t1] (all of them when
    t0 is None)."""
    out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ts, line in lines:
        if t0 is not None and not (t0 <= ts <= t1):
            continue
        p = [q.strip() for q in line.split(",")]
        if len(p) < 9:
            continue
        try:
            sm.append(float(p[1]))
            mx.append(float(p[2]))
        except ValueError:
            continue
        for nm, flag in zip(names, p[5:9]):
            if flag.lower() == "active":
                reasons.add(nm)
    if sm:
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
               "reasons": sorted(reasons), "samples": len(sm)}
    if t0 is not None:
        out["window_s"] = t1 - t0
    return out


def oracle_steps(system, L, nsteps, nthreads):
    """Time ``nsteps`` Gauss-Newton steps of the CPU oracle (from x0 each)."""
    import oracle

    x0 = system.point("x0", L)
    times = []
    for _ in range(nsteps):
        t = time.perf_counter()
        oracle.newton_step(system, x0, L, nthreads=nthreads)
        times.append(time.perf_counter() - t)
    return times


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.machine()


def oracle_parts(system, L, cores):
    """The oracle's evaluation (reverse mode: common factor and sequential
    Speelpenning; definition mode: every partial by direct powering) and MGS
    least squares, each timed at one thread (the paper timed one core) and
    at all cores, on bounded samples scaled to the whole system: evaluation
    on a block of rows (its time is proportional to the rows), MGS whole."""
    import oracle

    x = system.point("x0", L)
    out = {}
    for mode, rows1, rows_all in (("reverse", 32, system.N), ("definition", 8, 64)):
        row = {}
        for threads, rows in ((1, rows1), (cores, rows_all)):
            rows = min(rows, system.N)
            t = time.perf_counter()
            oracle.evaluate(system, x, L, mode, rows=(0, rows), nthreads=threads)
            dt = time.perf_counter() - t
            row[f"{threads}_thread_ms"] = 1e3 * dt * system.N / rows
            row[f"{threads}_thread_sample_rows"] = rows
        out[f"eval_{mode}"] = row
    f, J, _ = oracle.evaluate(system, x, L, "reverse", nthreads=cores)
    A = oracle.augmented(f, J)
    mg = {}
    for threads in (cores, 1):
        t = time.perf_counter()
        oracle.mgs(A, L, nthreads=threads)
        mg[f"{threads}_thread_ms"] = 1e3 * (time.perf_counter() - t)
    out["mgs"] = mg
    one = out["eval_reverse"]["1_thread_ms"] + mg["1_thread_ms"]
    out["newton_steps_per_s_1_thread"] = 1e3 / one
    return out


def cpu_baseline(system, L, budget_s=15.0):
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    times = []
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s and len(times) < 20:
        times.extend(oracle_steps(system, L, 1, cores))
    return {"value": len(times) / sum(times), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} full Gauss-Newton steps of the {WORKLOAD} workload in "
                      f"{ {1: 'D', 2: 'DD', 4: 'QD'}[L]} ({sum(times):.1f} s)",
            "cpu": cpu_model(), "parts": oracle_parts(system, L, cores)}


def cpu_adjoint_baseline():
    """The oracle's coefficient gradient on the 128-variable workload (DD), at
    its own root, timed on the host cores: about one second of CPU work."""
    import oracle
    from paper_1402_2626_gb300 import inputs

    s = inputs.workload("adj128")
    cores = os.cpu_count() or 1
    x, _ = oracle.newton(s, s.point("x0", 2), 2, 4, nthreads=cores)
    t = time.perf_counter()
    oracle.adjoint(s, x, 2.0 * x, 2, nthreads=cores)
    return {"gradient_ms": 1e3 * (time.perf_counter() - t), "cores": cores, "kind": "oracle",
            "sample": "one coefficient gradient of the adj128 workload in DD"}


def run_section(args):
    """One extra section alone (``--only``), e.g. under a profiler."""
    import torch

    from paper_1402_2626_gb300 import build

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    build.build()
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    fn = {"rates": lambda: measured_rates(),
          "eval": lambda: eval_section(dev, flush, args),
          "mgs": lambda: mgs_section(dev, flush, args),
          "adjoint": lambda: adjoint_extra(dev, flush, args),
          "mixed": lambda: mixed_extra(dev, flush, args),
          "paper": lambda: paper_extra(dev, flush, args),
          "batched": lambda: batched(dev, args, device_peaks(dev))}[args.only]
    print(json.dumps({"section": args.only, args.only: fn()}), flush=True)
    return 0


def _timed_calls(fn, stream, flush, reps, prep=None):
    """Median device time (ms) of ``fn`` over ``reps`` calls, L2 flushed and
    ``prep`` run before each (outside the events), after one untimed call."""
    import torch

    if prep:
        prep()
    fn()
    ms = []
    for _ in range(reps):
        flush.zero_()
        if prep:
            prep()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def eval_section(dev, flush, args):
    """Evaluation and differentiation of the gn256 workload (gn_eval, f and
    the dense J, default arithmetic) at the precision of --prec, alone: for
    one-kernel profiles of the evaluation kernels."""
    import torch

    from paper_1402_2626_gb300 import gn

    L = PRECS[args.prec]
    system = rank_system(0)
    S = gn.System(system)
    x = torch.tensor(system.point("x0", L), device=dev)
    f = torch.empty((system.N, 2, L), dtype=torch.float64, device=dev)
    J = torch.empty((system.n, system.N, 2, L), dtype=torch.float64, device=dev)
    ms = _timed_calls(lambda: S.eval(args.prec, x, f, J), torch.cuda.current_stream(dev), flush,
                      max(3, min(args.steps, 5)))
    S.close()
    return {"workload": WORKLOAD, "precision": args.prec, "ms": ms,
            "monomials_per_s": system.T / (ms / 1e3), "algorithmic_bytes": eval_bytes(system, L)}


def mgs_section(dev, flush, args):
    """The factorisation alone (gn_mgs: k_mgs_int on the 256 x 257 matrix
    [J, -f] of the gn256 workload at x0) at the precision of --prec: for
    one-kernel profiles of the MGS kernel."""
    import torch

    from paper_1402_2626_gb300 import gn

    L = PRECS[args.prec]
    system = rank_system(0)
    S = gn.System(system)
    x = torch.tensor(system.point("x0", L), device=dev)
    f = torch.empty((system.N, 2, L), dtype=torch.float64, device=dev)
    J = torch.empty((system.n, system.N, 2, L), dtype=torch.float64, device=dev)
    S.eval(args.prec, x, f, J)
    Ab0 = torch.cat([J, -f[None]], 0).contiguous()
    Ab = Ab0.clone()
    R = torch.empty((system.n + 1, system.n + 1, 2, L), dtype=torch.float64, device=dev)
    status = torch.zeros((1,), dtype=torch.int32, device=dev)
    ms = _timed_calls(lambda: S.mgs(args.prec, Ab, R, status), torch.cuda.current_stream(dev),
                      flush, max(3, min(args.steps, 5)), prep=lambda: Ab.copy_(Ab0))
    ok = int(status.item()) == 0
    S.close()
    return {"workload": WORKLOAD, "precision": args.prec, "ms": ms, "status_ok": ok,
            "algorithmic_imad": algorithmic_imad_mgs(system.N, system.n + 1, L)}


def run_reference(args):
    """The CPU oracle on the same workload, metric and steps (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1402_2626_gb300 import inputs

    import oracle

    oracle.build()
    L = PRECS[args.prec]
    system = inputs.workload(WORKLOAD, 0)
    cores = os.cpu_count() or 1
    oracle_steps(system, L, args.warmup, cores)
    times = oracle_steps(system, L, args.steps, cores)
    total = sum(times)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": 256, "n": 256, "terms_per_poly": 256, "k": 16,
                   "dmax": 5, "precision": args.prec},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full Gauss-Newton steps, CPU oracle, {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="dd", choices=list(PRECS))
    ap.add_argument("--no-extras", action="store_true", help="skip per-precision breakdowns")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched configuration")
    ap.add_argument("--only", choices=["rates", "eval", "mgs", "adjoint", "mixed", "paper", "batched"],
                    help="run one extra section alone and print it as the JSON line (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_section(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_1402_2626_gb300 import build, gn, inputs

    if local == 0:
        build.build()
    if dist:
        dist.barrier()
    L = PRECS[args.prec]
    system = rank_system(rank)
    S = gn.System(system)
    x0 = torch.tensor(system.point("x0", L), device=dev)
    x = x0.clone()
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        S.newton(args.prec, x, 1)

    for _ in range(max(args.warmup, 3)):
        x.copy_(x0)
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps (outside the events)
    clocks = ClockSampler(torch.cuda.current_device())
    if rank == 0:
        clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    # the same steps, untimed, for ~1 s just before the timed region, so
    # that the 200 ms clock samples see the GPU under this load (a timed
    # region of a few tens of ms falls between two samples)
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < SOAK_S:
        for _ in range(10):
            flush.zero_()
            x.copy_(x0)
            step()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        x.copy_(x0)
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    clocks.region(t_soak, time.perf_counter())
    if dist:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else {}
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_local = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_local, dist, dev)
    value = job_throughput(world, args.steps, t_max)

    # ---- end to end through host buffers: H2D of x, gn_newton, D2H of x
    hx0 = torch.tensor(system.point("x0", L)).pin_memory()
    hx = torch.empty_like(hx0).pin_memory()
    e2e_ms = []
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        x.copy_(hx0, non_blocking=True)
        step()
        hx.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t))
    e2e_local = max_over_ranks(sum(e2e_ms) / 1e3, dist, dev)
    e2e = {"value": job_throughput(world, args.steps, e2e_local), "unit": UNIT,
           "h2d_bytes_per_step": int(hx0.numel() * 8), "d2h_bytes_per_step": int(hx.numel() * 8 + 8 * 2 * 64 * 3)}

    extras = {}
    roofline = None
    head = {}
    if rank == 0 and not args.no_extras:
        peaks = device_peaks(dev)
        peaks["hbm_gbs"] = measured_hbm_gbs()
        rates = measured_rates()
        extras, roofline = breakdown(S, system, dev, flush, args, peaks, rates)
        # the evaluation half of the metric, first in the line
        head["eval_diff_monomials_per_s"] = {
            p: {"int": extras["eval_diff"][p]["int"]["monomials_per_s"],
                "fp64": extras["eval_diff"][p]["fp64"]["monomials_per_s"]} for p in PRECS}
        extras["peaks"] = peaks
        extras["measured_rates"] = rates
        extras["adjoint"] = adjoint_extra(dev, flush, args)
        extras["mixed"] = mixed_extra(dev, flush, args)
        extras["paper_workloads"] = paper_extra(dev, flush, args)
        if not args.no_batch:
            extras["batched"] = batched(dev, args, peaks)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, **head, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": system.N, "n": system.n, "terms_per_poly": 256,
                       "k": 16, "dmax": 5, "T": system.T, "precision": args.prec,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "flushed between timed steps (256 MiB write)"},
            "e2e": e2e, "gpu_launches": LAUNCHES_PER_STEP * args.steps,
            "clocks": clk, "roofline": roofline, **extras,
        }
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(system, L)
            if "adjoint" in line:
                line["adjoint"]["cpu_baseline"] = cpu_adjoint_baseline()
        print(json.dumps(line), flush=True)
    S.close()
    if dist:
        dist.destroy_process_group()
    return 0


# Table 5 of the paper: evaluation and differentiation of cyclic n-roots on
# one NVIDIA K20C, ms (context only: another GPU, another decade)
PAPER_CYCLIC_MS = {"d": {128: 1.13, 256: 6.97, 384: 21.59, 448: 32.68, 512: 46.43},
                   "dd": {128: 6.45, 256: 37.15, 384: 120.48, 448: 182.19, 512: 267.39},
                   "qd": {128: 29.45, 256: 152.82, 384: 513.78, 448: 809.15}}


def paper_extra(dev, flush, args):
    """The paper's own benchmark systems (Section 5): evaluation and
    differentiation of cyclic n-roots at the sizes of Table 5 in D, DD and QD
    (gn_eval, f and the full Jacobian), seven DD Newton iterations on the
    homotopy f(x) - t f(z) of cyclic 512-roots from z, and six DD Newton
    iterations on the Chandrasekhar H-equation (c = 33/64, H = 1) at n = 1024
    (Table 3's first size).  Device events, L2 flushed first."""
    import torch

    from paper_1402_2626_gb300 import gn, inputs

    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps, prep=None):
        if prep:
            prep()
        fn()
        ms = []
        for _ in range(reps):
            flush.zero_()
            if prep:
                prep()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    out = {"cyclic_eval_diff_ms": {}, "paper_k20c_ms": PAPER_CYCLIC_MS}
    for n in (128, 256, 384, 448, 512):
        s = inputs.cyclic(n, seed=1)
        S = gn.System(s)
        row = {}
        for prec, L in PRECS.items():
            x = torch.tensor(s.point("x0", L), device=dev)
            f = torch.empty((s.N, 2, L), dtype=torch.float64, device=dev)
            J = torch.empty((s.n, s.N, 2, L), dtype=torch.float64, device=dev)
            row[prec] = timed(lambda: S.eval(prec, x, f, J), 3)
        out["cyclic_eval_diff_ms"][n] = row
        S.close()
    s = inputs.cyclic_homotopy(512)
    S = gn.System(s)
    x0 = torch.tensor(s.point("x0", 2), device=dev)
    x = x0.clone()
    ms = timed(lambda: S.newton("dd", x, 7), 3, lambda: x.copy_(x0))
    x.copy_(x0)
    rep = S.newton("dd", x, 7)
    out["cyclic512_homotopy_dd_7_iterations"] = {"ms": ms, "dx_norms": rep["dx_norm"],
                                                 "paper_k20c_s": 5930.96}
    S.close()
    s = inputs.chandrasekhar(1024)
    S = gn.System(s)
    x0 = torch.tensor(s.point("x0", 2), device=dev)
    x = x0.clone()
    ms = timed(lambda: S.newton("dd", x, 6), 2, lambda: x.copy_(x0))
    x.copy_(x0)
    rep = S.newton("dd", x, 6)
    out["chandrasekhar1024_dd_6_iterations"] = {"ms": ms, "dx_norms": rep["dx_norm"],
                                                "paper_k20c_gpu2_s": 20.083, "paper_cpu_s": 322.360}
    S.close()
    return out


def mixed_extra(dev, flush, args):
    """Time to a quad-double root on the mixed-precision workload (N = 1536
    polynomials, n = 1024 variables, 63 terms of 8 variables plus a constant
    per polynomial, exponents 1..4, consistent): gn_newton_mixed with two
    double-precision steps and five QD refinement steps against four plain
    QD Gauss-Newton steps (gn_newton), both from x0 = x* + 1e-6.  Device
    events, L2 flushed first; the error of each result against the exact
    root x* built into the system is reported beside its time."""
    import numpy as np
    import torch

    from paper_1402_2626_gb300 import gn, inputs

    s = inputs.workload("mix1536")
    S = gn.System(s)
    stream = torch.cuda.current_stream(dev)
    x0 = torch.tensor(s.point("x0", 4), device=dev)
    x = x0.clone()
    xs = torch.zeros_like(x0)
    xs[:, :, 0] = torch.tensor(s.xstar, device=dev)

    def timed(fn, reps):
        fn()
        ms = []
        for _ in range(reps):
            flush.zero_()
            x.copy_(x0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    def err():
        d = (x - xs).cpu().numpy()
        return float(np.abs(d[:, 0, :].sum(-1) + 1j * d[:, 1, :].sum(-1)).max())

    # two double steps leave the frozen Jacobian about 1e-10 from J(x*), so
    # each refinement step gains about ten digits: five reach the QD floor
    # (1.8e-66 from x*, as plain QD; a sixth changes nothing).  With one
    # double step the frozen Jacobian is 2e-10 from J(x*) and a refinement
    # step gains only five digits.
    D_STEPS, REFINE, QD_STEPS = 2, 5, 4
    mixed_ms = timed(lambda: S.newton_mixed("qd", x, D_STEPS, REFINE), 3)
    x.copy_(x0)
    rep = S.newton_mixed("qd", x, D_STEPS, REFINE)
    err_mixed = err()
    plain_ms = timed(lambda: S.newton("qd", x, QD_STEPS), 2)
    x.copy_(x0)
    S.newton("qd", x, QD_STEPS)
    err_plain = err()
    S.close()
    return {"workload": "mix1536", "N": s.N, "n": s.n, "T": s.T, "precision": "qd",
            "mixed": {"double_steps": D_STEPS, "refine_steps": REFINE, "ms": mixed_ms,
                      "err_vs_root": err_mixed, "dx_norms": rep["dx_norm"]},
            "plain_qd": {"steps": QD_STEPS, "ms": plain_ms, "err_vs_root": err_plain},
            "speedup_vs_plain_qd": plain_ms / mixed_ms}


def adjoint_extra(dev, flush, args):
    """The coefficient gradient at the converged root on the 128-variable
    workload (N = n = 128, 128 terms of 12 variables per polynomial plus a
    constant, exponents 1..3, complex DD): four Newton steps from x0, then
    gn_adjoint (evaluation and MGS at the root, forward substitution with R^H,
    lambda = Q w, one gradient per term).  Device events, L2 flushed first."""
    import torch

    from paper_1402_2626_gb300 import gn, inputs

    s = inputs.workload("adj128")
    L = 2
    S = gn.System(s)
    stream = torch.cuda.current_stream(dev)
    x0 = torch.tensor(s.point("x0", L), device=dev)
    x = x0.clone()
    grad = torch.empty((s.T, 2, L), dtype=torch.float64, device=dev)
    lam = torch.empty((s.N, 2, L), dtype=torch.float64, device=dev)
    reps = max(5, min(args.steps, 20))

    def timed(fn, prep):
        for _ in range(2):
            prep()
            fn()
        ms = []
        for _ in range(reps):
            flush.zero_()
            prep()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    newton_ms = timed(lambda: S.newton("dd", x, 4), lambda: x.copy_(x0))
    S.newton("dd", x, 4)
    xr = x.clone()
    g = 2.0 * xr
    grad_ms = timed(lambda: S.adjoint("dd", xr, g, grad, lam), lambda: None)
    # from the last Newton step's factorisation (the forward solve's own QR)
    reuse_ms = timed(lambda: S.adjoint("dd", xr, g, grad, lam, reuse=True), lambda: None)
    S.close()
    return {"workload": "adj128", "N": s.N, "n": s.n, "T": s.T, "precision": "dd",
            "newton_4_steps_ms": newton_ms, "gradient_ms": grad_ms,
            "gradient_reuse_ms": reuse_ms,
            "gradient_over_newton_step": grad_ms / (newton_ms / 4),
            "gradients_per_s": s.T / (grad_ms / 1e3),
            "loss": "sum |x_j|^2 at the root (g = 2x)"}


def batched(dev, args, peaks):
    """The batched configuration: 4096 independent systems (n in [16, 128],
    M in [n/2, 2n] per polynomial, k in [2, 16], exponents 1..4), complex DD,
    one graph per Newton step; against the same systems stepped one at a time
    through the single-system path (gn_newton on each system in turn)."""
    import numpy as np
    import torch

    from paper_1402_2626_gb300 import gn, inputs

    t0 = time.perf_counter()
    b = inputs.batch_workload("batch4096")
    gen_s = time.perf_counter() - t0
    g = gn.Batch(b)
    L = 2
    x0 = torch.tensor(b.point("x0", L), device=dev)
    x = x0.clone()
    status = torch.zeros((b.S,), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    g.newton("dd", x, 1, status)  # tunes the launches, captures the step
    torch.cuda.synchronize()
    tuning = g.tuning("dd")
    reps = max(3, min(args.steps, 10))
    ms = []
    for _ in range(reps):
        x.copy_(x0)
        status.zero_()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.newton("dd", x, 1, status)
        e.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(e))
    step_ms = statistics.median(ms)
    ok = not bool(status.any().item())
    g.close()
    # the plain path, one system at a time, over every system of the batch:
    # each system is loaded and its step captured first (untimed), then one
    # gn_newton step of each, back to back, timed as a whole (each call
    # synchronizes to read its status, as a user's loop would)
    t_load = time.perf_counter()
    plain = []
    for s in range(b.S):
        sy = b.system(s)
        S1 = gn.System(sy)
        xs0 = torch.tensor(sy.point("x0", L), device=dev)
        xs = xs0.clone()
        S1.newton("dd", xs, 1)  # allocates the workspace, captures the step
        plain.append((S1, xs0, xs))
    load_s = time.perf_counter() - t_load
    loop_ms = []
    for _ in range(2):
        for _S1, xs0, xs in plain:
            xs.copy_(xs0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for S1, _xs0, xs in plain:
            S1.newton("dd", xs, 1)
        torch.cuda.synchronize()
        loop_ms.append(1e3 * (time.perf_counter() - t))
    for S1, _xs0, _xs in plain:
        S1.close()
    loop_total_ms = min(loop_ms)
    imad = sum(algorithmic_imad_mgs(int(n), int(n) + 1, L) for n in b.n)
    return {"workload": "batch4096", "systems": b.S, "terms": b.T, "precision": "dd",
            "ms_per_step": step_ms, "system_steps_per_s": b.S / (step_ms / 1e3), "all_ok": ok,
            "tuning": tuning,
            "loop_plain_ms_per_step": loop_total_ms,
            "loop_plain": f"one gn_newton step on each of the {b.S} systems in turn, measured "
                          f"(best of 2 loops; loading the systems and capturing their steps, "
                          f"{load_s:.0f} s, untimed)",
            "speedup_vs_loop": loop_total_ms / step_ms,
            "mgs_imad_per_step": imad,
            "mgs_imad_rate_lower_bound": {"achieved": imad / (step_ms / 1e3) / 1e9, "unit": "G IMAD/s",
                                          "peak": peaks["imad_ginstr"],
                                          "frac": imad / (step_ms / 1e3) / 1e9 / peaks["imad_ginstr"],
                                          "note": "MGS work only over the whole step time (evaluation not counted)"},
            "generate_s": gen_s}


def eval_bytes(system, L):
    """Algorithmic DRAM bytes of one evaluation in this library's layout: the
    packed occurrences (4 B: variable and exponent), term offsets (4 B), the
    coefficients (16 L B per term), x, f and the dense J (16 L B per entry)."""
    W = 16 * L
    return (4 * system.nnz + 4 * (system.T + 1) + W * system.T
            + W * (system.n + system.N + system.N * system.n))


def breakdown(S, system, dev, flush, args, peaks, rates):
    """Per-precision eval+diff (integer and FP64 arithmetic), least-squares and
    step times, and the roofline of the factorisation kernel (device events,
    L2 flushed before every timed call)."""
    import torch

    reps = max(5, min(args.steps, 20))
    stream = torch.cuda.current_stream(dev)
    out = {"eval_diff": {}, "lstsq_ms": {}, "newton_step_ms": {}}
    roof = None

    def timed(fn, prep=None):
        for _ in range(2):
            if prep:
                prep()
            fn()
        ms = []
        for _ in range(reps):
            flush.zero_()
            if prep:
                prep()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    for prec, L in PRECS.items():
        x = torch.tensor(system.point("x0", L), device=dev)
        f = torch.empty((system.N, 2, L), dtype=torch.float64, device=dev)
        J = torch.empty((system.n, system.N, 2, L), dtype=torch.float64, device=dev)
        Ab = torch.empty((system.n + 1, system.N, 2, L), dtype=torch.float64, device=dev)
        R = torch.empty((system.n + 1, system.n + 1, 2, L), dtype=torch.float64, device=dev)
        dx = torch.empty((system.n, 2, L), dtype=torch.float64, device=dev)
        status = torch.zeros((1,), dtype=torch.int32, device=dev)
        ev_ops, _ = algorithmic_fp64(system, L)
        ev = {}
        for arith in ("fp64", "int"):
            S.set_arith(arith)
            t = timed(lambda: S.eval(prec, x, f, J))
            ev[arith] = {"ms": t, "monomials_per_s": system.T / (t / 1e3)}
        S.set_arith("auto")
        g = ev_ops / (ev["fp64"]["ms"] / 1e3) / 1e9
        ev["fp64"]["fp64_ginstr_per_s"] = g
        ev["fp64"]["frac_of_fp64_peak"] = g / peaks["fp64_ginstr"]
        fm = rates.get("fp64_fma", {}).get("rate")
        ev["fp64"]["frac_of_fp64_measured"] = g / fm if fm else None
        ev["int"]["speedup_vs_fp64"] = ev["fp64"]["ms"] / ev["int"]["ms"]
        if L == 1:
            # double: the binding roofline is the larger of the HBM time of the
            # algorithmic bytes and the FP64 time of the algorithmic
            # instructions (L2 flushed before each timed call)
            by = eval_bytes(system, L)
            t = ev["fp64"]["ms"] / 1e3
            t_hbm = by / (peaks["hbm_gbs"] * 1e9)
            t_fp = ev_ops / (peaks["fp64_ginstr"] * 1e9)
            ev["fp64"]["binding_roofline"] = {
                "bound": "hbm" if t_hbm >= t_fp else "fp64", "frac": max(t_hbm, t_fp) / t,
                "algorithmic_bytes": by, "achieved_gbs": by / t / 1e9, "hbm_peak_gbs": peaks["hbm_gbs"],
                "fp64_frac": t_fp / t, "hbm_frac": t_hbm / t}
        out["eval_diff"][prec] = ev
        S.eval(prec, x, f, J)
        Ab0 = torch.cat([J, -f[None]], 0).contiguous()

        def prep_ab():
            Ab.copy_(Ab0)

        out["lstsq_ms"][prec] = timed(lambda: S.lstsq(prec, Ab, R, dx), prep_ab)
        x0 = torch.tensor(system.point("x0", L), device=dev)
        out["newton_step_ms"][prec] = timed(lambda: S.newton(prec, x, 1), lambda: x.copy_(x0))
        if prec == args.prec:
            # the dominant kernel of the step: k_mgs_int, through gn_mgs (its
            # time includes the zeroing of R and the conversion of Q back to
            # cascades, together under 1% of the factorisation)
            t_mgs = timed(lambda: S.mgs(prec, Ab, R, status), prep_ab)
            assert int(status.item()) == 0
            work = algorithmic_imad_mgs(system.N, system.n + 1, L)
            achieved = work / (t_mgs / 1e3) / 1e9
            mi = rates.get("imad", {}).get("rate")
            roof = {"kernel": f"k_mgs_int<{L}> (MGS on [J, -f], {system.N} x {system.n + 1})",
                    "bound": "alu", "achieved": achieved, "peak": peaks["imad_ginstr"],
                    "unit": "G IMAD/s", "frac": achieved / peaks["imad_ginstr"],
                    "peak_source": "derived: " + peaks["derivation"],
                    "frac_of_measured_imad": achieved / mi if mi else None,
                    "traffic": MGS_TRAFFIC.get(L),
                    "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum per launch",
                    "algorithmic_imad": work, "launch_ms": t_mgs,
                    "us_per_column": 1e3 * t_mgs / (system.n + 1),
                    "note": "latency-bound: one dependent pivot step per column"}
    return out, roof


if __name__ == "__main__":
    sys.exit(main())
