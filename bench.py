#!/usr/bin/env python
"""Benchmark of the blocked Cholesky (Algorithm 1, arXiv:1812.02056) on GB300.

One step = one FP64 Cholesky factorization with step s of an n x n SPD matrix
A = G G^T + n I (G iid N(0,1)), through the C ABI (gb_chol_factor), A and L
resident in HBM.  Default n = 8192, s = 256.  The metric is factorization
GFLOP/s counted as n^3/3 flops per step.

Prints ONE JSON line (rank 0).  Besides the contract keys it carries:
  roofline      the dominant kernel (largest device-time phase), from CUDA
                events the library records around each launch on the
                factorization's stream during the timed region;
  cpu_baseline  the CPU oracle timed on a bounded sample on the host cores;
  e2e           the same metric through gb_chol_factor on pinned HOST
                buffers (host<->device copies inside the timed region);
  extra         s sweep (FP64 and FP32), pivot-free LU, accuracy figures.

--impl reference times the CPU oracle (the reference arm of this project)
on a bounded sample of the same workload and prints the same JSON line with
"impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Cholesky GFLOP/s (n^3/3 flops per factorization)"
UNIT = "GFLOP/s"


def dist_max(x: float, dist=None, device="cpu") -> float:
    """Max of x over the ranks of the process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, flops_per_step: float, ms_total: float) -> float:
    """Whole-job GFLOP/s: every rank did `steps` steps; the slowest rank's
    time bounds the job (weak scaling, replicas)."""
    return world * steps * flops_per_step / (ms_total * 1e-3) / 1e9


def chol_flops(n: int) -> float:
    return n ** 3 / 3.0


def lu_flops(n: int) -> float:
    return 2.0 * n ** 3 / 3.0


# DRAM traffic per launch of a kernel, from one ncu capture of the same
# workload (dram__bytes_read.sum + dram__bytes_write.sum); reported only while
# the kernel's source is unchanged since the capture (sha256 prefix).
MEASURED_TRAFFIC = {
    ("update", "f64", 8192, 256): {
        "bytes_per_launch": 32.80e6, "source": "paper_1812_02056_gb300/csrc/update_simt.cu",
        "sha256_16": "35d6ae8f28452258"},
}


def measured_traffic(kernel: str, dtype: str, n: int, s: int):
    import hashlib
    rec = MEASURED_TRAFFIC.get((kernel, dtype, n, s))
    if rec is None:
        return None
    with open(os.path.join(ROOT, rec["source"]), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest()[:16] != rec["sha256_16"]:
            return None
    return rec["bytes_per_launch"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = os.path.join("/tmp", f"gbchol_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.out) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
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
        try:
            os.remove(self.out)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(A, s: int, reps: int = 1):
    import oracle
    n = A.shape[0]
    oracle.chol(A[:64, :64], min(s, 64))  # load / build outside the timing
    t0 = time.perf_counter()
    for _ in range(reps):
        L, info = oracle.chol(A, s)
    dt = (time.perf_counter() - t0) / reps
    return {"value": chol_flops(n) / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"oracle FP64 Cholesky (Algorithm 1) n={n} s={s}, {reps} run(s), "
                      f"{dt:.2f} s each; GFLOP/s = (n^3/3)/time"}


def run_reference(args):
    """Reference arm: the CPU oracle on a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1812_02056_gb300 import inputs
    n = args.ref_n
    s = min(args.s, n)
    A = inputs.spd_gram(n, inputs.seed_for(inputs.W_N8192))
    oracle.chol(A[:64, :64], 8)
    for _ in range(args.warmup):
        oracle.chol(A, s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.chol(A, s)
    el = time.perf_counter() - t0
    ms = el / args.steps * 1e3
    value = chol_flops(n) * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"FP64 Cholesky (Algorithm 1), A = G G^T + n I, n={args.n}, "
                               f"s={args.s}; each reference step factors a bounded sample "
                               f"n={n}, s={s}", "n": args.n, "s": args.s, "sample_n": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle",
                         "cores": oracle.num_threads(),
                         "sample": f"oracle FP64 Cholesky n={n} s={s} per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch

    from paper_1812_02056_gb300 import _build, binding, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        _build.build()
    if dist:
        dist.barrier()
    h = binding.Handle(local)
    n, s = args.n, args.s
    dt = binding.DTYPES[args.dtype]
    A = inputs.spd_gram(n, inputs.seed_for(inputs.W_N8192, rank), device=dev)
    if args.dtype == "f32":
        A = A.float()
    L = torch.empty((n, n), dtype=torch.float64 if dt == binding.GB_F64 else torch.float32,
                    device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        binding.check(h.gb_chol_factor(n, s, dt, A, n, L, n, info, stream), "gb_chol_factor")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert int(info.item()) == 0, f"breakdown at column {int(info.item())}"

    # ---- timed region
    h.set_option(binding.GB_OPT_PROFILE, 1)
    h.profile_read()  # drop anything recorded before
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = binding.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = binding.kernel_launches() - launches0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    prof = h.profile_read().as_dict()
    h.set_option(binding.GB_OPT_PROFILE, 0)
    ms_total = dist_max(e0.elapsed_time(e1), dist, dev)
    ms_step = ms_total / args.steps
    flops = chol_flops(n)
    value = job_value(world, args.steps, flops, ms_total)
    assert int(info.item()) == 0

    peaks, peak_src = load_peaks()
    # FP64 / FP32 pipe peaks from unit counts and clock: SMs x flop/clk/SM x
    # max SM clock, with 4 FP64 flop/clk/SM (2 DFMA, the nominal 1.25 TFLOP/s
    # of GB300 at 152 SMs and 2.07 GHz) and 256 FP32 flop/clk/SM (128 FFMA);
    # the library's FMA loop measures both beside them.
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    derived = {"f64": sms * 4 * sm_mhz * 1e6, "f32": sms * 256 * sm_mhz * 1e6}
    fma64 = h.measure_fma_peak("f64")
    fma32 = h.measure_fma_peak("f32")
    pipe_peaks = {}
    for kind in ("dmma", "tc_bf16", "tc_f16", "tc_tf32"):
        try:
            pipe_peaks[kind] = h.measure_peak(kind) / 1e12
        except binding.GbError as e:
            pipe_peaks[kind] = f"unavailable: {e}"

    # dominant kernel = phase with the largest device time; the inner and the
    # delayed updates are launches of one kernel and count together
    def by_kernel(pr):
        kk = {k: dict(v) for k, v in pr.items() if k not in ("inner", "update")}
        kk["update"] = {f: pr["inner"][f] + pr["update"][f]
                        for f in ("launches", "ms", "flops", "bytes")}
        return kk

    kern = by_kernel(prof)
    dom = max(kern, key=lambda p: kern[p]["ms"])
    d = kern[dom]
    if args.dtype in ("f64", "f32") and dom in ("update", "inner", "panel", "diag"):
        # Under look-ahead the update launches share the SMs with the column
        # steps, so their event intervals overlap other work and their sum can
        # exceed the step.  The kernel's rate is therefore taken from one
        # serialised factorization after the timed region (look-ahead off:
        # nothing runs beside a launch), and bounded from below by the timed
        # steps themselves (all of the kernel's flops within ms_per_step).
        la = h.get_option(binding.GB_OPT_LOOKAHEAD)
        ila = h.get_option(binding.GB_OPT_INNER_LOOKAHEAD)
        h.set_option(binding.GB_OPT_LOOKAHEAD, 0)
        h.set_option(binding.GB_OPT_INNER_LOOKAHEAD, 0)  # the same sums, one stream
        h.set_option(binding.GB_OPT_PROFILE, 1)
        step()
        torch.cuda.synchronize()
        h.profile_read()
        step()
        torch.cuda.synchronize()
        ser = by_kernel(h.profile_read().as_dict())[dom]
        h.set_option(binding.GB_OPT_PROFILE, 0)
        h.set_option(binding.GB_OPT_LOOKAHEAD, la)
        h.set_option(binding.GB_OPT_INNER_LOOKAHEAD, ila)
        ach = ser["flops"] / (ser["ms"] * 1e-3) / 1e12
        flops_per_step = d["flops"] / args.steps
        ach_lo = flops_per_step / (ms_step * 1e-3) / 1e12
        peak = derived[args.dtype] / 1e12
        tr = measured_traffic(dom, args.dtype, n, s)
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": tr, "kernel": dom,
                "achieved_source": "serialised factorization (both look-aheads off: the same "
                                   "sums on one stream), CUDA events around each launch",
                "serialised_launches": ser["launches"], "serialised_ms": ser["ms"],
                "serialised_flops": ser["flops"],
                "ms_per_launch": ser["ms"] / max(ser["launches"], 1),
                "algorithmic_flops_per_launch": ser["flops"] / max(ser["launches"], 1),
                "algorithmic_bytes_per_launch": ser["bytes"] / max(ser["launches"], 1),
                "timed_flops_per_step": flops_per_step,
                "achieved_lower_bound_in_step": ach_lo, "frac_lower_bound": ach_lo / peak,
                "whole_job_frac": value / (derived[args.dtype] / 1e9),
                "peak_source": f"{args.dtype} FMA pipe: {sms} SMs x "
                               f"{4 if args.dtype == 'f64' else 256} flop/clk x {sm_mhz:.0f} MHz "
                               f"(measured FMA loop: {(fma64 if args.dtype == 'f64' else fma32) / 1e12:.3f})"}
    else:
        ach = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "kernel": dom,
                "peak_source": f"hbm_gbs ({peak_src})", "launches": d["launches"]}

    # ---- accuracy of the timed factor (FP64 backward error on the device)
    extra = {"phases": prof, "fma_peak_tflops": {"f64": fma64 / 1e12, "f32": fma32 / 1e12},
             "pipe_peak_tflops": pipe_peaks,
             "derived_peak_tflops": {k: v / 1e12 for k, v in derived.items()}}
    if not args.quick:
        A64 = A.double() if A.dtype != torch.float64 else A
        extra["backward_error"] = h.backward_error(A64, L, args.dtype)

    # ---- end to end through host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        Ah = torch.empty((n, n), dtype=A.dtype, pin_memory=True)
        Ah.copy_(A)
        Lh = torch.empty((n, n), dtype=L.dtype, pin_memory=True)
        infoh = torch.zeros(1, dtype=torch.int32, pin_memory=True)
        esteps = max(1, min(args.steps, args.e2e_steps))
        binding.check(h.gb_chol_factor(n, s, dt, Ah, n, Lh, n, infoh, stream), "e2e warmup")
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(esteps):
            binding.check(h.gb_chol_factor(n, s, dt, Ah, n, Lh, n, infoh, stream), "e2e")
        torch.cuda.synchronize()
        el = dist_max(time.perf_counter() - t0, dist, dev)
        assert int(infoh[0]) == 0
        esz = A.element_size()
        # the CPU-GPU link on this machine: whole-matrix pinned copies each way
        link = {}
        for name, dst, src in (("h2d_ms", A, Ah), ("d2h_ms", Lh, L)):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            c0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            link[name] = (time.perf_counter() - c0) * 1e3
        # the library moves the lower triangle only, in column slabs of s
        # columns (rows from the slab's first column down), both ways; the
        # zeros above are written on the host
        tri = sum((n - q) * min(s, n - q) for q in range(0, n, s))
        e2e = {"value": world * esteps * flops / el / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": tri * esz,
               "d2h_bytes_per_step": tri * L.element_size() + 4,
               "steps": esteps, "ms_per_step": el / esteps * 1e3,
               "link_full_matrix_copy_ms": link}
        del Ah, Lh

    # ---- sweeps (not part of the timed value)
    if not args.quick:
        sweep = {}
        for sdt in ("f64", "f32"):
            Asw = A if sdt == args.dtype else (A.float() if sdt == "f32" else A.double())
            Lsw = torch.empty((n, n), dtype=Asw.dtype, device=dev)
            for ss in (64, 117, 256, 512):
                reps = 1 if sdt == "f64" else 3
                binding.check(h.gb_chol_factor(n, ss, binding.DTYPES[sdt], Asw, n, Lsw, n, info,
                                               stream), "sweep")
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                for _ in range(reps):
                    h.gb_chol_factor(n, ss, binding.DTYPES[sdt], Asw, n, Lsw, n, info, stream)
                a1.record(stream)
                torch.cuda.synchronize()
                sweep[f"chol_{sdt}_s{ss}"] = flops / (a0.elapsed_time(a1) / reps * 1e-3) / 1e9
            del Lsw
        Alu = torch.from_numpy(inputs.lu_diag_dominant(n, inputs.seed_for(inputs.W_N8192, 50))).to(dev)
        LU = torch.empty_like(Alu)
        for ss in (256,):
            h.gb_lu_factor(n, ss, binding.GB_F64, Alu, n, LU, n, info, stream)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            h.gb_lu_factor(n, ss, binding.GB_F64, Alu, n, LU, n, info, stream)
            a1.record(stream)
            torch.cuda.synchronize()
            sweep[f"lu_f64_s{ss}"] = lu_flops(n) / (a0.elapsed_time(a1) * 1e-3) / 1e9
        extra["sweep_gflops"] = sweep
        del Alu, LU
        # FP64 accuracy with the delayed and inner updates from exact digit
        # products on the tensor cores (GB_OPT_F64_UPDATE = 1), same input
        if args.dtype == "f64":
            Ld = torch.empty_like(A)
            dig = {}
            h.set_option(binding.GB_OPT_F64_UPDATE, 1)
            try:
                for ss in (256, 512):
                    h.gb_chol_factor(n, ss, binding.GB_F64, A, n, Ld, n, info, stream)
                    a0 = torch.cuda.Event(enable_timing=True)
                    a1 = torch.cuda.Event(enable_timing=True)
                    a0.record(stream)
                    for _ in range(3):
                        h.gb_chol_factor(n, ss, binding.GB_F64, A, n, Ld, n, info, stream)
                    a1.record(stream)
                    torch.cuda.synchronize()
                    ms = a0.elapsed_time(a1) / 3
                    dig[f"s{ss}"] = {"ms": ms, "gflops": flops / (ms * 1e-3) / 1e9,
                                     "backward_error": h.backward_error(A, Ld, "f64"),
                                     "info": int(info.item())}
            finally:
                h.set_option(binding.GB_OPT_F64_UPDATE, 0)
            # Algorithm 2 (pivot-free LU) likewise
            Alu = torch.from_numpy(inputs.lu_diag_dominant(n, inputs.seed_for(inputs.W_N8192, 50))).to(dev)
            LUd = torch.empty_like(Alu)
            h.set_option(binding.GB_OPT_F64_UPDATE, 1)
            try:
                h.gb_lu_factor(n, 256, binding.GB_F64, Alu, n, LUd, n, info, stream)
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                for _ in range(3):
                    h.gb_lu_factor(n, 256, binding.GB_F64, Alu, n, LUd, n, info, stream)
                a1.record(stream)
                torch.cuda.synchronize()
                ms = a0.elapsed_time(a1) / 3
                dig["lu_s256"] = {"ms": ms, "gflops": lu_flops(n) / (ms * 1e-3) / 1e9,
                                  "backward_error": h.backward_error(Alu, LUd, "f64", lu=True),
                                  "info": int(info.item())}
            finally:
                h.set_option(binding.GB_OPT_F64_UPDATE, 0)
            extra["f64_digit_update"] = dig
            del Ld, Alu, LUd

    if rank == 0 and world == 1 and not args.quick and not args.no_extras:
        extra["workloads"] = other_workloads(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cn = min(args.cpu_n, n)
        Ah = A[:cn, :cn].double().cpu().numpy()  # leading block of the timed input
        cpu = cpu_oracle_sample(Ah, min(s, cn))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": f"{args.dtype.upper()} Cholesky (Algorithm 1), "
                                   f"A = G G^T + n I, n={n}, s={s}",
                       "n": n, "s": s, "inner_step": h.get_option(binding.GB_OPT_INNER_STEP),
                       "l2": f"inputs larger than L2 (A and L {n * n * A.element_size() >> 20} MiB each)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "gpu_launches": launches, "clocks": clk, "roofline": roof, "e2e": e2e,
            "cpu_baseline": cpu, "extra": extra,
        }
        print(json.dumps(line))
    h.close()
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------- the other workloads
def other_workloads(args):
    """The other workloads the benchmark is quoted on, each with its own clock
    record, run after the headline's timed region in the same process:
    mixed precision + FP64 refinement at n = 16384 against the plain FP64
    form, the tensor-core update at n = 16384, K = 2048, the batched 10,000
    matrices (FP32 and FP64) and a short served run at 25% and 80% load."""
    import copy

    import torch

    runs = {
        "mixed_n16384": (run_mixed, {"n": 16384, "mixed_dtypes": "f64,mix_f16,mix_bf16x3",
                                     "reps": 1, "tune": True}),
        "update_tc_n16384_k2048": (run_update, {"n": 16384, "ks": "2048", "tc_modes": "2",
                                                "reps": 10, "warmup": 3,
                                                "update_dtype": "mix_bf16"}),
        "batched_10000": (run_batched, {"batch_count": 10000, "steps": 5, "warmup": 3,
                                        "batch_cpu_sample": 0}),
        "served_200": (run_served, {"served_count": 200, "served_rates": "0.25,0.8",
                                    "served_isolated": True}),
    }
    out = {}
    for name, (fn, over) in runs.items():
        a = copy.copy(args)
        for k, v in over.items():
            setattr(a, k, v)
        clocks = ClockSampler(0)
        clocks.start()
        t0 = time.perf_counter()
        try:
            res = fn(a)
        except Exception as e:  # reported, never hidden
            res = {"error": f"{type(e).__name__}: {e}"}
        res["wall_s"] = time.perf_counter() - t0
        res["clocks"] = clocks.stop()
        out[name] = res
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------ rank-s update only
def run_update(args):
    """Time gb_rank_update (C -= R R^T, lower, R = m x K) on the tensor cores:
    the delayed update of an n x n factorization's first block, m = n - K."""
    import torch

    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    h = binding.Handle(0)
    peaks, src = load_peaks()
    out = {"mode": "update", "n": args.n, "dtype": args.update_dtype, "results": []}
    dt = binding.DTYPES[args.update_dtype]
    g = torch.Generator(device=dev).manual_seed(5)
    for K in [int(k) for k in args.ks.split(",")]:
        m = args.n - K
        C = torch.randn((m, m), device=dev, generator=g)
        R = torch.randn((m, K), device=dev, generator=g)
        stream = torch.cuda.current_stream()

        def call():
            binding.check(h.gb_rank_update(dt, 1, 0, m, m, K, C, m, R, K, R, K, stream),
                          "gb_rank_update")

        default_mode = h.get_option(binding.GB_OPT_TC_UPDATE)
        for mode in [int(v) for v in args.tc_modes.split(",")]:
            h.set_option(binding.GB_OPT_TC_UPDATE, mode)
            for _ in range(args.warmup):
                call()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = binding.kernel_launches()
            e0.record(stream)
            for _ in range(args.reps):
                call()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.reps
            launches = (binding.kernel_launches() - l0) / args.reps
            # the same calls with the profile option: event pairs split each
            # call into its packing launches and the tensor-core kernel
            h.set_option(binding.GB_OPT_PROFILE, 1)
            h.profile_read()
            for _ in range(args.reps):
                call()
            torch.cuda.synchronize()
            prof = h.profile_read().as_dict()
            h.set_option(binding.GB_OPT_PROFILE, 0)
            flops = 2.0 * K * m * (m + 1) / 2.0
            cbytes = 8.0 * m * (m + 1) / 2.0  # FP32 lower triangle read + written
            tflops = flops / (ms * 1e-3) / 1e12
            kern_ms = prof["update"]["ms"] / max(1, prof["update"]["launches"])
            pack_ms = prof["copy"]["ms"] / max(1, prof["copy"]["launches"])
            kern_tflops = flops / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else None
            out["results"].append({
                "K": K, "m": m, "tc_mode": mode, "ms": ms, "tflops": tflops,
                "frac_of_bf16_peak": tflops / peaks["bf16_tflops"],
                "kernel_ms": kern_ms, "pack_ms": pack_ms, "kernel_tflops": kern_tflops,
                "kernel_frac_of_bf16_peak": (kern_tflops / peaks["bf16_tflops"]
                                             if kern_tflops else None),
                "hbm_bound_tflops": peaks["hbm_gbs"] * 1e9 * flops / cbytes / 1e12,
                "launches_per_call": launches})
        h.set_option(binding.GB_OPT_TC_UPDATE, default_mode)
        del C, R
        torch.cuda.empty_cache()
    out["peaks"] = {"bf16_tflops": peaks["bf16_tflops"], "hbm_gbs": peaks["hbm_gbs"], "source": src}
    h.close()
    return out


# ------------------------------------------------- mixed precision + IR
def run_mixed(args):
    """Time to an FP64-accurate solution (16 RHS) at n with cond(A) = 1e4:
    plain FP64 factor + solve against mixed factors + FP64 refinement."""
    import numpy as np
    import torch

    from paper_1812_02056_gb300 import _build, binding, inputs
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    h = binding.Handle(0)
    n, nrhs = args.n, 16
    t0 = time.perf_counter()
    if args.host_inputs:  # numpy QR on the host (no device QR library in the process)
        A = torch.from_numpy(inputs.spd_logspaced(n, inputs.seed_for(inputs.W_MIXED),
                                                  cond=1e4)).to(dev)
    else:
        A = inputs.spd_logspaced(n, inputs.seed_for(inputs.W_MIXED), cond=1e4, device=dev)
    B = torch.from_numpy(inputs.rhs(n, nrhs, inputs.seed_for(inputs.W_MIXED, 1))).to(dev)
    gen_s = time.perf_counter() - t0
    out = {"mode": "mixed", "n": n, "nrhs": nrhs, "cond": 1e4, "input_generation_s": gen_s,
           "results": {}}
    stream = torch.cuda.current_stream()
    xref = None
    wanted = args.mixed_dtypes.split(",")
    for name, s in [("f64", args.s_f64), ("f32", args.s_mixed), ("mix_f16", args.s_mixed),
                    ("mix_bf16", args.s_mixed), ("mix_bf16x3", args.s_mixed)]:
        if name not in wanted:
            continue
        dt = binding.DTYPES[name]
        tuned = None
        if args.tune and name != "f64":  # FP64 keeps its fixed step (tuning it takes ~20 s)
            tuned = h.tune_step("chol", name, n)  # later s = 0 calls use the tuned pair
            s = 0
        Ain = A.float() if name == "f32" else A
        L = torch.empty((n, n), dtype=torch.float64 if name == "f64" else torch.float32, device=dev)
        info = torch.zeros(1, dtype=torch.int32, device=dev)
        X = torch.empty_like(B)
        runs = []
        h.set_option(binding.GB_OPT_PROFILE, 1)
        for rep in range(1 + args.reps):
            h.profile_read()  # keep only the last repetition's phases
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            binding.check(h.gb_chol_factor(n, s, dt, Ain, n, L, n, info, stream), "factor")
            e1.record(stream)
            st, stats = h.gb_chol_solve(n, nrhs, dt, L, n, None if name == "f64" else A, n, B,
                                        nrhs, X, nrhs, 1e-14, 50, stream)
            e2.record(stream)
            torch.cuda.synchronize()
            runs.append((e0.elapsed_time(e1), e1.elapsed_time(e2), st, stats.iterations,
                         stats.eta, int(info.item())))
        prof = h.profile_read().as_dict()
        h.set_option(binding.GB_OPT_PROFILE, 0)
        fm, sm, st, it, eta, inf = runs[-1]
        if name == "f64":
            xref = X.clone()
        res = {"s": s if tuned is None else {"tuned_s": tuned[0], "tuned_inner": tuned[1]},
               "factor_ms": fm, "solve_ms": sm, "time_to_solution_ms": fm + sm,
               "status": st, "info": inf, "ir_iterations": it, "eta": eta,
               "factor_gflops": n ** 3 / 3 / (fm * 1e-3) / 1e9,
               "factor_phase_ms": {k: round(v["ms"], 3) for k, v in prof.items()},
               "factor_phase_launches": {k: v["launches"] for k, v in prof.items()}}
        if name != "f64":
            # the residual's method (GB_OPT_RESIDUAL), and the same solve with
            # the FP64 residual on the CUDA cores for comparison
            mode = h.get_option(binding.GB_OPT_RESIDUAL)
            digits = mode == 1 or (mode == 2 and n >= 2048)
            res["residual"] = "tensor-core digit products" if digits else "fp64 cuda cores"
            h.set_option(binding.GB_OPT_RESIDUAL, 0)
            X0 = torch.empty_like(B)
            torch.cuda.synchronize()
            e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
            e1.record(stream)
            st0, stats0 = h.gb_chol_solve(n, nrhs, dt, L, n, A, n, B, nrhs, X0, nrhs, 1e-14, 50,
                                          stream)
            e2.record(stream)
            torch.cuda.synchronize()
            h.set_option(binding.GB_OPT_RESIDUAL, mode)
            res["with_fp64_residual"] = {"solve_ms": e1.elapsed_time(e2),
                                         "time_to_solution_ms": fm + e1.elapsed_time(e2),
                                         "status": st0, "ir_iterations": stats0.iterations,
                                         "eta": stats0.eta}
            del X0
        Xh = X.double()
        R = B - A @ Xh
        den = A.abs().sum(1).max() * Xh.abs().max(0).values + B.abs().max(0).values
        res["eta_host"] = float((R.abs().max(0).values / den).max())
        if xref is not None:
            res["max_rel_diff_vs_fp64_solve"] = float((Xh - xref).abs().max() / xref.abs().max())
        out["results"][name] = res
        del L
        torch.cuda.empty_cache()
    h.close()
    return out


# ------------------------------------------------------------ batched
def run_batched(args):
    """10,000 SPD matrices, n uniform on [16, 512], FP32 and FP64, factored by
    one persistent launch (steps from the autotuner), captured in a CUDA graph
    and replayed; GFLOP/s = sum n^3/3 / time."""
    import numpy as np
    import torch

    import oracle
    from paper_1812_02056_gb300 import _build, binding, inputs
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    h = binding.Handle(0)
    sizes = inputs.batch_sizes(args.batch_count, 16, 512, inputs.seed_for(inputs.W_BATCHED))
    flops = float((sizes.astype(np.float64) ** 3).sum() / 3.0)
    out = {"mode": "batched", "count": int(len(sizes)), "n_range": [16, 512],
           "sum_n3_over_3": flops, "results": {}}
    peaks, _ = load_peaks()
    for dtype in ("f32", "f64"):
        tt = torch.float32 if dtype == "f32" else torch.float64
        buf, offs = inputs.batch_spd_device(sizes, inputs.seed_for(inputs.W_BATCHED, 1), dev, tt)
        outb = torch.empty_like(buf)
        esz = buf.element_size()
        dt = binding.DTYPES[dtype]
        steps = np.zeros(16, dtype=np.int32)
        t0 = time.perf_counter()
        if not args.no_tune:
            binding.check(h.gb_batched_tune(dt, 512, steps), "tune")
        tune_s = time.perf_counter() - t0
        a_arr = (buf.data_ptr() + offs * esz).astype(np.uint64)
        l_arr = (outb.data_ptr() + offs * esz).astype(np.uint64)
        n_arr = sizes.astype(np.int64)
        binding.check(h.gb_batched_plan(len(sizes), n_arr, a_arr, n_arr, l_arr, n_arr, dt, 0),
                      "plan")
        info = torch.zeros(len(sizes), dtype=torch.int32, device=dev)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            binding.check(h.gb_batched_run(info, st), "warm")
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            binding.check(h.gb_batched_run(info, st), "capture")
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        bad = int((info != 0).sum().item())
        rng = np.random.default_rng(1)
        errs = []
        for i in rng.choice(len(sizes), 4, replace=False):
            n = int(sizes[i])
            A = buf[offs[i]:offs[i] + n * n].view(n, n).double().cpu().numpy()
            L = outb[offs[i]:offs[i] + n * n].view(n, n).double().cpu().numpy()
            errs.append(oracle.chol_backward_error(A, L))
        gf = flops / (ms * 1e-3) / 1e9
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        alu = sms * (4 if dtype == "f64" else 256) * sm_mhz * 1e6 / 1e9
        out["results"][dtype] = {
            "ms_per_batch": ms, "gflops": gf, "alu_peak_gflops": alu, "frac_of_alu_peak": gf / alu,
            "breakdowns": bad, "tuned_steps_by_32": steps[:16].tolist(), "tune_s": tune_s,
            "sample_backward_error_max": max(errs), "graph_replays": args.steps,
            "bytes_in_out": 2 * int((sizes ** 2).sum()) * esz}
        # Algorithm 2 on the same matrices (SPD: every leading minor is positive)
        binding.check(h.gb_lu_batched_plan(len(sizes), n_arr, a_arr, n_arr, l_arr, n_arr, dt, 0),
                      "lu plan")
        with torch.cuda.stream(st):
            binding.check(h.gb_batched_run(info, st), "lu warm")
        torch.cuda.synchronize()
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g2, stream=st):
            binding.check(h.gb_batched_run(info, st), "lu capture")
        for _ in range(args.warmup):
            g2.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            g2.replay()
        e1.record()
        torch.cuda.synchronize()
        ms_lu = e0.elapsed_time(e1) / args.steps
        lu_errs = []
        for i in rng.choice(len(sizes), 4, replace=False):
            n = int(sizes[i])
            A = buf[offs[i]:offs[i] + n * n].view(n, n).double().cpu().numpy()
            F = outb[offs[i]:offs[i] + n * n].view(n, n).double().cpu().numpy()
            Lf = np.tril(F)
            Uf = np.triu(F, 1) + np.eye(n)
            lu_errs.append(oracle.lu_backward_error(A, Lf, Uf))
        gf_lu = 2.0 * flops / (ms_lu * 1e-3) / 1e9
        out["results"][dtype + "_lu"] = {
            "ms_per_batch": ms_lu, "gflops": gf_lu, "frac_of_alu_peak": gf_lu / alu,
            "breakdowns": int((info != 0).sum().item()), "step": "min(n, 32)",
            "sample_backward_error_max": max(lu_errs), "graph_replays": args.steps}
        del buf, outb, g, g2
        torch.cuda.empty_cache()
    # CPU oracle on a bounded sample of the same workload
    if args.batch_cpu_sample > 0:
        idx = np.random.default_rng(2).choice(len(sizes), args.batch_cpu_sample, replace=False)
        mats = [inputs.spd_gram(int(sizes[i]), inputs.seed_for(inputs.W_BATCHED, 2) + int(i))
                for i in idx]
        t0 = time.perf_counter()
        for A in mats:
            oracle.chol(A, 32)
        el = time.perf_counter() - t0
        fs = float(sum(int(sizes[i]) ** 3 for i in idx) / 3.0)
        out["cpu_baseline"] = {"value": fs / el / 1e9, "unit": "GFLOP/s", "kind": "oracle",
                               "cores": oracle.num_threads(),
                               "sample": f"{len(idx)} matrices of the workload, FP64, s=32"}
    h.close()
    return out


# ------------------------------------------------------------- served
def run_served(args):
    """Poisson stream of factor-and-solve jobs, n log-uniform on [32, 8192],
    1..64 right-hand sides, A = G G^T + n I, mixed-precision factor with FP64
    refinement, through the continuous-batching server with an HBM budget of
    80% of free memory.  Saturated throughput first (all jobs at once), then
    arrival rates at fractions of it; p50/p99 latency and solves/s."""
    import threading

    import numpy as np
    import torch

    from paper_1812_02056_gb300 import _build, binding, inputs
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    count = args.served_count
    _, n_all, k_all = inputs.served_requests(count, inputs.seed_for(inputs.W_SERVED),
                                              n_lo=32, n_hi=args.served_nmax)
    t0 = time.perf_counter()
    jobs = []
    for i in range(count):
        n, k = int(n_all[i]), int(k_all[i])
        A = inputs.spd_gram(n, inputs.seed_for(inputs.W_SERVED, 10 + i), device=dev)
        B = torch.from_numpy(inputs.rhs(n, k, inputs.seed_for(inputs.W_SERVED, 5000 + i))).to(dev)
        jobs.append((A, B, torch.empty_like(B)))
    torch.cuda.synchronize()
    out = {"mode": "served", "count": count, "dtype": args.served_dtype, "slots": args.slots,
           "n_range": [32, args.served_nmax], "input_generation_s": time.perf_counter() - t0,
           "runs": {}}
    srv = binding.Server(0, 0, args.slots)
    per_job = []

    def run(arrivals):
        srv.reset_stats()
        tickets = [None] * count
        start = time.perf_counter()

        def producer():
            for i in range(count):
                if arrivals is not None:
                    d = arrivals[i] - (time.perf_counter() - start)
                    if d > 0:
                        time.sleep(d)
                A, B, X = jobs[i]
                tickets[i] = srv.submit(A, B, X, dtype=args.served_dtype)

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        res = [srv.wait(t) for t in tickets]
        st = srv.stats()
        el = time.perf_counter() - start
        its = [r.iterations for r in res]
        per_job.clear()
        per_job.extend((int(n_all[i]), int(k_all[i]), res[i].queue_ms, res[i].compute_ms,
                        res[i].iterations) for i in range(count))
        return {"p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "max_ms": st.max_ms,
                "solves_per_s": count / el, "server_solves_per_s": st.solves_per_s,
                "max_running": st.max_running, "failed": sum(1 for r in res if r.status != 0),
                "mean_queue_ms": float(np.mean([r.queue_ms for r in res])),
                "mean_ir_iterations": float(np.mean(its)), "max_eta": max(r.eta for r in res)}

    run(None)  # warm-up: builds, autotunes nothing, fills the allocator pools
    sat = run(None)
    out["runs"]["saturated"] = sat
    rate_sat = sat["solves_per_s"]
    at25 = None
    for frac in [float(x) for x in args.served_rates.split(",")]:
        rate = frac * rate_sat
        arr = np.cumsum(inputs.rng(inputs.seed_for(inputs.W_SERVED, 77)).exponential(1.0 / rate,
                                                                                   size=count))
        r = run(arr)
        r["offered_rate"] = rate
        out["runs"][f"rate_{int(frac * 100)}pct"] = r
        if at25 is None:
            at25 = list(per_job)
    # The same jobs one at a time on a one-slot server: each job's isolated
    # compute time, their sum (the isolated-request bound on the saturated
    # makespan) and the slowest jobs of the 25% run against their isolated time.
    if args.served_isolated and at25 is not None:
        srv1 = binding.Server(0, 0, 1)
        iso = []
        for i in range(count):
            A, B, X = jobs[i]
            iso.append(srv1.wait(srv1.submit(A, B, X, dtype=args.served_dtype)).compute_ms)
        srv1.close()
        iso_sum_s = sum(iso) / 1e3
        out["isolated"] = {"sum_s": iso_sum_s, "solves_per_s": count / iso_sum_s,
                           "saturated_over_isolated": sat["solves_per_s"] / (count / iso_sum_s),
                           "max_ms": max(iso), "p99_ms": float(np.percentile(iso, 99))}
        slow = sorted(range(count), key=lambda i: -(at25[i][2] + at25[i][3]))[:12]
        out["slowest_at_first_rate"] = [
            {"n": at25[i][0], "nrhs": at25[i][1], "queue_ms": at25[i][2],
             "compute_ms": at25[i][3], "iterations": at25[i][4], "isolated_ms": iso[i]}
            for i in slow]
    # host check of a sample of the last run's results
    worst = 0.0
    for i in range(0, count, max(1, count // 8)):
        A, B, X = jobs[i]
        R = B - A @ X
        den = A.abs().sum(1).max() * X.abs().max(0).values + B.abs().max(0).values
        worst = max(worst, float((R.abs().max(0).values / den).max()))
    out["sample_eta_host_max"] = worst
    srv.close()
    return out


# ------------------------------------------------------------- Strassen
def run_strassen(args):
    """One Strassen level in the delayed update against the classical update:
    FP64 and FP32 pivot-free LU and Cholesky at n, s (time, GFLOP/s counted
    with the classical n^3/3 and 2n^3/3, backward error)."""
    import torch

    from paper_1812_02056_gb300 import _build, binding, inputs
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    h = binding.Handle(0)
    n, s = args.n, args.s
    out = {"mode": "strassen", "n": n, "s": s, "results": {}}
    Ac = inputs.spd_gram(n, inputs.seed_for(inputs.W_N8192, 0), device=dev)
    Al = torch.from_numpy(inputs.lu_diag_dominant(n, inputs.seed_for(inputs.W_N8192, 50))).to(dev)
    for kind, A64 in (("lu", Al), ("chol", Ac)):
        for dtype in ("f64", "f32"):
            A = A64 if dtype == "f64" else A64.float()
            F = torch.empty_like(A)
            info = torch.zeros(1, dtype=torch.int32, device=dev)
            dt = binding.DTYPES[dtype]
            fn = h.gb_lu_factor if kind == "lu" else h.gb_chol_factor
            for st_on in (0, 1):
                h.set_option(binding.GB_OPT_STRASSEN, st_on)
                fn(n, s, dt, A, n, F, n, info)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(args.reps):
                    fn(n, s, dt, A, n, F, n, info)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.reps
                fl = (2.0 if kind == "lu" else 1.0) * n ** 3 / 3.0
                be = h.backward_error(A64, F, dtype, lu=(kind == "lu"))
                out["results"][f"{kind}_{dtype}_{'strassen' if st_on else 'classical'}"] = {
                    "ms": ms, "gflops": fl / (ms * 1e-3) / 1e9, "backward_error": be,
                    "info": int(info.item())}
            h.set_option(binding.GB_OPT_STRASSEN, 0)
    h.close()
    return out


def run_qr(args):
    """Algorithm 3 (fast QR): FP64 and FP32 at n for each step s; GFLOP/s
    counted as 3 n^3 (Gram-Schmidt Q: 2 n^3, R = Q^T A upper triangle: n^3),
    per-phase device time, orthogonality ||Q^T Q - I||_F and backward error
    ||A - Q R||_F / ||A||_F (checked with torch matmuls outside the timing),
    and the oracle on a bounded sample."""
    import time

    import numpy as np
    import torch

    from paper_1812_02056_gb300 import _build, binding, inputs
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    h = binding.Handle(0)
    n = args.n
    G = torch.from_numpy(inputs.gaussian(n, n, inputs.seed_for(inputs.W_N8192, 70))).to(dev)
    A64 = G + 2.0 * np.sqrt(n) * torch.eye(n, dtype=torch.float64, device=dev)
    out = {"mode": "qr", "n": n, "flop_count": "3 n^3", "results": {}}
    for dtype in ("f64", "f32"):
        A = A64 if dtype == "f64" else A64.float()
        Q = torch.empty_like(A)
        R = torch.empty_like(A)
        info = torch.zeros(1, dtype=torch.int32, device=dev)
        dt = binding.DTYPES[dtype]
        for s, b in [(int(v), int(w)) for v in args.qr_steps.split(",")
                     for w in args.qr_inner.split(",")]:
            if b > s:
                continue
            h.set_option(binding.GB_OPT_QR_INNER_STEP, b)
            binding.check(h.gb_qr_factor(n, s, dt, A, n, Q, n, R, n, info), "qr warm-up")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.reps):
                h.gb_qr_factor(n, s, dt, A, n, Q, n, R, n, info)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.reps
            h.set_option(binding.GB_OPT_PROFILE, 1)
            h.profile_read()
            h.gb_qr_factor(n, s, dt, A, n, Q, n, R, n, info)
            prof = h.profile_read()
            h.set_option(binding.GB_OPT_PROFILE, 0)
            Qd, Rd, Ad = Q.double(), R.double(), A.double()
            orth = torch.linalg.norm(Qd.T @ Qd - torch.eye(n, dtype=torch.float64, device=dev)).item()
            berr = (torch.linalg.norm(Ad - Qd @ Rd) / torch.linalg.norm(Ad)).item()
            out["results"][f"{dtype}_s{s}_b{b}"] = {
                "ms": ms, "gflops": 3.0 * n ** 3 / (ms * 1e-3) / 1e9, "info": int(info.item()),
                "orthogonality": orth, "backward_error": berr,
                "phase_ms": {"panel": prof.ms[2], "inner": prof.ms[3], "update_and_r": prof.ms[4]}}
        h.set_option(binding.GB_OPT_QR_INNER_STEP, 16)
    if not args.no_cpu:
        import oracle
        cn = min(2048, n)  # a bounded sample of the same input (seconds of CPU work)
        Ah = A64[:cn, :cn].cpu().numpy()
        t0 = time.perf_counter()
        oracle.qr(Ah, min(64, cn))
        dt_s = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": 3.0 * cn ** 3 / dt_s / 1e9, "unit": "GFLOP/s",
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": f"FP64 QR n={cn}, s=64, leading block of the input"}
    h.close()
    return out


def run_left(args):
    """Left-looking tile accumulation against the right-looking delayed
    update, tensor-core Cholesky (mix_bf16, mix_f16) at n for several s:
    factor time, TFLOP/s (n^3/3), per-phase device time, backward error."""
    import torch

    from paper_1812_02056_gb300 import _build, binding, inputs
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    h = binding.Handle(0)
    n = args.n
    A = inputs.spd_gram(n, inputs.seed_for(inputs.W_MIXED, 5), device=dev)
    out = {"mode": "left", "n": n, "results": {}}
    L = torch.empty((n, n), dtype=torch.float32, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    for dtype in ("mix_bf16", "mix_f16"):
        dt = binding.DTYPES[dtype]
        for s in [int(v) for v in args.left_steps.split(",")]:
            for left in (0, 1):
                h.set_option(binding.GB_OPT_LEFT_LOOKING, left)
                binding.check(h.gb_chol_factor(n, s, dt, A, n, L, n, info), "warm-up")
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(args.reps):
                    h.gb_chol_factor(n, s, dt, A, n, L, n, info)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.reps
                h.set_option(binding.GB_OPT_PROFILE, 1)
                h.profile_read()
                h.gb_chol_factor(n, s, dt, A, n, L, n, info)
                prof = h.profile_read().as_dict()
                h.set_option(binding.GB_OPT_PROFILE, 0)
                out["results"][f"{dtype}_s{s}_{'left' if left else 'right'}"] = {
                    "ms": ms, "tflops": n ** 3 / 3 / (ms * 1e-3) / 1e12, "info": int(info.item()),
                    "backward_error": h.backward_error(A, L, dtype),
                    "phase_ms": {k: round(v["ms"], 3) for k, v in prof.items()}}
        h.set_option(binding.GB_OPT_LEFT_LOOKING, 0)
    h.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--s", type=int, default=256)
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--cpu-n", type=int, default=8192)
    ap.add_argument("--ref-n", type=int, default=8192)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--quick", action="store_true", help="skip sweeps and accuracy figures")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--mode", choices=["chol", "update", "mixed", "batched", "served", "strassen",
                                       "qr", "left"],
                    default="chol",
                    help="chol: the benchmark line; update: the tensor-core rank-s update "
                         "alone; mixed: FP64 vs mixed-precision time to solution")
    ap.add_argument("--ks", default="256,512,1024,2048")
    ap.add_argument("--qr-steps", default="32,64,128,256")
    ap.add_argument("--left-steps", default="256,512,1024")
    ap.add_argument("--qr-inner", default="8,16,32")
    ap.add_argument("--update-dtype", default="mix_bf16")
    ap.add_argument("--tc-modes", default="1,2",
                    help="update mode: tensor-core kernel variants to time (1 one CTA per tile, "
                         "2 CTA pairs with pair MMAs)")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--s-f64", type=int, default=256)
    ap.add_argument("--s-mixed", type=int, default=1024)
    ap.add_argument("--mixed-dtypes", default="f64,f32,mix_f16,mix_bf16,mix_bf16x3")
    ap.add_argument("--tune", action="store_true",
                    help="mixed mode: pick (s, inner step) with gb_tune_step, then factor with s = 0")
    ap.add_argument("--batch-count", type=int, default=10000)
    ap.add_argument("--host-inputs", action="store_true",
                    help="mixed: build A with numpy on the host instead of on the device")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched: keep the library's default step rule (no autotuner launches)")
    ap.add_argument("--batch-cpu-sample", type=int, default=200)
    ap.add_argument("--served-count", type=int, default=400)
    ap.add_argument("--served-nmax", type=int, default=8192)
    ap.add_argument("--served-dtype", default="mix_bf16")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--served-rates", default="0.25,0.5,0.8,0.95",
                    help="served: offered rates as fractions of the saturated rate")
    ap.add_argument("--served-isolated", action="store_true",
                    help="served: also run every job alone (isolated compute time per job)")
    ap.add_argument("--no-extras", action="store_true",
                    help="chol: skip the other workloads (mixed, update, batched, served) after the headline")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    modes = {"update": run_update, "mixed": run_mixed, "batched": run_batched,
             "served": run_served, "qr": run_qr, "left": run_left, "strassen": run_strassen}
    if args.mode in modes:
        print(json.dumps(modes[args.mode](args)))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
