#!/usr/bin/env python
"""Benchmark of the GB300 randomized ID: one step = one whole ID (sketch,
pivoted QR, triangular solve, probe error estimate) of the 32 GiB complex128
matrix m = 262144, n = 8192 (k = 200, l = 208), inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank decomposes
its own matrix (independent problems, no collective on the data path) and
the value is the total over ranks (weak scaling).  --impl reference times
the CPU oracle on a bounded column slab of the same workload.  At N = 1 the
line also carries, after the timed region, the end-to-end figure from host
buffers (`e2e`), the 24-bit test matrix variant, the CPU oracle and a
serving sample (`serving`: served IDs/s with p50 / p99 latency); the other
workloads run with --config (mixed_c64, batched, serving, ...).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "complex ID GB-of-A/s & fraction of roofline; served IDs/s at p99 latency"
# FP64 FMA peak of GB300 from unit counts and clocks: 152 SMs x 2 DFMA/clock
# x 2 flops x 2.07 GHz maximum SM clock (a DFMA probe measured 1.20 TF/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes of one sketch_tc_kernel launch of the 32 GiB workload (one column
# panel of 2048 columns): the 65536 x 2048 capture of
# profiles/sketch_tc_kernel_65536x2048.md, 4 x (4.897 + 0.129) GB, scaled by
# the panel's 4x rows; reported only for the sources it was measured on (hash
# of rid_sketch_tc.cu, rid_tc_digits.cuh and rid_tc.cuh)
TC_TRAFFIC = {"bytes_per_launch": 20.11e9,
              "source_sha1": "c6a5aef34e42c6854aab596daa3b9c8175c2a33d"}


TC_SOURCES = ("rid_sketch_tc.cu", "rid_tc_digits.cuh", "rid_tc.cuh")     # the product kernel's source


def tc_source_sha1():
    import hashlib
    h = hashlib.sha1()
    for name in TC_SOURCES:
        with open(os.path.join(ROOT, "paper_1205_3830_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def tc_source_unchanged():
    try:
        return TC_TRAFFIC["source_sha1"] == tc_source_sha1()
    except OSError:
        return False


NVSMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={NVSMI_FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, flag in zip(names, parts[5:9]):
                    if flag.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def init_dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if _cuda_ok() else "gloo")
    return world, rank, local


def _cuda_ok():
    import torch
    return torch.cuda.is_available()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _cuda_ok() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle on a bounded column slab (the cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_slab_setup(cfg, A_slab_host, omega_bits=0):
    import oracle
    Omega = oracle.gaussian_test_matrix(cfg.l, cfg.m, cfg.seed)   # untimed: plan creation
    if omega_bits:
        Omega = oracle.round_test_matrix(Omega, omega_bits)
    probes = oracle.probe_matrix(A_slab_host.shape[1], 8, 1)
    return Omega, probes


def oracle_slab_step(cfg, Omega, A_slab, probes):
    import oracle
    Y = oracle.randomize(Omega, A_slab)
    R, tau, perm = oracle.qr_select(Y, cfg.k)
    T = oracle.factor_r(R[:cfg.k, :cfg.k], R[:cfg.k, cfg.k:])
    est, upper, _ = oracle.error_estimate(A_slab, perm, T, probes)
    return est


def cpu_cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count()


def run_reference(args, cfg, world, rank):
    """The oracle as it stands, on host cores, on a column slab of the workload."""
    if rank != 0:
        return
    import numpy as np
    import torch
    import synth
    ns = args.ref_cols
    if _cuda_ok():
        import synth.device
        A = synth.device.device_matrix(cfg)
        A_slab = np.asfortranarray(A[:, :ns].cpu().numpy())
        del A
        torch.cuda.empty_cache()
    else:   # no GPU: the same recipe on the host at the slab's width
        small = synth.scaled_config(cfg, cfg.m, ns)
        A_slab = synth.host_matrix(small)
    Omega, probes = oracle_slab_setup(cfg, A_slab, args.omega_bits)
    for _ in range(args.warmup):
        oracle_slab_step(cfg, Omega, A_slab, probes)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_slab_step(cfg, Omega, A_slab, probes)
    dt = (time.perf_counter() - t0) / args.steps
    bytes_per_step = cfg.a_bytes * ns / cfg.n
    value = bytes_per_step / dt / 1e9
    sample = f"oracle ID of the column slab A[:, :{ns}] (m={cfg.m}, k={cfg.k}, l={cfg.l}); Omega drawn untimed"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(cfg, args),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(cfg, args):
    kind = (f"A = U V^H + tail (sigma_j = 1 for j <= {cfg.rank}, tail ~{cfg.eps:g})" if cfg.kind == "spectrum"
            else f"A = X Y + {cfg.eps:g} N (rank {cfg.rank})")
    ctype = "complex64" if cfg.dtype == "c64" else "complex128"
    return {"workload": f"{cfg.name}: {ctype} {kind}, m={cfg.m}, n={cfg.n}, k={cfg.k}, l={cfg.l}, "
                        f"{cfg.a_bytes / 2**30:.0f} GiB",
            "m": cfg.m, "n": cfg.n, "k": cfg.k, "l": cfg.l, "nprobe": args.nprobe, "mode": args.mode, "estimator": args.estimator,
            "omega": (("subsampled randomized Fourier transform S F D" if args.omega == "srft" else "complex Gaussian")
                      + (" (FP64)" if not args.omega_bits else
                         f" rounded to {args.omega_bits} bits below each row's maximum")),
            "l2": "inputs larger than L2 (A is %.0f GiB, L2 129 MB)" % (cfg.a_bytes / 2**30)}


# ---------------------------------------------------------------------------
# The GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, cfg, world, rank, local):
    import torch
    import synth
    import synth.device
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, n, k, l = cfg.m, cfg.n, cfg.k, cfg.l
    A = synth.device.device_matrix(cfg, device=dev)
    stream = torch.cuda.current_stream(dev)
    a_dtype = torch.complex64 if cfg.dtype == "c64" else torch.complex128
    rows = args.estimator == "rows"
    # the error's products ride along in the sketch: the plan is built with its row probes
    plan = rid.Plan(m, n, k, l, seed=cfg.seed + rank, dtype=a_dtype, mode=args.mode, stream=stream,
                    nprobe=args.nprobe if rows else 0, probe_seed=1)
    plan.enable_timing()
    if args.omega == "srft":
        plan.use_srft(cfg.seed + 1)           # the paper's S F D in place of the Gaussian rows
    if args.omega_bits:
        plan.round_omega(args.omega_bits)     # Omega (and the probes) rounded: bits / 8 digits
    Y = rid.colmajor_empty(l, n, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    T = rid.colmajor_empty(k, n - k, device=dev)

    def step(ev=None):
        if ev: ev[0].record(stream)
        plan.sketch(A, Y)
        if ev: ev[1].record(stream)
        plan.select(Y, perm)
        if ev: ev[2].record(stream)
        plan.solve(Y, T)
        if ev: ev[3].record(stream)
        res = plan.error_sketched(perm, T) if rows else plan.error(A, perm, T, args.nprobe, 1)
        if ev: ev[4].record(stream)
        return res

    for _ in range(args.warmup):
        step()
    plan.sync_status()
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    start.record(stream)
    kernel_ms = []
    for s in range(args.steps):
        est, upper = step(events[s])          # rid_error has synchronized the stream
        kernel_ms.append(plan.sketch_times())
    stop.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier(world)
    plan.sync_status()
    ms = max_over_ranks(start.elapsed_time(stop), world)
    ms_step = ms / args.steps
    per = {name: statistics.mean(ev[i].elapsed_time(ev[i + 1]) for ev in events)
           for i, name in enumerate(("sketch", "select", "solve", "error"))}
    st = plan.stats()
    launches = args.steps * (st["sketch_launches"] + st["select_launches"] + st["solve_launches"] +
                             (2 if rows else st["error_launches"]))
    # the column-probe estimator (a second pass over A), timed once for context
    col_ms = None
    if rows:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.error(A, perm, T, args.nprobe, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        col_ms = e0.elapsed_time(e1)
    value = world * cfg.a_bytes / 1e9 / (ms_step / 1e3)

    # roofline of the dominant kernel (the sketch's product) and of the whole ID
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bf16_sust = float(peaks.get("bf16_tflops_sustained", 1724.5))
    ls = l + (args.nprobe if rows else 0)               # rows of the product: Omega, then the row probes
    sketch_flops = 8.0 * ls * m * n                      # complex ls x m x n product
    k_ms = [statistics.mean(t[i] for t in kernel_ms) for i in range(3)]
    t_prod = k_ms[1] / 1e3
    fp64_equiv = {"achieved": sketch_flops / t_prod / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s"}
    fp64_equiv["frac"] = fp64_equiv["achieved"] / FP64_PEAK_TFLOPS
    if args.mode == "fp64":
        roof = {"bound": "alu", "achieved": fp64_equiv["achieved"], "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": fp64_equiv["frac"], "traffic": None, "kernel": "sketch_fp64_kernel",
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz (a DFMA probe measured 1.20)",
                "per_launch": "8 (l + r) m n flops (complex product, r row probes)" if rows else "8 l m n flops"}
        tc_flops = None
    else:
        # the emulation's own work: BF16 slice-pair products of the real
        # (2l x 2m) x (2m x n) problem, 2 flops per multiply-add (28 pairs for the
        # FP64-grade digits, 6 for the BF16x3 splits of the mixed mode)
        so = (args.omega_bits + 7) // 8 if args.omega_bits else 7
        pairs = sum(1 for s_ in range(so) for t_ in range(7) if s_ + t_ <= 6) if args.mode == "fp64_emulated" else 6
        tc_flops = pairs * 2.0 * (2 * ls) * (2 * m) * n
        achieved = tc_flops / t_prod / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf16_sust, "unit": "TFLOP/s",
                "frac": achieved / bf16_sust,
                "traffic": (TC_TRAFFIC.get("bytes_per_launch") if args.mode == "fp64_emulated" and tc_source_unchanged()
                            and cfg.name == "large_tall" and not (args.m or args.n) and rows else None),
                "kernel": "sketch_tc_kernel" if args.mode == "fp64_emulated" else "sketch_mixed_kernel",
                "peak_source": "of measured: MEASURED_PEAKS.json bf16_tflops_sustained (kernel timed inside a long step)",
                "per_launch": (f"{pairs} slice pairs x 2 x (2 ls)(2m)(n / panels) flops, ls = l + r row probes, "
                               f"one launch per column panel" if rows else
                               f"{pairs} slice pairs x 2 x (2l)(2m)(n / panels) flops, one launch per column panel"),
                "fp64_equivalent": fp64_equiv}
    # whole-ID roofline: sum over steps of max(bytes / HBM, flops / the peak of the pipe used)
    p64 = FP64_PEAK_TFLOPS * 1e12
    a_b = float(cfg.a_bytes)
    sketch_roof = (max(a_b / (hbm * 1e9), sketch_flops / p64) if tc_flops is None
                   else max(a_b / (hbm * 1e9), tc_flops / (bf16_sust * 1e12)))
    err_roof = (max(16.0 * k * (n - k) / (hbm * 1e9), 8.0 * k * (n - k) * args.nprobe / p64) if rows
                else max(a_b / (hbm * 1e9), 8.0 * m * n * args.nprobe / p64))
    t_roof = (sketch_roof +
              max(2 * 16.0 * l * n * k / (hbm * 1e9), 16.0 * n * (l * k - k * k / 2) / p64) +
              4.0 * k * k * (n - k) / p64 + err_roof)
    id_frac = t_roof / (ms_step / 1e3)

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if args.mode == "bf16" else "f64",
        "data": "synthetic (seeded, generated on the device)",
        "config": workload_config(cfg, args),
        "roofline": roof,
        "id_roofline_frac": id_frac,
        # algorithmic FP64 work of the whole ID: sketch (with the row probes), QR, solve, error
        "gflops": world * (sketch_flops + 16.0 * n * (l * k - k * k / 2) + 4.0 * k * k * (n - k) +
                           (8.0 * k * (n - k) * args.nprobe if rows else 8.0 * m * n * args.nprobe)) / (ms_step / 1e3) / 1e9,
        "step_ms": per,
        "sketch_kernel_ms": ({"slice": k_ms[0], "product": k_ms[1], "reduce": k_ms[2]} if args.mode != "bf16" else
                             {"slice": k_ms[0], "product": k_ms[1], "reduce": k_ms[2],
                              # the rest of the sketch: the row probes' own product (digits of
                              # A cut on chip) and its reduction
                              "probe_rows": max(0.0, per["sketch"] - k_ms[0] - k_ms[1] - k_ms[2])}),
        "gpu_launches": launches,
        "error_estimate": {"est": est, "upper": upper,
                           "estimator": ("row probes multiplied in the sketch's pass over A" if rows
                                         else "column probes, a second pass over A"),
                           "column_probe_pass_ms": col_ms},
        "clocks": clocks,
    }

    if args.e2e_steps > 0:
        line["e2e"] = run_e2e(args, cfg, plan, A, Y, perm, T, stream, world)
    if args.mode == "fp64_emulated" and not args.omega_bits and args.omega == "gaussian" and args.rounded_variant:
        line["omega_rounded_24bit"] = time_rounded_omega(args, cfg, A, stream, world, rank)
    if args.mode == "bf16":
        line["vs_fp64_path"] = compare_with_fp64(args, cfg, A, perm, T, stream, rank)
        # the plan's own verdict on the last ID: rho (the pivoted QR's estimate
        # of sigma_{k+1} / sigma_1) against the mode's measured floor
        rho, floor, accepted = plan.accuracy(Y)
        line["accuracy"] = {"rho": rho, "floor": floor, "accepted": accepted,
                            "reading": ("above the mixed mode's measured floor: the FP64 path's J and an ID error "
                                        "within 2x of it" if accepted else
                                        "below the mixed mode's measured floor: recompute in an FP64 mode")}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, cfg, A)
    plan.close()
    if world == 1 and args.serving_requests > 0 and args.mode == "fp64_emulated":
        # the metric's second part: served IDs/s at p99 latency, one rate past saturation
        del A, Y, perm, T
        torch.cuda.empty_cache()
        try:
            rates = [float(x) for x in args.serving_rates.split(",")]
            sweep, select_shape = serve_sweep(args, rates, args.serving_requests, rank, local, args.pool)
            s = max(sweep, key=lambda x: x["served_per_s"])     # saturation: the highest served rate
            line["serving"] = {"value": s["served_per_s"], "unit": "IDs/s", "p50_ms": s["p50_ms"],
                               "p99_ms": s["p99_ms"], "gb_per_s": s["gb_per_s"], "offered_per_s": s["offered_per_s"],
                               "errors": sum(x["errors"] for x in sweep), "slots": args.slots,
                               "select": select_shape, "sweep": sweep,
                               "workload": f"{args.serving_requests} requests per rate, {SERVING_WORKLOAD}, "
                                           f"cycling through {args.pool} device-resident matrices, FP64-emulated"}
        except Exception as exc:            # reported in the line; the headline above stands
            line["serving"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def time_rounded_omega(args, cfg, A, stream, world, rank):
    """The same step with the test matrix (and row probes) rounded to 24 bits
    below each row's maximum: the emulated product then multiplies 18 digit
    pairs instead of 28 and stays exact for that Omega.  Reported beside the
    headline, which uses the unrounded Gaussian Omega."""
    import torch
    import paper_1205_3830_gb300 as rid
    m, n, k, l = cfg.m, cfg.n, cfg.k, cfg.l
    plan = rid.Plan(m, n, k, l, seed=cfg.seed + rank, dtype=A.dtype, mode="fp64_emulated", stream=stream)
    plan.enable_timing()
    rows = args.estimator == "rows"
    if rows:
        plan.set_probes(args.nprobe, 1)
    plan.round_omega(24)
    Y = rid.colmajor_empty(l, n, device=A.device)
    perm = torch.empty(n, dtype=torch.int32, device=A.device)
    T = rid.colmajor_empty(k, n - k, device=A.device)

    def step():
        plan.sketch(A, Y)
        plan.select(Y, perm)
        plan.solve(Y, T)
        return plan.error_sketched(perm, T) if rows else plan.error(A, perm, T, args.nprobe, 1)

    for _ in range(3):
        step()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    prod = []
    for _ in range(reps):
        est, upper = step()
        prod.append(plan.sketch_times()[1])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world) / reps
    plan.close()
    return {"value": world * cfg.a_bytes / 1e9 / (ms / 1e3), "unit": "GB/s", "ms_per_step": ms, "steps": reps,
            "product_ms": statistics.mean(prod), "digit_pairs": 18, "error_estimate": {"est": est, "upper": upper},
            "omega": "complex Gaussian rounded to 24 bits below each row's maximum (ties to even)"}


def run_select_phase(args, cfg, world, rank, local):
    """The pivoted QR alone on a seeded random l x n complex Y (the sketch's
    shape for the config), with the plan's default launch shape; one JSON
    line with the per-call time (CUDA events).  For profiling the select
    without the config's A on the device."""
    import torch
    import synth
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.MASTER_SEED + 11 + rank)
    Y0 = torch.randn((cfg.n, cfg.l), dtype=torch.complex128, device=dev, generator=gen).t()
    plan = rid.Plan(cfg.m, cfg.n, cfg.k, cfg.l, seed=cfg.seed + rank, mode=args.mode)
    if args.select_ctas is not None:
        plan.set_select_grid(args.select_ctas)
    Y = rid.colmajor_empty(cfg.l, cfg.n, device=dev)
    perm = torch.empty(cfg.n, dtype=torch.int32, device=dev)
    times = []
    for s in range(args.warmup + args.steps):
        Y.copy_(Y0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.select(Y, perm)
        e1.record()
        torch.cuda.synchronize()
        if s >= args.warmup:
            times.append(e0.elapsed_time(e1))
    plan.sync_status()
    if rank == 0:
        print(json.dumps({"phase": "select", "config": cfg.name, "l": cfg.l, "n": cfg.n, "k": cfg.k,
                          "select_ctas": args.select_ctas, "select_ms": statistics.mean(times),
                          "select_ms_min": min(times), "launches": plan.stats()["select_launches"],
                          "perm_head": perm[:4].tolist()}), flush=True)
    plan.close()


def run_e2e(args, cfg, plan, A, Y, perm, T, stream, world):
    """Same metric with host buffers: every step copies A in from pinned host
    memory and reads perm, T and the estimate back.  With the row-probe
    estimator nothing after the sketch reads A, so A travels in column panels
    on a copy stream: the sketch of a panel starts as soon as it has landed,
    and the next step's copy of a panel starts as soon as this step's sketch
    of it is done (the host->device link, about 211 GB/s, is the bound)."""
    import torch
    allowed = os.sched_getaffinity(0)
    placement = pin_near_gpu(A.device)          # before the pinned buffer is allocated and first touched
    A_host = torch.empty((cfg.n, cfg.m), dtype=A.dtype, pin_memory=True).t()
    A_host.copy_(A)
    torch.cuda.synchronize()
    os.sched_setaffinity(0, allowed)
    perm_h = torch.empty(cfg.n, dtype=torch.int32, pin_memory=True)
    T_h = torch.empty((cfg.n - cfg.k, cfg.k), dtype=torch.complex128, pin_memory=True).t()
    torch.cuda.synchronize()
    rows = args.estimator == "rows"
    pipelined = rows and args.mode in ("fp64", "fp64_emulated", "bf16")     # modes with column-range sketches
    n = cfg.n
    width = max(128, (n // 8 + 127) // 128 * 128)
    panels = [(c0, min(width, n - c0)) for c0 in range(0, n, width)] if pipelined else [(0, n)]
    copy_stream = torch.cuda.Stream(A.device)
    landed = [torch.cuda.Event() for _ in panels]
    done = [torch.cuda.Event() for _ in panels]
    # this machine's host->device rate for this buffer: the whole of A, copied
    # panel by panel with nothing else running (the rate differs between boxes
    # and between parts of a large pinned buffer); the better of a copy before
    # and one after the untimed pass, so first-touch costs of the pinned
    # buffer do not lower it
    def link_rate():
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        l0.record(copy_stream)
        with torch.cuda.stream(copy_stream):
            for c0, nc in panels:
                A[:, c0:c0 + nc].copy_(A_host[:, c0:c0 + nc], non_blocking=True)
        l1.record(copy_stream)
        torch.cuda.synchronize()
        return A.numel() * A.element_size() / 1e9 / (l0.elapsed_time(l1) / 1e3)

    link_first = link_rate()

    # optional trace of the timed passes: per step and panel, the copy's start
    # and end (copy stream) and the sketch's start and end (compute stream)
    trace = []

    def timed_event(stream_):
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream_)
        return ev

    def copy_in(rec=None):
        for i, (c0, nc) in enumerate(panels):
            copy_stream.wait_event(done[i])          # this panel's previous sketch has read A
            t0 = timed_event(copy_stream) if rec is not None else None
            with torch.cuda.stream(copy_stream):
                A[:, c0:c0 + nc].copy_(A_host[:, c0:c0 + nc], non_blocking=True)
            landed[i].record(copy_stream)
            if rec is not None:
                rec.append({"panel": i, "copy": (t0, timed_event(copy_stream))})

    def passes(steps, traced=False):
        copy_stream.wait_stream(stream)
        recs = [[] for _ in range(steps)] if traced else None
        copy_in(recs[0] if traced else None)
        for step in range(steps):
            for i, (c0, nc) in enumerate(panels):
                stream.wait_event(landed[i])
                s0 = timed_event(stream) if traced else None
                if pipelined:
                    plan.sketch_cols(A, Y, c0, nc)
                else:
                    plan.sketch(A, Y)
                done[i].record(stream)
                if traced and i < len(recs[step]):
                    recs[step][i]["sketch"] = (s0, timed_event(stream))
            if rows and step + 1 < steps:
                copy_in(recs[step + 1] if traced else None)   # the next step's A, behind this step's sketch
            plan.select(Y, perm)
            plan.solve(Y, T)
            if rows:
                plan.error_sketched(perm, T)
            else:
                plan.error(A, perm, T, args.nprobe, 1)
            perm_h.copy_(perm, non_blocking=True)
            T_h.copy_(T, non_blocking=True)
            if not rows and step + 1 < steps:
                copy_stream.wait_stream(stream)     # the column-probe error read A: the next copy follows it
                copy_in(recs[step + 1] if traced else None)
        return recs

    passes(1)                                        # untimed: the first pass of this pattern
    torch.cuda.synchronize()
    link_gbs = max(link_first, link_rate())
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    start.record(stream)
    passes(args.e2e_steps)
    stop.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(start.elapsed_time(stop), world) / args.e2e_steps
    # a traced pass after the timed region (events add little, but none sit in it)
    t_start = timed_event(copy_stream)
    recs = passes(max(2, args.e2e_steps), traced=True)
    torch.cuda.synchronize()
    trace = e2e_trace_summary(recs, t_start, [nc for _, nc in panels], cfg.m, A.element_size())
    del A_host
    h2d = cfg.a_bytes
    d2h = 4 * cfg.n + 16 * cfg.k * (cfg.n - cfg.k) + 16
    value = world * cfg.a_bytes / 1e9 / (ms / 1e3)
    return {"value": value, "unit": "GB/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms, "steps": args.e2e_steps,
            "h2d_link_gbs": link_gbs, "frac_of_link": value / (world * link_gbs),
            "pipeline": (f"A in {len(panels)} column panels on a copy stream, overlapped with the sketch"
                         if pipelined else ("A copied whole; the next step's copy overlaps select, solve and "
                                            "error" if rows else "A copied whole, then the ID")),
            "trace": trace, "host_placement": placement}


def pin_near_gpu(device):
    """Run this process on the CPUs that sysfs lists as local to the GPU's PCI
    device, so the pinned host buffer allocated next lands in that node's
    memory; returns what was found (the bus id, the NUMA node, the CPU list)."""
    import torch
    out = {"affinity_set": False}
    try:
        p = torch.cuda.get_device_properties(device)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        out["pci"] = bus
        base = f"/sys/bus/pci/devices/{bus}"
        with open(f"{base}/numa_node") as f:
            out["numa_node"] = int(f.read().strip())
        with open(f"{base}/local_cpulist") as f:
            cpulist = f.read().strip()
        out["local_cpus"] = cpulist
        cpus = set()
        for part in cpulist.split(","):
            if "-" in part:
                lo, hi = part.split("-")
                cpus.update(range(int(lo), int(hi) + 1))
            elif part:
                cpus.add(int(part))
        allowed = os.sched_getaffinity(0)
        if cpus and cpus & allowed and cpus & allowed != allowed:
            os.sched_setaffinity(0, cpus & allowed)
            out["affinity_set"] = True
    except (OSError, ValueError, AttributeError) as exc:
        out["note"] = f"{type(exc).__name__}: {exc}"
    return out


def e2e_trace_summary(recs, t_start, widths, m, esize):
    """Per-panel copy and sketch intervals of a traced end-to-end pass: the
    copy rate of each panel, the copy engine's busy share, the time the
    sketch of a panel waited for its copy and the copy for the sketch."""
    steps = []
    for rec in recs:
        t = [(r["copy"][0], r["copy"][1], r["sketch"][0], r["sketch"][1]) for r in rec if "sketch" in r]
        if not t:
            continue
        c_ms = [a.elapsed_time(b) for a, b, _, _ in t]
        s_ms = [c.elapsed_time(d) for _, _, c, d in t]
        span = t[0][0].elapsed_time(t[-1][3])
        rates = [w * m * esize / 1e9 / (ms / 1e3) for w, ms in zip(widths, c_ms) if ms > 0]
        # idle gaps of the copy engine between consecutive panels' copies
        gaps = [t[i][1].elapsed_time(t[i + 1][0]) for i in range(len(t) - 1)]
        steps.append({"span_ms": span, "copy_ms": sum(c_ms), "sketch_ms": sum(s_ms),
                      "copy_busy_frac": sum(c_ms) / span if span > 0 else None,
                      "copy_gbs_min": min(rates) if rates else None, "copy_gbs_max": max(rates) if rates else None,
                      "copy_gap_ms_max": max(gaps) if gaps else 0.0})
    return {"steps": steps}


def compare_with_fp64(args, cfg, A, perm, T, stream, rank):
    """The plain FP64 GPU path (FP64-emulated sketch, FP64 QR / solve / error) on
    the same inputs upcast to complex128: its throughput and how far the mixed
    path's ID lies from it."""
    import torch
    import paper_1205_3830_gb300 as rid
    m, n, k, l = cfg.m, cfg.n, cfg.k, cfg.l
    A128 = A.t().to(torch.complex128).t()
    plan = rid.Plan(m, n, k, l, seed=cfg.seed + rank, mode="fp64_emulated", stream=stream)
    rows = args.estimator == "rows"
    if rows:
        plan.set_probes(args.nprobe, 1)
    Y = rid.colmajor_empty(l, n, device=A.device)
    perm2 = torch.empty(n, dtype=torch.int32, device=A.device)
    T2 = rid.colmajor_empty(k, n - k, device=A.device)

    def step():
        plan.sketch(A128, Y)
        plan.select(Y, perm2)
        plan.solve(Y, T2)
        return plan.error_sketched(perm2, T2) if rows else plan.error(A128, perm2, T2, args.nprobe, 1)

    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = 2
    for _ in range(reps):
        est, upper = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    same_J = bool(torch.equal(torch.sort(perm[:k]).values, torch.sort(perm2[:k]).values))
    same_perm = bool(torch.equal(perm[:k], perm2[:k]))
    dT = None
    if same_perm and n > k:
        dT = float((T - T2).abs().max() / T2.abs().max())
    plan.close()
    del A128
    return {"fp64_path_value": cfg.a_bytes / 1e9 / (ms / 1e3), "fp64_path_ms_per_step": ms, "unit": "GB/s",
            "same_J": same_J, "same_pivot_order": same_perm, "max_dT_rel": dT, "fp64_path_error_estimate": est,
            "stated_accuracy": "mixed sketch (BF16x3, FP32 sums) vs FP64-emulated sketch, same Omega and A"}


def cpu_baseline(args, cfg, A):
    import numpy as np
    ns = args.ref_cols
    A_slab = np.asfortranarray(A[:, :ns].cpu().numpy())
    Omega, probes = oracle_slab_setup(cfg, A_slab, args.omega_bits)
    t0 = time.perf_counter()
    oracle_slab_step(cfg, Omega, A_slab, probes)
    dt = time.perf_counter() - t0
    return {"value": cfg.a_bytes * ns / cfg.n / dt / 1e9, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"oracle ID of the column slab A[:, :{ns}] (m={cfg.m}, k={cfg.k}, l={cfg.l}), "
                      f"{dt:.1f} s; Omega drawn untimed"}


# ---------------------------------------------------------------------------
# Batched and served forms
# ---------------------------------------------------------------------------
def device_lowrank(m, n, rank, eps, gen, device):
    import torch
    X = torch.randn((m, rank), generator=gen, dtype=torch.complex128, device=device)
    Yf = torch.randn((rank, n), generator=gen, dtype=torch.complex128, device=device)
    A = torch.randn((n, m), generator=gen, dtype=torch.complex128, device=device).t().mul_(eps)
    return A.addmm_(X, Yf)


def run_batched(args, world, rank, local):
    """4096 independent complex128 IDs (m, n ~ U[64, 1024], k ~ U[4, 64],
    l = k + 8, A = X Y + 1e-10 N) per step.  Timed: the tensor-core batch (all
    sketches in one persistent launch, then one persistent launch of select,
    solve and the row-probe error, replayed as one CUDA graph, tile shapes
    from the autotuner); beside it the FP64 persistent batch (one launch, CUDA
    graph) and the plan path."""
    import torch
    import synth
    import paper_1205_3830_gb300 as rid
    from paper_1205_3830_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    shapes = synth.batched_shapes(args.count, synth.MASTER_SEED + 4 + rank)
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.MASTER_SEED + 4 + rank)
    problems = [(device_lowrank(m, n, k, 1e-10, gen, dev), k, l, 1000 + i) for i, (m, n, k, l) in enumerate(shapes)]
    r = args.nprobe
    stream = torch.cuda.current_stream(dev)
    # tile shapes per size class from the autotuner (its cache file, tuned
    # here for classes it does not hold yet), outside the timed region
    tuning = rid.TcTuning(os.path.join(ROOT, "paper_1205_3830_gb300", "_build", "tc_tiles.json"))
    t_tune = time.perf_counter()
    tuned = tuning.tune(problems, nprobe=r, probe_seed=1, force=False) if args.tune else {}
    t_tune = time.perf_counter() - t_tune
    tcb = rid.BatchTC(problems, nprobe=r, probe_seed=1, tuning=tuning if args.tune else None)
    tc_info = tcb.info()
    choices = {}
    for t, s in zip(tcb.tile_n, tcb.ksplit):
        key = f"tile_n={t or 128},ksplit={s or 1}"
        choices[key] = choices.get(key, 0) + 1
    for _ in range(args.warmup):
        tcb.run()
    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        tcb.run()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world) / args.steps
    sketch_ms, post_ms = tcb.times()
    res = tcb.results()
    ok = int(sum(1 for x in res if x["status"] == 0))
    tcb.close()
    del tcb
    torch.cuda.synchronize()

    a_bytes = sum(16.0 * m * n for (m, n, k, l) in shapes)
    pair_flops = sum(28 * 2.0 * (2 * (l + r)) * (2 * m) * n for (m, n, k, l) in shapes)
    post_flops = sum(16.0 * n * (l * k - k * k / 2) + 4.0 * k * k * (n - k) + 8.0 * k * (n - k) * r
                     for (m, n, k, l) in shapes)
    peaks = measured_peaks()
    bf16_sust = float(peaks.get("bf16_tflops_sustained", 1724.5))
    tc_roof = {"bound": "tensor", "achieved": pair_flops / (sketch_ms / 1e3) / 1e12, "peak": bf16_sust,
               "unit": "TFLOP/s", "traffic": None, "kernel": "sketch_tc_kernel (all problems, with slicing)",
               "per_launch": "28 digit pairs x 2 x 2(l + r) x 2m x n per problem; time of the whole sketch phase",
               "peak_source": "of measured: MEASURED_PEAKS.json bf16_tflops_sustained"}
    tc_roof["frac"] = tc_roof["achieved"] / bf16_sust
    post_roof = {"bound": "alu", "achieved": post_flops / (post_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                 "unit": "TFLOP/s", "traffic": None, "kernel": "batch_post_kernel",
                 "per_launch": "sum over problems of QR 16n(lk - k^2/2) + solve 4k^2(n-k) + error 8k(n-k)r flops"}
    post_roof["frac"] = post_roof["achieved"] / FP64_PEAK_TFLOPS
    dominant, other = (post_roof, tc_roof) if post_ms >= sketch_ms else (tc_roof, post_roof)

    # the FP64 persistent batch (one launch, captured in a CUDA graph)
    batch = rid.Batch(problems, nprobe=r, probe_seed=1)
    tile, _ = batch.autotune()
    batch.capture(tile)
    batch.replay()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(2):
        batch.replay()
    f1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = f0.elapsed_time(f1) / 2
    del batch
    # the plain FP64 GPU path on the same inputs: one plan per problem, in turn
    sub = min(64, len(problems))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (A, k, l, sd) in problems[:sub]:
        rid.decompose(A, k, l, seed=sd, mode="fp64", nprobe=r, probe_seed=1)
    torch.cuda.synchronize()
    plan_ids_s = sub / (time.perf_counter() - t0)
    line = {
        "metric": METRIC, "value": world * a_bytes / 1e9 / (ms / 1e3), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded, generated on the device)",
        "config": {"workload": f"batched: {len(shapes)} complex128 IDs, m, n ~ U[64, 1024], k ~ U[4, 64], l = k + 8, "
                               f"A = X Y + 1e-10 N ({a_bytes / 2**30:.1f} GiB in all)",
                   "count": len(shapes), "nprobe": r, "estimator": "rows",
                   "path": "tensor-core batch: all sketches in one persistent cooperative launch (waves of "
                           "digit cutting, grid barrier, longest-first work lists of tcgen05 products), then one "
                           "persistent launch of select / solve / error; both in one CUDA graph",
                   "cuda_graph": True, "l2": "inputs larger than L2 (%.1f GiB)" % (a_bytes / 2**30)},
        "ids_per_s": world * len(shapes) / (ms / 1e3),
        "phase_ms": {"sketches": sketch_ms, "select_solve_error": post_ms},
        "workspace": {"device_bytes": tc_info["bytes"], "gib": tc_info["bytes"] / 2**30, "waves": tc_info["waves"],
                      "work_items": tc_info["items"], "ctas": tc_info["ctas"],
                      "holds": "Omega and probe rows of every problem, X, two digit buffers of at most 2 GiB"},
        "tuning": {"autotuned": bool(args.tune), "classes_timed_now": len(tuned), "tune_s": t_tune,
                   "problems_per_choice": choices},
        "roofline": dominant,
        "roofline_other_phase": other,
        "gpu_launches": args.steps * 2,
        "ranks_ok": ok,
        "vs_fp64_batch": {"ids_per_s": world * len(shapes) / (fp64_ms / 1e3), "ms_per_step": fp64_ms, "tile": tile,
                          "path": "one persistent FP64 launch (CTA per problem), CUDA graph"},
        "vs_fp64_plan_path": {"ids_per_s": plan_ids_s, "problems_timed": sub,
                              "accuracy": "same J, T within 1e-12 (tests/test_gpu_batched.py)"},
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def serve_sweep(args, rates, requests, rank, local, pool=64):
    """Serve `requests` seeded requests at each offered rate (Poisson arrivals)
    and return the sweep (served IDs/s, GB of A/s, p50 / p99 ms, the plans'
    share per rate) and the server's select launch shape.  The requests cycle
    through `pool` distinct device matrices drawn from the workload's shape
    distribution (request i: matrix i % pool, its own seed 2000 + i), so a
    thousand requests per rate fit beside the server's memory."""
    import numpy as np
    import torch
    import synth
    from paper_1205_3830_gb300 import serve
    dev = torch.device("cuda", local)
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.MASTER_SEED + 5 + rank)
    pool = max(1, min(pool, requests))
    specs = synth.serving_requests(pool, 1.0, synth.MASTER_SEED + 5 + rank)      # shapes of the pool
    mats = [device_lowrank(m, n, k, 1e-10, gen, dev) for (_, m, n, k, l) in specs]
    a_bytes = sum(16.0 * specs[i % pool][1] * specs[i % pool][2] for i in range(requests))
    # warm-up: every kernel once
    serve.run_one(mats[0], specs[0][3], specs[0][4], 1, args.nprobe, 1, args.mode)
    sweep = []
    for rate in rates:
        opts = {} if args.select_ctas is None else {"select_ctas": args.select_ctas}
        srv = serve.Server(slots=args.slots, mode=args.mode, **opts)
        gaps = np.random.default_rng(synth.MASTER_SEED + 7 + rank).exponential(1.0 / rate, size=requests)
        t0 = time.perf_counter()
        due = 0.0
        for i in range(requests):
            _, m, n, k, l = specs[i % pool]
            due += gaps[i]
            wait = t0 + due - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            srv.submit(i, mats[i % pool], k, l, 2000 + i, args.nprobe, 1)
        done = srv.drain(timeout=900)            # a stuck request ends the sweep with an error, not a hang
        wall = time.perf_counter() - t0
        srv.close()
        errs = sum(1 for r in done if r.error is not None)
        st = serve.latency_stats(done)
        sweep.append({"offered_per_s": rate, "requests": len(done), "served_per_s": len(done) / wall,
                      "gb_per_s": a_bytes / 1e9 / wall, "p50_ms": st.get("p50_ms"), "p99_ms": st.get("p99_ms"),
                      "plan_dev_p50_ms": st.get("plan_dev_p50_ms"), "plan_host_p50_ms": st.get("plan_host_p50_ms"),
                      "id_dev_p50_ms": st.get("id_dev_p50_ms"), "plans_reused": st.get("plans_reused"),
                      "peak_concurrent": srv.peak_running,
                      "peak_hbm_gb": srv.peak_used / 1e9, "errors": errs})
    ctas = srv.select_ctas
    select_shape = ("the plan's default (one cooperative launch)" if ctas is None or ctas < 0 else
                    "one launch per step" if ctas == 0 else f"one cooperative launch of at most {ctas} CTAs")
    del mats
    torch.cuda.empty_cache()
    return sweep, select_shape


SERVING_WORKLOAD = ("complex128 ID requests, Poisson arrivals, m, n log-uniform [256, 16384], "
                    "k log-uniform [8, 256], l = k + 10")


def run_serving(args, world, rank, local):
    """Poisson stream of complex128 ID requests (m, n log-uniform in [256, 16384],
    k log-uniform in [8, 256], l = k + 10, A = X Y + 1e-10 N) at a sweep of
    rates; continuous batching admitted by HBM footprint; p50 / p99 latency."""
    import torch
    from paper_1205_3830_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    rates = [float(x) for x in args.rates.split(",")]
    sweep, select_shape = serve_sweep(args, rates, args.requests, rank, local, args.pool)
    best = max(sweep, key=lambda x: x["served_per_s"])
    line = {
        "metric": METRIC, "value": best["served_per_s"], "unit": "IDs/s", "n_gpus": world, "steps": len(rates),
        "warmup": 1, "ms_per_step": 1e3 / best["served_per_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.mode != "bf16" else "bf16",
        "data": "synthetic (seeded, generated on the device)",
        "config": {"workload": f"serving: {args.requests} {SERVING_WORKLOAD}",
                   "mode": args.mode, "slots": args.slots, "rates": rates,
                   "select": select_shape},
        "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "sweep": sweep,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--config", default="large_tall")
    ap.add_argument("--mode", default="fp64_emulated", choices=("fp64", "fp64_emulated", "bf16"))
    ap.add_argument("--nprobe", type=int, default=8)
    ap.add_argument("--no-rounded-variant", dest="rounded_variant", action="store_false",
                    help="skip the secondary measurement with a 24-bit rounded test matrix")
    ap.add_argument("--omega", choices=("gaussian", "srft"), default="gaussian",
                    help="test matrix: complex Gaussian or the paper's subsampled randomized Fourier transform")
    ap.add_argument("--omega-bits", type=int, default=0,
                    help="round the test matrix to this many bits below each row's maximum (0: unrounded)")
    ap.add_argument("--estimator", choices=("rows", "columns"), default=None,
                    help="error estimate from row probes multiplied in the sketch's pass over A (default; FP64-grade "
                         "in every mode) or from column probes in a second pass over A")
    ap.add_argument("--ref-cols", type=int, default=2048, help="column slab of the CPU oracle sample")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--count", type=int, default=4096, help="problems per batch (--config batched)")
    ap.add_argument("--tune", type=int, default=1,
                    help="--config batched: tile shapes per size class from the autotuner (1) or the defaults (0)")
    ap.add_argument("--requests", type=int, default=1000, help="requests per rate (--config serving)")
    ap.add_argument("--rates", default="40,160,320,640,1280,2560",
                    help="offered request rates per second (--config serving)")
    ap.add_argument("--pool", type=int, default=64,
                    help="distinct request matrices the requests cycle through (serving)")
    ap.add_argument("--slots", type=int, default=8, help="concurrent requests (--config serving)")
    ap.add_argument("--serving-requests", type=int, default=1000,
                    help="requests per rate of the serving sweep added to the headline line (0: none)")
    ap.add_argument("--serving-rates", default="160,320,640,1280,2560",
                    help="offered rates per second of the serving sweep added to the headline line")
    ap.add_argument("--select-ctas", type=int, default=None,
                    help="launch shape of the select: 0 one launch per step, N > 0 one cooperative launch of at "
                         "most N CTAs through L2, -1 the plan's default (--config serving: each served request's "
                         "select, default the server's, one launch per step; --phase select: default the plan's)")
    ap.add_argument("--phase", choices=("id", "select"), default="id",
                    help="select: time the pivoted QR alone on a random sketch-shaped Y (l x n of the config; "
                         "profiling without the config's A on the device)")
    ap.add_argument("--m", type=int, default=0, help="override m (profiling of smaller cases)")
    ap.add_argument("--n", type=int, default=0, help="override n (profiling of smaller cases)")
    args = ap.parse_args()
    if args.estimator is None:
        args.estimator = "rows"
    import dataclasses
    import synth
    world, rank, local = init_dist()
    if args.config in ("batched", "serving"):
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable":
                                  "the CPU oracle is timed on the single-ID workloads only"}), flush=True)
        elif args.config == "batched":
            run_batched(args, world, rank, local)
        else:
            run_serving(args, world, rank, local)
        return
    cfg = synth.CONFIGS[args.config]
    if args.m or args.n:
        cfg = dataclasses.replace(cfg, m=args.m or cfg.m, n=args.n or cfg.n)
    if args.impl == "reference":
        run_reference(args, cfg, world, rank)
    elif args.phase == "select":
        run_select_phase(args, cfg, world, rank, local)
    else:
        run_ours(args, cfg, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
