"""Benchmark: Metropolis spin-update attempts/ns of the single-spin sweep of the
3-D anisotropic Heisenberg model (arXiv 2106.11286) on one GB300, and the
fraction of the HBM roofline reached by the colour-pass kernel.

Workload (the headline configuration): sc 256^3 periodic (16,777,216 spins),
J = 1, K = 0.05, e = z, T = 1.2, random start from seed 2, FP32 spin storage
with FP64 reductions.  One step = one Metropolis sweep = both colour passes
with the fused E / M reductions into the FP64 accumulator.  The same
workload in plain FP64 is timed beside it ("fp64").  The state (201 MB in
FP32, 403 MB in FP64) is larger than the 129 MB L2, so no flush is needed
between steps.

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank advances
its own replica of the workload (replica index = rank; no data-path
collective) and the whole-job value is the attempts of all ranks over the
slowest rank's time ("scaling": "weak"); beside it, variants.slab_strong
times one sc 1024^3 lattice split into z-slabs over the ranks, halos
exchanged by NCCL after every colour pass (strong scaling; one rank: one
slab, its own periodic neighbour), and the same with the boundary planes
updated first and their exchange beside the interior update.  The headline is
the median of --repeats regions of exactly --steps steps.

``--impl reference`` times the CPU oracle (the plain FP64 C program that
defines the expected results) on this machine's host cores instead, each step
one oracle sweep of a bounded sub-lattice with the same parameters.
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

WORKLOAD = dict(name="sc256_fp32", kind="sc", L=256, J=1.0, K=0.05, e=(0.0, 0.0, 1.0), T=1.2, seed=2)
METRIC = "Metropolis spin-update attempts/ns (sc 256^3, FP32 spins, FP64 reductions)"
UNIT = "attempts/ns"
BYTES_PER_SPIN = {"fp64": 24, "fp32": 12, "fp16": 6}
# bytes per attempt the FP32 neighbour-table layout moves: 16-byte padded spin 4-vectors read twice and
# written once, 8 int32 table entries
TABLE_LAYOUT_BYTES = 3 * 16 + 8 * 4
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sc_pass_fp32_sc256_traffic.txt")


def config_dict(args, n_gpus):
    w = WORKLOAD
    return {"workload": f"sc {w['L']}^3 periodic, J={w['J']}, K={w['K']}, e=z, T={w['T']}, seed {w['seed']}, "
                        f"FP32 spins + FP64 reductions; step = 1 sweep (2 colour passes, fused E/M)",
            "lattice": "sc", "L": w["L"], "n_spins": w["L"] ** 3, "precision": "fp32",
            "sweeps_per_step": 1, "l2_policy": "inputs larger than L2 (201 MB state vs 129 MB L2)",
            "parallelism": f"replicas x{n_gpus}" if n_gpus > 1 else "1 GPU"}


# ------------------------------------------------------------------ helpers
KERNEL_SOURCES = ("kernels.cu", "device.cuh", "hs_impl.h")  # the dominant kernel's sources


def kernels_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_11286_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


# colour-pass kernel of each hs_kernel kind (hs_get_launch's "kernel")
KERNEL_NAMES = {1: "sc_pass_kernel", 3: "table_pass_kernel", 4: "sc_march_kernel", 5: "sc_pipe_kernel"}


def kernel_label(launch, precision_code=1, measure=1, zaxis=False):
    """Template label of the colour-pass kernel a launch configuration runs
    (as ncu names it), for matching the stored traffic to the timed kernel.
    zaxis: the lattice's easy axis is (0, 0, 1), for which FP32 V = 4 without
    prefetch runs its S.e = S_z variant (the last template argument)."""
    name = KERNEL_NAMES.get(launch["kernel"], "sc_pass_kernel")
    if launch["kernel"] == 1:
        pf = {1: 1, 3: 2}.get(launch["prefetch"], 0)
        ax = int(bool(zaxis) and precision_code == 1 and launch["vec_width"] == 4 and pf == 0)
        # then the direction-capable variant flag (every lattice up to 2^31 sites) and the axis variant
        return f"{name}<{precision_code}, {launch['vec_width']}, {measure}, {pf}, 0, 1, {ax}>"
    return name


ORDERS = {1: "ascending", 2: "alternating"}


def read_traffic(kernel=None, order=None, key="dram_bytes_per_launch"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources, on this kernel and in this order of the
    work items (hs_launch.order), else None.  key: the live figure (caches
    as the previous pass left them) or cold_dram_bytes_per_launch."""
    try:
        kv = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("sources_sha") != kernels_sha():
            return None
        if kernel is not None and kv.get("kernel", "") != kernel and not kv.get("kernel", "").startswith(kernel + "<"):
            return None
        if order is not None and kv.get("order") != ORDERS.get(order):
            return None
        return float(kv[key])
    except (OSError, KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.strip().splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(local_attempts: float, local_seconds: float, world: int, device=None):
    """Whole-job throughput: attempts of all ranks / slowest rank's time."""
    if world == 1:
        return local_attempts, local_seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_attempts, local_seconds], dtype=torch.float64, device=device)
    a = t[0:1].clone()
    s = t[1:2].clone()
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(a.item()), float(s.item())


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import numpy as np
    import torch

    from paper_2106_11286_gb300 import hs

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        import datetime
        # between two collectives of this program the ranks work for seconds at most, so a rank whose peer
        # failed on its own (out of memory, say) gives up after minutes instead of the default ten
        dist.init_process_group("nccl", device_id=dev, timeout=datetime.timedelta(minutes=5))
    w = WORKLOAD
    L = w["L"]
    N = L ** 3
    beta = 1.0 / w["T"]
    stream = torch.cuda.Stream(device=dev)
    params = dict(J=w["J"], K=w["K"], e=w["e"], seed=w["seed"], replica=rank, stream=stream)

    def barrier_sync():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- headline: FP32, step = one sweep with fused reductions
    lat = hs.Lattice("sc", dims=(L, L, L), precision="fp32", **params)
    lat.init()
    lat.accumulate(True)
    # project autotuner (restores the chain); off for profiling runs, which
    # want a fixed launch sequence
    launch = lat.launch if args.no_autotune else lat.autotune(beta, 3)
    fold = lat.info.fold_sweeps
    lat.sweep(beta, args.warmup)
    lat.reset_accumulator()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    # args.repeats regions of exactly K steps each, every one bracketed by a
    # barrier and a device synchronisation; the headline is the median region
    region_ms = []
    with ClockSampler(local) as clk:
        for _ in range(args.repeats):
            barrier_sync()
            t0.record(stream)
            lat.sweep(beta, args.steps)
            t1.record(stream)
            barrier_sync()
            region_ms.append(t0.elapsed_time(t1))
    ms = statistics.median(region_ms)
    mom, count = lat.read_accumulator()
    # Mean launch duration of the dominant kernel from the CUDA events of the
    # timed region: it holds colour-pass launches of that kernel (2 per step)
    # and the ring folds of the fused sums (two small launches per fold_sweeps
    # steps), so region time / launches, inter-launch gaps included, bounds the
    # achieved bandwidth from below.  A second, identical run with
    # every launch bracketed by its own events is reported beside it (those
    # events delay each launch and break the overlap of consecutive passes).
    hs.hs_enable_timing(lat.h, True)
    lat.sweep(beta, args.steps)
    k_ms_br, k_launches = hs.hs_read_timing(lat.h)
    hs.hs_enable_timing(lat.h, False)
    meas = lat.measure()
    tot_attempts, tot_s = aggregate(float(N) * args.steps, ms / 1e3, world, dev)
    value = tot_attempts / (tot_s * 1e9)
    kernel_ms = ms / (2 * args.steps)
    kernel_ms_bracketed = k_ms_br / max(k_launches, 1)
    alg_bytes = 3 * BYTES_PER_SPIN["fp32"] * (N // 2)   # per launch: N/2 attempts x 3 s
    peaks, peak_kind = measured_peaks()
    achieved_gbs = alg_bytes / (kernel_ms * 1e-3) / 1e9
    kname = KERNEL_NAMES.get(launch["kernel"], "sc_pass_kernel") if launch else "sc_pass_kernel"
    zax = tuple(w["e"]) == (0.0, 0.0, 1.0)
    traffic = read_traffic(kernel_label(launch, zaxis=zax), launch.get("order")) if launch else None
    traffic_cold = (read_traffic(kernel_label(launch, zaxis=zax), launch.get("order"), "cold_dram_bytes_per_launch")
                    if launch else None)
    roofline = {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved_gbs / peaks["hbm_gbs"], 4), "traffic": traffic,
                "peak_source": f"{peak_kind} copy bandwidth", "kernel": kernel_label(launch, zaxis=zax) if launch else kname,
                "kernel_ms": round(kernel_ms, 5), "alg_bytes_per_launch": alg_bytes,
                "kernel_timing": "timed-region CUDA events / colour-pass launches (the region holds only them and "
                                 f"the ring folds of the fused sums, one per {fold} sweeps)",
                "kernel_ms_bracketed": round(kernel_ms_bracketed, 5),
                "regions_ms": [round(x, 4) for x in region_ms],
                "frac_of_8TBs_nominal": round(achieved_gbs / 8000.0, 4), "launch": launch,
                "traffic_what": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch with the caches as the "
                                "previous pass left them (--cache-control none), the timed steady state; "
                                "traffic_cold: the same launch from a flushed L2",
                "traffic_cold": traffic_cold}
    # the other bounds of the same launches: the acceptance-weighted minimum 2 s + a s per attempt (rejected
    # sites need no store) and the traffic measured by ncu
    acc_rate = meas["accept_rate"]
    s_fp32 = BYTES_PER_SPIN["fp32"]
    min_bytes = (2 * s_fp32 + acc_rate * s_fp32) * (N // 2)
    roofline["alg_bytes_per_launch_acceptance_weighted"] = int(min_bytes)
    roofline["frac_acceptance_weighted"] = round(min_bytes / (kernel_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)
    if traffic:
        roofline["frac_ncu_traffic"] = round(traffic / (kernel_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)
    physics = {"E_per_spin": mom[0] / count / N, "absM": mom[2] / count, "accept_rate": meas["accept_rate"],
               "sweeps_averaged": count}
    lat.close()

    # ---- plain FP64 form of the same workload
    fp64 = None
    if not args.no_fp64:
        lat64 = hs.Lattice("sc", dims=(L, L, L), precision="fp64", **params)
        lat64.init()
        lat64.accumulate(True)
        lat64.sweep(beta, 3)
        barrier_sync()
        t0.record(stream)
        lat64.sweep(beta, args.fp64_steps)
        t1.record(stream)
        barrier_sync()
        ms64 = t0.elapsed_time(t1)
        a64, s64 = aggregate(float(N) * args.fp64_steps, ms64 / 1e3, world, dev)
        km64 = ms64 / (2 * args.fp64_steps)  # the region holds colour-pass launches and the ring folds
        gbs64 = 3 * BYTES_PER_SPIN["fp64"] * (N // 2) / (km64 * 1e-3) / 1e9
        v64 = a64 / (s64 * 1e9)
        fp64 = {"value": round(v64, 4), "unit": UNIT, "steps": args.fp64_steps,
                "ms_per_step": round(ms64 / args.fp64_steps, 4), "kernel_ms": round(km64, 4),
                "hbm_GBs": round(gbs64, 1), "hbm_frac": round(gbs64 / peaks["hbm_gbs"], 4),
                "launch": lat64.launch}
        fp64.update(fp64_roofline(v64, stream, kernel_label(lat64.launch, precision_code=0)))
        lat64.close()

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = e2e_pipelined(args, w, params, L, N, beta, world, dev, barrier_sync)
        e2e["serial_fp64"] = e2e_serial(args, w, params, L, N, beta, world, dev, barrier_sync)

    variants = None if args.no_variants else run_variants(args, rank, stream, barrier_sync, world, dev)
    if variants is not None:
        variants["noalloc"] = noalloc_run(args, stream)
        try:
            strong = slab_strong_run(args, rank, world, stream, barrier_sync, overlap=False)
            strong["overlap_value"] = slab_strong_run(args, rank, world, stream, barrier_sync, overlap=True)["value"]
            variants["slab_strong"] = strong
        except Exception as ex:  # the replica figure above stands on its own
            variants["slab_strong"] = {"error": repr(ex)[:300]}

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if rank != 0:
        return None
    # kernels launched in one timed region: two colour passes per sweep and the ring folds of the fused
    # sums (a per-sweep sum kernel and an apply kernel per fold_sweeps sweeps)
    gpu_launches = 2 * args.steps + 2 * ((args.steps + fold - 1) // fold)
    cpu, spin_err = (None, None) if (args.no_cpu_baseline or world > 1) else cpu_baseline(args)
    precision = None if (args.no_precision or world > 1) else precision_runs(args)
    tc = None if (args.no_precision or world > 1) else tc_runs(args)
    config1 = None if (args.no_precision or world > 1) else config1_run(args)
    beta_exp = None if (args.no_beta or world > 1) else beta_runs(args)
    # the compact summaries come last, so the tail of the line shows them
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(tot_s * 1e3 / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(args, world), "gpu_launches": gpu_launches, "clocks": clk.summary(),
            "variants": variants, "e2e": e2e, "cpu_baseline": cpu, "physics": physics, "fp64": fp64,
            "tc": tc, "beta_exponent": beta_exp, "config1_sc16_fp64": config1, "precision": precision,
            "spin_error_per_sweep": spin_err, "roofline": roofline}
    return line


# ------------------------------------------------------------------ other forms of the metric
BATCH_SIZES = (16, 24, 32, 48, 64, 96)
# M(T) scan of the critical exponent: temperatures (J = 1, k_B = 1) and the highest one in the power-law fit
BETA_TEMPS = (1.20, 1.25, 1.30, 1.34, 1.37, 1.40, 1.42, 1.43, 1.44, 1.45, 1.46)
BETA_FIT_TMAX = 1.40


def _timed(stream, fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def run_variants(args, rank, stream, barrier_sync, world, dev):
    """The batched form, the 464^3 precision ladder and the bcc nanoparticle,
    each timed on the device (attempts/ns), with its physics beside it."""
    from paper_2106_11286_gb300 import hs, inputs
    out = {}
    peaks, _ = measured_peaks()
    # (1) batched: 64 sc replicas, L = sizes[r mod 6], T_r = 1.30 + 0.30 r / 63, K = 0,
    #     2000 sweeps (1000 equilibration + 1000 measured) in one persistent launch
    lats = [hs.Lattice("sc", dims=(BATCH_SIZES[r % 6],) * 3, J=1.0, K=0.0, precision="fp32", seed=4,
                       replica=64 * rank + r, stream=stream) for r in range(64)]
    betas = [1.0 / (1.30 + 0.30 * r / 63) for r in range(64)]
    for m in lats:
        m.init()
    batch = hs.hs_batch_create([m.h for m in lats])
    # the project autotuner picks the batch's work split (restores every member)
    layout = hs.hs_batch_get_layout(batch) if args.no_autotune else hs.hs_batch_autotune(batch, betas, 5)
    hs.hs_batch_run(batch, betas, 5, 5)  # warm-up (captures a graph for these counts)
    for m in lats:
        m.reset_accumulator()
    n_spins = sum(BATCH_SIZES[r % 6] ** 3 for r in range(64))
    sec = _timed(stream, lambda: hs.hs_batch_run(batch, betas, args.batch_sweeps // 2, args.batch_sweeps // 2))
    u4 = {}
    for r, m in enumerate(lats):
        mom, cnt = m.read_accumulator()
        L = BATCH_SIZES[r % 6]
        u4.setdefault(L, []).append((round(1.0 / betas[r], 4), round(1 - (mom[4] / cnt) / (3 * (mom[3] / cnt) ** 2), 4)))
    hs.hs_batch_destroy(batch)
    for m in lats:
        m.close()
    out["batched"] = {"value": round(n_spins * args.batch_sweeps / (sec * 1e9), 3), "unit": UNIT,
                      "replicas": 64, "n_spins_total": n_spins, "sweeps": args.batch_sweeps, "layout": layout,
                      "hbm_frac": round(n_spins * args.batch_sweeps * 36 / sec / 1e9 / peaks["hbm_gbs"], 4),
                      "what": "one persistent cooperative kernel (CUDA graph), FP32 spins, FP64 moments",
                      "binder_u4": {str(L): v for L, v in u4.items()}}
    # (1b) the same 64 replicas as FP64 and as FP16 batches (the FP32 batch against plain FP64 in one form),
    #      their default layout, fewer sweeps for FP64 (bound by the FP64 pipe)
    per_prec = {}
    for prec, sweeps in (("fp64", max(2, args.batch_sweeps // 20)), ("fp16", args.batch_sweeps // 2)):
        lats = [hs.Lattice("sc", dims=(BATCH_SIZES[r % 6],) * 3, J=1.0, K=0.0, precision=prec, seed=4,
                           replica=64 * rank + r, stream=stream) for r in range(64)]
        for m in lats:
            m.init()
        batch = hs.hs_batch_create([m.h for m in lats])
        hs.hs_batch_run(batch, betas, 2, 2)
        sec = _timed(stream, lambda: hs.hs_batch_run(batch, betas, sweeps, 0))
        per_prec[prec] = {"value": round(n_spins * sweeps / (sec * 1e9), 3), "sweeps": sweeps,
                          "layout": hs.hs_batch_get_layout(batch),
                          "hbm_frac": round(n_spins * sweeps * 3 * BYTES_PER_SPIN[prec] / sec / 1e9 / peaks["hbm_gbs"], 4)}
        hs.hs_batch_destroy(batch)
        for m in lats:
            m.close()
    out["batched"]["precisions"] = per_prec
    # (1c) many small lattices: 304 replicas of 16^3 (K = 0, T 1.30 ... 1.60), the resident schedule (the default
    #      for 16 or more members that fit a CTA's shared memory) against the persistent one
    lats = [hs.Lattice("sc", dims=(16,) * 3, J=1.0, K=0.0, precision="fp32", seed=8, replica=304 * rank + r,
                       stream=stream) for r in range(304)]
    betas16 = [1.0 / (1.30 + 0.30 * r / 303) for r in range(304)]
    for m in lats:
        m.init()
    batch = hs.hs_batch_create([m.h for m in lats])
    small = {"replicas": 304, "n_spins_total": 304 * 16 ** 3, "sweeps": args.batch_sweeps // 4}
    for name, sched in (("resident", 2), ("persistent", 0)):
        hs.hs_batch_set_layout(batch, 2, 2, 0, sched)
        hs.hs_batch_run(batch, betas16, 2, 2)
        sec = _timed(stream, lambda: hs.hs_batch_run(batch, betas16, small["sweeps"], 0))
        small[name] = round(small["n_spins_total"] * small["sweeps"] / (sec * 1e9), 3)
    small["value"] = small["resident"]
    small["unit"] = UNIT
    small["what"] = ("one CTA per replica, its 48 KB of FP32 planes in shared memory for every sweep (batch "
                     "schedule 2); persistent: the streaming kernel with a grid barrier per colour pass")
    hs.hs_batch_destroy(batch)
    for m in lats:
        m.close()
    out["batched_small"] = small
    # (2) sc 464^3, K = 0.1, T = 1.0, 200 sweeps: FP16 vs FP32 vs FP64 (bias against FP64)
    L5 = 464
    N5 = L5 ** 3
    ladder = {}
    for prec, sweeps in (("fp16", args.big_sweeps), ("fp32", args.big_sweeps), ("fp64", args.big_sweeps)):
        lat = hs.Lattice("sc", dims=(L5,) * 3, J=1.0, K=0.1, e=(0, 0, 1), precision=prec, seed=5, replica=rank,
                         stream=stream)
        lat.init()
        lat.accumulate(True)
        lat.sweep(1.0, 10)  # tune on a state past the random start (the acceptance rate, and with it the
        #                    store traffic, falls as the lattice orders)
        launch = lat.launch if args.no_autotune else lat.autotune(1.0, 2)
        lat.sweep(1.0, 3)
        lat.reset_accumulator()
        sec = _timed(stream, lambda: lat.sweep(1.0, sweeps))
        mom, cnt = lat.read_accumulator()
        ladder[prec] = {"value": round(N5 * sweeps / (sec * 1e9), 3), "unit": UNIT, "sweeps": sweeps,
                        "hbm_frac": round(3 * BYTES_PER_SPIN[prec] * N5 * sweeps / sec / 1e9 / peaks["hbm_gbs"], 4),
                        "E_per_spin": mom[0] / cnt / N5, "absM": mom[2] / cnt,
                        "kernel": KERNEL_NAMES.get(launch["kernel"], "?"), "launch": launch}
        lat.close()
    ladder["note"] = "one seed each; the bias against FP64 with errors over seeds is under precision.sc464"
    out["sc464"] = ladder
    # (2b) beyond 10^8 spins on one GPU: sc 1024^3 (1,073,741,824 spins, 12.9 GB of FP32 state),
    #      the headline's parameters, autotuned launch
    if not args.no_big:
        L6 = 1024
        N6 = L6 ** 3
        lat = hs.Lattice("sc", dims=(L6,) * 3, J=WORKLOAD["J"], K=WORKLOAD["K"], e=WORKLOAD["e"], precision="fp32",
                         seed=6, replica=rank, stream=stream)
        beta6 = 1.0 / WORKLOAD["T"]
        lat.init()
        lat.accumulate(True)
        launch = lat.launch if args.no_autotune else lat.autotune(beta6, 2)
        lat.sweep(beta6, 3)
        lat.reset_accumulator()
        sec = _timed(stream, lambda: lat.sweep(beta6, args.huge_sweeps))
        mom, cnt = lat.read_accumulator()
        out["sc1024"] = {"value": round(N6 * args.huge_sweeps / (sec * 1e9), 3), "unit": UNIT, "n_spins": N6,
                         "sweeps": args.huge_sweeps, "device_bytes": 3 * 2 * (N6 // 2) * 4,
                         "hbm_frac": round(3 * BYTES_PER_SPIN["fp32"] * N6 * args.huge_sweeps / sec / 1e9 /
                                           peaks["hbm_gbs"], 4),
                         "E_per_spin": mom[0] / cnt / N6, "absM": mom[2] / cnt, "launch": launch}
        lat.close()
    # (2c) sc 2048^3 FP32 (8,589,934,592 spins, 103 GB of state): beyond 2^31 sites, register stencil
    if not args.no_big:
        L7 = 2048
        N7 = L7 ** 3
        lat = hs.Lattice("sc", dims=(L7,) * 3, J=WORKLOAD["J"], K=WORKLOAD["K"], e=WORKLOAD["e"], precision="fp32",
                         seed=7, replica=rank, stream=stream)
        beta7 = 1.0 / WORKLOAD["T"]
        lat.init()
        lat.accumulate(True)
        lat.sweep(beta7, 2)
        lat.reset_accumulator()
        sweeps7 = max(2, args.huge_sweeps // 4)
        sec = _timed(stream, lambda: lat.sweep(beta7, sweeps7))
        mom, cnt = lat.read_accumulator()
        out["sc2048"] = {"value": round(N7 * sweeps7 / (sec * 1e9), 3), "unit": UNIT, "n_spins": N7,
                         "sweeps": sweeps7, "device_bytes": 3 * 2 * (N7 // 2) * 4,
                         "hbm_frac": round(3 * BYTES_PER_SPIN["fp32"] * N7 * sweeps7 / sec / 1e9 /
                                           peaks["hbm_gbs"], 4),
                         "E_per_spin": mom[0] / cnt / N7, "absM": mom[2] / cnt, "launch": lat.launch}
        lat.close()
    # (3) bcc nanoparticle: radius 110 in a 232^3-cell box, open surface, 1 % vacancies (seed 3),
    #     CSR neighbour list, K = 0.2 along (1,1,1), T = 0.9, FP32
    if not args.no_csr:
        rp, col, mask = inputs.bcc_nanoparticle(radius=110, box=232, vacancy_fraction=0.01, seed=3)
        lat = hs.Lattice("csr", row_ptr=rp, col_idx=col, site_mask=mask, J=1.0, K=0.2, e=(1, 1, 1),
                         precision="fp32", seed=3, replica=rank, stream=stream)
        n_present = lat.info.n_present
        del rp, col
        lat.init()
        lat.accumulate(True)
        launch = lat.launch if args.no_autotune else lat.autotune(1 / 0.9, 10)
        lat.sweep(1 / 0.9, 3)
        lat.reset_accumulator()
        sec = _timed(stream, lambda: lat.sweep(1 / 0.9, args.csr_sweeps))
        mom, cnt = lat.read_accumulator()
        # algorithmic bytes per attempt: 3 s with s = 12 B of FP32 spin, plus z = 8 int32 neighbour
        # indices and the row's 4-byte offset (the FP32 path keys Philox by colour rank)
        per_attempt = 3 * BYTES_PER_SPIN["fp32"] + 8 * 4 + 4
        v = n_present * args.csr_sweeps / (sec * 1e9)
        out["bcc_nanoparticle"] = {"value": round(v, 3), "unit": UNIT,
                                   "n_spins": n_present, "colours": lat.info.n_colours, "sweeps": args.csr_sweeps,
                                   "alg_bytes_per_attempt": per_attempt,
                                   "hbm_frac": round(per_attempt * v / peaks["hbm_gbs"], 4),
                                   "layout_bytes_per_attempt": TABLE_LAYOUT_BYTES,
                                   "hbm_frac_layout_bytes": round(TABLE_LAYOUT_BYTES * v / peaks["hbm_gbs"], 4),
                                   "E_per_spin": mom[0] / cnt / n_present, "absM": mom[2] / cnt,
                                   "launch": launch}
        lat.close()
    return out


# ------------------------------------------------------------------ FP64 roofline
FP64_OPS_FILE = os.path.join(ROOT, "profiles", "sc_pass_fp64_sc256_ops.txt")


def read_fp64_ops(kernel=None):
    """FP64 pipe instructions per attempt of the FP64 colour-pass kernel, from
    the committed ncu instruction counts, if they were taken on the current
    kernel sources and on this kernel (template label); else None.  inst:
    DADD + DMUL + DFMA (each one issue slot of the FP64 pipe); pipe_inst:
    every instruction the FP64 pipe executed (the arithmetic plus the
    conversions and comparisons it also runs), when recorded."""
    try:
        kv = {}
        for line in open(FP64_OPS_FILE):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("sources_sha") != kernels_sha():
            return None
        if kernel is not None and kv.get("kernel", "") != kernel:
            return None
        out = {"inst": float(kv["fp64_inst_per_attempt"]), "flop": float(kv["fp64_flop_per_attempt"]),
               "kernel": kv.get("kernel", "")}
        if "fp64_pipe_inst_per_attempt" in kv:
            out["pipe_inst"] = float(kv["fp64_pipe_inst_per_attempt"])
        return out
    except (OSError, KeyError, ValueError):
        return None


def fp64_roofline(value, stream, kernel=None):
    """The FP64 path against the FP64 pipe.  hs_measure_alu_peak times DFMA
    chains on every SM in the same run; one DFMA is one FP64 pipe
    instruction, so peak instructions/s = measured FLOP/s / 2.  With the
    kernel's FP64 instructions per attempt (ncu counts of DADD + DMUL + DFMA)
    that bounds the attempts/ns; frac = achieved FP64 instructions/s over
    that peak.  frac_pipe counts every instruction of the FP64 pipe instead
    (the conversions and comparisons as well)."""
    from paper_2106_11286_gb300 import hs
    peak = max(hs.hs_measure_alu_peak(hs.ALU_FP64, stream) for _ in range(3))
    out = {"fp64_peak_tflops_measured": round(peak / 1e12, 4)}
    ops = read_fp64_ops(kernel)
    if ops:
        peak_inst = peak / 2.0
        achieved = value * 1e9 * ops["inst"]
        out.update({"bound": "alu", "unit": "FP64 inst/s", "fp64_inst_per_attempt": ops["inst"],
                    "fp64_flop_per_attempt": ops["flop"], "achieved": round(achieved / 1e12, 4),
                    "peak": round(peak_inst / 1e12, 4), "frac": round(achieved / peak_inst, 4),
                    "alu_bound_attempts_per_ns": round(peak_inst / ops["inst"] / 1e9, 3),
                    "peak_source": "measured DFMA chains (hs_measure_alu_peak), 1 instruction = 2 FLOP",
                    "kernel": ops["kernel"]})
        if "pipe_inst" in ops:
            out.update({"fp64_pipe_inst_per_attempt": ops["pipe_inst"],
                        "frac_pipe": round(value * 1e9 * ops["pipe_inst"] / peak_inst, 4)})
    return out


def noalloc_run(args, stream):
    """The allocation-free entry point on the headline workload (sc 256^3
    FP32, caller-held planes, static reduction scratch): attempts/ns of
    args.steps sweeps in one call, beside the handle path's."""
    import torch

    from paper_2106_11286_gb300 import hs
    w = WORKLOAD
    L = w["L"]
    dims = (L, L, L)
    planes = torch.empty(6 * L * L * (L // 2), dtype=torch.float32, device="cuda")
    with hs.Lattice("sc", dims=dims, precision="fp32", seed=w["seed"], J=w["J"], K=w["K"], e=w["e"],
                    stream=stream) as lat:
        lat.init()
        S = lat.get_spins()
    # the stencil layout: planes [colour][xyz][z][y][x/2], colour (x + y + z) & 1
    St = torch.from_numpy(S.reshape(L, L, L, 3)).to("cuda", torch.float32)
    z, y, x = torch.meshgrid(torch.arange(L, device="cuda"), torch.arange(L, device="cuda"),
                             torch.arange(L, device="cuda"), indexing="ij")
    col = (x + y + z) & 1
    P = planes.view(2, 3, L, L, L // 2)
    for c in (0, 1):
        m = col == c
        for q in range(3):
            P[c, q][z[m], y[m], x[m] // 2] = St[..., q][m]
    out = torch.zeros(hs.HS_N_MOMENTS + 2, dtype=torch.float64, device="cuda")
    beta = 1.0 / w["T"]
    kw = dict(J=w["J"], K=w["K"], e=w["e"], seed=w["seed"], stream=stream)
    hs.hs_sweep_sc_fp32_noalloc(planes, dims, beta, args.warmup, out, first_sweep=0, **kw)
    sec = _timed(stream, lambda: hs.hs_sweep_sc_fp32_noalloc(planes, dims, beta, args.steps, out,
                                                              first_sweep=args.warmup, **kw))
    del St, z, y, x, col
    return {"value": round(L ** 3 * args.steps / (sec * 1e9), 3), "unit": UNIT, "sweeps": args.steps,
            "what": "hs_sweep_sc_fp32_noalloc on the headline workload: register stencil, no prefetch, alternating "
                    "order, reductions finished by the last-arriving CTA of each sweep in static scratch"}


def slab_strong_run(args, rank, world, stream, barrier_sync, overlap=True):
    """One sc 1024^3 FP32 lattice split into z-slabs, one per rank, halos
    exchanged with NCCL after every colour pass (shards.DistributedSlab):
    strong scaling of one lattice, beside the replica figure.  overlap: the
    boundary planes first, their exchange on a communication stream beside
    the interior update (one rank: the slab's own halo copies)."""
    from paper_2106_11286_gb300 import shards
    L = 1024
    w = WORKLOAD
    ds = shards.DistributedSlab((L, L, L), J=w["J"], K=w["K"], e=w["e"], precision="fp32", seed=6,
                                stream=stream, overlap=overlap)
    try:
        ds.init()
        beta = 1.0 / w["T"]
        ds.sweep(beta, 3)
        barrier_sync()
        t = time.perf_counter()
        ds.sweep(beta, args.huge_sweeps)
        barrier_sync()
        sec = time.perf_counter() - t
        import torch
        _, s_max = aggregate(0.0, sec, world, torch.device("cuda", torch.cuda.current_device()))
    finally:
        ds.close()
    return {"value": round(float(L) ** 3 * args.huge_sweeps / (s_max * 1e9), 3), "unit": UNIT, "ranks": world,
            "n_spins": L ** 3, "sweeps": args.huge_sweeps, "scaling": "strong", "overlap": overlap,
            "what": "one sc 1024^3 FP32 lattice in z-slabs, packed halo planes by stream-ordered NCCL "
                    "send/recv after every colour pass" + (", boundary planes first, the exchange beside the "
                                                           "interior update" if overlap else "") +
                    "; wall clock over the slowest rank (overlap_value: boundary planes first, the exchange "
                    "beside the interior update)"}


# ------------------------------------------------------------------ CPU oracle
def _one_sweep_gpu(precision, L, params, beta):
    """Storage-rounded start state and the state after one GPU sweep."""
    from paper_2106_11286_gb300 import hs
    with hs.Lattice("sc", dims=(L, L, L), precision=precision, **params) as lat:
        lat.init()
        S0 = lat.get_spins()
        lat.sweep(beta, 1)
        return S0, lat.get_spins()


def _spin_error(S0, G, O):
    """One sweep from S0 on the GPU (G) and in the oracle (O): the fraction of
    sites whose accept decision differs, and |G - O| over the sites where both
    took the same decision (accepted: trial rounding; rejected: exactly 0)."""
    import numpy as np
    acc_g = np.any(G != S0, axis=1)
    acc_o = np.any(O != S0, axis=1)
    same = acc_g == acc_o
    d = np.linalg.norm(G[same] - O[same], axis=1)
    return {"decision_mismatch_frac": float((~same).mean()), "err_max": float(d.max()),
            "err_rms": float(np.sqrt((d * d).mean())), "accept_rate": float(acc_o.mean())}


def host_cores() -> int:
    """Host cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(args, sweeps=None, L=None):
    """The oracle as it stands on a bounded sample of the workload (sweeps of
    the full 256^3 lattice, started from the FP32 path's own rounded initial
    state): once on one thread and once with each colour class shared among
    every host core (the oracle's OpenMP sweep, bit-identical to the serial
    one).  The all-core figure is the baseline value.  The same leg measures
    the spin error per sweep of each GPU precision against the FP64 oracle:
    one sweep of the full lattice from the same state in both (the FP32 and
    FP16 paths against the oracle run with their random-number schedule and
    storage rounding)."""
    import numpy as np

    from oracle import oracle as orc
    w = WORKLOAD
    L = L or w["L"]
    sweeps = sweeps or args.cpu_sweeps
    beta = 1.0 / w["T"]
    params = dict(J=w["J"], K=w["K"], e=w["e"], seed=w["seed"])
    g = orc.lattice("sc", (L, L, L))
    starts = {p: _one_sweep_gpu(p, L, params, beta) for p in ("fp32", "fp16", "fp64")}
    cores = host_cores()
    kw = dict(J=w["J"], K=w["K"], e=w["e"], beta=beta, seed=w["seed"], mode=orc.MODE_FP32)
    S1 = starts["fp32"][0].copy()
    t = time.perf_counter()
    for s in range(sweeps):
        orc.sweep(g, S1, sweep_index=s, **kw)
        if s == 0:
            after_one = S1.copy()
    dt1 = time.perf_counter() - t
    par_sweeps = max(sweeps, args.cpu_parallel_sweeps)
    Sp = starts["fp32"][0].copy()
    t = time.perf_counter()
    for s in range(par_sweeps):
        orc.sweep_parallel(g, Sp, sweep_index=s, threads=cores, **kw)
        if s == sweeps - 1:
            same = bool(np.array_equal(Sp, S1))
    dtp = time.perf_counter() - t
    n1, npar = g.n * sweeps, g.n * par_sweeps
    out = {"value": round(npar / (dtp * 1e9), 6), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{par_sweeps} sweeps of the sc {L}^3 lattice ({npar} attempts), FP64 oracle with the FP32 "
                     f"random-number schedule, each colour class shared among {cores} OpenMP threads, {dtp:.1f} s",
           "nproc": os.cpu_count(), "bit_identical_to_serial": same,
           "single_thread": {"value": round(n1 / (dt1 * 1e9), 6), "cores": 1,
                             "sample": f"{sweeps} sweeps of the same lattice ({n1} attempts), {dt1:.1f} s"}}
    errors = {"fp32": _spin_error(starts["fp32"][0], starts["fp32"][1], after_one)}
    for prec, mode in (("fp16", orc.MODE_FP16), ("fp64", orc.MODE_FP64)):
        S0, G = starts[prec]
        O = S0.copy()
        orc.sweep_parallel(g, O, J=w["J"], K=w["K"], e=w["e"], beta=beta, seed=w["seed"], sweep_index=0, mode=mode,
                           threads=cores)
        errors[prec] = _spin_error(S0, G, O)
    errors["what"] = (f"one sweep of the sc {L}^3 workload from the same state on the GPU and in the FP64 oracle "
                      "(FP32 / FP16: the oracle with that path's random-number schedule and storage rounding)")
    return out, errors


def tc_runs(args):
    """T_c of each precision path from the Binder-cumulant crossing of sc
    L = 8 and 16 (K = 0, T = 1.38 .. 1.50, 6 replicas, 2000 + 8 x 1000
    sweeps), with jackknife errors: FP32 batched, FP64 and FP16 lattice by
    lattice."""
    from paper_2106_11286_gb300 import scan
    out = {}
    for prec in ("fp64", "fp32", "fp16"):
        sc = scan.run_scan((8, 16), (1.38, 1.42, 1.46, 1.50), n_equil=2000, n_blocks=8, block_sweeps=1000,
                           replicas=6, precision=prec, seed=91)
        tc, err = scan.binder_crossing(sc, 0, 1)
        out[prec] = {"tc": round(tc, 5), "err": round(err, 5)}
    for prec in ("fp32", "fp16"):
        out[prec]["diff_vs_fp64_sigma"] = round((out[prec]["tc"] - out["fp64"]["tc"]) /
                                                (out[prec]["err"] ** 2 + out["fp64"]["err"] ** 2) ** 0.5, 2)
    out["what"] = "Binder-cumulant crossing of sc L = 8 and 16, K = 0; literature T_c = 1.443 J"
    return out


def _seeded_means(L, K, T, sweeps, precision, seeds, n_equil=0):
    """<E>/N and <|M|> of an sc L^3 lattice (J = 1, e = z) over `sweeps`
    measured sweeps after n_equil unmeasured ones, one independent chain per
    seed from its own random start; returns the per-seed means."""
    from paper_2106_11286_gb300 import hs
    E, M, Mz = [], [], []
    for seed in seeds:
        with hs.Lattice("sc", dims=(L, L, L), J=1.0, K=K, e=(0.0, 0.0, 1.0), precision=precision, seed=seed) as lat:
            lat.init()
            if n_equil:
                lat.sweep(1.0 / T, n_equil)
            lat.accumulate(True)
            lat.sweep(1.0 / T, sweeps)
            mom, count = lat.read_accumulator()
        E.append(mom[hs.MOMENTS.index("sum_E")] / count / float(L) ** 3)
        M.append(mom[hs.MOMENTS.index("sum_absM")] / count)
        Mz.append(mom[hs.MOMENTS.index("sum_absMe")] / count)
    return E, M, Mz


def _mean_err(x):
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    return float(x.mean()), float(x.std(ddof=1) / np.sqrt(len(x))) if len(x) > 1 else float("nan")


def _compare(per_prec):
    """Means with their standard errors over seeds, and each reduced
    precision's difference from FP64 in units of the combined error."""
    out = {}
    for prec, (E, M) in per_prec.items():
        e, de = _mean_err(E)
        m, dm = _mean_err(M)
        out[prec] = {"E_per_spin": e, "E_err": de, "absM": m, "absM_err": dm}
    for prec in out:
        if prec == "fp64":
            continue
        r, f = out[prec], out["fp64"]
        r["E_diff_sigma"] = round((r["E_per_spin"] - f["E_per_spin"]) / (r["E_err"] ** 2 + f["E_err"] ** 2) ** 0.5, 2)
        r["absM_diff_sigma"] = round((r["absM"] - f["absM"]) / (r["absM_err"] ** 2 + f["absM_err"] ** 2) ** 0.5, 2)
    return out


def precision_runs(args):
    """The precision comparison at the two workloads that state it, each path
    over the same independent seeds (the FP64 path is pinned to the oracle
    element by element in the tests):
      sc256: sc 256^3, K = 0.05, T = 1.2, 500 sweeps measured from the start;
      sc464: sc 464^3, K = 0.1, T = 1.0, 200 sweeps measured from the start.
    <E>/N and <|M|> per seed, their mean and standard error over seeds, and the
    FP32 / FP16 difference from FP64 in units of the combined error (the
    spec bar is |diff| < 3 sigma)."""
    seeds = [1000 + k for k in range(args.precision_seeds)]
    out = {}
    for name, L, K, T, sweeps in (("sc256", WORKLOAD["L"], WORKLOAD["K"], WORKLOAD["T"], args.precision_sweeps),
                                  ("sc464", 464, 0.1, 1.0, args.big_sweeps)):
        per = {}
        for prec in ("fp64", "fp32", "fp16"):
            E, M, _ = _seeded_means(L, K, T, sweeps, prec, seeds)
            per[prec] = (E, M)
        out[name] = _compare(per)
        out[name]["sweeps"] = sweeps
    out["seeds"] = len(seeds)
    out["what"] = "means over independent seeds (random starts, every sweep measured), errors = std / sqrt(seeds)"
    return out


def config1_run(args):
    """sc 16^3 periodic, J = 1, K = 0.1, e = z, T = 1.0, random start from
    seed 1, 1000 equilibration + 1000 measured sweeps, FP64: <E>/N, <|M|>,
    <M_z> and <|M_z|>, with the attempts/ns of the 2000 sweeps (CUDA events;
    a 4096-spin lattice is launch- and latency-bound, so no HBM fraction).
    The FP32 and FP16 paths over the same independent seeds give the 3-sigma
    comparison at this size."""
    import torch

    from paper_2106_11286_gb300 import hs
    L, K, T = 16, 0.1, 1.0
    N = L ** 3
    stream = torch.cuda.current_stream()
    with hs.Lattice("sc", dims=(L, L, L), J=1.0, K=K, e=(0.0, 0.0, 1.0), precision="fp64", seed=1) as lat:
        lat.init()
        launch = lat.autotune(1.0 / T, 20)   # restores the state and the sweep counter
        lat.sweep(1.0 / T, 5)
        lat.init()   # the chain below starts from the seed's random state again
        lat.set_sweep_counter(0)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        lat.sweep(1.0 / T, 1000)
        lat.accumulate(True)
        lat.sweep(1.0 / T, 1000)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        mom, cnt = lat.read_accumulator()
    out = {"E_per_spin": mom[hs.MOMENTS.index("sum_E")] / cnt / N, "absM": mom[hs.MOMENTS.index("sum_absM")] / cnt,
           "Mz": mom[hs.MOMENTS.index("sum_Mz")] / cnt, "absMz": mom[hs.MOMENTS.index("sum_absMe")] / cnt,
           "sweeps": [1000, 1000], "value": round(N * 2000 / (ms * 1e6), 4), "unit": UNIT,
           "ms": round(ms, 3), "launch": launch}
    seeds = list(range(1, 1 + args.precision_seeds))
    per = {}
    for prec in ("fp64", "fp32", "fp16"):
        E, M, _ = _seeded_means(L, K, T, 1000, prec, seeds, n_equil=1000)
        per[prec] = (E, M)
    out["precision"] = _compare(per)
    return out


def beta_runs(args):
    """The paper's M(T) curves and its critical exponent: sc 64^3 and 128^3
    (and 256^3 and 512^3 below T_c), K = 0.01 (the paper's anisotropy), ordered start,
    temperatures from 1.20 to just above T_c, all in one persistent FP32
    batch per call.  T_c comes from the Binder crossing of 64^3 and 128^3;
    beta from the paper's log-log fit of <|M|> on T_c - T over the points
    T <= 1.40, jackknife errors over blocks (T_c's error included)."""
    from paper_2106_11286_gb300 import scan
    temps = BETA_TEMPS
    fit_idx = [j for j, T in enumerate(temps) if T <= BETA_FIT_TMAX]
    t = time.perf_counter()
    sc = scan.run_scan((64, 128), temps, n_equil=args.beta_equil, n_blocks=args.beta_blocks,
                       block_sweeps=args.beta_block_sweeps, replicas=2, K=0.01, seed=77, init="aligned")
    tc, tc_err = scan.binder_crossing(sc, 0, 1)
    b128, e128, _ = scan.beta_fit(sc, 1, fit_idx, tc_sizes=(0, 1))
    p128, pe128, _ = scan.beta_fit(sc, 1, fit_idx, tc=1.445)
    out = {"tc": round(tc, 4), "tc_err": round(tc_err, 4), "tc_from": "Binder crossing of 64^3 and 128^3",
           "beta_128": round(b128, 4), "beta_128_err": round(e128, 4),
           "beta_128_at_paper_tc": round(p128, 4), "beta_128_at_paper_tc_err": round(pe128, 4)}
    curves = {"64": [round(float(sc.absM[(0, j)].mean()), 5) for j in range(len(temps))],
              "128": [round(float(sc.absM[(1, j)].mean()), 5) for j in range(len(temps))]}
    if not args.no_big:
        big = scan.run_scan((256,), [temps[j] for j in fit_idx], n_equil=args.beta_equil // 2,
                            n_blocks=max(4, args.beta_blocks // 2), block_sweeps=args.beta_block_sweeps, replicas=1,
                            K=0.01, seed=78, init="aligned")
        b256, e256, _ = scan.beta_fit(big, 0, range(len(fit_idx)), tc=tc)
        out.update({"beta_256_at_tc": round(b256, 4), "beta_256_stat_err": round(e256, 4)})
        curves["256"] = [round(float(big.absM[(0, j)].mean()), 5) for j in range(len(fit_idx))]
        # the paper's largest lattice: 512^3 (1.3 x 10^8 spins per temperature, 9.7 GB for the six)
        huge = scan.run_scan((512,), [temps[j] for j in fit_idx], n_equil=args.beta_equil // 3,
                             n_blocks=4, block_sweeps=args.beta_block_sweeps // 2, replicas=1, K=0.01, seed=79,
                             init="aligned")
        b512, e512, _ = scan.beta_fit(huge, 0, range(len(fit_idx)), tc=tc)
        out.update({"beta_512_at_tc": round(b512, 4), "beta_512_stat_err": round(e512, 4)})
        curves["512"] = [round(float(huge.absM[(0, j)].mean()), 5) for j in range(len(fit_idx))]
    out.update({"paper": {"beta": "0.364 +- 0.002", "tc": 1.445, "K": 0.01},
                "fit_temps": [temps[j] for j in fit_idx], "temps": list(temps), "absM": curves,
                "seconds": round(time.perf_counter() - t, 1),
                "what": "paper's log-log fit of <|M|> on T_c - T; K = 0.01, J = 1, e = z; 2 replicas of 64^3 and "
                        "128^3 per temperature, 1 of 256^3 and of 512^3 (fit at the crossing T_c, its error not "
                        "propagated)"})
    return out


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return None
    from oracle import oracle as orc
    w = WORKLOAD
    cores = host_cores()
    # bounded sample per step: the workload's lattice, or an even sub-lattice of it sized so all steps take
    # about a minute at ~150 ns per attempt and core
    total = max(args.steps + args.warmup, 1)
    L = int(round((4e8 * cores / total) ** (1 / 3)))
    L = max(8, min(w["L"], L - (L % 2)))
    g = orc.lattice("sc", (L, L, L))
    S = orc.init_spins(g, seed=w["seed"])

    def step(s):
        orc.sweep_parallel(g, S, J=w["J"], K=w["K"], e=w["e"], beta=1.0 / w["T"], seed=w["seed"], sweep_index=s,
                           mode=orc.MODE_FP32, threads=cores)
    for s in range(args.warmup):
        step(s)
    t = time.perf_counter()
    for s in range(args.steps):
        step(args.warmup + s)
    dt = time.perf_counter() - t
    n = g.n * args.steps
    value = n / (dt * 1e9)
    sample = (f"each step one oracle sweep of an sc {L}^3 " + ("lattice (the workload itself)" if L == w["L"] else
                                                               "sub-lattice of the workload") +
              f", each colour class shared among {cores} OpenMP threads")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / max(args.steps, 1), 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, world),
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "nproc": os.cpu_count()},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ single cases for ncu captures
CASES = {
    # name: (L, precision, K, T, seed)
    "sc256_fp32": (256, "fp32", 0.05, 1.2, 2),
    "sc256_fp64": (256, "fp64", 0.05, 1.2, 2),
    "sc464_fp16": (464, "fp16", 0.1, 1.0, 5),
    "sc464_fp32": (464, "fp32", 0.1, 1.0, 5),
}


# batch cases: name -> (replicas, L, precision, schedule); L None: the bench's 64-replica mix
# (L = BATCH_SIZES[r mod 6], K = 0)
BATCH_CASES = {"batch304x16_resident": (304, 16, "fp32", 2), "batch304x16_persistent": (304, 16, "fp32", 0),
               "batch64_mix": (64, None, "fp32", 0)}


def run_batch_case(args):
    """One batch of small replicas (K = 0, T 1.30 ... 1.60) in a fixed
    schedule: 2 + 2 warm-up sweeps, then one batch run of args.steps sweeps
    (one kernel launch in the resident schedule), for an ncu capture."""
    import torch

    from paper_2106_11286_gb300 import hs
    n, L, prec, sched = BATCH_CASES[args.case]
    sizes = [L if L else BATCH_SIZES[r % 6] for r in range(n)]
    lats = [hs.Lattice("sc", dims=(sizes[r],) * 3, J=1.0, K=0.0, precision=prec, seed=8, replica=r) for r in range(n)]
    try:
        betas = [1.0 / (1.30 + 0.30 * r / (n - 1)) for r in range(n)]
        for m in lats:
            m.init()
        batch = hs.hs_batch_create([m.h for m in lats])
        try:
            hs.hs_batch_set_layout(batch, 2, 2, 0, sched)
            hs.hs_batch_run(batch, betas, 2, 2)
            sec = _timed(torch.cuda.current_stream(), lambda: hs.hs_batch_run(batch, betas, args.steps, 0))
            layout = hs.hs_batch_get_layout(batch)
        finally:
            hs.hs_batch_destroy(batch)
    finally:
        for m in lats:
            m.close()
    return {"case": args.case, "layout": layout, "value": round(sum(x ** 3 for x in sizes) * args.steps / (sec * 1e9), 3),
            "unit": UNIT, "steps": args.steps}


def run_case(args):
    """One workload alone in its autotuned launch (tuned after 10 sweeps, as
    the bench's variants are), then args.steps sweeps: a fixed, short launch
    sequence for an ncu capture of its colour-pass kernel.  Prints the launch
    and the attempts/ns of the swept region."""
    import torch

    from paper_2106_11286_gb300 import hs
    if args.case in BATCH_CASES:
        return run_batch_case(args)
    L, prec, K, T, seed = CASES[args.case]
    with hs.Lattice("sc", dims=(L,) * 3, J=1.0, K=K, e=(0, 0, 1), precision=prec, seed=seed) as lat:
        lat.init()
        lat.accumulate(True)
        lat.sweep(1.0 / T, 10)
        if args.launch:
            f = [int(x) for x in args.launch.split(",")]
            kernel, vec, blocks = f[:3]
            prefetch, order = (f[3:] + [0, 0])[:2]
            lat.set_launch(kernel=kernel, vec_width=vec, blocks_per_sm=blocks, prefetch=prefetch, order=order)
            launch = lat.launch
        else:
            launch = lat.launch if args.no_autotune else lat.autotune(1.0 / T, 2)
        lat.sweep(1.0 / T, args.warmup)
        sec = _timed(torch.cuda.current_stream(), lambda: lat.sweep(1.0 / T, args.steps))
    return {"case": args.case, "launch": launch, "kernel": KERNEL_NAMES.get(launch["kernel"], "?"),
            "value": round(L ** 3 * args.steps / (sec * 1e9), 3), "unit": UNIT, "steps": args.steps}


def e2e_serial(args, w, params, L, N, beta, world, dev, barrier_sync):
    """Each step: hs_set_spins of the FP64 state from pinned host memory (synchronous), the sweeps, the
    moments read back; wall clock over the steps."""
    import numpy as np
    import torch

    from paper_2106_11286_gb300 import hs

    rng = np.random.default_rng(w["seed"])
    S0 = rng.standard_normal((N, 3))
    S0 /= np.linalg.norm(S0, axis=1, keepdims=True)
    host = torch.from_numpy(S0).pin_memory()
    lat = hs.Lattice("sc", dims=(L, L, L), precision="fp32", **params)
    lat.accumulate(True)
    mom_out = np.zeros(hs.HS_N_MOMENTS)
    cnt = hs.ctypes.c_int64(0)
    sweeps = args.e2e_sweeps

    def e2e_step():
        hs.load().hs_set_spins(lat.h, host.data_ptr())                 # H2D of the step's input state
        lat.reset_accumulator()
        lat.sweep(beta, sweeps)
        hs.load().hs_read_accumulator(lat.h, mom_out.ctypes.data_as(hs._dp), hs.ctypes.byref(cnt))  # D2H
    for _ in range(2):
        e2e_step()
    regions = []
    for _ in range(3):   # the median of three regions, as for the pipelined form
        barrier_sync()
        te = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        barrier_sync()
        regions.append(time.perf_counter() - te)
    se = statistics.median(regions)
    # the host-to-device part alone (copy + conversion into the planes), for the breakdown: median of 3
    h2d = []
    for _ in range(3):
        barrier_sync()
        th = time.perf_counter()
        hs.load().hs_set_spins(lat.h, host.data_ptr())
        barrier_sync()
        h2d.append((time.perf_counter() - th) * 1e3)
    h2d_ms = statistics.median(h2d)
    ea, es = aggregate(float(N) * sweeps * args.e2e_steps, se, world, dev)
    lat.close()
    return {"value": round(ea / (es * 1e9), 4), "unit": UNIT, "h2d_bytes_per_step": int(N * 3 * 8),
            "d2h_bytes_per_step": int(hs.HS_N_MOMENTS * 8 + 8), "sweeps_per_step": sweeps,
            "steps": args.e2e_steps, "ms_per_step": round(se * 1e3 / args.e2e_steps, 3),
            "set_spins_ms": round(h2d_ms, 3),
            "regions_ms": [round(r * 1e3, 3) for r in regions],
            "what": "hs_set_spins from pinned host FP64 state, hs_sweep x sweeps_per_step, "
                    "hs_read_accumulator to host; wall clock, median of three regions of `steps` steps"}


def e2e_pipelined(args, w, params, L, N, beta, world, dev, barrier_sync):
    """Each step takes its own FP32 input state from pinned host memory (two states used alternately) and
    returns its moments to the host.  Step k+1's upload (hs_set_spins_async) is queued while step k's
    sweeps run, so its copy overlaps them; the first step's copy is inside the timed region and
    overlaps nothing.  Wall clock over the steps."""
    import numpy as np
    import torch

    from paper_2106_11286_gb300 import hs

    hosts = []
    for k in range(2):
        rng = np.random.default_rng(w["seed"] + 100 * k)
        S0 = rng.standard_normal((N, 3))
        S0 /= np.linalg.norm(S0, axis=1, keepdims=True)
        hosts.append(torch.from_numpy(S0.astype(np.float32).reshape(-1)).pin_memory())
    lat = hs.Lattice("sc", dims=(L, L, L), precision="fp32", **params)
    lat.accumulate(True)
    mom_out = np.zeros(hs.HS_N_MOMENTS)
    cnt = hs.ctypes.c_int64(0)
    sweeps = args.e2e_sweeps
    lib = hs.load()

    def run(steps):
        hs._check(lib.hs_set_spins_async(lat.h, hosts[0].data_ptr(), hs.HS_FP32))      # H2D of step 0's input
        for k in range(steps):
            lat.reset_accumulator()
            lat.sweep(beta, sweeps)
            if k + 1 < steps:
                hs._check(lib.hs_set_spins_async(lat.h, hosts[(k + 1) % 2].data_ptr(), hs.HS_FP32))  # step k+1's
            lib.hs_read_accumulator(lat.h, mom_out.ctypes.data_as(hs._dp), hs.ctypes.byref(cnt))  # D2H
    run(2)
    regions = []
    for _ in range(3):   # the median of three regions, so that one host stall does not decide the figure
        barrier_sync()
        te = time.perf_counter()
        run(args.e2e_steps)
        barrier_sync()
        regions.append(time.perf_counter() - te)
    se = statistics.median(regions)
    h2d = []
    for _ in range(3):   # the upload alone, for the breakdown: median of 3
        barrier_sync()
        th = time.perf_counter()
        hs._check(lib.hs_set_spins_async(lat.h, hosts[0].data_ptr(), hs.HS_FP32))
        barrier_sync()   # a device-wide synchronisation: the copy stream and the conversion are done
        h2d.append((time.perf_counter() - th) * 1e3)
    h2d_ms = statistics.median(h2d)
    ea, es = aggregate(float(N) * sweeps * args.e2e_steps, se, world, dev)
    lat.close()
    return {"value": round(ea / (es * 1e9), 4), "unit": UNIT, "h2d_bytes_per_step": int(N * 3 * 4),
            "d2h_bytes_per_step": int(hs.HS_N_MOMENTS * 8 + 8), "sweeps_per_step": sweeps,
            "steps": args.e2e_steps, "ms_per_step": round(se * 1e3 / args.e2e_steps, 3),
            "set_spins_ms": round(h2d_ms, 3),
            "regions_ms": [round(r * 1e3, 3) for r in regions],
            "what": "hs_set_spins_async of each step's FP32 input state from pinned host memory (step k+1's "
                    "copy queued while step k's sweeps run), hs_sweep x sweeps_per_step, hs_read_accumulator "
                    "to host; wall clock, median of three regions of `steps` steps"}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=30)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--e2e-sweeps", type=int, default=100)
    ap.add_argument("--cpu-sweeps", type=int, default=3)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the FP64/FP32/FP16 runs of the workload and the T_c scans")
    ap.add_argument("--precision-sweeps", type=int, default=500)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-big", action="store_true", help="skip the sc 1024^3 variant")
    ap.add_argument("--huge-sweeps", type=int, default=20, help="timed sweeps of the sc 1024^3 variant")
    ap.add_argument("--no-csr", action="store_true")
    ap.add_argument("--batch-sweeps", type=int, default=2000)
    ap.add_argument("--big-sweeps", type=int, default=200)
    ap.add_argument("--csr-sweeps", type=int, default=500)
    ap.add_argument("--repeats", type=int, default=5, help="timed regions of K steps; the headline is their median")
    ap.add_argument("--precision-seeds", type=int, default=8)
    ap.add_argument("--cpu-parallel-sweeps", type=int, default=10)
    ap.add_argument("--no-beta", action="store_true", help="skip the M(T) scan and the fit of beta")
    ap.add_argument("--beta-equil", type=int, default=3000)
    ap.add_argument("--beta-blocks", type=int, default=10)
    ap.add_argument("--beta-block-sweeps", type=int, default=500)
    ap.add_argument("--case", choices=sorted(CASES) + sorted(BATCH_CASES), help="run one workload alone (for ncu captures)")
    ap.add_argument("--launch", help="with --case: fixed launch 'kernel,vec_width,blocks_per_sm[,prefetch[,order]]' "
                                     "(hs_launch codes), no autotuning")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.repeats < 1:
        ap.error("--repeats must be >= 1")
    if args.case:
        line = run_case(args)
    else:
        line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
