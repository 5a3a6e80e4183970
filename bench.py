"""Benchmark of the 2D-PT hot path on GB300.

Workload (default, --workload n200): a planted Wishart instance with N = 200
logical spins, alpha = 0.5, copy-chain sparsified to at most 3 original edges
per copy (13,400 physical spins), an I = 32 x J = 8 replica grid (geometric
beta 0.1..5.0 / scale, linear P 0.5..64 x 32767), 64 independent runs (16,384
replicas), swap interval 50.  One step = one swap event of Algorithm 1 for all
runs: 50 heat-bath sweeps of every replica, f and g of the final sweep, one
round of P- or beta-swaps and the bottom-right record.  The int8 spin state
(220 MB) is larger than L2, so no flush is needed between steps.
--workload n800: N = 800 (213,551 physical spins), I = 64 x J = 16, 16 runs
(3.5 GB of spins), same ladders and interval.
--workload batched / serving: the uneven batch and the request stream.
--workload constrained: 3-colouring of a random cubic graph with one-hot
constraints (general penalty terms), I = 16 x J = 8, 256 runs.
--workload membw: L2 and HBM read ceilings from the library's read probe.
--workload threecopy: the runtime-degree kernels on three copies per node.

Metric: spin updates per second (physical spins x replicas x sweeps / time).

Arms: the default arm times the CUDA library; --impl reference times the CPU
oracle (a plain restatement of the method, the only reference this project
has) on the host cores for a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "spin updates/sec and time-to-planted-ground-state (batched vs plain, same GB300)"
UNIT = "spin-updates/s"
WORKLOADS = {
    "n200": dict(N=200, alpha=0.5, inst_seed=2, I=32, J=8, runs=64, interval=50),
    "n800": dict(N=800, alpha=0.5, inst_seed=3, I=64, J=16, runs=16, interval=50),
}


def workload_name(key, n, runs=None):
    w = WORKLOADS[key]
    return (f"wishart-planted N={w['N']} alpha={w['alpha']}, <=3 edges/copy ({n} spins), "
            f"I={w['I']} x J={w['J']}, {runs or w['runs']} runs, swap every {w['interval']} sweeps")


# Algorithmic lane-operations of one spin update under the heat-bath contract,
# the minimal sequence with a quad of walkers sharing one Philox call: Philox
# share 10 (10 rounds x 2 wide multiplies + 2 three-input xors, / 4), field 11
# (3 couplings x (sign, multiply-add) + 2 links x (sign, add) + the P product),
# decision 8 (convert, scale, exp2, uniform 2, 1 + e, fused test, sign), state
# traffic 3 (neighbour and record loads, pack and store, per walker).
OPS_PER_UPDATE = 32.0
# Algorithmic DRAM bytes per update if the state made one round trip per sweep:
# one int8 read and one write, plus the neighbour record (5 x 8 B) over 128 walkers.
BYTES_PER_UPDATE = 2.0 + 40.0 / 128.0

# DRAM bytes per sweep launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum),
# valid only while the kernel sources hash to `src`; the summaries are under profiles/.
PROFILED_TRAFFIC = {
    ("n200", "k_sweep_smem"): dict(src="d9fe13f0f233316c", dram_bytes_per_launch=389_639_680,
                                   profile="profiles/k_sweep_smem_n200.md"),
    # captured at 4 of the 16 runs and scaled by the walkers
    ("n800", "k_sweep_bits8"): dict(src="d9fe13f0f233316c", dram_bytes_per_launch=14_168_667_136,
                                    profile="profiles/k_sweep_bits8_n800.md (4 runs x 4)"),
    ("constrained", "k_sweep_penalty_smem"): dict(src="abe90108dc60f7eb", dram_bytes_per_launch=342_726_144,
                                                  profile="profiles/k_sweep_penalty_smem_colouring.md"),
    # V = 40000 colouring: captured at 16 of the 64 runs and scaled by the walkers
    ("constrained", "k_sweep_penalty_bits8"): dict(src="abe90108dc60f7eb", dram_bytes_per_launch=5_691_546_624,
                                                   profile="profiles/k_sweep_penalty_bits8_colouring40k.md (16 runs x 4)"),
}
KERNEL_SOURCES = ("pt2d_kernels.cu", "pt2d_sweep.cuh", "pt2d_device.cuh", "pt2d_internal.h", "pt2d_wide.cuh")
# kernels defined outside pt2d_kernels.cu hash their own file as well
KERNEL_EXTRA_SOURCES = {"k_sweep_penalty_smem": ("pt2d_penalty.cu",), "k_sweep_penalty_bits": ("pt2d_penalty.cu",),
                        "k_sweep_penalty_bits8": ("pt2d_penalty.cu",)}


def kernel_source_hash(kernel=None):
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES + KERNEL_EXTRA_SOURCES.get(kernel, ()):
        with open(os.path.join(ROOT, "paper_2506_14781_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def sweep_kernel_name(tiling):
    """Name of the sweep kernel a context's tiling selects."""
    if tiling["kernel"] in ("bits", "penalty_bits") and tiling.get("walkers_per_thread") == 8:
        return "k_sweep_bits8" if tiling["kernel"] == "bits" else "k_sweep_penalty_bits8"
    return {"smem": "k_sweep_smem", "bits": "k_sweep_bits", "global": "k_sweep_global",
            "generic": "k_sweep_generic", "generic_smem": "k_sweep_generic_smem",
            "penalty_smem": "k_sweep_penalty_smem", "penalty_bits": "k_sweep_penalty_bits"}[tiling["kernel"]]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# Ladders of the larger workloads (the tiny configuration fixes beta 0.1..2.0 and
# P 0.5..4.0 x max|J|; the larger ones leave the ranges open).  P reaches 64 x
# max|J| so that the last column is feasible (the column criterion of the
# paper's adaptive schedule), beta reaches 5.
BETA_MIN, BETA_MAX, P_MIN, P_MAX = 0.1, 5.0, 0.5, 64.0
RHO_TARGETS = (0.2, 0.1, 0.05)


def make_workload(key="n200"):
    import synth

    w = WORKLOADS[key]
    inst = synth.wishart_planted(w["N"], w["alpha"], w["inst_seed"])
    beta = synth.beta_ladder(w["I"], BETA_MIN, BETA_MAX, inst.scale)
    P = synth.penalty_ladder(w["J"], P_MIN, P_MAX, 32767)
    return dict(inst=inst, beta=beta, P=P, runs=w["runs"], interval=w["interval"], I=w["I"], J=w["J"],
                key=key)


def residual_tts(trace_f, trace_g, events_done, E_planted, N, scale, interval):
    """Per run: sweeps until the bottom-right replica is feasible (g = 0) with
    residual energy per spin (f - E_planted) / (N s) <= rho, for each target rho
    (the residual energy of the paper's ground-state experiments), and until it
    is feasible at or below the planted energy.  -1 where not reached."""
    T = min(events_done, trace_f.shape[1])
    out = {}
    rho = (trace_f[:, :T] - E_planted) / (N * scale)
    feas = trace_g[:, :T] == 0
    for target in list(RHO_TARGETS) + [0.0]:
        hit = feas & (rho <= target)
        first = np.where(hit.any(1), hit.argmax(1) + 1, -1)
        out["planted" if target == 0.0 else f"rho<={target}"] = np.where(first > 0, first * interval, -1)
    return out


def tts_summary(per_target, sec_per_sweep):
    s = {}
    for k, v in per_target.items():
        ok = v >= 0
        s[k] = {"reached": int(ok.sum()), "runs": int(v.size),
                "median_sweeps": float(np.median(v[ok])) if ok.any() else None,
                "median_seconds": float(np.median(v[ok]) * sec_per_sweep) if ok.any() else None}
    return s


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(), f"pt2d_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus: int, backend: str | None = None):
    """One process per GPU under torchrun (RANK / WORLD_SIZE / MASTER_* from the
    environment).  NCCL when CUDA is present, gloo otherwise (the CPU tests of
    the multi-process path).  Returns (rank, world, torch.distributed or None)."""
    if n_gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch
    import torch.distributed as dist

    rank = int(os.environ["RANK"])
    world = int(os.environ["WORLD_SIZE"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend, init_method="env://")
    return rank, world, dist


def max_over_ranks(x: float, dist) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (runs are replicated per rank: weak scaling)."""
    return units_per_rank * world / max_seconds


def run_gpu(args):
    import torch

    import paper_2506_14781_gb300 as pt

    rank, world, dist = dist_setup(args.gpus)
    dev = torch.cuda.current_device()
    wl = make_workload(args.workload)
    if args.runs:  # smaller cases of the same kernel, for profiling captures
        wl["runs"] = args.runs
    inst, beta, P, runs, interval = wl["inst"], wl["beta"], wl["P"], wl["runs"], wl["interval"]
    phys = pt.sparsify(inst.Jq, "max_edges", 3)
    n = phys.n
    R = len(beta) * len(P)
    updates_per_step = n * R * runs * interval
    stream = torch.cuda.Stream()
    ctx = pt.PT2D(phys, beta, P, runs, stream=stream, workspace="torch", trace_capacity=4096,
                  profile=True)
    ctx.write(pt.TARGET, np.full(runs, inst.E_planted, np.int64))
    seed = 100 + rank
    with torch.cuda.stream(stream):
        ctx.run(interval * args.warmup, interval, seed)
    ctx.sync()
    ms0, launches0 = ctx.kernel_time(0)
    swap_ms0, _ = ctx.kernel_time(1)
    n_launch0 = ctx.launch_count
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        start.record(stream)
        ctx.run(interval * args.steps, interval, seed)
        end.record(stream)
        end.synchronize()
    torch.cuda.synchronize()
    elapsed_ms = start.elapsed_time(end)
    elapsed_ms = max_over_ranks(elapsed_ms, dist)
    if dist is not None:
        dist.barrier()
    sweep_ms, sweep_launches = ctx.kernel_time(0)
    swap_ms, _ = ctx.kernel_time(1)
    gpu_launches = ctx.launch_count - n_launch0
    sweep_ms -= ms0
    sweep_launches -= launches0
    swap_ms -= swap_ms0
    value = job_throughput(updates_per_step * args.steps, world, elapsed_ms / 1e3)
    # roofline of the sweep kernel
    peaks, peak_src = _peaks()
    avg_launch_ms = sweep_ms / max(sweep_launches, 1)
    updates_per_launch = n * R * runs * interval
    algo_bytes = updates_per_launch * BYTES_PER_UPDATE
    hbm_achieved = algo_bytes / (avg_launch_ms / 1e3) / 1e9
    ops_per_update = OPS_PER_UPDATE
    tiling = ctx.tiling
    kernel = sweep_kernel_name(tiling)
    prof = PROFILED_TRAFFIC.get((args.workload, kernel))
    src_hash = kernel_source_hash(kernel)
    traffic = prof["dram_bytes_per_launch"] if prof and prof["src"] == src_hash else None
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sm_count * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # Tops/s
    alu_achieved = updates_per_launch * ops_per_update / (avg_launch_ms / 1e3) / 1e12
    clocks = clk.summary()
    e2e = run_e2e(pt, phys, wl, args) if rank == 0 else None
    cpu = cpu_baseline(wl, args) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    # The metric's second half, measured outside the timed region on one GPU
    # (under torchrun the line carries the update rate only): (a) time to
    # target of these runs, continued; (b) the uneven batch, batched vs one
    # context per instance; (c) time to the planted ground state, batched vs
    # plain, on small instances where it is reached.
    legs = args.legs == "all" and world == 1 and args.workload == "n200"
    if legs:
        tts = leg_tts(pt, ctx, inst, wl, seed, args.warmup + args.steps, args.tts_sweeps, stream, dev)
    else:
        per = residual_tts(ctx.read(pt.TRACE_F), ctx.read(pt.TRACE_G), args.warmup + args.steps,
                           inst.E_planted, inst.N, inst.scale, interval)
        tts = {"targets": tts_summary(per, elapsed_ms / 1e3 / (args.steps * interval)),
               "sweeps_run": int((args.warmup + args.steps) * interval), "note": PROXY_NOTE}
    ctx.close()
    batched = leg_batched(pt, args, stream, dev) if legs else None
    ground = leg_ground_state(pt, args, stream, dev) if legs else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int8 spins, int32 fields, f32 decisions",
        "data": "synthetic (seeded planted Wishart instance)",
        "config": {"workload": workload_name(args.workload, n, runs), "physical_spins": n,
                   "replicas": R * runs, "sweeps_per_step": interval,
                   "l2": f"state {n * R * runs / 1e6:.0f} MB > L2 (129 MB); no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "tiling": tiling},
        "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak,
                     "unit": "Tops/s (lane-ops)", "frac": alu_achieved / alu_peak,
                     "traffic": traffic, "kernel": kernel, "kernel_src": src_hash,
                     "traffic_source": prof["profile"] if traffic is not None else
                     "null: no ncu capture of this kernel source",
                     "peak_source": f"{sm_count} SMs x 128 lanes x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({peak_src} max clock)",
                     "ops_per_update": ops_per_update,
                     "hbm": {"achieved_gbs": hbm_achieved, "peak_gbs": peaks.get("hbm_gbs"),
                             "frac": hbm_achieved / peaks.get("hbm_gbs", 6800.0),
                             "bytes_per_update": BYTES_PER_UPDATE,
                             "measured_gbs": (traffic / (avg_launch_ms / 1e3) / 1e9) if traffic else None},
                     "avg_launch_ms": avg_launch_ms, "launches": sweep_launches,
                     "share_of_step": sweep_ms / max(elapsed_ms, 1e-9)},
        "e2e": e2e,
        "gpu_launches": int(gpu_launches),
        "clocks": clocks,
        "tts": tts,
        "batched": batched,
        "ground_state": ground,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def run_e2e(pt, phys, wl, args):
    """The same metric through the C ABI with host buffers: each job creates a
    context from the host instance (host -> device copies), runs E events and
    reads the results back (device -> host); wall time covers everything."""
    import torch

    inst, beta, P, runs, interval = wl["inst"], wl["beta"], wl["P"], wl["runs"], wl["interval"]
    events = max(1, min(args.steps, 20))
    jobs = 2
    R = len(beta) * len(P)
    h2d = (phys.cp_ptr.nbytes + phys.cp_col.nbytes + phys.cp_J.nbytes + phys.lk_ptr.nbytes
           + phys.lk_col.nbytes + beta.nbytes + P.nbytes + runs * 8)
    d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(jobs):
        ctx = pt.PT2D(phys, beta, P, runs, trace_capacity=events)
        ctx.write(pt.TARGET, np.full(runs, inst.E_planted, np.int64))
        ctx.run(interval * events, interval, 500 + j)
        res = [ctx.read(pt.BEST_F), ctx.read(pt.BEST_STATE), ctx.read(pt.SOLVED_EVENT),
               ctx.read(pt.TRACE_F), ctx.read(pt.TRACE_G)]
        d2h = sum(r.nbytes for r in res)
        ctx.close()
    wall = time.perf_counter() - t0
    updates = phys.n * R * runs * interval * events * jobs
    return {"value": updates / wall, "unit": UNIT, "h2d_bytes_per_step": int(h2d / events),
            "d2h_bytes_per_step": int(d2h / events),
            "job": f"create from host CSR + {events} events + read best/trace, x{jobs}"}


def _oracle_sample(wl, threads, sweeps, state=None):
    """Time the CPU oracle on `threads` runs of the workload (one thread per run),
    `sweeps` sweeps each (one event of that length)."""
    import threading

    import oracle

    if state is None:
        phys = oracle.sparsify(wl["inst"].Jq, "max_edges", 3)
        oinst = oracle.OracleInstance(phys)
        orcs = [oracle.OracleRun(oinst, wl["beta"], wl["P"], [r], 100 + r) for r in range(threads)]
        state = (phys, orcs)
    phys, orcs = state
    t0 = time.perf_counter()
    ths = [threading.Thread(target=o.run, args=(sweeps, sweeps)) for o in orcs]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    wall = time.perf_counter() - t0
    R = len(wl["beta"]) * len(wl["P"])
    updates = phys.n * R * sweeps * threads
    return updates / wall, wall, state


def cpu_baseline(wl, args):
    threads = min(os.cpu_count() or 1, wl["runs"])
    sweeps = args.cpu_sweeps if wl["key"] == "n200" else 1
    rate, wall, _ = _oracle_sample(wl, threads, sweeps)
    R = wl["I"] * wl["J"]
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{threads} runs x {R} replicas x {sweeps} sweeps of the N={wl['inst'].N} "
                      f"instance (one thread per run), {wall:.1f} s wall"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    key = args.workload if args.workload in WORKLOADS else "n200"
    wl = make_workload(key)
    threads = min(os.cpu_count() or 1, wl["runs"])
    sweeps = 2 if key == "n200" else 1
    R = wl["I"] * wl["J"]
    state = None
    for _ in range(args.warmup):
        _, _, state = _oracle_sample(wl, threads, sweeps, state)
    total_updates = 0.0
    total_wall = 0.0
    for _ in range(args.steps):
        rate, wall, state = _oracle_sample(wl, threads, sweeps, state)
        total_updates += rate * wall
        total_wall += wall
    value = total_updates / total_wall
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_wall / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int8 spins, int64 energies, f32 decisions", "data": "synthetic (seeded planted Wishart instance)",
        "config": {"workload": workload_name(key, state[0].n),
                   "sample": f"per step: {threads} runs x {R} replicas x {sweeps} sweeps"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{threads} runs x {R} replicas x {sweeps} sweeps per step, one thread per run"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _cuda_events():
    import torch

    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _timed(stream, fn):
    """CUDA-event seconds of the work `fn` queues on `stream`."""
    e0, e1 = _cuda_events()
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


PROXY_NOTE = ("rho<=x targets (bottom-right replica feasible with residual energy per spin "
              "(f - E_planted)/(N s) <= x) are proxies for the planted ground state; 'planted' is the "
              "target the metric names: g = 0 and f <= E_planted")


def leg_tts(pt, ctx, inst, wl, seed, events_done, total_sweeps, stream, dev):
    """Time to target on the timed workload: the same runs continue (outside the
    timed region) until `total_sweeps`; per run, sweeps until the bottom-right
    replica first meets each target, and seconds = sweeps x the whole job's
    measured wall time per sweep (all runs advance together)."""
    interval = wl["interval"]
    total_events = max(events_done, total_sweeps // interval)
    more = total_events - events_done
    with ClockSampler(dev) as clk:
        secs = _timed(stream, lambda: ctx.run(more * interval, interval, seed)) if more else 0.0
    sec_per_sweep = secs / max(more * interval, 1)
    per = residual_tts(ctx.read(pt.TRACE_F), ctx.read(pt.TRACE_G), total_events,
                       inst.E_planted, inst.N, inst.scale, interval)
    best = ctx.read(pt.BEST_F)
    feasible = best < np.iinfo(np.int64).max
    rho = (best[feasible] - inst.E_planted) / (inst.N * inst.scale)
    targets = tts_summary(per, sec_per_sweep)
    for v in targets.values():
        v["censored"] = v["runs"] - v["reached"]
    return {"targets": targets, "sweeps_run": int(total_events * interval),
            "seconds_per_sweep_all_runs": sec_per_sweep, "seconds_continued": secs,
            "median_best_feasible_residual_per_spin": float(np.median(rho)) if rho.size else None,
            "note": PROXY_NOTE + "; seconds = sweeps x the job's wall time per sweep (CUDA events)",
            "clocks": clk.summary()}


def batched_vs_plain(pt, probs, interval, *, batched_events, plain_events, tts_events, autotune,
                     max_degree, stream, dev, chunk=20, plain=True):
    """The batched persistent form against the one-instance-per-launch form on
    the same problems (identical trajectories).

    probs: (inst, phys, beta, P, seed).  The batch runs every problem in one
    kernel launch per event (CUDA graph); the plain form is one context per
    problem, run one after the other on the same stream.  Both forms are timed
    with CUDA events over whole events of every problem; the plain form's
    bottom-right (f, g) record of every event it ran is compared with the
    batch's.  The batch then continues to `tts_events` events: per problem,
    sweeps until each target (identical in both forms), and seconds = sweeps x
    each form's measured wall time per sweep of the whole set."""
    spins = sum(p[1].n for p in probs)
    R = len(probs[0][2]) * len(probs[0][3])
    upd_per_event = spins * R * interval
    cap = max(tts_events, batched_events + 32)
    probe = pt.Batch(1 << 22, max_degree, 8, stream=stream, trace_capacity=cap)
    need = sum(probe.instance_bytes(p[1], len(p[2]), len(p[3]), 1) for p in probs)
    probe.close()
    batch = pt.Batch(int(need * 1.02) + (64 << 20), max_degree, len(probs), stream=stream,
                     trace_capacity=cap)
    ids = [batch.add(p[1], p[2], p[3], 1, p[4], p[0].E_planted) for p in probs]
    tuned = batch.autotune(1, interval) if autotune else None
    batch.run(1, interval)
    done = int(batch.read(ids[0], pt.COUNTERS)[1])  # autotune trials advance the chains
    with ClockSampler(dev) as clk_b:
        t_batched = _timed(stream, lambda: batch.run(batched_events, interval))
    done += batched_events
    out = {"batched": {"seconds": t_batched, "events": batched_events,
                       "updates_per_s": upd_per_event * batched_events / t_batched,
                       "seconds_per_sweep": t_batched / (batched_events * interval),
                       "shape": batch.shape, "autotuned": tuned is not None, "clocks": clk_b.summary()}}
    if plain:
        ctxs = [pt.PT2D(p[1], p[2], p[3], 1, stream=stream, trace_capacity=plain_events + 1)
                for p in probs]
        for c, p in zip(ctxs, probs):
            c.run(interval, interval, p[4])  # warm-up event
        stream.synchronize()

        def plain_events_fn():
            for c, p in zip(ctxs, probs):
                c.run(plain_events * interval, interval, p[4])

        with ClockSampler(dev) as clk_p:
            t_plain = _timed(stream, plain_events_fn)
        same, checked = 0, 0
        for c, i in zip(ctxs, ids):
            k = plain_events + 1
            bt = (batch.read(i, pt.TRACE_F)[0, :k], batch.read(i, pt.TRACE_G)[0, :k])
            ct = (c.read(pt.TRACE_F)[0, :k], c.read(pt.TRACE_G)[0, :k])
            checked += 1
            same += bool(np.array_equal(bt[0], ct[0]) and np.array_equal(bt[1], ct[1]))
        launches = sum(c.launch_count for c in ctxs)
        for c in ctxs:
            c.close()
        out["plain"] = {"seconds": t_plain, "events": plain_events,
                        "updates_per_s": upd_per_event * plain_events / t_plain,
                        "seconds_per_sweep": t_plain / (plain_events * interval),
                        "launches_total": int(launches), "clocks": clk_p.summary(),
                        "identical_records": f"{same} of {checked} problems: bottom-right (f, g) "
                                             f"of all {plain_events + 1} events equal to the batch's"}
        out["speedup_wall"] = out["plain"]["seconds_per_sweep"] / out["batched"]["seconds_per_sweep"]
    t_more = 0.0
    while done < tts_events:
        k = min(chunk, tts_events - done)
        t_more += _timed(stream, lambda: batch.run(k, interval))
        done += k
    per = {}
    for i, p in zip(ids, probs):
        r = residual_tts(batch.read(i, pt.TRACE_F), batch.read(i, pt.TRACE_G), done,
                         p[0].E_planted, p[0].N, p[0].scale, interval)
        for k, v in r.items():
            per.setdefault(k, []).append(int(v[0]))
    batch.close()
    per = {k: np.array(v) for k, v in per.items()}
    tts = {"events_run": int(done), "sweeps_run": int(done * interval),
           "targets_batched": tts_summary(per, out["batched"]["seconds_per_sweep"]),
           "seconds_continued_batched": t_more}
    if plain:
        tts["targets_plain"] = tts_summary(per, out["plain"]["seconds_per_sweep"])
        tts["tts_speedup"] = {k: (tts["targets_plain"][k]["median_seconds"] /
                                  tts["targets_batched"][k]["median_seconds"])
                              if tts["targets_batched"][k]["median_seconds"] else None for k in per}
        tts["plain_seconds_source"] = ("identical sweep counts x the plain form's measured wall time per "
                                       f"sweep ({plain_events} events of every problem)")
    out["tts"] = tts
    out["per_problem_sweeps"] = per
    out["spins_total"] = int(spins)
    out["updates_per_event"] = int(upd_per_event)
    return out


def batched_problems(count, seed0=1000):
    """The uneven batch: planted Wishart instances with N uniform on {50..400}
    and alpha in {0.25, 0.5, 0.75}, each copy-chain sparsified to physical
    degree <= 4, I = 16 x J = 8."""
    import paper_2506_14781_gb300 as pt
    import synth

    probs = []
    for N, alpha, seed in synth.batch_specs(count, seed0):
        inst = synth.wishart_planted(N, alpha, seed)
        phys = pt.sparsify(inst.Jq, "max_degree", 4)
        probs.append((inst, phys, synth.beta_ladder(16, BETA_MIN, BETA_MAX, inst.scale),
                      synth.penalty_ladder(8, P_MIN, P_MAX, 32767), seed))
    return probs


def ground_state_problems(Ns, per_N, alpha=0.75):
    """Small planted Wishart instances with three copies per node (the paper's
    sparsification for its ground-state runs), I = 16 x J = 8: sizes at which
    2D-PT reaches the planted energy within 10^5 sweeps."""
    import paper_2506_14781_gb300 as pt
    import synth

    probs = []
    for N in Ns:
        for k in range(per_N):
            inst = synth.wishart_planted(N, alpha, 5000 + 100 * N + k)
            phys = pt.sparsify(inst.Jq, "fixed", 3)
            probs.append((inst, phys, synth.beta_ladder(16, BETA_MIN, BETA_MAX, inst.scale),
                          synth.penalty_ladder(8, P_MIN, P_MAX, 32767), 777 + k))
    return probs


def _strip(out):
    out = dict(out)
    out.pop("per_problem_sweeps", None)
    return out


def leg_batched(pt, args, stream, dev):
    """The uneven 1024-instance batch, batched vs one context per instance."""
    t0 = time.perf_counter()
    probs = batched_problems(args.instances)
    gen_s = time.perf_counter() - t0
    out = batched_vs_plain(pt, probs, 50, batched_events=args.batched_events,
                           plain_events=args.plain_events, tts_events=args.tts_events,
                           autotune=True, max_degree=3, stream=stream, dev=dev)
    out = _strip(out)
    out["workload"] = (f"{len(probs)} planted Wishart instances, N~U{{50..400}}, alpha in {{0.25,0.5,0.75}}, "
                       "physical degree <= 4, I=16 x J=8, 1 run each, swap every 50 sweeps")
    out["instance_generation_s"] = gen_s
    out["tts"]["note"] = PROXY_NOTE
    return out


def leg_ground_state(pt, args, stream, dev):
    """Time to the planted ground state, batched vs plain, where it is reached."""
    probs = ground_state_problems(args.gs_ns, args.gs_instances)
    degree = max(64, max(int(np.diff(p[1].cp_ptr).max()) for p in probs))
    out = batched_vs_plain(pt, probs, 50, batched_events=args.gs_timed_events,
                           plain_events=args.plain_events, tts_events=args.gs_events, autotune=True,
                           max_degree=degree, stream=stream, dev=dev, chunk=100)
    per = out["per_problem_sweeps"]["planted"]
    out = _strip(out)
    out["workload"] = (f"{len(probs)} planted Wishart instances (N in {list(args.gs_ns)}, alpha 0.75), "
                       "three copies per node, I=16 x J=8, 1 run each, swap every 50 sweeps, "
                       f"{args.gs_events * 50} sweeps")
    out["planted_reached"] = int((per >= 0).sum())
    out["tts"]["note"] = ("'planted': the bottom-right replica feasible (g = 0) with f <= E_planted, "
                          "the planted ground state (or lower)")
    return out


def run_batched(args):
    """Uneven-batch workload: planted Wishart instances with N uniform on
    {50..400} and alpha in {0.25, 0.5, 0.75}, each copy-chain sparsified to
    physical degree <= 4, I = 16 x J = 8, one run each, swap interval 50.
    Times the batched persistent form against the one-instance-per-launch form
    on the same events (identical trajectories), then continues the batched
    form to `--tts-events` events for time to target."""
    if int(os.environ.get("RANK", "0")) != 0:
        return  # a one-GPU workload: under torchrun the other ranks do no work
    import torch

    import paper_2506_14781_gb300 as pt

    stream = torch.cuda.Stream()
    dev = torch.cuda.current_device()
    t0 = time.perf_counter()
    probs = batched_problems(args.instances)
    gen_s = time.perf_counter() - t0
    E = args.steps
    out = batched_vs_plain(pt, probs, 50, batched_events=E, plain_events=args.plain_events,
                           tts_events=args.tts_events, autotune=args.autotune, max_degree=3,
                           stream=stream, dev=dev, plain=not args.no_plain)
    Ns = np.array([p[0].N for p in probs])
    per = out["per_problem_sweeps"]
    out["tts"]["reached_by_N"] = {k: {f"{lo}-{lo + 49}": int((v[(Ns >= lo) & (Ns < lo + 50)] >= 0).sum())
                                      for lo in range(50, 401, 50)} for k, v in per.items()}
    out["tts"]["note"] = PROXY_NOTE
    out = _strip(out)
    t_b = out["batched"]["seconds"]
    line = {
        "metric": METRIC,
        "value": out["batched"]["updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": E,
        "warmup": 1, "ms_per_step": t_b / E * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8 spins, int32 fields, f32 decisions",
        "data": "synthetic (seeded planted Wishart instances)",
        "config": {"workload": f"{len(probs)} planted Wishart instances, N~U{{50..400}}, alpha in "
                               f"{{0.25,0.5,0.75}}, physical degree <= 4, I=16 x J=8, 1 run each, "
                               f"swap every 50 sweeps", "physical_spins_total": out["spins_total"],
                   "instance_generation_s": gen_s},
        **out,
    }
    peaks, peak_src = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sm_count * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    alu = out["batched"]["updates_per_s"] * OPS_PER_UPDATE / 1e12
    line["roofline"] = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "Tops/s (lane-ops)",
                        "frac": alu / alu_peak, "traffic": None, "kernel": "k_batch",
                        "ops_per_update": OPS_PER_UPDATE,
                        "traffic_source": "profiles/k_batch_uneven137.md (137-instance capture, not scaled)",
                        "peak_source": f"{sm_count} SMs x 128 lanes x max clock ({peak_src})"}
    print(json.dumps(line))


def run_compare(args):
    """2D-PT against the J-column PT baseline (the paper's Fig. 3 comparison
    shape) on synthetic planted Wishart instances: N in `--cmp-ns` (20, 30, 40, 50),
    alpha = 0.75, I = 16 x J = 8, sparsified either to <= 3 original edges per
    copy (`--cmp-sparsify max_edges3`) or to three copies per node, the paper's
    setting (`fixed3`: ~N/3 couplings per copy, on the batch's runtime-degree
    kernel).  Each arm runs as one batch.  2D-PT uses a
    linear P ladder; J-column PT runs the same beta ladder in every column at
    the mean of those penalties, with beta-swaps only, and keeps the best
    feasible replica of its last row.  `--cmp-events` events of 50 sweeps;
    reported: the median over instances of the residual
    energy per spin of the best feasible state so far, rho = (f - E_gs) / (N s),
    at log-spaced sweep counts, and the sweeps to reach rho <= 0.2 / 0.1 /
    0.05 / 0 (E_gs: the planted energy or anything lower either method found)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return  # a one-GPU workload: under torchrun the other ranks do no work
    import torch

    import paper_2506_14781_gb300 as pt
    import synth

    I, J, interval, E = 16, 8, 50, args.cmp_events
    per_N = args.cmp_instances
    Ns = tuple(args.cmp_ns)
    probs = []
    for N in Ns:
        for k in range(per_N):
            inst = synth.wishart_planted(N, 0.75, 5000 + 100 * N + k)
            rule = ("max_edges", 3) if args.cmp_sparsify == "max_edges3" else ("fixed", 3)
            phys = pt.sparsify(inst.Jq, *rule)
            probs.append((inst, phys, synth.beta_ladder(I, BETA_MIN, BETA_MAX, inst.scale),
                          synth.penalty_ladder(J, P_MIN, P_MAX, 32767)))
    stream = torch.cuda.Stream()
    out = {}
    traces = {}
    for mode in ("2d", "jcolumn"):
        ladders = [(P if mode == "2d" else np.full(J, int(np.rint(P.mean())), np.int32))
                   for _, _, _, P in probs]
        degree = 3 if args.cmp_sparsify == "max_edges3" else max(
            64, max(int(np.diff(phys.cp_ptr).max()) for _, phys, _, _ in probs))
        b = pt.Batch(1 << 30, degree, len(probs), stream=stream, trace_capacity=E, swap_mode=mode)
        ids = [b.add(phys, beta, Pm, 1, 777 + k, inst.E_planted)
               for k, ((inst, phys, beta, _), Pm) in enumerate(zip(probs, ladders))]
        t0 = time.perf_counter()
        b.run(E, interval)
        b.sync()
        secs = time.perf_counter() - t0
        tf = np.stack([b.read(i, pt.TRACE_F)[0] for i in ids])
        tg = np.stack([b.read(i, pt.TRACE_G)[0] for i in ids])
        b.close()
        traces[mode] = (tf, tg)
        out[mode] = {"seconds": secs, "feasible_record_fraction": float((tg == 0).mean())}
    # ground-state estimate per instance: the planted energy or anything lower found
    big = np.iinfo(np.int64).max
    E_gs = []
    for k, (inst, _, _, _) in enumerate(probs):
        found = min(int(np.where(traces[m][1][k] == 0, traces[m][0][k], big).min()) for m in traces)
        E_gs.append(min(int(inst.E_planted), found))
    E_gs = np.array(E_gs)
    norm = np.array([inst.N * inst.scale for inst, _, _, _ in probs])
    checkpoints = sorted({int(x) for x in np.unique(np.round(np.geomspace(1, E, 12)))})
    Narr = np.array([inst.N for inst, _, _, _ in probs])
    for mode, (tf, tg) in traces.items():
        best = np.minimum.accumulate(np.where(tg == 0, tf, big), axis=1)
        rho = np.where(best < big, (best - E_gs[:, None]) / norm[:, None], np.inf)
        curve = {}
        for N in Ns:
            sel = Narr == N
            curve[str(N)] = {str(c * interval): float(np.median(rho[sel, c - 1])) for c in checkpoints}
        tts = {}
        for target in (0.2, 0.1, 0.05, 0.0):
            hit = rho <= target + 1e-12
            first = np.where(hit.any(1), hit.argmax(1) + 1, -1) * interval
            tts[f"rho<={target}"] = {str(N): {"reached": int((first[Narr == N] > 0).sum()),
                                              "of": int((Narr == N).sum()),
                                              "median_sweeps": float(np.median(first[(Narr == N) & (first > 0)]))
                                              if ((Narr == N) & (first > 0)).any() else None}
                                     for N in Ns}
        out[mode].update({"median_rho_by_sweeps": curve, "sweeps_to_target": tts})
    line = {
        "metric": "residual energy per spin vs sweeps, 2D-PT vs J-column PT (same replicas)",
        "value": None, "unit": "rho", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
        "config": {"workload": f"{per_N} planted Wishart instances per N in {list(Ns)}, alpha 0.75, "
                               f"{'<=3 edges per copy' if args.cmp_sparsify == 'max_edges3' else '3 copies per node'}, "
                               f"I={I} x J={J}, {E} events of {interval} sweeps; "
                               "J-column PT at the mean 2D-PT penalty"},
        "results": out,
    }
    print(json.dumps(line))


def run_adaptive(args):
    """Algorithm 2's adaptive ladders at length (the paper's ground-state
    setting): planted Wishart instances, alpha = 0.75, three copies per node,
    N in `--ad-ns` (100, 200), `--ad-instances` per N.  Per instance the
    library's pt2d_adaptive_schedule builds the beta and P ladders (capped at
    20 x 20; beta0 = 0.1 / s, P0 = 0.5 x 32767, alpha_beta = alpha_P =
    2 erfc^-1(1/2) for swap rates near 1/2, populations of `--ad-chains`
    chains x `--ad-mcs` sweeps, the row walk stopping at sigma_E <=
    `--ad-sigma-min` couplings of 32767).  Then, on the same instances and
    seeds, three arms run `--ad-events` events of 50 sweeps: 2D-PT on the
    adaptive ladders, J-column PT on the same beta ladder at the mean of the
    adaptive penalties, and 2D-PT on the fixed ladders of the other workloads
    (I = 16 x J = 8).  Ladders of up to 400 replicas exceed the batch's 128 per
    run, so each instance is one context; 16 run at a time on their own
    streams.  Reported per N and arm: the median over instances of the residual
    energy per spin of the best feasible bottom-right state so far, rho =
    (f - E_gs) / (N s), against sweeps, and the instances reaching rho <= 0.1,
    0.05 and 0 (E_gs: the planted energy or anything lower any arm found)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return  # a one-GPU workload
    import concurrent.futures as cf

    import torch
    from scipy.special import erfcinv

    import paper_2506_14781_gb300 as pt
    import synth

    interval, E, per_N = 50, args.ad_events, args.ad_instances
    Ns = tuple(args.ad_ns)
    probs = []
    for N in Ns:
        for k in range(per_N):
            inst = synth.wishart_planted(N, 0.75, 7000 + 100 * N + k)
            probs.append((inst, pt.sparsify(inst.Jq, "fixed", 3), 4242 + k))
    alpha = float(2 * erfcinv(0.5))

    def schedule(p):
        inst, phys, seed = p
        stream = torch.cuda.Stream()
        t0 = time.perf_counter()
        beta, P, samples = pt.adaptive_schedule(
            phys, beta0=BETA_MIN / inst.scale, P0=int(P_MIN * 32767), max_rows=20, max_cols=20,
            sigma_min=args.ad_sigma_min * 32767, alpha_beta=alpha, alpha_P=alpha, n_chain=args.ad_chains,
            mcs=args.ad_mcs, seed=seed * 1000, stream=stream)
        stream.synchronize()
        return beta, P, samples, time.perf_counter() - t0

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(16) as ex:
        ladders = list(ex.map(schedule, probs))
    sched_s = time.perf_counter() - t0
    arms = {
        "2d_adaptive": [(b, P, "2d") for b, P, _, _ in ladders],
        "jcolumn_adaptive": [(b, np.full(P.size, int(np.rint(P.mean())), np.int32), "jcolumn")
                             for b, P, _, _ in ladders],
        "2d_fixed": [(synth.beta_ladder(16, BETA_MIN, BETA_MAX, p[0].scale),
                      synth.penalty_ladder(8, P_MIN, P_MAX, 32767), "2d") for p in probs],
    }

    def run_one(job):
        (inst, phys, seed), (beta, P, mode) = job
        stream = torch.cuda.Stream()
        ctx = pt.PT2D(phys, beta, P, 1, stream=stream, trace_capacity=E, swap_mode=mode)
        ctx.write(pt.TARGET, [inst.E_planted])
        ctx.run(E * interval, interval, seed)
        out = (ctx.read(pt.TRACE_F)[0], ctx.read(pt.TRACE_G)[0])
        ctx.close()
        return out

    traces, arm_s = {}, {}
    for arm, lad in arms.items():
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(16) as ex:
            res = list(ex.map(run_one, zip(probs, lad)))
        arm_s[arm] = time.perf_counter() - t0
        traces[arm] = (np.stack([r[0] for r in res]), np.stack([r[1] for r in res]))
    big = np.iinfo(np.int64).max
    E_gs = np.array([min(int(p[0].E_planted),
                         min(int(np.where(traces[a][1][k] == 0, traces[a][0][k], big).min()) for a in traces))
                     for k, p in enumerate(probs)])
    norm = np.array([p[0].N * p[0].scale for p in probs])
    Narr = np.array([p[0].N for p in probs])
    checkpoints = sorted({int(x) for x in np.unique(np.round(np.geomspace(1, E, 14)))})
    results = {}
    for arm, (tf, tg) in traces.items():
        best = np.minimum.accumulate(np.where(tg == 0, tf, big), axis=1)
        rho = np.where(best < big, (best - E_gs[:, None]) / norm[:, None], np.inf)
        planted = np.minimum.accumulate(np.where(tg == 0, tf, big), axis=1) <= np.array(
            [p[0].E_planted for p in probs])[:, None]
        res = {"seconds": arm_s[arm], "feasible_record_fraction": float((tg == 0).mean())}
        for N in Ns:
            sel = Narr == N
            curve = {str(c * interval): float(np.median(rho[sel, c - 1])) for c in checkpoints}
            reach = {}
            for target in (0.1, 0.05, 0.0):
                hit = rho[sel] <= target + 1e-12
                first = np.where(hit.any(1), hit.argmax(1) + 1, -1) * interval
                reach[f"rho<={target}"] = {"reached": int((first > 0).sum()), "of": int(sel.sum()),
                                           "median_sweeps": float(np.median(first[first > 0]))
                                           if (first > 0).any() else None}
            hitp = planted[sel]
            firstp = np.where(hitp.any(1), hitp.argmax(1) + 1, -1) * interval
            reach["planted"] = {"reached": int((firstp > 0).sum()), "of": int(sel.sum()),
                                "median_sweeps": float(np.median(firstp[firstp > 0])) if (firstp > 0).any() else None}
            res[str(N)] = {"median_rho_by_sweeps": curve, "sweeps_to_target": reach}
        results[arm] = res
    lad_stats = {}
    for N in Ns:
        sel = [k for k, p in enumerate(probs) if p[0].N == N]
        Is = [ladders[k][0].size for k in sel]
        Js = [ladders[k][1].size for k in sel]
        lad_stats[str(N)] = {"I_median": float(np.median(Is)), "I_range": [int(min(Is)), int(max(Is))],
                             "J_median": float(np.median(Js)), "J_range": [int(min(Js)), int(max(Js))],
                             "beta_max_times_s_median": float(np.median([ladders[k][0][-1] * probs[k][0].scale
                                                                         for k in sel])),
                             "P_max_over_32767_median": float(np.median([ladders[k][1][-1] / 32767 for k in sel])),
                             "samples_median": float(np.median([ladders[k][2] for k in sel]))}
    line = {
        "metric": "residual energy per spin vs sweeps on Algorithm 2's adaptive ladders",
        "value": None, "unit": "rho", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
        "config": {"workload": f"{per_N} planted Wishart instances per N in {list(Ns)}, alpha 0.75, three "
                               f"copies per node; adaptive ladders capped at 20 x 20 (populations of "
                               f"{args.ad_chains} chains x {args.ad_mcs} sweeps, sigma_min = "
                               f"{args.ad_sigma_min} x 32767); {E} events of {interval} sweeps per arm"},
        "schedule_seconds": sched_s, "ladders": lad_stats, "results": results,
    }
    print(json.dumps(line))


def run_fig2(args):
    """The paper's Fig. 2 experiment shape: a 5-node all-to-all instance with two
    copies per node (10 physical spins, physical degree 3), one row at beta = 1,
    penalties P in {2, 4, 6, 8} (in the paper's units of g = (S1 - S2)^2) with
    P-swaps every 500 sweeps, against the P = 8 replica alone; 100 chains each.  The Full Adder couplings are not given, so
    the instance is seeded with couplings in {+-1, +-2, +-3}.  The last
    replica's state is sampled after every 500-sweep event; its feasible (g = 0)
    samples map to logical states (first copy of each chain), and the KL
    divergence D(p_hat || p) to the exact 5-node Boltzmann distribution at
    beta = 1 is reported against sweeps, per chain (mean over chains) and pooled
    over the chains."""
    if int(os.environ.get("RANK", "0")) != 0:
        return  # a one-GPU workload: under torchrun the other ranks do no work
    import torch  # noqa: F401  (CUDA context for the library)

    import paper_2506_14781_gb300 as pt

    rng = np.random.default_rng(3)
    A = rng.integers(1, 4, size=(5, 5)) * rng.choice([-1, 1], size=(5, 5))
    Jq = np.triu(A, 1)
    Jq = (Jq + Jq.T).astype(np.int16)
    phys = pt.sparsify(Jq, "fixed", 2)
    # exact logical Boltzmann distribution at beta = 1: f(s) = -sum_{i<j} J_ij s_i s_j
    states = np.array([[1 - 2 * ((k >> i) & 1) for i in range(5)] for k in range(32)])
    f_log = -0.5 * np.einsum("ki,ij,kj->k", states, Jq.astype(np.int64), states)
    w = np.exp(-(f_log - f_log.min()))
    p_exact = w / w.sum()
    first = np.array([int(np.nonzero(phys.copy_of == i)[0].min()) for i in range(5)])
    chains, interval, events = 100, 500, args.fig2_events
    checkpoints = sorted({int(x) for x in np.unique(np.round(np.geomspace(1, events, 16)))})
    out = {}
    # the paper's g = (S1 - S2)^2 is 4 per broken link where this library's g is 1,
    # so its penalties {2, 4, 6, 8} are {8, 16, 24, 32} here
    for arm, P in (("with_P_swaps", 4 * np.array([2, 4, 6, 8], np.int32)),
                   ("P8_alone", 4 * np.array([8], np.int32))):
        ctx = pt.PT2D(phys, np.array([1.0], np.float32), P, chains, trace_capacity=0)
        counts = np.zeros((chains, 32), np.int64)
        curve_chain, curve_pooled = {}, {}
        for e in range(1, events + 1):
            ctx.run(interval, interval, 2024)
            at = ctx.read(pt.WALKER_AT)[:, -1]
            S = ctx.read(pt.STATES)            # [chains][R][n], by walker
            s_last = S[np.arange(chains), at]  # the last slot's state per chain
            g = np.zeros(chains, np.int64)
            for a in range(phys.n):
                for k in range(phys.lk_ptr[a], phys.lk_ptr[a + 1]):
                    g += s_last[:, a] != s_last[:, phys.lk_col[k]]
            feas = g == 0
            idx = ((s_last[:, first] < 0).astype(np.int64) << np.arange(5)).sum(1)
            np.add.at(counts, (np.nonzero(feas)[0], idx[feas]), 1)
            if e in checkpoints:
                def kl(c):
                    q = c / max(c.sum(), 1)
                    m = q > 0
                    return float((q[m] * np.log(q[m] / p_exact[m])).sum()) if c.sum() else None
                per = [kl(counts[c]) for c in range(chains)]
                per = [x for x in per if x is not None]
                curve_chain[str(e * interval)] = float(np.mean(per)) if per else None
                curve_pooled[str(e * interval)] = kl(counts.sum(0))
        ctx.close()
        out[arm] = {"kl_mean_over_chains": curve_chain, "kl_pooled": curve_pooled,
                    "feasible_fraction": float(counts.sum() / (chains * events))}
    line = {
        "metric": "KL divergence of the last replica vs sweeps (Fig. 2 shape)", "value": None,
        "unit": "nats", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
        "config": {"workload": "seeded 5-node all-to-all instance, 2 copies per node (10 spins), "
                               f"beta = 1, P in 4 x {{2,4,6,8}} vs 4 x 8 alone, {chains} chains, "
                               f"swap every {interval} sweeps, {events} events, one sample per event"},
        "results": out,
    }
    print(json.dumps(line))


def run_constrained(args):
    """General constraint functions (Eq. 1 with g beyond copy links): 3-colouring
    of a random cubic graph, V = 2000 vertices (`--col-vertices`; n = 6000 spins, coupling
    degree 3, two one-hot links per spin), one-hot groups expanded by the
    library (pt2d_onehot_penalty), I = 16 x J = 8 (the batch's largest grid),
    256 runs (32,768 replicas, 197 MB of spins, larger than L2), swap
    interval 50.  The plain context runs it on the degree-specialised
    penalty kernel (int8 slab in shared memory, or bit-packed when the int8
    slab does not fit, e.g. --col-vertices 40000 --runs 64; weighted links,
    penalty fields, g0); the same runs then go through the runtime-degree
    batch (identical trajectories).  Reports spin
    updates/s with the sweep kernel's ALU roofline and how many runs found a
    proper colouring (g = 0, f = -k W)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return  # a one-GPU workload
    import torch

    import paper_2506_14781_gb300 as pt
    import synth

    V, k, I, J, runs, interval = args.col_vertices, 3, 16, 8, args.runs or 256, 50
    prob = synth.colouring(V, k, 7)
    lk_ptr, lk_col, lk_w, hk, g0 = pt.onehot_penalty(prob.n, prob.groups)
    phys = pt.PhysicalInstance(prob.n, prob.cp_ptr, prob.cp_col, prob.cp_J, lk_ptr, lk_col, h=prob.h,
                               lk_w=lk_w, hk=hk, g0=g0)
    # f moves by at most 12 per flip; the last column's penalty outweighs that
    beta = np.geomspace(0.05, 2.0, I).astype(np.float32)
    P = np.array([1, 2, 3, 5, 8, 12, 17, 24], np.int32)[:J]
    n, R = prob.n, I * J
    updates_per_event = n * R * runs * interval
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    ctx = pt.PT2D(phys, beta, P, runs, stream=stream, trace_capacity=args.warmup + args.steps, profile=True)
    ctx.write(pt.TARGET, np.full(runs, prob.f_proper, np.int64))
    seed = 2024
    with torch.cuda.stream(stream):
        ctx.run(interval * args.warmup, interval, seed)
    ctx.sync()
    ms0, l0 = ctx.kernel_time(0)
    n_launch0 = ctx.launch_count
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        start.record(stream)
        ctx.run(interval * args.steps, interval, seed)
        end.record(stream)
        end.synchronize()
    elapsed_ms = start.elapsed_time(end)
    sweep_ms, launches = ctx.kernel_time(0)
    sweep_ms -= ms0
    launches -= l0
    gpu_launches = ctx.launch_count - n_launch0
    value = updates_per_event * args.steps / (elapsed_ms / 1e3)
    avg_launch_ms = sweep_ms / max(launches, 1)
    tiling = ctx.tiling
    kernel = sweep_kernel_name(tiling)
    peaks, peak_src = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sm_count * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    alu = updates_per_event * OPS_PER_UPDATE / (avg_launch_ms / 1e3) / 1e12
    prof = PROFILED_TRAFFIC.get(("constrained", kernel))
    src_hash = kernel_source_hash(kernel)
    traffic = prof["dram_bytes_per_launch"] if prof and prof["src"] == src_hash else None
    best = ctx.read(pt.BEST_F)
    solved = ctx.read(pt.SOLVED_EVENT)
    feasible = best < np.iinfo(np.int64).max
    F_best = prob.same_colour_weight(best[feasible])
    events_done = args.warmup + args.steps
    # the same runs through the runtime-degree batch
    batch = pt.Batch(max(1 << 31, 3 * n * R * runs), max_coupling_degree=64, max_runs=runs, stream=stream,
                     trace_capacity=events_done)
    bid = batch.add(phys, beta, P, runs, seed, prob.f_proper)
    batch.run(args.warmup, interval)
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    batch.run(args.steps, interval)
    b1.record(stream)
    b1.synchronize()
    batch_ms = b0.elapsed_time(b1)
    same = bool(np.array_equal(batch.read(bid, pt.BEST_F), best) and
                np.array_equal(batch.read(bid, pt.F), ctx.read(pt.F)))
    batch.close()
    ctx.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8 spins, int32 fields, f32 decisions",
        "data": "synthetic (seeded random cubic graph, 3-colouring with one-hot constraints)",
        "config": {"workload": f"3-colouring of a random cubic graph, V={V} ({n} spins, one-hot groups), "
                               f"I={I} x J={J}, {runs} runs, swap every {interval} sweeps",
                   "physical_spins": n, "replicas": R * runs, "tiling": tiling,
                   "l2": f"state {n * R * runs / 1e6:.0f} MB > L2 (129 MB); no flush"},
        "roofline": {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "Tops/s (lane-ops)",
                     "frac": alu / alu_peak, "traffic": traffic, "kernel": kernel, "kernel_src": src_hash,
                     "traffic_source": prof["profile"] if traffic is not None else
                     "null: no ncu capture of this kernel source",
                     "ops_per_update": OPS_PER_UPDATE, "avg_launch_ms": avg_launch_ms, "launches": launches,
                     "peak_source": f"{sm_count} SMs x 128 lanes x max clock ({peak_src})"},
        "batched_runtime_degree": {"updates_per_s": updates_per_event * args.steps / (batch_ms / 1e3),
                                   "identical_results": same},
        "quality": {"runs_with_proper_colouring": int((solved >= 0).sum()), "runs": runs,
                    "median_event_solved": float(np.median(solved[solved >= 0])) if (solved >= 0).any() else None,
                    "runs_feasible": int(feasible.sum()),
                    "best_same_colour_edges_median": float(np.median(F_best)) if F_best.size else None,
                    "edges": int(prob.edges.shape[0]), "sweeps_run": events_done * interval},
        "gpu_launches": int(gpu_launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line))


def run_threecopy(args):
    """The runtime-degree kernels on the paper's sparsification for its
    ground-state runs: planted Wishart instances with alpha = 0.75 and N = 50
    and 100 (`--threecopy-ns`), three copies per node (about N/3
    couplings per copy), I = 20 x J = 20 ladders, 64 runs, swap interval 50;
    each on the shared-memory kernel (automatic tiling) and on the
    global-memory one.  Reports spin updates/s per kernel (3 warm-up events,
    then 10 timed events, CUDA-event time of the sweep launches)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return  # a one-GPU workload
    import torch  # noqa: F401  (CUDA context for the library)

    import paper_2506_14781_gb300 as pt
    import synth

    Ns = args.threecopy_ns
    rows = []
    for N in Ns:
        inst = synth.wishart_planted(N, 0.75, 3)
        phys = pt.sparsify(inst.Jq, "fixed", 3)
        beta = synth.beta_ladder(20, BETA_MIN, BETA_MAX, inst.scale)
        P = synth.penalty_ladder(20, P_MIN, P_MAX, 32767)
        for kernel in ("auto", "global"):
            ctx = pt.PT2D(phys, beta, P, 64, profile=True, trace_capacity=8, sweep_kernel=kernel)
            ctx.run(150, 50, 100)
            ctx.sync()
            ms0, n0 = ctx.kernel_time(0)
            ctx.run(500, 50, 100)
            ms1, n1 = ctx.kernel_time(0)
            per = (ms1 - ms0) / (n1 - n0)
            rows.append({"N": N, "spins": phys.n, "max_couplings_per_copy": int(np.diff(phys.cp_ptr).max()),
                         "tiling": ctx.tiling, "ms_per_launch": per,
                         "updates_per_s": phys.n * 400 * 64 * 50 / (per / 1e3)})
            ctx.close()
    line = {"metric": "spin updates/sec, runtime-degree kernels on three copies per node",
            "value": rows[0]["updates_per_s"], "unit": "spin-updates/s", "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic (seeded planted Wishart instances)",
            "config": {"workload": f"alpha 0.75, N in {list(Ns)}, three copies per node, I=20 x J=20, 64 runs, "
                                   f"swap every 50 sweeps"},
            "kernels": rows}
    print(json.dumps(line))


def run_membw(args):
    """Read ceilings of L2 and HBM from the library's read probe
    (pt2d_diag_read_bandwidth): 16-byte loads cached in L2 only, 8 CTAs of 256
    threads per SM, over buffers of 24, 48 and 96 MB (L2-resident after a
    warm-up pass; L2 is 129 MB) and of 8 GB (HBM).  GB/s = bytes x passes /
    time, best of three timings; the ceilings against which the L2 and HBM
    traffic of the sweep kernels (from ncu) is judged."""
    if int(os.environ.get("RANK", "0")) != 0:
        return  # a one-GPU workload
    import torch

    import paper_2506_14781_gb300 as pt

    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    res = {}
    for mb, passes in ((24, 2000), (48, 1000), (96, 500), (8192, 6)):
        buf = torch.ones(mb << 20, dtype=torch.uint8, device="cuda")
        pt.diag_read_bandwidth(buf, 2, out)  # warm-up: bring an L2-sized buffer into L2
        best = min(pt.diag_read_bandwidth(buf, passes, out) for _ in range(3))
        res[mb] = (mb << 20) * passes / (best / 1e3) / 1e9
        del buf
    peaks, src = _peaks()
    line = {
        "metric": "read bandwidth ceilings: L2-resident buffers and HBM (project read probe)",
        "value": max(res[m] for m in (24, 48, 96)), "unit": "GB/s", "n_gpus": 1, "higher_is_better": True,
        "data": "device buffers of ones",
        "config": {"workload": "pt2d_diag_read_bandwidth over 24, 48, 96 MB and 8 GB, best of 3"},
        "l2_read_gbs": {f"{m} MB": res[m] for m in (24, 48, 96)},
        "hbm_read_gbs": res[8192],
        "hbm_copy_gbs_measured": peaks.get("hbm_gbs"), "peaks_source": src,
    }
    print(json.dumps(line))


def run_serving(args):
    """Serving workload: a Poisson stream of constrained Ising requests at
    `--rates` requests per minute for `--duration` seconds each, then up to
    `--drain` seconds to finish what was admitted.  A request is a planted
    Wishart problem (N uniform on 50..800, alpha uniform on [0.25, 0.75], <= 3
    original edges per copy) with an I = 16 x J = 8 grid, run until its
    bottom-right replica is feasible at its target energy or 5 x 10^4 sweeps.
    `--serve-stops` lists the targets, each a separate pass over every rate:
    "planted" (f <= E_planted, the target the metric names) and "rho0.1" (f <=
    E_planted + 0.1 N s, residual energy per spin <= 0.1, so that latency is
    the time to that residual and solves/s counts the requests reaching it).
    At most `--max-requests` requests are resident (they share the GPU in one
    batched launch per step); the rest wait in FIFO order.  Problems are drawn
    from 256 pre-generated instances, each request with its own seed, so
    instance generation stays out of the timed loop."""
    if int(os.environ.get("RANK", "0")) != 0:
        return  # a one-GPU workload: under torchrun the other ranks do no work
    import torch  # noqa: F401  (CUDA context for the library)

    import paper_2506_14781_gb300 as pt
    import synth

    specs = synth.request_specs(256, 5)
    pool = []
    for N, alpha, seed in specs:
        inst = synth.wishart_planted(N, alpha, seed)
        phys = pt.sparsify(inst.Jq, "max_edges", 3)
        pool.append((inst, phys, synth.beta_ladder(16, BETA_MIN, BETA_MAX, inst.scale),
                     synth.penalty_ladder(8, P_MIN, P_MAX, 32767)))
    max_sweeps, interval = 50000, 50
    results = []
    for stop in args.serve_stops:
        for rate in args.rates:
            results.append(_serve_load(pt, synth, pool, stop, rate, max_sweeps, interval, args))
    line = {
        "metric": "serving p50/p99 latency and solves/sec", "value": results[0]["solves_per_s"],
        "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
        "config": {"workload": "Poisson stream of planted Wishart requests, N~U[50,800], "
                               "alpha~U[0.25,0.75], <=3 edges/copy, I=16 x J=8, stop at g=0 + "
                               "target energy or 5e4 sweeps", "duration_s": args.duration,
                   "drain_s": args.drain, "events_per_step": args.events_per_step,
                   "swap_interval": interval, "pool_gb": args.pool_gb,
                   "max_resident": args.max_requests, "stops": list(args.serve_stops)},
        "loads": results,
    }
    print(json.dumps(line))


def _serve_load(pt, synth, pool, stop, rate, max_sweeps, interval, args):
    """One offered load: Poisson arrivals for `duration` s, then drain."""
    arrivals = synth.poisson_arrivals(rate, args.duration, 5 + int(rate))
    rng = np.random.default_rng(int(rate))
    picks = rng.integers(0, len(pool), arrivals.size)

    def target(inst):
        if stop == "planted":
            return int(inst.E_planted)
        return int(inst.E_planted) + int(np.floor(0.1 * inst.N * inst.scale))

    srv = pt.Server(args.pool_gb << 30, 3, args.max_requests, interval, args.events_per_step)
    ids = []
    t0 = time.perf_counter()
    nxt = 0
    steps = 0
    pool_bytes = args.pool_gb << 30
    free0 = srv.free_bytes
    peak_used, peak_active = 0, 0
    while True:
        now = time.perf_counter() - t0
        while nxt < arrivals.size and arrivals[nxt] <= now:
            inst, phys, beta, P = pool[picks[nxt]]
            ids.append((srv.submit(phys, beta, P, 77 + nxt, target(inst), max_sweeps), picks[nxt]))
            nxt += 1
        if now > args.duration + args.drain:
            break
        active, queued, _ = srv.step()
        steps += 1
        peak_active = max(peak_active, active)
        peak_used = max(peak_used, free0 - srv.free_bytes)
        if active == 0 and queued == 0:
            if nxt >= arrivals.size:
                break
            time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    lat, wait, service, rho, solved_lat, solved, done, updates = [], [], [], [], [], 0, 0, 0
    executed = 0  # sweeps of every admitted request, finished or still resident at the end
    for rid, k in ids:
        st = srv.status(rid)
        inst, phys = pool[k][0], pool[k][1]
        if st["state"] in ("done", "running"):
            executed += phys.n * 128 * st["sweeps_done"]
        if st["state"] == "done":
            done += 1
            lat.append(st["t_done"] - st["t_submit"])
            wait.append(st["t_admit"] - st["t_submit"])
            service.append(st["t_done"] - st["t_admit"])
            if st["solved_event"] >= 0:
                solved += 1
                solved_lat.append(st["t_done"] - st["t_submit"])
            updates += phys.n * 128 * st["sweeps_done"]
            if st["best_event"] >= 0:
                rho.append((st["best_f"] - inst.E_planted) / (inst.N * inst.scale))
    srv.close()

    def pct(v, q):
        return float(np.percentile(np.array(v), q)) if v else None

    return {
        "stop": stop, "rate_per_min": rate, "submitted": len(ids), "completed": done, "solved": int(solved),
        "unfinished_at_end": len(ids) - done, "wall_s": wall, "steps": steps,
        "p50_latency_s": pct(lat, 50), "p99_latency_s": pct(lat, 99),
        "p50_latency_solved_s": pct(solved_lat, 50), "p99_latency_solved_s": pct(solved_lat, 99),
        "p50_queue_wait_s": pct(wait, 50), "p50_service_s": pct(service, 50),
        "solves_per_s": solved / wall, "completed_per_s": done / wall,
        "completed_per_min": 60.0 * done / wall,
        "spin_updates_per_s_completed": updates / wall,
        "spin_updates_per_s_executed": executed / wall,
        "median_best_residual_per_spin": pct(rho, 50),
        "resident_peak": int(peak_active), "memory_admitted_peak_bytes": int(peak_used),
        "pool_bytes": int(pool_bytes),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sweeps", type=int, default=100, help="oracle sample, N=200 workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="n200", choices=["n200", "n800", "batched", "serving", "compare", "fig2", "constrained", "membw", "threecopy", "adaptive"])
    ap.add_argument("--fig2-events", type=int, default=8000)
    ap.add_argument("--cmp-events", type=int, default=2000)
    ap.add_argument("--cmp-instances", type=int, default=64)
    ap.add_argument("--cmp-sparsify", default="max_edges3", choices=["max_edges3", "fixed3"])
    ap.add_argument("--cmp-ns", type=int, nargs="+", default=[20, 30, 40, 50])
    ap.add_argument("--col-vertices", type=int, default=2000, help="constrained: vertices of the cubic graph")
    ap.add_argument("--threecopy-ns", type=int, nargs="+", default=[50, 100])
    ap.add_argument("--rates", type=float, nargs="+", default=[100.0, 1000.0, 5000.0])
    ap.add_argument("--serve-stops", nargs="+", default=["planted", "rho0.1"], choices=["planted", "rho0.1"])
    ap.add_argument("--duration", type=float, default=30.0)
    ap.add_argument("--drain", type=float, default=30.0)
    ap.add_argument("--events-per-step", type=int, default=20)
    ap.add_argument("--pool-gb", type=int, default=16)
    ap.add_argument("--max-requests", type=int, default=128, help="serving: most resident requests")
    ap.add_argument("--instances", type=int, default=1024)
    ap.add_argument("--runs", type=int, default=0, help="override the workload's run count")
    ap.add_argument("--tts-events", type=int, default=160,
                    help="batched: events (of 50 sweeps) the batch runs for time to target")
    ap.add_argument("--tts-sweeps", type=int, default=20000,
                    help="default workload: sweeps the timed runs continue to for time to target")
    ap.add_argument("--batched-events", type=int, default=4, help="batched leg: timed batched events")
    ap.add_argument("--plain-events", type=int, default=2,
                    help="batched legs: timed events of the one-context-per-instance form")
    ap.add_argument("--gs-ns", type=int, nargs="+", default=[20])
    ap.add_argument("--gs-instances", type=int, default=256)
    ap.add_argument("--gs-events", type=int, default=2000)
    ap.add_argument("--gs-timed-events", type=int, default=20)
    ap.add_argument("--ad-ns", type=int, nargs="+", default=[100, 200])
    ap.add_argument("--ad-instances", type=int, default=64)
    ap.add_argument("--ad-events", type=int, default=2000)
    ap.add_argument("--ad-chains", type=int, default=64)
    ap.add_argument("--ad-mcs", type=int, default=500)
    ap.add_argument("--ad-sigma-min", type=float, default=1.0)
    ap.add_argument("--legs", default="all", choices=["all", "none"],
                    help="default workload: also measure time to target, the batched vs plain forms "
                         "and the ground-state leg (outside the timed region), or not")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "compare":
        run_compare(args)
    elif args.workload == "fig2":
        run_fig2(args)
    elif args.workload == "constrained":
        run_constrained(args)
    elif args.workload == "membw":
        run_membw(args)
    elif args.workload == "threecopy":
        run_threecopy(args)
    elif args.workload == "adaptive":
        run_adaptive(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
