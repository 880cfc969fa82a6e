#!/usr/bin/env python
"""Benchmark of the VeST coordinate-descent hot path on the Zipf workload.

Workload (default): 3-order 100,000^3 tensor, 1e7 observed entries with
Zipf(1.2) indices per mode, FP32 values from a planted sparse Tucker model,
ranks (10, 10, 10), L_F lambda = 0.01; the fitted model starts U(0,1) dense.

One step = one iteration of Algorithm 2, the whole path: factor sweep over
every mode, core sweep, loss, responsibility scores, and the prune at
pr = 0.01 (the schedule's first rate, 1 % of each segment's unpruned
elements).  value = (order * nnz) entry-mode updates per second of whole
steps, all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

Other workloads: uniform_1e4x4_5e7 (4-order, 5e7 entries, L_1), batch_256_jobs
(independent jobs, batched against one at a time), serve_200rps (a request
trace, p50/p99 latency), scalability (iteration time against order, mode size
and entry count) and sparsity_curve (RE and held-out RE against the target
sparsity).  --impl reference times the FP64 oracle on the host instead.

With N > 1 (torchrun, one rank per GPU) every rank fits its own independent
instance of the workload (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1904_02603_gb300 import datagen  # noqa: E402

METRIC = "CD-sweep nnz-updates/s"
UNIT = "entry-mode updates/s"
PRUNE_RATE = 0.01  # pr_1 = min(0.01 t, 0.1) at t = 1 (Algorithm 2)
BATCH = "batch_256_jobs"
SERVE = "serve_200rps"
SCALABILITY = "scalability"
SPARSITY = "sparsity_curve"
FP32_LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="vest", choices=["vest", "reference"])
    p.add_argument("--workload", default="zipf_1e5x3_1e7", choices=sorted(datagen.WORKLOADS) + [BATCH, SERVE, SCALABILITY, SPARSITY],
                   help=f"{BATCH}: 256 independent jobs (jobs/s); {SERVE}: a request trace (p50/p99 latency); "
                        f"{SCALABILITY}: iteration time against order, mode size and entry count; "
                        f"{SPARSITY}: training and held-out error against the target sparsity")
    p.add_argument("--duration", type=float, default=5.0, help=f"{SERVE}: seconds of Poisson arrivals")
    p.add_argument("--streams", type=int, default=16, help="stream slots of the batched and served forms")
    p.add_argument("--autosearch", type=int, default=0,
                   help="after the timed steps, run vest_autosearch (Algorithm 2, VeST_auto) for up to this many "
                        "iterations from the initial model and report it")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--profile", default=None, choices=["sweep", "iteration"],
                   help="run a short fixed sequence for an ncu capture instead of the benchmark: build the "
                        "workload's index, then --steps factor sweeps of mode 0 (sweep) or --steps calls of "
                        "vest_iteration with pr = 0.01 (iteration); no timing, no JSON line")
    p.add_argument("--start", default="init", choices=["init", "pruned"],
                   help="init: the U(0,1) start of Algorithm 2; pruned: 5 sweeps, then 90%% of every segment "
                        "pruned by responsibility (the sparse state where the HBM roofline applies)")
    p.add_argument("--accuracy-sweeps", type=int, default=20,
                   help="sweeps of the FP32-against-FP64 GPU comparison after the timed region (0: skip)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline")
    p.add_argument("--cpu-all-cores", type=int, default=1,
                   help="1: also time the oracle on every host core (one process per core, own samples)")
    return p.parse_args()


def workload_config(w: datagen.Workload, extra=None):
    c = {"workload": w.name, "dims": list(w.dims), "ranks": list(w.ranks), "nnz": w.nnz, "index_dist": w.dist,
         "zipf_s": w.zipf_s if w.dist == "zipf" else None, "reg": w.reg, "lambda": w.lam,
         "core_density_planted": w.core_density, "factor_density_planted": w.factor_density, "noise": w.noise,
         "init": "U(0,1) dense (the random start of Algorithm 2)", "data_seed": w.data_seed, "init_seed": w.init_seed}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------ CPU oracle timing
def sample_problem(t: datagen.SparseTensor, n: int, seed: int = 0):
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(t.nnz, size=min(n, t.nnz), replace=False))
    return t.idx[:, sel], t.val[sel].astype(np.float64)


def oracle_step_time(t, st, n_sample: int, reg: int, lam: float):
    """One full oracle iteration (factor sweep, core sweep, loss, responsibility, prune) on a sample."""
    import oracle as O
    idx, x = sample_problem(t, n_sample)
    prob = O.Problem(t.dims, idx, x)
    om = O.Model([f.astype(np.float64) for f in st.factors], st.core.astype(np.float64))
    t0 = time.perf_counter()
    O.sweep_factors(prob, om, reg, lam, -1)
    O.sweep_core(prob, om, reg, lam)
    O.loss(prob, om, reg, lam)
    df, dc, _, _ = O.responsibility(prob, om)
    O.prune(om, df, dc, PRUNE_RATE)
    return time.perf_counter() - t0, prob.nnz


def _oracle_worker(job):
    """One full oracle iteration on one sample, in its own process (spawned): (seconds, entries)."""
    import oracle as O
    dims, idx, x, factors, core, reg, lam = job
    prob = O.Problem(dims, idx, x)
    om = O.Model([f.astype(np.float64) for f in factors], core.astype(np.float64))
    t0 = time.perf_counter()
    O.sweep_factors(prob, om, reg, lam, -1)
    O.sweep_core(prob, om, reg, lam)
    O.loss(prob, om, reg, lam)
    df, dc, _, _ = O.responsibility(prob, om)
    O.prune(om, df, dc, PRUNE_RATE)
    return time.perf_counter() - t0, prob.nnz


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_rate_all_cores(t, st, w, target_seconds: float, single_rate: float, procs: int | None = None):
    """The oracle, unchanged, on every host core at once: one process per core, each running one
    full iteration on its own sample of the workload (independent problems, as the paper's threads
    take independent rows).  Rate = all processes' entry-mode updates / the slowest process's
    time.  The processes are spawned (never forked after the GPU was used)."""
    import multiprocessing as mp
    procs = procs or host_cores()
    reg = 0 if w.reg == "LF" else 1
    n = int(min(t.nnz, max(1000, single_rate * target_seconds / len(t.dims))))
    jobs = []
    for i in range(procs):
        idx, x = sample_problem(t, n, seed=100 + i)
        jobs.append((t.dims, idx, x, st.factors, st.core, reg, w.lam))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_worker, jobs)
    slowest = max(dt for dt, _ in res)
    return len(t.dims) * sum(k for _, k in res) / slowest, procs, n, slowest


def oracle_rate(t, st, w, target_seconds: float):
    reg = 0 if w.reg == "LF" else 1
    probe_n = 4000
    dt, n = oracle_step_time(t, st, probe_n, reg, w.lam)
    n_target = int(min(t.nnz, max(probe_n, probe_n * target_seconds / max(dt, 1e-3))))
    dt, n = oracle_step_time(t, st, n_target, reg, w.lam)
    return len(t.dims) * n / dt, n, dt


def run_reference(args):
    """The oracle as it stands, timed on the host cores, on bounded samples of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload not in datagen.WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the one-tensor workloads only"}))
        return
    w = datagen.WORKLOADS[args.workload]
    # the inputs are the same numbers either way; a device only forms the planted values faster
    dev = None
    try:
        import torch
        dev = "cuda" if torch.cuda.is_available() else None
    except ImportError:
        pass
    t, st, _ = datagen.make(w, device=dev)
    reg = 0 if w.reg == "LF" else 1
    per_step = min(10.0, 150.0 / max(args.steps + args.warmup, 1))
    dt, n = oracle_step_time(t, st, 4000, reg, w.lam)
    n_sample = int(min(t.nnz, max(4000, 4000 * per_step / max(dt, 1e-3))))
    # every host core at once: one spawned process per core, each a full iteration on its own sample
    import multiprocessing as mp
    procs = host_cores()
    jobs = []
    for i in range(procs):
        idx, x = sample_problem(t, n_sample, seed=i)
        jobs.append((t.dims, idx, x, st.factors, st.core, reg, w.lam))
    times = []
    with mp.get_context("spawn").Pool(procs) as pool:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, jobs)
            if k >= args.warmup:
                times.append(time.perf_counter() - t0)
    total = sum(times)
    units = len(t.dims) * sum(e for _, e in res)
    value = args.steps * units / total
    sample = (f"{procs} processes (one per host core), each one full iteration per step on its own {n_sample} "
              f"entries drawn uniformly from the workload's {t.nnz} (same dims, ranks, values, init)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, {"sample_entries": n_sample * procs,
                                          "parallelism": f"{procs} host processes"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
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
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index_for_smi(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


# ------------------------------------------------------------------ replicas (weak scaling)
def replica_seeds(w: datagen.Workload, rank: int):
    """Every rank fits its own instance of the workload: data and init seeds offset by the rank."""
    return w.data_seed + rank, w.init_seed + rank


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time: all ranks run the same steps, the job ends with the last."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    tt = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(world: int, units_per_step: int, steps: int, ms: float) -> float:
    """Units all ranks processed per second (each rank runs its own replica of the workload)."""
    return world * units_per_step * steps / (ms / 1e3)


def precision_gap(w: datagen.Workload, sweeps: int, data=None) -> dict:
    """The FP32 path against the FP64 GPU path on the same data and from the same start.

    The tensor values and the initial model are the FP32 numbers of the workload, cast up for the
    FP64 run, so both runs start from identical values.  Each sweep is the factor sweep over every
    mode followed by the core sweep (no pruning); the objective (Eq. 1 / Eq. 2) and RE (Eq. 4) are
    taken after every sweep.  Returns the per-sweep relative objective gap |f32 - f64| / f64, the
    RE gap, the largest relative factor and core differences after the last sweep, and the FP64
    objective's relative change over the last sweep (how far from convergence the comparison is)."""
    import torch

    from paper_1904_02603_gb300 import vest as V
    t, st = data if data is not None else datagen.make(w, device="cuda")[:2]
    reg = V.REG_LF if w.reg == "LF" else V.REG_L1
    idx = torch.from_numpy(np.ascontiguousarray(t.idx)).cuda()
    v32 = torch.from_numpy(np.ascontiguousarray(t.val.astype(np.float32))).cuda()
    st32 = st.astype(np.float32)
    runs = {}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        ix = V.vest_build_index(V.Tensor(t.dims, idx, v32.to(dt)))
        m = V.Model.from_host(st32, dtype=dt)
        sc = V.make_scratch(ix, m)
        losses = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(sweeps):
            V.vest_sweep_factors(ix, m, reg, w.lam, -1, sc)
            V.vest_sweep_core(ix, m, reg, w.lam, sc)
            losses.append(V.vest_loss(ix, m, reg, w.lam, sc))
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        f, c, _, _ = m.to_host()
        runs[name] = {"loss": torch.stack(losses).cpu().numpy(), "factors": f, "core": c, "s_per_sweep": sec / sweeps}
        del ix, m, sc
        torch.cuda.empty_cache()
    o32, o64 = runs["f32"]["loss"][:, 3], runs["f64"]["loss"][:, 3]
    r32, r64 = runs["f32"]["loss"][:, 4], runs["f64"]["loss"][:, 4]

    def rel(a, b):
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))

    gap = np.abs(o32 - o64) / np.abs(o64)
    return {"workload": w.name, "sweeps": sweeps, "reg": w.reg, "lambda": w.lam,
            "rel_obj_gap": gap.tolist(), "final_rel_obj_gap": float(gap[-1]), "max_rel_obj_gap": float(gap.max()),
            "re_gap": (np.abs(r32 - r64) / np.abs(r64)).tolist(),
            "obj_f64": o64.tolist(), "re_f64": r64.tolist(),
            "f64_last_sweep_rel_change": float(abs(o64[-1] - o64[-2]) / o64[-2]) if sweeps > 1 else None,
            "factor_rel_gap": max(rel(a, b) for a, b in zip(runs["f32"]["factors"], runs["f64"]["factors"])),
            "core_rel_gap": rel(runs["f32"]["core"], runs["f64"]["core"]),
            "s_per_sweep": {"f32": runs["f32"]["s_per_sweep"], "f64": runs["f64"]["s_per_sweep"]}}


def profiled_traffic(workload: str, tensor_cores: bool):
    """DRAM bytes per launch of the factor-sweep task kernel from the committed ncu summary of this
    workload (the tensor-core kernel's summary on the FP32 path, the FMA kernel's otherwise).

    The summary records the files it was taken from and a hash of each; once one changes the
    counters no longer describe the kernel and the traffic is reported as null."""
    name = "sweep_task_tc_kernel" if tensor_cores else "sweep_task_kernel"
    path = os.path.join(ROOT, "profiles", f"{name}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None, f"no ncu summary for {name} on this workload"
    fields = dict(line.split(":", 1) for line in text.splitlines()
                  if line.startswith(("source_sha256_16:", "sources:", "dram_bytes_per_launch:")))
    if len(fields) != 3:
        return None, "ncu summary lacks sources, source hash or traffic"
    want = fields["source_sha256_16"].split()
    srcs = [os.path.join(ROOT, "paper_1904_02603_gb300", "csrc", f) for f in fields["sources"].split()]
    have = [hashlib.sha256(open(f, "rb").read()).hexdigest()[:16] if os.path.exists(f) else "-" for f in srcs]
    if want != have:
        return None, "kernel sources changed since the ncu capture"
    return float(fields["dram_bytes_per_launch"]), f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {path[len(ROOT) + 1:]}"


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ batched jobs
BATCH_SWEEPS = 10


def main_batch(args):
    """256 independent jobs, 10 sweeps each: the batched form (one graph per job, replayed over
    a pool of streams) against the plain form (one job after another, every call launched as it
    goes).  A step is the whole batch; value = jobs per second."""
    import torch

    from paper_1904_02603_gb300 import batch as B
    from paper_1904_02603_gb300 import build as Bd
    from paper_1904_02603_gb300 import vest as V
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return  # the batched workload runs on one GPU
    torch.cuda.set_device(0)
    Bd.build()
    V.load()
    ws = datagen.batch_workloads()
    t0 = time.perf_counter()
    specs = []
    for w in ws:
        t, st, _ = datagen.make(w, device="cuda")
        specs.append((t, st, V.REG_LF, w.lam))
    gen_s = time.perf_counter() - t0
    plain = B.prepare(specs)
    batched = B.prepare(specs)
    entries = sum(w.nnz for w in ws)
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    steps, warm = max(1, args.steps), max(1, args.warmup)
    for _ in range(warm):
        B.run_plain(plain, BATCH_SWEEPS)
    plain_ms = timed(lambda: B.run_plain(plain, BATCH_SWEEPS), steps)
    captured0 = V.vest_launch_count()
    run = B.BatchedRun(batched, BATCH_SWEEPS, n_streams=args.streams)
    per_replay = V.vest_launch_count() - captured0  # kernels recorded in the graphs, launched by every replay
    for _ in range(warm):
        run.replay()
    clocks = ClockSampler(gpu_index_for_smi(0))
    time.sleep(0.5)
    batched_ms = timed(run.replay, steps)
    launches = per_replay * steps
    # the autotuned batched form: per shape class, the faster kernel for Eq. 11 from trial sweeps
    tuned = B.prepare(specs)
    t_tune = time.perf_counter()
    table = B.autotune(tuned)
    tune_s = time.perf_counter() - t_tune
    captured1 = V.vest_launch_count()
    run_t = B.BatchedRun(tuned, BATCH_SWEEPS, n_streams=args.streams)
    launches = (V.vest_launch_count() - captured1) * steps  # the timed (autotuned) replays
    for _ in range(warm):
        run_t.replay()
    tuned_ms = timed(run_t.replay, steps)
    clk = clocks.stop()
    choices = [v["path"] for v in table.values()]
    # e2e: host inputs of one job copied in, indexed, swept and its loss read back, job by job
    # (the serving path a caller without resident data takes)
    idx_h = [torch.from_numpy(t.idx).pin_memory() for t, _, _, _ in specs[:32]]
    val_h = [torch.from_numpy(t.val).pin_memory() for t, _, _, _ in specs[:32]]
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    h2d = d2h = 0
    for (t, st, reg, lam), ih, vh in zip(specs[:32], idx_h, val_h):
        ten = V.Tensor(t.dims, ih.to("cuda", non_blocking=True), vh.to("cuda", non_blocking=True))
        job = B.prepare([(t, st, reg, lam)])[0]
        ixe = V.vest_build_index(ten)
        job = B.Job(ten, job.model, ixe, job.scratch, reg, lam)
        B.sweeps(job, BATCH_SWEEPS)
        loss = V.vest_loss(ixe, job.model, reg, lam, job.scratch).cpu()
        h2d += ih.numel() * ih.element_size() + vh.numel() * vh.element_size()
        d2h += loss.numel() * loss.element_size()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t_e
    line = {
        "metric": "jobs/s (batched factorisations, 10 sweeps each)", "value": len(ws) / (tuned_ms / 1e3),
        "unit": "jobs/s", "n_gpus": 1, "steps": steps, "warmup": warm, "ms_per_step": tuned_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCH, "jobs": len(ws), "sweeps": BATCH_SWEEPS, "entries": entries,
                   "streams": args.streams,
                   "form": "one CUDA graph per job, replayed round-robin over streams; the kernel for Eq. 11 "
                           "chosen per shape class by the autotuner (batch.autotune)",
                   "l2": "the batch's CSR arrays and factors (several GB) exceed the 129 MB L2",
                   "input_generation_s": gen_s},
        "plain": {"value": len(ws) / (plain_ms / 1e3), "unit": "jobs/s", "ms_per_step": plain_ms,
                  "form": "one job after another on one stream, each call launched as it goes"},
        "untuned": {"value": len(ws) / (batched_ms / 1e3), "unit": "jobs/s", "ms_per_step": batched_ms,
                    "form": "the same graphs with the library's default kernel choice (tensor cores wherever they "
                            "apply)"},
        "autotune": {"classes": len(table), "tensor_core_classes": sum(1 for c in choices if c == V.DELTA_AUTO),
                     "fma_classes": sum(1 for c in choices if c == V.DELTA_FMA), "seconds": tune_s},
        "speedup_vs_plain": plain_ms / tuned_ms,
        "entry_mode_updates_per_s": sum(w.nnz * len(w.dims) for w in ws) * BATCH_SWEEPS / (tuned_ms / 1e3),
        "e2e": {"value": 32 / e2e_s, "unit": "jobs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "includes": "32 jobs one by one: H2D of idx+val, index build, 10 sweeps, D2H of the loss"},
        "clocks": clk,
        "gpu_launches": launches,
        "gpu_launches_note": "kernels recorded in the jobs' graphs times the timed replays",
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving
def main_serve(args):
    """A Poisson trace at 200 requests/s, half factorisation jobs (drawn as in the batched
    configuration, 10 sweeps each) and half completion queries (1..1e5 tuples, log-uniform)
    against resident models, served by the continuous-batching loop under a 150 GB budget and,
    for comparison, one request at a time."""
    import torch

    from paper_1904_02603_gb300 import build as Bd
    from paper_1904_02603_gb300 import serve as S
    from paper_1904_02603_gb300 import vest as V
    if int(os.environ.get("RANK", "0")) != 0:
        return  # the serving workload runs on one GPU
    torch.cuda.set_device(0)
    Bd.build()
    V.load()
    specs = []
    for w in datagen.batch_workloads():
        t, st, _ = datagen.make(w, device="cuda")
        specs.append((t, st, V.REG_LF, w.lam))
    trace = S.make_trace(specs, rate=200.0, duration=args.duration)
    warm = S.make_trace(specs, rate=200.0, duration=0.3, seed=99)
    server = S.Server(specs, budget_bytes=150 << 30, slots=args.streams)
    server.serve(warm)
    clocks = ClockSampler(gpu_index_for_smi(0))
    time.sleep(0.5)
    launches0 = V.vest_launch_count()
    server.serve(trace)
    launches = V.vest_launch_count() - launches0
    clk = clocks.stop()
    served = S.latency_stats(trace)
    base_trace = S.make_trace(specs, rate=200.0, duration=args.duration)
    base = S.latency_stats(S.serve_one_at_a_time(S.Server(specs, slots=1), base_trace))
    h2d = sum(specs[r.spec][0].idx.nbytes + specs[r.spec][0].val.nbytes if r.kind == "job" else r.q_idx.nbytes
              for r in trace)
    d2h = sum(40 if r.kind == "job" else 4 * r.q_idx.shape[1] for r in trace)
    line = {
        "metric": "p99 latency (continuous batching, 200 req/s)", "value": served["p99_ms"], "unit": "ms",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": served["span_s"] * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": SERVE, "rate_per_s": 200, "duration_s": args.duration, "job_fraction": 0.5,
                   "slots": args.streams, "hbm_budget_gb": 150, "sweeps_per_job": 10,
                   "l2": "each job's inputs are copied in from host memory; the batch exceeds the 129 MB L2"},
        "served": served, "one_at_a_time": base,
        "p50_ms": served["p50_ms"], "jobs_per_s": served["jobs_per_s"],
        "e2e": {"value": served["p99_ms"], "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "includes": "every request from its arrival: H2D of its inputs, index build, sweeps or "
                            "reconstruction, D2H of its result"},
        "clocks": clk, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ scalability series
def loglog_slope(xs, ys) -> float:
    lx, ly = np.log(np.asarray(xs, np.float64)), np.log(np.asarray(ys, np.float64))
    return float(np.polyfit(lx, ly, 1)[0]) if len(xs) > 1 else float("nan")


def main_scalability(args):
    """The data-scalability series of Section 4.4 on one GPU: one Algorithm 2 iteration (factor
    sweep, core sweep, loss, responsibility, prune at pr = 0.01) timed at every point of three
    series (order 3..10; mode size 1e3..1e8 with |Omega| = I; |Omega| 1e3..1e7), ranks 3, values
    U(0,1), FP32.  value = entry-mode updates/s at the largest point (I = |Omega| = 1e8)."""
    import torch

    from paper_1904_02603_gb300 import build as Bd
    from paper_1904_02603_gb300 import vest as V
    if int(os.environ.get("RANK", "0")) != 0:
        return  # the series runs on one GPU
    torch.cuda.set_device(0)
    Bd.build()
    V.load()
    stream = torch.cuda.current_stream()
    steps, warm = max(1, min(args.steps, 5)), max(1, min(args.warmup, 3))
    lam = 0.01
    pts, launches, cpu_pts, cpu_total = [], 0, [], 0.0
    clocks = ClockSampler(gpu_index_for_smi(0))
    for k, (series, order, dim, nnz) in enumerate(datagen.scalability_points()):
        t, st = datagen.uniform_tensor(order, dim, nnz, seed=3000 + k)
        ten = V.Tensor.from_host(t)
        mdl = V.Model.from_host(st)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ix = V.vest_build_index(ten)
        e1.record(stream)
        torch.cuda.synchronize()
        index_ms = e0.elapsed_time(e1)
        sc = V.make_scratch(ix, mdl)
        for _ in range(warm):
            V.vest_iteration(ix, mdl, V.REG_LF, lam, PRUNE_RATE, sc)
        torch.cuda.synchronize()
        l0 = V.vest_launch_count()
        e0.record(stream)
        for _ in range(steps):
            loss, _, _, _ = V.vest_iteration(ix, mdl, V.REG_LF, lam, PRUNE_RATE, sc)
        e2.record(stream)
        torch.cuda.synchronize()
        n_launch = V.vest_launch_count() - l0
        launches += n_launch
        ms = e0.elapsed_time(e2) / steps
        re = float(loss.cpu().numpy()[4])
        pts.append({"series": series, "order": order, "dim": dim, "nnz": nnz, "ms_per_iteration": ms,
                    "index_build_ms": index_ms, "updates_per_s": order * nnz / (ms / 1e3),
                    "launches_per_iteration": n_launch // steps, "re_after": re})
        del ix, sc, mdl, ten
        torch.cuda.empty_cache()
    clk = clocks.stop()
    # the oracle on the order series, cheapest points first, within the CPU time budget
    if not args.no_cpu_baseline:
        for k, (series, order, dim, nnz) in enumerate(datagen.scalability_points()):
            if series != "order" or cpu_total * 4 > args.cpu_seconds:
                continue
            t, st = datagen.uniform_tensor(order, dim, nnz, seed=3000 + k)
            dt, _ = oracle_step_time(t, st.astype(np.float64), nnz, 0, lam)
            cpu_total += dt
            cpu_pts.append({"order": order, "dim": dim, "nnz": nnz, "ms_per_iteration": dt * 1e3})
    slopes = {}
    for series, key in (("order", "order"), ("dims", "dim"), ("nnz", "nnz")):
        s_pts = [p for p in pts if p["series"] == series]
        top = s_pts[len(s_pts) // 2:]
        slopes[series] = {"all": loglog_slope([p[key] for p in s_pts], [p["ms_per_iteration"] for p in s_pts]),
                          "upper_half": loglog_slope([p[key] for p in top], [p["ms_per_iteration"] for p in top])}
    big = max((p for p in pts if p["series"] == "dims"), key=lambda p: p["dim"])
    line = {
        "metric": METRIC, "value": big["updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warm,
        "ms_per_step": big["ms_per_iteration"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": SCALABILITY, "ranks": datagen.SCALABILITY_RANK, "values": "U(0,1)",
                   "index_dist": "uniform", "reg": "LF", "lambda": lam, "init": "U(0,1) dense",
                   "step": "one iteration of Algorithm 2 (vest_iteration, pr=%g)" % PRUNE_RATE,
                   "value_at": "order 3, I = |Omega| = 1e8",
                   "l2": "points up to 1e5 entries fit in L2 (no flush: the series measures the iteration as run)"},
        "series": pts,
        "loglog_slope_ms": slopes,
        "cpu_baseline": {"value": None, "unit": "ms per iteration", "cores": 1, "kind": "oracle",
                         "sample": "one full oracle iteration at each order-series point within the CPU budget",
                         "points": cpu_pts} if cpu_pts else None,
        "clocks": clk, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ sparsity against error
SPARSITY_TARGETS = (0.0, 0.2, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 0.95, 0.99)


def main_sparsity_curve(args):
    """Section 4.3 on planted data: VeST_man at each target sparsity and VeST_auto (the elbow
    rule), for L_F and L_1, fitted on 90 % of the observed entries; RE on the training entries
    and Test RE on the held-out 10 %, both from vest_loss over the respective index.  The Value
    Pruning baseline of Section 4.1 (the s = 0 fit, then the 60 % smallest-magnitude elements of
    every segment removed, no refit) is scored the same way."""
    import torch

    from paper_1904_02603_gb300 import build as Bd
    from paper_1904_02603_gb300 import vest as V
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(0)
    Bd.build()
    V.load()
    w = datagen.SPARSITY_CURVE
    t, st, planted = datagen.make(w, device="cuda")
    train, test = datagen.split_entries(t, 0.1)
    ix_tr = V.vest_build_index(V.Tensor.from_host(train))
    ix_te = V.vest_build_index(V.Tensor.from_host(test))
    truth_zeros = sum(int((f == 0).sum()) for f in planted.factors) + int((planted.core == 0).sum())
    truth_sparsity = truth_zeros / (planted.core.size + sum(f.size for f in planted.factors))
    max_iter = 256  # CD from the U(0,1) start needs a few hundred sweeps on this tensor
    total_elems = planted.core.size + sum(f.size for f in planted.factors)
    curves, launches, total_s = {}, 0, 0.0
    clocks = ClockSampler(gpu_index_for_smi(0))
    # the converged unpruned fit (VeST_man with s = 0 prunes nothing), from which the second set of
    # runs starts: pruning a settled model is where the paper's flat-then-rising RE curve appears
    fits = {}
    for reg_name, reg in (("LF", V.REG_LF), ("L1", V.REG_L1)):
        # plain sweeps (factor sweep, core sweep) until RE changes by less than 1e-6 relative over
        # 50 sweeps, at most 4000: the auto-search's 256-iteration cap is too short from U(0,1)
        fm = V.Model.from_host(st)
        fsc = V.make_scratch(ix_tr, fm)
        t0 = time.perf_counter()
        prev, sweeps, re_now = None, 0, None
        while sweeps < 4000:
            for _ in range(50):
                V.vest_sweep_factors(ix_tr, fm, reg, w.lam, -1, fsc)
                V.vest_sweep_core(ix_tr, fm, reg, w.lam, fsc)
            sweeps += 50
            re_now = float(V.vest_loss(ix_tr, fm, reg, w.lam, fsc)[4].item())
            if prev is not None and abs(prev - re_now) <= 1e-6 * prev:
                break
            prev = re_now
        torch.cuda.synchronize()
        fits[reg_name] = (fm, {"sweeps": sweeps, "re": re_now, "seconds": time.perf_counter() - t0})
        del fsc
    for (reg_name, reg), start in [(rg, sname) for sname in ("init", "fit")
                                   for rg in (("LF", V.REG_LF), ("L1", V.REG_L1))]:
        rows = []
        for target, rise in [(x, 0) for x in SPARSITY_TARGETS] + [(-1.0, 0), (-1.0, 1)]:
            mdl = V.Model.from_host(st) if start == "init" else fits[reg_name][0].clone()
            sc = V.make_scratch(ix_tr, mdl, autosearch=True)
            sc_te = V.make_scratch(ix_te, mdl)
            torch.cuda.synchronize()
            l0 = V.vest_launch_count()
            t0 = time.perf_counter()
            rep = V.vest_autosearch(ix_tr, mdl, V.params(reg=reg, lam=w.lam, target_sparsity=target,
                                                         max_iter=max_iter, elbow_rise=rise), sc)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            launches += V.vest_launch_count() - l0
            total_s += secs
            tr = V.vest_loss(ix_tr, mdl, reg, w.lam, sc).cpu().numpy()
            te = V.vest_loss(ix_te, mdl, reg, w.lam, sc_te).cpu().numpy()
            mode = "man" if target >= 0 else ("auto_rise" if rise else "auto")
            rows.append({"start": start, "target": None if target < 0 else target, "mode": mode,
                         "sparsity": rep["final_sparsity"], "re_train": float(tr[4]), "re_test": float(te[4]),
                         "iters": rep["iters"], "stop_iter": rep["stop_iter"], "seconds": secs})
            if target == 0.0:  # Value Pruning: the unpruned fit, then |value| keys at ratio 0.6
                kf, kc = V.vest_value_keys(mdl)
                V.vest_prune(mdl, kf, kc, 0.6, sc, count_mode=1)
                zeros = int(V.vest_count_zeros(mdl, sc).sum().item())
                tr = V.vest_loss(ix_tr, mdl, reg, w.lam, sc).cpu().numpy()
                te = V.vest_loss(ix_te, mdl, reg, w.lam, sc_te).cpu().numpy()
                rows.append({"start": start, "target": 0.6, "mode": "value_pruning", "sparsity": zeros / total_elems,
                             "re_train": float(tr[4]), "re_test": float(te[4]), "iters": rep["iters"],
                             "stop_iter": 0, "seconds": 0.0})
            del mdl, sc, sc_te
        curves[f"{reg_name}_from_{start}"] = rows
    clk = clocks.stop()
    n_runs = sum(1 for rows in curves.values() for r in rows if r["mode"] != "value_pruning")
    auto = next(r for r in curves["LF_from_fit"] if r["mode"] == "auto")
    line = {
        "metric": "Test RE of VeST_auto (L_F, from the converged fit) on held-out entries", "value": auto["re_test"],
        "unit": "RE",
        "n_gpus": 1, "steps": n_runs, "warmup": 0, "ms_per_step": 1e3 * total_s / n_runs,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": w.dtype, "data": "synthetic",
        "config": {**workload_config(w), "workload": SPARSITY, "tensor": w.name, "test_fraction": 0.1,
                   "max_iter": max_iter, "truth_sparsity": truth_sparsity,
                   "schedule": "pr_t = min(0.01 t, 0.1) of all elements; VeST_man stops pruning at the target, "
                               "VeST_auto at the elbow (threshold 0.05; auto_rise also needs RE to rise); "
                               "value_pruning: the s = 0 fit with the 60 % "
                               "smallest |element| of each segment pruned, no refit"},
        "curves": curves,
        "fits": {k: v[1] for k, v in fits.items()},
        "seconds_total": total_s,
        "clocks": clk, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ profiling driver
def main_profile(args):
    """A short fixed sequence of library calls on the workload, for an ncu capture (the launches
    to capture are selected with ncu's -k / -s / -c)."""
    import torch

    from paper_1904_02603_gb300 import build as Bd
    from paper_1904_02603_gb300 import vest as V
    torch.cuda.set_device(0)
    Bd.build()
    V.load()
    w = datagen.WORKLOADS[args.workload]
    reg = V.REG_LF if w.reg == "LF" else V.REG_L1
    t, st, _ = datagen.make(w, device="cuda")
    ix = V.vest_build_index(V.Tensor.from_host(t))
    m = V.Model.from_host(st)
    sc = V.make_scratch(ix, m)
    for _ in range(args.steps):
        if args.profile == "sweep":
            V.vest_sweep_factors(ix, m, reg, w.lam, 0, sc)
        else:
            V.vest_iteration(ix, m, reg, w.lam, PRUNE_RATE, sc)
    torch.cuda.synchronize()
    print(f"profile run: {args.profile} x {args.steps} on {w.name}, device status {V.vest_device_status()}")


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    if args.profile:
        main_profile(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == BATCH:
        main_batch(args)
        return
    if args.workload == SERVE:
        main_serve(args)
        return
    if args.workload == SCALABILITY:
        main_scalability(args)
        return
    if args.workload == SPARSITY:
        main_sparsity_curve(args)
        return
    import torch
    import torch.distributed as dist

    from paper_1904_02603_gb300 import vest as V

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1904_02603_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    V.load()

    w = datagen.WORKLOADS[args.workload]
    # every rank fits its own instance of the workload (weak scaling)
    ds, iseed = replica_seeds(w, rank)
    t, st, _ = datagen.make(w, device="cuda", data_seed=ds, init_seed=iseed)
    tdt = torch.float64 if w.dtype == "f64" else torch.float32
    reg = V.REG_LF if w.reg == "LF" else V.REG_L1
    ten = V.Tensor.from_host(t)
    mdl = V.Model.from_host(st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    stream = torch.cuda.current_stream()
    N, nnz = len(t.dims), t.nnz
    units_per_step = N * nnz
    start_note = "U(0,1) dense (the random start of Algorithm 2)"
    if args.start == "pruned":
        # the state pruning leads to: a short fit, then 90 % of every segment (each A^(n) and G)
        # pruned by responsibility in one step (count_mode total)
        for _ in range(5):
            V.vest_sweep_factors(ix, mdl, reg, w.lam, -1, sc)
            V.vest_sweep_core(ix, mdl, reg, w.lam, sc)
        dfp, dcp, _, _ = V.vest_responsibility(ix, mdl, sc, with_resp=False)
        V.vest_prune(mdl, dfp, dcp, 0.9, sc, count_mode=1)
        zeros = V.vest_count_zeros(mdl, sc).cpu().numpy()
        size = sum(d * r for d, r in zip(w.dims, w.ranks)) + math.prod(w.ranks)
        start_note = ("5 sweeps from U(0,1), then 90%% of every segment pruned by responsibility "
                      "(sparsity %.3f)" % (float(zeros.sum()) / size))
        f_h, c_h, fm_h, cm_h = mdl.to_host()
        st = datagen.ModelState(f_h, c_h, fm_h, cm_h)  # the oracle baseline and the accuracy run start here too

    def step(model, index, evs=None):
        # one iteration of Algorithm 2: the factor sweep mode by mode (each mode's sweep timed on
        # its own for the roofline), then the core sweep, loss, responsibility and prune in one call
        if evs:
            evs[0].record(stream)
        for n in range(N):
            V.vest_sweep_factors(index, model, reg, w.lam, n, sc)
            if evs:
                evs[1 + n].record(stream)
        loss, _, _, _ = V.vest_iteration(index, model, reg, w.lam, PRUNE_RATE, sc, factor_sweep=False)
        if evs:
            evs[N + 1].record(stream)
        return loss

    def step_separate(model, index, evs):
        # the same iteration through the separate entry points, for the per-operation breakdown
        evs[0].record(stream)
        V.vest_sweep_factors(index, model, reg, w.lam, -1, sc)
        evs[1].record(stream)
        V.vest_sweep_core(index, model, reg, w.lam, sc)
        evs[2].record(stream)
        V.vest_loss(index, model, reg, w.lam, sc)
        evs[3].record(stream)
        df, dc, _, _ = V.vest_responsibility(index, model, sc, with_resp=False)
        evs[4].record(stream)
        V.vest_prune(model, df, dc, PRUNE_RATE, sc)
        evs[5].record(stream)

    for _ in range(args.warmup):
        step(mdl, ix)
    torch.cuda.synchronize()

    ops = [f"sweep_factors_mode{n}" for n in range(N)] + ["core_sweep+loss+responsibility+prune"]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(ops) + 1)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(gpu_index_for_smi(local))
    time.sleep(0.5)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = V.vest_launch_count()
    start.record(stream)
    for k in range(args.steps):
        loss = step(mdl, ix, evs[k])
    end.record(stream)
    torch.cuda.synchronize()
    launches = V.vest_launch_count() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = start.elapsed_time(end)
    op_ms = {op: statistics.mean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps))
             for i, op in enumerate(ops)}
    mode_ms = [op_ms[f"sweep_factors_mode{n}"] for n in range(N)]
    op_ms["sweep_factors"] = sum(mode_ms)
    elapsed_ms = max_over_ranks(elapsed_ms, world)
    value = whole_job_rate(world, units_per_step, args.steps, elapsed_ms)
    final_loss = loss.cpu().numpy().tolist()

    # Algorithm 2 end to end (VeST_auto) from the initial model, after the timed region
    auto = None
    if args.autosearch > 0:
        am = V.Model.from_host(st)
        asc = V.make_scratch(ix, am, autosearch=True)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        rep = V.vest_autosearch(ix, am, V.params(reg=reg, lam=w.lam, max_iter=args.autosearch), asc)
        torch.cuda.synchronize()
        ta = time.perf_counter() - ta
        auto = {"iters": rep["iters"], "stop_iter": rep["stop_iter"], "final_sparsity": rep["final_sparsity"],
                "re": [float(x) for x in rep["re"]], "pr": [float(x) for x in rep["pr"]],
                "sparsity": [float(x) for x in rep["sparsity"]], "seconds": ta,
                "ms_per_iteration": 1e3 * ta / max(rep["iters"], 1),
                "mode": "VeST_auto: pr_t = min(0.01 t, 0.1), elbow threshold 0.05, count_mode total, normalised"}
        del am, asc

    # per-operation breakdown through the separate entry points (after the timed region, on a copy)
    sep_model = mdl.clone()
    sep_evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    step_separate(sep_model, ix, sep_evs)
    torch.cuda.synchronize()
    sep_ms = {op: sep_evs[i].elapsed_time(sep_evs[i + 1])
              for i, op in enumerate(["sweep_factors", "sweep_core", "loss", "responsibility", "prune"])}
    del sep_model

    # ---------------- end to end: host buffers in, loss out, through the public API
    idx_h = torch.from_numpy(t.idx).pin_memory()
    val_h = torch.from_numpy(t.val).pin_memory()
    loss_h = torch.empty(5, dtype=torch.float64).pin_memory()
    e2e_model = mdl.clone()
    h2d = idx_h.numel() * idx_h.element_size() + val_h.numel() * val_h.element_size()
    d2h = loss_h.numel() * loss_h.element_size()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall = time.perf_counter()
    e0.record(stream)
    for _ in range(args.e2e_steps):
        tdev = V.Tensor(t.dims, idx_h.to("cuda", non_blocking=True), val_h.to("cuda", non_blocking=True))
        ixe = V.vest_build_index(tdev)
        le = step(e2e_model, ixe)
        loss_h.copy_(le, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t_wall))
    e2e_ms = max_over_ranks(e2e_ms, world)
    e2e_value = whole_job_rate(world, units_per_step, args.e2e_steps, e2e_ms) if args.e2e_steps > 0 else None

    # ---------------- the FP32 path against the FP64 GPU path (after the timed region)
    accuracy = None
    if w.dtype == "f32" and args.accuracy_sweeps > 0 and rank == 0:
        accuracy = precision_gap(w, args.accuracy_sweeps, (t, st))

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---------------- roofline of the dominant kernel: one mode's factor sweep (task kernel + fix-up)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    probe_buf = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    probed = {"fp32_fma_tflops": V.vest_probe_peak(V.PROBE_FP32_FMA),
              "fp64_fma_tflops": V.vest_probe_peak(V.PROBE_FP64_FMA),
              "tf32_mma_tflops": V.vest_probe_peak(V.PROBE_TF32_MMA),
              "l2_gather_tbs": V.vest_probe_peak(V.PROBE_L2_GATHER, probe_buf),
              "sms": sms,
              "how": "vest_probe_peak: self-timed FMA chains / tcgen05 TF32 MMAs (A in TMEM) / 16-byte L2 gathers "
                     "on every SM, CUDA events, second of two runs, clocks as found"}
    del probe_buf
    fp32_peak = probed["fp32_fma_tflops"]  # TFLOP/s
    # algorithmic work per entry and mode (dense core): delta = |G| + |G|/J_n FMAs, row sums J_n + J_n(J_n+1)/2 FMAs
    G = math.prod(w.ranks)
    s = 4 if w.dtype == "f32" else 8
    flops_mode, bytes_mode = [], []
    for n in range(N):
        Jn = w.ranks[n]
        flops_mode.append(2.0 * nnz * (G + G // Jn + Jn + Jn * (Jn + 1) // 2))
        # per mode: nnz ((N-1) 4 + s_val) + (I_n+1) 8 + 2 I_n J_n s_f + I_n J_n (mask) + sum_{k != n} I_k J_k s_f
        bytes_mode.append(nnz * ((N - 1) * 4 + s) + (w.dims[n] + 1) * 8 + 2 * w.dims[n] * Jn * s
                          + w.dims[n] * Jn + sum(w.dims[k] * w.ranks[k] * s for k in range(N) if k != n))
    launch_s = statistics.mean(mode_ms) / 1e3
    flops_launch, bytes_launch = statistics.mean(flops_mode), statistics.mean(bytes_mode)
    achieved = flops_launch / launch_s / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    traffic, traffic_note = profiled_traffic(args.workload, w.dtype == "f32" and
                                             os.environ.get("VEST_TENSOR_CORES", "1") != "0")
    roofline = {"bound": "alu", "kernel": "vest_sweep_factors, one mode (task kernel, fix-up, row finish), mean over modes",
                "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                "peak_source": "measured: vest_probe_peak FP32 FMA on this GPU (nominal %d SMs x %d lanes x 2 x %.0f MHz"
                               " = %.1f)" % (sms, FP32_LANES_PER_SM, sm_max,
                                            sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12),
                "flops_note": "algorithmic flops of the staged contraction and the row sums (Eq. 10-11), whichever "
                              "unit runs them: on the FP32 path 1000 of the 1100 delta FMAs per entry run on the "
                              "tensor cores in split TF32 (section 6b)",
                "traffic": traffic, "traffic_source": traffic_note,
                "launch_ms": launch_s * 1e3,
                "algorithmic_flops_per_launch": flops_launch, "algorithmic_bytes_per_launch": bytes_launch,
                "hbm_achieved_gbs": bytes_launch / launch_s / 1e9, "hbm_peak_gbs": hbm,
                "hbm_frac": bytes_launch / launch_s / 1e9 / hbm,
                "hbm_peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, n_s, dt = oracle_rate(t, st, w, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one full oracle iteration on {n_s} entries drawn from the workload ({dt:.1f} s)"}
        if args.cpu_all_cores:
            prate, procs, n_p, dt_p = oracle_rate_all_cores(t, st, w, args.cpu_seconds, rate)
            cpu["all_cores"] = {"value": prate, "unit": UNIT, "cores": procs, "kind": "oracle",
                                "sample": f"{procs} processes, each one full oracle iteration on its own sample "
                                          f"of {n_p} entries (slowest {dt_p:.1f} s)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": w.dtype, "data": "synthetic",
        "config": workload_config(w, {"start": start_note,
                                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                      "l2": "inputs larger than L2 (CSR per mode %.0f MB > 129 MB)" %
                                            ((N - 1) * 4 * nnz / 1e6 + s * nnz / 1e6),
                                      "step": "one iteration of Algorithm 2: factor sweep (all modes) + core sweep + "
                                              "loss + responsibility + prune (pr=%g, its first pruning rate)"
                                              % PRUNE_RATE}),
        "op_ms": op_ms,
        "separate_calls_ms": sep_ms,
        "autosearch": auto,
        "sweep_only": {"value": world * units_per_step / (op_ms["sweep_factors"] / 1e3), "unit": UNIT},
        "final_loss": {"sq_err": final_loss[0], "objective": final_loss[3], "re": final_loss[4]},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "peaks_probed": probed,
        "accuracy": accuracy,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": args.e2e_steps, "includes": "H2D of idx+val, vest_build_index, one step, D2H of the loss"},
        "clocks": clk,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
