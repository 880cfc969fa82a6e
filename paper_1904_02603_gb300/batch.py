"""Many independent factorisations on one GPU.

Each job is a tensor, its index, its model and its own scratch buffer.  The plain form runs
the jobs one after another on one stream, every call launching its kernels as it goes.  The
batched form records each job's sweeps once as a CUDA graph on a stream of its own and then
replays the graphs round-robin over a pool of streams, so the small jobs of the mix run side
by side on the GPU's SMs and no host launch overhead sits between their kernels.  An autotuner
picks, per shape class of the job mix, whether the factor sweep's contraction (Eq. 11) runs on
the tensor cores or on FMA kernels, from timed trial sweeps, and keeps the choices in a table.  Every kernel
is deterministic and a job's buffers are its own, so a job's results are bitwise the same
alone, in the plain form and in the batched form.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass

import torch

from . import vest as V


@dataclass
class Job:
    tensor: V.Tensor
    model: V.Model
    index: V.Index
    scratch: torch.Tensor
    reg: int
    lam: float
    path: int = V.DELTA_AUTO  # kernel for Eq. 11 in the factor sweep (set by autotune)


def prepare(specs, device="cuda") -> list[Job]:
    """specs: (SparseTensor, ModelState, reg, lam) per job; builds every index (one sync each)."""
    jobs = []
    for t, st, reg, lam in specs:
        ten = V.Tensor.from_host(t)
        mdl = V.Model.from_host(st)
        ix = V.vest_build_index(ten)
        jobs.append(Job(ten, mdl, ix, V.make_scratch(ix, mdl), reg, lam))
    return jobs


def sweeps(job: Job, iterations: int, stream=None):
    """`iterations` rounds of the factor sweep (every mode) and the core sweep."""
    for _ in range(iterations):
        V.vest_sweep_factors(job.index, job.model, job.reg, job.lam, -1, job.scratch, stream=stream, path=job.path)
        V.vest_sweep_core(job.index, job.model, job.reg, job.lam, job.scratch, stream=stream)


def _bucket(J: int) -> int:
    return 4 if J <= 4 else 8 if J <= 8 else 10 if J <= 10 else 12 if J <= 12 else 16 if J <= 16 else 32


def shape_key(job: Job) -> str:
    """The shape class a tuned choice is shared by: order, the rank buckets the kernels are
    instantiated for, the dtype, and the entry count to the nearest power of two."""
    ranks = "x".join(str(_bucket(r)) for r in job.model.ranks)
    nnz = max(job.tensor.nnz, 1)
    return f"N{job.model.order}_J{ranks}_{str(job.model.core.dtype).replace('torch.', '')}_nnz2^{round(math.log2(nnz))}"


def _time_path(job: Job, path: int, trials: int) -> float:
    """Seconds per factor sweep of one job with `path`, on a copy of its model (the job's own
    model is left as it is); inf when the path does not apply."""
    m = job.model.clone()
    try:
        V.vest_sweep_factors(job.index, m, job.reg, job.lam, -1, job.scratch, path=path)  # warm-up
    except V.VestError:
        return math.inf
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(trials):
        V.vest_sweep_factors(job.index, m, job.reg, job.lam, -1, job.scratch, path=path)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3 / trials


def autotune(jobs: list[Job], table: dict | None = None, cache_path: str | None = None, trials: int = 3) -> dict:
    """Picks, for every shape class, the faster kernel for Eq. 11 (the FMA kernels, or the tensor
    cores wherever they apply) by timing both on the first job of the class, and sets `path` on
    every job of it.  `table` (or the JSON
    file at `cache_path`) holds earlier choices, which are reused without timing; the updated
    table is returned (and written back to `cache_path`).  Both kernels compute the same update
    to within FP32 rounding, so the choice changes speed, not results beyond rounding."""
    table = dict(table or {})
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            table.update(json.load(f))
    for j in jobs:
        key = shape_key(j)
        if key not in table:
            # the tensor-core choice is AUTO (tensor cores on every mode where they apply): jobs of one
            # class share rank buckets, not exact ranks, so a strict choice could fail on another job
            t_fma = _time_path(j, V.DELTA_FMA, trials)
            t_tc = _time_path(j, V.DELTA_AUTO, trials)
            table[key] = {"path": V.DELTA_AUTO if t_tc < t_fma else V.DELTA_FMA,
                          "fma_ms": t_fma * 1e3, "tensor_ms": t_tc * 1e3}
        j.path = table[key]["path"]
    if cache_path:
        with open(cache_path, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return table


def run_plain(jobs: list[Job], iterations: int):
    """One job after another on the current stream."""
    for j in jobs:
        sweeps(j, iterations)


class BatchedRun:
    """Each job's sweeps captured once as a graph on its own stream; `replay()` launches them
    all, job j on stream j mod n_streams, and joins the streams to the current one."""

    def __init__(self, jobs: list[Job], iterations: int, n_streams: int = 16):
        self.jobs = jobs
        self.streams = [torch.cuda.Stream() for _ in range(max(1, n_streams))]
        self.graphs = []
        for j in jobs:
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                    sweeps(j, iterations, stream=s)
            torch.cuda.current_stream().wait_stream(s)
            self.graphs.append(g)

    def replay(self):
        cur = torch.cuda.current_stream()
        for s in self.streams:
            s.wait_stream(cur)
        for i, g in enumerate(self.graphs):
            with torch.cuda.stream(self.streams[i % len(self.streams)]):
                g.replay()
        for s in self.streams:
            cur.wait_stream(s)
