"""Many independent factorisations on one GPU.

Each job is a tensor, its index, its model and its own scratch buffer.  The plain form runs
the jobs one after another on one stream, every call launching its kernels as it goes.  The
batched form records each job's sweeps once as a CUDA graph on a stream of its own and then
replays the graphs round-robin over a pool of streams, so the small jobs of the mix run side
by side on the 152 SMs and no host launch overhead sits between their kernels.  Every kernel
is deterministic and a job's buffers are its own, so a job's results are bitwise the same
alone, in the plain form and in the batched form.
"""
from __future__ import annotations

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
        V.vest_sweep_factors(job.index, job.model, job.reg, job.lam, -1, job.scratch, stream=stream)
        V.vest_sweep_core(job.index, job.model, job.reg, job.lam, job.scratch, stream=stream)


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
