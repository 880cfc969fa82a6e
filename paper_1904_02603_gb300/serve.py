"""A request loop over one GPU: factorisation jobs and completion queries.

Requests arrive over time (a seeded Poisson trace).  A factorisation job brings a sparse tensor
and an initial model: it is copied in, indexed, swept (factor sweep over every mode, then the
core sweep, 10 times) and its model stays resident.  A completion query asks for the
reconstruction (Eq. 7) at index tuples against a resident model.

The continuous-batching server admits every request that has arrived as soon as a stream slot
is free, the request's target model (for a query) is resident and its estimated memory fits the
HBM budget; admitted work runs on a stream of its own, so requests overlap on the device and
the host only launches, polls completion events and retires.  The baseline serves the same trace
one request at a time, each to completion before the next starts.  Kernels are deterministic and
requests share no buffer: a request's result is bitwise the same alone and in the mix.
"""
from __future__ import annotations

import math
import time
from collections import OrderedDict, deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np
import torch

from . import batch as B
from . import vest as V


@dataclass
class Request:
    rid: int
    kind: str            # "job" or "query"
    arrival: float       # seconds after the start of the trace
    spec: int = -1       # job: index into the job specs
    target: int = -1     # query: rid of the job whose model is queried
    q_idx: np.ndarray | None = None  # query: [N][m] int32
    # filled in by the server
    start: float = math.nan
    done: float = math.nan
    result: object = None
    evicted: bool = False


def make_trace(specs, rate: float, duration: float, seed: int = 1004, job_fraction: float = 0.5):
    """Poisson arrivals at `rate` per second for `duration` seconds; each request a job (spec drawn
    round-robin) with probability job_fraction, else a query of m ~ log-uniform [1, 1e5] tuples
    against the model of a uniformly chosen earlier job (a job if there is none yet)."""
    rng = np.random.default_rng(seed)
    t, reqs, jobs, ns = 0.0, [], [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        rid = len(reqs)
        if rng.random() < job_fraction or not jobs:
            reqs.append(Request(rid, "job", t, spec=ns % len(specs)))
            jobs.append(rid)
            ns += 1
        else:
            target = int(rng.choice(jobs))
            dims = specs[reqs[target].spec][0].dims
            m = int(round(math.exp(rng.uniform(0.0, math.log(1e5)))))
            q = np.stack([rng.integers(0, d, size=m) for d in dims]).astype(np.int32)
            reqs.append(Request(rid, "query", t, target=target, q_idx=q))
    return reqs


class Budget:
    """Device-memory accounting of the server against one budget (bytes).

    Two kinds of holdings count: the in-flight requests (a job's tensor, index, scratch and model;
    a query's tuples and answers) and the resident models of finished jobs.  When a request does
    not fit, resident models are evicted least recently used first (a query uses its model), never
    one that a waiting or running request refers to."""

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.inflight = 0
        self.resident = OrderedDict()  # rid -> bytes, least recently used first

    @property
    def used(self) -> int:
        return self.inflight + sum(self.resident.values())

    def fits(self, nbytes: int) -> bool:
        return self.used + nbytes <= self.budget

    def reserve(self, nbytes: int):
        self.inflight += nbytes

    def release(self, nbytes: int):
        self.inflight -= nbytes

    def add_resident(self, rid: int, nbytes: int):
        self.resident[rid] = nbytes

    def touch(self, rid: int):
        if rid in self.resident:
            self.resident.move_to_end(rid)

    def make_room(self, nbytes: int, pinned) -> list:
        """Evicts least recently used resident models outside `pinned` until `nbytes` fits or no
        candidate is left; returns the evicted rids (empty when nothing needed to go)."""
        out = []
        for rid in list(self.resident):
            if self.fits(nbytes):
                break
            if rid in pinned:
                continue
            del self.resident[rid]
            out.append(rid)
        return out


class _Inflight:
    def __init__(self, req, stream, nbytes, future=None, state=None, event=None):
        self.req, self.stream, self.nbytes = req, stream, nbytes
        self.future, self.state, self.event = future, state, event


class Server:
    """Continuous batching over `slots` streams under an HBM budget (bytes)."""

    def __init__(self, specs, budget_bytes: int = 150 << 30, slots: int = 16, sweeps: int = 10,
                 launch_threads: int = 4):
        self.specs = specs
        self.budget_bytes = budget_bytes
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.sweeps = sweeps
        self.launch_threads = launch_threads
        self.models = {}  # rid of a finished job -> (Model, dims)
        # pinned host copies of every job's inputs, made before the clock starts
        self.host = [(torch.from_numpy(t.idx).pin_memory(), torch.from_numpy(t.val).pin_memory())
                     for t, _, _, _ in specs]
        # device bytes of each job and of its resident model, from the library's size queries
        self.sizes = []
        for t, st, _, _ in specs:
            b = V.device_bytes_for_shape(t.dims, st.ranks, t.nnz, torch.from_numpy(t.val[:0]).dtype)
            self.sizes.append((sum(b.values()), b["model"]))

    def _launch_job(self, req, stream):
        t, st, reg, lam = self.specs[req.spec]
        ih, vh = self.host[req.spec]
        with torch.cuda.stream(stream):
            ten = V.Tensor(t.dims, ih.to("cuda", non_blocking=True), vh.to("cuda", non_blocking=True))
            mdl = V.Model.from_host(st)
            ix = V.vest_build_index(ten, stream=stream)  # waits for this stream only
            sc = V.make_scratch(ix, mdl)
            job = B.Job(ten, mdl, ix, sc, reg, lam)
            B.sweeps(job, self.sweeps, stream=stream)
            loss = V.vest_loss(ix, mdl, reg, lam, sc, stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return (job, loss), ev

    def _launch_query(self, req, stream):
        mdl, _ = self.models[req.target]
        with torch.cuda.stream(stream):
            q = torch.from_numpy(req.q_idx).pin_memory().to("cuda", non_blocking=True)
            out = V.vest_reconstruct(mdl, q, stream=stream)
            host = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)
            host.copy_(out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return (q, out, host), ev

    def serve(self, reqs):
        """Runs the trace; fills each request's start, done and result.  Jobs are launched from a
        small thread pool, since building an index waits for its own stream (the range check), so
        the admission loop never blocks on one job; queries launch inline.  A query whose model was
        evicted gets result None and `evicted` set.  Device memory in use (in-flight requests plus
        resident models) stays within the budget as long as every single request fits in it; a
        request larger than the whole budget runs alone."""
        self.models = {}  # a trace's queries refer to that trace's jobs only
        budget = Budget(self.budget_bytes)
        pending = deque(sorted(reqs, key=lambda r: r.arrival))
        waiting = []  # arrived, not yet admitted
        inflight = []
        free = list(range(len(self.streams)))
        evicted = set()
        pool = ThreadPoolExecutor(max_workers=self.launch_threads)
        max_used = 0
        t0 = time.perf_counter()
        try:
            while pending or waiting or inflight:
                now = time.perf_counter() - t0
                while pending and pending[0].arrival <= now:
                    waiting.append(pending.popleft())
                progressed = False
                keep = []
                for req in waiting:  # admit in arrival order while slots and memory allow
                    if req.kind == "query" and req.target in evicted:
                        req.start = req.done = time.perf_counter() - t0
                        req.result, req.evicted = None, True
                        progressed = True
                        continue
                    if not free or (req.kind == "query" and req.target not in self.models):
                        keep.append(req)  # no slot, or its model is not resident yet
                        continue
                    nbytes = self.sizes[req.spec][0] if req.kind == "job" else 16 * req.q_idx.size
                    if not budget.fits(nbytes):
                        running = {f.req.target for f in inflight if f.req.kind == "query"}
                        pinned = running | {r.target for r in waiting if r.kind == "query"}
                        gone = budget.make_room(nbytes, pinned)
                        if not budget.fits(nbytes) and not inflight:
                            # nothing will finish to free memory: models that only waiting queries
                            # need go too (those queries are answered as evicted)
                            gone += budget.make_room(nbytes, running)
                        for rid in gone:
                            self.models.pop(rid, None)
                            evicted.add(rid)
                    if not budget.fits(nbytes) and inflight:
                        keep.append(req)
                        continue
                    si = free.pop()
                    s = self.streams[si]
                    req.start = time.perf_counter() - t0
                    if req.kind == "job":
                        inflight.append(_Inflight(req, si, nbytes, future=pool.submit(self._launch_job, req, s)))
                    else:
                        budget.touch(req.target)
                        state, ev = self._launch_query(req, s)
                        inflight.append(_Inflight(req, si, nbytes, state=state, event=ev))
                    budget.reserve(nbytes)
                    max_used = max(max_used, budget.used)
                    progressed = True
                waiting = keep
                still = []
                for f in inflight:
                    if f.event is None and f.future.done():
                        f.state, f.event = f.future.result()  # re-raises a failed launch
                    if f.event is not None and f.event.query():
                        f.req.done = time.perf_counter() - t0
                        budget.release(f.nbytes)
                        if f.req.kind == "job":
                            job, loss = f.state
                            self.models[f.req.rid] = (job.model, job.tensor.dims)
                            budget.add_resident(f.req.rid, self.sizes[f.req.spec][1])
                            f.req.result = loss.cpu().numpy()
                        else:
                            f.req.result = f.state[2].numpy().copy()
                        free.append(f.stream)
                        progressed = True
                    else:
                        still.append(f)
                inflight = still
                if not progressed:
                    time.sleep(0.0001)
        finally:
            pool.shutdown(wait=True)
        self.max_used_bytes, self.resident_bytes = max_used, sum(budget.resident.values())
        self.evicted = sorted(evicted)
        return reqs


def serve_one_at_a_time(server: Server, reqs):
    """The baseline: each request to completion before the next one starts (arrival order)."""
    server.models = {}
    t0 = time.perf_counter()
    s = server.streams[0]
    for req in sorted(reqs, key=lambda r: r.arrival):
        wait = req.arrival - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        req.start = time.perf_counter() - t0
        if req.kind == "job":
            (job, loss), _ = server._launch_job(req, s)
            s.synchronize()
            server.models[req.rid] = (job.model, job.tensor.dims)
            req.result = loss.cpu().numpy()
        else:
            (_, _, host), _ = server._launch_query(req, s)
            s.synchronize()
            req.result = host.numpy().copy()
        req.done = time.perf_counter() - t0
    return reqs


def latency_stats(reqs) -> dict:
    lat = np.array([r.done - r.arrival for r in reqs]) * 1e3
    jobs = [r for r in reqs if r.kind == "job"]
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"requests": len(reqs), "jobs": len(jobs), "queries": len(reqs) - len(jobs),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "jobs_per_s": len(jobs) / span, "span_s": span,
            "job_p99_ms": float(np.percentile([(r.done - r.arrival) * 1e3 for r in jobs], 99)) if jobs else None}
