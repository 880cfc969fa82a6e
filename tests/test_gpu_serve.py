"""The request loop: every job's model and loss, and every query's values, are bitwise the same
when served in the mix (continuous batching) as when run alone."""
import numpy as np
import pytest
import torch

from paper_1904_02603_gb300 import batch as B
from paper_1904_02603_gb300 import datagen
from paper_1904_02603_gb300 import serve as S
from paper_1904_02603_gb300 import vest as V

pytestmark = pytest.mark.gpu


def _specs():
    shapes = [((60, 50, 40), (3, 4, 5), 3000), ((30, 20, 25, 15), (3, 3, 4, 2), 2500),
              ((200, 90, 70), (10, 8, 6), 9000), ((500, 400, 300), (6, 7, 5), 20000)]
    out = []
    for j, (dims, ranks, nnz) in enumerate(shapes):
        t, st = datagen.random_problem(4000 + j, dims, ranks, nnz, dtype=np.float32)
        out.append((t, st, V.REG_LF, 0.02))
    return out


def _alone(spec, sweeps):
    job = B.prepare([spec])[0]
    B.sweeps(job, sweeps)
    loss = V.vest_loss(job.index, job.model, job.reg, job.lam, job.scratch).cpu().numpy()
    return job.model, loss


def test_served_results_equal_alone_results():
    specs = _specs()
    reqs = S.make_trace(specs, rate=400.0, duration=0.08, seed=7)
    assert any(r.kind == "query" for r in reqs) and any(r.kind == "job" for r in reqs)
    server = S.Server(specs, slots=4, sweeps=3)
    server.serve(reqs)
    torch.cuda.synchronize()
    alone = {}
    for r in reqs:
        if r.kind == "job":
            mdl, loss = _alone(specs[r.spec], 3)
            alone[r.rid] = mdl
            np.testing.assert_array_equal(r.result, loss)
            f1, c1, _, _ = server.models[r.rid][0].to_host()
            f2, c2, _, _ = mdl.to_host()
            assert all(np.array_equal(a, b) for a, b in zip(f1, f2)) and np.array_equal(c1, c2)
    for r in reqs:
        if r.kind == "query":
            ref = V.vest_reconstruct(alone[r.target], torch.from_numpy(r.q_idx).cuda()).cpu().numpy()
            np.testing.assert_array_equal(r.result, ref)
    st = S.latency_stats(reqs)
    assert st["requests"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0


def test_budget_holds_and_evicts_resident_models():
    """A budget that holds one job and a few models: the server never admits past it, evicts the
    least recently used models no waiting request needs, and every answered request still equals
    its alone result."""
    specs = _specs()
    reqs = S.make_trace(specs, rate=400.0, duration=0.08, seed=7)
    server = S.Server(specs, slots=4, sweeps=3)
    job_max = max(j for j, _ in server.sizes)
    model_min = min(m for _, m in server.sizes)
    query_max = max(16 * r.q_idx.size for r in reqs if r.kind == "query")
    server.budget_bytes = job_max + query_max + 2 * model_min
    server.serve(reqs)
    torch.cuda.synchronize()
    assert server.max_used_bytes <= server.budget_bytes
    assert server.evicted, "the small budget should force evictions"
    for r in reqs:
        if r.kind == "query" and not r.evicted:
            mdl, _ = _alone(specs[reqs[r.target].spec], 3)
            ref = V.vest_reconstruct(mdl, torch.from_numpy(r.q_idx).cuda()).cpu().numpy()
            np.testing.assert_array_equal(r.result, ref)
        if r.kind == "query" and r.evicted:
            assert r.result is None and r.target in server.evicted
