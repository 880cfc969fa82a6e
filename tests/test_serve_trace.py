"""Host logic of the serving loop: the seeded request trace."""
import numpy as np

from paper_1904_02603_gb300 import datagen
from paper_1904_02603_gb300 import serve as S


def _specs():
    out = []
    for j, (dims, ranks) in enumerate([((60, 50, 40), (3, 4, 5)), ((30, 20, 25, 15), (3, 3, 4, 2))]):
        t, st = datagen.random_problem(5000 + j, dims, ranks, 500, dtype=np.float32)
        out.append((t, st, 0, 0.01))
    return out


def test_trace_is_seeded_ordered_and_well_formed():
    specs = _specs()
    a = S.make_trace(specs, rate=200.0, duration=5.0, seed=3)
    b = S.make_trace(specs, rate=200.0, duration=5.0, seed=3)
    assert [(r.kind, r.arrival, r.spec, r.target) for r in a] == [(r.kind, r.arrival, r.spec, r.target) for r in b]
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0) and arr[-1] <= 5.0
    assert 800 < len(a) < 1200  # Poisson(1000)
    jobs = [r for r in a if r.kind == "job"]
    assert 0.4 < len(jobs) / len(a) < 0.6
    assert a[0].kind == "job"
    for r in a:
        if r.kind == "query":
            tgt = a[r.target]
            assert tgt.kind == "job" and tgt.arrival < r.arrival
            dims = specs[tgt.spec][0].dims
            assert r.q_idx.shape[0] == len(dims) and 1 <= r.q_idx.shape[1] <= 100_000
            assert all(int(r.q_idx[n].max()) < dims[n] and int(r.q_idx[n].min()) >= 0 for n in range(len(dims)))


def test_latency_stats():
    reqs = [S.Request(0, "job", 0.0), S.Request(1, "query", 0.5, target=0)]
    reqs[0].done, reqs[1].done = 1.0, 0.75
    st = S.latency_stats(reqs)
    assert st["requests"] == 2 and st["jobs"] == 1 and st["queries"] == 1
    assert abs(st["p50_ms"] - 625.0) < 1e-9 and st["span_s"] == 1.0 and st["jobs_per_s"] == 1.0


def test_budget_counts_resident_models_and_evicts_least_recently_used_unpinned():
    b = S.Budget(100)
    b.reserve(30)
    assert b.fits(70) and not b.fits(71)
    b.release(30)
    for rid, nb in ((1, 20), (2, 20), (3, 20)):
        b.add_resident(rid, nb)
    assert b.used == 60
    b.touch(1)  # order of use now 2, 3, 1
    assert b.make_room(30, pinned=set()) == []  # 60 + 30 fits
    assert b.make_room(50, pinned={2}) == [3]  # 2 is pinned: 3 goes, then 40 + 50 fits
    assert list(b.resident) == [2, 1] and b.used == 40
    b.reserve(50)
    assert b.make_room(30, pinned={1, 2}) == [] and not b.fits(30)  # nothing may go
    b.release(50)
    assert b.used == 40
