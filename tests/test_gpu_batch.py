"""Batched jobs (CUDA graphs over a pool of streams) against the plain one-job-at-a-time form and
the oracle: every job's result must be bitwise the same in both forms."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1904_02603_gb300 import batch as B
from paper_1904_02603_gb300 import datagen
from paper_1904_02603_gb300 import vest as V
from gpu_common import model_err, oracle_pair

pytestmark = pytest.mark.gpu


def _specs(dtype, count=7):
    out = []
    shapes = [((60, 50, 40), (3, 4, 5), 3000), ((30, 20, 25, 15), (3, 3, 4, 2), 2500), ((200, 90, 70), (10, 8, 6), 9000),
              ((40, 40, 40), (5, 5, 5), 1200), ((25, 30, 20, 18), (4, 5, 3, 3), 4000), ((500, 400, 300), (6, 7, 5), 20000),
              ((12, 10, 9, 8), (2, 3, 2, 4), 700)]
    for j, (dims, ranks, nnz) in enumerate(shapes[:count]):
        t, st = datagen.random_problem(3000 + j, dims, ranks, nnz, dtype=dtype)
        out.append((t, st, V.REG_LF if j % 3 else V.REG_L1, 0.02))
    return out


def _state(job):
    f, c, fm, cm = job.model.to_host()
    return f, c, fm, cm


def test_batched_equals_plain_bitwise():
    specs = _specs(np.float32)
    plain = B.prepare(specs)
    batched = B.prepare(specs)
    B.run_plain(plain, 3)
    run = B.BatchedRun(batched, 3, n_streams=4)
    run.replay()
    torch.cuda.synchronize()
    for a, b in zip(plain, batched):
        fa, ca, _, _ = _state(a)
        fb, cb, _, _ = _state(b)
        assert all(np.array_equal(x, y) for x, y in zip(fa, fb))
        assert np.array_equal(ca, cb)


def test_batched_replay_continues_and_matches_the_oracle_f64():
    specs = _specs(np.float64, count=3)
    jobs = B.prepare(specs)
    run = B.BatchedRun(jobs, 2, n_streams=2)
    run.replay()
    run.replay()  # four iterations in all
    torch.cuda.synchronize()
    for (t, st, reg, lam), job in zip(specs, jobs):
        prob, om = oracle_pair(t, st)
        for _ in range(4):
            O.sweep_factors(prob, om, reg, lam, -1)
            O.sweep_core(prob, om, reg, lam)
        assert model_err(job.model, om) < 1e-9, model_err(job.model, om)


def test_autotuned_batch_equals_plain_with_the_same_choices():
    """The autotuner sets one kernel per shape class; the batched form with those choices equals
    the plain form with the same choices bitwise, and every job stays within FP32 rounding of the
    library's default choice."""
    specs = _specs(np.float32)
    tuned = B.prepare(specs)
    table = B.autotune(tuned, trials=1)
    assert {B.shape_key(j) for j in tuned} == set(table)
    assert all(v["path"] in (V.DELTA_FMA, V.DELTA_AUTO) for v in table.values())
    plain = B.prepare(specs)
    for j, t in zip(plain, tuned):
        j.path = t.path
    B.run_plain(plain, 3)
    B.BatchedRun(tuned, 3, n_streams=4).replay()
    default = B.prepare(specs)
    B.run_plain(default, 3)
    torch.cuda.synchronize()
    for a, b, c in zip(plain, tuned, default):
        fa, ca, _, _ = a.model.to_host()
        fb, cb, _, _ = b.model.to_host()
        fc, cc, _, _ = c.model.to_host()
        assert all(np.array_equal(x, y) for x, y in zip(fa, fb)) and np.array_equal(ca, cb)
        scale = max(float(np.abs(x).max()) for x in fc)
        assert max(float(np.abs(x - y).max()) for x, y in zip(fa, fc)) <= 1e-3 * scale
