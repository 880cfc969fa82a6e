"""Host logic of the batch autotuner: shape classes and reuse of a stored table (no GPU: every
class is already in the table, so nothing is timed)."""
import json

import numpy as np
import torch

from paper_1904_02603_gb300 import batch as B
from paper_1904_02603_gb300 import datagen
from paper_1904_02603_gb300 import vest as V


def _job(dims, ranks, nnz, seed):
    t, st = datagen.random_problem(seed, dims, ranks, nnz, dtype=np.float32)
    ten = V.Tensor(t.dims, torch.from_numpy(t.idx), torch.from_numpy(t.val))
    return B.Job(ten, V.Model.from_host(st, device="cpu"), None, None, V.REG_LF, 0.01)


def test_shape_key_groups_by_order_rank_bucket_dtype_and_entry_scale():
    a = _job((40, 30, 20), (10, 9, 10), 3000, 1)
    b = _job((50, 60, 70), (9, 10, 10), 3100, 2)  # same buckets (10), same power-of-two scale
    c = _job((40, 30, 20), (10, 9, 10), 12000, 3)  # four times the entries
    d = _job((40, 30, 20, 5), (10, 9, 10, 3), 3000, 4)
    assert B.shape_key(a) == B.shape_key(b) == "N3_J10x10x10_float32_nnz2^12"
    assert B.shape_key(c) != B.shape_key(a) and B.shape_key(d).startswith("N4_J10x10x10x4")


def test_stored_table_is_reused_without_timing(tmp_path):
    jobs = [_job((40, 30, 20), (10, 9, 10), 3000, 1), _job((30, 20, 25, 15), (3, 3, 4, 2), 2500, 5)]
    table = {B.shape_key(jobs[0]): {"path": V.DELTA_FMA, "fma_ms": 1.0, "tensor_ms": 2.0},
             B.shape_key(jobs[1]): {"path": V.DELTA_AUTO, "fma_ms": 2.0, "tensor_ms": 1.0}}
    cache = tmp_path / "tune.json"
    cache.write_text(json.dumps(table))
    out = B.autotune(jobs, cache_path=str(cache))
    assert [j.path for j in jobs] == [V.DELTA_FMA, V.DELTA_AUTO]
    assert out == table and json.loads(cache.read_text()) == table
