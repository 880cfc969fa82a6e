"""CPU checks of the input generators the scalability and sparsity-curve runs use."""
import math

import numpy as np

from paper_1904_02603_gb300 import datagen


def test_scalability_series_match_the_study():
    pts = datagen.scalability_points()
    order = [p for p in pts if p[0] == "order"]
    dims = [p for p in pts if p[0] == "dims"]
    nnz = [p for p in pts if p[0] == "nnz"]
    assert [p[1] for p in order] == list(range(3, 11)) and all(p[2] == p[3] == 1000 for p in order)
    assert [p[2] for p in dims] == [10 ** e for e in range(3, 9)] and all(p[1] == 3 and p[2] == p[3] for p in dims)
    assert [p[3] for p in nnz] == [10 ** e for e in range(3, 8)] and all(p[1] == 3 and p[2] == 1000 for p in nnz)


def test_uniform_tensor_shapes_ranges_and_distinct_positions():
    t, st = datagen.uniform_tensor(4, 30, 5000, seed=11)
    assert t.idx.shape == (4, 5000) and t.idx.dtype == np.int32
    assert t.idx.min() >= 0 and t.idx.max() < 30
    assert t.val.min() >= 0.0 and t.val.max() < 1.0
    keys = sum(t.idx[n].astype(np.int64) * 30 ** n for n in range(4))
    assert np.unique(keys).size == 5000
    assert st.ranks == (3,) * 4 and st.core.size == 81
    assert all(0.0 <= f.min() and f.max() < 1.0 for f in st.factors)
    # above 2^62 cells positions are independent draws, still in range
    t, _ = datagen.uniform_tensor(10, 1000, 300, seed=12)
    assert t.idx.shape == (10, 300) and t.idx.max() < 1000
    # seeded: the same seed gives the same tensor
    a, _ = datagen.uniform_tensor(3, 50, 700, seed=13)
    b, _ = datagen.uniform_tensor(3, 50, 700, seed=13)
    assert np.array_equal(a.idx, b.idx) and np.array_equal(a.val, b.val)


def test_split_entries_is_a_partition_in_input_order():
    t, _ = datagen.uniform_tensor(3, 40, 2000, seed=14)
    tr, te = datagen.split_entries(t, 0.1, seed=5)
    assert tr.nnz + te.nnz == t.nnz and te.nnz == 200
    key = lambda x: sum(x.idx[n].astype(np.int64) * 40 ** n for n in range(3))
    k_all, k_tr, k_te = key(t), key(tr), key(te)
    assert not set(k_tr) & set(k_te)
    assert set(k_tr) | set(k_te) == set(k_all)
    pos = {k: i for i, k in enumerate(k_all)}
    assert all(np.diff([pos[k] for k in k_tr]) > 0) and all(np.diff([pos[k] for k in k_te]) > 0)
    lookup = dict(zip(k_all, t.val))
    assert all(lookup[k] == v for k, v in zip(k_te, te.val))


def test_sparsity_curve_truth_sparsity():
    w = datagen.SPARSITY_CURVE
    elems = math.prod(w.ranks) + sum(d * r for d, r in zip(w.dims, w.ranks))
    zeros = (1 - w.core_density) * math.prod(w.ranks) + (1 - w.factor_density) * sum(
        d * r for d, r in zip(w.dims, w.ranks))
    assert abs(zeros / elems - 0.71) < 0.01


def test_planted_values_on_a_torch_device_are_the_same_numbers():
    rng = np.random.default_rng(21)
    dims, ranks = (40, 30, 20), (4, 3, 5)
    idx = datagen.sample_indices(rng, dims, 3000)
    planted = datagen.planted_model(rng, dims, ranks, 0.3, 0.5)
    a = datagen.planted_values(idx, planted, 0.01, np.random.default_rng(5))
    b = datagen.planted_values_on("cpu", idx, planted, 0.01, np.random.default_rng(5))
    np.testing.assert_array_equal(a, b)
