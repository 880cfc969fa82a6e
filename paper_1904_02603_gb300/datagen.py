"""Seeded synthetic workloads shaped like the paper's tensors (Section 4.1, Table 2).

This module only draws inputs: observed index sets, values from a *planted*
sparse Tucker model plus Gaussian noise, and the U(0,1) initial state of the
model being fitted (the random start of Algorithm 2).  It is shared by the CUDA tests,
the bench and the oracle tests, and holds none of the fitted method's
arithmetic: no update rule, no responsibility, no pruning, no loss.  The one
contraction here evaluates the planted ground-truth model to synthesise X.

Layouts match the library's: idx is (N, nnz) int32, 0-based, one row per
mode; the core is flat with j_1 fastest; factors are (I_n, J_n) row-major.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class SparseTensor:
    dims: tuple
    idx: np.ndarray  # (N, nnz) int32
    val: np.ndarray  # (nnz,) float64 or float32

    @property
    def N(self):
        return len(self.dims)

    @property
    def nnz(self):
        return int(self.val.shape[0])


@dataclass
class ModelState:
    factors: list  # (I_n, J_n) arrays
    core: np.ndarray  # flat, j_1 fastest
    factor_masks: list = field(default=None)  # uint8, 1 = pruned
    core_mask: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.factor_masks is None:
            self.factor_masks = [np.zeros(f.shape, np.uint8) for f in self.factors]
        if self.core_mask is None:
            self.core_mask = np.zeros(self.core.shape, np.uint8)

    @property
    def ranks(self):
        return tuple(f.shape[1] for f in self.factors)

    @property
    def dims(self):
        return tuple(f.shape[0] for f in self.factors)

    def astype(self, dtype):
        return ModelState([f.astype(dtype) for f in self.factors], self.core.astype(dtype),
                          [m.copy() for m in self.factor_masks], self.core_mask.copy())

    def copy(self):
        return self.astype(self.core.dtype)


def _linear_keys(idx: np.ndarray, dims) -> np.ndarray | None:
    total = 1
    for d in dims:
        total *= int(d)
    if total >= 2 ** 62:
        return None
    key = np.zeros(idx.shape[1], np.int64)
    stride = 1
    for n, d in enumerate(dims):
        key += idx[n].astype(np.int64) * stride
        stride *= int(d)
    return key


def _draw_mode(rng, dim: int, count: int, dist: str, zipf_s: float, rank_perm) -> np.ndarray:
    if dist == "uniform":
        return rng.integers(0, dim, size=count, dtype=np.int64)
    if dist == "zipf":
        # P(rank r) proportional to r^-s over r = 1..dim; ranks mapped to ids by a seeded permutation
        w = np.arange(1, dim + 1, dtype=np.float64) ** (-zipf_s)
        cdf = np.cumsum(w)
        cdf /= cdf[-1]
        r = np.searchsorted(cdf, rng.random(count), side="right")
        r = np.minimum(r, dim - 1)
        return rank_perm[r]
    raise ValueError(f"unknown index distribution {dist!r}")


def sample_indices(rng, dims, nnz: int, dist: str = "uniform", zipf_s: float = 1.2,
                   distinct: bool = True) -> np.ndarray:
    """(N, nnz) int32 observed positions, distinct unless asked otherwise, in random order."""
    dims = tuple(int(d) for d in dims)
    total = math.prod(dims)
    if distinct and nnz > total:
        raise ValueError("more distinct entries requested than the tensor holds")
    perms = [rng.permutation(d) if dist == "zipf" else None for d in dims]
    have = np.zeros((len(dims), 0), np.int64)
    for _ in range(200):
        need = nnz - have.shape[1]
        if need <= 0:
            break
        draw = max(need + need // 8 + 16, 16)
        cand = np.stack([_draw_mode(rng, d, draw, dist, zipf_s, perms[n]) for n, d in enumerate(dims)])
        have = np.concatenate([have, cand], axis=1)
        if distinct:
            key = _linear_keys(have, dims)
            if key is None:
                _, first = np.unique(have.T, axis=0, return_index=True)
            else:
                _, first = np.unique(key, return_index=True)
            have = have[:, np.sort(first)]
    if have.shape[1] < nnz:
        raise RuntimeError("could not draw enough distinct entries")
    have = have[:, :nnz]
    order = rng.permutation(nnz)
    return np.ascontiguousarray(have[:, order].astype(np.int32))


def _sparse_normal(rng, shape, density: float, exact_zero_fraction: float | None = None) -> np.ndarray:
    size = math.prod(shape)
    a = rng.standard_normal(size)
    if exact_zero_fraction is not None:
        nz = size - int(math.floor(exact_zero_fraction * size))
    else:
        nz = int(round(density * size))
    keep = np.zeros(size, bool)
    keep[rng.permutation(size)[:nz]] = True
    a[~keep] = 0.0
    return a.reshape(shape)


def planted_model(rng, dims, ranks, core_density: float, factor_density: float,
                  exact_zero_fraction: float | None = None) -> ModelState:
    core = _sparse_normal(rng, (math.prod(ranks),), core_density, exact_zero_fraction)
    factors = [_sparse_normal(rng, (d, r), factor_density, exact_zero_fraction) for d, r in zip(dims, ranks)]
    return ModelState(factors, core)


def planted_values(idx: np.ndarray, planted: ModelState, noise: float, rng) -> np.ndarray:
    """X_alpha = planted Tucker model at alpha + N(0, noise^2), float64."""
    ranks = planted.ranks
    N = len(ranks)
    x = np.zeros(idx.shape[1], np.float64)
    cols = [np.ascontiguousarray(f.T) for f in planted.factors]  # (J_n, I_n)
    nzb = np.nonzero(planted.core)[0]
    for b in nzb:
        rest = int(b)
        term = np.full(idx.shape[1], planted.core[b], np.float64)
        for n in range(N):
            j = rest % ranks[n]
            rest //= ranks[n]
            term *= cols[n][j][idx[n]]
        x += term
    if noise > 0:
        x += rng.normal(0.0, noise, size=x.shape)
    return x


def planted_values_on(device, idx: np.ndarray, planted: ModelState, noise: float, rng) -> np.ndarray:
    """planted_values with the per-term products on a torch device (same terms, same order, FP64:
    the same numbers), for generating large batches of inputs quickly."""
    import torch
    ranks = planted.ranks
    N = len(ranks)
    it = [torch.from_numpy(np.ascontiguousarray(idx[n]).astype(np.int64)).to(device) for n in range(N)]
    cols = [torch.from_numpy(np.ascontiguousarray(f.T)).to(device) for f in planted.factors]
    x = torch.zeros(idx.shape[1], dtype=torch.float64, device=device)
    for b in np.nonzero(planted.core)[0]:
        rest = int(b)
        term = torch.full((idx.shape[1],), float(planted.core[b]), dtype=torch.float64, device=device)
        for n in range(N):
            j = rest % ranks[n]
            rest //= ranks[n]
            term *= cols[n][j][it[n]]
        x += term
    out = x.cpu().numpy()
    if noise > 0:
        out = out + rng.normal(0.0, noise, size=out.shape)
    return out


def random_init(dims, ranks, seed: int, dtype=np.float64) -> ModelState:
    """The random start of Algorithm 2: every core and factor element drawn U(0,1)."""
    rng = np.random.default_rng(seed)
    factors = [rng.random((int(d), int(r))).astype(dtype) for d, r in zip(dims, ranks)]
    core = rng.random(math.prod(ranks)).astype(dtype)
    return ModelState(factors, core)


@dataclass
class Workload:
    name: str
    dims: tuple
    ranks: tuple
    nnz: int
    dist: str = "uniform"
    zipf_s: float = 1.2
    core_density: float = 0.5
    factor_density: float = 0.5
    exact_zero_fraction: float | None = None
    noise: float = 0.01
    dtype: str = "f64"
    reg: str = "LF"
    lam: float = 0.01
    data_seed: int = 1000
    init_seed: int = 2000


# The workloads the library is measured and checked on, named by their index
# distribution, mode sizes and entry count: synthetic stand-ins for the paper's
# workload shapes (Table 2); the small ones keep the same structure at sizes the
# FP64 oracle finishes in seconds.
WORKLOADS = {
    "uniform_100x3_1e4": Workload("uniform_100x3_1e4", (100, 100, 100), (5, 5, 5), 10_000, "uniform", exact_zero_fraction=0.5,
                   noise=0.01, dtype="f64", reg="LF", lam=0.01, data_seed=1000, init_seed=2000),
    "zipf_1e5x3_1e7": Workload("zipf_1e5x3_1e7", (100_000,) * 3, (10, 10, 10), 10_000_000, "zipf", 1.2, core_density=0.1,
                   factor_density=0.3, noise=0.01, dtype="f32", reg="LF", lam=0.01, data_seed=1001,
                   init_seed=2001),
    "uniform_1e4x4_5e7": Workload("uniform_1e4x4_5e7", (10_000,) * 4, (8, 8, 8, 8), 50_000_000, "uniform", core_density=0.05,
                   factor_density=0.4, noise=0.05, dtype="f32", reg="L1", lam=0.1, data_seed=1002,
                   init_seed=2002),
    "zipf_2000x3_4e4": Workload("zipf_2000x3_4e4", (2000,) * 3, (10, 10, 10), 40_000, "zipf", 1.2, core_density=0.1,
                         factor_density=0.3, noise=0.01, dtype="f32", reg="LF", lam=0.01, data_seed=1011,
                         init_seed=2011),
    "uniform_2000x4_5e6": Workload("uniform_2000x4_5e6", (2000,) * 4, (8, 8, 8, 8), 5_000_000, "uniform",
                          core_density=0.05, factor_density=0.4, noise=0.05, dtype="f32", reg="L1", lam=0.1,
                          data_seed=1013, init_seed=2013),
    "uniform_300x4_2e4": Workload("uniform_300x4_2e4", (300,) * 4, (8, 8, 8, 8), 20_000, "uniform", core_density=0.05,
                         factor_density=0.4, noise=0.05, dtype="f32", reg="L1", lam=0.1, data_seed=1012,
                         init_seed=2012),
}


def batch_workloads(count: int = 256, seed: int = 1003, init_seed: int = 2003) -> list:
    """The batched configuration: independent jobs of order 3 or 4 (equal odds), mode sizes
    log-uniform in [50, 5000], nnz log-uniform in [1e3, 1e6] capped at half the tensor, ranks
    uniform in 3..10 per mode, planted sparse Tucker values (core 20 %, factors 40 %, noise
    0.01), FP32, L_F with lambda 0.01.  Job j draws its data from seed * 1000 + j and its
    initial model from init_seed + j."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(count):
        N = int(rng.choice([3, 4]))
        dims = tuple(int(round(math.exp(rng.uniform(math.log(50), math.log(5000))))) for _ in range(N))
        nnz = int(round(math.exp(rng.uniform(math.log(1e3), math.log(1e6)))))
        nnz = int(min(nnz, 0.5 * math.prod(dims)))
        ranks = tuple(int(rng.integers(3, 11)) for _ in range(N))
        jobs.append(Workload(f"batch_job_{j}", dims, ranks, nnz, "uniform", core_density=0.2, factor_density=0.4,
                             noise=0.01, dtype="f32", reg="LF", lam=0.01, data_seed=seed * 1000 + j,
                             init_seed=init_seed + j))
    return jobs


def make(w: Workload | str, device=None, **overrides):
    """Returns (tensor, initial model state, planted model) for a workload.  With a torch
    device the planted values are formed there (same numbers, faster)."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    if overrides:
        w = Workload(**{**w.__dict__, **overrides})
    ss = np.random.SeedSequence(w.data_seed)
    r_idx, r_model, r_noise = (np.random.default_rng(s) for s in ss.spawn(3))
    idx = sample_indices(r_idx, w.dims, w.nnz, w.dist, w.zipf_s)
    planted = planted_model(r_model, w.dims, w.ranks, w.core_density, w.factor_density, w.exact_zero_fraction)
    if device is None:
        x = planted_values(idx, planted, w.noise, r_noise)
    else:
        x = planted_values_on(device, idx, planted, w.noise, r_noise)
    np_dtype = np.float64 if w.dtype == "f64" else np.float32
    tensor = SparseTensor(tuple(w.dims), idx, x.astype(np_dtype))
    init = random_init(w.dims, w.ranks, w.init_seed, np_dtype)
    return tensor, init, planted


def random_problem(seed: int, dims, ranks, nnz: int, dtype=np.float64, dist: str = "uniform",
                   distinct: bool = True):
    """Small random instance for parity tests: planted dense model, U(0,1) init."""
    rng = np.random.default_rng(seed)
    idx = sample_indices(rng, dims, nnz, dist, 1.2, distinct=distinct)
    planted = planted_model(rng, dims, ranks, 0.6, 0.7)
    x = planted_values(idx, planted, 0.01, rng)
    init = random_init(dims, ranks, seed + 7919, dtype)
    return SparseTensor(tuple(int(d) for d in dims), idx, x.astype(dtype)), init


# ---------------------------------------------------------------- scalability series (Section 4.4)
# The paper's data-scalability study: every mode the same size I, every rank 3, entry values
# uniform in [0, 1]; three series, each varying one quantity.
SCALABILITY_RANK = 3


def scalability_points() -> list:
    """(series, order N, mode size I, |Omega|) of the three series: the order 3..10 at
    I = |Omega| = 1e3; the mode size 1e3..1e8 at N = 3 with |Omega| = I; |Omega| 1e3..1e7 at
    N = 3, I = 1e3."""
    pts = [("order", n, 1000, 1000) for n in range(3, 11)]
    pts += [("dims", 3, 10 ** e, 10 ** e) for e in range(3, 9)]
    pts += [("nnz", 3, 1000, 10 ** e) for e in range(3, 8)]
    return pts


def uniform_tensor(order: int, dim: int, nnz: int, seed: int, dtype=np.float32):
    """A `order`-way tensor with every mode of size `dim`, `nnz` observed positions drawn uniformly
    and values U(0,1), with a U(0,1) initial model of rank 3 per mode.  Positions are distinct
    where the tensor has fewer than 2^62 cells; above that they are independent draws (the
    expected number of repeated positions, nnz^2 / (2 dim^order), is below 1e-7 at every
    point of the series)."""
    ss = np.random.SeedSequence(seed)
    r_idx, r_val, r_init = (np.random.default_rng(s) for s in ss.spawn(3))
    dims = (int(dim),) * order
    if math.prod(dims) < 2 ** 62:
        idx = sample_indices(r_idx, dims, nnz, "uniform")
    else:
        idx = r_idx.integers(0, dim, size=(order, nnz), dtype=np.int32)
    val = r_val.random(nnz, dtype=np.float64).astype(dtype)
    ranks = (SCALABILITY_RANK,) * order
    factors = [r_init.random((dim, SCALABILITY_RANK), dtype=np.float32).astype(dtype) for _ in range(order)]
    core = r_init.random(SCALABILITY_RANK ** order, dtype=np.float32).astype(dtype)
    assert tuple(f.shape[1] for f in factors) == ranks
    return SparseTensor(dims, idx, val), ModelState(factors, core)


# ---------------------------------------------------------------- held-out split (Section 4.2)
def split_entries(t: SparseTensor, test_fraction: float = 0.1, seed: int = 1005):
    """The observed entries split at random into a training tensor (1 - test_fraction of them)
    and a held-out tensor (the rest), each keeping the input's order of entries."""
    rng = np.random.default_rng(seed)
    n_test = int(round(test_fraction * t.nnz))
    test = np.zeros(t.nnz, bool)
    test[rng.permutation(t.nnz)[:n_test]] = True
    train_t = SparseTensor(t.dims, np.ascontiguousarray(t.idx[:, ~test]), np.ascontiguousarray(t.val[~test]))
    test_t = SparseTensor(t.dims, np.ascontiguousarray(t.idx[:, test]), np.ascontiguousarray(t.val[test]))
    return train_t, test_t


# A planted sparse Tucker tensor for the sparsity-versus-error curves (Section 4.3): the truth
# has 90 % of its core and 70 % of its factor elements at zero (overall sparsity 0.71), so the
# reconstruction error of a fit should stay flat as the target sparsity grows to about there.
SPARSITY_CURVE = Workload("planted_1000x3_1e6", (1000, 1000, 1000), (10, 10, 10), 1_000_000, "uniform",
                          core_density=0.1, factor_density=0.3, noise=0.01, dtype="f32", reg="LF", lam=0.01,
                          data_seed=1006, init_seed=2006)


# ---------------------------------------------------------------- pruning scores for selection tests
def tied_scores(sizes, seed: int) -> list:
    """One float64 score array per segment size: values on a coarse grid (many ties), a tenth of
    them negative and some -0.0, so a selection by (score, index) meets every ordering case."""
    rng = np.random.default_rng(seed)
    out = []
    for size in sizes:
        v = np.round(rng.standard_normal(int(size)) * 50.0) / 10.0
        v[rng.random(int(size)) < 0.01] = -0.0
        out.append(v.astype(np.float64))
    return out
