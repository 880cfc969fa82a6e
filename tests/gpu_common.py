"""Shared helpers for the GPU parity tests: moving seeded inputs to both sides and comparing."""
import numpy as np
import torch

import oracle as O
from paper_1904_02603_gb300 import datagen
from paper_1904_02603_gb300 import vest as V


def oracle_pair(t: datagen.SparseTensor, st: datagen.ModelState):
    prob = O.Problem(t.dims, t.idx, t.val.astype(np.float64))
    model = O.Model([f.astype(np.float64) for f in st.factors], st.core.astype(np.float64),
                    [m.copy() for m in st.factor_masks], st.core_mask.copy())
    return prob, model


def device_pair(t: datagen.SparseTensor, st: datagen.ModelState, dtype=torch.float64):
    npdt = np.float64 if dtype == torch.float64 else np.float32
    ten = V.Tensor(t.dims, torch.from_numpy(t.idx).cuda(), torch.from_numpy(t.val.astype(npdt)).cuda())
    mdl = V.Model.from_host(st.astype(npdt))
    return ten, mdl


def oracle_from_device(m: V.Model) -> O.Model:
    f, c, fm, cm = m.to_host()
    return O.Model([a.astype(np.float64) for a in f], c.astype(np.float64), fm, cm)


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(float(np.max(np.abs(ref))) if ref.size else 0.0, 1e-300)
    return float(np.max(np.abs(got - ref))) / scale if ref.size else 0.0


def model_err(dev: V.Model, ref: O.Model) -> float:
    f, c, _, _ = dev.to_host()
    return max([rel_err(a, b) for a, b in zip(f, ref.A)] + [rel_err(c, ref.G)])


def masks_equal(dev: V.Model, ref: O.Model) -> bool:
    _, _, fm, cm = dev.to_host()
    return all(np.array_equal(a, b) for a, b in zip(fm, ref.Amask)) and np.array_equal(cm, ref.Gmask)


def with_masks(st: datagen.ModelState, frac: float, seed: int) -> datagen.ModelState:
    """Marks a random fraction of elements as pruned (value 0)."""
    rng = np.random.default_rng(seed)
    st = st.copy()
    for n, f in enumerate(st.factors):
        mk = rng.random(f.shape) < frac
        st.factor_masks[n][:] = mk
        f[mk] = 0
    mk = rng.random(st.core.shape) < frac
    st.core_mask[:] = mk
    st.core[mk] = 0
    return st


# Small problems that span several sweep tasks, ragged tails, the generic
# (N >= 5) path, every rank bucket, heavy rows cut across many tasks, empty rows.
CASES = {
    "n3_ragged": dict(dims=(40, 30, 20), ranks=(3, 4, 5), nnz=3001),
    "n2": dict(dims=(120, 90), ranks=(4, 6), nnz=2500),
    "n4": dict(dims=(12, 10, 9, 8), ranks=(2, 3, 2, 4), nnz=3000),
    "n5_generic": dict(dims=(7, 6, 5, 6, 5), ranks=(2, 2, 3, 2, 2), nnz=2000),
    "rank16": dict(dims=(60, 50, 40), ranks=(16, 3, 2), nnz=2500),
    "rank32": dict(dims=(80, 60), ranks=(32, 9), nnz=2000),
    "zipf_heavy": dict(dims=(60, 3000, 3000), ranks=(5, 4, 3), nnz=40000, dist="zipf"),
    "empty_rows": dict(dims=(500, 40, 30), ranks=(3, 3, 3), nnz=300),
}


def make_case(name: str, dtype=np.float64, seed: int = 0):
    c = CASES[name]
    return datagen.random_problem(100 + seed + sum(map(ord, name)), c["dims"], c["ranks"], c["nnz"], dtype=dtype,
                                  dist=c.get("dist", "uniform"))
