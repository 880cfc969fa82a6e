"""Parity at the full size of the Zipf 100,000^3 / 1e7-entry FP32 workload (ranks 10, the
benchmark's default), through the calls and launch configuration the benchmark times.

The oracle cannot redo whole passes at this size, so the checks take outputs it can compute one
by one, or properties that hold at any size:
  - index of every mode: bit-exact against the oracle's stable counting sort (it is O(nnz));
  - factor sweep of each mode from the initial model: sampled rows (four of the heaviest Zipf
    rows, which span hundreds of tasks, plus random and empty rows) against the oracle's row
    update (Algorithm 4) on the same rows;
  - loss: sampled residuals against the oracle's B(alpha) (Eq. 7), the sums against the
    returned residual array;
  - factor responsibility: the sampled rows' Delta (Eq. 6) against the oracle on those rows'
    entries;
  - prune: tied scores on the full-size segments, bit-exact against the oracle's selection;
  - core sweep: repeatable bitwise, objective not increased, marking table untouched.
Tolerances for the FP32 path against the FP64 oracle are relative to the largest magnitude of
the compared values: 5e-4 for swept rows and for Delta, 1e-4 for residuals.  FP32 products with
compensated sums put the expected error near 1e-6 (an FP32 emulation of the row update on this
workload stays below 2e-7); a wrong index or a dropped term gives errors of order one.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1904_02603_gb300 import datagen
from paper_1904_02603_gb300 import vest as V

pytestmark = pytest.mark.gpu
WORKLOAD = "zipf_1e5x3_1e7"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02603_gb300 import build as B
    B.build()
    V.load()


@pytest.fixture(scope="module")
def full():
    w = datagen.WORKLOADS[WORKLOAD]
    t, st, _ = datagen.make(w, device="cuda")
    ix = V.vest_build_index(V.Tensor.from_host(t))
    prob = O.Problem(t.dims, t.idx, t.val.astype(np.float64))
    index = [O.build_index(prob, n) for n in range(t.N)]
    return w, t, st, ix, prob, index


def _oracle_model(st):
    return O.Model([f.astype(np.float64) for f in st.factors], st.core.astype(np.float64))


def _sample_rows(row_ptr, seed):
    lens = np.diff(row_ptr)
    by_len = np.argsort(-lens, kind="stable")
    heavy = by_len[[5, 20, 100, 1000]]
    rng = np.random.default_rng(seed)
    light = rng.choice(np.nonzero(lens)[0], size=24, replace=False)
    empty = np.nonzero(lens == 0)[0][:2]
    return np.unique(np.concatenate([heavy, light, empty]))


def _rel(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref)) / max(float(np.max(np.abs(ref))), 1e-300))


def test_index_bit_exact_at_full_size(full):
    w, t, st, ix, prob, index = full
    for n in range(t.N):
        view = ix.mode_view(n)
        row_ptr, perm = index[n]
        np.testing.assert_array_equal(view["row_ptr"].numpy(), row_ptr)
        np.testing.assert_array_equal(view["perm"].numpy(), perm)
        others = [k for k in range(t.N) if k != n]
        np.testing.assert_array_equal(view["oidx"].numpy(), t.idx[others][:, perm])
        np.testing.assert_array_equal(view["val"].numpy(), t.val[perm])


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_factor_sweep_sampled_rows_at_full_size(full, mode):
    w, t, st, ix, prob, index = full
    mdl = V.Model.from_host(st)
    sc = V.make_scratch(ix, mdl)
    V.vest_sweep_factors(ix, mdl, V.REG_LF, w.lam, mode, sc)
    got = mdl.factors[mode].cpu().numpy()
    row_ptr, perm = index[mode]
    rows = _sample_rows(row_ptr, 50 + mode)
    om = _oracle_model(st)
    for r in rows:
        O.update_row(prob, om, mode, int(r), row_ptr, perm, V.REG_LF, w.lam)
    assert np.diff(row_ptr)[rows].max() > 100_000  # the sample holds rows cut across many tasks
    err = _rel(got[rows], om.A[mode][rows])
    assert err < 5e-4, err
    untouched = np.setdiff1d(np.arange(t.dims[mode]), np.nonzero(np.diff(row_ptr))[0])[:5]
    np.testing.assert_array_equal(got[untouched], 0.0)  # rows without entries are set to 0


def test_loss_sampled_residuals_at_full_size(full):
    w, t, st, ix, prob, index = full
    mdl = V.Model.from_host(st)
    sc = V.make_scratch(ix, mdl)
    resid = torch.empty(t.nnz, dtype=torch.float32, device="cuda")
    out = V.vest_loss(ix, mdl, V.REG_LF, w.lam, sc, resid=resid).cpu().numpy()
    r = resid.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(60)
    pick = rng.choice(t.nnz, size=2000, replace=False)
    sub = O.Problem(t.dims, t.idx[:, pick], t.val[pick].astype(np.float64))
    ref = sub.x - O.reconstruct(sub, _oracle_model(st))
    assert _rel(r[pick], ref) < 1e-4
    assert abs(out[0] - np.sum(r * r)) <= 1e-5 * out[0]
    x = t.val.astype(np.float64)
    assert abs(out[1] - np.sum(x * x)) <= 1e-6 * out[1]


def test_factor_responsibility_sampled_rows_at_full_size(full):
    w, t, st, ix, prob, index = full
    mdl = V.Model.from_host(st)
    sc = V.make_scratch(ix, mdl)
    df, _, _, _ = V.vest_responsibility(ix, mdl, sc, with_resp=False)
    for n in range(t.N):
        row_ptr, perm = index[n]
        rows = _sample_rows(row_ptr, 70 + n)
        rows = rows[np.diff(row_ptr)[rows] < 60_000]  # the oracle pass below is |G| work per entry
        ent = np.concatenate([perm[row_ptr[r]:row_ptr[r + 1]] for r in rows])
        sub = O.Problem(t.dims, t.idx[:, ent], t.val[ent].astype(np.float64))
        odf, _, _, _ = O.responsibility(sub, _oracle_model(st))
        err = _rel(df[n].cpu().numpy()[rows], odf[n][rows])
        assert err < 5e-4, (n, err)


def test_prune_tied_scores_bit_exact_at_full_size(full):
    w, t, st, ix, prob, index = full
    mdl = V.Model.from_host(st)
    sc = V.make_scratch(ix, mdl)
    sizes = [d * r for d, r in zip(w.dims, w.ranks)] + [int(np.prod(w.ranks))]
    keys = datagen.tied_scores(sizes, seed=80)
    df = [torch.from_numpy(k.reshape(f.shape)).cuda() for k, f in zip(keys[:-1], st.factors)]
    dc = torch.from_numpy(keys[-1]).cuda()
    npr = V.vest_prune(mdl, df, dc, 0.01, sc, count_mode=1).cpu().numpy()
    om = _oracle_model(st)
    onp = O.prune(om, [k.reshape(f.shape) for k, f in zip(keys[:-1], st.factors)], keys[-1], 0.01, 1)
    np.testing.assert_array_equal(npr, onp)
    f, c, fm, cm = mdl.to_host()
    for a, b in zip(fm, om.Amask):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(cm, om.Gmask)


def test_core_sweep_properties_at_full_size(full):
    w, t, st, ix, prob, index = full
    runs = []
    for _ in range(2):
        mdl = V.Model.from_host(st)
        sc = V.make_scratch(ix, mdl)
        before = V.vest_loss(ix, mdl, V.REG_LF, w.lam, sc).cpu().numpy()
        V.vest_sweep_core(ix, mdl, V.REG_LF, w.lam, sc)
        after = V.vest_loss(ix, mdl, V.REG_LF, w.lam, sc).cpu().numpy()
        runs.append((mdl.to_host(), before, after))
    (f1, c1, fm1, cm1), before, after = runs[0]
    (f2, c2, _, _), _, _ = runs[1]
    np.testing.assert_array_equal(c1, c2)  # deterministic
    assert after[3] <= before[3] * (1 + 1e-6)  # coordinate descent does not raise the objective
    assert after[3] < before[3]
    np.testing.assert_array_equal(cm1, st.core_mask)
    for a, b in zip(f1, st.factors):
        np.testing.assert_array_equal(a, b)  # the core sweep leaves the factors alone
