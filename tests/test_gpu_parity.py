"""GPU parity: every C-ABI call against the FP64 CPU oracle on the same seeded inputs.

Tolerances: integer and index outputs bit-exact; FP64 results within 1e-9 of
the oracle, measured as max |gpu - oracle| / max |oracle| per array (the two
sides differ only in summation order, ~1e-16 per operation, amplified by the
CD iterations); masks selected from identical scores bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1904_02603_gb300 import datagen
from paper_1904_02603_gb300 import vest as V
from gpu_common import (CASES, device_pair, make_case, masks_equal, model_err, oracle_from_device, oracle_pair,
                        rel_err, with_masks)

pytestmark = pytest.mark.gpu
TOL64 = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02603_gb300 import build as B
    B.build()
    V.load()


# ---------------------------------------------------------------- a1: index
@pytest.mark.parametrize("name", list(CASES))
def test_index_bit_exact(name):
    t, st = make_case(name)
    ten, _ = device_pair(t, st)
    ix = V.vest_build_index(ten)
    prob, _ = oracle_pair(t, st)
    for mode in range(t.N):
        view = ix.mode_view(mode)
        row_ptr, perm = O.build_index(prob, mode)
        np.testing.assert_array_equal(view["row_ptr"].numpy(), row_ptr)
        np.testing.assert_array_equal(view["perm"].numpy(), perm)
        others = [k for k in range(t.N) if k != mode]
        np.testing.assert_array_equal(view["oidx"].numpy(), t.idx[others][:, perm])
        np.testing.assert_array_equal(view["val"].numpy(), t.val[perm])
        nonempty = np.nonzero(np.diff(row_ptr))[0]
        np.testing.assert_array_equal(view["nzrow"].numpy(), nonempty)
        np.testing.assert_array_equal(view["nzptr"].numpy(), np.append(row_ptr[nonempty], t.nnz))


def test_index_rejects_out_of_range():
    t, st = make_case("n3_ragged")
    ten, _ = device_pair(t, st)
    ten.idx[1, 5] = t.dims[1]
    with pytest.raises(V.VestError) as e:
        V.vest_build_index(ten)
    assert e.value.status == 1


# ---------------------------------------------------------------- a6: loss
@pytest.mark.parametrize("reg", [V.REG_LF, V.REG_L1])
@pytest.mark.parametrize("name", list(CASES))
def test_loss_f64(name, reg):
    t, st = make_case(name)
    st = with_masks(st, 0.1, 3)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    resid = torch.empty(t.nnz, dtype=torch.float64, device="cuda")
    out = V.vest_loss(ix, mdl, reg, 0.3, sc, resid=resid).cpu().numpy()
    prob, om = oracle_pair(t, st)
    ref = O.loss(prob, om, reg, 0.3)
    assert rel_err(out, ref) < 1e-12, (out, ref)
    assert rel_err(resid.cpu().numpy(), prob.x - O.reconstruct(prob, om)) < 1e-12


# ---------------------------------------------------------------- a2-a4: factor sweep
@pytest.mark.parametrize("reg", [V.REG_LF, V.REG_L1])
@pytest.mark.parametrize("name", list(CASES))
def test_sweep_factors_f64(name, reg):
    lam = 0.05 if reg == V.REG_LF else 0.5
    t, st = make_case(name)
    st = with_masks(st, 0.15, 5)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    prob, om = oracle_pair(t, st)
    for mode in range(t.N):  # mode by mode, then all modes at once
        V.vest_sweep_factors(ix, mdl, reg, lam, mode, sc)
        O.sweep_factors(prob, om, reg, lam, mode)
        assert model_err(mdl, om) < TOL64, (mode, model_err(mdl, om))
    V.vest_sweep_factors(ix, mdl, reg, lam, -1, sc)
    O.sweep_factors(prob, om, reg, lam, -1)
    assert model_err(mdl, om) < TOL64
    assert masks_equal(mdl, om)


# ---------------------------------------------------------------- a5: core sweep
@pytest.mark.parametrize("reg", [V.REG_LF, V.REG_L1])
@pytest.mark.parametrize("name", list(CASES))
def test_sweep_core_f64(name, reg):
    lam = 0.05 if reg == V.REG_LF else 0.5
    t, st = make_case(name)
    st = with_masks(st, 0.15, 7)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    prob, om = oracle_pair(t, st)
    for _ in range(2):
        V.vest_sweep_core(ix, mdl, reg, lam, sc)
        O.sweep_core(prob, om, reg, lam)
        assert model_err(mdl, om) < TOL64, model_err(mdl, om)
    assert masks_equal(mdl, om)


# ---------------------------------------------------------------- a7: responsibility
@pytest.mark.parametrize("name", list(CASES))
def test_responsibility_f64(name):
    t, st = make_case(name)
    st = with_masks(st, 0.1, 9)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    df, dc, rf, rc = V.vest_responsibility(ix, mdl, sc)
    prob, om = oracle_pair(t, st)
    odf, odc, orf, orc = O.responsibility(prob, om)
    for n in range(t.N):
        assert rel_err(df[n].cpu().numpy(), odf[n]) < TOL64
        assert rel_err(rf[n].cpu().numpy(), orf[n]) < 1e-7
    assert rel_err(dc.cpu().numpy(), odc) < TOL64
    assert rel_err(rc.cpu().numpy(), orc) < 1e-7


# ---------------------------------------------------------------- a8: prune
@pytest.mark.parametrize("count_mode", [0, 1])
@pytest.mark.parametrize("name", ["n3_ragged", "rank32", "n5_generic"])
def test_prune_bit_exact(name, count_mode):
    t, st = make_case(name)
    st = with_masks(st, 0.2, 11)
    rng = np.random.default_rng(4)
    df = [np.round(rng.standard_normal(f.shape), 2) for f in st.factors]  # many ties
    df[0].flat[0] = -0.0
    dc = np.round(rng.standard_normal(st.core.shape), 2)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    n_gpu = V.vest_prune(mdl, [torch.from_numpy(d).cuda() for d in df], torch.from_numpy(dc).cuda(), 0.37, sc,
                         count_mode=count_mode).cpu().numpy()
    _, om = oracle_pair(t, st)
    n_ref = O.prune(om, df, dc, 0.37, count_mode)
    np.testing.assert_array_equal(n_gpu, n_ref)
    assert masks_equal(mdl, om)
    assert model_err(mdl, om) == 0.0


def test_prune_threshold_mode():
    t, st = make_case("n4")
    rng = np.random.default_rng(5)
    df = [rng.standard_normal(f.shape) for f in st.factors]
    dc = rng.standard_normal(st.core.shape)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    n_gpu = V.vest_prune(mdl, [torch.from_numpy(d).cuda() for d in df], torch.from_numpy(dc).cuda(), 0.0, sc,
                         threshold_mode=1, tau=-0.5).cpu().numpy()
    _, om = oracle_pair(t, st)
    n_ref = O.prune(om, df, dc, 0.0, 0, 1, -0.5)
    np.testing.assert_array_equal(n_gpu, n_ref)
    assert masks_equal(mdl, om)


# ---------------------------------------------------------------- a9: auto-search, config-0 workload
def test_manual_pruning_run_f64_uniform_100x3():
    """The 100^3 / 10^4-entry FP64 workload: 10 iterations, 20% of the remaining pruned each step."""
    t, st, _ = datagen.make("uniform_100x3_1e4")
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl, autosearch=True)
    p = V.params(reg=V.REG_LF, lam=0.01, max_iter=10, fixed_pr_mode=1, fixed_pr=0.2, count_mode=0,
                 target_sparsity=1.0, conv_tol=0.0, normalize=1)
    rep = V.vest_autosearch(ix, mdl, p, sc)
    prob, om = oracle_pair(t, st)
    orep = O.autosearch(prob, om, O.Params(reg=O.REG_LF, lam=0.01, max_iter=10, fixed_pr_mode=1, fixed_pr=0.2,
                                           count_mode=0, target_sparsity=1.0, conv_tol=0.0, normalize=1))
    assert rep["iters"] == orep["iters"] == 10
    assert rel_err(rep["re"], orep["re"]) < TOL64
    np.testing.assert_array_equal(rep["sparsity"], orep["sparsity"])
    assert masks_equal(mdl, om)
    assert model_err(mdl, om) < TOL64


def test_autosearch_auto_mode_f64():
    t, st = make_case("n3_ragged")
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl, autosearch=True)
    rep = V.vest_autosearch(ix, mdl, V.params(reg=V.REG_L1, lam=0.2, max_iter=40, conv_tol=1e-7), sc)
    prob, om = oracle_pair(t, st)
    orep = O.autosearch(prob, om, O.Params(reg=O.REG_L1, lam=0.2, max_iter=40, conv_tol=1e-7))
    assert rep["iters"] == orep["iters"] and rep["stop_iter"] == orep["stop_iter"]
    assert rel_err(rep["re"], orep["re"]) < TOL64
    assert masks_equal(mdl, om)
    assert model_err(mdl, om) < TOL64


def test_autosearch_revive_on_stop_f64():
    """VeST_auto with revive_on_stop against the oracle: the elbow fires at iteration 4 on this
    problem, and the masks go back to those before the prune of iteration 3."""
    t, st = datagen.random_problem(42, (30, 25, 20), (3, 3, 3), 3000)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl, autosearch=True)
    kw = dict(lam=0.05, init_pr=0.05, max_pr=0.2, max_iter=12, conv_tol=1e-9, normalize=0, revive_on_stop=1)
    rep = V.vest_autosearch(ix, mdl, V.params(reg=V.REG_LF, **kw), sc)
    prob, om = oracle_pair(t, st)
    orep = O.autosearch(prob, om, O.Params(reg=O.REG_LF, **kw))
    assert rep["stop_iter"] == orep["stop_iter"] >= 3 and rep["iters"] == orep["iters"]
    assert rel_err(rep["re"], orep["re"]) < TOL64
    np.testing.assert_array_equal(rep["sparsity"], orep["sparsity"])
    assert masks_equal(mdl, om)
    assert model_err(mdl, om) < TOL64


def test_autosearch_elbow_rise_f64():
    """VeST_auto with elbow_rise against the oracle: pruning runs until RE rises (iteration 11 on
    this problem), not just until its second difference is large."""
    t, st = datagen.random_problem(42, (30, 25, 20), (3, 3, 3), 3000)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl, autosearch=True)
    kw = dict(reg=V.REG_LF, lam=0.05, max_iter=20, conv_tol=1e-7, normalize=1, elbow_rise=1)
    rep = V.vest_autosearch(ix, mdl, V.params(**kw), sc)
    prob, om = oracle_pair(t, st)
    orep = O.autosearch(prob, om, O.Params(**kw))
    assert rep["stop_iter"] == orep["stop_iter"] > 3 and rep["iters"] == orep["iters"]
    assert rel_err(rep["re"], orep["re"]) < TOL64
    np.testing.assert_array_equal(rep["sparsity"], orep["sparsity"])
    assert masks_equal(mdl, om)
    assert model_err(mdl, om) < TOL64


def test_autosearch_resume_from_checkpoint_f64(tmp_path):
    """A run stopped after 5 iterations, checkpointed to a file, loaded and resumed to 12 ends
    bitwise where one run to 12 ends, and both match the oracle's uninterrupted run."""
    from paper_1904_02603_gb300 import checkpoint
    t, st = datagen.random_problem(42, (30, 25, 20), (3, 3, 3), 3000)
    ten, whole = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, whole, autosearch=True)
    kw = dict(reg=V.REG_LF, lam=0.05, init_pr=0.05, max_pr=0.2, target_sparsity=0.5, conv_tol=1e-9)
    rep_whole = V.vest_autosearch(ix, whole, V.params(max_iter=12, normalize=1, **kw), sc)
    _, part = device_pair(t, st)
    first = V.vest_autosearch(ix, part, V.params(max_iter=5, normalize=0, **kw), sc)
    checkpoint.save(tmp_path / "run.npz", part, first)
    del part
    resumed, rep0 = checkpoint.load(tmp_path / "run.npz")
    rep = V.vest_autosearch(ix, resumed, V.params(max_iter=12, normalize=1, resume=1, **kw), sc, resume_from=rep0)
    assert rep["iters"] == rep_whole["iters"] == 12 and rep["stop_iter"] == rep_whole["stop_iter"]
    for key in ("re", "obj", "pr", "sparsity"):
        np.testing.assert_array_equal(rep[key], rep_whole[key])
    for a, b in zip(resumed.to_host(), whole.to_host()):
        for x, y in zip(a if isinstance(a, list) else [a], b if isinstance(b, list) else [b]):
            np.testing.assert_array_equal(x, y)
    prob, om = oracle_pair(t, st)
    orep = O.autosearch(prob, om, O.Params(max_iter=12, normalize=1, **{k: v for k, v in kw.items()}))
    assert orep["stop_iter"] == rep["stop_iter"]
    assert rel_err(rep["re"], orep["re"]) < TOL64
    assert masks_equal(resumed, om)
    assert model_err(resumed, om) < TOL64


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_value_pruning_keys_and_prune(dtype):
    """Value Pruning: |element| keys bit-exact, then the 60 % smallest per segment pruned as the
    oracle's prune does with the same keys."""
    t, st = make_case("zipf_heavy")
    st = with_masks(st, 0.1, 17)
    ten, mdl = device_pair(t, st, dtype)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    V.vest_sweep_factors(ix, mdl, V.REG_LF, 0.05, -1, sc)
    V.vest_sweep_core(ix, mdl, V.REG_LF, 0.05, sc)
    om = oracle_from_device(mdl)
    kf, kc = V.vest_value_keys(mdl)
    for n in range(t.N):
        np.testing.assert_array_equal(kf[n].cpu().numpy(), np.abs(om.A[n]))
    np.testing.assert_array_equal(kc.cpu().numpy(), np.abs(om.G))
    npr = V.vest_prune(mdl, kf, kc, 0.6, sc, count_mode=1)
    onp = O.prune(om, [np.abs(a) for a in om.A], np.abs(om.G), 0.6, 1)
    np.testing.assert_array_equal(npr.cpu().numpy(), onp)
    assert masks_equal(mdl, om)
    assert model_err(mdl, om) == 0.0


# ---------------------------------------------------------------- FP32 path vs FP64 oracle
def test_fp32_objective_within_1e4_on_zipf_workload():
    """FP32 storage and products, FP64 row finishing: objective within 1e-4 of the FP64 oracle."""
    t, st, _ = datagen.make("zipf_2000x3_4e4")
    ten, mdl = device_pair(t, st, torch.float32)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    prob, om = oracle_pair(t, st)
    errs = []
    for it in range(4):
        V.vest_sweep_factors(ix, mdl, V.REG_LF, 0.01, -1, sc)
        V.vest_sweep_core(ix, mdl, V.REG_LF, 0.01, sc)
        O.sweep_factors(prob, om, O.REG_LF, 0.01, -1)
        O.sweep_core(prob, om, O.REG_LF, 0.01)
        got = V.vest_loss(ix, mdl, V.REG_LF, 0.01, sc).cpu().numpy()[3]
        ref = O.loss(prob, om, O.REG_LF, 0.01)[3]
        errs.append(abs(got - ref) / ref)
    print("fp32 relative objective error per iteration:", errs)
    assert max(errs) < 1e-4


# ---------------------------------------------------------------- one iteration in one call (Algorithm 2)
@pytest.mark.parametrize("reg", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_iteration_f64(name, reg):
    """vest_iteration against the oracle's sweeps, loss, responsibility and prune in turn."""
    if reg == 1 and name not in ("n3_ragged", "zipf_heavy", "n5_generic"):
        pytest.skip("L1 on a subset")
    t, st = make_case(name)
    st = with_masks(st, 0.05, 13)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    prob, om = oracle_pair(t, st)
    lam = 0.05
    for it in range(2):
        loss, df, dc, npr = V.vest_iteration(ix, mdl, reg, lam, 0.05, sc)
        O.sweep_factors(prob, om, reg, lam, -1)
        O.sweep_core(prob, om, reg, lam)
        oloss = O.loss(prob, om, reg, lam)
        odf, odc, _, _ = O.responsibility(prob, om)
        onp = O.prune(om, odf, odc, 0.05, 0)
        assert rel_err(loss.cpu().numpy(), oloss) < TOL64, (it, loss.cpu().numpy(), oloss)
        for n in range(t.N):
            assert rel_err(df[n].cpu().numpy(), odf[n]) < TOL64
        assert rel_err(dc.cpu().numpy(), odc) < TOL64
        np.testing.assert_array_equal(npr.cpu().numpy(), onp)
        assert masks_equal(mdl, om)
        assert model_err(mdl, om) < TOL64


def test_iteration_without_responsibility_matches_separate_calls():
    t, st = make_case("zipf_heavy")
    ten, m1 = device_pair(t, st)
    _, m2 = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, m1)
    loss, df, dc, npr = V.vest_iteration(ix, m1, V.REG_LF, 0.01, 0.0, sc, with_responsibility=False)
    assert df is None and dc is None and npr is None
    V.vest_sweep_factors(ix, m2, V.REG_LF, 0.01, -1, sc)
    V.vest_sweep_core(ix, m2, V.REG_LF, 0.01, sc)
    ref = V.vest_loss(ix, m2, V.REG_LF, 0.01, sc)
    assert rel_err(loss.cpu().numpy(), ref.cpu().numpy()) < 1e-12
    f1, c1, _, _ = m1.to_host()
    f2, c2, _, _ = m2.to_host()
    assert all(np.array_equal(a, b) for a, b in zip(f1, f2)) and np.array_equal(c1, c2)


def test_iteration_fp32_objective_within_1e4_on_zipf_workload():
    """The residual kept by the core sweep (FP32, updated block by block) gives the loss within 1e-4."""
    t, st, _ = datagen.make("zipf_2000x3_4e4")
    ten, mdl = device_pair(t, st, torch.float32)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    prob, om = oracle_pair(t, st)
    for it in range(3):
        loss, _, _, _ = V.vest_iteration(ix, mdl, V.REG_LF, 0.01, 0.0, sc)
        O.sweep_factors(prob, om, O.REG_LF, 0.01, -1)
        O.sweep_core(prob, om, O.REG_LF, 0.01)
        ref = O.loss(prob, om, O.REG_LF, 0.01)
        got = loss.cpu().numpy()
        assert abs(got[3] - ref[3]) / ref[3] < 1e-4, (it, got, ref)
        assert abs(got[4] - ref[4]) / ref[4] < 1e-4


# ---------------------------------------------------------------- edge cases
def test_empty_tensor_zeroes_everything():
    dims, ranks = (5, 4, 3), (2, 2, 2)
    t = datagen.SparseTensor(dims, np.zeros((3, 0), np.int32), np.zeros(0))
    st = datagen.random_init(dims, ranks, 1)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    V.vest_sweep_factors(ix, mdl, V.REG_LF, 0.1, -1, sc)
    V.vest_sweep_core(ix, mdl, V.REG_LF, 0.1, sc)
    f, c, _, _ = mdl.to_host()
    assert all(np.all(a == 0) for a in f) and np.all(c == 0)
    out = V.vest_loss(ix, mdl, V.REG_LF, 0.1, sc).cpu().numpy()
    np.testing.assert_array_equal(out, [0, 0, 0, 0, 0])


def test_single_entry_and_fully_pruned_rows():
    dims, ranks = (3, 3, 3), (2, 2, 2)
    t = datagen.SparseTensor(dims, np.array([[1], [2], [0]], np.int32), np.array([1.5]))
    st = datagen.random_init(dims, ranks, 2)
    st.factor_masks[0][1, :] = 1
    st.factors[0][1, :] = 0
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    prob, om = oracle_pair(t, st)
    V.vest_sweep_factors(ix, mdl, V.REG_LF, 0.1, -1, sc)
    V.vest_sweep_core(ix, mdl, V.REG_LF, 0.1, sc)
    O.sweep_factors(prob, om, O.REG_LF, 0.1, -1)
    O.sweep_core(prob, om, O.REG_LF, 0.1)
    assert model_err(mdl, om) < TOL64


def test_sweeps_are_deterministic():
    t, st = make_case("zipf_heavy", np.float32)
    ten, mdl = device_pair(t, st, torch.float32)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    outs = []
    for _ in range(2):
        m = mdl.clone()
        V.vest_sweep_factors(ix, m, V.REG_LF, 0.01, -1, sc)
        V.vest_sweep_core(ix, m, V.REG_LF, 0.01, sc)
        outs.append(m.to_host())
    for a, b in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(outs[0][1], outs[1][1])


def test_reconstruct_normalize_count_zeros():
    t, st = make_case("n4")
    st = with_masks(st, 0.3, 13)
    ten, mdl = device_pair(t, st)
    prob, om = oracle_pair(t, st)
    q = np.stack([np.random.default_rng(1).integers(0, d, 500) for d in t.dims]).astype(np.int32)
    got = V.vest_reconstruct(mdl, torch.from_numpy(q).cuda()).cpu().numpy()
    ref = np.array([O.entry(om, q[:, i]) for i in range(500)])
    assert rel_err(got, ref) < 1e-12
    bad = q[:, :4].copy()
    bad[0, 0], bad[1, 1], bad[2, 2] = t.dims[0], -1, 1 << 30  # outside the tensor: NaN, nothing read
    got_bad = V.vest_reconstruct(mdl, torch.from_numpy(bad).cuda()).cpu().numpy()
    assert np.isnan(got_bad[:3]).all() and got_bad[3] == got[3]
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    z = V.vest_count_zeros(mdl, sc).cpu().numpy()
    ref_z = [int(np.sum(a == 0)) for a in om.A] + [int(np.sum(om.G == 0))]
    np.testing.assert_array_equal(z, ref_z)
    V.vest_normalize(mdl, sc)
    O.normalize(om)
    assert model_err(mdl, om) < 1e-12


def test_invalid_arguments_are_rejected_on_the_host():
    t, st = make_case("n3_ragged")
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    with pytest.raises(V.VestError) as e:
        V.vest_sweep_factors(ix, mdl, V.REG_LF, 0.0, -1, sc)  # lambda must be > 0
    assert e.value.status == 1
    with pytest.raises(V.VestError) as e:
        V.vest_sweep_factors(ix, mdl, V.REG_LF, 0.1, -1, sc[:100])
    assert e.value.status == 4
    with pytest.raises(V.VestError):
        V.vest_sweep_factors(ix, mdl, V.REG_LF, 0.1, 7, sc)
