"""Pins of the FP64 CPU oracle against things other than itself.

Each test checks one oracle function against what the paper and plain
mathematics fix: the hand-worked examples in tests/golden/, the textbook
n-mode-product reconstruction (Section 2.1), brute-force 1-D minimisation of
the objective (Eq. 1 / Eq. 2) for every coordinate update, ridge closed forms
that repeated Gauss-Seidel sweeps must reach, brute-force zeroing for the
responsibility (Definition 1-2), numpy sorts for the index and the prune.
No test here re-types an oracle formula; the objective is evaluated through a
dense reconstruction built with numpy tensordot.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1904_02603_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


# ---------------------------------------------------------------- numpy references
def dense_recon(model: O.Model) -> np.ndarray:
    """G x_1 A^(1) x_2 ... x_N A^(N), one n-mode product at a time (Section 2.1)."""
    X = model.core_tensor()
    for n, A in enumerate(model.A):
        X = np.moveaxis(np.tensordot(A, X, axes=([1], [n])), 0, n)
    return X


def sq_err(prob: O.Problem, model: O.Model) -> float:
    pred = dense_recon(model)[tuple(prob.idx)]
    r = prob.x - pred
    return float(r @ r)


def objective(prob, model, reg, lam) -> float:
    elems = np.concatenate([model.G] + [a.ravel() for a in model.A])
    pen = np.sum(np.abs(elems)) if reg == O.REG_L1 else float(elems @ elems)
    return sq_err(prob, model) + lam * pen


def golden_min(f, lo, hi, iters=400):
    g = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        if fc <= fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
        if b - a < 1e-15 * max(1.0, abs(a)):
            break
    return 0.5 * (a + b)


def coord_argmin(f, reg, x0):
    if reg == O.REG_LF:
        # the objective is exactly quadratic along one coordinate: fit it from 3 evaluations
        h = max(1.0, abs(x0))
        fm, f0, fp = f(x0 - h), f(x0), f(x0 + h)
        c2 = (fp + fm - 2.0 * f0) / (2.0 * h * h)
        c1 = (fp - fm) / (2.0 * h)
        return x0 - c1 / (2.0 * c2)
    # L_1: piecewise quadratic with a kink at 0.  Locate the minimum by golden
    # section, then refine on its side of the kink, where f is exactly quadratic.
    R = 10.0 * (abs(x0) + 10.0)
    x = golden_min(f, -R, R)
    if abs(x) < 1e-6:
        return 0.0
    h = abs(x) / 2.0
    fm, f0, fp = f(x - h), f(x), f(x + h)
    c2 = (fp + fm - 2.0 * f0) / (2.0 * h * h)
    c1 = (fp - fm) / (2.0 * h)
    return x - c1 / (2.0 * c2)


def small_problem(seed, dims, ranks, nnz, masks=0.0):
    t, init = datagen.random_problem(seed, dims, ranks, nnz)
    prob = O.Problem(t.dims, t.idx, t.val.astype(np.float64))
    model = O.Model(init.factors, init.core)
    if masks > 0:
        rng = np.random.default_rng(seed + 1)
        for n in range(model.N):
            mk = rng.random(model.A[n].shape) < masks
            model.Amask[n][:] = mk
            model.A[n][mk] = 0.0
        mk = rng.random(model.G.shape) < masks
        model.Gmask[:] = mk
        model.G[mk] = 0.0
    return prob, model


# ---------------------------------------------------------------- golden hand examples
def _frac_array(rows):
    return np.array([[float(Fraction(v)) for v in r] for r in rows])


def _golden_cases():
    return json.load(open(GOLDEN))["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_hand_examples(case, oracle_lib):
    d = json.load(open(GOLDEN))
    prob = O.Problem(d["tensor"]["dims"], np.array(d["tensor"]["idx"]), np.array(d["tensor"]["x"], float))
    model = O.Model([np.array(a, float) for a in d["init"]["A"]], np.array(d["init"]["G"], float))
    reg = O.REG_L1 if case.get("reg") == "L1" else O.REG_LF
    lam = float(Fraction(case.get("lambda", "1")))
    e = case["expect"]
    if case["op"] == "responsibility":
        df, dc, rf, rc = O.responsibility(prob, model)
        np.testing.assert_allclose(df[0], _frac_array(e["dA0"]), rtol=1e-14)
        np.testing.assert_allclose(df[1], _frac_array(e["dA1"]), rtol=1e-14)
        np.testing.assert_allclose(dc, [float(Fraction(v)) for v in e["dG"]], rtol=1e-14)
        re2 = float(Fraction(e["RE2"]))
        np.testing.assert_allclose(rf[0], np.sqrt((14 + _frac_array(e["dA0"])) / 14) - 1, rtol=1e-13)
        assert abs(O.loss(prob, model, 0, 1.0)[4] ** 2 - re2) < 1e-15
        return
    if case["op"] == "sweep_factors":
        O.sweep_factors(prob, model, reg, lam, case["mode"])
    elif case["op"] == "sweep_core":
        O.sweep_core(prob, model, reg, lam)
    elif case["op"] == "sweep_factors_then_core":
        O.sweep_factors(prob, model, reg, lam, -1)
        O.sweep_core(prob, model, reg, lam)
    np.testing.assert_allclose(model.A[0], _frac_array(e["A0"]), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(model.A[1], _frac_array(e["A1"]), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(model.G, [float(Fraction(v)) for v in e["G"]], rtol=1e-14)


# ---------------------------------------------------------------- Eq. 7 and the loss
@pytest.mark.parametrize("dims,ranks", [((4, 5), (2, 3)), ((4, 3, 5), (2, 3, 2)), ((3, 4, 2, 3), (2, 1, 2, 3))])
def test_entry_matches_dense_nmode_product(dims, ranks, oracle_lib):
    rng = np.random.default_rng(11)
    A = [rng.standard_normal((d, r)) for d, r in zip(dims, ranks)]
    model = O.Model(A, rng.standard_normal(int(np.prod(ranks))))
    full = np.array(np.unravel_index(np.arange(int(np.prod(dims))), dims))
    prob = O.Problem(dims, full, np.zeros(full.shape[1]))
    ref = dense_recon(model)[tuple(full)]
    np.testing.assert_allclose(O.reconstruct(prob, model), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("reg", [O.REG_LF, O.REG_L1])
def test_loss_matches_definition(reg, oracle_lib):
    prob, model = small_problem(3, (7, 6, 5), (3, 2, 4), 90, masks=0.2)
    out = O.loss(prob, model, reg, 0.37)
    sq = sq_err(prob, model)
    assert out[0] == pytest.approx(sq, rel=1e-12)
    assert out[1] == pytest.approx(float(prob.x @ prob.x), rel=1e-14)
    assert out[3] == pytest.approx(objective(prob, model, reg, 0.37), rel=1e-12)
    assert out[4] == pytest.approx(np.sqrt(sq) / np.linalg.norm(prob.x), rel=1e-12)


# ---------------------------------------------------------------- index
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_build_index_matches_stable_argsort(seed, oracle_lib):
    rng = np.random.default_rng(seed)
    dims = (13, 40, 7)
    nnz = 300
    idx = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.int32)  # repeats allowed
    idx[0][idx[0] == 5] = 6  # an empty row
    prob = O.Problem(dims, idx, rng.standard_normal(nnz))
    for mode in range(3):
        row_ptr, perm = O.build_index(prob, mode)
        np.testing.assert_array_equal(perm, np.argsort(idx[mode], kind="stable"))
        np.testing.assert_array_equal(row_ptr, np.concatenate([[0], np.cumsum(np.bincount(idx[mode], minlength=dims[mode]))]))


# ---------------------------------------------------------------- update rules vs brute force
@pytest.mark.parametrize("reg", [O.REG_LF, O.REG_L1])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_factor_rows_are_sequential_coordinate_minimisers(reg, mode, oracle_lib):
    lam = 0.05 if reg == O.REG_LF else 0.8
    prob, model = small_problem(5, (6, 5, 4), (3, 2, 3), 70, masks=0.15)
    row_ptr, perm = O.build_index(prob, mode)
    rows = [r for r in range(model.dims[mode]) if row_ptr[r + 1] > row_ptr[r]][:3] + [
        r for r in range(model.dims[mode]) if row_ptr[r + 1] == row_ptr[r]][:1]
    for row in rows:
        before = model.copy()
        O.update_row(prob, model, mode, row, row_ptr, perm, reg, lam)
        walk = before.copy()
        for j in range(model.J[mode]):
            if walk.Amask[mode][row, j]:
                assert model.A[mode][row, j] == 0.0
                continue

            def f(a):
                walk.A[mode][row, j] = a
                return objective(prob, walk, reg, lam)

            best = coord_argmin(f, reg, before.A[mode][row, j])
            got = model.A[mode][row, j]
            assert abs(got - best) <= 1e-7 * max(1.0, abs(best)), (row, j, got, best)
            walk.A[mode][row, j] = got


@pytest.mark.parametrize("reg", [O.REG_LF, O.REG_L1])
def test_core_sweep_is_sequential_coordinate_minimiser(reg, oracle_lib):
    lam = 0.05 if reg == O.REG_LF else 0.8
    prob, model = small_problem(8, (5, 6, 4), (2, 3, 2), 80, masks=0.15)
    before = model.copy()
    O.sweep_core(prob, model, reg, lam)
    walk = before.copy()
    for b in range(model.G.size):  # linear order, j_1 fastest
        if walk.Gmask[b]:
            assert model.G[b] == 0.0
            continue

        def f(g):
            walk.G[b] = g
            return objective(prob, walk, reg, lam)

        best = coord_argmin(f, reg, before.G[b])
        assert abs(model.G[b] - best) <= 1e-7 * max(1.0, abs(best)), (b, model.G[b], best)
        walk.G[b] = model.G[b]


def _design_rows(model, prob, mode, row, row_ptr, perm):
    """Rows delta_alpha of the mode-`mode` least-squares problem for one factor row, via einsum."""
    Gt = model.core_tensor()
    D = []
    for p in range(row_ptr[row], row_ptr[row + 1]):
        a = perm[p]
        T = np.moveaxis(Gt, mode, 0)
        others = [k for k in range(model.N) if k != mode]
        for k in reversed(others):
            T = T @ model.A[k][prob.idx[k, a]]
        D.append(T)
    return np.array(D)


def test_row_gauss_seidel_reaches_ridge_solution(oracle_lib):
    lam = 0.3
    prob, model = small_problem(9, (5, 6, 7), (3, 2, 2), 120)
    mode = 0
    row_ptr, perm = O.build_index(prob, mode)
    row = int(np.argmax(np.diff(row_ptr)))
    D = _design_rows(model, prob, mode, row, row_ptr, perm)
    x = prob.x[perm[row_ptr[row]:row_ptr[row + 1]]]
    ridge = np.linalg.solve(D.T @ D + lam * np.eye(D.shape[1]), D.T @ x)
    for _ in range(3000):
        O.update_row(prob, model, mode, row, row_ptr, perm, O.REG_LF, lam)
    np.testing.assert_allclose(model.A[mode][row], ridge, rtol=1e-9, atol=1e-11)


def test_core_gauss_seidel_reaches_ridge_solution(oracle_lib):
    lam = 0.2
    prob, model = small_problem(10, (5, 4, 6), (2, 2, 2), 90)
    P = np.einsum("ai,aj,ak->aijk", model.A[0][prob.idx[0]], model.A[1][prob.idx[1]], model.A[2][prob.idx[2]])
    P = P.reshape(prob.nnz, -1, order="F")  # column = core linear index, j_1 fastest
    ridge = np.linalg.solve(P.T @ P + lam * np.eye(P.shape[1]), P.T @ prob.x)
    for _ in range(3000):
        O.sweep_core(prob, model, O.REG_LF, lam)
    np.testing.assert_allclose(model.G, ridge, rtol=1e-9, atol=1e-11)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("reg", [O.REG_LF, O.REG_L1])
def test_objective_monotone_and_masks_frozen(reg, oracle_lib):
    lam = 0.05 if reg == O.REG_LF else 0.5
    prob, model = small_problem(12, (15, 12, 10), (3, 4, 3), 600, masks=0.2)
    frozen = [m.copy() for m in model.Amask], model.Gmask.copy()
    prev = objective(prob, model, reg, lam)
    for _ in range(4):
        for mode in range(3):
            O.sweep_factors(prob, model, reg, lam, mode)
            cur = objective(prob, model, reg, lam)
            assert cur <= prev * (1 + 1e-12), (mode, prev, cur)
            prev = cur
        O.sweep_core(prob, model, reg, lam)
        cur = objective(prob, model, reg, lam)
        assert cur <= prev * (1 + 1e-12)
        prev = cur
    for n in range(3):
        assert np.all(model.A[n][frozen[0][n] == 1] == 0.0)
    assert np.all(model.G[frozen[1] == 1] == 0.0)


def test_responsibility_matches_brute_force_zeroing(oracle_lib):
    prob, model = small_problem(14, (6, 5, 4), (2, 3, 2), 70, masks=0.1)
    df, dc, rf, rc = O.responsibility(prob, model)
    base = sq_err(prob, model)
    xx = float(prob.x @ prob.x)
    re = np.sqrt(base / xx)
    for n in range(3):
        for (i, j), d in np.ndenumerate(df[n]):
            w = model.copy()
            w.A[n][i, j] = 0.0
            bf = sq_err(prob, w) - base
            assert abs(d - bf) <= 1e-10 * (base + abs(bf)), (n, i, j, d, bf)
            assert rf[n][i, j] == pytest.approx((np.sqrt((base + bf) / xx) - re) / re, rel=1e-8, abs=1e-12)
    for b in range(model.G.size):
        w = model.copy()
        w.G[b] = 0.0
        bf = sq_err(prob, w) - base
        assert abs(dc[b] - bf) <= 1e-10 * (base + abs(bf))


@pytest.mark.parametrize("count_mode", [0, 1])
def test_prune_matches_lexsort_selection(count_mode, oracle_lib):
    rng = np.random.default_rng(21)
    model = O.Model([rng.standard_normal((9, 4)), rng.standard_normal((7, 3))], rng.standard_normal(12))
    model.Amask[0][rng.random((9, 4)) < 0.3] = 1
    model.A[0][model.Amask[0] == 1] = 0.0
    df = [np.round(rng.standard_normal((9, 4)), 1), np.round(rng.standard_normal((7, 3)), 1)]  # many ties
    df[1][0, 0] = -0.0
    dc = np.round(rng.standard_normal(12), 1)
    pr = 0.3
    ref_masks = [m.copy() for m in model.Amask] + [model.Gmask.copy()]
    deltas = [d.ravel() for d in df] + [dc]
    n_ref = []
    for s, d in enumerate(deltas):
        m = ref_masks[s].reshape(-1)
        cand = np.nonzero(m == 0)[0]
        k = int(np.floor(pr * (m.size if count_mode else cand.size)))
        order = np.lexsort((cand, d[cand] + 0.0))
        m[cand[order[:k]]] = 1
        n_ref.append(k)
    n = O.prune(model, df, dc, pr, count_mode)
    np.testing.assert_array_equal(n, n_ref)
    for s in range(2):
        np.testing.assert_array_equal(model.Amask[s], ref_masks[s])
        assert np.all(model.A[s][model.Amask[s] == 1] == 0.0)
    np.testing.assert_array_equal(model.Gmask, ref_masks[2])
    # threshold mode
    m2 = O.Model([np.ones((3, 2)), np.ones((2, 2))], np.ones(4))
    n2 = O.prune(m2, [np.array([[0, 1], [2, -1], [5, 0.5]]), np.full((2, 2), 3.0)], np.array([0.1, 0.9, 2, 3]),
                 0.0, 0, 1, 1.0)
    np.testing.assert_array_equal(n2, [3, 0, 2])
    np.testing.assert_array_equal(m2.Amask[0], [[1, 0], [0, 1], [0, 1]])


def test_normalize_keeps_reconstruction(oracle_lib):
    rng = np.random.default_rng(5)
    A = [rng.standard_normal((5, 3)), rng.standard_normal((4, 2)), rng.standard_normal((6, 2))]
    A[1][:, 1] = 0.0  # a zero column
    model = O.Model(A, rng.standard_normal(12))
    ref = dense_recon(model)
    O.normalize(model)
    np.testing.assert_allclose(dense_recon(model), ref, rtol=1e-12, atol=1e-12)
    for n in range(3):
        norms = np.linalg.norm(model.A[n], axis=0)
        for j, v in enumerate(norms):
            assert v == pytest.approx(0.0 if (n == 1 and j == 1) else 1.0, abs=1e-14)


def test_elbow_stat_hand_values(oracle_lib):
    # (RE_t + RE_{t-2} - 2 RE_{t-1}) / pr_t
    assert O.elbow_stat(0.7, 0.8, 1.0, 0.03) == pytest.approx(0.1 / 0.03, rel=1e-14)
    assert O.elbow_stat(0.5, 0.5, 0.5, 0.01) == 0.0
    assert O.elbow_stat(0.6, 0.5, 0.5, 0.1) == pytest.approx(1.0, rel=1e-14)


def test_autosearch_manual_mode(oracle_lib):
    prob, model = small_problem(31, (12, 10, 8), (3, 3, 2), 500)
    target = 0.3
    p = O.Params(reg=O.REG_LF, lam=0.05, target_sparsity=target, max_iter=40, conv_tol=1e-9, normalize=0)
    rep = O.autosearch(prob, model, p)
    k = rep["stop_iter"]
    assert k > 0 and rep["sparsity"][k - 2] >= target and (k < 3 or rep["sparsity"][k - 3] < target)
    for t in range(1, k):  # pruned iterations follow pr_t = min(INIT_PR * t, MAX_PR)
        assert rep["pr"][t - 1] == pytest.approx(min(0.01 * t, 0.1))
    assert np.all(np.diff(rep["sparsity"]) >= 0)
    assert rep["final_sparsity"] >= target


def test_autosearch_auto_mode_stops_at_first_elbow(oracle_lib):
    prob, model = small_problem(32, (12, 10, 8), (3, 3, 2), 500)
    p = O.Params(reg=O.REG_LF, lam=0.05, target_sparsity=-1.0, max_iter=60, conv_tol=1e-7, normalize=0)
    rep = O.autosearch(prob, model, p)
    re = rep["re"]
    fire = None
    for t in range(3, rep["iters"] + 1):
        pr = min(0.01 * t, 0.1)
        if (re[t - 1] + re[t - 3] - 2 * re[t - 2]) / pr > 0.05:
            fire = t
            break
    assert rep["stop_iter"] == (fire or 0)


def test_autosearch_elbow_rise_waits_for_a_rising_error(oracle_lib):
    """With elbow_rise the stop is the first t >= 3 whose second difference exceeds the threshold
    while RE_t > RE_{t-1}; RE falls at every pruned iteration before it."""
    prob, model = small_problem(42, (30, 25, 20), (3, 3, 3), 3000)
    p = O.Params(reg=O.REG_LF, lam=0.05, target_sparsity=-1.0, max_iter=30, conv_tol=1e-7, normalize=0, elbow_rise=1)
    rep = O.autosearch(prob, model, p)
    re = rep["re"]
    fire = None
    for t in range(3, rep["iters"] + 1):
        pr = min(0.01 * t, 0.1)
        if re[t - 1] > re[t - 2] and (re[t - 1] + re[t - 3] - 2 * re[t - 2]) / pr > 0.05:
            fire = t
            break
    assert fire is not None and rep["stop_iter"] == fire
    assert np.all(np.diff(re[:fire - 1]) < 0)
    assert rep["sparsity"][fire - 2] > rep["sparsity"][1]  # pruning went on past the early sweeps


def test_autosearch_revive_restores_the_masks_before_the_last_prune(oracle_lib):
    """VeST_auto with revive_on_stop: when the elbow fires at iteration k, the masks go back to
    those after iteration k-2 (before the prune of iteration k-1); the run up to k is unchanged."""
    def run(revive, max_iter):
        prob, model = small_problem(42, (30, 25, 20), (3, 3, 3), 3000)
        p = O.Params(reg=O.REG_LF, lam=0.05, init_pr=0.05, max_pr=0.2, target_sparsity=-1.0, max_iter=max_iter,
                     conv_tol=1e-9, normalize=0, revive_on_stop=revive)
        return O.autosearch(prob, model, p), model

    plain, m_plain = run(0, 30)
    rev, m_rev = run(1, 30)
    k = rev["stop_iter"]
    assert k == plain["stop_iter"] and k >= 3
    np.testing.assert_array_equal(rev["re"][:k], plain["re"][:k])
    np.testing.assert_array_equal(rev["sparsity"][:k], plain["sparsity"][:k])
    before, m_before = run(0, k - 2)  # stops right after the prune of iteration k-2
    assert before["iters"] == k - 2
    for a, b in zip(m_rev.Amask, m_before.Amask):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(m_rev.Gmask, m_before.Gmask)
    assert any((a != b).any() for a, b in zip(m_plain.Amask + [m_plain.Gmask], m_before.Amask + [m_before.Gmask]))
    # revived elements are refit by the next sweep: the value sparsity drops back to that of k-2
    assert rev["sparsity"][k] == plain["sparsity"][k - 3] < plain["sparsity"][k]


@pytest.mark.parametrize("split", [5, 8])
def test_autosearch_resume_equals_one_run(oracle_lib, split):
    """A run stopped after `split` iterations (no normalisation) and resumed from its report to
    max_iter gives the same report and model as one run to max_iter; the manual-mode stop falls
    at iteration 6, so the two splits resume before and after it."""
    def params(max_iter, normalize, resume):
        return O.Params(reg=O.REG_LF, lam=0.05, init_pr=0.05, max_pr=0.2, target_sparsity=0.5, max_iter=max_iter,
                        conv_tol=1e-9, normalize=normalize, resume=resume)

    prob, one = small_problem(42, (30, 25, 20), (3, 3, 3), 3000)
    whole = O.autosearch(prob, one, params(12, 1, 0))
    _, two = small_problem(42, (30, 25, 20), (3, 3, 3), 3000)
    first = O.autosearch(prob, two, params(split, 0, 0))
    assert first["iters"] == split and whole["stop_iter"] == 6
    rest = O.autosearch(prob, two, params(12, 1, 1), resume_from=first)
    assert rest["iters"] == whole["iters"] and rest["stop_iter"] == whole["stop_iter"]
    for key in ("re", "obj", "pr", "sparsity"):
        np.testing.assert_array_equal(rest[key], whole[key])
    for a, b in zip(one.A + [one.G], two.A + [two.G]):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(one.Amask + [one.Gmask], two.Amask + [two.Gmask]):
        np.testing.assert_array_equal(a, b)


def test_planted_model_is_recovered(oracle_lib):
    # noiseless, fully observed, rank-matched: CD drives RE towards 0 (a sanity check,
    # not a pin: the problem is non-convex and some starts plateau for a long time)
    rng = np.random.default_rng(4)
    dims, ranks = (6, 6, 6), (2, 2, 2)
    truth = O.Model([rng.standard_normal((d, r)) for d, r in zip(dims, ranks)], rng.standard_normal(8))
    full = np.array(np.unravel_index(np.arange(216), dims))
    prob = O.Problem(dims, full, dense_recon(truth)[tuple(full)])
    init = datagen.random_init(dims, ranks, 4)
    model = O.Model(init.factors, init.core)
    for _ in range(300):
        O.sweep_factors(prob, model, O.REG_LF, 1e-6, -1)
        O.sweep_core(prob, model, O.REG_LF, 1e-6)
    assert O.loss(prob, model, O.REG_LF, 1e-6)[4] < 1e-2


def test_ctypes_structs_match_the_oracle_header(tmp_path):
    """Every field of the oracle's C structs, as gcc lays them out, equals its ctypes mirror."""
    import ctypes as C
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    pairs = [(O._Tensor, "or_tensor"), (O._Model, "or_model"), (O._Params, "or_params"), (O._Report, "or_report")]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vest_oracle.h"', "int main(void) {"]
    for st, cname in pairs:
        for name, _ in st._fields_:
            field = "lambda" if name == "lambda_" else name
            lines.append(f'  printf("{cname} {name} %zu %zu\\n", offsetof({cname}, {field}), '
                         f"sizeof((({cname}*)0)->{field}));")
        lines.append(f'  printf("{cname} SIZE %zu 0\\n", sizeof({cname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    here = os.path.dirname(os.path.abspath(O.__file__))
    subprocess.run(["gcc", "-std=c11", "-I", here, str(src), "-o", str(exe)], check=True)
    out = [x for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n") if x]
    assert len(out) == sum(len(st._fields_) + 1 for st, _ in pairs)
    by_name = {cname: st for st, cname in pairs}
    for line in out:
        cname, field, off, size = line.split()
        st = by_name[cname]
        if field == "SIZE":
            assert C.sizeof(st) == int(off), cname
        else:
            f = getattr(st, field)
            assert (f.offset, f.size) == (int(off), int(size)), (cname, field)
