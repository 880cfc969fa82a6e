"""More shapes for one full iteration against the oracle: rank 1 in a mode, orders 6 and 8,
rank 16 beside rank 1 (the rank buckets' extremes), each with pruned elements."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1904_02603_gb300 import datagen
from paper_1904_02603_gb300 import vest as V
from gpu_common import device_pair, masks_equal, model_err, oracle_pair, rel_err, with_masks

pytestmark = pytest.mark.gpu
TOL64 = 1e-9

SHAPES = {
    "rank1_n3": dict(dims=(50, 40, 30), ranks=(1, 4, 3), nnz=3000),
    "rank1_first_two": dict(dims=(30, 30, 30), ranks=(1, 1, 5), nnz=2500),
    "n6": dict(dims=(6, 5, 6, 5, 6, 5), ranks=(2, 2, 3, 2, 2, 2), nnz=2500),
    "n8": dict(dims=(4,) * 8, ranks=(2,) * 8, nnz=2000),
    "rank16_rank1": dict(dims=(40, 50, 30), ranks=(16, 1, 2), nnz=3000),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02603_gb300 import build as B
    B.build()
    V.load()


@pytest.mark.parametrize("name", list(SHAPES))
def test_iteration_f64_more_shapes(name):
    c = SHAPES[name]
    t, st = datagen.random_problem(300 + sum(map(ord, name)), c["dims"], c["ranks"], c["nnz"])
    st = with_masks(st, 0.05, 19)
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    prob, om = oracle_pair(t, st)
    lam, pr = 0.05, 0.05
    for it in range(2):
        loss, df, dc, npr = V.vest_iteration(ix, mdl, V.REG_LF, lam, pr, sc)
        O.sweep_factors(prob, om, V.REG_LF, lam, -1)
        O.sweep_core(prob, om, V.REG_LF, lam)
        oloss = O.loss(prob, om, V.REG_LF, lam)
        odf, odc, _, _ = O.responsibility(prob, om)
        onp = O.prune(om, odf, odc, pr, 0)
        assert rel_err(loss.cpu().numpy(), oloss) < TOL64, (it, loss.cpu().numpy(), oloss)
        for n in range(t.N):
            assert rel_err(df[n].cpu().numpy(), odf[n]) < TOL64, (it, n)
        assert rel_err(dc.cpu().numpy(), odc) < TOL64
        np.testing.assert_array_equal(npr.cpu().numpy(), onp)
        assert masks_equal(mdl, om)
        assert model_err(mdl, om) < TOL64
