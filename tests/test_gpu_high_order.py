"""Order 10 with every rank 3, the top of the order series of the scalability study (Section 4.4).

At this order the permuted core (3^10 elements, padded to 4 per mode-n fibre) no longer fits in
shared memory, so the factor sweep and the loss read it from global memory, and the core
sweep runs 3^8 = 6561 blocks of 9 elements.  No other parity case reaches these paths.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1904_02603_gb300 import datagen
from paper_1904_02603_gb300 import vest as V
from gpu_common import device_pair, masks_equal, model_err, oracle_pair, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02603_gb300 import build as B
    B.build()
    V.load()


@pytest.fixture(scope="module")
def order10():
    return datagen.uniform_tensor(10, 5, 200, seed=4242, dtype=np.float64)


def test_order10_iteration_f64(order10):
    """One vest_iteration (both sweeps, loss, responsibility, prune) against the oracle's steps."""
    t, st = order10
    ten, mdl = device_pair(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    prob, om = oracle_pair(t, st)
    lam, pr = 0.05, 0.05
    loss, df, dc, npr = V.vest_iteration(ix, mdl, V.REG_LF, lam, pr, sc)
    O.sweep_factors(prob, om, V.REG_LF, lam, -1)
    O.sweep_core(prob, om, V.REG_LF, lam)
    oloss = O.loss(prob, om, V.REG_LF, lam)
    odf, odc, _, _ = O.responsibility(prob, om)
    onp = O.prune(om, odf, odc, pr, 0)
    assert rel_err(loss.cpu().numpy(), oloss) < TOL64, (loss.cpu().numpy(), oloss)
    for n in range(t.N):
        assert rel_err(df[n].cpu().numpy(), odf[n]) < TOL64, n
    assert rel_err(dc.cpu().numpy(), odc) < TOL64
    np.testing.assert_array_equal(npr.cpu().numpy(), onp)
    assert masks_equal(mdl, om)
    assert model_err(mdl, om) < TOL64


def test_order10_fp32_loss_and_iteration(order10):
    """FP32: the loss kernel (global-memory core) against the oracle's loss of the same model,
    and one iteration's objective against the FP64 path's (same start, rounding apart)."""
    t, st = order10
    ten32, m32 = device_pair(t, st, torch.float32)
    ix32 = V.vest_build_index(ten32)
    sc32 = V.make_scratch(ix32, m32)
    ten64, m64 = device_pair(t, st)
    ix64 = V.vest_build_index(ten64)
    sc64 = V.make_scratch(ix64, m64)
    lam = 0.05
    l32, _, _, _ = V.vest_iteration(ix32, m32, V.REG_LF, lam, 0.0, sc32, with_responsibility=False)
    l64, _, _, _ = V.vest_iteration(ix64, m64, V.REG_LF, lam, 0.0, sc64, with_responsibility=False)
    obj32, obj64 = float(l32.cpu().numpy()[3]), float(l64.cpu().numpy()[3])
    assert abs(obj32 - obj64) <= 1e-2 * abs(obj64), (obj32, obj64)
    # the FP32 model as it stands, scored by the FP32 loss kernel and by the oracle in FP64
    f, c, fm, cm = m32.to_host()
    prob, _ = oracle_pair(t, st)
    om = O.Model([a.astype(np.float64) for a in f], c.astype(np.float64), fm, cm)
    got = V.vest_loss(ix32, m32, V.REG_LF, lam, sc32).cpu().numpy()
    ref = O.loss(prob, om, V.REG_LF, lam)
    assert rel_err(got[:4], ref[:4]) < 1e-5, (got, ref)
