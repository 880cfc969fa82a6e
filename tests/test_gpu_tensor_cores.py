"""Parity of the tensor-core FP32 factor sweep (Eq. 11 on tcgen05 in split TF32) with the FP64 oracle.

The FP32 factor sweep takes the tensor-core kernel whenever the model's other modes split into one
or two "A" modes and at most one remaining mode (ranks up to 16); the cases below cover both splits
(3-order and 2-order models take one A mode, 4-order models two), every rank bucket (4, 8, 10, 12,
16), ragged task tails, heavy Zipf rows cut across many tasks, pruned elements and empty rows.
Each mode's sweep and each mode's responsibility (Eq. 6) are compared with the oracle element by
element, relative to the largest magnitude, within 1e-4: FP32 storage with about 21-bit products
and FP32 row sums put the error near 1e-6, while a wrong index, column or core permutation gives
errors of order one.  A last test runs the same sweep with the tensor cores switched off
(VEST_TENSOR_CORES=0, the FMA kernels) in a child process: both paths agree within the same
tolerance and are not bitwise equal, which shows the tensor-core kernel is the one that ran.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1904_02603_gb300 import datagen  # noqa: E402
from paper_1904_02603_gb300 import vest as V  # noqa: E402
from gpu_common import oracle_pair, rel_err, with_masks  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4

# name: dims, ranks, nnz, index law; the A-mode split each mode takes is noted
TC_CASES = {
    "n3_rank10_zipf": dict(dims=(300, 2000, 2000), ranks=(10, 10, 10), nnz=30000, dist="zipf"),  # 1 A mode
    "n4_rank8": dict(dims=(40, 30, 30, 25), ranks=(8, 8, 8, 8), nnz=20011),  # 2 A modes
    "n3_mixed": dict(dims=(200, 150, 90), ranks=(3, 7, 10), nnz=12345),  # buckets 4, 8, 10
    "n3_rank12_16": dict(dims=(120, 100, 80), ranks=(12, 16, 5), nnz=9000),  # buckets 12, 16
    "n2_rank9": dict(dims=(700, 500), ranks=(9, 6), nnz=20000),  # no remaining mode
    "n4_mixed": dict(dims=(30, 25, 20, 15), ranks=(5, 6, 7, 3), nnz=6000),
    "n3_tail": dict(dims=(50, 40, 30), ranks=(6, 5, 4), nnz=257),  # one full task and one entry
    # a rank above 16: no padded factor copies, so mode 0 (bucket 32) reads the caller's rows,
    # of odd length (7 and 5), one element at a time; modes 1 and 2 take the FMA kernels
    "n3_rank20_odd": dict(dims=(60, 50, 40), ranks=(20, 7, 5), nnz=7000),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02603_gb300 import build as B
    B.build()
    V.load()


def _case(name, masked=False):
    c = TC_CASES[name]
    t, st = datagen.random_problem(300 + sum(map(ord, name)), c["dims"], c["ranks"], c["nnz"], dtype=np.float32,
                                   dist=c.get("dist", "uniform"))
    if masked:
        st = with_masks(st, 0.2, seed=7)
    return t, st


def _device(t, st):
    ten = V.Tensor(t.dims, torch.from_numpy(t.idx).cuda(), torch.from_numpy(t.val.astype(np.float32)).cuda())
    return ten, V.Model.from_host(st.astype(np.float32))


@pytest.mark.parametrize("name", sorted(TC_CASES))
@pytest.mark.parametrize("reg", [V.REG_LF, V.REG_L1])
def test_tensor_core_factor_sweep_matches_oracle(name, reg):
    t, st = _case(name, masked=(reg == V.REG_L1))
    ten, mdl = _device(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    prob, om = oracle_pair(t, st.astype(np.float32).astype(np.float64))
    lam = 0.05
    for n in range(t.N):
        V.vest_sweep_factors(ix, mdl, reg, lam, n, sc)
        O.sweep_factors(prob, om, reg, lam, n)
        got = mdl.factors[n].cpu().numpy()
        err = rel_err(got, om.A[n])
        assert err < TOL, (name, n, err)
        # the device result feeds the next mode on both sides, so errors do not compound
        om.A[n] = got.astype(np.float64)
    assert V.vest_device_status() == 0


@pytest.mark.parametrize("name", sorted(TC_CASES))
def test_tensor_core_responsibility_matches_oracle(name):
    t, st = _case(name)
    ten, mdl = _device(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    df, dc, _, _ = V.vest_responsibility(ix, mdl, sc, with_resp=False)
    prob, om = oracle_pair(t, st.astype(np.float32).astype(np.float64))
    odf, odc, _, _ = O.responsibility(prob, om)
    for n in range(t.N):
        assert rel_err(df[n].cpu().numpy(), odf[n]) < TOL, (name, n)
    assert rel_err(dc.cpu().numpy(), odc) < TOL


def test_tensor_core_sweep_is_deterministic():
    t, st = _case("n3_rank10_zipf")
    outs = []
    for _ in range(2):
        ten, mdl = _device(t, st)
        ix = V.vest_build_index(ten)
        sc = V.make_scratch(ix, mdl)
        V.vest_sweep_factors(ix, mdl, V.REG_LF, 0.05, -1, sc)
        outs.append([f.cpu().numpy() for f in mdl.factors])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


_CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1904_02603_gb300 import vest as V
sys.path.insert(0, {root!r} + "/tests")
from test_gpu_tensor_cores import _case, _device
V.load()
t, st = _case("n3_rank10_zipf")
ten, mdl = _device(t, st)
ix = V.vest_build_index(ten)
sc = V.make_scratch(ix, mdl)
V.vest_sweep_factors(ix, mdl, V.REG_LF, 0.05, -1, sc)
print(json.dumps([f.cpu().numpy().tolist() for f in mdl.factors]))
"""


def test_tensor_core_and_fma_paths_agree_but_differ():
    env = dict(os.environ, VEST_TENSOR_CORES="0")
    out = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], capture_output=True, text=True, env=env,
                         cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    fma = [np.array(a, np.float32) for a in json.loads(out.stdout.strip().splitlines()[-1])]
    t, st = _case("n3_rank10_zipf")
    ten, mdl = _device(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    V.vest_sweep_factors(ix, mdl, V.REG_LF, 0.05, -1, sc)
    tcs = [f.cpu().numpy() for f in mdl.factors]
    assert max(rel_err(a, b) for a, b in zip(tcs, fma)) < TOL
    assert any(not np.array_equal(a, b) for a, b in zip(tcs, fma))


@pytest.mark.parametrize("name", sorted(TC_CASES))
def test_tensor_core_loss_matches_oracle(name):
    """vest_loss on an FP32 model takes the tensor-core loss kernel (delta^(0) by the MMA, dotted
    with the mode-0 row): the residuals (Eq. 7) and the five loss values against the oracle."""
    t, st = _case(name, masked=True)
    ten, mdl = _device(t, st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    resid = torch.empty(t.nnz, dtype=torch.float32, device="cuda")
    out = V.vest_loss(ix, mdl, V.REG_L1, 0.05, sc, resid=resid).cpu().numpy()
    prob, om = oracle_pair(t, st.astype(np.float32).astype(np.float64))
    ref = O.loss(prob, om, O.REG_L1, 0.05)
    r_ref = prob.x - O.reconstruct(prob, om)
    assert rel_err(resid.cpu().numpy(), r_ref) < TOL, name
    assert np.all(np.abs(out - ref) <= TOL * np.abs(ref)), (out, ref)
    assert V.vest_device_status() == 0
