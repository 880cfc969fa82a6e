"""vest_loss_noalloc: the loss computed with the library's fixed device scratch
array instead of a caller buffer, for callers that cannot allocate device memory
when they need the loss.  Checked through the C ABI against vest_loss on the
same inputs, on two calls in a row (the second call reuses the array the first
one left behind).  Collected last so a stop-at-first-failure run has already
run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02603_gb300 import build as B
    from paper_1904_02603_gb300 import vest as V
    B.build()
    return V.load()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_loss_matches_scratch_loss_twice(lib, dtype):
    from paper_1904_02603_gb300 import datagen
    from paper_1904_02603_gb300 import vest as V
    npdt = np.float64 if dtype == torch.float64 else np.float32
    t, st = datagen.random_problem(77, (300, 200, 150), (6, 5, 4), 20000, dtype=npdt, dist="zipf")
    ten = V.Tensor(t.dims, torch.from_numpy(t.idx).cuda(), torch.from_numpy(t.val).cuda())
    mdl = V.Model.from_host(st)
    ix = V.vest_build_index(ten)
    sc = V.make_scratch(ix, mdl)
    ref = V.vest_loss(ix, mdl, V.REG_L1, 0.25, sc).cpu().numpy()
    ref_r = torch.empty(t.nnz, dtype=dtype, device="cuda")
    V.vest_loss(ix, mdl, V.REG_L1, 0.25, sc, resid=ref_r)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        resid = torch.full((t.nnz,), float("nan"), dtype=dtype, device="cuda")
        rc = lib.vest_loss_noalloc(ix.handle, C.byref(mdl.cstruct()), V.REG_L1, 0.25, C.c_void_p(out.data_ptr()),
                                   C.c_void_p(resid.data_ptr()), stream)
        assert rc == 0, lib.vest_last_error()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0), call
        np.testing.assert_allclose(resid.cpu().numpy(), ref_r.cpu().numpy(), rtol=1e-12, atol=1e-12), call


def test_noalloc_rejects_a_core_beyond_its_limit(lib):
    from paper_1904_02603_gb300 import vest as V
    dims, ranks = (4, 4, 4, 4, 4), (32, 32, 16, 16, 1)  # permuted core of 262144 doubles > 1 MiB
    t = V.Tensor(dims, torch.zeros((5, 1), dtype=torch.int32, device="cuda"),
                 torch.ones(1, dtype=torch.float64, device="cuda"))
    ix = V.vest_build_index(t)
    m = V.Model([torch.rand(d, r, dtype=torch.float64, device="cuda") for d, r in zip(dims, ranks)],
                torch.rand(int(np.prod(ranks)), dtype=torch.float64, device="cuda"))
    with pytest.raises(V.VestError) as e:
        V.vest_loss_noalloc(ix, m, V.REG_LF, 0.1)
    assert e.value.status == 4 and "1 MiB" in str(e.value)
