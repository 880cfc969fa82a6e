"""CPU round trip of an auto-search checkpoint file (model, marking tables, report)."""
import numpy as np

from paper_1904_02603_gb300 import checkpoint, datagen
from paper_1904_02603_gb300 import vest as V


def test_checkpoint_round_trip(tmp_path):
    st = datagen.random_init((7, 5, 4), (3, 2, 2), seed=3)
    st.factor_masks[1][2, 1] = 1
    st.core_mask[5] = 1
    model = V.Model.from_host(st, device="cpu")
    report = {"iters": 4, "stop_iter": 3, "re": np.array([0.9, 0.8, 0.75, 0.74]), "obj": np.arange(4.0),
              "pr": np.array([0.01, 0.02, 0.0, 0.0]), "sparsity": np.array([0.0, 0.05, 0.1, 0.1])}
    checkpoint.save(tmp_path / "c.npz", model, report)
    back, rep = checkpoint.load(tmp_path / "c.npz", device="cpu")
    for a, b in zip(model.to_host(), back.to_host()):
        for x, y in zip(a if isinstance(a, list) else [a], b if isinstance(b, list) else [b]):
            assert x.dtype == y.dtype
            np.testing.assert_array_equal(x, y)
    assert rep["iters"] == 4 and rep["stop_iter"] == 3
    for k in ("re", "obj", "pr", "sparsity"):
        np.testing.assert_array_equal(rep[k], report[k])
