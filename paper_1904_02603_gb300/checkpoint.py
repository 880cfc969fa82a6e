"""Checkpoints of long auto-search runs (Algorithm 2).

A checkpoint is the model as it stands (factors, core and both marking tables) and the report of
the run so far (iterations done, where pruning stopped, the RE, objective, pruning-rate and
sparsity histories), written to one .npz file on the host.  `load` puts the model back on the
device; `vest_autosearch(..., params(resume=1, ...), resume_from=report)` then continues the run
from the next iteration.  A run of K iterations without the final normalisation, saved, loaded
and resumed, ends bitwise where one uninterrupted run ends.
"""
from __future__ import annotations

import numpy as np

from . import vest as V

_HIST = ("re", "obj", "pr", "sparsity")


class _State:
    def __init__(self, factors, core, factor_masks, core_mask):
        self.factors, self.core, self.factor_masks, self.core_mask = factors, core, factor_masks, core_mask


def save(path, model: V.Model, report: dict) -> None:
    f, c, fm, cm = model.to_host()
    arrays = {f"factor{n}": a for n, a in enumerate(f)}
    arrays.update({f"mask{n}": a for n, a in enumerate(fm)})
    arrays.update(core=c, core_mask=cm, order=np.array(len(f), np.int64),
                  counts=np.array([report["iters"], report["stop_iter"]], np.int64))
    arrays.update({f"hist_{k}": np.asarray(report[k], np.float64) for k in _HIST})
    np.savez(path, **arrays)


def load(path, device="cuda"):
    """Returns (model on `device`, report to resume from)."""
    with np.load(path) as z:
        n = int(z["order"])
        st = _State([z[f"factor{i}"] for i in range(n)], z["core"], [z[f"mask{i}"] for i in range(n)], z["core_mask"])
        report = {"iters": int(z["counts"][0]), "stop_iter": int(z["counts"][1])}
        report.update({k: z[f"hist_{k}"].copy() for k in _HIST})
    return V.Model.from_host(st, device=device), report
