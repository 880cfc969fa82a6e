"""ctypes front end of the FP64 CPU oracle (``oracle/vest_oracle.c``).

TEST INFRASTRUCTURE ONLY: ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product library never does.  Nothing here shares code with the
CUDA path.  The arithmetic lives in the C file; this module only marshals
numpy arrays into the C structs and back.

Parity status per function (what pins each one is in ``tests/test_oracle_pins.py``
and ``tests/golden/``):
  or_entry / or_loss            pinned: dense n-mode-product reconstruction
  or_build_index                pinned: numpy stable argsort
  or_update_row / sweep_factors pinned: brute-force 1-D minimisation, ridge closed form, hand example
  or_sweep_core                 pinned: brute-force 1-D minimisation, ridge closed form, hand example
  or_responsibility             pinned: brute-force zeroing of each element
  or_prune                      pinned: numpy lexsort selection
  or_normalize                  pinned: reconstruction invariance, unit column norms
  or_elbow_stat / or_autosearch pinned: hand-built RE sequences, monotonicity, sparsity invariants
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

MAX_ORDER = 10
REG_LF, REG_L1 = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    src = os.path.join(_HERE, "vest_oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(os.path.join(_HERE, "vest_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Tensor(C.Structure):
    _fields_ = [("N", C.c_int32), ("I", C.c_int64 * MAX_ORDER), ("nnz", C.c_int64),
                ("idx", C.POINTER(C.c_int32)), ("x", C.POINTER(C.c_double))]


class _Model(C.Structure):
    _fields_ = [("N", C.c_int32), ("I", C.c_int64 * MAX_ORDER), ("J", C.c_int32 * MAX_ORDER),
                ("A", C.POINTER(C.c_double) * MAX_ORDER), ("Amask", C.POINTER(C.c_uint8) * MAX_ORDER),
                ("G", C.POINTER(C.c_double)), ("Gmask", C.POINTER(C.c_uint8))]


class _Params(C.Structure):
    _fields_ = [("reg", C.c_int32), ("lambda_", C.c_double), ("init_pr", C.c_double),
                ("max_pr", C.c_double), ("elbow_thresh", C.c_double), ("target_sparsity", C.c_double),
                ("conv_tol", C.c_double), ("max_iter", C.c_int32), ("fixed_pr_mode", C.c_int32),
                ("fixed_pr", C.c_double), ("count_mode", C.c_int32), ("normalize", C.c_int32),
                ("revive_on_stop", C.c_int32), ("resume", C.c_int32), ("elbow_rise", C.c_int32)]


class _Report(C.Structure):
    _fields_ = [("iters", C.c_int32), ("stop_iter", C.c_int32), ("re_hist", C.c_double * 256),
                ("obj_hist", C.c_double * 256), ("pr_hist", C.c_double * 256),
                ("sparsity_hist", C.c_double * 256), ("final_sparsity", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            d, i32, i64 = C.c_double, C.c_int32, C.c_int64
            PT, PM = C.POINTER(_Tensor), C.POINTER(_Model)
            PD, PI32, PI64 = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
            PPD = C.POINTER(C.POINTER(C.c_double))
            sig = {
                "or_entry": (d, [PM, PI32]),
                "or_reconstruct": (C.c_int, [PT, PM, PD]),
                "or_loss": (C.c_int, [PT, PM, i32, d, PD]),
                "or_build_index": (C.c_int, [PT, i32, PI64, PI32]),
                "or_delta": (None, [PM, i32, PI32, PD]),
                "or_update_row": (C.c_int, [PT, PM, i32, i64, PI64, PI32, i32, d]),
                "or_sweep_factors": (C.c_int, [PT, PM, i32, d, i32]),
                "or_sweep_core": (C.c_int, [PT, PM, i32, d]),
                "or_responsibility": (C.c_int, [PT, PM, PPD, PD, PPD, PD]),
                "or_prune": (C.c_int, [PM, PPD, PD, d, i32, i32, d, PI64]),
                "or_normalize": (C.c_int, [PM]),
                "or_sparsity": (d, [PM]),
                "or_elbow_stat": (d, [d, d, d, d]),
                "or_autosearch": (C.c_int, [PT, PM, C.POINTER(_Params), C.POINTER(_Report)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


@dataclass
class Problem:
    """Observed entries: idx (N, nnz) int32 0-based, x (nnz,) float64."""
    dims: tuple
    idx: np.ndarray
    x: np.ndarray

    def __post_init__(self):
        self.idx = np.ascontiguousarray(self.idx, dtype=np.int32)
        self.x = np.ascontiguousarray(self.x, dtype=np.float64)
        self.dims = tuple(int(d) for d in self.dims)

    @property
    def N(self):
        return len(self.dims)

    @property
    def nnz(self):
        return int(self.x.shape[0])

    def cstruct(self):
        t = _Tensor()
        t.N = self.N
        for n, d in enumerate(self.dims):
            t.I[n] = d
        t.nnz = self.nnz
        t.idx = _ptr(self.idx, C.c_int32)
        t.x = _ptr(self.x, C.c_double)
        return t


@dataclass
class Model:
    """A: list of (I_n, J_n) float64; G: flat core (j_1 fastest); masks uint8 (1 = pruned)."""
    A: list
    G: np.ndarray
    Amask: list = field(default=None)
    Gmask: np.ndarray = field(default=None)

    def __post_init__(self):
        self.A = [np.ascontiguousarray(a, dtype=np.float64) for a in self.A]
        self.G = np.ascontiguousarray(np.asarray(self.G, dtype=np.float64).reshape(-1))
        if self.Amask is None:
            self.Amask = [np.zeros(a.shape, np.uint8) for a in self.A]
        self.Amask = [np.ascontiguousarray(m, dtype=np.uint8) for m in self.Amask]
        if self.Gmask is None:
            self.Gmask = np.zeros(self.G.shape, np.uint8)
        self.Gmask = np.ascontiguousarray(np.asarray(self.Gmask, dtype=np.uint8).reshape(-1))
        assert self.G.size == int(np.prod(self.J))

    @property
    def N(self):
        return len(self.A)

    @property
    def J(self):
        return tuple(a.shape[1] for a in self.A)

    @property
    def dims(self):
        return tuple(a.shape[0] for a in self.A)

    def copy(self):
        return Model([a.copy() for a in self.A], self.G.copy(), [m.copy() for m in self.Amask], self.Gmask.copy())

    def core_tensor(self):
        """Core as an ndarray indexed [j_1, ..., j_N]."""
        return self.G.reshape(self.J, order="F")

    def cstruct(self):
        m = _Model()
        m.N = self.N
        for n, a in enumerate(self.A):
            m.I[n] = a.shape[0]
            m.J[n] = a.shape[1]
            m.A[n] = _ptr(a, C.c_double)
            m.Amask[n] = _ptr(self.Amask[n], C.c_uint8)
        m.G = _ptr(self.G, C.c_double)
        m.Gmask = _ptr(self.Gmask, C.c_uint8)
        return m


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def entry(model: Model, i) -> float:
    i = np.ascontiguousarray(i, dtype=np.int32)
    m = model.cstruct()
    return lib().or_entry(C.byref(m), _ptr(i, C.c_int32))


def reconstruct(prob: Problem, model: Model) -> np.ndarray:
    out = np.zeros(prob.nnz, np.float64)
    t, m = prob.cstruct(), model.cstruct()
    _check(lib().or_reconstruct(C.byref(t), C.byref(m), _ptr(out, C.c_double)), "reconstruct")
    return out


def loss(prob: Problem, model: Model, reg: int, lam: float) -> np.ndarray:
    """[sum r^2, sum x^2, reg term, objective, RE]."""
    out = np.zeros(5, np.float64)
    t, m = prob.cstruct(), model.cstruct()
    _check(lib().or_loss(C.byref(t), C.byref(m), reg, lam, _ptr(out, C.c_double)), "loss")
    return out


def build_index(prob: Problem, mode: int):
    row_ptr = np.zeros(prob.dims[mode] + 1, np.int64)
    t = prob.cstruct()
    perm_buf = np.zeros(max(prob.nnz, 1), np.int32)
    _check(lib().or_build_index(C.byref(t), mode, _ptr(row_ptr, C.c_int64), _ptr(perm_buf, C.c_int32)),
           "build_index")
    perm = perm_buf[: prob.nnz].copy()
    return row_ptr, perm


def delta(model: Model, mode: int, i) -> np.ndarray:
    i = np.ascontiguousarray(i, dtype=np.int32)
    out = np.zeros(model.J[mode], np.float64)
    m = model.cstruct()
    lib().or_delta(C.byref(m), mode, _ptr(i, C.c_int32), _ptr(out, C.c_double))
    return out


def update_row(prob: Problem, model: Model, mode: int, row: int, row_ptr, perm, reg: int, lam: float):
    t, m = prob.cstruct(), model.cstruct()
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    if perm.size == 0:
        perm = np.zeros(1, np.int32)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    _check(lib().or_update_row(C.byref(t), C.byref(m), mode, row, _ptr(row_ptr, C.c_int64),
                               _ptr(perm, C.c_int32), reg, lam), "update_row")


def sweep_factors(prob: Problem, model: Model, reg: int, lam: float, mode: int = -1):
    t, m = prob.cstruct(), model.cstruct()
    _check(lib().or_sweep_factors(C.byref(t), C.byref(m), reg, lam, mode), "sweep_factors")


def sweep_core(prob: Problem, model: Model, reg: int, lam: float):
    t, m = prob.cstruct(), model.cstruct()
    _check(lib().or_sweep_core(C.byref(t), C.byref(m), reg, lam), "sweep_core")


def responsibility(prob: Problem, model: Model):
    """Returns (delta_factor list, delta_core, resp_factor list, resp_core)."""
    t, m = prob.cstruct(), model.cstruct()
    df = [np.zeros(a.shape, np.float64) for a in model.A]
    rf = [np.zeros(a.shape, np.float64) for a in model.A]
    dc = np.zeros(model.G.shape, np.float64)
    rc = np.zeros(model.G.shape, np.float64)
    dfp = (C.POINTER(C.c_double) * model.N)(*[_ptr(a, C.c_double) for a in df])
    rfp = (C.POINTER(C.c_double) * model.N)(*[_ptr(a, C.c_double) for a in rf])
    _check(lib().or_responsibility(C.byref(t), C.byref(m), dfp, _ptr(dc, C.c_double), rfp,
                                   _ptr(rc, C.c_double)), "responsibility")
    return df, dc, rf, rc


def prune(model: Model, delta_factor, delta_core, pr: float, count_mode: int = 0,
          threshold_mode: int = 0, tau: float = 0.0) -> np.ndarray:
    m = model.cstruct()
    df = [np.ascontiguousarray(a, dtype=np.float64) for a in delta_factor]
    dc = np.ascontiguousarray(delta_core, dtype=np.float64)
    dfp = (C.POINTER(C.c_double) * model.N)(*[_ptr(a, C.c_double) for a in df])
    n_pruned = np.zeros(model.N + 1, np.int64)
    _check(lib().or_prune(C.byref(m), dfp, _ptr(dc, C.c_double), pr, count_mode, threshold_mode, tau,
                          _ptr(n_pruned, C.c_int64)), "prune")
    return n_pruned


def normalize(model: Model):
    m = model.cstruct()
    _check(lib().or_normalize(C.byref(m)), "normalize")


def sparsity(model: Model) -> float:
    m = model.cstruct()
    return lib().or_sparsity(C.byref(m))


def elbow_stat(re_t, re_t1, re_t2, pr_t) -> float:
    return lib().or_elbow_stat(re_t, re_t1, re_t2, pr_t)


@dataclass
class Params:
    reg: int = REG_LF
    lam: float = 0.01
    init_pr: float = 0.01
    max_pr: float = 0.1
    elbow_thresh: float = 0.05
    target_sparsity: float = -1.0
    conv_tol: float = 1e-6
    max_iter: int = 50
    fixed_pr_mode: int = 0
    fixed_pr: float = 0.0
    count_mode: int = 1
    normalize: int = 1
    revive_on_stop: int = 0
    resume: int = 0
    elbow_rise: int = 0

    def cstruct(self):
        p = _Params()
        p.reg, p.lambda_, p.init_pr, p.max_pr = self.reg, self.lam, self.init_pr, self.max_pr
        p.elbow_thresh, p.target_sparsity, p.conv_tol = self.elbow_thresh, self.target_sparsity, self.conv_tol
        p.max_iter, p.fixed_pr_mode, p.fixed_pr = self.max_iter, self.fixed_pr_mode, self.fixed_pr
        p.count_mode, p.normalize, p.revive_on_stop = self.count_mode, self.normalize, self.revive_on_stop
        p.resume, p.elbow_rise = self.resume, self.elbow_rise
        return p


def autosearch(prob: Problem, model: Model, params: Params, resume_from: dict | None = None) -> dict:
    """Algorithm 2 on `model` in place.  With params.resume, `resume_from` is the report of the
    run being continued (as returned by an earlier call)."""
    t, m, p = prob.cstruct(), model.cstruct(), params.cstruct()
    rep = _Report()
    if resume_from is not None:
        k = int(resume_from["iters"])
        rep.iters, rep.stop_iter = k, int(resume_from["stop_iter"])
        for name, key in (("re_hist", "re"), ("obj_hist", "obj"), ("pr_hist", "pr"), ("sparsity_hist", "sparsity")):
            getattr(rep, name)[:k] = [float(v) for v in resume_from[key][:k]]
    _check(lib().or_autosearch(C.byref(t), C.byref(m), C.byref(p), C.byref(rep)), "autosearch")
    it = rep.iters
    return {"iters": it, "stop_iter": rep.stop_iter, "re": np.array(rep.re_hist[:it]),
            "obj": np.array(rep.obj_hist[:it]), "pr": np.array(rep.pr_hist[:it]),
            "sparsity": np.array(rep.sparsity_hist[:it]), "final_sparsity": rep.final_sparsity}
