"""Python binding of libvest (include/vest.h): argument marshalling only.

Every function named ``vest_*`` here calls the C entry point of the same name;
all compute runs in the library's CUDA kernels.  PyTorch provides device
memory and the current stream.  If libvest.so is missing or no CUDA device is
present, the binding raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

MAX_ORDER = 10
MAX_RANK = 32
F64, F32 = 0, 1
REG_LF, REG_L1 = 0, 1
STATUS = {0: "OK", 1: "INVALID", 2: "CUDA", 3: "NOMEM", 4: "WORKSPACE", 5: "TIMEOUT", 6: "UNSUPPORTED",
          7: "NUMERIC"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvest.so")


class VestError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} failed: VEST_ERR_{STATUS.get(status, status)}: {msg}")
        self.status = status


class vest_tensor(C.Structure):
    _fields_ = [("order", C.c_int32), ("val_dtype", C.c_int32), ("dims", C.c_int64 * MAX_ORDER),
                ("nnz", C.c_int64), ("idx", C.c_void_p), ("val", C.c_void_p)]


class vest_model(C.Structure):
    _fields_ = [("order", C.c_int32), ("dtype", C.c_int32), ("dims", C.c_int64 * MAX_ORDER),
                ("ranks", C.c_int32 * MAX_ORDER), ("factor", C.c_void_p * MAX_ORDER),
                ("factor_mask", C.c_void_p * MAX_ORDER), ("core", C.c_void_p), ("core_mask", C.c_void_p)]


class vest_mode_view(C.Structure):
    _fields_ = [("row_ptr", C.c_void_p), ("perm", C.c_void_p), ("oidx", C.c_void_p), ("val", C.c_void_p),
                ("nzptr", C.c_void_p), ("nzrow", C.c_void_p), ("nrows_nonempty", C.c_void_p)]


class vest_params(C.Structure):
    _fields_ = [("reg", C.c_int32), ("lambda_", C.c_double), ("init_pr", C.c_double), ("max_pr", C.c_double),
                ("elbow_thresh", C.c_double), ("target_sparsity", C.c_double), ("conv_tol", C.c_double),
                ("max_iter", C.c_int32), ("fixed_pr_mode", C.c_int32), ("fixed_pr", C.c_double),
                ("count_mode", C.c_int32), ("normalize", C.c_int32), ("revive_on_stop", C.c_int32),
                ("resume", C.c_int32), ("elbow_rise", C.c_int32)]


class vest_report(C.Structure):
    _fields_ = [("iters", C.c_int32), ("stop_iter", C.c_int32), ("re_hist", C.c_double * 256),
                ("obj_hist", C.c_double * 256), ("pr_hist", C.c_double * 256),
                ("sparsity_hist", C.c_double * 256), ("final_sparsity", C.c_double)]


# name -> (restype, argtypes); the ABI surface declared in include/vest.h
_P = C.c_void_p
_SIGS = {
    "vest_version": (C.c_char_p, []),
    "vest_last_error": (C.c_char_p, []),
    "vest_launch_count": (C.c_uint64, []),
    "vest_index_workspace_bytes": (C.c_size_t, [C.POINTER(vest_tensor)]),
    "vest_build_index": (C.c_int, [C.POINTER(vest_tensor), _P, C.c_size_t, C.POINTER(_P), _P]),
    "vest_index_destroy": (C.c_int, [_P]),
    "vest_index_mode": (C.c_int, [_P, C.c_int32, C.POINTER(vest_mode_view)]),
    "vest_scratch_bytes": (C.c_size_t, [_P, C.POINTER(vest_model)]),
    "vest_scratch_bytes_for": (C.c_size_t, [C.POINTER(vest_tensor), C.POINTER(vest_model)]),
    "vest_sweep_factors": (C.c_int, [_P, C.POINTER(vest_model), C.c_int32, C.c_double, C.c_int32, _P,
                                     C.c_size_t, _P]),
    "vest_sweep_factors_ex": (C.c_int, [_P, C.POINTER(vest_model), C.c_int32, C.c_double, C.c_int32, C.c_int32, _P,
                                        C.c_size_t, _P]),
    "vest_sweep_core": (C.c_int, [_P, C.POINTER(vest_model), C.c_int32, C.c_double, _P, C.c_size_t, _P]),
    "vest_loss": (C.c_int, [_P, C.POINTER(vest_model), C.c_int32, C.c_double, _P, _P, _P, C.c_size_t, _P]),
    "vest_responsibility": (C.c_int, [_P, C.POINTER(vest_model), _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "vest_iteration": (C.c_int, [_P, C.POINTER(vest_model), C.c_int32, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                 _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "vest_prune": (C.c_int, [C.POINTER(vest_model), _P, _P, C.c_double, C.c_int32, C.c_int32, C.c_double, _P, _P,
                             C.c_size_t, _P]),
    "vest_normalize": (C.c_int, [C.POINTER(vest_model), _P, C.c_size_t, _P]),
    "vest_count_zeros": (C.c_int, [C.POINTER(vest_model), _P, _P, C.c_size_t, _P]),
    "vest_value_keys": (C.c_int, [C.POINTER(vest_model), _P, _P, _P]),
    "vest_autosearch_scratch_bytes": (C.c_size_t, [_P, C.POINTER(vest_model)]),
    "vest_autosearch": (C.c_int, [_P, C.POINTER(vest_model), C.POINTER(vest_params), C.POINTER(vest_report), _P,
                                  C.c_size_t, _P]),
    "vest_reconstruct": (C.c_int, [C.POINTER(vest_model), _P, C.c_int64, _P, _P]),
    "vest_loss_noalloc": (C.c_int, [_P, C.POINTER(vest_model), C.c_int32, C.c_double, _P, _P, _P]),
    "vest_device_status": (C.c_int, [C.POINTER(C.c_uint32), C.c_int32]),
    "vest_probe_peak": (C.c_int, [C.c_int32, C.POINTER(C.c_double), _P, C.c_size_t, _P]),
}

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Loads libvest.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libvest.so not found at {path}; build it with paper_1904_02603_gb300.build.build()")
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("libvest needs a CUDA device; there is no CPU fallback")


def _call(name, *args):
    rc = getattr(load(), name)(*args)
    if rc != 0:
        raise VestError(name, rc, load().vest_last_error().decode())
    return rc


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dtype_code(dt):
    if dt == torch.float64:
        return F64
    if dt == torch.float32:
        return F32
    raise ValueError(f"unsupported dtype {dt}")


# ------------------------------------------------------------------ device-resident objects
class Tensor:
    """Observed entries on the device: idx (N, nnz) int32, val (nnz,) float32/float64."""

    def __init__(self, dims, idx: torch.Tensor, val: torch.Tensor):
        self.dims = tuple(int(d) for d in dims)
        self.idx = idx.to(torch.int32).contiguous()
        self.val = val.contiguous()
        assert self.idx.shape == (len(self.dims), self.val.shape[0])

    @classmethod
    def from_host(cls, st, device="cuda"):
        return cls(st.dims, torch.from_numpy(np.ascontiguousarray(st.idx)).to(device),
                   torch.from_numpy(np.ascontiguousarray(st.val)).to(device))

    @property
    def order(self):
        return len(self.dims)

    @property
    def nnz(self):
        return int(self.val.shape[0])

    def cstruct(self):
        t = vest_tensor()
        t.order = self.order
        t.val_dtype = _dtype_code(self.val.dtype)
        for n, d in enumerate(self.dims):
            t.dims[n] = d
        t.nnz = self.nnz
        t.idx = self.idx.data_ptr() if self.nnz else None
        t.val = self.val.data_ptr() if self.nnz else None
        return t


class Model:
    """Factors (I_n, J_n), masks (uint8, 1 = pruned), flat core (j_1 fastest) and core mask on the device."""

    def __init__(self, factors, core, factor_masks=None, core_mask=None):
        self.factors = [f.contiguous() for f in factors]
        self.core = core.reshape(-1).contiguous()
        dev = self.core.device
        self.factor_masks = [m.to(torch.uint8).contiguous() for m in factor_masks] if factor_masks is not None \
            else [torch.zeros(f.shape, dtype=torch.uint8, device=dev) for f in self.factors]
        self.core_mask = core_mask.reshape(-1).to(torch.uint8).contiguous() if core_mask is not None \
            else torch.zeros(self.core.shape, dtype=torch.uint8, device=dev)

    @classmethod
    def from_host(cls, state, device="cuda", dtype=None):
        cv = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device) if dtype is None
              else torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dtype))
        return cls([cv(f) for f in state.factors], cv(state.core),
                   [torch.from_numpy(np.ascontiguousarray(m)).to(device) for m in state.factor_masks],
                   torch.from_numpy(np.ascontiguousarray(state.core_mask)).to(device))

    @property
    def order(self):
        return len(self.factors)

    @property
    def ranks(self):
        return tuple(int(f.shape[1]) for f in self.factors)

    @property
    def dims(self):
        return tuple(int(f.shape[0]) for f in self.factors)

    def clone(self):
        return Model([f.clone() for f in self.factors], self.core.clone(), [m.clone() for m in self.factor_masks],
                     self.core_mask.clone())

    def to_host(self):
        return ([f.cpu().numpy() for f in self.factors], self.core.cpu().numpy(),
                [m.cpu().numpy() for m in self.factor_masks], self.core_mask.cpu().numpy())

    def cstruct(self):
        m = vest_model()
        m.order = self.order
        m.dtype = _dtype_code(self.core.dtype)
        for n, f in enumerate(self.factors):
            m.dims[n] = f.shape[0]
            m.ranks[n] = f.shape[1]
            m.factor[n] = f.data_ptr()
            m.factor_mask[n] = self.factor_masks[n].data_ptr()
        m.core = self.core.data_ptr()
        m.core_mask = self.core_mask.data_ptr()
        return m


class Index:
    """Mode-n index built by vest_build_index; keeps its device workspace alive."""

    def __init__(self, handle, ws, tensor: Tensor):
        self.handle = handle
        self.ws = ws
        self.dims = tensor.dims
        self.nnz = tensor.nnz
        self.dtype = tensor.val.dtype

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.vest_index_destroy(self.handle)
            self.handle = None

    def mode_view(self, mode: int) -> dict:
        """Host copies of the mode's CSR arrays (they live inside this index's workspace tensor)."""
        v = vest_mode_view()
        _call("vest_index_mode", self.handle, mode, C.byref(v))
        N, nnz, I = len(self.dims), self.nnz, self.dims[mode]
        torch.cuda.synchronize()
        R = int(self._slice(v.nrows_nonempty, 1, torch.int32)[0])
        return {
            "row_ptr": self._slice(v.row_ptr, I + 1, torch.int64),
            "perm": self._slice(v.perm, nnz, torch.int32),
            "oidx": self._slice(v.oidx, (N - 1) * nnz, torch.int32).reshape(N - 1, nnz),
            "val": self._slice(v.val, nnz, self.dtype),
            "nzptr": self._slice(v.nzptr, R + 1, torch.int64),
            "nzrow": self._slice(v.nzrow, R, torch.int32),
        }

    def _slice(self, ptr, count, dtype):
        esize = torch.empty(0, dtype=dtype).element_size()
        off = int(ptr) - self.ws.data_ptr()
        assert 0 <= off and off + count * esize <= self.ws.numel(), "view outside the index workspace"
        return self.ws[off:off + count * esize].view(dtype).cpu()


# ------------------------------------------------------------------ entry points (same names as vest.h)
def vest_version() -> str:
    return load().vest_version().decode()


def vest_device_status(clear: bool = True) -> int:
    """Synchronises the device and returns the status bits its kernels raised since the last
    clear (0: none; bit 0: a bounded tensor-core wait of the factor sweep gave up)."""
    f = C.c_uint32(0)
    getattr(load(), "vest_device_status")(C.byref(f), int(clear))
    return int(f.value)


PROBE_FP32_FMA, PROBE_FP64_FMA, PROBE_TF32_MMA, PROBE_L2_GATHER = 0, 1, 2, 3


def vest_probe_peak(kind: int, buffer: torch.Tensor | None = None, stream=None) -> float:
    """Measured peak rate of one unit (TFLOP/s for kinds 0-2, TB/s for the L2 gather, kind 3)."""
    r = C.c_double(0.0)
    _call("vest_probe_peak", int(kind), C.byref(r), _dptr(buffer), buffer.numel() * buffer.element_size()
          if buffer is not None else 0, _stream(stream))
    return float(r.value)


def vest_launch_count() -> int:
    return int(load().vest_launch_count())


def vest_index_workspace_bytes(t: Tensor) -> int:
    return int(load().vest_index_workspace_bytes(C.byref(t.cstruct())))


def vest_build_index(t: Tensor, stream=None) -> Index:
    _require_cuda()
    nbytes = vest_index_workspace_bytes(t)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
    h = C.c_void_p()
    _call("vest_build_index", C.byref(t.cstruct()), _dptr(ws), nbytes, C.byref(h), _stream(stream))
    return Index(h, ws, t)


def vest_scratch_bytes(ix: Index, m: Model) -> int:
    return int(load().vest_scratch_bytes(ix.handle, C.byref(m.cstruct())))


def vest_scratch_bytes_for(t: Tensor, m: Model) -> int:
    """vest_scratch_bytes for the index that vest_build_index(t) would make, without building it."""
    return int(load().vest_scratch_bytes_for(C.byref(t.cstruct()), C.byref(m.cstruct())))


def _shape_structs(dims, ranks, nnz: int, dtype):
    t, m = vest_tensor(), vest_model()
    t.order = m.order = len(dims)
    t.val_dtype = m.dtype = _dtype_code(dtype)
    t.nnz = int(nnz)
    for n, (d, r) in enumerate(zip(dims, ranks)):
        t.dims[n] = m.dims[n] = int(d)
        m.ranks[n] = int(r)
    return t, m


def device_bytes_for_shape(dims, ranks, nnz: int, dtype=torch.float32) -> dict:
    """Device memory a factorisation of this shape takes, from the library's own size queries,
    before anything is allocated: the tensor (indices and values), the index workspace, the
    scratch and the model (factors, core and their masks), in bytes."""
    t, m = _shape_structs(dims, ranks, nnz, dtype)
    es = torch.empty(0, dtype=dtype).element_size()
    G = 1
    for r in ranks:
        G *= int(r)
    model = sum(int(d) * int(r) * (es + 1) for d, r in zip(dims, ranks)) + G * (es + 1)
    return {"tensor": int(nnz) * (4 * len(dims) + es),
            "index": int(load().vest_index_workspace_bytes(C.byref(t))),
            "scratch": int(load().vest_scratch_bytes_for(C.byref(t), C.byref(m))),
            "model": model}


def vest_autosearch_scratch_bytes(ix: Index, m: Model) -> int:
    return int(load().vest_autosearch_scratch_bytes(ix.handle, C.byref(m.cstruct())))


def make_scratch(ix: Index, m: Model, autosearch: bool = False) -> torch.Tensor:
    n = vest_autosearch_scratch_bytes(ix, m) if autosearch else vest_scratch_bytes(ix, m)
    if n == 0:
        raise VestError("vest_scratch_bytes", 1, load().vest_last_error().decode())
    return torch.empty(n, dtype=torch.uint8, device="cuda")


DELTA_AUTO, DELTA_FMA, DELTA_TENSOR = 0, 1, 2


def vest_sweep_factors(ix: Index, m: Model, reg: int, lam: float, mode: int, scratch: torch.Tensor, stream=None,
                       path: int = DELTA_AUTO):
    if path == DELTA_AUTO:
        _call("vest_sweep_factors", ix.handle, C.byref(m.cstruct()), reg, lam, mode, _dptr(scratch), scratch.numel(),
              _stream(stream))
    else:
        _call("vest_sweep_factors_ex", ix.handle, C.byref(m.cstruct()), reg, lam, mode, path, _dptr(scratch),
              scratch.numel(), _stream(stream))


def vest_sweep_core(ix: Index, m: Model, reg: int, lam: float, scratch: torch.Tensor, stream=None):
    _call("vest_sweep_core", ix.handle, C.byref(m.cstruct()), reg, lam, _dptr(scratch), scratch.numel(),
          _stream(stream))


def vest_loss(ix: Index, m: Model, reg: int, lam: float, scratch: torch.Tensor, out=None, resid=None, stream=None):
    """Returns the device double[5] {sum r^2, sum X^2, reg term, objective, RE}."""
    if out is None:
        out = torch.empty(5, dtype=torch.float64, device="cuda")
    _call("vest_loss", ix.handle, C.byref(m.cstruct()), reg, lam, _dptr(out), _dptr(resid), _dptr(scratch),
          scratch.numel(), _stream(stream))
    return out


def vest_loss_noalloc(ix: Index, m: Model, reg: int, lam: float, out=None, resid=None, stream=None):
    """vest_loss without a scratch buffer: the library's fixed 1 MiB device array is used instead."""
    if out is None:
        out = torch.empty(5, dtype=torch.float64, device="cuda")
    _call("vest_loss_noalloc", ix.handle, C.byref(m.cstruct()), reg, lam, _dptr(out), _dptr(resid), _stream(stream))
    return out


def _ptr_array(ts):
    arr = (C.c_void_p * MAX_ORDER)()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr()
    return arr


def vest_responsibility(ix: Index, m: Model, scratch: torch.Tensor, with_resp: bool = True, stream=None):
    """Returns (delta_factor list, delta_core, resp_factor list or None, resp_core or None), device float64."""
    df = [torch.empty(f.shape, dtype=torch.float64, device="cuda") for f in m.factors]
    dc = torch.empty(m.core.shape, dtype=torch.float64, device="cuda")
    rf = [torch.empty(f.shape, dtype=torch.float64, device="cuda") for f in m.factors] if with_resp else None
    rc = torch.empty(m.core.shape, dtype=torch.float64, device="cuda") if with_resp else None
    dfa, rfa = _ptr_array(df), (_ptr_array(rf) if with_resp else None)
    _call("vest_responsibility", ix.handle, C.byref(m.cstruct()), C.cast(dfa, C.c_void_p), _dptr(dc),
          C.cast(rfa, C.c_void_p) if rfa is not None else None, _dptr(rc), _dptr(scratch), scratch.numel(),
          _stream(stream))
    return df, dc, rf, rc


def vest_value_keys(m: Model, stream=None):
    """Returns (|A^(n)| per mode, |G|) as device float64: the Value Pruning keys for vest_prune."""
    kf = [torch.empty(f.shape, dtype=torch.float64, device="cuda") for f in m.factors]
    kc = torch.empty(m.core.shape, dtype=torch.float64, device="cuda")
    kfa = _ptr_array(kf)
    _call("vest_value_keys", C.byref(m.cstruct()), C.cast(kfa, C.c_void_p), _dptr(kc), _stream(stream))
    return kf, kc


def vest_prune(m: Model, delta_factor, delta_core, pr: float, scratch: torch.Tensor, count_mode: int = 0,
               threshold_mode: int = 0, tau: float = 0.0, stream=None) -> torch.Tensor:
    """Returns the device int64[order+1] pruned counts."""
    n_pruned = torch.zeros(m.order + 1, dtype=torch.int64, device="cuda")
    dfa = _ptr_array([d.contiguous() for d in delta_factor])
    _call("vest_prune", C.byref(m.cstruct()), C.cast(dfa, C.c_void_p), _dptr(delta_core.contiguous()), pr,
          count_mode, threshold_mode, tau, _dptr(n_pruned), _dptr(scratch), scratch.numel(), _stream(stream))
    return n_pruned


def vest_iteration(ix: Index, m: Model, reg: int, lam: float, pr: float, scratch: torch.Tensor, count_mode: int = 0,
                   with_responsibility: bool = True, factor_sweep: bool = True, stream=None):
    """One iteration of Algorithm 2 in one call.

    Returns (loss, delta_factor list or None, delta_core or None, n_pruned or None): loss is the
    device double[5] of vest_loss for the swept model (before the prune)."""
    loss = torch.empty(5, dtype=torch.float64, device="cuda")
    df = dc = n_pruned = None
    dfa = None
    if with_responsibility:
        df = [torch.empty(f.shape, dtype=torch.float64, device="cuda") for f in m.factors]
        dc = torch.empty(m.core.shape, dtype=torch.float64, device="cuda")
        n_pruned = torch.zeros(m.order + 1, dtype=torch.int64, device="cuda")
        dfa = _ptr_array(df)
    _call("vest_iteration", ix.handle, C.byref(m.cstruct()), reg, lam, pr, count_mode, int(factor_sweep),
          _dptr(loss), C.cast(dfa, C.c_void_p) if dfa is not None else None, _dptr(dc), _dptr(n_pruned),
          _dptr(scratch), scratch.numel(), _stream(stream))
    return loss, df, dc, n_pruned


def vest_normalize(m: Model, scratch: torch.Tensor, stream=None):
    _call("vest_normalize", C.byref(m.cstruct()), _dptr(scratch), scratch.numel(), _stream(stream))


def vest_count_zeros(m: Model, scratch: torch.Tensor, stream=None) -> torch.Tensor:
    out = torch.zeros(m.order + 1, dtype=torch.int64, device="cuda")
    _call("vest_count_zeros", C.byref(m.cstruct()), _dptr(out), _dptr(scratch), scratch.numel(), _stream(stream))
    return out


def vest_reconstruct(m: Model, q_idx: torch.Tensor, stream=None) -> torch.Tensor:
    q = q_idx.to(torch.int32).contiguous()
    count = int(q.shape[1])
    out = torch.empty(count, dtype=m.core.dtype, device="cuda")
    _call("vest_reconstruct", C.byref(m.cstruct()), _dptr(q) if count else None, count,
          _dptr(out) if count else None, _stream(stream))
    return out


def params(reg=REG_LF, lam=0.01, init_pr=0.01, max_pr=0.1, elbow_thresh=0.05, target_sparsity=-1.0,
           conv_tol=1e-6, max_iter=50, fixed_pr_mode=0, fixed_pr=0.0, count_mode=1, normalize=1,
           revive_on_stop=0, resume=0, elbow_rise=0) -> vest_params:
    p = vest_params()
    p.reg, p.lambda_, p.init_pr, p.max_pr = reg, lam, init_pr, max_pr
    p.elbow_thresh, p.target_sparsity, p.conv_tol, p.max_iter = elbow_thresh, target_sparsity, conv_tol, max_iter
    p.fixed_pr_mode, p.fixed_pr, p.count_mode, p.normalize = fixed_pr_mode, fixed_pr, count_mode, normalize
    p.revive_on_stop, p.resume, p.elbow_rise = revive_on_stop, resume, elbow_rise
    return p


def vest_autosearch(ix: Index, m: Model, p: vest_params, scratch: torch.Tensor, stream=None,
                    resume_from: dict | None = None) -> dict:
    """Algorithm 2 on `m` in place; with p.resume, `resume_from` is the report being continued."""
    rep = vest_report()
    if resume_from is not None:
        k = int(resume_from["iters"])
        rep.iters, rep.stop_iter = k, int(resume_from["stop_iter"])
        for name, key in (("re_hist", "re"), ("obj_hist", "obj"), ("pr_hist", "pr"), ("sparsity_hist", "sparsity")):
            getattr(rep, name)[:k] = [float(v) for v in resume_from[key][:k]]
    _call("vest_autosearch", ix.handle, C.byref(m.cstruct()), C.byref(p), C.byref(rep), _dptr(scratch),
          scratch.numel(), _stream(stream))
    it = rep.iters
    return {"iters": it, "stop_iter": rep.stop_iter, "re": np.array(rep.re_hist[:it]),
            "obj": np.array(rep.obj_hist[:it]), "pr": np.array(rep.pr_hist[:it]),
            "sparsity": np.array(rep.sparsity_hist[:it]), "final_sparsity": rep.final_sparsity}


def exported_symbols():
    """The ABI names this binding wraps (must match include/vest.h)."""
    return sorted(_SIGS)
