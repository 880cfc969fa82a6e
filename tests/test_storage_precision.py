"""Precision studies behind two design choices, run on the CPU.

1. Whether the factors can be stored in BF16 (a variant considered for the 4-order workload):
one iteration of Algorithm 2's sweeps on the oracle, with the factor matrices rounded to the
storage format after the factor sweep, against the same iteration kept in FP64.

FP32 storage stays within 1e-6 of the FP64 objective; BF16 storage misses the 1e-4 relative
objective tolerance of the FP32 path by more than ten times already after one iteration (and
the gap grows over later iterations), so the library keeps FP32 factors.

2. Whether the delta contraction (Eq. 11) could move to the tensor cores in TF32: as one
(entries x |G|/J_n) by (|G|/J_n x J_n) product with Khatri-Rao rows, one TF32 product errs by
about 1e-4 relative while three (hi*hi + hi*lo + lo*hi, FP32 accumulation) match FP32 FMAs."""
import numpy as np

import oracle as O
from paper_1904_02603_gb300 import datagen


def _round_bf16(a):
    """Round to the nearest BF16 value, ties to even: the upper 16 bits of the FP32 pattern."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _round_tf32(a):
    """Round to the nearest TF32 value (10 explicit mantissa bits), ties to even, as FP32."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0xFFF + ((u >> 13) & 1)) >> 13) << 13
    return r.astype(np.uint32).view(np.float32)


def _round_fp32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def test_bf16_rounding_helper():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0, 1e-3])
    got = _round_bf16(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa wins (1); 1 + 3*2^-9 rounds up
    np.testing.assert_array_equal(got[:5], [1.0, 1.0, 1.0 + 2 ** -7, -2.5, 0.0])
    assert abs(got[5] - 1e-3) <= 2 ** -9 * 1e-3


def test_bf16_factor_storage_misses_the_objective_tolerance():
    w = datagen.WORKLOADS["uniform_300x4_2e4"]
    t, st, _ = datagen.make(w)
    prob = O.Problem(t.dims, t.idx, t.val.astype(np.float64))
    reg = O.REG_L1 if w.reg == "L1" else O.REG_LF

    def one_iteration(store):
        m = O.Model([store(f.astype(np.float64)) for f in st.factors], st.core.astype(np.float64))
        O.sweep_factors(prob, m, reg, w.lam, -1)
        for n in range(len(m.A)):
            m.A[n][:] = store(m.A[n])
        O.sweep_core(prob, m, reg, w.lam)
        return O.loss(prob, m, reg, w.lam)[3]

    ref = one_iteration(lambda a: a)
    gap32 = abs(one_iteration(_round_fp32) - ref) / ref
    gap16 = abs(one_iteration(_round_bf16) - ref) / ref
    assert gap32 < 1e-6, gap32
    assert gap16 > 1e-3, gap16


def test_three_tf32_products_match_fp32_on_the_delta_contraction():
    rng = np.random.default_rng(0)
    E, Jf, Jo, Jn = 4096, 10, 10, 10  # the 3-order rank-10 workload: |G|/J_n = 100
    G = rng.random((Jo * Jf, Jn))  # permuted core of the U(0,1) start
    A = (rng.random((E, Jo))[:, :, None] * rng.random((E, Jf))[:, None, :]).reshape(E, Jo * Jf)
    ref = A @ G
    A32, G32 = A.astype(np.float32), G.astype(np.float32)
    err = lambda v: float((np.abs(v.astype(np.float64) - ref) / np.abs(ref)).max())
    fp32 = err(A32 @ G32)
    a_hi, g_hi = _round_tf32(A32), _round_tf32(G32)
    a_lo, g_lo = _round_tf32(A32 - a_hi), _round_tf32(G32 - g_hi)
    one = err(a_hi @ g_hi)
    three = err(a_hi @ g_hi + a_hi @ g_lo + a_lo @ g_hi)
    assert one > 1e-5 and three < 3 * fp32 and three < 2e-6, (fp32, one, three)
