"""The identity the GPU core sweep rests on (Section 3.5 keeps the core update sequential).

Updating a run of consecutive core elements as a block -- g_k = sum_alpha r_alpha P_alpha(k)
and the block Gram M = sum_alpha P_alpha P_alpha^T taken once before the block, then for each
k in order sum_alpha r'_alpha P_alpha(k) = g_k - sum_{l<k} Delta_l M_lk -- gives, in exact
arithmetic, the element-at-a-time sweep of Eq. 12 / Eq. 14.  This checks it on the CPU in FP64
against the oracle's sequential sweep, for the block shape the kernels use (J_1 x m elements at
one suffix of the higher modes) and for blocks that span several suffixes (the shape that would
take fewer passes when the leading ranks are small).  The block arithmetic is written here in
numpy from the update rules; it shares nothing with the CUDA code or the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1904_02603_gb300 import datagen


def _soft(g, d, lam):
    """Minimiser of (d/2) a^2 + g a + lam |a| (the L_1 rules, Eq. 13 / Eq. 14 as read)."""
    if g > lam:
        return (lam - g) / d
    if g < -lam:
        return -(lam + g) / d
    return 0.0


def _blocked_core_sweep(idx, x, A, G, Gmask, reg, lam, blocks):
    N = len(A)
    ranks = [a.shape[1] for a in A]
    G = G.copy()
    # P[alpha, beta] = prod_n A^(n)[i_n, beta_n]; each new mode's digit goes outermost, so the
    # column index is beta's linear index with j_1 fastest
    P = np.ones((x.size, 1))
    for n in range(N):
        P = (A[n][idx[n]][:, :, None] * P[:, None, :]).reshape(x.size, -1)
    assert P.shape[1] == int(np.prod(ranks))
    r = x - P @ G
    for blk in blocks:
        Pb = P[:, blk]
        g = Pb.T @ r
        M = Pb.T @ Pb
        delta = np.zeros(len(blk))
        for k, beta in enumerate(blk):
            if Gmask[beta]:
                continue
            s = g[k] - delta[:k] @ M[:k, k]  # sum_alpha r_alpha P_alpha(beta), r as updated so far
            num = s + G[beta] * M[k, k]
            new = num / (lam + M[k, k]) if reg == O.REG_LF else _soft(-2.0 * num, 2.0 * M[k, k], lam)
            delta[k] = new - G[beta]
            G[beta] = new
        r -= Pb @ delta
    return G


def _blocks_at_one_suffix(ranks, m):
    """J_1 x m consecutive elements at a fixed suffix (j_3, ..., j_N), as the kernels block."""
    J1, J2 = ranks[0], ranks[1]
    S = int(np.prod(ranks[2:]))
    out = []
    for s in range(S):
        for q0 in range(0, J2, m):
            q1 = min(J2, q0 + m)
            out.append([j1 + J1 * (q + J2 * s) for q in range(q0, q1) for j1 in range(J1)])
    return out


def _blocks_of(size, total):
    return [list(range(b, min(total, b + size))) for b in range(0, total, size)]


@pytest.mark.parametrize("reg", [O.REG_LF, O.REG_L1])
@pytest.mark.parametrize("dims,ranks", [((9, 8, 7), (3, 4, 2)), ((6, 5, 4, 5), (2, 3, 2, 3))])
def test_blocked_core_sweep_equals_the_sequential_sweep(reg, dims, ranks):
    lam = 0.05 if reg == O.REG_LF else 0.5
    t, st = datagen.random_problem(77, dims, ranks, 200)
    rng = np.random.default_rng(78)
    Gmask = (rng.random(st.core.size) < 0.15).astype(np.uint8)
    G0 = np.where(Gmask, 0.0, st.core)
    model = O.Model([f.copy() for f in st.factors], G0.copy(), None, Gmask.copy())
    O.sweep_core(O.Problem(t.dims, t.idx, t.val), model, reg, lam)
    total = G0.size
    partitions = {
        "one suffix, m = 2": _blocks_at_one_suffix(ranks, 2),
        "one suffix, whole j_2 range": _blocks_at_one_suffix(ranks, ranks[1]),
        "blocks of 7 across suffixes": _blocks_of(7, total),
        "one block": _blocks_of(total, total),
        "single elements": _blocks_of(1, total),
    }
    for name, blocks in partitions.items():
        assert sorted(sum(blocks, [])) == list(range(total)), name
        got = _blocked_core_sweep(t.idx, t.val, st.factors, G0, Gmask, reg, lam, blocks)
        scale = max(np.abs(model.G).max(), 1e-300)
        assert np.abs(got - model.G).max() / scale < 1e-11, name
