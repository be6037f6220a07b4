"""Pins of the oracle's PC construction by randomized SVD of the SVIR (Section 2.4): exact
recovery of a rank-m SVIR, the Eckart-Young lower bound and a near-optimal error on a smoothly
varying blur, the convention linking the SVIR to the operator (against the oracle's own H), and
the singular values against numpy's full SVD."""
import numpy as np

import oracle
import pc_inputs as P
from oracle import pc_svir as SV


def _omega(K, cols, seed):
    return P.normal(seed, K * cols).reshape(K, cols)


def test_rank_m_svir_is_recovered():
    op = P.workload("small-2d", n=16, levels=2)          # m = 9 terms, r = 3
    S = SV.svir_of_pc(op.u, op.v)
    u, v, s = SV.randomized_pc(S, op.m, _omega(S.shape[1], op.m + 5, P.BASE_SEED + 700))
    assert np.abs(v.T @ u - S).max() < 1e-12 * np.abs(S).max()
    assert s[op.m] < 1e-12 * s[0]                         # nothing beyond rank m


def test_svir_convention_matches_the_operator():
    op = P.workload("small-2d", n=16, levels=2)
    S = SV.svir_of_pc(op.u, op.v)
    f = P.normal(P.BASE_SEED + 701, op.N)
    assert np.abs(SV.apply_svir(S, f, 2, op.n, op.r) - oracle.pc_apply(op, f)).max() < 1e-12
    op1 = P.workload("small-1d", n=64)
    S1 = SV.svir_of_pc(op1.u, op1.v)
    f1 = P.normal(P.BASE_SEED + 702, op1.N)
    assert np.abs(SV.apply_svir(S1, f1, 1, op1.n, op1.r) - oracle.pc_apply(op1, f1)).max() < 1e-12


def test_near_optimal_on_a_smooth_blur():
    # sigma growing along axis 0 (the first blur of Section 4.1, in miniature)
    n, r = 24, 5
    S = SV.svir_space_varying_gaussian(2, n, r, lambda y0, y1: 0.6 + 2.0 * y0)
    sv = np.linalg.svd(S, compute_uv=False)
    for m in (2, 4, 6):
        u, v, s = SV.randomized_pc(S, m, _omega(S.shape[1], m + 8, P.BASE_SEED + 703 + m), power_iters=2)
        err = np.linalg.norm(S - v.T @ u)
        best = np.sqrt(np.sum(sv[m:] ** 2))               # Eckart-Young: the best rank-m error
        assert err >= best * (1 - 1e-9)
        assert err <= 1.05 * best + 1e-14
        assert np.allclose(s[:m], sv[:m], rtol=1e-6)
    # the expansion error decays with m
    errs = [np.linalg.norm(S - (lambda uv: uv[1].T @ uv[0])(SV.randomized_pc(S, m, _omega(S.shape[1], m + 8, 9)))) for m in (1, 2, 4, 8)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
