"""GPU construction of a product-convolution expansion by randomized SVD of the space-varying
impulse response (Section 2.4), pc_svir_expansion, against the FP64 oracle
(oracle/pc_svir.py) with the same test matrix: the rank-m reconstruction v^T u and the singular
values; exact recovery of a rank-m SVIR; and the expansion used as the kernels and windows of
an operator whose Theta matches the oracle's Theta of the same expansion."""
import numpy as np
import pytest

import pc_inputs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as m
    return m


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _omega(K, cols, seed):
    return P.normal(seed, K * cols).reshape(K, cols)


@pytest.mark.parametrize("name,kw", [("small-2d", {"n": 32, "levels": 2}), ("small-1d", {"n": 512})])
def test_rank_m_svir_is_recovered(pw, name, kw):
    from oracle import pc_svir as SV
    op = P.workload(name, **kw)
    S = SV.svir_of_pc(op.u, op.v)
    om = _omega(S.shape[1], op.m + 4, P.BASE_SEED + 710)
    u, v, s = pw.pc_svir_expansion(_dev(S), op.m, _dev(om))
    Sm = v.double().cpu().numpy().T @ u.double().cpu().numpy()
    assert np.abs(Sm - S).max() <= 1e-5 * np.abs(S).max()
    assert s[op.m] <= 1e-5 * s[0]                       # nothing beyond rank m


@pytest.mark.parametrize("n,m,l,q", [(32, 4, 12, 2), (128, 6, 16, 2), (128, 3, 8, 0)])
def test_matches_oracle_on_a_smooth_blur(pw, n, m, l, q):
    """sigma growing along axis 0 (the first blur of Section 4.1, in miniature): the GPU's rank-m
    reconstruction and leading singular values equal the oracle's (same test matrix, same power
    iterations) within the FP32 sketch's accuracy."""
    from oracle import pc_svir as SV
    r = 5
    S = SV.svir_space_varying_gaussian(2, n, r, lambda y0, y1: 0.6 + 2.0 * y0)
    om = _omega(S.shape[1], l, P.BASE_SEED + 720 + n + m)
    u_ref, v_ref, s_ref = SV.randomized_pc(S, m, om, power_iters=q)
    u, v, s = pw.pc_svir_expansion(_dev(S), m, _dev(om), power_iters=q)
    Sm = v.double().cpu().numpy().T @ u.double().cpu().numpy()
    Sm_ref = v_ref.T @ u_ref
    assert np.abs(Sm - Sm_ref).max() <= 1e-4 * np.abs(S).max()
    assert np.allclose(s[:m], s_ref[:m], rtol=1e-4)


def test_expansion_as_operator(pw):
    """The GPU expansion (u, v) of a smooth blur's SVIR as the kernels and windows of an
    operator (paper order): its assembled Theta equals the oracle's Theta of the same (u, v) on
    seeded columns of every band."""
    import torch
    from oracle import pc_svir as SV
    from helpers import compare_columns, sample_columns
    n, r, m = 64, 4, 5
    S = SV.svir_space_varying_gaussian(2, n, r, lambda y0, y1: 0.8 + 1.5 * y1)
    u, v, _ = pw.pc_svir_expansion(_dev(S), m, _dev(_omega(S.shape[1], m + 6, P.BASE_SEED + 730)))
    op = P.Operator("svir", 2, n, 4, 3, r, u.double().cpu().numpy(), v.double().cpu().numpy(), gap=2, order=0)
    g = pw.PCOperator(pw.desc_of(op), u.contiguous(), v.contiguous())
    g.assemble()
    err, ref = compare_columns(g, op, sample_columns(op, per_band=2, seed=3))
    assert err <= 1e-5 * ref, err / ref
    g.close()


def test_rejects_bad_sizes(pw):
    import torch
    S = torch.zeros((64, 9), dtype=torch.float32, device="cuda")
    om = torch.zeros((9, 12), dtype=torch.float32, device="cuda")
    with pytest.raises(pw.PCError):
        pw.pc_svir_expansion(S, 4, om)            # l = 12 > K = 9
    om2 = torch.zeros((9, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(pw.PCError):
        pw.pc_svir_expansion(S, 4, om2)           # l < m
