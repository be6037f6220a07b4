"""Degenerate operators on the GPU, checked against what the mathematics fixes rather than
against the oracle's numbers: point kernels with windows summing to one give H = I, so Theta
is the identity on the pattern; point kernels alone give the multiplier B = Psi^* V Psi, which
is symmetric; one kernel shared by every term gives a convolution, whose sub-bands are
circulant (Lemma 5.1).  The shapes are those of the parity cases (64^2, L = 3)."""
import numpy as np
import pytest

import pc_inputs as P
from helpers import make_gpu_op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as m
    return m


def _op(u, v, order=0, family=0, delta=4, r=0, n=64, L=3):
    return P.Operator("degenerate", 2, n, delta, L, r, u, v, gap=2, order=order, family=family)


def _entries(pw, g, op, mus, lams):
    pos = g.lookup(np.asarray(mus, dtype=np.int64), np.asarray(lams, dtype=np.int64))
    assert np.all(pos >= 0)
    import torch
    return g.values()[torch.tensor(pos, device="cuda")].double().cpu().numpy()


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("family,delta", [(0, 4), (1, 4), (0, 2)])
def test_partition_of_unity_with_point_kernels_is_identity(pw, order, family, delta):
    n = 64
    v = P.hat_windows(2, n, 3)                      # 9 windows summing to 1 at every pixel
    u = np.ones((9, 1))
    op = _op(u, v, order, family, delta)
    g = make_gpu_op(pw, op)
    g.assemble()
    g.sync()
    vals = g.values().double().cpu().numpy()
    # every stored row holds exactly one 1 (its diagonal) and zeros elsewhere
    pos = g.lookup(np.arange(op.N, dtype=np.int64), np.arange(op.N, dtype=np.int64))
    assert np.all(pos >= 0)
    assert np.abs(vals[pos] - 1.0).max() <= 1e-5      # the FP32 bar: 1e-5 of max |Theta| = 1
    vals[pos] = 0.0
    assert np.abs(vals).max() <= 1e-5
    g.close()


def test_multiplier_is_symmetric(pw):
    n = 64
    v = P.hat_windows(2, n, 3) * (0.5 + P.uniform(P.BASE_SEED + 600, 9)[:, None])
    op = _op(np.ones((9, 1)), v)
    g = make_gpu_op(pw, op)
    g.assemble()
    g.sync()
    rng = np.random.default_rng(9)
    rows = rng.integers(0, op.N, 60)
    mus, lams = [], []
    for s in rows:
        cols = pw.pc_plan_row(g.desc, int(s))
        pick = cols[rng.integers(0, cols.size, 20)]
        mus += [int(s)] * pick.size
        lams += pick.tolist()
    a = _entries(pw, g, op, mus, lams)
    b = _entries(pw, g, op, lams, mus)          # the pattern is symmetric
    scale = np.abs(a).max()
    assert np.abs(a - b).max() <= 1e-5 * scale
    g.close()


def test_convolution_subbands_are_circulant(pw):
    n, L = 64, 3
    v = P.hat_windows(2, n, 3)
    k = P.gaussian_kernel(2, 3, 1.2).reshape(-1)
    op = _op(np.stack([k] * 9), v, r=3)
    g = make_gpu_op(pw, op)
    g.assemble()
    g.sync()
    rng = np.random.default_rng(10)
    # a detail band of level 2 (translates 16 x 16) against the same band: shift both indices
    nj = n >> 2
    off = nj * nj * 1                               # level-2 band (0,1) starts after the approximation
    base_mu = off + rng.integers(0, nj, 30) * nj + rng.integers(0, nj, 30)
    worst = 0.0
    for mu in base_mu:
        cols = pw.pc_plan_row(g.desc, int(mu))
        lam = cols[(cols >= off) & (cols < off + nj * nj)]
        lam = lam[rng.integers(0, lam.size, 8)]
        t0, t1 = rng.integers(1, nj, 2)
        def shift(i):
            a, b = divmod(int(i) - off, nj)
            return off + ((a + t0) % nj) * nj + (b + t1) % nj
        x = _entries(pw, g, op, [int(mu)] * lam.size, lam)
        y = _entries(pw, g, op, [shift(mu)] * lam.size, [shift(l) for l in lam])
        worst = max(worst, float(np.abs(x - y).max()))
    assert worst <= 1e-5 * float(np.abs(g.values().double().cpu().numpy()).max())
    g.close()
