"""Full-size runs of the large workload (2-D 1024^2, db4, L=5, m=64, 31x31 Gaussian * motion
kernels; 3,555,397,632 stored entries): assembly parity on seeded columns of every band against
the FP64 oracle, and the BF16 apply to 16 right-hand sides against the definition of the
product on the stored matrix (FP64 sums over each sampled row's stored entries)."""
import numpy as np
import pytest

import pc_inputs as P
from helpers import make_gpu_op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as pw
    op = P.workload("c5")
    g = make_gpu_op(pw, op, precision=0, bf16=1)
    assert g.nnz == 3555397632
    g.assemble()
    g.sync()
    yield pw, op, g
    g.close()


def test_large_assembly_columns(large):
    import oracle
    pw, op, g = large
    rng = np.random.default_rng(21)
    n, L = op.n, op.levels
    cols = []
    # one seeded column per band (coarse bands are the expensive ones for the oracle)
    starts = [(0, (n >> L) ** 2)] + [((n >> j) ** 2 * (1 + t), (n >> j) ** 2) for j in range(L, 0, -1) for t in range(3)]
    for off, size in starts:
        cols.append(off + int(rng.integers(0, size)))
    cols = np.array(cols, dtype=np.int64)
    T = oracle.theta_columns(op, cols)
    mus = np.arange(op.N, dtype=np.int64)
    import torch
    vals = g.values()
    err = ref = 0.0
    for c, lam in enumerate(cols):
        mask = oracle.pattern_column(op, lam)
        pos = g.lookup(mus, np.full(op.N, lam, dtype=np.int64))
        assert np.array_equal(pos >= 0, mask), lam
        got = vals[torch.tensor(pos[mask], device="cuda")].double().cpu().numpy()
        want = T[c][mask]
        err = max(err, float(np.abs(got - want).max()))
        ref = max(ref, float(np.abs(want).max()))
    assert err <= 1e-5 * ref, err / ref


def test_large_apply_16rhs(large):
    import torch
    pw, op, g = large
    nrhs = 16
    x = torch.tensor(P.normal(P.BASE_SEED + 55, op.N * nrhs), dtype=torch.float32, device="cuda").reshape(op.N, nrhs)
    y = g.apply(x)
    g.sync()
    vals = g.values()
    rptr = pw.pc_theta(g.h)[2]
    rng = np.random.default_rng(8)
    rows = [0, op.N - 1] + rng.integers(0, op.N, 40).tolist()
    desc = g.desc
    worst = 0.0
    for s in rows:
        cols = pw.pc_plan_row(desc, int(s))
        pos = g.lookup(np.full(cols.size, s, dtype=np.int64), cols)   # paper order: stored row = mu
        v = vals[torch.tensor(pos, device="cuda")].double()
        ref = (v[:, None] * x[torch.tensor(cols, device="cuda")].double()).sum(0)
        worst = max(worst, float(torch.linalg.norm(y[s].double() - ref) / torch.linalg.norm(ref)))
    assert worst <= 1e-2, worst
