"""Full-size runs of the large workload (2-D 1024^2, db4, L=5, m=64, 31x31 Gaussian * motion
kernels; 3,555,397,632 stored entries), each against the FP64 oracle: the assembly on seeded
columns of every band; the BF16 apply to 16 right-hand sides on sampled rows (the oracle's rows
of Theta come from the order-flag identity Theta_0(u)^T = Theta_1(flip u)); the backward for a
seeded dL/dTheta on sampled columns against the oracle's adjoint; and the BF16 apply against the
definition of the product on the stored matrix."""
import numpy as np
import pytest

import pc_inputs as P
from helpers import assert_elementwise, make_gpu_op, oracle_rows

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


def _band_columns(op, seed):
    """One seeded column per band (coarse bands are the expensive ones for the oracle)."""
    rng = np.random.default_rng(seed)
    n, L = op.n, op.levels
    starts = [(0, (n >> L) ** 2)] + [((n >> j) ** 2 * (1 + t), (n >> j) ** 2) for j in range(L, 0, -1) for t in range(3)]
    return np.array([off + int(rng.integers(0, size)) for off, size in starts], dtype=np.int64)


def test_large_apply_vs_oracle(large):
    """y = Theta x (16 right-hand sides, BF16 Theta, FP32 accumulation) on one seeded row of
    every band against the oracle's rows of Theta in FP64: max over right-hand sides of
    ||y - y_ref|| / ||y_ref|| <= 1e-2 per row."""
    import torch
    import oracle
    pw, op, g = large
    nrhs = 16
    x = P.normal(P.BASE_SEED + 56, op.N * nrhs).reshape(op.N, nrhs)
    y = g.apply(torch.tensor(x, dtype=torch.float32, device="cuda"))
    g.sync()
    rows = _band_columns(op, 22)
    R = oracle_rows(op, rows)
    worst = 0.0
    for i, mu in enumerate(rows):
        mask = oracle.pattern_column(op, int(mu))      # the pattern is symmetric
        ref = R[i][mask] @ x[mask]
        got = y[int(mu)].double().cpu().numpy()
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        worst = max(worst, rel)
    assert worst <= 1e-2, worst


def test_large_backward_vs_oracle(large):
    """dL/du, dL/dv for a seeded dL/dTheta (N(0,1) values on the pattern entries of one seeded
    column per band, zero elsewhere) against the oracle's adjoint on the same columns (FP64),
    element-wise within 1e-5 of the largest magnitude."""
    import torch
    import oracle
    pw, op, g = large
    cols = _band_columns(op, 23)
    G = np.zeros((cols.size, op.N))
    G_d = torch.zeros(g.nnz, dtype=torch.float32, device="cuda")
    for c, lam in enumerate(cols):
        mus = np.nonzero(oracle.pattern_column(op, int(lam)))[0].astype(np.int64)
        vals = P.normal(P.BASE_SEED + 600 + c, mus.size)
        G[c, mus] = vals
        pos = g.lookup(mus, np.full(mus.size, lam, dtype=np.int64))
        assert (pos >= 0).all()
        G_d[torch.tensor(pos, device="cuda")] = torch.tensor(vals, dtype=torch.float32, device="cuda")
    du, dv = g.backward(G_d)
    g.sync()
    du_ref, dv_ref = oracle.theta_grad(op, cols, G, nthreads=4)
    e1 = assert_elementwise(du.double().cpu().numpy(), du_ref, 1e-5, "dL/du")
    e2 = assert_elementwise(dv.double().cpu().numpy(), dv_ref, 1e-5, "dL/dv")
    print(f"c5 backward vs oracle: max err / max|g| du {e1:.2e} dv {e2:.2e}")


@pytest.mark.parametrize("name,kw", [("op2", {"n": 512}), ("c5", {"n": 512, "levels": 4})],
                         ids=["m25-512", "m64-512"])
def test_backward_many_terms_vs_oracle(name, kw):
    """Operators with many terms (25 Symmlet-6 terms and 64 terms on 512^2, several groups of
    terms in the dL/dv gather): seeded dL/dTheta on one column per band, dL/du and dL/dv against
    the oracle's adjoint element-wise within 1e-5 of the largest magnitude."""
    import torch
    import oracle
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as pw
    op = P.workload(name, **kw)
    g = make_gpu_op(pw, op)
    cols = _band_columns(op, 24)
    G = np.zeros((cols.size, op.N))
    G_d = torch.zeros(g.nnz, dtype=torch.float32, device="cuda")
    for c, lam in enumerate(cols):
        mus = np.nonzero(oracle.pattern_column(op, int(lam)))[0].astype(np.int64)
        vals = P.normal(P.BASE_SEED + 650 + c, mus.size)
        G[c, mus] = vals
        pos = g.lookup(mus, np.full(mus.size, lam, dtype=np.int64))
        assert (pos >= 0).all()
        G_d[torch.tensor(pos, device="cuda")] = torch.tensor(vals, dtype=torch.float32, device="cuda")
    du, dv = g.backward(G_d)
    g.sync()
    du_ref, dv_ref = oracle.theta_grad(op, cols, G, nthreads=8)
    assert_elementwise(du.double().cpu().numpy(), du_ref, 1e-5, "dL/du")
    assert_elementwise(dv.double().cpu().numpy(), dv_ref, 1e-5, "dL/dv")
    g.close()
