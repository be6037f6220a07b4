"""GPU parity of pc_backward (dL/du_k, dL/dv_k from dL/dTheta) against the oracle's adjoint,
element-wise, and against the oracle's FP64 central finite differences on the differentiation
workload."""
import numpy as np
import pytest

import oracle
import pc_inputs as P
from helpers import assert_elementwise, make_gpu_op, sample_columns, storage_map

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as m
    return m


def _random_G(op, g, seed):
    """dL/dTheta: seeded values on the pattern, as a dense (N, N) array and in storage order."""
    N = op.N
    G = np.zeros((N, N))
    store = np.zeros(g.nnz)
    mus = np.arange(N, dtype=np.int64)
    vals = P.normal(seed, N * N).reshape(N, N)
    for lam in range(N):
        mask = oracle.pattern_column(op, lam)
        pos = g.lookup(mus, np.full(N, lam, dtype=np.int64))
        G[mask, lam] = vals[mask, lam]
        store[pos[mask]] = vals[mask, lam]
    return G, store


@pytest.mark.parametrize("name,kw", [("small-1d", {}), ("small-1d", {"order": 1}),
                                     ("small-1d", {"n": 64, "levels": 5, "r": 7}),
                                     ("small-2d", {"n": 32, "levels": 3}), ("small-2d", {"n": 32, "levels": 3, "order": 1}),
                                     ("small-2d", {"n": 32, "levels": 4, "r": 4}), ("small-2d", {"n": 64, "levels": 4, "gap": 1}),
                                     ("small-2d", {"n": 32, "levels": 3, "delta": 3}),
                                     ("small-2d", {"n": 32, "levels": 3, "delta": 1}),
                                     ("small-2d", {"n": 32, "levels": 3, "delta": 4, "family": 1}),   # Symmlet 4
                                     ("c1", {})])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp32", "fp64"])
def test_backward_matches_oracle(pw, name, kw, precision):
    import torch
    op = P.workload(name, **kw)
    g = make_gpu_op(pw, op, precision=precision)
    G, store = _random_G(op, g, P.BASE_SEED + 77)
    dt = torch.float64 if precision else torch.float32
    du, dv = g.backward(torch.tensor(store, dtype=dt, device="cuda"))
    g.sync()
    cols = np.arange(op.N)
    du_ref, dv_ref = oracle.theta_grad(op, cols, G.T.copy())
    tol = 1e-5 if precision == 0 else 1e-11
    assert_elementwise(du.double().cpu().numpy(), du_ref, tol, "dL/du")
    assert_elementwise(dv.double().cpu().numpy(), dv_ref, tol, "dL/dv")


def _c3_pair():
    op = P.workload("c3")
    tgt = P.workload("c3")
    tgt.u = op.extra["u_target"]
    return op, tgt


def test_c3_gradient_matches_oracle(pw):
    """Differentiation workload (2-D 128^2, db4, L = 3, m = 9, 11x11 learnable kernels), loss
    ||Theta_P(u, v) - Theta_P(u_target, v)||_F^2 over every column.  dL/dTheta = 2 (Theta -
    Theta_target) on the pattern is computed by the oracle (FP64, Algorithm 2) and given to both
    sides; pc_backward's FP32 dL/du and dL/dv equal the oracle's adjoint (FP64) element-wise
    within 1e-5 of the largest magnitude."""
    import torch
    import oracle
    op, tgt = _c3_pair()
    g = make_gpu_op(pw, op)
    rows, cols = storage_map(pw, g.desc, op.N)
    assert rows.size == g.nnz
    store = np.zeros(g.nnz)
    du_ref = np.zeros(op.u.shape)
    dv_ref = np.zeros(op.v.shape)
    chunk = 2048
    for c0 in range(0, op.N, chunk):
        cs = np.arange(c0, min(op.N, c0 + chunk), dtype=np.int64)
        Gc = 2.0 * (oracle.theta_columns(op, cs) - oracle.theta_columns(tgt, cs))
        for i, lam in enumerate(cs):
            Gc[i, ~oracle.pattern_column(op, lam)] = 0.0
        sel = (cols >= c0) & (cols < c0 + cs.size)
        store[sel] = Gc[cols[sel] - c0, rows[sel]]
        a, b = oracle.theta_grad(op, cs, Gc)
        du_ref += a
        dv_ref += b
    du, dv = g.backward(torch.tensor(store, dtype=torch.float32, device="cuda"))
    g.sync()
    e1 = assert_elementwise(du.double().cpu().numpy(), du_ref, 1e-5, "dL/du")
    e2 = assert_elementwise(dv.double().cpu().numpy(), dv_ref, 1e-5, "dL/dv")
    print(f"c3 gradient vs oracle: max err / max|g| du {e1:.2e} dv {e2:.2e}")
    g.close()


def test_c3_gradient_finite_differences(pw):
    """Differentiation workload, loss ||Theta_P(u, v) - Theta_P(u_target, v)||_F^2 over a seeded
    sample of columns stratified over the bands.  The GPU's FP32 forward and backward (dL/dTheta
    from its own FP32 Theta) against central differences (step 1e-6) of the same loss
    evaluated by the FP64 oracle, on 64 seeded parameters (32 kernel taps, 32 window pixels
    inside the supports of the sampled columns): per parameter within 1e-4, relative to
    max(|fd|, 1e-3 max|g|)."""
    import torch
    import oracle
    op, tgt = _c3_pair()
    cols = sample_columns(op, per_band=6, seed=9)
    masks = np.array([oracle.pattern_column(op, lam) for lam in cols])
    Tt = oracle.theta_columns(tgt, cols)

    def loss(u, v):
        T = oracle.theta_columns(op, cols, u=u, v=v)
        return float((((T - Tt) * masks) ** 2).sum())

    # FP32 gradient of the sampled loss: dL/dTheta = 2 (Theta - Theta_target) on the sampled
    # columns' pattern entries, zero elsewhere
    g32 = make_gpu_op(pw, op)
    t32 = make_gpu_op(pw, tgt)
    g32.assemble()
    t32.assemble()
    mus = np.arange(op.N, dtype=np.int64)
    pos = np.concatenate([g32.lookup(mus[m], np.full(int(m.sum()), lam, dtype=np.int64))
                          for lam, m in zip(cols, masks)])
    assert (pos >= 0).all()
    pos_d = torch.tensor(pos, device="cuda")
    G = torch.zeros(g32.nnz, dtype=torch.float32, device="cuda")
    G[pos_d] = 2.0 * (g32.values()[pos_d] - t32.values()[pos_d])
    du, dv = g32.backward(G)
    g32.sync()
    du = du.double().cpu().numpy()
    dv = dv.double().cpu().numpy()
    scale = max(np.abs(du).max(), np.abs(dv).max())
    rng = np.random.default_rng(P.BASE_SEED + 3)
    h = 1e-6
    u0, v0 = op.u.copy(), op.v.copy()
    worst = 0.0
    for i in range(64):
        k = int(rng.integers(op.m))
        if i % 2 == 0:
            t = int(rng.integers(op.u.shape[1]))
            up, um = u0.copy(), u0.copy()
            up[k, t] += h
            um[k, t] -= h
            fd = (loss(up, v0) - loss(um, v0)) / (2 * h)
            got = du[k, t]
        else:
            # a pixel of the support of a sampled column's wavelet
            lam = int(cols[int(rng.integers(cols.size))])
            e = np.zeros(op.N)
            e[lam] = 1.0
            supp = np.nonzero(oracle.idwt(op.d, op.n, op.levels, op.delta, e))[0]
            x = int(supp[int(rng.integers(supp.size))])
            vp, vm = v0.copy(), v0.copy()
            vp[k, x] += h
            vm[k, x] -= h
            fd = (loss(u0, vp) - loss(u0, vm)) / (2 * h)
            got = dv[k, x]
        err = abs(got - fd) / max(abs(fd), 1e-3 * scale)
        worst = max(worst, err)
    assert worst <= 1e-4, worst
    g32.close()
    t32.close()


def test_autograd_function(pw):
    import torch
    op = P.workload("small-2d", n=32, levels=3)
    g = make_gpu_op(pw, op)
    u = torch.tensor(op.u, dtype=torch.float32, device="cuda", requires_grad=True)
    v = torch.tensor(op.v, dtype=torch.float32, device="cuda", requires_grad=True)
    th = pw.theta(u, v, g)
    w = torch.linspace(-1, 1, th.numel(), device="cuda")
    (th * w).sum().backward()
    du, dv = g.backward(w.contiguous())
    # dv is accumulated with FP32 atomics, so two runs agree up to summation order
    for a, b in ((u.grad, du), (v.grad, dv)):
        assert (a - b).abs().max() <= 1e-5 * b.abs().max()
