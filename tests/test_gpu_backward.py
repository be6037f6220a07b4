"""GPU parity of pc_backward (dL/du_k, dL/dv_k from dL/dTheta) against the oracle's adjoint,
and against FP64 central finite differences on the differentiation workload."""
import numpy as np
import pytest

import oracle
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
    for got, ref in ((du, du_ref), (dv, dv_ref)):
        got = got.double().cpu().numpy()
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (np.linalg.norm(got - ref) / np.linalg.norm(ref))


def test_c3_gradient_finite_differences(pw):
    """Differentiation workload: 2-D 128^2, db4, L=3, m=9, 11x11 learnable kernels.  Loss
    ||Theta_P(u, v) - Theta_P(u_target, v)||^2.  The FP32 gradient from pc_backward matches FP64
    central differences (step 1e-6) on 64 seeded parameters (mixed u and v) to 1e-4."""
    import torch
    op = P.workload("c3")
    tgt = P.workload("c3")
    tgt.u = op.extra["u_target"]
    g64 = make_gpu_op(pw, op, precision=1)
    t64 = make_gpu_op(pw, tgt, precision=1)
    t64.assemble()
    T64 = t64.values().clone()
    u64 = torch.tensor(op.u, dtype=torch.float64, device="cuda")
    v64 = torch.tensor(op.v, dtype=torch.float64, device="cuda")

    def loss(u, v):
        pw.pc_set_params(g64.h, u, v)
        g64.assemble()
        return float(((g64.values() - T64) ** 2).sum())

    # FP32 gradient
    g32 = make_gpu_op(pw, op, precision=0)
    t32 = make_gpu_op(pw, tgt, precision=0)
    t32.assemble()
    g32.assemble()
    G = 2.0 * (g32.values() - t32.values())
    du, dv = g32.backward(G.contiguous())
    g32.sync()
    du = du.double().cpu().numpy()
    dv = dv.double().cpu().numpy()
    rng = np.random.default_rng(P.BASE_SEED + 3)
    h = 1e-6
    worst = 0.0
    scale = max(np.abs(du).max(), np.abs(dv).max())
    for i in range(64):
        k = int(rng.integers(op.m))
        if i % 2 == 0:
            t = int(rng.integers(op.u.shape[1]))
            up, um = u64.clone(), u64.clone()
            up[k, t] += h
            um[k, t] -= h
            fd = (loss(up, v64) - loss(um, v64)) / (2 * h)
            got = du[k, t]
        else:
            # a pixel where the window is nonzero half of the time, anywhere otherwise
            x = int(rng.integers(op.N))
            vp, vm = v64.clone(), v64.clone()
            vp[k, x] += h
            vm[k, x] -= h
            fd = (loss(u64, vp) - loss(u64, vm)) / (2 * h)
            got = dv[k, x]
        err = abs(got - fd) / max(abs(fd), 1e-3 * scale)
        worst = max(worst, err)
    assert worst <= 1e-4, worst


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
