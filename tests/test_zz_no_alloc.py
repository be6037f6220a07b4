"""pc_backward_noalloc: the allocation-free backward.

It serves callers that cannot call cudaMalloc: a framework that has reserved the whole device
for its own pool allocator, or a training loop that cannot afford the implicit device
synchronisation of an allocation.  Its scratch is one static device array that every call on a
device shares.  The tests below call it first on a freshly created handle (so no scratch of
pc_backward exists yet) and check that it allocates nothing (the handle's device bytes and
torch's allocated bytes are unchanged), then that its dL/du and dL/dv match the FP64 oracle's
adjoint element-wise and pc_backward's results, on two calls in a row with different dL/dTheta
(no state leaks from one call into the next), for FP32 and FP64 handles, 1-D and 2-D operators
and several filter templates.  An operator whose scratch exceeds the
array's size gets PC_ERR_UNSUPPORTED with the size it needs, and its outputs are left alone.
This file is collected last so that a failure here stops a `-x` run only after every other test.
"""
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


def _seeded_dtheta(op, g, seed):
    """Seeded N(0,1) dL/dTheta on the pattern: dense (N, N) for the oracle, storage order for
    the library."""
    import oracle
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


@pytest.mark.parametrize("name,kw", [("small-2d", {"n": 64, "levels": 3}),
                                     ("small-1d", {}),
                                     ("small-2d", {"n": 32, "levels": 3, "delta": 6, "family": 1}),   # Symmlet 6
                                     ("small-2d", {"n": 32, "levels": 3, "delta": 10})])              # 20 taps
@pytest.mark.parametrize("precision", [0, 1], ids=["fp32", "fp64"])
def test_backward_noalloc_matches_oracle_and_pc_backward(pw, name, kw, precision):
    import torch
    import oracle
    from helpers import assert_elementwise
    op = P.workload(name, **kw)
    dt = torch.float64 if precision else torch.float32
    tol = 1e-11 if precision else 1e-5
    u = torch.tensor(op.u, dtype=dt, device="cuda")
    v = torch.tensor(op.v, dtype=dt, device="cuda")
    g = pw.PCOperator(pw.desc_of(op, precision), u, v)       # fresh handle: no backward scratch yet
    K = (2 * op.r + 1) ** op.d
    for call in range(2):
        Gd, store = _seeded_dtheta(op, g, P.BASE_SEED + 500 + call)
        G = torch.tensor(store, dtype=dt, device="cuda")
        du = torch.full((op.m, K), float("nan"), dtype=dt, device="cuda")
        dv = torch.full((op.m, op.N), float("nan"), dtype=dt, device="cuda")
        torch.cuda.synchronize()
        before = (pw.pc_info(g.h)[1], torch.cuda.memory_allocated())
        pw.pc_backward_noalloc(g.h, G, du, dv)
        g.sync()
        after = (pw.pc_info(g.h)[1], torch.cuda.memory_allocated())
        assert before == after, (call, before, after)
        du_ref, dv_ref = oracle.theta_grad(op, np.arange(op.N), Gd.T.copy())
        assert_elementwise(du.double().cpu().numpy(), du_ref, tol, f"dL/du call {call}")
        assert_elementwise(dv.double().cpu().numpy(), dv_ref, tol, f"dL/dv call {call}")
        # the allocating entry point on the same input
        du_b, dv_b = g.backward(G)
        g.sync()
        assert_elementwise(du.double().cpu().numpy(), du_b.double().cpu().numpy(), tol, f"du vs pc_backward {call}")
        assert_elementwise(dv.double().cpu().numpy(), dv_b.double().cpu().numpy(), tol, f"dv vs pc_backward {call}")
    g.close()


def test_backward_noalloc_rejects_oversize(pw):
    """An operator with 64 terms of 31x31 kernels (the large workload's terms on a 256^2 grid)
    needs about 27 MB of scratch, more than the static array holds: PC_ERR_UNSUPPORTED, the
    required size in the message, du and dv untouched."""
    import torch
    op = P.workload("c5", n=256, levels=4)
    g = pw.PCOperator(pw.desc_of(op), torch.tensor(op.u, dtype=torch.float32, device="cuda"),
                      torch.tensor(op.v, dtype=torch.float32, device="cuda"))
    K = (2 * op.r + 1) ** 2
    G = torch.zeros(g.nnz, dtype=torch.float32, device="cuda")
    du = torch.full((op.m, K), 7.0, dtype=torch.float32, device="cuda")
    dv = torch.full((op.m, op.N), 7.0, dtype=torch.float32, device="cuda")
    with pytest.raises(pw.PCError) as ei:
        pw.pc_backward_noalloc(g.h, G, du, dv)
    assert ei.value.status == pw.PC_ERR_UNSUPPORTED
    msg = str(ei.value)
    assert "needs" in msg and str(8 << 20) in msg, msg
    torch.cuda.synchronize()
    assert bool((du == 7.0).all()) and bool((dv == 7.0).all())
    g.close()
