"""pc_backward_noalloc: the allocation-free backward, for callers that cannot call cudaMalloc
(a framework that reserved the device for its own pool, or a loop that cannot afford the
device synchronisation of an allocation).  Its scratch is a static device array shared by
all calls; this test checks, on two calls in a row with different dL/dTheta, that its
dL/du and dL/dv match pc_backward's within the backward tests' FP32 tolerance (1e-5
relative, norm-wise), so no state leaks from one call into the next."""
import numpy as np
import pytest

import pc_inputs as P

pytestmark = pytest.mark.gpu


def test_backward_noalloc_matches_pc_backward():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as pw

    op = P.workload("small-2d", n=64, levels=3)
    u = torch.tensor(op.u, dtype=torch.float32, device="cuda")
    v = torch.tensor(op.v, dtype=torch.float32, device="cuda")
    g = pw.PCOperator(pw.desc_of(op), u, v)
    K = (2 * op.r + 1) ** op.d
    for call in range(2):
        G = torch.tensor(P.normal(P.BASE_SEED + 500 + call, g.nnz), dtype=torch.float32, device="cuda")
        du_ref, dv_ref = g.backward(G)
        du = torch.full((op.m, K), float("nan"), dtype=torch.float32, device="cuda")
        dv = torch.full((op.m, op.N), float("nan"), dtype=torch.float32, device="cuda")
        pw.pc_backward_noalloc(g.h, G, du, dv)
        g.sync()
        for got, ref in ((du, du_ref), (dv, dv_ref)):
            err = torch.linalg.norm((got - ref).double()) / torch.linalg.norm(ref.double())
            assert err <= 1e-5, (call, float(err))
    g.close()
