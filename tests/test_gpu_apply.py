"""GPU parity of pc_apply (y = Theta x on the stored pattern) against the oracle's Theta."""
import numpy as np
import pytest

import pc_inputs as P
from helpers import dense_theta_pattern, make_gpu_op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as m
    return m


@pytest.mark.parametrize("name,kw", [("small-1d", {}), ("small-2d", {"n": 32, "levels": 3}),
                                     ("small-2d", {"n": 32, "levels": 3, "order": 1}), ("c1", {})])
@pytest.mark.parametrize("nrhs", [1, 3, 16, 21, 64])
@pytest.mark.parametrize("mode", ["fp32", "bf16", "fp64"])
def test_apply_matches_oracle(pw, name, kw, nrhs, mode):
    import torch
    op = P.workload(name, **kw)
    prec = 1 if mode == "fp64" else 0
    g = make_gpu_op(pw, op, precision=prec, bf16=(mode == "bf16"))
    g.assemble()
    T = dense_theta_pattern(op)
    x = P.normal(P.BASE_SEED + 31, op.N * nrhs).reshape(op.N, nrhs)
    dt = torch.float64 if prec else torch.float32
    xd = torch.tensor(x, dtype=dt, device="cuda")
    y = g.apply(xd)
    g.sync()
    ref = T @ x
    rel = np.linalg.norm(y.double().cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    tol = {"fp32": 1e-5, "bf16": 1e-2, "fp64": 1e-12}[mode]
    assert rel.max() <= tol, rel


def test_apply_strided(pw):
    """ldx, ldy larger than nrhs: only the first nrhs columns are read / written."""
    import torch
    op = P.workload("small-1d")
    g = make_gpu_op(pw, op)
    g.assemble()
    T = dense_theta_pattern(op)
    x = torch.randn(op.N, 7, dtype=torch.float32, device="cuda")
    y = torch.full((op.N, 9), 7.0, dtype=torch.float32, device="cuda")
    pw.pc_apply(g.h, x, y, nrhs=5, ldx=7, ldy=9)
    g.sync()
    ref = T @ x[:, :5].double().cpu().numpy()
    got = y[:, :5].double().cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    assert torch.all(y[:, 5:] == 7.0)


@pytest.mark.parametrize("nrhs,ld", [(8, 8), (12, 12), (21, 24), (5, 8), (16, 20)])
def test_apply_vector_groups(pw, nrhs, ld):
    """16-byte aligned x/y with ld % 4 == 0 take the float4 path in groups of 16/8/4 columns,
    the remainder (< 4) the scalar path; padding columns are left untouched."""
    import torch
    op = P.workload("small-2d", n=32, levels=3)
    g = make_gpu_op(pw, op, bf16=1)
    g.assemble()
    T = dense_theta_pattern(op)
    x = torch.randn(op.N, ld, dtype=torch.float32, device="cuda")
    y = torch.full((op.N, ld), 3.0, dtype=torch.float32, device="cuda")
    pw.pc_apply(g.h, x, y, nrhs=nrhs, ldx=ld, ldy=ld)
    g.sync()
    ref = T @ x[:, :nrhs].double().cpu().numpy()
    got = y[:, :nrhs].double().cpu().numpy()
    rel = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rel.max() <= 1e-2
    assert torch.all(y[:, nrhs:] == 3.0)


def test_apply_errors(pw):
    """pc_apply before the first assembly, and right-hand-side counts outside 1..64."""
    import torch
    op = P.workload("small-2d", n=32, levels=3)
    g = make_gpu_op(pw, op, bf16=1)
    x = torch.zeros((op.N, 4), dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(pw.PCError) as e:
        pw.pc_apply(g.h, x, y, nrhs=4)
    assert e.value.status == pw.PC_ERR_NOT_ASSEMBLED
    g.assemble()
    for bad in (0, 65):
        with pytest.raises(pw.PCError) as e:
            pw.pc_apply(g.h, x, y, nrhs=bad, ldx=max(bad, 1), ldy=max(bad, 1))
        assert e.value.status == pw.PC_ERR_INVALID_ARG
    g.sync()
