"""Batched persistent assembly (pc_batch_*) and the autotuner, through the C-ABI.

A batch re-runs each operator's own row code, so its values must equal the operator's
single assembly bit for bit; both are checked against the FP64 oracle on sampled columns.
"""
import numpy as np
import pytest

import pc_inputs as P
from helpers import compare_columns, make_gpu_op, sample_columns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as m
    return m


def _mixed_ops():
    """Uneven batch: 1-D and 2-D, db2/db4, several m, radii, levels, a region wrapping the torus."""
    ops = P.batch_workload(count=12, max_side_2d=128, max_pow_1d=12)
    ops.append(P.workload("small-2d", n=32, levels=4, r=4))
    ops.append(P.workload("small-1d", n=64, levels=5, r=7, order=1))
    return ops


def test_batch_equals_single_assembly(pw):
    import torch
    ops = _mixed_ops()
    singles = []
    for op in ops:
        g = make_gpu_op(pw, op, bf16=1)
        g.assemble()
        singles.append(g.values().clone())
        g.close()
    gs = [make_gpu_op(pw, op, bf16=1) for op in ops]
    batch = pw.PCBatch(gs)
    assert batch.items >= len(ops)
    for g, ref in zip(gs, singles):
        g.sync()
        assert torch.equal(g.values(), ref)
        assert torch.equal(g.values_bf16(), ref.to(torch.bfloat16))
    # new parameters, graph replay
    for g, op in zip(gs, ops):
        op.u = op.u * 0.5 + 0.01
        pw.pc_set_params(g.h, torch.tensor(op.u, dtype=torch.float32, device="cuda"), None)
    batch.run()
    torch.cuda.synchronize()
    for g, op in list(zip(gs, ops))[::4]:
        err, ref = compare_columns(g, op, sample_columns(op, per_band=2, seed=5))
        assert err <= 1e-5 * ref, (op.name, err / ref)
    batch.close()


def test_batch_rejects_fp64(pw):
    op = P.workload("small-1d")
    g = make_gpu_op(pw, op, precision=1)
    with pytest.raises(pw.PCError):
        pw.PCBatch([g])


def test_autotune_keeps_values(pw):
    import torch
    op = P.workload("small-2d")
    g = make_gpu_op(pw, op)
    g.assemble()
    before = g.values().clone()
    pw.pc_autotune(g.h)
    g.sync()
    assert torch.equal(g.values(), before)      # every row's arithmetic is independent of the group shape
    g.assemble()
    g.sync()
    assert torch.equal(g.values(), before)
    err, ref = compare_columns(g, op, sample_columns(op, per_band=2))
    assert err <= 1e-5 * ref
