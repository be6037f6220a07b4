"""Batched persistent assembly (pc_batch_*) and the autotuner, through the C-ABI.

A batch re-runs each operator's own row code, so its values must equal the operator's
single assembly bit for bit; both are checked against the FP64 oracle on sampled columns.
"""
import numpy as np
import pytest

import pc_inputs as P
from helpers import compare_columns, compare_columns_dev, make_gpu_op, sample_columns

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


def test_full_batch_workload_vs_oracle(pw):
    """The batching workload at its own size: 64 operators (32 1-D with n = 2^10..2^16, 32 2-D
    with side 64..512; m 4..25, kernel widths 5..31, db2/db4, L 3..6) assembled by one batch
    (persistent launches captured in a CUDA graph), then replayed.  Every operator is checked
    against the FP64 oracle (Algorithm 2) on columns stratified over its bands (first, last and
    one seeded translate of each band): element-wise within 1e-5 of max|Theta|, with the stored
    pattern equal to the oracle's (over every row for two columns per operator, and every
    oracle entry present for the others)."""
    import torch
    ops = P.batch_workload(64)
    gs = [make_gpu_op(pw, op) for op in ops]
    batch = pw.PCBatch(gs)
    batch.run()
    torch.cuda.synchronize()
    worst = 0.0
    for i, (g, op) in enumerate(zip(gs, ops)):
        g.sync()
        cols = sample_columns(op, per_band=1, seed=100 + i)
        err, ref = compare_columns_dev(g, op, cols[:2], full_pattern=True)
        e2, r2 = compare_columns_dev(g, op, cols[2:], full_pattern=False)
        rel = max(err, e2) / max(ref, r2)
        worst = max(worst, rel)
        assert rel <= 1e-5, (op.name, op.d, op.n, op.m, op.r, op.delta, op.levels, rel)
    batch.close()
    for g in gs:
        g.close()
    print(f"batch workload: worst max rel err {worst:.2e} over 64 operators")
