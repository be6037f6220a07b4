"""GPU parity of pc_assemble against the FP64 oracle (Algorithm 2), through the C-ABI.

Bar: the stored pattern equals the oracle's exactly; FP32 values within max|err| <= 1e-5
max|ref| (the FP32 target), FP64 values within 1e-12 max|ref|; the BF16 copy is the
round-to-nearest of the FP32 value.
"""
import numpy as np
import pytest

import pc_inputs as P
from helpers import compare_columns, make_gpu_op, sample_columns

pytestmark = pytest.mark.gpu

CASES = [
    ("small-1d", {}),
    ("small-1d", {"delta": 2, "levels": 5}),
    ("small-1d", {"n": 64, "levels": 5, "r": 7}),        # heavy periodic wrap at coarse levels
    ("small-1d", {"order": 1}),
    ("small-2d", {}),
    ("small-2d", {"order": 1}),
    ("small-2d", {"gap": 1}),
    ("small-2d", {"delta": 2, "levels": 4}),
    ("small-2d", {"n": 32, "levels": 4, "r": 4}),        # supports wrap the torus
    ("small-2d", {"n": 128, "levels": 5, "r": 5}),       # LL-only first levels for coarse rows
    ("small-2d", {"delta": 3}),                          # db3: 6 taps in the 8-tap template (zero-padded)
    ("small-2d", {"delta": 1, "levels": 4}),             # Haar: 2-tap template
    ("small-2d", {"delta": 5, "n": 128, "levels": 3}),   # db5: 10 taps in the 20-tap template
    ("small-2d", {"r": 0}),                              # point kernels (no widening of the supports)
    ("small-2d", {"gap": 0}),                            # same-level blocks only
    ("small-2d", {"n": 16, "levels": 2, "r": 1}),        # smallest grid: every range wraps
    ("small-2d", {"levels": 1}),                         # one level: approximation + one detail level
    ("small-1d", {"levels": 1}),
    ("c1", {}),                                          # dense 256 x 256
    ("small-2d", {"delta": 6, "family": 1, "n": 64, "levels": 3}),   # Symmlet 6: 12 taps, 20-tap template
    ("small-2d", {"delta": 4, "family": 1}),             # Symmlet 4: 8-tap template
    ("small-1d", {"delta": 6, "family": 1}),
    ("op1", {"n": 64}),                                  # stand-ins for the paper's two blurs (Symmlet 6)
    ("op2", {"n": 64}),
]


@pytest.fixture(scope="module")
def pw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as m
    return m


@pytest.mark.parametrize("name,kw", CASES, ids=[f"{n}-{k}" for n, k in CASES])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp32", "fp64"])
def test_assemble_matches_oracle(pw, name, kw, precision):
    op = P.workload(name, **kw)
    g = make_gpu_op(pw, op, precision=precision, bf16=(precision == 0))
    g.assemble()
    g.sync()
    cols = np.arange(op.N) if op.N <= 1024 else sample_columns(op, per_band=6)
    err, ref = compare_columns(g, op, cols)
    tol = 1e-5 if precision == 0 else 1e-12
    assert err <= tol * ref, (err, ref, err / ref)
    if precision == 0:
        import torch
        v32 = g.values()
        v16 = g.values_bf16()
        assert torch.equal(v32.to(torch.bfloat16), v16)


def test_c2_full_size_sampled(pw):
    """The benchmark workload (2-D 256^2, db4, L=4, m=16, 15x15 Gaussians, gap 2) in the
    launch configuration the benchmark times, on seeded columns of every band."""
    op = P.workload("c2")
    g = make_gpu_op(pw, op, precision=0, bf16=1)
    assert g.nnz == 123896832
    g.assemble()
    g.sync()
    cols = sample_columns(op, per_band=3, seed=11)
    err, ref = compare_columns(g, op, cols)
    assert err <= 1e-5 * ref, (err, ref, err / ref)


def test_reassemble_after_set_params(pw):
    import torch
    op = P.workload("small-2d")
    g = make_gpu_op(pw, op)
    g.assemble()
    op.u = op.u[::-1].copy()                    # different kernels, same shapes
    pw.pc_set_params(g.h, torch.tensor(op.u, dtype=torch.float32, device="cuda"), None)
    g.assemble()
    g.sync()
    err, ref = compare_columns(g, op, sample_columns(op, per_band=3))
    assert err <= 1e-5 * ref
