"""pc_export: Theta as host CSR (ascending columns per row, rows = outputs, in either operator
order) against the oracle's pattern and values (Algorithm 2), and its product against pc_apply."""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("name,kw", [("small-2d", {"n": 32, "levels": 3}), ("small-2d", {"n": 32, "levels": 3, "order": 1}),
                                     ("small-1d", {}), ("op1", {"n": 32, "levels": 3})])
@pytest.mark.parametrize("prec", [0, 1])
def test_export_matches_oracle(pw, name, kw, prec):
    import torch
    op = P.workload(name, **kw)
    g = make_gpu_op(pw, op, precision=prec)
    g.assemble()
    rp, cols, vals = g.export()
    assert rp[0] == 0 and rp[-1] == g.nnz and np.all(np.diff(rp) > 0)
    T = dense_theta_pattern(op)
    for mu in range(op.N):
        c = cols[rp[mu]:rp[mu + 1]]
        assert np.all(np.diff(c) > 0), mu
        assert np.array_equal(c, np.flatnonzero(oracle.pattern_column(op, mu))), mu
    rows = np.repeat(np.arange(op.N), np.diff(rp))
    err = np.abs(vals - T[rows, cols]).max()
    assert err <= (1e-12 if prec else 1e-5) * np.abs(T).max()
    # the exported matrix times x equals pc_apply (same stored values)
    x = P.normal(P.BASE_SEED + 640, op.N)
    y = np.zeros(op.N)
    np.add.at(y, rows, vals * x[cols])
    dt = torch.float64 if prec else torch.float32
    yg = g.apply(torch.tensor(x, dtype=dt, device="cuda").reshape(op.N, 1)).double().cpu().numpy().ravel()
    assert np.abs(yg - y).max() <= (1e-12 if prec else 1e-5) * np.abs(y).max()
    g.close()


def test_export_before_assembly_fails(pw):
    op = P.workload("small-1d")
    g = make_gpu_op(pw, op)
    with pytest.raises(pw.PCError) as e:
        g.export()
    assert e.value.status == pw.PC_ERR_NOT_ASSEMBLED
    g.close()
