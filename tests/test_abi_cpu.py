"""CPU tests of the C-ABI library: it loads, exports every entry point that include/pcwave.h
declares, validates descriptors, and its host planner's pattern equals the oracle's pattern
(bit-exact index sets).  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import pc_inputs as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pw():
    import importlib.util
    spec = importlib.util.spec_from_file_location("pcwave_build", os.path.join(ROOT, "paper_2005_09870_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_2005_09870_gb300 as m
    return m


def test_exports_every_declared_symbol(pw):
    header = open(os.path.join(ROOT, "include", "pcwave.h")).read()
    declared = set(re.findall(r"^\s*(?:pc_status|void|const char\*|int64_t)\s+(pc_\w+)\s*\(", header, re.M))
    assert len(declared) >= 20
    lib = ctypes.CDLL(pw.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), name


def test_plan_check_rejects_bad_descriptors(pw):
    good = pw.make_desc(2, 64, 3, 4, 9, 3)
    pw.pc_plan_check(good)
    bad = [pw.make_desc(3, 64, 3, 4, 9, 3), pw.make_desc(2, 60, 3, 4, 9, 3), pw.make_desc(2, 64, 7, 4, 9, 3),
           pw.make_desc(2, 64, 3, 0, 9, 3), pw.make_desc(2, 64, 3, 4, 0, 3), pw.make_desc(2, 64, 3, 4, 300, 3),
           pw.make_desc(2, 64, 3, 4, 9, -1), pw.make_desc(2, 64, 3, 4, 9, 3, gap=-2),
           pw.make_desc(2, 64, 3, 4, 9, 3, order=2), pw.make_desc(2, 64, 3, 4, 9, 3, precision=1, store_bf16=1),
           pw.make_desc(2, 256, 3, 4, 9, 3, gap=-1), pw.make_desc(2, 64, 3, 4, 9, 3, family=2),
           pw.make_desc(2, 64, 3, 4, 9, 3, family=-1)]
    for d in bad:
        with pytest.raises(pw.PCError):
            pw.pc_plan_check(d)


@pytest.mark.parametrize("name,kw", [("small-1d", {}), ("small-1d", {"delta": 2, "levels": 5}),
                                     ("small-1d", {"n": 64, "levels": 5, "r": 7}), ("c1", {}),
                                     ("small-2d", {"n": 32}), ("small-2d", {"n": 32, "gap": 1}),
                                     ("small-2d", {"n": 16, "levels": 4, "r": 4}), ("small-2d", {"n": 32, "order": 1})])
def test_planner_pattern_equals_oracle(pw, name, kw):
    op = P.workload(name, **kw)
    desc = pw.desc_of(op)
    total = 0
    for lam in range(op.N):
        cols = pw.pc_plan_row(desc, lam)         # stored row lam: the pattern is symmetric
        assert len(set(cols.tolist())) == len(cols)
        assert set(cols.tolist()) == set(np.nonzero(oracle.pattern_column(op, lam))[0].tolist()), lam
        total += len(cols)
    assert pw.pc_plan_nnz(desc) == total


def test_plan_nnz_of_the_benchmark_workloads(pw):
    """Pattern sizes of the 256^2, 128^2 and 1024^2 workloads (regression values of the
    planner; the sampled test below checks rows of the 256^2 workload against the oracle)."""
    assert pw.pc_plan_nnz(pw.make_desc(2, 256, 4, 4, 16, 7)) == 123896832
    assert pw.pc_plan_nnz(pw.make_desc(2, 128, 3, 4, 9, 5)) == 25412608
    assert pw.pc_plan_nnz(pw.make_desc(2, 1024, 5, 4, 64, 15)) == 3555397632


def test_oracle_pattern_row_counts_sampled(pw):
    """On the 256^2 workload, sampled rows of every band: the planner's row equals the oracle's
    pattern column (bit-exact)."""
    op = P.workload("c2")
    desc = pw.desc_of(op)
    rng = np.random.default_rng(3)
    for lam in list(rng.integers(0, op.N, 12)) + [0, op.N - 1, 16 * 16, 4096]:
        cols = pw.pc_plan_row(desc, int(lam))
        assert set(cols.tolist()) == set(np.nonzero(oracle.pattern_column(op, int(lam)))[0].tolist())


@pytest.mark.parametrize("family", [0, 1])
def test_host_filter_taps_equal_oracle(pw, family):
    """The library's host taps (C++, Laguerre roots) against the oracle's (C, Durand-Kerner
    roots): two implementations of the same spectral factor choice."""
    for delta in range(1, 11):
        got = pw.pc_filter_taps(family, delta)
        want = oracle.symmlet(delta) if family else oracle.daubechies(delta)
        assert np.abs(got - want).max() < 1e-13, delta
    with pytest.raises(pw.PCError):
        pw.pc_filter_taps(2, 4)
    with pytest.raises(pw.PCError):
        pw.pc_filter_taps(family, 11)


def test_planner_pattern_equals_oracle_symmlet(pw):
    for name, kw in (("op1", {"n": 32, "levels": 3}), ("small-1d", {"delta": 6, "family": 1})):
        op = P.workload(name, **kw)
        desc = pw.desc_of(op)
        assert desc.family == 1
        for lam in np.random.default_rng(4).integers(0, op.N, 40):
            cols = pw.pc_plan_row(desc, int(lam))
            mask = oracle.pattern_column(op, int(lam))
            assert np.array_equal(np.sort(cols), np.flatnonzero(mask))
