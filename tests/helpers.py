"""Shared helpers of the GPU parity tests: build an operator through the C-ABI binding and
compare its stored entries with the FP64 oracle, column by column (Algorithm 2)."""
import numpy as np

import oracle


def make_gpu_op(pw, op, precision=0, bf16=0):
    import torch
    dt = torch.float64 if precision == pw.PC_FP64 else torch.float32
    u = torch.tensor(op.u, dtype=dt, device="cuda").contiguous()
    v = torch.tensor(op.v, dtype=dt, device="cuda").contiguous()
    return pw.PCOperator(pw.desc_of(op, precision, bf16), u, v)


def sample_columns(op, per_band=4, seed=0):
    """Seeded columns stratified over bands (every band, first/last translate included)."""
    rng = np.random.default_rng(seed)
    n, L, d = op.n, op.levels, op.d
    cols = []
    nL = n >> L
    starts = [(0, nL ** d)]
    for j in range(L, 0, -1):
        nj = n >> j
        nb = nj ** d
        for t in range(1 if d == 1 else 3):
            starts.append((nb * (1 + t) if d == 2 else nj, nb))
    for off, size in starts:
        pick = {off, off + size - 1}
        pick.update((off + rng.integers(0, size, per_band)).tolist())
        cols += sorted(pick)
    return np.array(sorted(set(cols)), dtype=np.int64)


def compare_columns(pcop, op, cols, values=None, nthreads=0):
    """Returns (max |err|, max |ref|) over the pattern entries of the given columns, after
    checking that the stored pattern equals the oracle's pattern exactly."""
    vals = (pcop.values() if values is None else values).double().cpu().numpy()
    T = oracle.theta_columns(op, cols, nthreads=nthreads)
    err = 0.0
    ref = 0.0
    N = op.N
    mus = np.arange(N, dtype=np.int64)
    for c, lam in enumerate(cols):
        mask = oracle.pattern_column(op, lam)
        pos = pcop.lookup(mus, np.full(N, lam, dtype=np.int64))
        assert np.array_equal(pos >= 0, mask), f"pattern differs in column {lam}"
        got = vals[pos[mask]]
        want = T[c][mask]
        err = max(err, float(np.abs(got - want).max(initial=0.0)))
        ref = max(ref, float(np.abs(want).max(initial=0.0)))
        # entries outside the pattern are not stored; the oracle's must be beyond the band gap
    return err, ref


def dense_theta_pattern(op, nthreads=0):
    """Oracle Theta restricted to the pattern, dense (small N only)."""
    cols = np.arange(op.N)
    T = oracle.theta_columns(op, cols, nthreads=nthreads).T.copy()
    for lam in cols:
        T[~oracle.pattern_column(op, lam), lam] = 0.0
    return T
