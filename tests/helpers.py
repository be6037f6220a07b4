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


def compare_columns_dev(pcop, op, cols, nthreads=0, full_pattern=True):
    """compare_columns for large operators: only the compared entries are gathered from the
    device.  full_pattern: check the stored pattern of each column against the oracle's over
    every row (otherwise only that every oracle pattern entry is stored)."""
    import torch
    vals = pcop.values()
    T = oracle.theta_columns(op, cols, nthreads=nthreads)
    err = ref = 0.0
    N = op.N
    for c, lam in enumerate(cols):
        mask = oracle.pattern_column(op, lam)
        if full_pattern:
            mus = np.arange(N, dtype=np.int64)
            pos = pcop.lookup(mus, np.full(N, lam, dtype=np.int64))
            assert np.array_equal(pos >= 0, mask), f"pattern differs in column {lam}"
            pos = pos[mask]
        else:
            mus = np.nonzero(mask)[0].astype(np.int64)
            pos = pcop.lookup(mus, np.full(mus.size, lam, dtype=np.int64))
            assert (pos >= 0).all(), f"oracle pattern entry not stored in column {lam}"
        got = vals[torch.as_tensor(pos, device=vals.device)].double().cpu().numpy()
        want = T[c][mask]
        err = max(err, float(np.abs(got - want).max(initial=0.0)))
        ref = max(ref, float(np.abs(want).max(initial=0.0)))
    return err, ref


def assert_elementwise(got, ref, tol, what=""):
    """Element-wise bound: every |got - ref| <= tol * max |ref| (the metric the tests use for
    Theta, applied to each entry of a gradient: a wrong entry larger than tol * max |ref|
    fails however many correct entries surround it)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    scale = float(np.abs(ref).max())
    err = np.abs(got - ref)
    worst = int(np.argmax(err))
    assert err.flat[worst] <= tol * scale, (
        f"{what}: entry {np.unravel_index(worst, ref.shape)} got {got.flat[worst]!r} want {ref.flat[worst]!r}; "
        f"max err {err.flat[worst]:.3e} > {tol:.1e} x max|ref| {scale:.3e}")
    return float(err.flat[worst] / scale) if scale else 0.0


def storage_map(pw, desc, N):
    """(rows, cols) of every stored entry in storage order, from the host planner
    (pc_plan_row): entry i of the stored values is S[rows[i], cols[i]] (S = Theta in the
    paper's order)."""
    rows, cols = [], []
    for s in range(N):
        c = pw.pc_plan_row(desc, s)
        rows.append(np.full(c.size, s, dtype=np.int32))
        cols.append(c.astype(np.int32))
    return np.concatenate(rows), np.concatenate(cols)


def flipped(op):
    """The operator with every kernel mirrored (u_k(t) -> u_k(-t)) and the other order: by the
    order-flag identity Theta_1(u, v) = Theta_0(flip u, v)^T, column mu of its Theta is row
    mu of op's Theta."""
    import copy
    o = copy.copy(op)
    o.u = np.ascontiguousarray(op.u[:, ::-1])
    o.order = 1 - op.order
    return o


def oracle_rows(op, rows, nthreads=0):
    """Rows Theta[rows, :] of the oracle's Theta (Algorithm 2 columns of the flipped operator)."""
    return oracle.theta_columns(flipped(op), rows, nthreads=nthreads)
