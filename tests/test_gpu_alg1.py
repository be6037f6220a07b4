"""The GPU's thresholded Algorithm 1 (Section 3.2; pc_alg1_create) against the FP64 oracle's
dense Algorithm 1 (oracle.alg1_dense, reading R21: the Schur-certified rule 0 and the plain cut
tau_k = eps_k, rule 1) on the same seeded operators.

Where several results are correct.  The threshold tau_k ends next to the magnitude of one entry of
A_k; entries whose magnitudes are equal (the translates of a row, and coincident values) can fall
on either side between two FP64 evaluations that round differently.  So every case checks:
  - tau_k against the oracle's (relative 1e-9), the kept counts against the oracle's up to the
    entries tied with tau (|a| within 1e-12 of tau); at eta ~ 0 the threshold falls among the
    rounding-noise entries (below 1e-13 max|A_k|), which count as tied; at eta = 0 the certified
    rule may stop at 0 or just below the smallest significant entry, so there the check is that
    no entry above the noise is discarded;
  - Theta~ element-wise against sum_k (A_k restricted to |a| >= tau_k(GPU)) B_k built from the
    oracle's dense A_k = Psi^T U_k Psi and B_k = Psi^T V_k Psi (numpy products), with an allowance
    for the tied entries only: |dT| <= 1e-12 max|Theta| + sum_k |A_k on ties| |B_k|;
  - where no entry is tied (every tie-free case), Theta~ against the oracle's own Theta~
    element-wise at 1e-12;
  - the guarantee ||Theta - Theta~||_2 <= eta (Section 5.5) with Theta from the oracle."""
import numpy as np
import pytest

import oracle
import pc_inputs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_09870_gb300 as m
    return m


def _tiny(d, n, L, delta, r, m, seed=0, family=0):
    N, K = n ** d, (2 * r + 1) ** d
    u = P.normal(P.BASE_SEED + 100 + seed, m * K).reshape(m, K)
    v = P.uniform(P.BASE_SEED + 200 + seed, m * N).reshape(m, N) + 0.1
    return P.Operator("tiny", d, n, delta, L, r, u, v, gap=-1, family=family)


def _smooth(d, n, L, delta, r, g, family=0):
    """Gaussian kernels of growing width on hat windows (the smooth operators of Section 4.1)."""
    u = np.stack([P.gaussian_kernel(d, r, 0.8 + 0.6 * k).reshape(-1) for k in range(g ** d)])
    v = P.hat_windows(d, n, g)
    return P.Operator("smooth", d, n, delta, L, r, u, v, gap=-1, family=family)


def _one_term(op, u, v, r):
    return P.Operator("term", op.d, op.n, op.delta, op.levels, r, u[None, :], v[None, :], gap=-1,
                      family=op.family)


def _dense_parts(op):
    """The oracle's dense A_k and B_k (row-major N x N) for every term."""
    N = op.N
    cols = np.arange(N)
    A, B = [], []
    for k in range(op.m):
        A.append(oracle.theta_columns(_one_term(op, op.u[k], np.ones(N), op.r), cols).T.copy())
        B.append(oracle.theta_columns(_one_term(op, np.ones(1), op.v[k], 0), cols).T.copy())
    return A, B


def _run(pw, op, eta, fp32=False, rule=0):
    desc = pw.make_desc(op.d, op.n, op.levels, op.delta, op.m, op.r, gap=-1, order=0,
                        precision=pw.PC_FP32 if fp32 else pw.PC_FP64, family=op.family)
    a = pw.PCAlg1(desc, op.u, op.v, eta, rule=rule)
    T = a.dense()
    out = (T, a.kept.copy(), a.tau.copy(), a.nnz)
    a.close()
    return out


def _check_case(pw, op, eta, strict_when_untied=True, fp32=False, rule=0):
    tol = 1e-5 if fp32 else 1e-12
    T, kept, tau, nnz = _run(pw, op, eta, fp32, rule)
    To, kept_o, tau_o = oracle.alg1_dense(op, eta, rule=rule)
    A, B = _dense_parts(op)
    scale = max(np.abs(To).max(), 1e-300)
    expect = np.zeros_like(T)
    allow = np.zeros_like(T)
    tied_any = False
    for k in range(op.m):
        a = np.abs(A[k])
        amax = a.max()
        top = amax * (1 + 1e-15) + 1e-300
        noise = 1e-13 * amax
        ties = (np.abs(a - tau[k]) <= 1e-12 * tau[k]) & (a > 0)
        sig = a > noise
        if rule == 1:
            assert tau[k] == tau_o[k], (k, tau[k], tau_o[k])      # both eta / (m max|v_k|)
            amb = ties
        elif eta == 0.0:
            # eps_k = 0: nothing significant may go; where each side's rounding leaves exact zeros or
            # ~1e-17 noise decides whether its threshold stops at 0 or just below the smallest entry
            assert tau[k] <= a[sig].min(initial=np.inf) * (1 + 1e-9), (k, tau[k])
            assert int(kept[k]) >= int(np.count_nonzero(sig)), (k, kept[k])
            amb = ties | ((a > 0) & ~sig)
            tied_any |= bool(amb.any()) or tau[k] != tau_o[k]
            expect += np.where(sig, A[k], 0.0) @ B[k]
            if amb.any():
                allow += np.where(amb, a, 0.0) @ np.abs(B[k])
            continue
        elif tau_o[k] <= noise or tau[k] <= noise:
            # eta ~ 0: the threshold sits among rounding-noise entries (exact zeros of A_k that
            # each FP64 evaluation leaves at its own ~1e-17 level), which both sides may keep
            assert tau[k] <= noise and tau_o[k] <= noise, (k, tau[k], tau_o[k])
            amb = ties | ((a > 0) & (a <= noise))
        else:
            # the GPU's threshold: the oracle's within the bisection's resolution, or the top
            assert abs(tau[k] - tau_o[k]) <= 1e-9 * tau_o[k] or (tau[k] >= amax and tau_o[k] >= amax), \
                (k, tau[k], tau_o[k])
            amb = ties
        tied_any |= bool(amb.any())
        keep = (a >= tau[k]) & (a > 0)
        n_amb = int(np.count_nonzero(amb))
        assert abs(int(kept[k]) - int(np.count_nonzero(keep))) <= n_amb, (k, kept[k])
        if tau_o[k] > 0.0:
            assert abs(int(kept[k]) - int(kept_o[k])) <= n_amb, (k, kept[k], kept_o[k])
        else:
            # a zero threshold (the bisection never left lo = 0) keeps every entry, zeros included
            assert kept_o[k] == op.N * op.N and kept[k] <= op.N * op.N
        expect += np.where(keep & ~amb, A[k], 0.0) @ B[k]
        if amb.any():
            allow += np.where(amb, a, 0.0) @ np.abs(B[k])
        if rule == 0 and tau[k] < top:
            # the kept part is what the threshold certifies: discarded Schur bound within eps_k
            D = np.where(a < tau[k] * (1 - 1e-12), a, 0.0)
            eps = eta / (op.m * np.abs(op.v[k]).max())
            assert np.sqrt(D.sum(0).max() * D.sum(1).max()) <= eps * (1 + 1e-9) + 1e-12 * amax
    err = np.abs(T - expect)
    assert np.all(err <= tol * scale + allow * (1 + 1e-9)), err.max() / scale
    if strict_when_untied and not tied_any:
        assert np.array_equal(kept, kept_o)
        assert np.abs(T - To).max() <= tol * scale, np.abs(T - To).max() / scale
    return T, To


CASES = [
    # d, n, L, delta, r, m, family
    (1, 32, 3, 2, 2, 2, 0),
    (1, 64, 4, 4, 3, 3, 0),
    (1, 1024, 5, 4, 4, 3, 0),
    (1, 256, 8, 2, 3, 2, 0),        # L = log2 n: every row its own class
    (2, 16, 2, 2, 1, 2, 0),
    (2, 32, 3, 3, 2, 3, 0),
    (2, 32, 3, 3, 2, 2, 1),         # Symmlet 6
    (2, 32, 5, 2, 1, 2, 0),         # L = log2 n
    (2, 8, 1, 1, 0, 1, 0),          # Haar, one level, a delta kernel (A_k = I), one term
    (1, 16, 4, 1, 0, 1, 0),         # Haar, full depth, delta kernel
    (2, 16, 3, 1, 2, 3, 0),         # Haar, radius 2
]


@pytest.mark.parametrize("eta", [0.0, 1e-3, 1e-1, 1e3])
@pytest.mark.parametrize("d,n,L,delta,r,m,family", CASES)
def test_alg1_matches_oracle(pw, d, n, L, delta, r, m, family, eta):
    op = _tiny(d, n, L, delta, r, m, seed=d * 7 + n + L, family=family)
    T, To = _check_case(pw, op, eta)
    if eta >= 1e3:
        assert not np.any(T)


@pytest.mark.parametrize("eta", [1e-4, 1e-2, 1e-1])
@pytest.mark.parametrize("d,n,L,delta,r,m,family", CASES)
def test_alg1_hard_rule_matches_oracle(pw, d, n, L, delta, r, m, family, eta):
    """The plain cut tau_k = eps_k (rule 1), FP64 and FP32 products."""
    op = _tiny(d, n, L, delta, r, m, seed=d * 7 + n + L, family=family)
    _check_case(pw, op, eta, rule=1)
    _check_case(pw, op, eta, rule=1, fp32=True)


@pytest.mark.parametrize("eta", [1e-3, 1e-1])
@pytest.mark.parametrize("d,n,L,delta,r,m,family", [CASES[1], CASES[2], CASES[5], CASES[6], CASES[7]])
def test_alg1_fp32_matches_oracle(pw, d, n, L, delta, r, m, family, eta):
    """FP32 products (the same FP64 thresholds): Theta~ within 1e-5 of max|Theta~| element-wise."""
    op = _tiny(d, n, L, delta, r, m, seed=d * 7 + n + L, family=family)
    _check_case(pw, op, eta, fp32=True)


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("L,r,rule,eta", [(3, 3, 0, 1e-2), (2, 1, 1, 1e-3), (3, 1, 1, 1e-2)])
def test_alg1_4096_pixels(pw, fp32, L, r, rule, eta):
    """A 64 x 64 image, db2: support boxes narrower than the image (the unchecked interior taps)
    next to full-period ones at the coarse levels."""
    op = _tiny(2, 64, L, 2, r, 2, seed=5 + L + r)
    _check_case(pw, op, eta, fp32=fp32, rule=rule)


@pytest.mark.parametrize("d,n,L,delta,r,g", [(1, 256, 5, 3, 8, 4), (2, 32, 3, 2, 4, 2)])
def test_alg1_guarantee(pw, d, n, L, delta, r, g):
    """||Theta - Theta~||_2 <= eta on smooth operators, with fewer kept entries of A~_k and
    larger thresholds as eta grows."""
    op = _smooth(d, n, L, delta, r, g)
    Theta = oracle.theta_columns(op, np.arange(op.N)).T
    prev = None
    for eta in (1e-6, 1e-4, 1e-2, 1e-1):
        T, kept, tau, nnz = _run(pw, op, eta)
        assert np.linalg.norm(Theta - T, 2) <= eta * (1 + 1e-9), eta
        if prev is not None:
            assert nnz <= prev[0] and np.all(kept <= prev[1]) and np.all(tau >= prev[2])
        prev = (nnz, kept, tau)


def test_alg1_storage_shrinks_with_eta(pw):
    """A 128 x 128 smooth operator: the stored support follows the thresholds (boxes narrower
    than the period), so Theta~ holds a part of N^2 and less as eta grows."""
    op = _smooth(2, 128, 3, 2, 4, 2)
    nnzs = []
    desc = pw.make_desc(2, 128, 3, 2, op.m, 4, gap=-1, precision=pw.PC_FP64)
    for eta in (1e-6, 1e-3, 1e-1):
        a = pw.PCAlg1(desc, op.u, op.v, eta)
        nnzs.append(a.nnz)
        a.close()
    assert nnzs[0] >= nnzs[1] >= nnzs[2] and nnzs[2] < 0.9 * nnzs[0]
    assert nnzs[0] < op.N * op.N // 4, nnzs


def test_alg1_eta_zero_is_theta(pw):
    op = _tiny(2, 32, 3, 3, 2, 3, seed=11)
    T, _, _, _ = _run(pw, op, 0.0)
    Theta = oracle.theta_columns(op, np.arange(op.N)).T
    assert np.abs(T - Theta).max() <= 1e-12 * np.abs(Theta).max()


def test_alg1_device_inputs_and_zero_window(pw):
    """Inputs from device memory give the same Theta~; a zero window contributes nothing."""
    import torch
    op = _tiny(2, 16, 2, 2, 1, 3, seed=3)
    op.v[1] = 0.0
    T_host, kept_h, tau_h, _ = _run(pw, op, 1e-3)
    desc = pw.make_desc(2, 16, 2, 2, 3, 1, gap=-1, precision=pw.PC_FP64)
    a = pw.PCAlg1(desc, torch.tensor(op.u, device="cuda"), torch.tensor(op.v, device="cuda"), 1e-3)
    assert np.array_equal(a.dense(), T_host)
    assert np.array_equal(a.kept, kept_h) and np.array_equal(a.tau, tau_h)
    assert a.kept[1] == 0
    a.close()


def test_alg1_rejects(pw):
    op = _tiny(2, 16, 2, 2, 1, 2)
    bad_order = pw.make_desc(2, 16, 2, 2, 2, 1, gap=-1, order=1, precision=pw.PC_FP64)
    with pytest.raises(pw.PCError) as e:
        pw.PCAlg1(bad_order, op.u, op.v, 1e-3)
    assert e.value.status == pw.PC_ERR_UNSUPPORTED
    bad_prec = pw.make_desc(2, 16, 2, 2, 2, 1, gap=-1, precision=7)
    with pytest.raises(pw.PCError) as e:
        pw.PCAlg1(bad_prec, op.u, op.v, 1e-3)
    assert e.value.status == pw.PC_ERR_INVALID_ARG
    ok = pw.make_desc(2, 16, 2, 2, 2, 1, gap=-1, precision=pw.PC_FP64)
    with pytest.raises(pw.PCError) as e:
        pw.PCAlg1(ok, op.u, op.v, -1.0)
    assert e.value.status == pw.PC_ERR_INVALID_ARG
    with pytest.raises(pw.PCError) as e:
        pw.PCAlg1(ok, op.u, op.v, 1e-3, rule=2)
    assert e.value.status == pw.PC_ERR_INVALID_ARG


def test_alg1_oversize_reports_oom_and_leaves_the_context_usable(pw):
    """A 2048 x 2048 Symmlet-6 operator at eta = 5e-4 needs ~10^11 stored entries (rows reach the
    coarse wavelets' supports): PC_ERR_OOM, no pending CUDA error, and the next calls work."""
    import torch
    op = P.workload("op1", n=2048)
    desc = pw.make_desc(2, 2048, op.levels, op.delta, op.m, op.r, gap=-1, precision=pw.PC_FP32, family=op.family)
    with pytest.raises(pw.PCError) as e:
        pw.PCAlg1(desc, op.u, op.v, 5e-4, rule=pw.PC_ALG1_HARD)
    assert e.value.status == pw.PC_ERR_OOM
    x = torch.ones(1 << 20, device="cuda")
    assert float(x.sum()) == float(1 << 20)
    small = _tiny(2, 16, 2, 2, 1, 2, seed=4)
    T, _, _, _ = _run(pw, small, 1e-3)
    assert np.isfinite(T).all()


def _oracle_rows(op, tau, rows):
    """Rows of sum_k A~_k B_k from the oracle's transforms (FP64, full periodic length): row mu is
    Psi^*(sum_k v_k . Psi A~_k[mu, :]) since B_k = Psi^* diag(v_k) Psi, with A_k[mu, :] = Psi^* F
    and F(z) = sum_t u_k(t) psi_mu(z + t); A~_k keeps |a| >= tau_k.  Returns, per row, the row with
    the entries tied with tau_k (within 1e-9) kept, the row with them dropped, and their number."""
    d, n, L, r = op.d, op.n, op.levels, op.r
    K1 = 2 * r + 1
    shape = (n, n) if d == 2 else (n,)
    out = []
    for mu in rows:
        e = np.zeros(op.N)
        e[mu] = 1.0
        psi = oracle.idwt(d, n, L, op.delta, e, family=op.family).reshape(shape)
        s = np.zeros(op.N)
        s_drop = np.zeros(op.N)
        ties = 0
        for k in range(op.m):
            uk = op.u[k].reshape((K1, K1) if d == 2 else (K1,))
            F = np.zeros(shape)
            if d == 2:
                for t0 in range(-r, r + 1):
                    for t1 in range(-r, r + 1):
                        if uk[t0 + r, t1 + r] != 0.0:
                            F += uk[t0 + r, t1 + r] * np.roll(psi, (-t0, -t1), (0, 1))
            else:
                for t in range(-r, r + 1):
                    F += uk[t + r] * np.roll(psi, -t)
            a = oracle.dwt(d, n, L, op.delta, F.reshape(-1), family=op.family)
            tied = np.abs(np.abs(a) - tau[k]) <= 1e-9 * tau[k]
            ties += int(np.count_nonzero(tied))
            keep = np.abs(a) >= tau[k]
            s += op.v[k] * oracle.idwt(d, n, L, op.delta, np.where(keep | tied, a, 0.0), family=op.family)
            s_drop += op.v[k] * oracle.idwt(d, n, L, op.delta, np.where(keep & ~tied, a, 0.0), family=op.family)
        out.append((oracle.dwt(d, n, L, op.delta, s, family=op.family),
                    oracle.dwt(d, n, L, op.delta, s_drop, family=op.family), ties))
    return out


def _check_rows(a, op, rows, tau, tol):
    """Sampled rows of the GPU's Theta~ against _oracle_rows: element-wise within tol of the row's
    largest magnitude (tied entries: either variant), zero where the GPU stores nothing."""
    for mu, (ref, ref_drop, ties) in zip(rows, _oracle_rows(op, tau, rows)):
        cols, vals = a.row(mu)
        got = np.zeros(op.N)
        got[cols] = vals
        off = np.ones(op.N, dtype=bool)
        off[cols] = False
        res = []
        for r in ((ref, ref_drop) if ties else (ref,)):
            scale = np.abs(r).max()
            err = np.abs(got - r).max() / scale
            outside = np.abs(r[off]).max(initial=0.0) / scale
            res.append((err, outside))
        assert any(err <= tol and outside <= 1e-12 for err, outside in res), (mu, ties, res)


@pytest.mark.parametrize("name,n,fp32", [("op1", 256, True), ("op2", 256, True), ("op1", 256, False),
                                         ("op1", 1024, True)])
def test_alg1_rows_large(pw, name, n, fp32):
    """The Symmlet-6 stand-ins at 256^2 and 1024^2 (the benchmark's cases; support boxes too large
    for shared memory, so the global-scratch product path runs), eta = 5e-4, the plain cut:
    sampled rows of every level against the oracle's transforms, element-wise; the columns the GPU
    does not store are zero there.  (op1 at 1024^2 holds 4.8e10 FP32 entries, 192 GB.)"""
    op = P.workload(name, n=n)
    desc = pw.make_desc(2, n, op.levels, op.delta, op.m, op.r, gap=-1,
                        precision=pw.PC_FP32 if fp32 else pw.PC_FP64, family=op.family)
    a = pw.PCAlg1(desc, op.u, op.v, 5e-4, rule=pw.PC_ALG1_HARD)
    eps = 5e-4 / (op.m * np.abs(op.v).max(1))
    assert np.array_equal(a.tau, eps)
    L = op.levels
    nL = n >> L
    rows = [3 * nL + 5,                                    # approximation
            nL * nL + 7 * nL + 2,                           # level L, band (0,1)
            3 * (n >> 2) ** 2 + 11 * (n >> 2) + 40,        # level 2, band (1,1)
            (n >> 1) ** 2 + 77 * (n >> 1) + 101,           # level 1, band (0,1)
            2 * (n >> 1) ** 2 + 128 * (n >> 1) - 1]        # level 1, band (1,0), end of line 127
    _check_rows(a, op, rows, a.tau, 1e-5 if fp32 else 1e-12)
    a.close()


def test_alg1_discard_mode(pw):
    """PC_ALG1_DISCARD on the 256^2 op1 stand-in (FP32 Theta~ of ~10 GB, two groups of classes
    in the 8 GB buffer): the same thresholds, kept counts and stored-entry count as the kept run,
    and the matrix calls refuse."""
    import torch
    op = P.workload("op1", n=256)
    desc = pw.make_desc(2, 256, op.levels, op.delta, op.m, op.r, gap=-1, precision=pw.PC_FP32, family=op.family)
    a = pw.PCAlg1(desc, op.u, op.v, 5e-4, rule=pw.PC_ALG1_HARD)
    b = pw.PCAlg1(desc, op.u, op.v, 5e-4, rule=pw.PC_ALG1_HARD, flags=pw.PC_ALG1_DISCARD)
    assert a.nnz * 4 > (8 << 30)
    assert np.array_equal(a.tau, b.tau) and np.array_equal(a.kept, b.kept) and a.nnz == b.nnz
    for call in (lambda: b.row(0), b.export):
        with pytest.raises(pw.PCError) as e:
            call()
        assert e.value.status == pw.PC_ERR_UNSUPPORTED
    cols, vals = a.row(1000)
    assert len(cols) > 0 and np.isfinite(vals).all()
    a.close()
    b.close()
    assert float(torch.ones(8, device="cuda").sum()) == 8.0


@pytest.mark.parametrize("rule,fp32", [(1, True), (0, False)])
def test_alg1_rows_1d_65536(pw, rule, fp32):
    """A 1-D signal of 2^16 samples, six levels, db3: sampled rows of every level against the
    oracle's transforms (both rules; the certified threshold is taken from the GPU and checked
    on the sampled rows only through Theta~)."""
    op = P.workload("small-1d", n=1 << 16, levels=6, delta=3)
    desc = pw.make_desc(1, op.n, op.levels, op.delta, op.m, op.r, gap=-1,
                        precision=pw.PC_FP32 if fp32 else pw.PC_FP64, family=op.family)
    a = pw.PCAlg1(desc, op.u, op.v, 1e-3, rule=rule)
    if rule == 1:
        assert np.array_equal(a.tau, 1e-3 / (op.m * np.abs(op.v).max(1)))
    n, L = op.n, op.levels
    rows = [5, (n >> L) + 17]                                        # approximation, level L
    rows += [(n >> j) + (n >> j) // 3 for j in (4, 2, 1)]           # levels 4, 2, 1
    rows += [n - 1]                                                  # last row of level 1
    _check_rows(a, op, rows, a.tau, 1e-5 if fp32 else 1e-12)
    a.close()
