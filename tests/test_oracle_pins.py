"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks an oracle function against the mathematics the paper fixes: closed-form
filter taps, orthonormality of the basis built by an independent matrix form of the
cascade recursion (Section 2.1), brute-force dense Theta = Psi^T H Psi, the closed
forms Theta = I and B = Psi^T V Psi, the circulant (translation) structure of
convolution sub-bands (Lemma 5.1), trace / Frobenius invariants, the count bounds of
Lemmas 5.2-5.3, Algorithm 1's exact identity Theta = sum_k A_k B_k, and central finite
differences for the gradient.
"""
import math

import numpy as np
import pytest

import oracle
import pc_inputs as P


# ----------------------------------------------------------------- independent basis
def _periodised(taps, first, M):
    """vector of length M with taps[i] added at (first + i) mod M"""
    out = np.zeros(M)
    for i, t in enumerate(taps):
        out[(first + i) % M] += t
    return out


def _cascade_1d(h, n, L):
    """Matrix form of phi_{j,l} = sum_n h[n-2l] phi_{j-1,n}, psi_{j,l} = sum_n g[n-2l] phi_{j-1,n}
    (Section 2.1) on the circle of length n, starting from phi_{0,n} = Dirac at n.
    Returns (Phi_L, [Psi_1..Psi_L]) as n x n_j matrices of sampled basis vectors."""
    Lf = len(h)
    g = np.array([(-1) ** (1 - i) * h[1 - i] for i in range(2 - Lf, 2)])   # g on [2-Lf, 1]
    Phi = np.eye(n)
    Psis = []
    for j in range(1, L + 1):
        M = n >> (j - 1)
        Hm = np.stack([_periodised(h, 2 * l, M) for l in range(M // 2)], 1)
        Gm = np.stack([_periodised(g, 2 * l + 2 - Lf, M) for l in range(M // 2)], 1)
        Psis.append(Phi @ Gm)
        Phi = Phi @ Hm
    return Phi, Psis


def dense_psi(d, n, L, delta, family=0):
    """N x N matrix whose column lambda is psi_lambda, canonical order."""
    h = oracle.symmlet(delta) if family else oracle.daubechies(delta)
    Phi, Psis = _cascade_1d(h, n, L)
    if d == 1:
        return np.concatenate([Phi] + [Psis[j - 1] for j in range(L, 0, -1)], 1)
    cols = [np.kron(Phi, Phi)]
    for j in range(L, 0, -1):
        A, D = (Phi if j == L else None), Psis[j - 1]
        # phi at level j for the detail bands of level j
        Ph = _cascade_1d(h, n, j)[0]
        cols += [np.kron(Ph, D), np.kron(D, Ph), np.kron(D, D)]
    return np.concatenate(cols, 1)


def dense_H(op, u=None, v=None):
    """H[y, x] from Eq. (2): order 0: sum_k u_k(y-x) v_k(x); order 1: sum_k v_k(y) u_k(y-x)."""
    u = op.u if u is None else u
    v = op.v if v is None else v
    n, d, r, N = op.n, op.d, op.r, op.N
    K = 2 * r + 1
    H = np.zeros((N, N))
    for k in range(u.shape[0]):
        U = np.zeros((N, N))
        for t0 in (range(-r, r + 1) if d == 2 else [0]):
            for t1 in range(-r, r + 1):
                c = u[k, (t0 + r) * K + (t1 + r)] if d == 2 else u[k, t1 + r]
                if d == 1:
                    idx = np.arange(n)
                    U[(idx + t1) % n, idx] += c
                else:
                    x0, x1 = np.divmod(np.arange(N), n)
                    U[((x0 + t0) % n) * n + (x1 + t1) % n, np.arange(N)] += c
        V = np.diag(v[k])
        H += U @ V if op.order == 0 else V @ U
    return H


def tiny(d, n, L, delta, r, m, order=0, seed=0, gap=-1, family=0):
    N = n ** d
    K = (2 * r + 1) ** d
    u = P.normal(P.BASE_SEED + 100 + seed, m * K).reshape(m, K)
    v = P.uniform(P.BASE_SEED + 200 + seed, m * N).reshape(m, N) + 0.1
    return P.Operator("tiny", d, n, delta, L, r, u, v, gap=gap, order=order, family=family)


# ----------------------------------------------------------------- filter taps
def test_db2_closed_form():
    s = math.sqrt(3.0)
    ref = np.array([1 + s, 3 + s, 3 - s, 1 - s]) / (4 * math.sqrt(2.0))
    assert np.abs(oracle.daubechies(2) - ref).max() < 1e-15


def test_haar_is_db1():
    assert np.abs(oracle.daubechies(1) - [2 ** -0.5, 2 ** -0.5]).max() < 1e-16


@pytest.mark.parametrize("delta", [1, 2, 3, 4, 5, 6])
def test_taps_properties(delta):
    h = oracle.daubechies(delta)
    Lf = len(h)
    assert Lf == 2 * delta
    assert abs(h.sum() - math.sqrt(2)) < 1e-14
    for k in range(delta):
        s = sum(h[i] * h[i + 2 * k] for i in range(Lf - 2 * k))
        assert abs(s - (1.0 if k == 0 else 0.0)) < 1e-14
    # delta vanishing moments of the high-pass g[i] = (-1)^(1-i) h[1-i]
    for p in range(delta):
        mom = sum((-1) ** (1 - i) * h[1 - i] * float(i) ** p for i in range(2 - Lf, 2))
        assert abs(mom) < 1e-10 * (Lf ** p)
    # minimum phase: zeros of sum h[n] z^n other than z = -1 lie outside the unit circle
    q, rem = np.polydiv(h[::-1], np.poly1d([1.0, 1.0]) ** delta)   # divide out (1+z)^delta
    assert np.abs(rem).max() < 1e-12
    assert np.all(np.abs(np.roots(q)) > 1.0)


# ----------------------------------------------------------------- transforms
@pytest.mark.parametrize("d,n,L,delta", [(1, 64, 4, 2), (1, 32, 5, 4), (1, 16, 2, 3),
                                         (2, 16, 3, 2), (2, 16, 2, 4), (2, 8, 3, 4)])
def test_transform_is_independent_orthonormal_basis(d, n, L, delta):
    N = n ** d
    Psi = dense_psi(d, n, L, delta)
    assert np.abs(Psi.T @ Psi - np.eye(N)).max() < 1e-13
    rng = np.random.default_rng(1)
    f = rng.standard_normal(N)
    c = oracle.dwt(d, n, L, delta, f)
    assert np.abs(c - Psi.T @ f).max() < 1e-13
    assert np.abs(oracle.idwt(d, n, L, delta, c) - f).max() < 1e-13
    assert abs(np.dot(c, c) - np.dot(f, f)) < 1e-12 * np.dot(f, f)     # Parseval


def test_haar_textbook():
    x = np.random.default_rng(2).standard_normal(16)
    c = oracle.dwt(1, 16, 1, 1, x)
    a = (x[0::2] + x[1::2]) / math.sqrt(2)
    dd = (x[1::2] - x[0::2]) / math.sqrt(2)
    assert np.abs(c[:8] - a).max() < 1e-15 and np.abs(c[8:] - dd).max() < 1e-15


# ----------------------------------------------------------------- operator and Theta
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("d,n", [(1, 32), (2, 8)])
def test_pc_apply_dense(order, d, n):
    op = tiny(d, n, 2, 2, 2, 3, order=order)
    H = dense_H(op)
    f = np.random.default_rng(3).standard_normal(op.N)
    assert np.abs(oracle.pc_apply(op, f) - H @ f).max() < 1e-13


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("d,n,L,delta,r,m", [(1, 16, 2, 2, 2, 2), (1, 32, 3, 2, 3, 3), (1, 64, 4, 4, 4, 2),
                                             (2, 8, 2, 2, 1, 2), (2, 16, 2, 4, 2, 3), (2, 16, 3, 2, 2, 2)])
def test_theta_bruteforce(order, d, n, L, delta, r, m):
    op = tiny(d, n, L, delta, r, m, order=order)
    Psi = dense_psi(d, n, L, delta)
    Theta = Psi.T @ dense_H(op) @ Psi
    cols = np.arange(op.N)
    T = oracle.theta_columns(op, cols).T
    assert np.abs(T - Theta).max() < 1e-13 * max(1.0, np.abs(Theta).max())


def test_alg1_exact_identity():
    """Algorithm 1 without thresholding: sum_k A_k B_k = Theta, A_k = Psi^T U_k Psi,
    B_k = Psi^T V_k Psi (Section 3.2); and ||B_k||_2 = ||v_k||_inf (Lemma 5.9)."""
    op = tiny(2, 16, 2, 2, 2, 3)
    Psi = dense_psi(2, 16, 2, 2)
    T = oracle.theta_columns(op, np.arange(op.N)).T
    acc = np.zeros_like(T)
    for k in range(op.m):
        one_u = P.Operator("u", 2, 16, 2, 2, op.r, op.u[k:k + 1], np.ones((1, op.N)))
        one_v = P.Operator("v", 2, 16, 2, 2, 0, np.ones((1, 1)), op.v[k:k + 1])
        A = Psi.T @ dense_H(one_u) @ Psi
        B = Psi.T @ dense_H(one_v) @ Psi
        assert abs(np.linalg.norm(B, 2) - np.abs(op.v[k]).max()) < 1e-12
        acc += A @ B
    assert np.abs(acc - T).max() < 1e-12


@pytest.mark.parametrize("d,n,L,delta", [(1, 64, 4, 2), (2, 16, 3, 4)])
def test_identity_closed_form(d, n, L, delta):
    """one term, v = 1, u = Dirac  =>  Theta = I"""
    N = n ** d
    op = P.Operator("id", d, n, delta, L, 0, np.ones((1, 1)), np.ones((1, N)))
    T = oracle.theta_columns(op, np.arange(N)).T
    assert np.abs(T - np.eye(N)).max() < 1e-13


def test_multiplier_closed_form():
    """u = Dirac, general v  =>  Theta = B = Psi^T diag(v) Psi: symmetric, eigenvalues = v."""
    n, L, delta = 16, 2, 4
    v = P.uniform(P.BASE_SEED + 7, n * n).reshape(1, -1) * 3 - 1
    op = P.Operator("B", 2, n, delta, L, 0, np.ones((1, 1)), v)
    T = oracle.theta_columns(op, np.arange(n * n)).T
    assert np.abs(T - T.T).max() < 1e-13
    ev = np.sort(np.linalg.eigvalsh((T + T.T) / 2))
    assert np.abs(ev - np.sort(v[0])).max() < 1e-12


@pytest.mark.parametrize("d,n,L,delta", [(1, 64, 3, 2), (2, 16, 2, 4)])
def test_convolution_subbands_circulant(d, n, L, delta):
    """Constant window => convolution operator => sub-bands are circulant (Lemma 5.1):
    shifting both basis functions by 2^L pixels along any axis leaves Theta unchanged."""
    op = tiny(d, n, L, delta, 2, 1)
    op.v[:] = 1.7
    N = op.N
    T = oracle.theta_columns(op, np.arange(N)).T
    # permutation of the canonical index induced by a pixel shift of s = 2^L on axis 1
    s = 2 ** L
    e = np.zeros(N)
    perm = np.zeros(N, dtype=np.int64)
    for i in range(N):
        e[:] = 0
        e[i] = 1
        f = oracle.idwt(d, n, L, delta, e)
        fs = np.roll(f.reshape((n,) * d), s, axis=d - 1).reshape(-1)
        c = oracle.dwt(d, n, L, delta, fs)
        perm[i] = int(np.argmax(np.abs(c)))
        assert abs(c[perm[i]] - 1) < 1e-12
    assert sorted(perm) == list(range(N)) and np.any(perm != np.arange(N))
    assert np.abs(T[np.ix_(perm, perm)] - T).max() < 1e-13


def test_trace_and_frobenius_invariants():
    """Psi orthonormal => trace Theta = trace H = sum_k u_k(0) sum_x v_k(x) and
    ||Theta||_F^2 = ||H||_F^2 = sum_x sum_t (sum_k u_k(t) v_k(x))^2 (order 0, 2r+1 <= n)."""
    op = P.workload("c1")
    T = oracle.theta_columns(op, np.arange(op.N)).T
    r = op.r
    tr = sum(op.u[k, r] * op.v[k].sum() for k in range(op.m))
    assert abs(np.trace(T) - tr) < 1e-11 * abs(tr)
    fro = ((op.u.T @ op.v) ** 2).sum()
    assert abs((T ** 2).sum() - fro) < 1e-11 * fro


@pytest.mark.parametrize("d,n", [(1, 32), (2, 8)])
def test_order_flag_transpose(d, n):
    """v . (u * f) is the transpose of flip(u) * (v . f): Theta_1(u, v) = Theta_0(flip u, v)^T"""
    op1 = tiny(d, n, 2, 2, 2, 3, order=1)
    op0 = tiny(d, n, 2, 2, 2, 3, order=0)
    op0.u = op1.u[:, ::-1].copy()
    T1 = oracle.theta_columns(op1, np.arange(op1.N)).T
    T0 = oracle.theta_columns(op0, np.arange(op0.N)).T
    assert np.abs(T1 - T0.T).max() < 1e-14 * max(1, np.abs(T0).max()) * 10


# ----------------------------------------------------------------- pattern
@pytest.mark.parametrize("d,n,L,delta,r", [(1, 128, 4, 2, 3), (1, 64, 5, 4, 2), (2, 32, 3, 2, 2), (2, 16, 3, 4, 1)])
def test_pattern_contains_every_nonzero(d, n, L, delta, r):
    """With the band gap opened to L, the pattern's spatial rule keeps every entry that
    can be nonzero: entries it drops are exactly 0 in Theta."""
    op = tiny(d, n, L, delta, r, 2, gap=L)
    T = oracle.theta_columns(op, np.arange(op.N)).T
    for lam in range(op.N):
        mask = oracle.pattern_column(op, lam)
        assert np.all(T[~mask, lam] == 0.0), lam
    # the pattern is symmetric
    rng = np.random.default_rng(4)
    for mu, lam in rng.integers(0, op.N, (200, 2)):
        assert oracle.in_pattern(op, mu, lam) == oracle.in_pattern(op, lam, mu)


@pytest.mark.parametrize("d,n,delta", [(1, 256, 2), (1, 128, 4), (2, 32, 2), (2, 16, 3)])
def test_pattern_count_bounds(d, n, delta):
    """r = 0, no band limit, full depth: the pattern is the intersecting-support set I.
    Row counts obey Lemma 5.2 and the total obeys Lemma 5.3."""
    J = int(math.log2(n))
    op = P.Operator("I", d, n, delta, J, 0, np.ones((1, 1)), np.ones((1, n ** d)), gap=J)
    total = 0
    for lam in range(op.N):
        cnt = int(oracle.pattern_column(op, lam).sum())
        total += cnt
        # level of lam in the paper's numbering (j_paper = J - level); approximation -> 0
        if d == 1:
            jm = J if lam < 1 else J - int(math.floor(math.log2(lam)))
        else:
            jm = J if lam < 1 else J - int(math.floor(math.log2(lam) / 2))
        jp = J - jm
        assert cnt <= (2 * delta) ** d * ((2 ** d - 1) * jp + 2 ** (d * (J - jp))) + (2 * delta) ** d
    assert total <= 2 * (2 ** d - 1) * 2 ** d * delta ** d * J * 2 ** (d * J)


# ----------------------------------------------------------------- gradient
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("d,n,L,delta,r,m", [(1, 32, 3, 2, 2, 2), (2, 16, 2, 4, 1, 2)])
def test_gradient_finite_differences(order, d, n, L, delta, r, m):
    """L = 1/2 ||Theta_P - T||^2 is quadratic in each of u and v, so central differences
    are exact up to rounding."""
    op = tiny(d, n, L, delta, r, m, order=order, gap=1)
    cols = np.arange(op.N)
    mask = np.stack([oracle.pattern_column(op, c) for c in cols])          # (cols, N)
    tgt = P.normal(5, op.N * op.N).reshape(op.N, op.N)

    def loss(u, v):
        T = oracle.theta_columns(op, cols, u=u, v=v)
        return 0.5 * (((T - tgt) * mask) ** 2).sum()

    T = oracle.theta_columns(op, cols)
    G = (T - tgt) * mask
    du, dv = oracle.theta_grad(op, cols, G)
    rng = np.random.default_rng(6)
    h = 1e-6
    # quadratic loss: the central difference is exact up to rounding, |err| ~ eps * L / h
    tol = 50 * np.finfo(float).eps * loss(op.u, op.v) / h
    for _ in range(8):
        k = rng.integers(op.m)
        i = rng.integers(op.u.shape[1])
        up, um = op.u.copy(), op.u.copy()
        up[k, i] += h
        um[k, i] -= h
        fd = (loss(up, op.v) - loss(um, op.v)) / (2 * h)
        assert abs(fd - du[k, i]) <= tol + 1e-9 * abs(fd)
        i = rng.integers(op.N)
        vp, vm = op.v.copy(), op.v.copy()
        vp[k, i] += h
        vm[k, i] -= h
        fd = (loss(op.u, vp) - loss(op.u, vm)) / (2 * h)
        assert abs(fd - dv[k, i]) <= tol + 1e-9 * abs(fd)


def test_gradient_adjoint_identity():
    """<G, dTheta(du, dv)> = <du, dL/du> + <dv, dL/dv> for the linearisation (exact
    dot-product test: Theta is bilinear in (u, v))."""
    op = tiny(2, 16, 2, 2, 1, 2, gap=1)
    cols = np.arange(0, op.N, 3)
    G = P.normal(8, cols.size * op.N).reshape(cols.size, op.N)
    G *= np.stack([oracle.pattern_column(op, c) for c in cols])
    du, dv = oracle.theta_grad(op, cols, G)
    Du = P.normal(9, op.u.size).reshape(op.u.shape)
    Dv = P.normal(10, op.v.size).reshape(op.v.shape)
    # dTheta along (Du, 0) is Theta(Du, v); along (0, Dv) is Theta(u, Dv) (bilinearity)
    lhs = (G * oracle.theta_columns(op, cols, u=Du)).sum() + (G * oracle.theta_columns(op, cols, v=Dv)).sum()
    rhs = (du * Du).sum() + (dv * Dv).sum()
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))


def test_golden_c1_regression():
    """Stored oracle values for c1 (written by tests/golden/make_golden.py, oracle only)
    reproduce on this machine; the trace equals the closed form sum_k u_k(0) sum_x v_k(x)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "c1_theta_entries.txt")
    op = P.workload("c1")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    tr = float([l for l in open(path) if l.startswith("# trace")][0].split()[2])
    assert abs(tr - sum(op.u[k, op.r] * op.v[k].sum() for k in range(op.m))) < 1e-11 * tr
    lams = sorted({int(r[1]) for r in rows})
    T = dict(zip(lams, oracle.theta_columns(op, lams)))
    for mu, lam, val in rows:
        assert abs(T[int(lam)][int(mu)] - float(val)) <= 1e-14 + 1e-12 * abs(float(val))
