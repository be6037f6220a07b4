"""Pins of the oracle's thresholded Algorithm 1 (Section 3.2; the guarantee of Theorem 3.1,
||Theta - Theta~||_2 <= eta) against facts outside the oracle: the brute-force Theta from dense
H and the independent cascade basis, numpy's spectral norm, and the threshold certificate
recomputed from A_k = Psi^T U_k Psi built with dense matrices."""
import numpy as np
import pytest

import oracle
import pc_inputs as P
from test_oracle_pins import dense_H, dense_psi, tiny


def _schur(D):
    return float(np.sqrt(np.abs(D).sum(0).max() * np.abs(D).sum(1).max()))


def _smooth(d, n, L, delta, r, m, order=0):
    """Gaussian kernels on hat windows (the smooth operators the algorithm is made for)."""
    g = int(round(m ** (1.0 / d)))
    u = np.stack([P.gaussian_kernel(d, r, 0.8 + 0.6 * k).reshape(-1) for k in range(g ** d)])
    v = P.hat_windows(d, n, g)
    return P.Operator("smooth", d, n, delta, L, r, u, v, gap=-1, order=order)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("d,n,L,delta,r,m", [(1, 64, 4, 4, 3, 3), (2, 16, 2, 2, 1, 2), (1, 32, 3, 2, 2, 2)])
def test_eta_zero_is_the_exact_matrix(order, d, n, L, delta, r, m):
    op = tiny(d, n, L, delta, r, m, order=order)
    Psi = dense_psi(d, n, L, delta)
    Theta = Psi.T @ dense_H(op) @ Psi
    T, nnz, tau = oracle.alg1_dense(op, 0.0)
    assert np.abs(T - Theta).max() < 1e-12 * max(1.0, np.abs(Theta).max())


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("make", ["tiny", "smooth"])
def test_spectral_error_within_eta(order, make):
    if make == "tiny":
        op = tiny(1, 64, 4, 4, 3, 3, order=order)
    else:
        op = _smooth(1, 128, 5, 4, 6, 4, order=order)
    Psi = dense_psi(op.d, op.n, op.levels, op.delta)
    Theta = Psi.T @ dense_H(op) @ Psi
    prev_nnz = None
    prev_tau = None
    for eta in (1e-5, 1e-4, 1e-3, 1e-2, 1e-1, 1.0):
        T, nnz, tau = oracle.alg1_dense(op, eta)
        assert np.linalg.norm(Theta - T, 2) <= eta * (1 + 1e-9), eta
        if prev_nnz is not None:               # larger eta: thresholds grow, fewer entries kept
            assert np.all(nnz <= prev_nnz) and np.all(tau >= prev_tau)
        prev_nnz, prev_tau = nnz, tau
    assert prev_nnz.sum() < 0.5 * op.m * op.N ** 2   # the thresholds do discard


def test_threshold_certificate_and_maximality():
    # tau_k is the largest threshold whose discarded part of A_k has Schur bound <= eta/(m ||v_k||)
    op = tiny(1, 64, 4, 4, 3, 3)
    Psi = dense_psi(1, 64, 4, 4)
    N, K = op.N, 2 * op.r + 1
    eta = 3e-3
    _, nnz, tau = oracle.alg1_dense(op, eta)
    for k in range(op.m):
        U = np.zeros((N, N))
        for t in range(-op.r, op.r + 1):
            U[(np.arange(N) + t) % N, np.arange(N)] += op.u[k, t + op.r]
        A = Psi.T @ U @ Psi
        eps = eta / (op.m * np.abs(op.v[k]).max())
        # (the bisection ends next to an entry's magnitude: entries within 1e-9 of tau may go
        # either way between this A and the oracle's, which differ by rounding)
        D = np.where(np.abs(A) < tau[k] * (1 - 1e-9), A, 0.0)
        assert _schur(D) <= eps * (1 + 1e-9)
        D2 = np.where(np.abs(A) < tau[k] * (1 + 1e-6), A, 0.0)
        assert _schur(D2) > eps or np.count_nonzero(D2) == np.count_nonzero(A)
        assert np.count_nonzero(np.abs(A) >= tau[k] * (1 + 1e-9)) <= nnz[k] <= np.count_nonzero(np.abs(A) >= tau[k] * (1 - 1e-9))


def test_large_eta_discards_everything():
    op = tiny(1, 32, 3, 2, 2, 2)
    Psi = dense_psi(1, 32, 3, 2)
    Theta = Psi.T @ dense_H(op) @ Psi
    eta = 1e3
    T, nnz, _ = oracle.alg1_dense(op, eta)
    assert np.all(nnz == 0) and np.all(T == 0.0)
    assert np.linalg.norm(Theta, 2) <= eta


@pytest.mark.parametrize("make", ["tiny", "smooth"])
def test_hard_rule_is_a_plain_cut(make):
    """Rule 1 (tau_k = eps_k): the kept entries are exactly those of A_k = Psi^T U_k Psi (dense,
    from the independent cascade basis) with |a| >= eps_k, and Theta~ = sum_k A~_k B_k with
    B_k = Psi^T diag(v_k) Psi, both orders."""
    for order in (0, 1):
        op = tiny(1, 64, 4, 4, 3, 3, order=order) if make == "tiny" else _smooth(1, 128, 5, 4, 6, 4, order=order)
        Psi = dense_psi(op.d, op.n, op.levels, op.delta)
        N, K = op.N, 2 * op.r + 1
        eta = 2e-3
        T, nnz, tau = oracle.alg1_dense(op, eta, rule=1)
        ref = np.zeros((N, N))
        for k in range(op.m):
            U = np.zeros((N, N))
            for t in range(-op.r, op.r + 1):
                U[(np.arange(N) + t) % N, np.arange(N)] += op.u[k, t + op.r]
            A = Psi.T @ U @ Psi
            B = Psi.T @ np.diag(op.v[k]) @ Psi
            eps = eta / (op.m * np.abs(op.v[k]).max())
            assert tau[k] == eps
            # entries within rounding of eps may go either way between this A and the oracle's
            assert np.count_nonzero(np.abs(A) >= eps * (1 + 1e-9)) <= nnz[k] <= np.count_nonzero(np.abs(A) >= eps * (1 - 1e-9))
            At = np.where(np.abs(A) >= eps, A, 0.0)
            assert np.abs(A - At).max() < eps
            assert nnz[k] < np.count_nonzero(np.abs(A) > 1e-14 * np.abs(A).max())   # the cut drops entries
            ref += At @ B if order == 0 else B @ At
        assert np.abs(T - ref).max() < 1e-12 * np.abs(ref).max()
