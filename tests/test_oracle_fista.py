"""Pins of the oracle's wavelet-domain deblurring solver (Section 4.3 and the FISTA-W /
FISTA-WP iterations of the appendix on deblurring algorithms) against facts that do not come
from the oracle itself: closed-form minimisers, the optimality conditions of the l1 problem,
library eigenvalues and the known O(1/k^2) objective bound of the accelerated method."""
import numpy as np
import pytest

import oracle


def soft(a, t):
    return np.sign(a) * np.maximum(np.abs(a) - t, 0.0)


def objective(T, z0, w, z):
    return 0.5 * float(np.sum((T @ z - z0) ** 2)) + float(np.sum(w * np.abs(z)))


def kkt_residual(T, z0, w, z):
    """Max violation of 0 in Theta^T (Theta z - z0) + w sign(z) (subdifferential at z)."""
    g = T.T @ (z0 - T @ z)
    on = z != 0
    r_on = np.abs(g[on] - w[on] * np.sign(z[on]))
    r_off = np.maximum(np.abs(g[~on]) - w[~on], 0.0)
    return max(float(r_on.max(initial=0.0)), float(r_off.max(initial=0.0)))


def nonsym(N, seed):
    rng = np.random.default_rng(seed)
    return np.eye(N) + 0.35 * rng.standard_normal((N, N)) / np.sqrt(N)


def test_identity_operator_is_one_soft_threshold():
    rng = np.random.default_rng(1)
    N = 37
    z0 = rng.standard_normal(N)
    w = rng.uniform(0.0, 0.8, N)
    for iters in (1, 2, 7):
        z = oracle.fista(np.eye(N), z0, w, iters, 1.0, z_init=rng.standard_normal(N))
        np.testing.assert_allclose(z, soft(z0, w), rtol=0, atol=1e-15)


def test_diagonal_operator_closed_form():
    # min 1/2 (d z - b)^2 + w |z| per entry: z = soft(d b, w) / d^2
    rng = np.random.default_rng(2)
    N = 40
    d = rng.uniform(0.5, 2.0, N)
    b = rng.standard_normal(N)
    w = rng.uniform(0.0, 0.6, N)
    tau = 1.0 / float(np.max(d * d))
    z = oracle.fista(np.diag(d), b, w, 3000, tau)
    np.testing.assert_allclose(z, soft(d * b, w) / (d * d), rtol=0, atol=1e-9)


@pytest.mark.parametrize("precond", [False, True])
def test_nonsymmetric_operator_meets_optimality(precond):
    # A transposed operand in the gradient (Theta y instead of Theta^T) changes the limit.
    N = 30
    T = nonsym(N, 3)
    rng = np.random.default_rng(4)
    z0 = rng.standard_normal(N)
    w = rng.uniform(0.05, 0.4, N)
    sigma = 1.0 / oracle.jacobi(T) if precond else None
    S = np.ones(N) if sigma is None else sigma
    M = np.sqrt(S)[:, None] * (T.T @ T) * np.sqrt(S)[None, :]
    tau = 1.0 / float(np.linalg.eigvalsh(M).max())
    z = oracle.fista(T, z0, w, 4000, tau, sigma=sigma)
    assert kkt_residual(T, z0, w, z) < 1e-9
    assert np.count_nonzero(z) < N          # the thresholds are active somewhere


def test_least_squares_limit_without_weights():
    N = 24
    T = nonsym(N, 5)
    z0 = np.random.default_rng(6).standard_normal(N)
    tau = 1.0 / float(np.linalg.norm(T, 2) ** 2)
    z = oracle.fista(T, z0, np.zeros(N), 4000, tau)
    np.testing.assert_allclose(z, np.linalg.solve(T, z0), rtol=0, atol=1e-9)


def test_objective_bound_and_acceleration():
    # Accelerated proximal gradient: F(z_k) - F* <= 2 ||z_init - z*||^2 / (tau (k + 1)^2); on an
    # ill-conditioned problem it is also far ahead of plain forward-backward (no momentum).
    N = 60
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    T = Q * np.logspace(0, -2, N)[None, :]
    z0 = rng.standard_normal(N)
    w = np.full(N, 0.01)
    tau = 1.0 / float(np.linalg.norm(T, 2) ** 2)
    zstar = oracle.fista(T, z0, w, 60000, tau)
    Fstar = objective(T, z0, w, zstar)
    R2 = float(np.sum(zstar ** 2))
    for k in (1, 2, 5, 10, 50, 200, 1000):
        gap = objective(T, z0, w, oracle.fista(T, z0, w, k, tau)) - Fstar
        assert gap <= 2.0 * R2 / (tau * (k + 1) ** 2) + 1e-12, k
    # plain forward-backward for comparison, written from the prox-gradient definition
    z = np.zeros(N)
    for _ in range(200):
        z = soft(z - tau * (T.T @ (T @ z - z0)), tau * w)
    assert objective(T, z0, w, oracle.fista(T, z0, w, 200, tau)) - Fstar < 0.5 * (objective(T, z0, w, z) - Fstar)


def test_power_norm_and_jacobi_against_library():
    N = 50
    T = nonsym(N, 8)
    est = oracle.power_norm(T, 500)
    true = float(np.linalg.norm(T, 2) ** 2)
    assert est <= true * (1 + 1e-12)
    assert abs(est - true) < 1e-8 * true
    for k in (1, 3, 10):                    # never above the eigenvalue, from the first iteration
        assert oracle.power_norm(T, k) <= true * (1 + 1e-12)
    J = oracle.jacobi(T)
    np.testing.assert_allclose(J, np.diag(T.T @ T), rtol=1e-13, atol=0)
    assert abs(J.sum() - np.linalg.norm(T, "fro") ** 2) < 1e-10
    sigma = 1.0 / J
    M = np.sqrt(sigma)[:, None] * (T.T @ T) * np.sqrt(sigma)[None, :]
    lam = float(np.linalg.eigvalsh(M).max())
    assert abs(oracle.power_norm(T, 500, sigma=sigma) - lam) < 1e-8 * lam


def test_first_momentum_weight_is_zero():
    # (i - 1)/(i + 2) vanishes at i = 1, so two accelerated iterations equal two plain
    # forward-backward steps; from the third on they differ.
    N = 32
    T = nonsym(N, 9)
    rng = np.random.default_rng(10)
    z0 = rng.standard_normal(N)
    w = rng.uniform(0.0, 0.3, N)
    zi = rng.standard_normal(N)
    tau = 0.9 / float(np.linalg.norm(T, 2) ** 2)
    z = zi.copy()
    fb = []
    for _ in range(3):
        z = soft(z - tau * (T.T @ (T @ z - z0)), tau * w)
        fb.append(z.copy())
    np.testing.assert_allclose(oracle.fista(T, z0, w, 1, tau, z_init=zi), fb[0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle.fista(T, z0, w, 2, tau, z_init=zi), fb[1], rtol=0, atol=1e-13)
    assert np.abs(oracle.fista(T, z0, w, 3, tau, z_init=zi) - fb[2]).max() > 1e-6
