"""Pins of the oracle's Symmlet filters (the least-asymmetric spectral factors; Section 4.3 uses
the Symmlet basis of order 6) against facts that do not come from the oracle: the filter-bank
conditions of Section 2.1, the shared power response |m0|^2 with Daubechies' filter, a brute
force over every real spectral factor with numpy's root finder, the known equalities for orders
1-3, and the basis built by the independent cascade matrices of test_oracle_pins."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import dense_H, dense_psi, tiny

K = 512


def _phase_residual(roots):
    """Mean squared residual of the least-squares line through the unwrapped phase of
    prod (e^{-iw} - z) on the midpoint grid of [0, pi]."""
    w = (np.arange(K) + 0.5) * np.pi / K
    ph = np.zeros(K)
    for z in roots:
        ph += np.unwrap(np.angle(np.exp(-1j * w) - z))
    A = np.stack([np.ones(K), w], 1)
    coef, *_ = np.linalg.lstsq(A, ph, rcond=None)
    return float(np.mean((ph - A @ coef) ** 2))


def _factors(delta):
    """Every real spectral factor of Daubechies' P (one root of each reciprocal pair per root of
    P, conjugate roots of P choosing alike): list of (taps, residual)."""
    P = [math.comb(delta - 1 + k, k) for k in range(delta)]
    ys = np.roots(P[::-1]) if delta > 1 else np.array([])
    groups = []
    used = set()
    for i, y in enumerate(ys):
        if i in used:
            continue
        if abs(y.imag) < 1e-9:
            groups.append([i])
        else:
            j = min((k for k in range(len(ys)) if k != i and k not in used), key=lambda k: abs(ys[k] - np.conj(y)))
            groups.append([i, j])
            used.add(j)
        used.add(i)
    out = []
    for mask in range(1 << len(groups)):
        roots = []
        for g, grp in enumerate(groups):
            for i in grp:
                b = 2 - 4 * ys[i]
                z = (b + np.sqrt(b * b - 4 + 0j)) / 2
                if abs(z) < 1:
                    z = 1 / z
                roots.append(1 / z if (mask >> g) & 1 else z)
        poly = np.poly1d([1.0])
        for _ in range(delta):
            poly = poly * np.poly1d([1.0, 1.0])
        for z in roots:
            poly = poly * np.poly1d([1.0, -z])
        h = np.real(poly.coeffs[::-1])          # h[n] is the coefficient of z^n
        h = h * math.sqrt(2) / h.sum()
        out.append((h, _phase_residual(roots)))
    return out


@pytest.mark.parametrize("delta", range(1, 11))
def test_filter_bank_conditions(delta):
    h = oracle.symmlet(delta)
    Lf = len(h)
    assert Lf == 2 * delta
    assert abs(h.sum() - math.sqrt(2)) < 1e-13
    for k in range(delta):
        s = sum(h[i] * h[i + 2 * k] for i in range(Lf - 2 * k))
        assert abs(s - (1.0 if k == 0 else 0.0)) < 1e-13
    for p in range(delta):
        mom = sum((-1) ** (1 - i) * h[1 - i] * float(i) ** p for i in range(2 - Lf, 2))
        assert abs(mom) < 1e-9 * (Lf ** p)
    # the same power response as Daubechies' filter of the same order
    w = np.linspace(0, np.pi, 301)
    E = np.exp(-1j * np.outer(w, np.arange(Lf)))
    assert np.abs(np.abs(E @ h) - np.abs(E @ oracle.daubechies(delta))).max() < 1e-12


@pytest.mark.parametrize("delta", range(2, 9))
def test_least_asymmetric_among_all_factors(delta):
    h = oracle.symmlet(delta)
    cands = _factors(delta)
    best = min(r for _, r in cands)
    # the oracle's taps are one of the factors, with the smallest residual ...
    match = [r for t, r in cands if np.abs(t - h).max() < 1e-9]
    assert len(match) == 1, "not a spectral factor of P"
    assert match[0] <= best * (1 + 1e-9) + 1e-15
    # ... and of the tied ones (a factor and its mirror) the one with the smaller energy centre
    tied = [t for t, r in cands if abs(r - best) <= 1e-9 * best + 1e-15]
    centre = lambda t: float(np.sum(np.arange(len(t)) * t * t))
    assert centre(h) <= min(centre(t) for t in tied) + 1e-12


@pytest.mark.parametrize("delta", [1, 2, 3])
def test_low_orders_equal_daubechies(delta):
    # orders 1-3 have at most one choice besides the mirror, and the least-asymmetric one is
    # the minimum-phase filter itself
    assert np.abs(oracle.symmlet(delta) - oracle.daubechies(delta)).max() < 1e-12


def test_symmlets_differ_from_daubechies_and_are_centred():
    for delta in (4, 5, 6, 8):
        h, hd = oracle.symmlet(delta), oracle.daubechies(delta)
        assert np.abs(h - hd).max() > 1e-3
        c = lambda t: float(np.sum(np.arange(len(t)) * t * t))
        # closer to the middle of the support than the minimum-phase filter
        mid = (2 * delta - 1) / 2
        assert abs(c(h) - mid) < abs(c(hd) - mid)


@pytest.mark.parametrize("d,n,L,delta", [(1, 64, 3, 6), (1, 32, 2, 4), (2, 16, 1, 6), (2, 32, 2, 4)])
def test_symmlet_transform_is_independent_orthonormal_basis(d, n, L, delta):
    N = n ** d
    Psi = dense_psi(d, n, L, delta, family=1)
    assert np.abs(Psi.T @ Psi - np.eye(N)).max() < 1e-12
    f = np.random.default_rng(5).standard_normal(N)
    c = oracle.dwt(d, n, L, delta, f, family=1)
    assert np.abs(c - Psi.T @ f).max() < 1e-12
    assert np.abs(oracle.idwt(d, n, L, delta, c, family=1) - f).max() < 1e-12


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("d,n,L,delta,r,m", [(1, 32, 2, 6, 3, 2), (1, 64, 3, 4, 2, 3), (2, 16, 2, 4, 1, 2)])
def test_symmlet_theta_bruteforce(order, d, n, L, delta, r, m):
    op = tiny(d, n, L, delta, r, m, order=order, family=1)
    Psi = dense_psi(d, n, L, delta, family=1)
    Theta = Psi.T @ dense_H(op) @ Psi
    T = oracle.theta_columns(op, np.arange(op.N)).T
    assert np.abs(T - Theta).max() < 1e-12 * max(1.0, np.abs(Theta).max())
