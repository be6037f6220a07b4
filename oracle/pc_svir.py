"""FP64 oracle for building a product-convolution expansion from a space-varying impulse
response (SVIR) by randomized SVD (the construction of Section 2.4, "singular value
decomposition", citing Halko, Martinsson and Tropp).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
reference leg may import it.  Plain numpy; numpy's QR and SVD serve as steps.

Conventions (paper order, H f = sum_k u_k * (v_k . f)):
  the SVIR is S[x, t] = impulse response of a source at pixel x, at offset t (row-major
  (2r+1)^d stencil, centre = offset 0), so (H f)(x + t) = sum_x f(x) S[x, t] on the torus,
  and a PC expansion is the rank-m factorisation S[x, t] = sum_k v_k(x) u_k(t).
"""
from __future__ import annotations

import numpy as np


def svir_of_pc(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """S = sum_k v_k u_k^T (N x K) of a product-convolution expansion (u: m x K, v: m x N)."""
    return np.asarray(v, dtype=np.float64).T @ np.asarray(u, dtype=np.float64)


def apply_svir(S: np.ndarray, f: np.ndarray, d: int, n: int, r: int) -> np.ndarray:
    """(H f)(y) = sum_x f(x) S[x, y - x] by its definition, on the periodic grid."""
    N = n ** d
    f = np.asarray(f, dtype=np.float64).reshape(N)
    out = np.zeros(N)
    offs = [(0, t1) for t1 in range(-r, r + 1)] if d == 1 else \
        [(t0, t1) for t0 in range(-r, r + 1) for t1 in range(-r, r + 1)]
    for i, (t0, t1) in enumerate(offs):
        if d == 1:
            idx = (np.arange(n) + t1) % n
        else:
            x0, x1 = np.divmod(np.arange(N), n)
            idx = ((x0 + t0) % n) * n + (x1 + t1) % n
        np.add.at(out, idx, f * S[:, i])
    return out


def randomized_pc(S: np.ndarray, m: int, omega: np.ndarray, power_iters: int = 2):
    """Rank-m expansion of the SVIR by randomized SVD: Y = S Omega, Q an orthonormal basis of
    its range refined by power iterations (S S^T)^q with re-orthonormalisation, B = Q^T S,
    B = U~ diag(s) W^T, then v_k = s_k (Q U~)[:, k] and u_k = W[:, k].
    omega: K x (m + p) test matrix (the random numbers, passed in).  Returns (u (m x K),
    v (m x N), s (the m + p singular values of B))."""
    S = np.asarray(S, dtype=np.float64)
    Q, _ = np.linalg.qr(S @ omega)
    for _ in range(power_iters):
        Z, _ = np.linalg.qr(S.T @ Q)
        Q, _ = np.linalg.qr(S @ Z)
    B = Q.T @ S
    Ut, s, Wt = np.linalg.svd(B, full_matrices=False)
    V = (Q @ Ut[:, :m]) * s[:m][None, :]
    return Wt[:m].copy(), V.T.copy(), s


def svir_space_varying_gaussian(d: int, n: int, r: int, sigma_of_x) -> np.ndarray:
    """SVIR of a blur whose impulse response at source x is a normalised Gaussian of standard
    deviation sigma_of_x(x0, x1) (x in [0, 1)^d), truncated to the (2r+1)^d stencil."""
    N = n ** d
    t = np.arange(-r, r + 1, dtype=np.float64)
    S = np.zeros((N, (2 * r + 1) ** d))
    for x in range(N):
        x0, x1 = divmod(x, n) if d == 2 else (0, x)
        s = float(sigma_of_x(x0 / n, x1 / n))
        g1 = np.exp(-0.5 * (t / s) ** 2)
        k = np.outer(g1, g1).reshape(-1) if d == 2 else g1
        S[x] = k / k.sum()
    return S
