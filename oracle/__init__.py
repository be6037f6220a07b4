"""FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may
import this package.  It shares no code with the CUDA path.  The arithmetic lives in
pc_oracle.c (plain double-precision loops following the paper's Algorithm 2, the
definitions of Sections 1-3, the thresholded Algorithm 1, the Symmlet filters and the FISTA
iterations of the deblurring appendix); this file only compiles and calls it.  pc_svir.py
(numpy) holds the randomized-SVD construction of a product-convolution expansion.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_ubyte)


def build(force: bool = False) -> str:
    """Compile pc_oracle.c with gcc + OpenMP into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        I, D = ctypes.c_int, ctypes.c_int64
        lib.or_daubechies.argtypes = [I, _dp]
        lib.or_symmlet.argtypes = [I, _dp]
        lib.or_dwt.argtypes = [I, I, I, I, _dp, _dp]
        lib.or_idwt.argtypes = [I, I, I, I, _dp, _dp]
        lib.or_pc_apply.argtypes = [I, I, I, I, I, _dp, _dp, _dp, _dp]
        lib.or_theta_columns.argtypes = [I, I, I, I, I, I, I, _dp, _dp, D, _i64p, _dp, I]
        lib.or_in_pattern.argtypes = [I, I, I, I, I, I, D, D]
        lib.or_pattern_mask.argtypes = [I, I, I, I, I, I, D, _u8p]
        lib.or_theta_grad.argtypes = [I, I, I, I, I, I, I, _dp, _dp, D, _i64p, _dp, _dp, _dp, I]
        lib.or_max_threads.argtypes = []
        lib.or_jacobi.argtypes = [D, _dp, _dp]
        lib.or_power_norm.argtypes = [D, _dp, _dp, I, _dp]
        lib.or_fista.argtypes = [D, _dp, _dp, _dp, _dp, I, ctypes.c_double, _dp]
        lib.or_alg1_dense.argtypes = [I, I, I, I, I, I, I, _dp, _dp, ctypes.c_double, I, _dp, _i64p, _dp]
        _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _check(rc, what):
    if rc < 0:
        raise ValueError(f"oracle: {what} failed (rc={rc})")


def max_threads() -> int:
    return int(_load().or_max_threads())


def daubechies(delta: int) -> np.ndarray:
    """Low-pass taps h[0..2 delta - 1] (minimum phase, sum sqrt 2)."""
    h = np.zeros(64)
    rc = _load().or_daubechies(delta, h.ctypes.data_as(_dp))
    _check(rc, "daubechies")
    return h[:rc].copy()


def symmlet(delta: int) -> np.ndarray:
    """Low-pass taps h[0..2 delta - 1] of the least-asymmetric spectral factor (sum sqrt 2)."""
    h = np.zeros(64)
    rc = _load().or_symmlet(delta, h.ctypes.data_as(_dp))
    _check(rc, "symmlet")
    return h[:rc].copy()


def _wcode(delta, family=0):
    """The library's filter code: delta + 100 * family (0 Daubechies, 1 Symmlet)."""
    return int(delta) + 100 * int(family)


def _opcode(op):
    return _wcode(op.delta, getattr(op, "family", 0))


def dwt(d, n, L, delta, f, family=0):
    """Forward periodic transform Psi^* of pixels f (n^d, row-major) -> canonical coefficients."""
    f, fp = _d(np.asarray(f).reshape(-1))
    c = np.zeros(f.size)
    _check(_load().or_dwt(d, n, L, _wcode(delta, family), fp, c.ctypes.data_as(_dp)), "dwt")
    return c


def idwt(d, n, L, delta, c, family=0):
    """Inverse periodic transform Psi: canonical coefficients -> pixels."""
    c, cp = _d(np.asarray(c).reshape(-1))
    f = np.zeros(c.size)
    _check(_load().or_idwt(d, n, L, _wcode(delta, family), cp, f.ctypes.data_as(_dp)), "idwt")
    return f


def pc_apply(op, f, u=None, v=None):
    """H f for the operator (direct periodic convolution)."""
    u, up = _d(op.u if u is None else u)
    v, vp = _d(op.v if v is None else v)
    f, fp = _d(np.asarray(f).reshape(-1))
    w = np.zeros(op.N)
    _check(_load().or_pc_apply(op.d, op.n, u.shape[0], op.r, op.order, up, vp, fp,
                               w.ctypes.data_as(_dp)), "pc_apply")
    return w


def theta_columns(op, cols, u=None, v=None, nthreads: int = 0):
    """Columns Theta[:, cols] of Psi^* H Psi by Algorithm 2.  Returns (len(cols), N)."""
    u, up = _d(op.u if u is None else u)
    v, vp = _d(op.v if v is None else v)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.zeros((cols.size, op.N))
    rc = _load().or_theta_columns(op.d, op.n, op.levels, _opcode(op), u.shape[0], op.r, op.order,
                                  up, vp, cols.size, cols.ctypes.data_as(_i64p),
                                  out.ctypes.data_as(_dp), nthreads)
    _check(rc, "theta_columns")
    return out


def in_pattern(op, mu: int, lam: int) -> bool:
    return bool(_load().or_in_pattern(op.d, op.n, op.levels, _opcode(op), op.r, op.gap, int(mu), int(lam)))


def pattern_column(op, lam: int) -> np.ndarray:
    """Boolean mask over mu of the pattern entries (mu, lam)."""
    mask = np.zeros(op.N, dtype=np.uint8)
    _load().or_pattern_mask(op.d, op.n, op.levels, _opcode(op), op.r, op.gap, int(lam),
                            mask.ctypes.data_as(_u8p))
    return mask.astype(bool)


def theta_grad(op, cols, G, u=None, v=None, nthreads: int = 0):
    """(dL/du, dL/dv) for a loss whose gradient w.r.t. Theta[:, cols] is G (len(cols), N);
    G must already be zero outside the pattern."""
    u, up = _d(op.u if u is None else u)
    v, vp = _d(op.v if v is None else v)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    G, Gp = _d(G)
    du = np.zeros(u.shape)
    dv = np.zeros(v.shape)
    rc = _load().or_theta_grad(op.d, op.n, op.levels, _opcode(op), u.shape[0], op.r, op.order,
                               up, vp, cols.size, cols.ctypes.data_as(_i64p), Gp,
                               du.ctypes.data_as(_dp), dv.ctypes.data_as(_dp), nthreads)
    _check(rc, "theta_grad")
    return du, dv


def _opt(a):
    if a is None:
        return None, None
    return _d(np.asarray(a).reshape(-1))


def jacobi(T):
    """diag(Theta^T Theta) of a dense Theta (N, N): the FISTA-WP preconditioner."""
    T, Tp = _d(T)
    out = np.zeros(T.shape[0])
    _check(_load().or_jacobi(T.shape[0], Tp, out.ctypes.data_as(_dp)), "jacobi")
    return out


def power_norm(T, iters, sigma=None):
    """Power-iteration estimate of the largest eigenvalue of S^(1/2) Theta^T Theta S^(1/2)."""
    T, Tp = _d(T)
    _, sp = _opt(sigma)
    out = ctypes.c_double(0.0)
    _check(_load().or_power_norm(T.shape[0], Tp, sp, int(iters), ctypes.byref(out)), "power_norm")
    return out.value


def fista(T, z0, w, iters, tau, z_init=None, sigma=None):
    """FISTA-W (sigma None) / FISTA-WP iterates on the dense Theta; returns z^(iters)."""
    T, Tp = _d(T)
    N = T.shape[0]
    z0, z0p = _d(np.asarray(z0).reshape(-1))
    w, wp = _d(np.asarray(w).reshape(-1))
    _, sp = _opt(sigma)
    z = np.zeros(N) if z_init is None else np.array(z_init, dtype=np.float64).reshape(-1)
    _check(_load().or_fista(N, Tp, z0p, wp, sp, int(iters), float(tau), z.ctypes.data_as(_dp)), "fista")
    return z


def alg1_dense(op, eta, u=None, v=None, rule=0):
    """Algorithm 1 with thresholding on dense matrices (N <= 4096): returns (Theta~ (N, N),
    entries kept per A~_k, threshold per k).  rule 0: the Schur-certified threshold; rule 1:
    tau_k = eps_k."""
    u, up = _d(op.u if u is None else u)
    v, vp = _d(op.v if v is None else v)
    N = op.N
    T = np.zeros((N, N))
    nnz = np.zeros(u.shape[0], dtype=np.int64)
    tau = np.zeros(u.shape[0])
    rc = _load().or_alg1_dense(op.d, op.n, op.levels, _opcode(op), u.shape[0], op.r, op.order, up, vp, float(eta),
                               int(rule), T.ctypes.data_as(_dp), nnz.ctypes.data_as(_i64p), tau.ctypes.data_as(_dp))
    _check(rc, "alg1_dense")
    return T, nnz, tau
