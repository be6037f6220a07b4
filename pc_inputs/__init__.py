"""Seeded synthetic inputs for product-convolution operators.

An operator is H f = sum_k u_k * (v_k . f) (paper order, Eq. (2), Section 1) or
H f = sum_k v_k . (u_k * f) (convolution first).  This module only *draws inputs*:
a counter-based PRNG, blur kernels u_k, multiplier windows v_k and the table of
workloads.  It holds no part of the method's arithmetic (no wavelet transform, no
product-convolution evaluation) and is the only module shared by the FP64 oracle
tests and the GPU path.

Stand-in for the paper's workloads (Section 4.1): the paper blurs a 1024^2 confocal
image with two measured space-varying blurs (Gaussian impulse responses with sigma
growing along one axis, supports up to 19x19 and 25x25, m = 5 and 25).  Those
operators are not available; the workloads below are synthetic operators of the same
kind (Gaussian / motion blurs, supports 5x5..31x31, partition-of-unity hat windows,
images 64^2..1024^2), drawn from fixed seeds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "splitmix64", "uniform", "normal", "gaussian_kernel", "motion_kernel",
    "hat_windows", "Operator", "workload", "batch_workload", "BASE_SEED",
]

BASE_SEED = 200509870
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): output i is the
    finaliser applied to seed + (offset+i+1)*0x9E3779B97F4A7C15 (mod 2^64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of uniforms."""
    npair = (count + 1) // 2
    u = uniform(seed, 2 * npair, 2 * offset)
    u1 = 1.0 - u[0::2]                      # in (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npair)
    z[0::2] = rad * np.cos(2.0 * math.pi * u2)
    z[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return z[:count]


def gaussian_kernel(d: int, r: int, sigma: float) -> np.ndarray:
    """Grid-sampled exp(-|t|^2 / 2 sigma^2) on [-r, r]^d, normalised to sum 1 after
    truncation.  Returned shape (2r+1,)*d; index r is offset 0."""
    t = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-(t * t) / (2.0 * sigma * sigma))
    if d == 2:
        g = np.outer(g, g)
    return g / g.sum()


def motion_kernel(r: int, length: float, theta: float) -> np.ndarray:
    """Linear motion blur: a centred segment of the given length at angle theta,
    rasterised with 4*length sub-samples splatted bilinearly on a (2r+1)^2 grid
    (axis 0 = rows), then normalised to sum 1.  Samples outside the grid are dropped."""
    k = np.zeros((2 * r + 1, 2 * r + 1))
    ns = max(1, int(round(4 * length)))
    for s in range(ns):
        a = (s + 0.5) / ns - 0.5
        p0 = r + a * length * math.sin(theta)
        p1 = r + a * length * math.cos(theta)
        i0, i1 = int(math.floor(p0)), int(math.floor(p1))
        f0, f1 = p0 - i0, p1 - i1
        for di, wi in ((0, 1.0 - f0), (1, f0)):
            for dj, wj in ((0, 1.0 - f1), (1, f1)):
                y, x = i0 + di, i1 + dj
                if 0 <= y <= 2 * r and 0 <= x <= 2 * r:
                    k[y, x] += wi * wj
    return k / k.sum()


def skewed_gaussian(r: int, s_long: float, s_short: float, theta: float, skew: float) -> np.ndarray:
    """(2r+1)^2 stencil of an anisotropic Gaussian: standard deviations s_long along the
    direction theta and s_short across it, skewed along the long axis by the factor
    (1 + skew * tanh(t / s_long)) (t the coordinate along theta); normalised to sum 1."""
    y0, y1 = np.mgrid[-r:r + 1, -r:r + 1].astype(np.float64)
    t = math.cos(theta) * y1 + math.sin(theta) * y0
    q = -math.sin(theta) * y1 + math.cos(theta) * y0
    k = np.exp(-0.5 * ((t / s_long) ** 2 + (q / s_short) ** 2)) * (1.0 + skew * np.tanh(t / s_long))
    return k / k.sum()


def _conv2_same(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Full 2-D convolution of two centred odd-size kernels, cropped back to a's size."""
    ra, rb = a.shape[0] // 2, b.shape[0] // 2
    out = np.zeros((a.shape[0] + 2 * rb, a.shape[1] + 2 * rb))
    for i in range(b.shape[0]):
        for j in range(b.shape[1]):
            out[i:i + a.shape[0], j:j + a.shape[1]] += b[i, j] * a
    return out[rb:rb + 2 * ra + 1, rb:rb + 2 * ra + 1]


def hat_windows(d: int, n: int, g: int) -> np.ndarray:
    """Piecewise-linear hats on the periodic grid of side n: g nodes per axis at
    c_i = i*n/g and v_i(x) = max(0, 1 - circdist(x, c_i) / (n/g)).  In 2-D the
    windows are tensor products (bilinear), ordered row-major over the node grid.
    The windows sum to 1 at every pixel (partition of unity).  Shape (g^d, n^d)."""
    x = np.arange(n, dtype=np.float64)
    h = n / g
    w1 = np.empty((g, n))
    for i in range(g):
        dist = np.abs(x - i * h)
        dist = np.minimum(dist, n - dist)
        w1[i] = np.maximum(0.0, 1.0 - dist / h)
    if d == 1:
        return w1
    return np.einsum("ia,jb->ijab", w1, w1).reshape(g * g, n * n)


@dataclass
class Operator:
    """One product-convolution operator and its wavelet-matrix settings.

    u: (m, (2r+1)^d) kernels, row-major stencil, centre index = offset 0.
    v: (m, n^d) windows, row-major pixels (axis 0 slow).
    delta: wavelet order (number of vanishing moments; 2*delta taps).
    family: 0 = Daubechies (minimum phase), 1 = Symmlet (least asymmetric), same support.
    levels: number of decomposition levels L (level 1 finest, L coarsest).
    gap: keep entries with | |mu| - |lambda| | <= gap; -1 keeps every entry.
    order: 0 = u_k * (v_k . f) (paper), 1 = v_k . (u_k * f).
    """
    name: str
    d: int
    n: int
    delta: int
    levels: int
    r: int
    u: np.ndarray
    v: np.ndarray
    gap: int = 2
    order: int = 0
    extra: dict = field(default_factory=dict)
    family: int = 0

    @property
    def m(self) -> int:
        return self.u.shape[0]

    @property
    def N(self) -> int:
        return self.n ** self.d


def _stack(kernels, d):
    return np.stack([k.reshape(-1) for k in kernels]).astype(np.float64)


def workload(name: str, seed_offset: int = 0, **over) -> Operator:
    """The named synthetic workloads.

    c1  1-D n=256, db2, L=5, m=4 Gaussians sigma in {1,2,3,4} (radius 4 sigma, all
        padded to r=16), 4 hats; dense wavelet matrix.
    c2  2-D 256^2, db4, L=4, m=16 (4x4 bilinear hats), 15x15 Gaussians
        sigma_k = 0.5 + 2.5 k/15; pattern gap 2.
    c3  2-D 128^2, db4, L=3, m=9 (3x3 hats), 11x11 kernels; 'u' is the learnable
        initialisation (Gaussian sigma=1.5 plus N(0,1e-2) noise), extra['u_target'] the
        target kernels (Gaussians sigma_k = 0.8 + 1.7 k/8).
    c5  2-D 1024^2, db4, L=5, m=64 (8x8 hats), 31x31 kernels = normalised
        Gaussian(sigma ~ U[0.5,4]) * motion(length ~ U{3..15}, angle ~ U[0,pi)).
    op1  stand-in for the paper's first blur (Section 4.1): isotropic Gaussians whose sigma
         grows along axis 0 only, sigma_k = 3 (k + 1/2) / 5 px for the m = 5 windows (hats
         along axis 0, constant along axis 1), 19x19 stencils (r = 9); Symmlet 6, L = 4.
    op2  stand-in for the second blur: m = 25 (5x5 bilinear hats), 25x25 stencils (r = 12)
         of rotated, skewed Gaussians whose elongation grows with the distance of the window
         centre from the field centre and whose long axis points to it; Symmlet 6, L = 4.
    small-1d / small-2d  parity cases that span several tiles with a ragged tail.
    Keyword overrides replace fields (n, levels, ...) before the inputs are drawn.
    """
    seed = BASE_SEED + {"c1": 1, "c2": 2, "c3": 3, "c4": 4, "c5": 5}.get(name, 17) + 1000 * seed_offset
    if name == "c1":
        n = over.get("n", 256)
        sig = [1.0, 2.0, 3.0, 4.0]
        r = 16
        u = np.zeros((4, 2 * r + 1))
        for k, s in enumerate(sig):
            rk = int(math.ceil(4 * s))
            u[k, r - rk:r + rk + 1] = gaussian_kernel(1, rk, s)
        v = hat_windows(1, n, 4)
        return Operator("c1", 1, n, over.get("delta", 2), over.get("levels", 5), r, u, v,
                        gap=over.get("gap", -1), order=over.get("order", 0), family=over.get("family", 0))
    if name == "c2":
        n, g, r = over.get("n", 256), 4, over.get("r", 7)
        m = g * g
        u = _stack([gaussian_kernel(2, r, 0.5 + 2.5 * k / (m - 1)) for k in range(m)], 2)
        return Operator("c2", 2, n, over.get("delta", 4), over.get("levels", 4), r, u,
                        hat_windows(2, n, g), gap=over.get("gap", 2), order=over.get("order", 0), family=over.get("family", 0))
    if name == "c3":
        n, g, r = over.get("n", 128), 3, 5
        m = g * g
        noise = normal(seed, m * (2 * r + 1) ** 2).reshape(m, -1) * 1e-2
        base = gaussian_kernel(2, r, 1.5).reshape(-1)
        u = base[None, :] + noise
        ut = _stack([gaussian_kernel(2, r, 0.8 + 1.7 * k / (m - 1)) for k in range(m)], 2)
        return Operator("c3", 2, n, over.get("delta", 4), over.get("levels", 3), r, u,
                        hat_windows(2, n, g), gap=over.get("gap", 2), order=over.get("order", 0),
                        extra={"u_target": ut}, family=over.get("family", 0))
    if name == "c5":
        n, g, r = over.get("n", 1024), 8, 15
        m = g * g
        un = uniform(seed, 4 * m).reshape(m, 4)
        ks = []
        for k in range(m):
            sigma = 0.5 + 3.5 * un[k, 0]
            length = 3 + int(un[k, 1] * 13)          # U{3..15}
            theta = math.pi * un[k, 2]
            ks.append(_conv2_same(motion_kernel(r, length, theta), gaussian_kernel(2, r, sigma)))
        u = _stack([k / k.sum() for k in ks], 2)
        return Operator("c5", 2, n, over.get("delta", 4), over.get("levels", 5), r, u,
                        hat_windows(2, n, g), gap=over.get("gap", 2), order=over.get("order", 0), family=over.get("family", 0))
    if name == "op1":
        n, g, r = over.get("n", 256), 5, over.get("r", 9)
        u = _stack([gaussian_kernel(2, r, 3.0 * (k + 0.5) / g) for k in range(g)], 2)
        w1 = hat_windows(1, n, g)
        v = np.repeat(w1, n, axis=1)             # v_k(y0, y1) = hat_k(y0)
        return Operator("op1", 2, n, over.get("delta", 6), over.get("levels", 4), r, u, v,
                        gap=over.get("gap", 2), order=over.get("order", 0), family=over.get("family", 1))
    if name == "op2":
        n, g, r = over.get("n", 256), 5, over.get("r", 12)
        ks = []
        for i in range(g):
            for j in range(g):
                c0, c1 = (i + 0.5) / g - 0.5, (j + 0.5) / g - 0.5     # window centre - field centre
                rho = math.hypot(c0, c1) / math.hypot(0.5, 0.5)
                ks.append(skewed_gaussian(r, 1.0 + 3.0 * rho, 1.0, math.atan2(c0, c1), 0.4 * rho))
        u = _stack(ks, 2)
        return Operator("op2", 2, n, over.get("delta", 6), over.get("levels", 4), r, u,
                        hat_windows(2, n, g), gap=over.get("gap", 2), order=over.get("order", 0),
                        family=over.get("family", 1))
    if name in ("small-1d", "small-2d"):
        d = 1 if name == "small-1d" else 2
        n = over.get("n", 512 if d == 1 else 64)
        r = over.get("r", 5 if d == 1 else 3)
        g = over.get("g", 5 if d == 1 else 3)
        m = g ** d
        un = uniform(seed, m)
        u = _stack([gaussian_kernel(d, r, 0.6 + 1.8 * un[k]) for k in range(m)], d)
        # a little seeded asymmetry so that kernel flips are visible
        u = u + 0.05 * normal(seed + 1, u.size).reshape(u.shape) * u.max()
        v = hat_windows(d, n, g) * (1.0 + 0.25 * uniform(seed + 2, m)[:, None])
        return Operator(name, d, n, over.get("delta", 4), over.get("levels", 3), r, u, v,
                        gap=over.get("gap", 2), order=over.get("order", 0), family=over.get("family", 0))
    raise KeyError(name)


def batch_workload(count: int = 64, seed_offset: int = 0, max_side_2d: int = 512,
                   max_pow_1d: int = 16) -> list[Operator]:
    """Uneven batch: the first half 1-D with n = 2^p, p ~ U{10..max_pow_1d}; the second
    half 2-D with side ~ U{64,128,256,512} (capped at max_side_2d); m ~ U{4,9,16,25}
    (sqrt(m) x sqrt(m) hats in 2-D, m hats in 1-D); odd width ~ U{5,...,31};
    Gaussian sigma_k = (width-1)/8 * (0.5 + k/(m-1)); db2/db4 ~ U; L ~ U{3..6} with
    n / 2^L >= 2; pattern gap 2."""
    seed = BASE_SEED + 4 + 1000 * seed_offset
    un = uniform(seed, 8 * count).reshape(count, 8)
    ops = []
    for i in range(count):
        d = 1 if i < count // 2 else 2
        if d == 1:
            n = 2 ** (10 + int(un[i, 0] * (max_pow_1d - 9)))
        else:
            sides = [s for s in (64, 128, 256, 512) if s <= max_side_2d]
            n = sides[int(un[i, 0] * len(sides))]
        m = (4, 9, 16, 25)[int(un[i, 1] * 4)]
        width = 5 + 2 * int(un[i, 2] * 14)            # 5..31 odd
        r = width // 2
        delta = (2, 4)[int(un[i, 3] * 2)]
        lmax = min(6, int(math.log2(n)) - 1)
        levels = 3 + int(un[i, 4] * (lmax - 2))
        base = (width - 1) / 8.0
        sig = [base * (0.5 + (k / (m - 1) if m > 1 else 0.0)) for k in range(m)]
        u = _stack([gaussian_kernel(d, r, max(s, 0.3)) for s in sig], d)
        g = int(round(math.sqrt(m))) if d == 2 else m
        v = hat_windows(d, n, g)
        ops.append(Operator(f"batch{i}", d, n, delta, levels, r, u, v, gap=2, order=0))
    return ops
