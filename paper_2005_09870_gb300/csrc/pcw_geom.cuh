// Geometry of the periodic separable Daubechies basis and of the prescribed pattern.
//
// Shared by the host planner and the device kernels of libpcwave (not by the oracle).
//
// Levels j = 1 (finest) .. L (coarsest); level j has n_j = n >> j translates per axis.
// The 1-D factor rho^e_{j,l} (e = 0: scaling function phi, e = 1: wavelet psi) is supported
// on 2^j l + off(j,e) + [0, len_j - 1] before periodisation, with
//   len_j = (2^j - 1)(Lf - 1) + 1,  off(j,0) = 0,  off(j,1) = 2^(j-1)(2 - Lf)
// which follows from supp h = [0, Lf-1], supp g = [2-Lf, 1] and the cascade recursion of
// Section 2.1.  Bands in canonical order: b = 0 is the approximation band (level L, e = 0);
// then levels L..1, each with bands e = (0,1), (1,0), (1,1) in 2-D (e = 1 in 1-D).
//
// Pattern (the "prescribed scale/space pattern"; Remark 5.3's truncation rule (i) with
// J(L) = gap, and the support test of Section 5.2 widened by the kernel radius r):
// (mu, lambda) is kept iff | |mu| - |lambda| | <= gap and, on each axis, the support of
// psi_lambda meets supp psi_mu widened by r on the torus.  Entries failing the spatial test
// are exactly zero.  For a row (filtered-side element) at level j, translate l, the kept
// translates l' of a column band at level j2 form one run of consecutive integers
// (mod n_j2) on each axis: the "stencil" computed below.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define PCW_HD __host__ __device__ __forceinline__
#else
#define PCW_HD inline
#endif

namespace pcw {

// Every divisor in this geometry is a power of two (grid sides, level lengths, strides 2^k):
// floor/ceil division are arithmetic shifts and the periodic residue is a mask.
PCW_HD int log2i(int b)
{
#ifdef __CUDA_ARCH__
    return __ffs(b) - 1;
#else
    return __builtin_ctz((unsigned)b);
#endif
}
PCW_HD int floor_div(int a, int b) { return a >> log2i(b); }     // b = 2^k
PCW_HD int ceil_div(int a, int b) { return -((-a) >> log2i(b)); }
PCW_HD int pmod(int a, int b) { return a & (b - 1); }            // b = 2^k, result in [0, b)

PCW_HD int wav_len(int j, int Lf) { return ((1 << j) - 1) * (Lf - 1) + 1; }
PCW_HD int wav_off(int j, int e, int Lf) { return e ? (1 << (j - 1)) * (2 - Lf) : 0; }

// Unwrapped index range of the coefficients kept at one level on one axis.  When the range
// covers the whole circle (cnt == n at that level) it is "full": every residue once, indices
// are then read modulo the level length.
struct Range {
    int lo;
    int cnt;
    int full;
};

// Outputs y of a stride-S filter out[y] = sum_{i<len} f[i] in[S*y + off + i] that can be
// nonzero when the input is supported on `in`.
PCW_HD Range range_filter(Range in, int S, int off, int len, int n_out)
{
    Range o;
    o.lo = ceil_div(in.lo - off - len + 1, S);
    int hi = floor_div(in.lo + in.cnt - 1 - off, S);
    o.cnt = hi - o.lo + 1;
    o.full = in.full;
    if (o.cnt >= n_out || in.full) {
        o.cnt = n_out;
        o.full = 1;
    }
    return o;
}

// One cascade step keeping both the low-pass (h, taps at [0, Lf-1]) and the high-pass
// (g, taps at [2-Lf, 1]) outputs: the union of the two ranges.
PCW_HD Range range_cascade(Range in, int Lf, int n_out)
{
    Range o;
    o.lo = ceil_div(in.lo - Lf + 1, 2);
    int hi = floor_div(in.lo + in.cnt - 1 + Lf - 2, 2);
    o.cnt = hi - o.lo + 1;
    o.full = in.full;
    if (o.cnt >= n_out || in.full) {
        o.cnt = n_out;
        o.full = 1;
    }
    return o;
}

// Level-0 (pixel) region of a filtered-side element at level j, factor e, translate l:
// supp rho^e_{j,l} widened by r; capped to the circle when it covers it.
PCW_HD Range region0(int j, int e, int l, int r, int Lf, int n)
{
    Range o;
    o.lo = (l << j) + wav_off(j, e, Lf) - r;
    o.cnt = wav_len(j, Lf) + 2 * r;
    o.full = 0;
    if (o.cnt >= n) {
        o.cnt = n;
        o.full = 1;
    }
    return o;
}

// Stencil on one axis: first unwrapped translate and count of the column translates at
// (j2, e2) kept for a row at (j, e, l).  dense: every translate.
PCW_HD void stencil(int j, int e, int l, int j2, int e2, int r, int Lf, int n, int dense,
                    int* first, int* count)
{
    int n2 = n >> j2;
    if (dense) {
        *first = 0;
        *count = n2;
        return;
    }
    int U = (l << j) + wav_off(j, e, Lf) - r;
    int E = U + wav_len(j, Lf) + 2 * r - 1;
    int a2 = wav_off(j2, e2, Lf), len2 = wav_len(j2, Lf);
    int lo = ceil_div(U - a2 - len2 + 1, 1 << j2);
    int hi = floor_div(E - a2, 1 << j2);
    int c = hi - lo + 1;
    if (c > n2) c = n2;
    *first = lo;
    *count = c;
}

struct Band {
    int j;       // level (approximation band: L)
    int e0, e1;  // factor per axis (1-D: e0 = 0)
    int nj;      // translates per axis
    int64_t off; // first canonical index
};

PCW_HD int num_bands(int d, int L) { return 1 + L * ((d == 1) ? 1 : 3); }

PCW_HD Band band_info(int d, int n, int L, int b)
{
    Band B;
    if (b == 0) {
        B.j = L;
        B.e0 = 0;
        B.e1 = 0;
        B.nj = n >> L;
        B.off = 0;
        return B;
    }
    int per = (d == 1) ? 1 : 3;
    int lev = L - (b - 1) / per;
    int t = (b - 1) % per;
    B.j = lev;
    B.nj = n >> lev;
    if (d == 1) {
        B.e0 = 0;
        B.e1 = 1;
        B.off = B.nj;
    } else {
        B.e0 = (t >= 1) ? 1 : 0;
        B.e1 = (t == 1) ? 0 : 1;
        B.off = (int64_t)B.nj * B.nj * (1 + t);
    }
    return B;
}

PCW_HD int band_of_level(int d, int L, int j, int t)
{  // t = 0..2 (2-D) or 0 (1-D); j = L with t = -1 gives the approximation band
    if (t < 0) return 0;
    return 1 + (L - j) * ((d == 1) ? 1 : 3) + t;
}

PCW_HD int abs_i(int a) { return a < 0 ? -a : a; }

// Is the column band b2 kept for rows of band b (band-gap rule)?
PCW_HD int block_kept(int d, int n, int L, int gap, int b, int b2)
{
    if (gap < 0) return 1;
    Band A = band_info(d, n, L, b), B = band_info(d, n, L, b2);
    return abs_i(A.j - B.j) <= gap;
}

// Number of stored entries of a row (band b, translate l0, l1) in column band b2.
PCW_HD int64_t block_count(int d, int n, int L, int Lf, int r, int gap, int b, int l0, int l1,
                           int b2)
{
    Band A = band_info(d, n, L, b), B = band_info(d, n, L, b2);
    int f, c1, c0 = 1;
    stencil(A.j, A.e1, l1, B.j, B.e1, r, Lf, n, gap < 0, &f, &c1);
    if (d == 2) stencil(A.j, A.e0, l0, B.j, B.e0, r, Lf, n, gap < 0, &f, &c0);
    return (int64_t)c0 * c1;
}

// Arrays of one level are stored row-major with the axis-1 range as pitch, and thread groups
// walk rows with consecutive lanes; an odd pitch keeps those accesses free of shared-memory bank
// conflicts.  A non-wrapping range is extended by one coefficient to an odd count: the extra
// cascade output lies past every filter tap of the input range, so it is exactly zero.
PCW_HD Range pad_odd(Range q, int n_out)
{
    if (!q.full && !(q.cnt & 1) && q.cnt + 1 < n_out) q.cnt += 1;
    return q;
}

// Padded line arrays in shared memory.  The 2-D low/high-pass passes read each output's
// window 2c + [2 - LF, LF - 1] (LF = filter template length >= Lf) without bounds checks; the
// union output range of an input line spans ceil((lo - Lf + 1) / 2) .. floor((hi + Lf - 2) / 2),
// so those windows reach at most Lf + LF - 3 elements past either end of the line.  An array
// of nl lines of len elements therefore keeps that many zeros before its first line and
// between lines (line l starts at margin + l * pitch, pitch >= len + margin, odd so that
// lanes walking lines hit distinct banks), and PASS_SLACK elements after the last line for
// the discarded outputs of a line's last chunk of PASS_CH outputs.
constexpr int PASS_CH = 4;
constexpr int PASS_SLACK = 2 * (PASS_CH - 1);
PCW_HD int pass_margin(int Lf, int LF) { return Lf + LF - 3; }
PCW_HD int odd_pitch(int len, int mg) { return (len + mg) | 1; }
PCW_HD int padded_size(int nl, int len, int mg) { return mg + nl * odd_pitch(len, mg) + PASS_SLACK; }

}  // namespace pcw
