// Thresholded Algorithm 1 (Section 3.2) on the GPU: Theta~ = sum_k A~_k B_k with
// A_k = Psi^* U_k Psi thresholded at tau_k, B_k = Psi^* V_k Psi, every product evaluated in
// pixel space on the support it can reach (the predicted positions of Section 5.3).
//
// Structure used.  Row mu = (band of level j, position x) of A_k is the wavelet transform of
// F_{k,mu}(z) = sum_t u_k(t) psi_mu(z + t).  Shifting x by 2^(J-j) t shifts F by 2^J t
// pixels, and a shift by 2^J t moves the coefficients of every level j' <= J by 2^(J-j') t
// exactly.  So the rows of A_k fall into 2^(J d) classes (band, x mod 2^(J-j)), the rows of a
// class being translates of its representative: one generator row per class and term (the
// sub-band circulant structure of Section 5.3).  Thresholding acts on generator values, the
// discarded part's row and column absolute sums are per row class and per column class, and
// for the product, row mu of A~_k B_k is Psi^*(v_k . F~_{k,mu}) with F~_{k,mu} = Psi A~_k[mu, :]
// (B_k's rows are <psi_q, v_k psi_lambda>), so a row of Theta~ is the wavelet transform of
// s~_mu = sum_k v_k . F~_{k,mu}.  F~ of a class is supported on the union R of its kept
// wavelets' supports; s~ then too, and the row of Theta~ holds the coefficients reaching R.
//
// Every transform runs on "boxes": per axis and level a run [a, a + w) of unwrapped positions
// (w = the period once the run covers it), the coefficients a run of the previous level reaches
// through the taps 2l + i, i in [2 - Lf, Lf - 1].  Values outside a box are zero.  Work is
// spread one CTA per (class, term) or per row, the transforms in FP64.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <vector>

namespace pcw {
namespace alg1 {

constexpr int A1_MAXJ = 16;
constexpr int A1_MAXLF = 20;
constexpr int A1_THREADS = 512;

// One axis of a box at one level: unwrapped start a, width w (w == period: the whole line).
struct Ax {
    int a, w;
};

__host__ __device__ inline int fl2(int x) { return x >> 1; }  // floor(x / 2), arithmetic shift

// floor(a / b) for b > 0
__host__ __device__ inline long long floordiv(long long a, long long b)
{
    const long long q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

// The coefficients of the next level reached by a box of a level of period M.
__host__ __device__ inline Ax next_ax(Ax b, int M, int Lf)
{
    const int M2 = M >> 1;
    if (b.w >= M) return {0, M2};
    const int lo = fl2(b.a - Lf + 2);        // ceil((a - Lf + 1) / 2)
    const int hi = fl2(b.a + b.w + Lf - 3);  // floor((a + w - 1 + Lf - 2) / 2)
    const int w = hi - lo + 1;
    if (w >= M2) return {0, M2};
    return {lo, w};
}

// Geometry of one class of rows (band, phase p): generator boxes (from the support of F,
// levels 0..J) and product boxes (from R), each row's segment offsets.  A row holds, in
// canonical band order, the approximation of level J then, for levels J..1, the detail bands
// (e0, e1) = (0,1), (1,0), (1,1) (2-D; one detail band in 1-D), each over its level's box,
// row-major.
struct A1Class {
    int j, e0, e1, p0, p1;      // band of the representative row and its phase
    int rows;                   // rows in the class (translates): (n >> J)^d
    Ax g[2][A1_MAXJ + 1];       // generator boxes per axis and level
    Ax c[2][A1_MAXJ + 1];       // product boxes per axis and level (c[.][0] = R)
    int goffl[A1_MAXJ + 1];     // offset of level l's detail bands in a generator row
    int coffl[A1_MAXJ + 1];     // the same in a product row
    int glen, tlen;             // entries of a generator row / of a product row
    int rsize;                  // |R| (pixels of the product box), 0 when nothing is kept
    int pad_;
    long long goff;             // first generator entry (per term stride gtotal)
    long long foff;             // first value of F~ (m x |R|)
    long long toff;             // first value of the class's rows of Theta~ (rows x tlen)
};

struct A1Params {
    int D, n, J, Lf, r, m, ncls, nJ;
    long long N, gtotal;
    double h[A1_MAXLF];          // h[i], i in [0, Lf - 1]
    double g[A1_MAXLF];          // g[i] at g[i - (2 - Lf)], i in [2 - Lf, 1]
    int tab_off[A1_MAXJ + 1][2]; // 1-D factor of level j, type e in tab
    int tab_len[A1_MAXJ + 1];
    const A1Class* cls;
    const double* tab;
    const double* u;             // m x (2r+1)^D kernels
    const double* v;             // m x N windows
    double* G;                   // m x gtotal generator entries
    const double* tau;           // m thresholds
    double* Fb;                  // F~ per class: m x |R|
    double* theta;               // Theta~ rows
    long long tbase;             // value offset of the Theta~ buffer's first element
    long long sA, sT, sR;        // scratch layout of a CTA (elements): two level buffers, a
                                 // work buffer, the 1-D factor samples
    // FP32 products (Theta~ in FP32): the taps, F~ and Theta~ in single precision
    float hf[A1_MAXLF], gf[A1_MAXLF];
    float* Fb32;
    float* theta32;
    // per-pixel lists of the terms whose window is nonzero there (slot-major, wslots x N; k = -1
    // ends a list), with the window values in the products' precision
    int wslots;
    const int* wk;
    const double* wv64;
    const float* wv32;
};

template <class T> __device__ __forceinline__ T tap_h(const A1Params& P, int i);
template <> __device__ __forceinline__ double tap_h<double>(const A1Params& P, int i) { return P.h[i]; }
template <> __device__ __forceinline__ float tap_h<float>(const A1Params& P, int i) { return P.hf[i]; }
template <class T> __device__ __forceinline__ T tap_g(const A1Params& P, int i);
template <> __device__ __forceinline__ double tap_g<double>(const A1Params& P, int i) { return P.g[i]; }
template <> __device__ __forceinline__ float tap_g<float>(const A1Params& P, int i) { return P.gf[i]; }

// ---------------------------------------------------------------------------------------
// Host geometry
// ---------------------------------------------------------------------------------------

// 1-D scaling function (e = 0) and wavelet (e = 1) of level j at translate 0 on the integer line,
// by the cascade phi_j(p) = sum_i h[i] phi_{j-1}(p - 2^(j-1) i), psi_j(p) = sum_i g[i]
// phi_{j-1}(p - 2^(j-1) i), phi_0 = the unit pixel.  phi_j lives on [0, (2^j - 1)(Lf - 1)],
// psi_j on 2^(j-1)(2 - Lf) + the same length; returned from its first sample.
inline void factor_tables(const double* h, int Lf, int J, std::vector<std::vector<double>>* phi,
                          std::vector<std::vector<double>>* psi)
{
    phi->assign(J + 1, {});
    psi->assign(J + 1, {});
    (*phi)[0] = {1.0};
    std::vector<double> gg(Lf);
    for (int i = 2 - Lf; i <= 1; ++i) gg[i - (2 - Lf)] = (((1 - i) % 2 == 0) ? 1.0 : -1.0) * h[1 - i];
    for (int j = 1; j <= J; ++j) {
        const int len = ((1 << j) - 1) * (Lf - 1) + 1;
        const std::vector<double>& pp = (*phi)[j - 1];
        const int step = 1 << (j - 1);
        std::vector<double> a(len, 0.0), b(len, 0.0);
        for (int i = 0; i < Lf; ++i)
            for (size_t q = 0; q < pp.size(); ++q) a[q + (size_t)step * i] += h[i] * pp[q];
        // psi_j from index 2^(j-1)(2 - Lf): g[i] at shift 2^(j-1) i, i = 2 - Lf .. 1
        for (int i = 2 - Lf; i <= 1; ++i)
            for (size_t q = 0; q < pp.size(); ++q) b[q + (size_t)step * (i - (2 - Lf))] += gg[i - (2 - Lf)] * pp[q];
        (*phi)[j] = a;
        (*psi)[j] = b;
    }
}

// Start (unwrapped) of the 1-D factor of level j, type e, translate p.
__host__ __device__ inline int factor_start(int j, int e, int p, int Lf)
{
    return (p << j) + (e ? (1 << (j - 1)) * (2 - Lf) : 0);
}

// Box chain from a level-0 box per axis; returns the row length and fills the level offsets.
inline int chain(int D, int n, int J, int Lf, const Ax b0[2], Ax out[2][A1_MAXJ + 1], int offl[A1_MAXJ + 1])
{
    for (int d = 0; d < D; ++d) {
        out[d][0] = b0[d];
        for (int l = 0; l < J; ++l) out[d][l + 1] = next_ax(out[d][l], n >> l, Lf);
    }
    if (D == 1)
        for (int l = 0; l <= J; ++l) out[1][l] = {0, 1};
    int off = out[0][J].w * out[1][J].w;  // approximation of level J first
    for (int l = J; l >= 1; --l) {
        offl[l] = off;
        off += (D == 2 ? 3 : 1) * out[0][l].w * out[1][l].w;
    }
    offl[0] = off;
    return off;
}

// ---------------------------------------------------------------------------------------
// Device transforms on boxes (block-wide; every thread of the CTA calls them)
// ---------------------------------------------------------------------------------------

// Value at unwrapped position p of a line stored on box b with period M (a power of two):
// zero unless p is an image of a stored position.
template <class T>
__device__ __forceinline__ T at(const T* line, int stride, Ax b, int M, int p)
{
    const int k = (p - b.a) & (M - 1);
    return k < b.w ? line[(long long)k * stride] : T(0);
}

// One analysis level of a 2-D box signal X (b0.w x b1.w, row-major, period M): the next
// approximation into Y (nb0.w x nb1.w) and the detail bands (0,1), (1,0), (1,1) into out,
// out + sz, out + 2 sz (sz = nb0.w nb1.w); T holds 2 b0.w nb1.w.  Axis 1 first, then axis 0.
// Filter taps as seen by the transforms: LF > 0 holds the LF taps of h and g in registers (the
// loops over them unroll); LF = 0 reads them from the parameters with the run-time length.
template <class F, int LF>
struct Taps {
    F h[LF], g[LF];
    __device__ explicit Taps(const A1Params& P)
    {
#pragma unroll
        for (int i = 0; i < LF; ++i) {
            h[i] = tap_h<F>(P, i);
            g[i] = tap_g<F>(P, i);
        }
    }
    __device__ int lf() const { return LF; }
    __device__ F H(int i) const { return h[i]; }
    __device__ F G(int i) const { return g[i]; }  // g at index i - (2 - Lf)
};
template <class F>
struct Taps<F, 0> {
    const A1Params& P;
    __device__ explicit Taps(const A1Params& p) : P(p) {}
    __device__ int lf() const { return P.Lf; }
    __device__ F H(int i) const { return tap_h<F>(P, i); }
    __device__ F G(int i) const { return tap_g<F>(P, i); }
};

// One analysis level of a 2-D box signal X (b0.w x b1.w, row-major, period M): the next
// approximation into Y (nb0.w x nb1.w) and the detail bands (0,1), (1,0), (1,1) into out,
// out + sz, out + 2 sz (sz = nb0.w nb1.w); T holds 2 b0.w nb1.w.  Axis 1 first, then axis 0.
// An output whose taps all fall on stored positions reads them unchecked (at() would return the
// same values); the others go through at().
template <class F, int LF = 0>
__device__ void analysis2(const A1Params& P, const F* X, Ax b0, Ax b1, int M, Ax nb0, Ax nb1, F* T, F* Y, F* out)
{
    const Taps<F, LF> tp(P);
    const int Lf = tp.lf();
    const int n01 = b0.w * nb1.w;
    for (int idx = threadIdx.x; idx < n01; idx += blockDim.x) {
        const int r = idx / nb1.w, q = idx - r * nb1.w;
        const int base = 2 * (nb1.a + q);
        const F* line = X + (long long)r * b1.w;
        F lo = 0, hi = 0;
        const int k0 = base + 2 - Lf - b1.a;
        if (k0 >= 0 && k0 + 2 * Lf - 3 < b1.w) {
            const F* xp = line + k0;
#pragma unroll
            for (int i = 2 - Lf; i < Lf; ++i) {
                const F x = xp[i - (2 - Lf)];
                if (i >= 0) lo = fma(tp.H(i), x, lo);
                if (i <= 1) hi = fma(tp.G(i - (2 - Lf)), x, hi);
            }
        } else {
            for (int i = 2 - Lf; i < Lf; ++i) {
                const F x = at(line, 1, b1, M, base + i);
                if (i >= 0) lo = fma(tp.H(i), x, lo);
                if (i <= 1) hi = fma(tp.G(i - (2 - Lf)), x, hi);
            }
        }
        T[idx] = lo;
        T[n01 + idx] = hi;
    }
    __syncthreads();
    const int sz = nb0.w * nb1.w;
    for (int idx = threadIdx.x; idx < sz; idx += blockDim.x) {
        const int r = idx / nb1.w, q = idx - r * nb1.w;
        const int base = 2 * (nb0.a + r);
        F ll = 0, d01 = 0, d10 = 0, d11 = 0;
        const int k0 = base + 2 - Lf - b0.a;
        if (k0 >= 0 && k0 + 2 * Lf - 3 < b0.w) {
            const F* tl = T + (long long)k0 * nb1.w + q;
            const F* th = tl + n01;
#pragma unroll
            for (int i = 2 - Lf; i < Lf; ++i) {
                const long long o = (long long)(i - (2 - Lf)) * nb1.w;
                const F xl = tl[o], xh = th[o];
                if (i >= 0) {
                    ll = fma(tp.H(i), xl, ll);
                    d01 = fma(tp.H(i), xh, d01);
                }
                if (i <= 1) {
                    const F gi = tp.G(i - (2 - Lf));
                    d10 = fma(gi, xl, d10);
                    d11 = fma(gi, xh, d11);
                }
            }
        } else {
            for (int i = 2 - Lf; i < Lf; ++i) {
                const F xl = at(T + q, nb1.w, b0, M, base + i);
                const F xh = at(T + n01 + q, nb1.w, b0, M, base + i);
                if (i >= 0) {
                    ll = fma(tp.H(i), xl, ll);
                    d01 = fma(tp.H(i), xh, d01);
                }
                if (i <= 1) {
                    const F gi = tp.G(i - (2 - Lf));
                    d10 = fma(gi, xl, d10);
                    d11 = fma(gi, xh, d11);
                }
            }
        }
        Y[idx] = ll;
        out[idx] = d01;
        out[sz + idx] = d10;
        out[2 * sz + idx] = d11;
    }
    __syncthreads();
}

// One analysis level of a 1-D box signal.
template <class F, int LF = 0>
__device__ void analysis1(const A1Params& P, const F* X, Ax b, int M, Ax nb, F* Y, F* out)
{
    const Taps<F, LF> tp(P);
    const int Lf = tp.lf();
    for (int idx = threadIdx.x; idx < nb.w; idx += blockDim.x) {
        const int base = 2 * (nb.a + idx);
        F lo = 0, hi = 0;
        const int k0 = base + 2 - Lf - b.a;
        if (k0 >= 0 && k0 + 2 * Lf - 3 < b.w) {
#pragma unroll
            for (int i = 2 - Lf; i < Lf; ++i) {
                const F x = X[k0 + i - (2 - Lf)];
                if (i >= 0) lo = fma(tp.H(i), x, lo);
                if (i <= 1) hi = fma(tp.G(i - (2 - Lf)), x, hi);
            }
        } else {
            for (int i = 2 - Lf; i < Lf; ++i) {
                const F x = at(X, 1, b, M, base + i);
                if (i >= 0) lo = fma(tp.H(i), x, lo);
                if (i <= 1) hi = fma(tp.G(i - (2 - Lf)), x, hi);
            }
        }
        Y[idx] = lo;
        out[idx] = hi;
    }
    __syncthreads();
}

// Detail coefficients of a thresholded generator row at one level: band b at (y0, y1), zero
// outside the row's box or below the threshold.
struct GenDet {
    const double* row;
    Ax g0, g1;
    int Mh, off, bsz;
    double tau;
    __device__ double operator()(int b, int y0, int y1) const
    {
        const int k0 = (y0 - g0.a) & (Mh - 1), k1 = (y1 - g1.a) & (Mh - 1);
        if (k0 >= g0.w || k1 >= g1.w) return 0.0;
        const double v = row[off + b * bsz + k0 * g1.w + k1];
        return fabs(v) >= tau ? v : 0.0;
    }
};

// One synthesis level restricted to an output box: from the approximation Y of level l on
// (cb0, cb1) (period Mh) and the detail bands det, the approximation of level l - 1 on
// (ob0, ob1) into X; x[p] = sum over i with p - i even of h[i] a[(p - i)/2] + g[i] d[(p - i)/2]
// per axis (the transpose of the analysis).  Axis 0 first, then axis 1; T holds
// 2 ob0.w cb1.w.  (cb0, cb1) must be the boxes the output box reaches, so that nothing else
// contributes to it.
__device__ void synthesis2(const A1Params& P, const double* Y, Ax cb0, Ax cb1, int Mh, Ax ob0, Ax ob1, double* T,
                           double* X, const GenDet& det)
{
    const int Lf = P.Lf;
    const int n01 = ob0.w * cb1.w;
    for (int idx = threadIdx.x; idx < n01; idx += blockDim.x) {
        const int r = idx / cb1.w, q = idx - r * cb1.w;
        const int p0 = ob0.a + r, y1 = cb1.a + q;
        double lo = 0.0, hi = 0.0;
        const int i0 = ((p0 - (2 - Lf)) & 1) ? 3 - Lf : 2 - Lf;
        for (int i = i0; i < Lf; i += 2) {
            const int l0 = (p0 - i) >> 1;
            if (i >= 0) {
                lo = fma(P.h[i], at(Y + q, cb1.w, cb0, Mh, l0), lo);
                hi = fma(P.h[i], det(0, l0, y1), hi);
            }
            if (i <= 1) {
                const double gi = P.g[i - (2 - Lf)];
                lo = fma(gi, det(1, l0, y1), lo);
                hi = fma(gi, det(2, l0, y1), hi);
            }
        }
        T[idx] = lo;
        T[n01 + idx] = hi;
    }
    __syncthreads();
    const int sz = ob0.w * ob1.w;
    for (int idx = threadIdx.x; idx < sz; idx += blockDim.x) {
        const int r = idx / ob1.w, q = idx - r * ob1.w;
        const int p1 = ob1.a + q;
        const double* rl = T + (long long)r * cb1.w;
        const double* rh = T + n01 + (long long)r * cb1.w;
        double x = 0.0;
        const int i0 = ((p1 - (2 - Lf)) & 1) ? 3 - Lf : 2 - Lf;
        for (int i = i0; i < Lf; i += 2) {
            const int l1 = (p1 - i) >> 1;
            if (i >= 0) x = fma(P.h[i], at(rl, 1, cb1, Mh, l1), x);
            if (i <= 1) x = fma(P.g[i - (2 - Lf)], at(rh, 1, cb1, Mh, l1), x);
        }
        X[idx] = x;
    }
    __syncthreads();
}

// One synthesis level of a 1-D box signal.
__device__ void synthesis1(const A1Params& P, const double* Y, Ax cb, int Mh, Ax ob, double* X, const GenDet& det)
{
    const int Lf = P.Lf;
    for (int idx = threadIdx.x; idx < ob.w; idx += blockDim.x) {
        const int p = ob.a + idx;
        double x = 0.0;
        const int i0 = ((p - (2 - Lf)) & 1) ? 3 - Lf : 2 - Lf;
        for (int i = i0; i < Lf; i += 2) {
            const int l = (p - i) >> 1;
            if (i >= 0) x = fma(P.h[i], at(Y, 1, cb, Mh, l), x);
            if (i <= 1) x = fma(P.g[i - (2 - Lf)], det(0, l, 0), x);
        }
        X[idx] = x;
    }
    __syncthreads();
}

// Copies a class record into shared memory.
__device__ inline void load_class(const A1Class* src, A1Class* dst)
{
    __syncthreads();
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(A1Class) / sizeof(int)); i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

// Analysis chain over the boxes bx (levels 0..J) from X, into a row (approximation of level J
// at 0, detail bands of level l at offl[l]).  X and Y are swapped between levels; returns the
// buffer holding the approximation.
template <int D, class F, int LF = 0>
__device__ F* analysis_chain(const A1Params& P, F* X, F* Y, F* T, const Ax (*bx)[A1_MAXJ + 1], const int* offl,
                             F* row)
{
    for (int l = 0; l < P.J; ++l) {
        const int M = P.n >> l;
        if (D == 2)
            analysis2<F, LF>(P, X, bx[0][l], bx[1][l], M, bx[0][l + 1], bx[1][l + 1], T, Y, row + offl[l + 1]);
        else
            analysis1<F, LF>(P, X, bx[0][l], M, bx[0][l + 1], Y, row + offl[l + 1]);
        F* t = X;
        X = Y;
        Y = t;
    }
    const int sz = bx[0][P.J].w * bx[1][P.J].w;
    for (int idx = threadIdx.x; idx < sz; idx += blockDim.x) row[idx] = X[idx];
    __syncthreads();
    return X;
}

// 1-D factor (type e, level j, translate p) at unwrapped pixel x, periodised with period n.
__device__ inline double factor_at(const A1Params& P, int j, int e, int p, int x)
{
    const int s = factor_start(j, e, p, P.Lf);
    const int len = P.tab_len[j];
    const double* t = P.tab + P.tab_off[j][e];
    double acc = 0.0;
    for (int k = (x - s) & (P.n - 1); k < len; k += P.n) acc += t[k];
    return acc;
}

// ---------------------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------------------

// Stage 1: generator rows.  One CTA per (class, term): F(z) = sum_t u_k(t) psi_c(z + t) on the
// class's level-0 generator box (psi_c = the separable product of 1-D factors, the sum over t
// split per axis), then its analysis chain into G[k][class].
template <int D, int LF = 0>
__global__ void __launch_bounds__(A1_THREADS) k_a1_generators(const __grid_constant__ A1Params P, double* gscratch)
{
    extern __shared__ double smem[];
    __shared__ A1Class C;
    double* S = gscratch ? gscratch + (long long)blockIdx.x * (2 * P.sA + P.sT + P.sR) : smem;
    double *A = S, *B = S + P.sA, *T = S + 2 * P.sA, *Rs = T + P.sT;
    const int r = P.r, K1 = 2 * r + 1;
    const int K = (D == 2) ? K1 * K1 : K1;
    for (int item = blockIdx.x; item < P.ncls * P.m; item += gridDim.x) {
        const int c = item % P.ncls, k = item / P.ncls;
        load_class(P.cls + c, &C);
        const Ax a0 = C.g[0][0], a1 = C.g[1][0];
        const int n0 = a0.w + 2 * r, n1 = (D == 2) ? a1.w + 2 * r : 0;
        double* R0 = Rs;
        double* R1 = Rs + n0;
        for (int i = threadIdx.x; i < n0 + n1; i += blockDim.x) {
            if (i < n0)
                R0[i] = factor_at(P, C.j, C.e0, C.p0, a0.a - r + i);
            else
                R1[i - n0] = factor_at(P, C.j, C.e1, C.p1, a1.a - r + (i - n0));
        }
        __syncthreads();
        const double* uk = P.u + (long long)k * K;
        if (D == 2) {
            // Y[t0][i1] = sum_t1 u(t0, t1) psi1(z1 + t1), then F[i0][i1] = sum_t0 psi0(z0 + t0) Y[t0][i1]
            for (int idx = threadIdx.x; idx < K1 * a1.w; idx += blockDim.x) {
                const int t0 = idx / a1.w, i1 = idx - t0 * a1.w;
                double acc = 0.0;
                for (int t1 = 0; t1 < K1; ++t1) acc = fma(uk[t0 * K1 + t1], R1[i1 + t1], acc);
                T[idx] = acc;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < a0.w * a1.w; idx += blockDim.x) {
                const int i0 = idx / a1.w, i1 = idx - i0 * a1.w;
                double acc = 0.0;
                for (int t0 = 0; t0 < K1; ++t0) acc = fma(R0[i0 + t0], T[t0 * a1.w + i1], acc);
                A[idx] = acc;
            }
        } else {
            for (int idx = threadIdx.x; idx < a0.w; idx += blockDim.x) {
                double acc = 0.0;
                for (int t = 0; t < K1; ++t) acc = fma(uk[t], R0[idx + t], acc);
                A[idx] = acc;
            }
        }
        __syncthreads();
        analysis_chain<D, double, LF>(P, A, B, T, C.g, C.goffl, P.G + (long long)k * P.gtotal + C.goff);
    }
}

// Per-pixel lists of the terms with v_k(x) != 0: pass 0 counts the longest list (atomicMax), pass
// 1 writes the lists (increasing k, -1 after the last) and the window values.
__global__ void k_a1_wlist(const double* v, int m, long long N, int slots, int* maxcnt, int* wk, double* wv64,
                           float* wv32)
{
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
        int cnt = 0;
        for (int k = 0; k < m; ++k) {
            const double a = v[(long long)k * N + x];
            if (a == 0.0) continue;
            if (slots > 0 && cnt < slots) {
                wk[(long long)cnt * N + x] = k;
                if (wv64) wv64[(long long)cnt * N + x] = a;
                if (wv32) wv32[(long long)cnt * N + x] = (float)a;
            }
            ++cnt;
        }
        if (slots > 0) {
            if (cnt < slots) wk[(long long)cnt * N + x] = -1;
        } else {
            atomicMax(maxcnt, cnt);
        }
    }
}

// Max |x| over each of gridDim.y runs of len values (stride apart), blocks of a run splitting it:
// out[blockIdx.y] holds the bits of the max (zeroed first); for non-negative doubles the bit
// patterns order like the values, so an integer atomicMax gives the exact maximum.
__global__ void k_a1_absmax(const double* x, long long stride, long long len, unsigned long long* out)
{
    __shared__ double red[32];
    const double* p = x + (long long)blockIdx.y * stride;
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(p[i]));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) atomicMax(out + blockIdx.y, (unsigned long long)__double_as_longlong(m));
    }
}

// Stage 2a: for the query threshold tq[k] of every term, the discarded absolute sum of each
// segment (the entries of one row class in one column class, listed by perm).  A warp per
// segment, each lane summing a fixed subsequence, then a fixed shuffle tree: deterministic.
__global__ void __launch_bounds__(A1_THREADS) k_a1_segsum(const __grid_constant__ A1Params P, const int* perm,
                                                          const long long* seg_start, const int* seg_len,
                                                          const int* seg_row_off, int nseg, const double* tq,
                                                          double* segsum)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int item = blockIdx.x; item < P.ncls * P.m; item += gridDim.x) {
        const int c = item % P.ncls, k = item / P.ncls;
        const double t = tq[k];
        const double* row = P.G + (long long)k * P.gtotal + P.cls[c].goff;
        for (int s = seg_row_off[c] + warp; s < seg_row_off[c + 1]; s += nw) {
            const long long st = seg_start[s];
            const int len = seg_len[s];
            double acc = 0.0;
            for (int i = lane; i < len; i += 32) {
                const double a = fabs(row[perm[st + i]]);
                if (a < t) acc += a;
            }
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) segsum[(long long)k * nseg + s] = acc;
        }
    }
}

// Stage 2b: one bisection step per term (one CTA per term).  The discarded part D of A_k has
// row sums = the row class sums and column sums = the column class sums (every row and
// column of a class has the same multiset of values); its Schur bound sqrt(||D||_1 ||D||_inf)
// decides: step 0 tries the top threshold (everything discarded), steps 1..last halve
// [lo, hi] keeping lo feasible; tau = lo at the end.
__global__ void k_a1_bisect(int ncls, int nseg, const int* seg_row_off, const int* colseg_off, const int* colseg,
                            const double* segsum, const double* eps, const double* top, double* lo, double* hi,
                            double* tq, double* tau, int* done, int step, int last)
{
    __shared__ double red[2][32];
    const int k = blockIdx.x;
    const double* ss = segsum + (long long)k * nseg;
    double mr = 0.0, mc = 0.0;
    for (int c = threadIdx.x; c < ncls; c += blockDim.x) {
        double a = 0.0;
        for (int s = seg_row_off[c]; s < seg_row_off[c + 1]; ++s) a += ss[s];
        double b = 0.0;
        for (int q = colseg_off[c]; q < colseg_off[c + 1]; ++q) b += ss[colseg[q]];
        mr = fmax(mr, a);
        mc = fmax(mc, b);
    }
    for (int o = 16; o; o >>= 1) {
        mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
        mc = fmax(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = mr;
        red[1][threadIdx.x >> 5] = mc;
    }
    __syncthreads();
    if (threadIdx.x != 0 || done[k]) return;
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        mr = fmax(mr, red[0][w]);
        mc = fmax(mc, red[1][w]);
    }
    const double schur = sqrt(mr * mc);
    if (step == 0) {
        if (schur <= eps[k]) {
            tau[k] = tq[k];
            done[k] = 1;
        } else {
            lo[k] = 0.0;
            hi[k] = tq[k];
            tq[k] = 0.5 * (lo[k] + hi[k]);
        }
        return;
    }
    if (schur <= eps[k])
        lo[k] = tq[k];
    else
        hi[k] = tq[k];
    if (step == last) {
        tau[k] = lo[k];
        done[k] = 1;
    } else {
        tq[k] = 0.5 * (lo[k] + hi[k]);
    }
}

// Walks the segments of a row on boxes bx: calls f(level, e0, e1, offset of the segment, box0,
// box1) for the approximation of level J, then levels J..1 and their detail bands.
template <int D, class Fn>
__device__ inline void for_segments(int J, const Ax (*bx)[A1_MAXJ + 1], const int* offl, Fn f)
{
    f(J, 0, 0, 0, bx[0][J], bx[1][J]);
    for (int l = J; l >= 1; --l) {
        const int sz = bx[0][l].w * bx[1][l].w;
        if (D == 2) {
            f(l, 0, 1, offl[l], bx[0][l], bx[1][l]);
            f(l, 1, 0, offl[l] + sz, bx[0][l], bx[1][l]);
            f(l, 1, 1, offl[l] + 2 * sz, bx[0][l], bx[1][l]);
        } else {
            f(l, 1, 0, offl[l], bx[0][l], bx[1][l]);
        }
    }
}

// Stage 2c: entries kept per (class, term) and the box R of each class: per axis the union of
// the kept wavelets' supports, each taken at the image nearest the class's F box (unwrapped).
template <int D>
__global__ void __launch_bounds__(A1_THREADS) k_a1_support(const __grid_constant__ A1Params P, long long* kept,
                                                           int* rbox)
{
    __shared__ A1Class C;
    __shared__ long long redc[32];
    __shared__ int redb[4][32];
    const int Lf = P.Lf, n = P.n;
    for (int item = blockIdx.x; item < P.ncls * P.m; item += gridDim.x) {
        const int c = item % P.ncls, k = item / P.ncls;
        load_class(P.cls + c, &C);
        const double* row = P.G + (long long)k * P.gtotal + C.goff;
        const double tau = P.tau[k];
        long long cnt = 0;
        int lo[2] = {INT_MAX, INT_MAX}, hi[2] = {INT_MIN, INT_MIN};
        const int cen2[2] = {2 * C.g[0][0].a + C.g[0][0].w - 1, 2 * C.g[1][0].a + C.g[1][0].w - 1};
        for_segments<D>(P.J, C.g, C.goffl, [&](int l, int e0, int e1, int off, Ax b0, Ax b1) {
            const int len = ((1 << l) - 1) * (Lf - 1) + 1;
            for (int idx = threadIdx.x; idx < b0.w * b1.w; idx += blockDim.x) {
                const double v = row[off + idx];
                if (!(fabs(v) >= tau) || v == 0.0) continue;
                ++cnt;
                const int i0 = idx / b1.w, i1 = idx - i0 * b1.w;
                const int yy[2] = {b0.a + i0, b1.a + i1};
                const int ee[2] = {e0, e1};
                for (int d = 0; d < D; ++d) {
                    long long s0 = (long long)yy[d] * (1 << l) + (ee[d] ? (1 << (l - 1)) * (2 - Lf) : 0);
                    long long s1 = s0 + len - 1;
                    const long long q = floordiv(cen2[d] - (s0 + s1) + n, 2LL * n);
                    s0 += q * n;
                    s1 += q * n;
                    lo[d] = min(lo[d], (int)s0);
                    hi[d] = max(hi[d], (int)s1);
                }
            }
        });
        for (int o = 16; o; o >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            for (int d = 0; d < 2; ++d) {
                lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
                hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
            }
        }
        if ((threadIdx.x & 31) == 0) {
            const int w = threadIdx.x >> 5;
            redc[w] = cnt;
            redb[0][w] = lo[0];
            redb[1][w] = hi[0];
            redb[2][w] = lo[1];
            redb[3][w] = hi[1];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                cnt += redc[w];
                lo[0] = min(lo[0], redb[0][w]);
                hi[0] = max(hi[0], redb[1][w]);
                lo[1] = min(lo[1], redb[2][w]);
                hi[1] = max(hi[1], redb[3][w]);
            }
            kept[(long long)k * P.ncls + c] = cnt;
            if (cnt) {
                for (int d = 0; d < D; ++d) {
                    atomicMin(rbox + 4 * c + 2 * d, lo[d]);
                    atomicMax(rbox + 4 * c + 2 * d + 1, hi[d]);
                }
            }
        }
    }
}

// Stage 3: F~_{k,c} = Psi A~_k[c, :] on the class's product box R, by the synthesis chain
// restricted to the boxes R reaches (level J down to 0), reading the thresholded generator.
template <int D>
__global__ void __launch_bounds__(A1_THREADS) k_a1_synth(const __grid_constant__ A1Params P, double* gscratch)
{
    extern __shared__ double smem[];
    __shared__ A1Class C;
    double* S = gscratch ? gscratch + (long long)blockIdx.x * (2 * P.sA + P.sT) : smem;
    double *X = S, *Y = S + P.sA, *T = S + 2 * P.sA;
    const int J = P.J;
    for (int item = blockIdx.x; item < P.ncls * P.m; item += gridDim.x) {
        const int c = item % P.ncls, k = item / P.ncls;
        load_class(P.cls + c, &C);
        if (C.rsize == 0) continue;
        const double* row = P.G + (long long)k * P.gtotal + C.goff;
        const double tau = P.tau[k];
        {
            const GenDet ap{row, C.g[0][J], C.g[1][J], P.n >> J, 0, 0, tau};
            const Ax c0 = C.c[0][J], c1 = C.c[1][J];
            for (int idx = threadIdx.x; idx < c0.w * c1.w; idx += blockDim.x) {
                const int r = idx / c1.w, q = idx - r * c1.w;
                X[idx] = ap(0, c0.a + r, c1.a + q);
            }
            __syncthreads();
        }
        for (int l = J; l >= 1; --l) {
            const int Mh = P.n >> l;
            const GenDet det{row, C.g[0][l], C.g[1][l], Mh, C.goffl[l], C.g[0][l].w * C.g[1][l].w, tau};
            if (D == 2)
                synthesis2(P, X, C.c[0][l], C.c[1][l], Mh, C.c[0][l - 1], C.c[1][l - 1], T, Y, det);
            else
                synthesis1(P, X, C.c[0][l], Mh, C.c[0][l - 1], Y, det);
            double* t = X;
            X = Y;
            Y = t;
        }
        if (P.Fb32) {
            float* out = P.Fb32 + C.foff + (long long)k * C.rsize;
            for (int idx = threadIdx.x; idx < C.rsize; idx += blockDim.x) out[idx] = (float)X[idx];
        } else {
            double* out = P.Fb + C.foff + (long long)k * C.rsize;
            for (int idx = threadIdx.x; idx < C.rsize; idx += blockDim.x) out[idx] = X[idx];
        }
        __syncthreads();
    }
}

// Stage 4: the rows of Theta~.  One CTA per row (class c, translate t): s~ = sum_k v_k . F~_{k,c}
// on R shifted by 2^J t (over the terms whose window is nonzero at the pixel, in increasing k),
// then its analysis chain on the class's product boxes.  F = double: FP64
// throughout; F = float: FP32 windows, F~ and transform, the sum over k compensated (Kahan).
// LF > 0: instantiated for one filter length (taps in registers).  The CTAs take the rows of the
// classes clist[0 .. nlist).
template <class F> struct ProdIO;
template <> struct ProdIO<double> {
    static __device__ const double* wv(const A1Params& P) { return P.wv64; }
    static __device__ const double* fb(const A1Params& P) { return P.Fb; }
    static __device__ double* theta(const A1Params& P) { return P.theta; }
};
template <> struct ProdIO<float> {
    static __device__ const float* wv(const A1Params& P) { return P.wv32; }
    static __device__ const float* fb(const A1Params& P) { return P.Fb32; }
    static __device__ float* theta(const A1Params& P) { return P.theta32; }
};

template <int D, class F, int LF = 0>
__global__ void __launch_bounds__(A1_THREADS) k_a1_product(const __grid_constant__ A1Params P, const int* clist,
                                                           int nlist, F* gscratch)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ A1Class C;
    F* S = gscratch ? gscratch + (long long)blockIdx.x * (2 * P.sA + P.sT) : reinterpret_cast<F*>(smem_raw);
    F *X = S, *Y = S + P.sA, *T = S + 2 * P.sA;
    const F* WV = ProdIO<F>::wv(P);
    const F* FB = ProdIO<F>::fb(P);
    F* TH = ProdIO<F>::theta(P);
    const int rows = (D == 2) ? P.nJ * P.nJ : P.nJ;
    const long long total = (long long)nlist * rows;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        const int ci = (int)(item / rows), t = (int)(item - (long long)ci * rows);
        load_class(P.cls + clist[ci], &C);
        if (C.tlen == 0) continue;
        const int t0 = (D == 2) ? t / P.nJ : t, t1 = (D == 2) ? t - t0 * P.nJ : 0;
        const Ax R0 = C.c[0][0], R1 = C.c[1][0];
        const F* Fc = FB + C.foff;
        for (int idx = threadIdx.x; idx < C.rsize; idx += blockDim.x) {
            const int i0 = idx / R1.w, i1 = idx - i0 * R1.w;
            const int x0 = (R0.a + i0 + (t0 << P.J)) & (P.n - 1);
            const long long pix = (D == 2) ? (long long)x0 * P.n + ((R1.a + i1 + (t1 << P.J)) & (P.n - 1)) : x0;
            F s = 0, comp = 0;
            for (int sl = 0; sl < P.wslots; ++sl) {
                const int k = P.wk[(long long)sl * P.N + pix];
                if (k < 0) break;
                const F term = WV[(long long)sl * P.N + pix] * Fc[(long long)k * C.rsize + idx];
                if (sizeof(F) == 4) {
                    const F y = term - comp;
                    const F z = s + y;
                    comp = (z - s) - y;
                    s = z;
                } else {
                    s += term;
                }
            }
            X[idx] = s;
        }
        __syncthreads();
        analysis_chain<D, F, LF>(P, X, Y, T, C.c, C.coffl, TH + (C.toff - P.tbase) + (long long)t * C.tlen);
    }
}

}  // namespace alg1
}  // namespace pcw
