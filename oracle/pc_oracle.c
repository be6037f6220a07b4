/*
 * FP64 CPU oracle for the wavelet matrix of a product-convolution operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares no code
 * with the CUDA path (paper_2005_09870_gb300/) and neither side includes the other.
 *
 * What it computes (Escande & Weiss, "Fast wavelet decomposition of linear operators
 * through product-convolution expansions"):
 *   H f = sum_k u_k * (v_k . f)                         Eq. (2), Section 1  (order 0)
 *   H f = sum_k v_k . (u_k * f)                         convolution first     (order 1)
 *   Theta = Psi^* H Psi,  Theta[mu, lambda] = <psi_mu, H psi_lambda>        Section 3.2
 * column by column, exactly as the paper's naive Algorithm 2 (Section 4.2): get
 * psi_lambda, apply H, take the forward wavelet transform.  Everything is plain
 * double-precision loops over the full periodic grid; no localisation, no blocking.
 *
 * Conventions (the paper leaves them open; see the readings in the design notes):
 *   - levels j = 1 (finest) .. L (coarsest); level j has n_j = n / 2^j translates per axis;
 *   - Daubechies low-pass h with Lf = 2*delta taps on [0, Lf-1], minimum phase, sum sqrt(2)
 *     (or the Symmlet of the same order: same support, least-asymmetric phase); functions
 *     take the filter as a code delta + 100 * family (family 0 Daubechies, 1 Symmlet);
 *     high-pass g[i] = (-1)^(1-i) h[1-i] on [2-Lf, 1]                    (Section 2.1);
 *   - analysis a_j[l] = sum_n h[n-2l] a_{j-1}[n],  d_j[l] = sum_n g[n-2l] a_{j-1}[n],
 *     indices mod n_{j-1} (the recursion of Section 2.1 on the torus);
 *   - 2-D separable bands e = (e0, e1), e0 on axis 0 (rows, slow index);
 *   - canonical coefficient order: approximation band (level L) first, then levels
 *     L..1, bands (0,1), (1,0), (1,1) within a level, translates row-major;
 *   - convolution (u * f)(y) = sum_t u(t) f(y - t), t in [-r, r]^d, stencil row-major.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXTAPS 40

/* ------------------------------------------------------------------------------------
 * Daubechies filter by spectral factorisation (Daubechies 1988; Section 2.1 cites
 * Mallat Thm 7.5 / 7.9 for supp h = [0, 2 delta - 1] and delta vanishing moments).
 * |m0|^2 = cos^(2 delta)(w/2) P(sin^2(w/2)),  P(y) = sum_{k<delta} C(delta-1+k, k) y^k.
 * Each root y_i of P gives z + 1/z = 2 - 4 y_i; keep the root with |z| > 1 for the
 * polynomial sum_n h[n] z^n (minimum phase), multiply by (1+z)^delta, normalise sum h = sqrt 2.
 * ---------------------------------------------------------------------------------- */
static double binom(int a, int b)
{
    double r = 1.0;
    for (int i = 1; i <= b; ++i) r = r * (double)(a - b + i) / (double)i;
    return r;
}

/* roots of the real polynomial sum_k c[k] y^k (degree deg) by Durand-Kerner */
static void poly_roots(const double *c, int deg, double complex *roots)
{
    double complex a[OR_MAXTAPS];
    for (int k = 0; k <= deg; ++k) a[k] = c[k] / c[deg];        /* monic */
    for (int i = 0; i < deg; ++i) roots[i] = cpow(0.4 + 0.9 * I, i);
    for (int it = 0; it < 2000; ++it) {
        double moved = 0.0;
        for (int i = 0; i < deg; ++i) {
            double complex p = 1.0, den = 1.0;
            for (int k = deg - 1; k >= 0; --k) p = p * roots[i] + a[k];
            /* p above evaluated a monic poly via Horner: start value 1 = leading coeff */
            for (int q = 0; q < deg; ++q)
                if (q != i) den *= roots[i] - roots[q];
            double complex step = p / den;
            roots[i] -= step;
            moved = fmax(moved, cabs(step));
        }
        if (moved < 1e-17) break;
    }
}

int or_daubechies(int delta, double *h)
{
    if (delta < 1 || 2 * delta > OR_MAXTAPS) return -1;
    double complex poly[OR_MAXTAPS + 1];
    for (int i = 0; i <= OR_MAXTAPS; ++i) poly[i] = 0.0;
    poly[0] = 1.0;
    int deg = 0;
    /* (1 + z)^delta */
    for (int k = 0; k < delta; ++k) {
        for (int i = deg + 1; i >= 1; --i) poly[i] += poly[i - 1];
        ++deg;
    }
    if (delta > 1) {
        double c[OR_MAXTAPS];
        for (int k = 0; k < delta; ++k) c[k] = binom(delta - 1 + k, k);
        double complex y[OR_MAXTAPS];
        poly_roots(c, delta - 1, y);
        for (int i = 0; i < delta - 1; ++i) {
            double complex b = 2.0 - 4.0 * y[i];                 /* z^2 - b z + 1 = 0 */
            double complex s = csqrt(b * b - 4.0);
            double complex z = (b + s) / 2.0;
            if (cabs(z) < 1.0) z = (b - s) / 2.0;
            /* multiply by (z_var - z) */
            for (int q = deg + 1; q >= 0; --q) {
                double complex lower = (q >= 1) ? poly[q - 1] : 0.0;
                poly[q] = lower - z * poly[q];
            }
            ++deg;
        }
    }
    double sum = 0.0;
    for (int i = 0; i <= deg; ++i) sum += creal(poly[i]);
    for (int i = 0; i <= deg; ++i) h[i] = creal(poly[i]) * sqrt(2.0) / sum;
    return 2 * delta;
}

/* ------------------------------------------------------------------------------------
 * Symmlet (least-asymmetric) filter (Section 4.3 uses the Symmlet basis of order 6).  Same
 * |m0|^2 as Daubechies' filter of the same order (same P), but for every root y_i of P -- each
 * conjugate pair once, so that the taps stay real -- the factor (z - z_i) takes the root z_i
 * of z^2 - (2 - 4 y_i) z + 1 = 0 outside or inside the unit circle, whichever makes the phase
 * of prod_i (e^{-iw} - z_i) closest to linear on [0, pi]: the smallest mean squared residual of
 * the least-squares line through the unwrapped phase at w_k = (k + 1/2) pi / 512, k < 512.
 * A choice and its mirror (all roots inverted: the reversed filter) have the same residual;
 * ties within 1e-9 (relative) go to the smaller energy centre sum_n n h[n]^2.
 * ------------------------------------------------------------------------------------ */
#define OR_SYM_K 512
#define OR_PI 3.14159265358979323846

static double phase_residual(const double complex *z, int nz)
{
    double ph[OR_SYM_K];
    for (int k = 0; k < OR_SYM_K; ++k) ph[k] = 0.0;
    for (int i = 0; i < nz; ++i) {
        double prev = 0.0, acc = 0.0;
        for (int k = 0; k < OR_SYM_K; ++k) {
            const double w = (k + 0.5) * OR_PI / OR_SYM_K;
            const double a = carg(cexp(-I * w) - z[i]);
            if (k == 0) acc = a;
            else {
                double dlt = a - prev;
                while (dlt > OR_PI) dlt -= 2.0 * OR_PI;
                while (dlt < -OR_PI) dlt += 2.0 * OR_PI;
                acc += dlt;
            }
            prev = a;
            ph[k] += acc;
        }
    }
    /* least-squares line a + b w */
    double sw = 0.0, sww = 0.0, sp = 0.0, swp = 0.0;
    for (int k = 0; k < OR_SYM_K; ++k) {
        const double w = (k + 0.5) * OR_PI / OR_SYM_K;
        sw += w; sww += w * w; sp += ph[k]; swp += w * ph[k];
    }
    const double n = OR_SYM_K, det = n * sww - sw * sw;
    const double b = (n * swp - sw * sp) / det, a = (sp - b * sw) / n;
    double r = 0.0;
    for (int k = 0; k < OR_SYM_K; ++k) {
        const double w = (k + 0.5) * OR_PI / OR_SYM_K;
        const double e = ph[k] - a - b * w;
        r += e * e;
    }
    return r / n;
}

/* taps of (1 + z)^delta prod_i (z - z_i), normalised to sum sqrt 2; returns the tap count */
static int taps_from_roots(int delta, const double complex *z, int nz, double *h)
{
    double complex poly[OR_MAXTAPS + 1];
    for (int i = 0; i <= OR_MAXTAPS; ++i) poly[i] = 0.0;
    poly[0] = 1.0;
    int deg = 0;
    for (int k = 0; k < delta; ++k) {
        for (int i = deg + 1; i >= 1; --i) poly[i] += poly[i - 1];
        ++deg;
    }
    for (int i = 0; i < nz; ++i) {
        for (int q = deg + 1; q >= 0; --q) {
            double complex lower = (q >= 1) ? poly[q - 1] : 0.0;
            poly[q] = lower - z[i] * poly[q];
        }
        ++deg;
    }
    double sum = 0.0;
    for (int i = 0; i <= deg; ++i) sum += creal(poly[i]);
    for (int i = 0; i <= deg; ++i) h[i] = creal(poly[i]) * sqrt(2.0) / sum;
    return deg + 1;
}

int or_symmlet(int delta, double *h)
{
    if (delta < 1 || 2 * delta > OR_MAXTAPS) return -1;
    if (delta == 1) return taps_from_roots(1, NULL, 0, h);
    double c[OR_MAXTAPS];
    for (int k = 0; k < delta; ++k) c[k] = binom(delta - 1 + k, k);
    double complex y[OR_MAXTAPS], zout[OR_MAXTAPS];
    const int ny = delta - 1;
    poly_roots(c, ny, y);
    for (int i = 0; i < ny; ++i) {
        double complex b = 2.0 - 4.0 * y[i];
        double complex s = csqrt(b * b - 4.0);
        zout[i] = (b + s) / 2.0;
        if (cabs(zout[i]) < 1.0) zout[i] = (b - s) / 2.0;
    }
    /* groups: a real root alone, a root with positive imaginary part with its conjugate */
    int g_first[OR_MAXTAPS], g_second[OR_MAXTAPS], ng = 0;
    for (int i = 0; i < ny; ++i) {
        const double tol = 1e-9 * (1.0 + cabs(y[i]));
        if (fabs(cimag(y[i])) <= tol) {
            g_first[ng] = i; g_second[ng] = -1; ++ng;
        } else if (cimag(y[i]) > 0.0) {
            int best = -1;
            double bd = 1e300;
            for (int j = 0; j < ny; ++j) {
                if (j == i || cimag(y[j]) >= 0.0) continue;
                const double dd = cabs(y[j] - conj(y[i]));
                if (dd < bd) { bd = dd; best = j; }
            }
            if (best < 0) return -1;
            g_first[ng] = i; g_second[ng] = best; ++ng;
        }
    }
    double best_r = 1e300, best_c = 1e300;
    double hb[OR_MAXTAPS];
    int Lf = 2 * delta;
    for (long mask = 0; mask < (1L << ng); ++mask) {
        double complex z[OR_MAXTAPS];
        int nz = 0;
        for (int g = 0; g < ng; ++g) {
            const int i = g_first[g];
            const double complex zi = ((mask >> g) & 1) ? 1.0 / zout[i] : zout[i];
            z[nz++] = zi;
            if (g_second[g] >= 0) z[nz++] = conj(zi);
        }
        double ht[OR_MAXTAPS];
        if (taps_from_roots(delta, z, nz, ht) != Lf) return -1;
        const double r = phase_residual(z, nz);
        double cen = 0.0;
        for (int n = 0; n < Lf; ++n) cen += n * ht[n] * ht[n];
        const int tie = fabs(r - best_r) <= 1e-9 * fmax(best_r, 1e-300);
        if (r < best_r && !tie) {
            best_r = r; best_c = cen;
            memcpy(hb, ht, sizeof(double) * Lf);
        } else if (tie && cen < best_c) {
            best_c = cen;
            memcpy(hb, ht, sizeof(double) * Lf);
        }
    }
    memcpy(h, hb, sizeof(double) * Lf);
    return Lf;
}

/* Filter code: delta + 100 * family (family 0 = Daubechies, 1 = Symmlet). */
static int filter_taps(int code, double *h)
{
    const int family = code / 100, delta = code % 100;
    if (family == 0) return or_daubechies(delta, h);
    if (family == 1) return or_symmlet(delta, h);
    return -1;
}

/* g[i] = (-1)^(1-i) h[1-i] for i in [2-Lf, 1], stored at g_arr[i - (2 - Lf)] */
static void highpass(const double *h, int Lf, double *g_arr)
{
    for (int i = 2 - Lf; i <= 1; ++i) {
        int s = ((1 - i) % 2 == 0) ? 1 : -1;
        g_arr[i - (2 - Lf)] = s * h[1 - i];
    }
}

static inline int64_t pmod(int64_t a, int64_t m) { int64_t r = a % m; return r < 0 ? r + m : r; }

/* ------------------------------------------------------------------------------------
 * One analysis / synthesis step on a strided periodic line of length M (M even).
 * ---------------------------------------------------------------------------------- */
static void analysis_line(const double *h, const double *g, int Lf, int64_t M,
                          const double *x, int64_t sx, double *a, double *d, int64_t so)
{
    for (int64_t l = 0; l < M / 2; ++l) {
        double sa = 0.0, sd = 0.0;
        for (int i = 0; i < Lf; ++i) sa += h[i] * x[pmod(2 * l + i, M) * sx];
        for (int i = 2 - Lf; i <= 1; ++i) sd += g[i - (2 - Lf)] * x[pmod(2 * l + i, M) * sx];
        a[l * so] = sa;
        d[l * so] = sd;
    }
}

/* transpose of analysis_line: x[(2l+i) mod M] += h[i] a[l] + g[i] d[l] (x zeroed first) */
static void synthesis_line(const double *h, const double *g, int Lf, int64_t M,
                           const double *a, const double *d, int64_t si, double *x, int64_t sx)
{
    for (int64_t q = 0; q < M; ++q) x[q * sx] = 0.0;
    for (int64_t l = 0; l < M / 2; ++l) {
        for (int i = 0; i < Lf; ++i) x[pmod(2 * l + i, M) * sx] += h[i] * a[l * si];
        for (int i = 2 - Lf; i <= 1; ++i) x[pmod(2 * l + i, M) * sx] += g[i - (2 - Lf)] * d[l * si];
    }
}

/* forward transform Psi^*: f (n^d pixels, row-major) -> c (canonical order) */
int or_dwt(int d, int n, int L, int wcode, const double *f, double *c)
{
    double h[OR_MAXTAPS], g[OR_MAXTAPS];
    int Lf = filter_taps(wcode, h);
    if (Lf < 0 || (n >> L) < 1 || (d != 1 && d != 2)) return -1;
    highpass(h, Lf, g);
    int64_t N = (d == 1) ? n : (int64_t)n * n;
    double *cur = malloc(sizeof(double) * N), *tmp = malloc(sizeof(double) * N);
    memcpy(cur, f, sizeof(double) * N);
    for (int j = 1; j <= L; ++j) {
        int64_t M = n >> (j - 1), Mh = M / 2;           /* current LL is M^d */
        if (d == 1) {
            /* a -> tmp[0..Mh), detail -> c[Mh .. 2Mh) = level j detail slot */
            analysis_line(h, g, Lf, M, cur, 1, tmp, c + Mh, 1);
            memcpy(cur, tmp, sizeof(double) * Mh);
        } else {
            /* axis 1 on every row: low -> tmp[r][0..Mh), high -> tmp[r][Mh..M) */
            for (int64_t r0 = 0; r0 < M; ++r0)
                analysis_line(h, g, Lf, M, cur + r0 * M, 1, tmp + r0 * M, tmp + r0 * M + Mh, 1);
            /* axis 0 on every column of both halves */
            int64_t Nb = Mh * Mh;                       /* band size at level j */
            double *LL = malloc(sizeof(double) * Nb);
            for (int64_t q1 = 0; q1 < Mh; ++q1) {
                /* low half column q1 (e1=0): axis0 low -> LL, axis0 high -> band (1,0) */
                analysis_line(h, g, Lf, M, tmp + q1, M, LL + q1, c + Nb + 1 * Nb + q1, Mh);
                /* high half column (e1=1): axis0 low -> band (0,1), high -> band (1,1) */
                analysis_line(h, g, Lf, M, tmp + Mh + q1, M, c + Nb + 0 * Nb + q1, c + Nb + 2 * Nb + q1, Mh);
            }
            memcpy(cur, LL, sizeof(double) * Nb);
            free(LL);
        }
    }
    int64_t NL = (d == 1) ? (n >> L) : (int64_t)(n >> L) * (n >> L);
    memcpy(c, cur, sizeof(double) * NL);
    free(cur);
    free(tmp);
    return 0;
}

/* inverse transform Psi: c (canonical) -> f (pixels) */
int or_idwt(int d, int n, int L, int wcode, const double *c, double *f)
{
    double h[OR_MAXTAPS], g[OR_MAXTAPS];
    int Lf = filter_taps(wcode, h);
    if (Lf < 0 || (n >> L) < 1 || (d != 1 && d != 2)) return -1;
    highpass(h, Lf, g);
    int64_t N = (d == 1) ? n : (int64_t)n * n;
    double *cur = malloc(sizeof(double) * N), *tmp = malloc(sizeof(double) * N);
    int64_t NL = (d == 1) ? (n >> L) : (int64_t)(n >> L) * (n >> L);
    memcpy(cur, c, sizeof(double) * NL);
    for (int j = L; j >= 1; --j) {
        int64_t M = n >> (j - 1), Mh = M / 2;
        if (d == 1) {
            synthesis_line(h, g, Lf, M, cur, c + Mh, 1, tmp, 1);
            memcpy(cur, tmp, sizeof(double) * M);
        } else {
            int64_t Nb = Mh * Mh;
            /* undo axis 0: columns of the low half from (LL, (1,0)), high half from ((0,1), (1,1)) */
            for (int64_t q1 = 0; q1 < Mh; ++q1) {
                synthesis_line(h, g, Lf, M, cur + q1, c + Nb + 1 * Nb + q1, Mh, tmp + q1, M);
                synthesis_line(h, g, Lf, M, c + Nb + 0 * Nb + q1, c + Nb + 2 * Nb + q1, Mh, tmp + Mh + q1, M);
            }
            /* undo axis 1 on every row */
            for (int64_t r0 = 0; r0 < M; ++r0)
                synthesis_line(h, g, Lf, M, tmp + r0 * M, tmp + r0 * M + Mh, 1, cur + r0 * M, 1);
            /* cur now holds the M x M LL of level j-1 (row stride M) */
        }
    }
    memcpy(f, cur, sizeof(double) * N);
    free(cur);
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Product-convolution operator applied to one signal (Eq. (2)), direct periodic
 * convolution: (u * f)(y) = sum_t u(t) f(y - t), evaluated as the scatter
 * w(x + t) += u(t) f(x) over the x where f(x) != 0.
 * ---------------------------------------------------------------------------------- */
static void scatter_conv(int d, int n, int r, const double *u, const double *f, double *w)
{
    int K = 2 * r + 1;
    int64_t N = (d == 1) ? n : (int64_t)n * n;
    for (int64_t x = 0; x < N; ++x) {
        double fx = f[x];
        if (fx == 0.0) continue;
        if (d == 1) {
            for (int t = -r; t <= r; ++t) w[pmod(x + t, n)] += u[t + r] * fx;
        } else {
            int64_t x0 = x / n, x1 = x % n;
            for (int t0 = -r; t0 <= r; ++t0)
                for (int t1 = -r; t1 <= r; ++t1)
                    w[pmod(x0 + t0, n) * n + pmod(x1 + t1, n)] += u[(t0 + r) * K + (t1 + r)] * fx;
        }
    }
}

int or_pc_apply(int d, int n, int m, int r, int order, const double *u, const double *v,
                const double *f, double *w)
{
    int64_t N = (d == 1) ? n : (int64_t)n * n;
    int64_t Ku = (d == 1) ? (2 * r + 1) : (int64_t)(2 * r + 1) * (2 * r + 1);
    double *t = malloc(sizeof(double) * N), *c = malloc(sizeof(double) * N);
    for (int64_t x = 0; x < N; ++x) w[x] = 0.0;
    for (int k = 0; k < m; ++k) {
        const double *uk = u + k * Ku, *vk = v + k * N;
        if (order == 0) {                    /* u_k * (v_k . f) */
            for (int64_t x = 0; x < N; ++x) t[x] = vk[x] * f[x];
            scatter_conv(d, n, r, uk, t, w);
        } else {                             /* v_k . (u_k * f) */
            for (int64_t x = 0; x < N; ++x) c[x] = 0.0;
            scatter_conv(d, n, r, uk, f, c);
            for (int64_t x = 0; x < N; ++x) w[x] += vk[x] * c[x];
        }
    }
    free(t);
    free(c);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Algorithm 2 (Section 4.2): for each requested lambda, psi_lambda = Psi e_lambda,
 * w = H psi_lambda, column lambda of Theta = Psi^* w.  out is ncols x N (column-major
 * by requested column: out[c*N + mu] = Theta[mu, cols[c]]).
 * ---------------------------------------------------------------------------------- */
int or_theta_columns(int d, int n, int L, int wcode, int m, int r, int order,
                     const double *u, const double *v, int64_t ncols, const int64_t *cols,
                     double *out, int nthreads)
{
    int64_t N = (d == 1) ? n : (int64_t)n * n;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *e = calloc(N, sizeof(double)), *psi = malloc(sizeof(double) * N),
               *w = malloc(sizeof(double) * N);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t c = 0; c < ncols; ++c) {
            int64_t lam = cols[c];
            if (lam < 0 || lam >= N) { bad = 1; continue; }
            e[lam] = 1.0;
            or_idwt(d, n, L, wcode, e, psi);
            e[lam] = 0.0;
            or_pc_apply(d, n, m, r, order, u, v, psi, w);
            or_dwt(d, n, L, wcode, w, out + c * N);
        }
        free(e);
        free(psi);
        free(w);
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------------------
 * Basis index <-> (level, band, translate) and the prescribed pattern.
 * ---------------------------------------------------------------------------------- */
/* returns level j (1..L; approximation band reported as level L) and e0, e1, l0, l1 */
static void decode(int d, int n, int L, int64_t idx, int *j, int *e0, int *e1, int64_t *l0, int64_t *l1)
{
    int64_t nL = n >> L;
    if (d == 1) {
        *e0 = 0;
        *l0 = 0;
        if (idx < nL) { *j = L; *e1 = 0; *l1 = idx; return; }
        for (int jj = L; jj >= 1; --jj) {
            int64_t nj = n >> jj;
            if (idx >= nj && idx < 2 * nj) { *j = jj; *e1 = 1; *l1 = idx - nj; return; }
        }
    } else {
        if (idx < nL * nL) { *j = L; *e0 = 0; *e1 = 0; *l0 = idx / nL; *l1 = idx % nL; return; }
        for (int jj = L; jj >= 1; --jj) {
            int64_t nj = n >> jj, Nb = nj * nj;
            if (idx >= Nb && idx < 4 * Nb) {
                int64_t b = (idx - Nb) / Nb, l = (idx - Nb) % Nb;
                *j = jj;
                *e0 = (b >= 1) ? 1 : 0;
                *e1 = (b == 1) ? 0 : 1;
                *l0 = l / nj;
                *l1 = l % nj;
                return;
            }
        }
    }
    *j = -1;
}

/* closed support [lo, hi] (unwrapped) of the 1-D factor rho^e_{j,l}:
 * phi_{j,l}: 2^j l + [0, (2^j-1)(Lf-1)],  psi_{j,l}: 2^j l + 2^(j-1)(2-Lf) + [0, (2^j-1)(Lf-1)] */
static void support(int j, int e, int64_t l, int Lf, int64_t *lo, int64_t *hi)
{
    int64_t len = ((int64_t)1 << j) - 1;
    len = len * (Lf - 1) + 1;
    int64_t a = e ? ((int64_t)1 << (j - 1)) * (2 - Lf) : 0;
    *lo = ((int64_t)1 << j) * l + a;
    *hi = *lo + len - 1;
}

/* 1 if some periodic image of [B0,B1] meets [A0-r, A1+r] on the circle of length n */
static int near_on_circle(int64_t A0, int64_t A1, int64_t B0, int64_t B1, int r, int n)
{
    int64_t span = (A1 - A0) + (B1 - B0) + 2 * r + llabs(A0) + llabs(B0);
    int64_t P = span / n + 2;
    for (int64_t p = -P; p <= P; ++p)
        if (B0 + p * n <= A1 + r && B1 + p * n >= A0 - r) return 1;
    return 0;
}

/* (mu, lambda) in P: gap < 0 keeps everything; otherwise | |mu| - |lambda| | <= gap and,
 * on every axis, the supports of psi_mu and psi_lambda are within r of each other on the
 * torus (entries failing this are exactly zero: the kernels have radius r). */
int or_in_pattern(int d, int n, int L, int wcode, int r, int gap, int64_t mu, int64_t lam)
{
    const int delta = wcode % 100;
    if (gap < 0) return 1;
    int Lf = 2 * delta;
    int jm, e0m, e1m, jl, e0l, e1l;
    int64_t l0m, l1m, l0l, l1l;
    decode(d, n, L, mu, &jm, &e0m, &e1m, &l0m, &l1m);
    decode(d, n, L, lam, &jl, &e0l, &e1l, &l0l, &l1l);
    if (jm < 0 || jl < 0) return -1;
    if (abs(jm - jl) > gap) return 0;
    int64_t A0, A1, B0, B1;
    support(jm, e1m, l1m, Lf, &A0, &A1);
    support(jl, e1l, l1l, Lf, &B0, &B1);
    if (!near_on_circle(A0, A1, B0, B1, r, n)) return 0;
    if (d == 2) {
        support(jm, e0m, l0m, Lf, &A0, &A1);
        support(jl, e0l, l0l, Lf, &B0, &B1);
        if (!near_on_circle(A0, A1, B0, B1, r, n)) return 0;
    }
    return 1;
}

int or_pattern_mask(int d, int n, int L, int wcode, int r, int gap, int64_t lam,
                    unsigned char *mask)
{
    int64_t N = (d == 1) ? n : (int64_t)n * n;
    for (int64_t mu = 0; mu < N; ++mu) mask[mu] = (unsigned char)or_in_pattern(d, n, L, wcode, r, gap, mu, lam);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Gradient of a loss of Theta restricted to given columns.  G is ncols x N (caller has
 * zeroed the entries outside the pattern).  With g = Psi G[:, lambda] (adjoint of the
 * forward transform) and w = H psi_lambda:
 *   order 0: dL/du_k(t) += sum_y g(y) (v_k psi)(y - t),  dL/dv_k(y) += psi(y) sum_t u_k(t) g(y + t)
 *   order 1: dL/du_k(t) += sum_y g(y) v_k(y) psi(y - t), dL/dv_k(y) += g(y) (u_k * psi)(y)
 * du (m x K) and dv (m x N) are overwritten.
 * ---------------------------------------------------------------------------------- */
int or_theta_grad(int d, int n, int L, int wcode, int m, int r, int order,
                  const double *u, const double *v, int64_t ncols, const int64_t *cols,
                  const double *G, double *du, double *dv, int nthreads)
{
    int64_t N = (d == 1) ? n : (int64_t)n * n;
    int K = 2 * r + 1;
    int64_t Ku = (d == 1) ? K : (int64_t)K * K;
    for (int64_t i = 0; i < m * Ku; ++i) du[i] = 0.0;
    for (int64_t i = 0; i < m * N; ++i) dv[i] = 0.0;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *e = calloc(N, sizeof(double)), *psi = malloc(sizeof(double) * N),
               *g = malloc(sizeof(double) * N), *c = malloc(sizeof(double) * N),
               *du_t = calloc(m * Ku, sizeof(double)), *dv_t = calloc(m * N, sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t ci = 0; ci < ncols; ++ci) {
            int64_t lam = cols[ci];
            if (lam < 0 || lam >= N) { bad = 1; continue; }
            e[lam] = 1.0;
            or_idwt(d, n, L, wcode, e, psi);
            e[lam] = 0.0;
            or_idwt(d, n, L, wcode, G + ci * N, g);
            for (int k = 0; k < m; ++k) {
                const double *uk = u + k * Ku, *vk = v + k * N;
                double *duk = du_t + k * Ku, *dvk = dv_t + k * N;
                for (int64_t x = 0; x < N; ++x) {
                    if (psi[x] == 0.0) continue;
                    int64_t x0 = (d == 1) ? 0 : x / n, x1 = (d == 1) ? x : x % n;
                    for (int t0 = (d == 1 ? 0 : -r); t0 <= (d == 1 ? 0 : r); ++t0)
                        for (int t1 = -r; t1 <= r; ++t1) {
                            int64_t y = (d == 1) ? pmod(x1 + t1, n) : pmod(x0 + t0, n) * n + pmod(x1 + t1, n);
                            int64_t ti = (d == 1) ? (t1 + r) : (int64_t)(t0 + r) * K + (t1 + r);
                            if (order == 0) {
                                /* y = x + t: du(t) += g(x+t) v(x) psi(x);  dv(x) += psi(x) u(t) g(x+t) */
                                duk[ti] += g[y] * vk[x] * psi[x];
                                dvk[x] += psi[x] * uk[ti] * g[y];
                            } else {
                                /* du(t) += g(x+t) v(x+t) psi(x) */
                                duk[ti] += g[y] * vk[y] * psi[x];
                            }
                        }
                }
                if (order == 1) {
                    for (int64_t x = 0; x < N; ++x) c[x] = 0.0;
                    scatter_conv(d, n, r, uk, psi, c);
                    for (int64_t x = 0; x < N; ++x) dvk[x] += g[x] * c[x];
                }
            }
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            for (int64_t i = 0; i < m * Ku; ++i) du[i] += du_t[i];
            for (int64_t i = 0; i < m * N; ++i) dv[i] += dv_t[i];
        }
        free(e); free(psi); free(g); free(c); free(du_t); free(dv_t);
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------------------
 * Deblurring in the wavelet domain (Section 4.3, problem min_z 1/2 ||Theta z - z0||^2 +
 * ||z||_{1,w}, and the FISTA iteration of the appendix on deblurring algorithms).
 * Theta is a dense row-major N x N array here: Theta[mu * N + lambda].
 * ------------------------------------------------------------------------------------ */

/* y = Theta x */
static void dense_mv(int64_t N, const double *T, const double *x, double *y)
{
    for (int64_t mu = 0; mu < N; ++mu) {
        double acc = 0.0;
        for (int64_t la = 0; la < N; ++la) acc += T[mu * N + la] * x[la];
        y[mu] = acc;
    }
}

/* y = Theta^T x */
static void dense_mtv(int64_t N, const double *T, const double *x, double *y)
{
    for (int64_t la = 0; la < N; ++la) y[la] = 0.0;
    for (int64_t mu = 0; mu < N; ++mu)
        for (int64_t la = 0; la < N; ++la) y[la] += T[mu * N + la] * x[mu];
}

/* Jacobi diagonal diag(Theta^T Theta): out[lambda] = sum_mu Theta[mu, lambda]^2 (the
 * preconditioner of FISTA-WP). */
int or_jacobi(int64_t N, const double *T, double *out)
{
    for (int64_t la = 0; la < N; ++la) {
        double acc = 0.0;
        for (int64_t mu = 0; mu < N; ++mu) acc += T[mu * N + la] * T[mu * N + la];
        out[la] = acc;
    }
    return 0;
}

/* Power iteration for the largest eigenvalue of M = S^(1/2) Theta^T Theta S^(1/2), with
 * S = diag(sigma) (identity when sigma is NULL); its inverse bounds the FISTA step.
 * Start u = (1, ..., 1) / sqrt(N); each iteration g = M u, estimate = ||g||, u = g / ||g||.
 * Writes the last estimate to *out. */
int or_power_norm(int64_t N, const double *T, const double *sigma, int iters, double *out)
{
    double *u = malloc(sizeof(double) * N), *r = malloc(sizeof(double) * N), *g = malloc(sizeof(double) * N);
    if (!u || !r || !g) { free(u); free(r); free(g); return -1; }
    for (int64_t i = 0; i < N; ++i) u[i] = 1.0 / sqrt((double)N);
    double est = 0.0;
    for (int it = 0; it < iters; ++it) {
        if (sigma)
            for (int64_t i = 0; i < N; ++i) u[i] *= sqrt(sigma[i]);
        dense_mv(N, T, u, r);
        dense_mtv(N, T, r, g);
        if (sigma)
            for (int64_t i = 0; i < N; ++i) g[i] *= sqrt(sigma[i]);
        double s = 0.0;
        for (int64_t i = 0; i < N; ++i) s += g[i] * g[i];
        est = sqrt(s);
        for (int64_t i = 0; i < N; ++i) u[i] = (s > 0.0) ? g[i] / est : 0.0;
    }
    *out = est;
    free(u); free(r); free(g);
    return 0;
}

/* FISTA in the wavelet domain: z holds z^(0) = y^(1) on entry and z^(iters) on return.
 * For i = 1..iters:
 *   z^(i)   = Prox^S (y^(i) - tau S Theta^T (Theta y^(i) - z0)),
 *   y^(i+1) = z^(i) + (i - 1) / (i + 2) (z^(i) - z^(i-1)),
 * with S = diag(sigma) (identity when sigma is NULL: FISTA-W; else FISTA-WP) and the prox of
 * tau ||.||_{1,w} in the metric S^-1: soft thresholding of entry lambda at tau sigma[lambda]
 * w[lambda]. */
int or_fista(int64_t N, const double *T, const double *z0, const double *w, const double *sigma,
             int iters, double tau, double *z)
{
    double *y = malloc(sizeof(double) * N), *r = malloc(sizeof(double) * N), *g = malloc(sizeof(double) * N);
    if (!y || !r || !g) { free(y); free(r); free(g); return -1; }
    for (int64_t i = 0; i < N; ++i) y[i] = z[i];
    for (int it = 1; it <= iters; ++it) {
        dense_mv(N, T, y, r);
        for (int64_t mu = 0; mu < N; ++mu) r[mu] -= z0[mu];
        dense_mtv(N, T, r, g);
        const double beta = (double)(it - 1) / (double)(it + 2);
        for (int64_t la = 0; la < N; ++la) {
            const double s = sigma ? sigma[la] : 1.0;
            const double a = y[la] - tau * s * g[la];
            const double t = tau * s * w[la];
            const double zn = (a > t) ? a - t : (a < -t) ? a + t : 0.0;
            y[la] = zn + beta * (zn - z[la]);
            z[la] = zn;
        }
    }
    free(y); free(r); free(g);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Algorithm 1 (Section 3.2) with thresholding, on dense matrices (small N only).
 *   eps_k = eta / (m ||v_k||_inf);  A_k = Psi^* U_k Psi;  B_k = Psi^* V_k Psi;
 *   A~_k = A_k with the entries below a threshold tau_k set to 0.  rule 0: tau_k the largest
 *          value whose discarded part D_k has Schur bound sqrt(||D_k||_1 ||D_k||_inf) <= eps_k
 *          (so ||A_k - A~_k||_2 <= eps_k; bisection on tau, 80 halvings).  rule 1: tau_k = eps_k
 *          (the threshold step read as a plain cut at eps_k; no 2-norm certificate);
 *   Theta~ = sum_k A~_k B_k  (paper order; B_k A~_k in the convolution-first order).
 * Rule 0: since ||B_k||_2 = ||v_k||_inf, ||Theta - Theta~||_2 <= sum_k eps_k ||v_k||_inf = eta.
 * theta: N x N row-major Theta~[mu * N + lambda]; nnz_a[k] = entries kept in A~_k;
 * tau[k] = the threshold.  Returns 0, or -1 on bad input or allocation failure.
 * ------------------------------------------------------------------------------------ */
static double schur_discard(int64_t N, const double *A, double t, double *rs, double *cs)
{
    for (int64_t i = 0; i < N; ++i) { rs[i] = 0.0; cs[i] = 0.0; }
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            const double a = fabs(A[i * N + j]);
            if (a < t) { rs[i] += a; cs[j] += a; }
        }
    double mr = 0.0, mc = 0.0;
    for (int64_t i = 0; i < N; ++i) { mr = fmax(mr, rs[i]); mc = fmax(mc, cs[i]); }
    return sqrt(mr * mc);
}

int or_alg1_dense(int d, int n, int L, int wcode, int m, int r, int order, const double *u, const double *v,
                  double eta, int rule, double *theta, int64_t *nnz_a, double *tau)
{
    const int64_t N = (d == 1) ? n : (int64_t)n * n;
    const int64_t Ku = (d == 1) ? (2 * r + 1) : (int64_t)(2 * r + 1) * (2 * r + 1);
    if (N > 4096 || m < 1 || eta < 0.0 || (rule != 0 && rule != 1)) return -1;
    double *colsA = malloc(sizeof(double) * N * N), *colsB = malloc(sizeof(double) * N * N);
    double *A = malloc(sizeof(double) * N * N), *B = malloc(sizeof(double) * N * N);
    double *ones = malloc(sizeof(double) * N), *rs = malloc(sizeof(double) * N), *cs = malloc(sizeof(double) * N);
    int64_t *all = malloc(sizeof(int64_t) * N);
    if (!colsA || !colsB || !A || !B || !ones || !rs || !cs || !all) {
        free(colsA); free(colsB); free(A); free(B); free(ones); free(rs); free(cs); free(all);
        return -1;
    }
    for (int64_t i = 0; i < N; ++i) { ones[i] = 1.0; all[i] = i; }
    for (int64_t i = 0; i < N * N; ++i) theta[i] = 0.0;
    const double delta1 = 1.0;   /* the point kernel of the multiplier */
    int rc = 0;
    for (int k = 0; k < m && rc == 0; ++k) {
        double vmax = 0.0;
        for (int64_t x = 0; x < N; ++x) vmax = fmax(vmax, fabs(v[k * N + x]));
        /* A_k = Psi^* U_k Psi (columns of the one-term operator u_k * (1 . f)) */
        rc |= or_theta_columns(d, n, L, wcode, 1, r, 0, u + k * Ku, ones, N, all, colsA, 0);
        /* B_k = Psi^* V_k Psi (columns of the one-term operator delta * (v_k . f)) */
        rc |= or_theta_columns(d, n, L, wcode, 1, 0, 0, &delta1, v + k * N, N, all, colsB, 0);
        if (rc) break;
        for (int64_t mu = 0; mu < N; ++mu)
            for (int64_t la = 0; la < N; ++la) {
                A[mu * N + la] = colsA[la * N + mu];
                B[mu * N + la] = colsB[la * N + mu];
            }
        /* threshold by bisection on tau */
        const double eps = (vmax > 0.0) ? eta / (m * vmax) : 1e300;
        double amax = 0.0;
        for (int64_t i = 0; i < N * N; ++i) amax = fmax(amax, fabs(A[i]));
        double t;
        const double top = amax * (1.0 + 1e-15) + 1e-300;
        if (rule == 1) {
            t = eps;
        } else if (schur_discard(N, A, top, rs, cs) <= eps) {
            t = top;
        } else {
            double lo = 0.0, hi = top;
            for (int it = 0; it < 80; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (schur_discard(N, A, mid, rs, cs) <= eps) lo = mid; else hi = mid;
            }
            t = lo;
        }
        tau[k] = t;
        int64_t kept = 0;
        for (int64_t i = 0; i < N * N; ++i) {
            if (fabs(A[i]) < t) A[i] = 0.0; else ++kept;
        }
        nnz_a[k] = kept;
        /* C_k = A~_k B_k (paper order) or B_k A~_k (convolution first), accumulated */
        const double *P1 = (order == 0) ? A : B, *P2 = (order == 0) ? B : A;
        for (int64_t mu = 0; mu < N; ++mu)
            for (int64_t q = 0; q < N; ++q) {
                const double a = P1[mu * N + q];
                if (a == 0.0) continue;
                for (int64_t la = 0; la < N; ++la) theta[mu * N + la] += a * P2[q * N + la];
            }
    }
    free(colsA); free(colsB); free(A); free(B); free(ones); free(rs); free(cs); free(all);
    return rc ? -1 : 0;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
