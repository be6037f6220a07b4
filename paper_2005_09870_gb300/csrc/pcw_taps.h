// Daubechies and Symmlet low-pass filter taps on the host, FP64.
//
// Section 2.1: the orthogonal wavelets come from a filter bank (h, g) with supp h =
// [0, 2 delta - 1], delta vanishing moments, and g[i] = (-1)^(1-i) h[1-i].  The taps are the
// minimum-phase spectral factor of |m0(w)|^2 = cos^(2 delta)(w/2) P(sin^2(w/2)), with
// P(y) = sum_{k<delta} C(delta-1+k, k) y^k (Daubechies' construction).  Roots of P are
// found by Laguerre iteration with deflation, polished by Newton on the full polynomial.
#pragma once
#include <complex>
#include <cmath>
#include <vector>

namespace pcw {

inline std::complex<double> poly_eval(const std::vector<std::complex<double>>& c,
                                      std::complex<double> x, std::complex<double>* d1,
                                      std::complex<double>* d2)
{
    // c[k] is the coefficient of x^k; returns p(x), p'(x), p''(x)
    std::complex<double> p = 0.0, dp = 0.0, ddp = 0.0;
    for (int k = (int)c.size() - 1; k >= 0; --k) {
        ddp = ddp * x + 2.0 * dp;
        dp = dp * x + p;
        p = p * x + c[k];
    }
    if (d1) *d1 = dp;
    if (d2) *d2 = ddp;
    return p;
}

inline std::complex<double> laguerre(const std::vector<std::complex<double>>& c,
                                     std::complex<double> x)
{
    const double deg = (double)c.size() - 1;
    for (int it = 0; it < 500; ++it) {
        std::complex<double> d1, d2;
        std::complex<double> p = poly_eval(c, x, &d1, &d2);
        if (std::abs(p) < 1e-300) return x;
        std::complex<double> G = d1 / p, H = G * G - d2 / p;
        std::complex<double> sq = std::sqrt((deg - 1.0) * (deg * H - G * G));
        std::complex<double> den = (std::abs(G + sq) > std::abs(G - sq)) ? G + sq : G - sq;
        std::complex<double> step = (std::abs(den) > 0) ? deg / den : std::complex<double>(1e-3, 1e-3);
        x -= step;
        if (std::abs(step) < 1e-16 * (1.0 + std::abs(x))) break;
    }
    return x;
}

// Roots y_i of P(y) = sum_{k<delta} C(delta-1+k, k) y^k: Laguerre with deflation, then a
// Newton polish on P.
inline std::vector<std::complex<double>> p_roots(int delta)
{
    std::vector<std::complex<double>> P(delta);
    for (int k = 0; k < delta; ++k) {
        double b = 1.0;  // C(delta-1+k, k)
        for (int i = 1; i <= k; ++i) b = b * (double)(delta - 1 + i) / (double)i;
        P[k] = b;
    }
    std::vector<std::complex<double>> roots, work = P;
    while (work.size() > 1) {
        std::complex<double> z = laguerre(work, std::complex<double>(-0.3, 0.2));
        roots.push_back(z);
        // synthetic division by (x - z)
        std::vector<std::complex<double>> q(work.size() - 1);
        std::complex<double> carry = work.back();
        for (int k = (int)work.size() - 2; k >= 0; --k) {
            q[k] = carry;
            carry = work[k] + carry * z;
        }
        work.swap(q);
    }
    for (auto& z : roots)
        for (int it = 0; it < 5; ++it) {
            std::complex<double> d1;
            std::complex<double> p = poly_eval(P, z, &d1, nullptr);
            if (std::abs(d1) > 0) z -= p / d1;
        }
    return roots;
}

// The root of z^2 - (2 - 4y) z + 1 = 0 outside the unit circle (z + 1/z = 2 - 4y).
inline std::complex<double> outer_root(std::complex<double> y)
{
    const std::complex<double> b = 2.0 - 4.0 * y;
    const std::complex<double> s = std::sqrt(b * b - 4.0);
    std::complex<double> z = 0.5 * (b + s);
    if (std::abs(z) < 1.0) z = 0.5 * (b - s);
    return z;
}

// h[n] = coefficient of z^n in (1 + z)^delta prod_i (z - z_i), scaled to sum sqrt 2.
inline int taps_of(int delta, const std::vector<std::complex<double>>& zs, double* h)
{
    std::vector<std::complex<double>> poly(1, 1.0);
    auto mul_linear = [&](std::complex<double> c0, std::complex<double> c1) {  // * (c0 + c1 z)
        std::vector<std::complex<double>> out(poly.size() + 1, 0.0);
        for (size_t i = 0; i < poly.size(); ++i) {
            out[i] += poly[i] * c0;
            out[i + 1] += poly[i] * c1;
        }
        poly.swap(out);
    };
    for (int k = 0; k < delta; ++k) mul_linear(1.0, 1.0);
    for (auto z : zs) mul_linear(-z, 1.0);
    const int Lf = (int)poly.size();
    double sum = 0.0;
    for (int i = 0; i < Lf; ++i) sum += poly[i].real();
    for (int i = 0; i < Lf; ++i) h[i] = poly[i].real() * std::sqrt(2.0) / sum;
    return Lf;
}

// Daubechies (minimum phase): every z_i outside the unit circle.  Fills h with 2*delta
// taps; returns the tap count, or -1 for an unsupported delta.
inline int daubechies_taps(int delta, double* h)
{
    if (delta < 1 || delta > 20) return -1;
    std::vector<std::complex<double>> zs;
    if (delta > 1)
        for (auto y : p_roots(delta)) zs.push_back(outer_root(y));
    return taps_of(delta, zs, h);
}

// Symmlet (least asymmetric; the basis of Section 4.3): the same |m0|^2, with z_i or 1/z_i
// per root of P (one choice per conjugate pair, so the taps stay real) chosen to make the
// phase of prod_i (e^{-iw} - z_i) closest to linear: the smallest mean squared residual of
// its least-squares line over w_k = (k + 1/2) pi / 512, k < 512.  A choice and its mirror
// (all roots inverted) tie; ties within 1e-9 (relative) go to the smaller energy centre
// sum_n n h[n]^2.  Returns the tap count, or -1 for an unsupported delta.
inline int symmlet_taps(int delta, double* h)
{
    if (delta < 1 || delta > 20) return -1;
    if (delta == 1) return daubechies_taps(1, h);
    const std::vector<std::complex<double>> ys = p_roots(delta);
    // one representative per real root and per conjugate pair (the member with Im > 0)
    std::vector<std::complex<double>> rep;
    std::vector<bool> pair;
    for (auto y : ys) {
        const double tol = 1e-9 * (1.0 + std::abs(y));
        if (std::abs(y.imag()) <= tol) {
            rep.push_back(y);
            pair.push_back(false);
        } else if (y.imag() > 0.0) {
            rep.push_back(y);
            pair.push_back(true);
        }
    }
    const int ng = (int)rep.size();
    constexpr int KW = 512;
    const double pi = 3.14159265358979323846;
    double best_r = 0.0, best_c = 0.0;
    bool have = false;
    std::vector<double> hb(2 * delta), ht(2 * delta);
    for (long mask = 0; mask < (1L << ng); ++mask) {
        std::vector<std::complex<double>> zs;
        for (int g = 0; g < ng; ++g) {
            std::complex<double> z = outer_root(rep[g]);
            if ((mask >> g) & 1) z = 1.0 / z;
            zs.push_back(z);
            if (pair[g]) zs.push_back(std::conj(z));
        }
        if (taps_of(delta, zs, ht.data()) != 2 * delta) return -1;
        // phase of prod_i (e^{-iw} - z_i), continued along the grid by the argument of the
        // ratio of consecutive factor values (each step well below pi)
        std::vector<double> ph(KW, 0.0);
        for (auto z : zs) {
            std::complex<double> prev = std::exp(std::complex<double>(0.0, -0.5 * pi / KW)) - z;
            double acc = std::arg(prev);
            ph[0] += acc;
            for (int k = 1; k < KW; ++k) {
                const std::complex<double> cur = std::exp(std::complex<double>(0.0, -(k + 0.5) * pi / KW)) - z;
                acc += std::arg(cur / prev);
                ph[k] += acc;
                prev = cur;
            }
        }
        // residual of the least-squares line (centred form)
        double wm = 0.0, pm = 0.0;
        for (int k = 0; k < KW; ++k) {
            wm += (k + 0.5) * pi / KW;
            pm += ph[k];
        }
        wm /= KW;
        pm /= KW;
        double sxx = 0.0, sxy = 0.0;
        for (int k = 0; k < KW; ++k) {
            const double dw = (k + 0.5) * pi / KW - wm;
            sxx += dw * dw;
            sxy += dw * (ph[k] - pm);
        }
        const double slope = sxy / sxx;
        double r = 0.0;
        for (int k = 0; k < KW; ++k) {
            const double e = (ph[k] - pm) - slope * ((k + 0.5) * pi / KW - wm);
            r += e * e;
        }
        r /= KW;
        double cen = 0.0;
        for (int n = 0; n < 2 * delta; ++n) cen += n * ht[n] * ht[n];
        const bool tie = have && std::abs(r - best_r) <= 1e-9 * best_r;
        if (!have || (r < best_r && !tie) || (tie && cen < best_c)) {
            if (!tie) best_r = r;
            best_c = cen;
            hb = ht;
            have = true;
        }
    }
    for (int n = 0; n < 2 * delta; ++n) h[n] = hb[n];
    return 2 * delta;
}

// Taps of the filter family (0 Daubechies, 1 Symmlet) of order delta.
inline int filter_taps(int family, int delta, double* h)
{
    if (family == 0) return daubechies_taps(delta, h);
    if (family == 1) return symmlet_taps(delta, h);
    return -1;
}

}  // namespace pcw
