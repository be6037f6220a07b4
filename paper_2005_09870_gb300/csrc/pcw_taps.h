// Daubechies low-pass filter taps on the host, FP64.
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

// Fills h with 2*delta taps; returns the tap count, or -1 for an unsupported delta.
inline int daubechies_taps(int delta, double* h)
{
    if (delta < 1 || delta > 20) return -1;
    const int Lf = 2 * delta;
    // P(y) coefficients
    std::vector<std::complex<double>> P(delta);
    for (int k = 0; k < delta; ++k) {
        double b = 1.0;  // C(delta-1+k, k)
        for (int i = 1; i <= k; ++i) b = b * (double)(delta - 1 + i) / (double)i;
        P[k] = b;
    }
    // roots of P by Laguerre + deflation, then Newton polish on P
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
    // sum_n h[n] z^n  proportional to  (1 + z)^delta  prod_i (z - z_i),  |z_i| > 1,
    // where z_i + 1/z_i = 2 - 4 y_i
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
    for (auto y : roots) {
        std::complex<double> b = 2.0 - 4.0 * y;
        std::complex<double> s = std::sqrt(b * b - 4.0);
        std::complex<double> z = 0.5 * (b + s);
        if (std::abs(z) < 1.0) z = 0.5 * (b - s);
        mul_linear(-z, 1.0);
    }
    double sum = 0.0;
    for (int i = 0; i < Lf; ++i) sum += poly[i].real();
    for (int i = 0; i < Lf; ++i) h[i] = poly[i].real() * std::sqrt(2.0) / sum;
    return Lf;
}

}  // namespace pcw
