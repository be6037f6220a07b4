// Host FP64 linear algebra for the randomized-SVD construction of a product-convolution
// expansion (pc_svir_expansion): the small factorisations of the range finder and of the
// projected matrix.  Sizes are the sketch width l = m + oversampling (<= 64) and the stencil
// size K (<= 961 for 31 x 31 kernels), so plain loops suffice.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

namespace pcw {

// Cholesky factor of the symmetric positive definite l x l matrix G (row-major): G = R^T R with
// R upper triangular (returned row-major).  Returns false when a pivot is not positive.
inline bool cholesky_upper(const std::vector<double>& G, int l, std::vector<double>* R)
{
    R->assign((size_t)l * l, 0.0);
    std::vector<double>& r = *R;
    for (int i = 0; i < l; ++i) {
        double d = G[(size_t)i * l + i];
        for (int k = 0; k < i; ++k) d -= r[(size_t)k * l + i] * r[(size_t)k * l + i];
        if (!(d > 0.0)) return false;
        const double rii = std::sqrt(d);
        r[(size_t)i * l + i] = rii;
        for (int j = i + 1; j < l; ++j) {
            double s = G[(size_t)i * l + j];
            for (int k = 0; k < i; ++k) s -= r[(size_t)k * l + i] * r[(size_t)k * l + j];
            r[(size_t)i * l + j] = s / rii;
        }
    }
    return true;
}

// Inverse of an upper triangular l x l matrix (row-major), by back substitution per column.
inline std::vector<double> upper_inverse(const std::vector<double>& R, int l)
{
    std::vector<double> X((size_t)l * l, 0.0);
    for (int c = 0; c < l; ++c) {
        for (int i = c; i >= 0; --i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = i + 1; k <= c; ++k) s -= R[(size_t)i * l + k] * X[(size_t)k * l + c];
            X[(size_t)i * l + c] = s / R[(size_t)i * l + i];
        }
    }
    return X;
}

// Singular value decomposition of the l x K matrix B (row-major) by one-sided Jacobi rotations
// (Hestenes) on the columns of A = B^T (K x l): rotate column pairs until every pair is
// orthogonal to relative precision, then A = W diag(s) U^T with s the column norms.  Returns
// s (descending), U (l x l, row-major: B = U diag(s) W^T, column j of U is the left singular
// vector j of B) and W (K x l, row-major: column j is the right singular vector j).
inline void jacobi_svd(const std::vector<double>& B, int l, int K, std::vector<double>* s, std::vector<double>* U,
                       std::vector<double>* W)
{
    std::vector<double> A((size_t)K * l), V((size_t)l * l, 0.0);
    for (int i = 0; i < l; ++i)
        for (int t = 0; t < K; ++t) A[(size_t)t * l + i] = B[(size_t)i * K + t];
    for (int i = 0; i < l; ++i) V[(size_t)i * l + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < l - 1; ++p)
            for (int q = p + 1; q < l; ++q) {
                double a = 0.0, b = 0.0, c = 0.0;
                for (int t = 0; t < K; ++t) {
                    const double x = A[(size_t)t * l + p], y = A[(size_t)t * l + q];
                    a += x * x;
                    b += y * y;
                    c += x * y;
                }
                if (c == 0.0) continue;
                const double rel = std::fabs(c) / std::sqrt(a * b);
                off = std::max(off, rel);
                if (rel < 1e-15) continue;
                // rotation that zeroes the (p, q) entry of A^T A
                const double zeta = (b - a) / (2.0 * c);
                const double tt = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / std::sqrt(1.0 + tt * tt), sn = cs * tt;
                for (int t = 0; t < K; ++t) {
                    const double x = A[(size_t)t * l + p], y = A[(size_t)t * l + q];
                    A[(size_t)t * l + p] = cs * x - sn * y;
                    A[(size_t)t * l + q] = sn * x + cs * y;
                }
                for (int t = 0; t < l; ++t) {
                    const double x = V[(size_t)t * l + p], y = V[(size_t)t * l + q];
                    V[(size_t)t * l + p] = cs * x - sn * y;
                    V[(size_t)t * l + q] = sn * x + cs * y;
                }
            }
        if (off < 1e-15) break;
    }
    std::vector<double> nrm(l);
    for (int j = 0; j < l; ++j) {
        double a = 0.0;
        for (int t = 0; t < K; ++t) a += A[(size_t)t * l + j] * A[(size_t)t * l + j];
        nrm[j] = std::sqrt(a);
    }
    std::vector<int> ord(l);
    for (int j = 0; j < l; ++j) ord[j] = j;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
    s->assign(l, 0.0);
    U->assign((size_t)l * l, 0.0);
    W->assign((size_t)K * l, 0.0);
    for (int jj = 0; jj < l; ++jj) {
        const int j = ord[jj];
        (*s)[jj] = nrm[j];
        for (int t = 0; t < l; ++t) (*U)[(size_t)t * l + jj] = V[(size_t)t * l + j];
        for (int t = 0; t < K; ++t) (*W)[(size_t)t * l + jj] = nrm[j] > 0.0 ? A[(size_t)t * l + j] / nrm[j] : 0.0;
    }
}

}  // namespace pcw
