// Product-convolution expansion of a space-varying blur by randomized SVD of its space-varying
// impulse response (the construction of Section 2.4; the randomized range finder of Halko,
// Martinsson and Tropp).  The tall products over the N pixels run as cuBLAS FP32 GEMMs on the
// device; the sketch-sized factorisations (l x l Gram matrices, the l x K projected matrix) run
// in FP64 on the host (pcw_svir.h).
#pragma once
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "pcw_svir.h"

namespace pcw {

// Row-major C (M x N) = op(A) (M x K) * op(B) (K x N) with cuBLAS (column-major): the row-major
// product is the column-major product C^T = op(B)^T op(A)^T.
inline cublasStatus_t gemm_rm(cublasHandle_t hb, bool ta, bool tb, int M, int N, int K, const float* A, int lda,
                              const float* B, int ldb, float* C, int ldc)
{
    const float one = 1.0f, zero = 0.0f;
    return cublasSgemm(hb, tb ? CUBLAS_OP_T : CUBLAS_OP_N, ta ? CUBLAS_OP_T : CUBLAS_OP_N, N, M, K, &one, B, ldb,
                       A, lda, &zero, C, ldc);
}

struct SvirWork {
    cublasHandle_t hb = nullptr;
    cudaStream_t st = nullptr;
    float* G = nullptr;  // l x l Gram matrix (device)
    float* T = nullptr;  // l x l transform (device)
    float* tmp = nullptr;  // rows x l scratch for the orthonormalised copy
    std::string err;
};

// Orthonormalises the first c columns of X (rows x c, row-major with row stride ld, device) in
// place by the Gram-matrix eigendecomposition (X^T X = E diag(lam) E^T, X <- X E diag(lam)^(-1/2)),
// twice; directions whose eigenvalue is below 1e-12 of the largest are dropped (a rank-deficient
// sketch).  Returns the number of columns kept (<= c), in the first columns; 0 on error.
inline int svir_orthonormalise(SvirWork& w, float* X, int64_t rows, int c, int ld)
{
    int keep = c;
    for (int pass = 0; pass < 2; ++pass) {
        if (gemm_rm(w.hb, true, false, keep, keep, (int)rows, X, ld, X, ld, w.G, keep) != CUBLAS_STATUS_SUCCESS) {
            w.err = "cuBLAS Gram product failed";
            return 0;
        }
        std::vector<float> gf((size_t)keep * keep);
        if (cudaMemcpyAsync(gf.data(), w.G, sizeof(float) * gf.size(), cudaMemcpyDeviceToHost, w.st) != cudaSuccess ||
            cudaStreamSynchronize(w.st) != cudaSuccess) {
            w.err = "Gram copy failed";
            return 0;
        }
        std::vector<double> G(gf.begin(), gf.end()), lam, E, E2;
        for (int i = 0; i < keep; ++i)  // symmetrise the FP32 product
            for (int j = 0; j < i; ++j) G[(size_t)i * keep + j] = G[(size_t)j * keep + i] = 0.5 * (G[(size_t)i * keep + j] + G[(size_t)j * keep + i]);
        jacobi_svd(G, keep, keep, &lam, &E, &E2);  // symmetric PSD: singular values = eigenvalues
        int r = 0;
        while (r < keep && lam[r] > 1e-12 * lam[0] && lam[r] > 0.0) ++r;
        if (r == 0) {
            w.err = "the sketch is zero";
            return 0;
        }
        // T (keep x r) = E[:, :r] diag(lam)^(-1/2)
        std::vector<float> Tf((size_t)keep * r);
        for (int i = 0; i < keep; ++i)
            for (int j = 0; j < r; ++j) Tf[(size_t)i * r + j] = (float)(E[(size_t)i * keep + j] / std::sqrt(lam[j]));
        if (cudaMemcpyAsync(w.T, Tf.data(), sizeof(float) * Tf.size(), cudaMemcpyHostToDevice, w.st) != cudaSuccess) {
            w.err = "transform copy failed";
            return 0;
        }
        // tmp (rows x r, stride ld) = X T, then back into X
        if (gemm_rm(w.hb, false, false, (int)rows, r, keep, X, ld, w.T, r, w.tmp, ld) != CUBLAS_STATUS_SUCCESS ||
            cudaMemcpyAsync(X, w.tmp, sizeof(float) * rows * ld, cudaMemcpyDeviceToDevice, w.st) != cudaSuccess) {
            w.err = "orthonormalisation product failed";
            return 0;
        }
        keep = r;
    }
    return keep;
}

}  // namespace pcw
