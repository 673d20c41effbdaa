// Skinny products of the Davidson subspace algebra: a few hundred vectors of
// length ov (ov in the tens of thousands) against each other.  Both kernels are
// bound by reading the vectors once; the generic tiled GEMM serialises too many
// shared-memory stages for these shapes.
#pragma once
#include "common.cuh"

namespace tddft {

// C[m][n] = alpha * sum_k A[m][k] B[n][k] + beta * C[m][n]   (m < M, n < N, k < K)
// A, B: rows of length K with strides lda, ldb (T = float or double).  K is cut
// into chunks (one CTA per chunk and 32x32 output tile); chunk sums are taken in
// T and added in FP64 in a fixed order, so results are deterministic.  C has
// type tc (F32 or F64) and row stride ldc.
template <typename T>
void sk_gram(const T* A, long long lda, int M, const T* B, long long ldb, int N, int K, void* C,
             DType tc, long long ldc, double alpha, double beta, cudaStream_t s);

// out[m][c] = alpha * sum_k coef(m, k) V[k][c] + beta * out[m][c]
// (m < M, k < K, c < ncols); coef(m, k) = coef[m*scm + k*sck] of type tcoef (F32
// or F64, converted to T on load); V rows of stride ldv; out rows of stride ldo.
// out must not overlap V.  One pass over V per block of 32 (float) or 16
// (double) output rows; the K sum is split over 8 warps and added in a fixed order.
template <typename T>
void sk_combo(const void* coef, DType tcoef, long long scm, long long sck, int M, int K, const T* V,
              long long ldv, int ncols, T* out, long long ldo, double alpha, double beta,
              cudaStream_t s);

}  // namespace tddft
