// Skinny products: a few hundred rows of length ov (tens of thousands) against
// each other -- the Davidson subspace algebra and the Coulomb contractions of
// the response operator.  Both kernels are bound by reading the long rows once;
// the generic tiled GEMM serialises too many shared-memory stages for these
// shapes.  Operands may be FP64, FP32 or BF16; the products are accumulated in
// FP64 when every operand is FP64 and in FP32 otherwise.
#pragma once
#include "common.cuh"

namespace tddft {

// C[m][n] = alpha * sum_k A[m][k] B[n][k] + beta * C[m][n]   (m < M, n < N, k < K)
// A, B: rows of length K with strides lda, ldb.  K is cut into chunks (one CTA
// per chunk and 32x32 output tile); chunk sums are added in FP64 in a fixed
// order, so results are deterministic.  C (type tc: F32 or F64) has row stride ldc.
void sk_gram(const void* A, DType ta, long long lda, int M, const void* B, DType tb, long long ldb, int N,
             int K, void* C, DType tc, long long ldc, double alpha, double beta, cudaStream_t s);

// out[m][c] = alpha * sum_k coef(m, k) V[k][c] + beta * out[m][c]
// (m < M, k < K, c < ncols); coef(m, k) = coef[m*scm + k*sck] of type tcoef (F32
// or F64); V rows of stride ldv (type tv); out rows of stride ldo (type tout,
// F32 or F64).  out must not overlap V.  One pass over V per block of 32 (FP32)
// or 16 (FP64) output rows; the K sum is split over 8 warps and added in a fixed
// order.
void sk_combo(const void* coef, DType tcoef, long long scm, long long sck, int M, int K, const void* V,
              DType tv, long long ldv, int ncols, void* out, DType tout, long long ldo, double alpha,
              double beta, cudaStream_t s);

// Typed conveniences for same-type vectors (T = float or double).
template <typename T> constexpr DType dtype_of();
template <> constexpr DType dtype_of<double>() { return DType::F64; }
template <> constexpr DType dtype_of<float>() { return DType::F32; }

template <typename T>
inline void sk_gram(const T* A, long long lda, int M, const T* B, long long ldb, int N, int K, void* C,
                    DType tc, long long ldc, double alpha, double beta, cudaStream_t s) {
  sk_gram(A, dtype_of<T>(), lda, M, B, dtype_of<T>(), ldb, N, K, C, tc, ldc, alpha, beta, s);
}
template <typename T>
inline void sk_combo(const void* coef, DType tcoef, long long scm, long long sck, int M, int K, const T* V,
                     long long ldv, int ncols, T* out, long long ldo, double alpha, double beta,
                     cudaStream_t s) {
  sk_combo(coef, tcoef, scm, sck, M, K, V, dtype_of<T>(), ldv, ncols, out, dtype_of<T>(), ldo, alpha, beta,
           s);
}

}  // namespace tddft
