// Streaming kernels over singles vectors (rows of length ov) and factor staging.
#pragma once
#include "common.cuh"

namespace tddft {

// Delta_ia = eps_a - eps_i (Eq. hessian, first term), ia = i*nv + a.
void delta_kernel(const double* eps_o, const double* eps_v, int no, int nv, double* delta,
                  cudaStream_t s);
// Rows r < k of out [k][n]: unit vector at column idx[r].
void unit_rows(double* out, int k, int n, const int* idx, cudaStream_t s);
// out[r] = sum_e X[r][e]^2 (deterministic; per-thread partial sums in T, the
// block sum in FP64), X rows of stride ldx.
template <typename T>
void row_sumsq(const T* X, long long ldx, int k, int n, double* out, cudaStream_t s);
// R = AX - diag(omega) X  (Eq. residual).
void resid_tda(const double* X, const double* AX, const double* omega, int k, int n, double* R,
               cudaStream_t s);
// Rp = PU - s W - b, Rm = MW - s U - bm (paired residuals; b, bm may be NULL).
template <typename T>
void resid_paired(const T* U, const T* W, const T* PU, const T* MW, const double* shift, const T* b,
                  const T* bm, int k, int n, T* Rp, T* Rm, cudaStream_t s);
// out = R / (Delta - omega)  (Eq. precondition with the diagonal T), guarded.
template <typename T>
void precond_tda(const T* R, const double* omega, const double* delta, int k, int n, T* out,
                 cudaStream_t s);
// Diagonal T for the paired systems: x = (g+ + g-)/2/(Delta - s), y = (g+ - g-)/2/(Delta + s),
// out_u = x + y, out_w = x - y.
template <typename T>
void precond_paired(const T* gp, const T* gm, const double* shift, const double* delta, int k, int n,
                    T* out_u, T* out_w, cudaStream_t s);
// Stream compaction of rows: the rows r < nc of src with keep[r] != 0 go, in
// order, to the leading rows of dst; count[0] = their number.
template <typename T>
void compact_rows(const T* src, const int* keep, int nc, int n, T* dst, int* count, cudaStream_t s);
// Zero row r of X [rows][n] when sqrt(a1[q] + a2[q]) / g[q] <= tol, q = r % nr
// (a2 may be NULL): masks the directions of converged systems on the device.
template <typename T>
void zero_converged(T* X, int rows, int nr, int n, const double* a1, const double* a2, const double* g,
                    double tol, cudaStream_t s);
// dst[r] = src[idx[r]] (rows of length n).
template <typename T>
void gather_rows(const T* src, const int* idx, int k, int n, T* dst, cudaStream_t s);
// Projected matrix a (ld) after its new columns [n_old, n_old+n_new) were written
// for all rows < n_old+n_new: mirror into the new rows and symmetrise the new block.
template <typename S>
void sym_fill(S* a, int ld, int n_old, int n_new, cudaStream_t s);
// X[r] *= scale[r].
template <typename T>
void scale_rows(T* X, const double* scale, int k, int n, cudaStream_t s);
// conversions
// y = a y + b x over n elements of type t (F64 or F32); y is not read when a == 0.
void axpby(void* y, const void* x, DType t, double a, double b, long long n, cudaStream_t s);

void cast_f64_to_f32(const double* in, float* out, long long n, cudaStream_t s);
void cast_f32_to_f64(const float* in, double* out, long long n, cudaStream_t s);
void cast_to_bf16(const void* in, DType tin, __nv_bfloat16* out, long long n, cudaStream_t s);
void convert(const void* in, DType tin, void* out, DType tout, long long n, cudaStream_t s);
// Zero the factor entries of orbitals outside the exchange window (Sec. 3.1):
// L [rows][n1][n2] *= m1[p] * m2[q].
void mask_block(void* L, DType t, int rows, int n1, int n2, const unsigned char* m1,
                const unsigned char* m2, cudaStream_t s);
// Operator combination (FP64 output):
//   out = Delta*X + c_j*J + c_1*K1 + c_2*K2   (J, K1, K2 of type `tw`, may be NULL)
void combine(const double* X, const double* delta, const void* J, const void* K1, const void* K2,
             DType tw, double c_j, double c_1, double c_2, long long m, int n, double* out,
             cudaStream_t s);
// FP32 variant (FP32 vectors in and out, FP32 parts).
void combine_f32(const float* X, const double* delta, const float* J, const float* K1, const float* K2,
                 double c_j, double c_1, double c_2, long long m, int n, float* out, cudaStream_t s);
// Sum `parts` partial buffers of n elements (type t) into the first.
void reduce_parts(void* buf, DType t, int parts, long long n, cudaStream_t s);
// Non-finite check: flag[0] |= 1 if any entry of X is NaN/Inf.
void check_finite(const void* X, DType t, long long n, int* flag, cudaStream_t s);

}  // namespace tddft

namespace tddft {
// out[r] += scale[r] * X[r] (rows of length n)
template <typename T>
void axpy_rows(T* out, const T* X, const double* scale, int k, int n, cudaStream_t s);
// X = (U + W)/2, Y = (U - W)/2
void half_sum_diff(const double* U, const double* W, long long n, double* X, double* Y,
                   cudaStream_t s);
// out = Y - shift[r] * X - B   (B may be NULL): the residual of (T - shift) x = b
template <typename T>
void resid_shift(const T* Y, const T* X, const double* shift, const T* B, int k, int n, T* out,
                 cudaStream_t s);
}  // namespace tddft
