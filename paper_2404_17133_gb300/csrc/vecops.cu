// Streaming kernels over singles vectors and factor staging.  All are bound by
// HBM bandwidth (or, for FP64 arithmetic, by the FP64 pipe): grid-stride loops,
// coalesced along the contiguous index, grids sized to a multiple of the SM count.
#include <algorithm>

#include "vecops.cuh"

namespace tddft {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  const long long cap = 152LL * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

__device__ __forceinline__ double guard(double d) {
  if (fabs(d) < 1e-8) return d < 0 ? -1e-8 : 1e-8;
  return d;
}

template <typename T> __device__ __forceinline__ double ldd(const T* p, long long i);
template <> __device__ __forceinline__ double ldd<double>(const double* p, long long i) { return p[i]; }
template <> __device__ __forceinline__ double ldd<float>(const float* p, long long i) { return (double)p[i]; }
template <> __device__ __forceinline__ double ldd<__nv_bfloat16>(const __nv_bfloat16* p, long long i) {
  return (double)__bfloat162float(p[i]);
}

__global__ void k_delta(const double* eo, const double* ev, int no, int nv, double* d) {
  long long n = (long long)no * nv;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / nv), a = (int)(t % nv);
    d[t] = ev[a] - eo[i];
  }
}

__global__ void k_unit_rows(double* out, int k, int n, const int* idx) {
  long long tot = (long long)k * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int r = (int)(t / n), e = (int)(t % n);
    out[t] = (e == idx[r]) ? 1.0 : 0.0;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_row_sumsq(const T* X, long long ldx, int n, double* out) {
  __shared__ double red[32];
  const T* x = X + blockIdx.x * ldx;
  // per-thread partials in the row's precision (FP32 rows: FP32 FMA rate); four
  // independent accumulators keep four loads in flight
  T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0);
  const int st = blockDim.x;
  int e = threadIdx.x;
  for (; e + 3 * st < n; e += 4 * st) {
    const T v0 = x[e], v1 = x[e + st], v2 = x[e + 2 * st], v3 = x[e + 3 * st];
    p0 = fma(v0, v0, p0); p1 = fma(v1, v1, p1); p2 = fma(v2, v2, p2); p3 = fma(v3, v3, p3);
  }
  for (; e < n; e += st) { const T v = x[e]; p0 = fma(v, v, p0); }
  double acc = ((double)p0 + (double)p1) + ((double)p2 + (double)p3);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

__global__ void k_resid_tda(const double* X, const double* AX, const double* om, int k, int n, double* R) {
  long long tot = (long long)k * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int r = (int)(t / n);
    R[t] = AX[t] - om[r] * X[t];
  }
}

template <typename T>
__global__ void k_resid_paired(const T* U, const T* W, const T* PU, const T* MW,
                               const double* sh, const T* b, const T* bm, int k, int n,
                               T* Rp, T* Rm) {
  long long tot = (long long)k * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int r = (int)(t / n);
    double s = sh[r];
    Rp[t] = (T)((double)PU[t] - s * (double)W[t] - (b ? (double)b[t] : 0.0));
    Rm[t] = (T)((double)MW[t] - s * (double)U[t] - (bm ? (double)bm[t] : 0.0));
  }
}

template <typename T>
__global__ void k_precond_tda(const T* R, const double* om, const double* d, int k, int n, T* out) {
  long long tot = (long long)k * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int r = (int)(t / n), e = (int)(t % n);
    out[t] = (T)((double)R[t] / guard(d[e] - om[r]));
  }
}

template <typename T>
__global__ void k_precond_paired(const T* gp, const T* gm, const double* sh, const double* d,
                                 int k, int n, T* ou, T* ow) {
  long long tot = (long long)k * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int r = (int)(t / n), e = (int)(t % n);
    double g1 = (double)gp[t], g2 = gm ? (double)gm[t] : 0.0;
    double rx = 0.5 * (g1 + g2), ry = 0.5 * (g1 - g2);
    double x = rx / guard(d[e] - sh[r]);
    double y = ry / guard(d[e] + sh[r]);
    ou[t] = (T)(x + y);
    ow[t] = (T)(x - y);
  }
}

template <typename T>
__global__ void k_gather_rows(const T* src, const int* idx, int k, int n, T* dst) {
  long long tot = (long long)k * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int r = (int)(t / n), e = (int)(t % n);
    dst[t] = src[(long long)idx[r] * n + e];
  }
}

// Row r of src goes to row (number of kept rows before r) of dst when keep[r].
// Grid: x over column blocks, y over source rows.
template <typename T>
__global__ void k_compact_rows(const T* __restrict__ src, const int* __restrict__ keep, int nc, int n,
                               T* __restrict__ dst, int* __restrict__ count) {
  const int r = blockIdx.y;
  __shared__ int pos;
  if (threadIdx.x == 0) {
    int p = 0;
    for (int q = 0; q < r; ++q) p += keep[q] ? 1 : 0;
    pos = p;
    if (r == nc - 1 && blockIdx.x == 0) *count = p + (keep[r] ? 1 : 0);
  }
  __syncthreads();
  if (!keep[r]) return;
  const T* in = src + (long long)r * n;
  T* out = dst + (long long)pos * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = in[e];
}

// Zero row r of X (rows of length n; row r uses flag index r % nr) when the
// relative residual sqrt(a1[q] + a2[q]) / g[q] is at most tol (a2 may be NULL).
template <typename T>
__global__ void k_zero_converged(T* X, int rows, int nr, int n, const double* __restrict__ a1,
                                 const double* __restrict__ a2, const double* __restrict__ g, double tol) {
  const int r = blockIdx.y;
  const int q = r % nr;
  const double rr = sqrt(a1[q] + (a2 ? a2[q] : 0.0)) / g[q];
  if (!(rr <= tol)) return;
  T* x = X + (long long)r * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[e] = T(0);
}

template <typename S>
__global__ void k_sym_fill(S* a, int ld, int n_old, int n_new) {
  int N = n_old + n_new;
  long long tot = (long long)N * n_new;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int r = (int)(t / n_new), j = (int)(t % n_new);
    int c = n_old + j;
    if (r < n_old) {
      a[(long long)c * ld + r] = a[(long long)r * ld + c];
    } else if (r < c) {
      S v = S(0.5) * (a[(long long)r * ld + c] + a[(long long)c * ld + r]);
      a[(long long)r * ld + c] = v;
      a[(long long)c * ld + r] = v;
    }
  }
}

template <typename T>
__global__ void k_scale_rows(T* X, const double* sc, int k, int n) {
  long long tot = (long long)k * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x)
    X[t] = (T)((double)X[t] * sc[t / n]);
}

// y = a y + b x (y is not read when a == 0)
template <typename T>
__global__ void k_axpby(T* y, const T* x, double a, double b, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] = (T)(a == 0.0 ? b * (double)x[t] : a * (double)y[t] + b * (double)x[t]);
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* in, TO* out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = (TO)ldd<TI>(in, t);
}

template <typename TI>
__global__ void k_to_bf16(const TI* in, __nv_bfloat16* out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = __double2bfloat16(ldd<TI>(in, t));
}

template <typename T>
__global__ void k_mask(T* L, int rows, int n1, int n2, const unsigned char* m1, const unsigned char* m2) {
  long long tot = (long long)rows * n1 * n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    long long pq = t % ((long long)n1 * n2);
    int p = (int)(pq / n2), q = (int)(pq % n2);
    if (!(m1[p] && m2[q])) L[t] = (T)0.0f;
  }
}

template <typename TX, typename TW, typename TO>
__global__ void k_combine(const TX* X, const double* d, const TW* J, const TW* K1, const TW* K2,
                          double cj, double c1, double c2, long long m, int n, TO* out) {
  long long tot = m * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    double v = d[t % n] * (double)X[t];
    if (J) v += cj * ldd<TW>(J, t);
    if (K1) v += c1 * ldd<TW>(K1, t);
    if (K2) v += c2 * ldd<TW>(K2, t);
    out[t] = (TO)v;
  }
}

template <typename T>
__global__ void k_reduce_parts(T* buf, int parts, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double acc = (double)buf[t];
    for (int p = 1; p < parts; ++p) acc += (double)buf[p * n + t];
    buf[t] = (T)acc;
  }
}

template <typename T>
__global__ void k_check_finite(const T* X, long long n, int* flag) {
  int bad = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double v = ldd<T>(X, t);
    if (!isfinite(v)) bad = 1;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

#define TD_GRID(n) grid_for(n), kThreads, 0, s

}  // namespace

void delta_kernel(const double* eo, const double* ev, int no, int nv, double* d, cudaStream_t s) {
  k_delta<<<TD_GRID((long long)no * nv)>>>(eo, ev, no, nv, d);
  count_launch(); TD_LAUNCH_CHECK();
}
void unit_rows(double* out, int k, int n, const int* idx, cudaStream_t s) {
  k_unit_rows<<<TD_GRID((long long)k * n)>>>(out, k, n, idx);
  count_launch(); TD_LAUNCH_CHECK();
}
template <typename T>
void row_sumsq(const T* X, long long ldx, int k, int n, double* out, cudaStream_t s) {
  if (k <= 0) return;
  k_row_sumsq<T><<<k, 1024, 0, s>>>(X, ldx, n, out);
  count_launch(); TD_LAUNCH_CHECK();
}
template void row_sumsq<double>(const double*, long long, int, int, double*, cudaStream_t);
template void row_sumsq<float>(const float*, long long, int, int, double*, cudaStream_t);
void resid_tda(const double* X, const double* AX, const double* om, int k, int n, double* R, cudaStream_t s) {
  k_resid_tda<<<TD_GRID((long long)k * n)>>>(X, AX, om, k, n, R);
  count_launch(); TD_LAUNCH_CHECK();
}
template <typename T>
void resid_paired(const T* U, const T* W, const T* PU, const T* MW, const double* sh,
                  const T* b, const T* bm, int k, int n, T* Rp, T* Rm, cudaStream_t s) {
  k_resid_paired<T><<<TD_GRID((long long)k * n)>>>(U, W, PU, MW, sh, b, bm, k, n, Rp, Rm);
  count_launch(); TD_LAUNCH_CHECK();
}
template void resid_paired<double>(const double*, const double*, const double*, const double*, const double*,
                                   const double*, const double*, int, int, double*, double*, cudaStream_t);
template void resid_paired<float>(const float*, const float*, const float*, const float*, const double*,
                                  const float*, const float*, int, int, float*, float*, cudaStream_t);
template <typename T>
void precond_tda(const T* R, const double* om, const double* d, int k, int n, T* out, cudaStream_t s) {
  k_precond_tda<T><<<TD_GRID((long long)k * n)>>>(R, om, d, k, n, out);
  count_launch(); TD_LAUNCH_CHECK();
}
template void precond_tda<double>(const double*, const double*, const double*, int, int, double*, cudaStream_t);
template void precond_tda<float>(const float*, const double*, const double*, int, int, float*, cudaStream_t);
template <typename T>
void precond_paired(const T* gp, const T* gm, const double* sh, const double* d, int k, int n,
                    T* ou, T* ow, cudaStream_t s) {
  k_precond_paired<T><<<TD_GRID((long long)k * n)>>>(gp, gm, sh, d, k, n, ou, ow);
  count_launch(); TD_LAUNCH_CHECK();
}
template void precond_paired<double>(const double*, const double*, const double*, const double*, int, int,
                                     double*, double*, cudaStream_t);
template void precond_paired<float>(const float*, const float*, const double*, const double*, int, int,
                                    float*, float*, cudaStream_t);
template <typename T>
void gather_rows(const T* src, const int* idx, int k, int n, T* dst, cudaStream_t s) {
  if (k <= 0) return;
  k_gather_rows<T><<<TD_GRID((long long)k * n)>>>(src, idx, k, n, dst);
  count_launch(); TD_LAUNCH_CHECK();
}
template void gather_rows<double>(const double*, const int*, int, int, double*, cudaStream_t);
template void gather_rows<float>(const float*, const int*, int, int, float*, cudaStream_t);
template <typename T>
void compact_rows(const T* src, const int* keep, int nc, int n, T* dst, int* count, cudaStream_t s) {
  if (nc <= 0) { TD_CUDA(cudaMemsetAsync(count, 0, sizeof(int), s)); return; }
  TD_REQUIRE(nc <= 65535, TDDFT_ERR_ARG, "compact_rows: too many rows");
  dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 64), nc);
  k_compact_rows<T><<<grid, 256, 0, s>>>(src, keep, nc, n, dst, count);
  count_launch(); TD_LAUNCH_CHECK();
}
template void compact_rows<double>(const double*, const int*, int, int, double*, int*, cudaStream_t);
template void compact_rows<float>(const float*, const int*, int, int, float*, int*, cudaStream_t);

template <typename T>
void zero_converged(T* X, int rows, int nr, int n, const double* a1, const double* a2, const double* g,
                    double tol, cudaStream_t s) {
  if (rows <= 0) return;
  TD_REQUIRE(rows <= 65535 && nr >= 1, TDDFT_ERR_ARG, "zero_converged: bad rows");
  dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 64), rows);
  k_zero_converged<T><<<grid, 256, 0, s>>>(X, rows, nr, n, a1, a2, g, tol);
  count_launch(); TD_LAUNCH_CHECK();
}
template void zero_converged<double>(double*, int, int, int, const double*, const double*, const double*,
                                     double, cudaStream_t);
template void zero_converged<float>(float*, int, int, int, const double*, const double*, const double*,
                                    double, cudaStream_t);

template <typename S>
void sym_fill(S* a, int ld, int n_old, int n_new, cudaStream_t s) {
  if (n_new <= 0) return;
  k_sym_fill<S><<<TD_GRID((long long)(n_old + n_new) * n_new)>>>(a, ld, n_old, n_new);
  count_launch(); TD_LAUNCH_CHECK();
}
template void sym_fill<double>(double*, int, int, int, cudaStream_t);
template void sym_fill<float>(float*, int, int, int, cudaStream_t);
template <typename T>
void scale_rows(T* X, const double* sc, int k, int n, cudaStream_t s) {
  k_scale_rows<T><<<TD_GRID((long long)k * n)>>>(X, sc, k, n);
  count_launch(); TD_LAUNCH_CHECK();
}
void axpby(void* y, const void* x, DType t, double a, double b, long long n, cudaStream_t s) {
  if (n <= 0) return;
  if (t == DType::F64) k_axpby<double><<<TD_GRID(n)>>>((double*)y, (const double*)x, a, b, n);
  else if (t == DType::F32) k_axpby<float><<<TD_GRID(n)>>>((float*)y, (const float*)x, a, b, n);
  else throw Error(TDDFT_ERR_ARG, "axpby: FP64 or FP32 only");
  count_launch();
  TD_LAUNCH_CHECK();
}

template void scale_rows<double>(double*, const double*, int, int, cudaStream_t);
template void scale_rows<float>(float*, const double*, int, int, cudaStream_t);
void cast_f64_to_f32(const double* in, float* out, long long n, cudaStream_t s) {
  k_convert<double, float><<<TD_GRID(n)>>>(in, out, n);
  count_launch(); TD_LAUNCH_CHECK();
}
void cast_f32_to_f64(const float* in, double* out, long long n, cudaStream_t s) {
  k_convert<float, double><<<TD_GRID(n)>>>(in, out, n);
  count_launch(); TD_LAUNCH_CHECK();
}
void convert(const void* in, DType tin, void* out, DType tout, long long n, cudaStream_t s) {
  if (tout == DType::BF16) { cast_to_bf16(in, tin, (__nv_bfloat16*)out, n, s); return; }
  if (tin == DType::F64 && tout == DType::F64) TD_CUDA(cudaMemcpyAsync(out, in, n * 8, cudaMemcpyDeviceToDevice, s));
  else if (tin == DType::F32 && tout == DType::F32) TD_CUDA(cudaMemcpyAsync(out, in, n * 4, cudaMemcpyDeviceToDevice, s));
  else if (tin == DType::F64 && tout == DType::F32) { k_convert<double, float><<<TD_GRID(n)>>>((const double*)in, (float*)out, n); count_launch(); }
  else if (tin == DType::F32 && tout == DType::F64) { k_convert<float, double><<<TD_GRID(n)>>>((const float*)in, (double*)out, n); count_launch(); }
  else throw Error(TDDFT_ERR_ARG, "convert: unsupported types");
  TD_LAUNCH_CHECK();
}
void cast_to_bf16(const void* in, DType tin, __nv_bfloat16* out, long long n, cudaStream_t s) {
  if (tin == DType::F64) k_to_bf16<double><<<TD_GRID(n)>>>((const double*)in, out, n);
  else k_to_bf16<float><<<TD_GRID(n)>>>((const float*)in, out, n);
  count_launch(); TD_LAUNCH_CHECK();
}
void mask_block(void* L, DType t, int rows, int n1, int n2, const unsigned char* m1, const unsigned char* m2,
                cudaStream_t s) {
  long long tot = (long long)rows * n1 * n2;
  if (tot == 0) return;
  if (t == DType::F64) k_mask<double><<<TD_GRID(tot)>>>((double*)L, rows, n1, n2, m1, m2);
  else if (t == DType::F32) k_mask<float><<<TD_GRID(tot)>>>((float*)L, rows, n1, n2, m1, m2);
  else k_mask<__nv_bfloat16><<<TD_GRID(tot)>>>((__nv_bfloat16*)L, rows, n1, n2, m1, m2);
  count_launch(); TD_LAUNCH_CHECK();
}
void combine(const double* X, const double* d, const void* J, const void* K1, const void* K2, DType tw,
             double cj, double c1, double c2, long long m, int n, double* out, cudaStream_t s) {
  if (tw == DType::F64)
    k_combine<double, double, double><<<TD_GRID(m * n)>>>(X, d, (const double*)J, (const double*)K1, (const double*)K2, cj, c1, c2, m, n, out);
  else
    k_combine<double, float, double><<<TD_GRID(m * n)>>>(X, d, (const float*)J, (const float*)K1, (const float*)K2, cj, c1, c2, m, n, out);
  count_launch(); TD_LAUNCH_CHECK();
}
void combine_f32(const float* X, const double* d, const float* J, const float* K1, const float* K2,
                 double cj, double c1, double c2, long long m, int n, float* out, cudaStream_t s) {
  k_combine<float, float, float><<<TD_GRID(m * n)>>>(X, d, J, K1, K2, cj, c1, c2, m, n, out);
  count_launch(); TD_LAUNCH_CHECK();
}
void reduce_parts(void* buf, DType t, int parts, long long n, cudaStream_t s) {
  if (parts <= 1) return;
  if (t == DType::F64) k_reduce_parts<double><<<TD_GRID(n)>>>((double*)buf, parts, n);
  else k_reduce_parts<float><<<TD_GRID(n)>>>((float*)buf, parts, n);
  count_launch(); TD_LAUNCH_CHECK();
}
void check_finite(const void* X, DType t, long long n, int* flag, cudaStream_t s) {
  if (n <= 0) return;
  if (t == DType::F64) k_check_finite<double><<<TD_GRID(n)>>>((const double*)X, n, flag);
  else if (t == DType::F32) k_check_finite<float><<<TD_GRID(n)>>>((const float*)X, n, flag);
  else k_check_finite<__nv_bfloat16><<<TD_GRID(n)>>>((const __nv_bfloat16*)X, n, flag);
  count_launch(); TD_LAUNCH_CHECK();
}


namespace {
template <typename T>
__global__ void k_axpy_rows(T* out, const T* X, const double* sc, int k, int n) {
  long long tot = (long long)k * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x)
    out[t] = (T)((double)out[t] + sc[t / n] * (double)X[t]);
}
__global__ void k_half_sum_diff(const double* U, const double* W, long long n, double* X, double* Y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double u = U[t], w = W[t];
    if (X) X[t] = 0.5 * (u + w);
    if (Y) Y[t] = 0.5 * (u - w);
  }
}
template <typename T>
__global__ void k_resid_shift(const T* Y, const T* X, const double* sh, const T* B, int k, int n, T* out) {
  long long tot = (long long)k * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x)
    out[t] = (T)((double)Y[t] - sh[t / n] * (double)X[t] - (B ? (double)B[t] : 0.0));
}
}  // namespace

template <typename T>
void axpy_rows(T* out, const T* X, const double* sc, int k, int n, cudaStream_t s) {
  if (k <= 0) return;
  k_axpy_rows<T><<<TD_GRID((long long)k * n)>>>(out, X, sc, k, n);
  count_launch(); TD_LAUNCH_CHECK();
}
template void axpy_rows<double>(double*, const double*, const double*, int, int, cudaStream_t);
template void axpy_rows<float>(float*, const float*, const double*, int, int, cudaStream_t);
void half_sum_diff(const double* U, const double* W, long long n, double* X, double* Y, cudaStream_t s) {
  if (n <= 0) return;
  k_half_sum_diff<<<TD_GRID(n)>>>(U, W, n, X, Y);
  count_launch(); TD_LAUNCH_CHECK();
}
template <typename T>
void resid_shift(const T* Y, const T* X, const double* sh, const T* B, int k, int n, T* out, cudaStream_t s) {
  if (k <= 0) return;
  k_resid_shift<T><<<TD_GRID((long long)k * n)>>>(Y, X, sh, B, k, n, out);
  count_launch(); TD_LAUNCH_CHECK();
}
template void resid_shift<double>(const double*, const double*, const double*, const double*, int, int, double*, cudaStream_t);
template void resid_shift<float>(const float*, const float*, const double*, const float*, int, int, float*, cudaStream_t);

}  // namespace tddft
