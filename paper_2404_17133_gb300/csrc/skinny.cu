// Skinny subspace products (see skinny.cuh).
#include <algorithm>

#include "skinny.cuh"

namespace tddft {

namespace {

constexpr int kTile = 32;        // output tile of sk_gram (32 x 32, 2 x 2 per thread)
constexpr int kGramThreads = 256;
constexpr int kComboThreads = 256;
constexpr int kComboGroups = kComboThreads / 32;   // warps splitting the K sum

// Partial Gram matrices: CTA (chunk, mt, nt) sums k in [chunk*kc, chunk*kc + kc)
// for the output tile (mt, nt) and writes part[chunk][m][n].
template <typename T>
__global__ void __launch_bounds__(kGramThreads)
k_sk_gram(const T* __restrict__ A, long long lda, int M, const T* __restrict__ B, long long ldb, int N,
          int K, int kc, T* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char gram_raw[];
  const int ld = kc + 1;
  T* As = reinterpret_cast<T*>(gram_raw);
  T* Bs = As + kTile * ld;
  const int tid = threadIdx.x;
  const int k0 = blockIdx.x * kc;
  const int kn = min(kc, K - k0);
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.z * kTile;
  for (int e = tid; e < kTile * kc; e += kGramThreads) {
    const int r = e / kc, k = e - r * kc;
    const bool kin = k < kn;
    As[r * ld + k] = (kin && m0 + r < M) ? A[(long long)(m0 + r) * lda + k0 + k] : T(0);
    Bs[r * ld + k] = (kin && n0 + r < N) ? B[(long long)(n0 + r) * ldb + k0 + k] : T(0);
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  T c00 = 0, c01 = 0, c10 = 0, c11 = 0;
  const T* a0 = As + ty * ld;
  const T* a1 = As + (ty + 16) * ld;
  const T* b0 = Bs + tx * ld;
  const T* b1 = Bs + (tx + 16) * ld;
#pragma unroll 4
  for (int k = 0; k < kn; ++k) {
    const T x0 = a0[k], x1 = a1[k], y0 = b0[k], y1 = b1[k];
    c00 = fma(x0, y0, c00);
    c01 = fma(x0, y1, c01);
    c10 = fma(x1, y0, c10);
    c11 = fma(x1, y1, c11);
  }
  T* P = part + (long long)blockIdx.x * M * N;
  const int ma = m0 + ty, mb = m0 + ty + 16, na = n0 + tx, nb = n0 + tx + 16;
  if (ma < M && na < N) P[(long long)ma * N + na] = c00;
  if (ma < M && nb < N) P[(long long)ma * N + nb] = c01;
  if (mb < M && na < N) P[(long long)mb * N + na] = c10;
  if (mb < M && nb < N) P[(long long)mb * N + nb] = c11;
}

template <typename T, typename TC>
__global__ void k_sk_gram_reduce(const T* __restrict__ part, int S, int M, int N, TC* __restrict__ C,
                                 long long ldc, double alpha, double beta) {
  const long long MN = (long long)M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < MN;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < S; ++c) acc += (double)part[(long long)c * MN + i];
    const int m = (int)(i / N), n = (int)(i - (long long)m * N);
    TC* p = C + (long long)m * ldc + n;
    double v = alpha * acc;
    if (beta != 0.0) v += beta * (double)*p;
    *p = (TC)v;
  }
}

// Combination: CTA = 32 columns x kComboGroups warps; warp g sums k = g, g+8, ...
// for its lane's column and all MB rows of the block; the warps' partial sums
// are added in a fixed order through shared memory.
template <typename T, typename TS, int MB>
__global__ void __launch_bounds__(kComboThreads)
k_sk_combo(const TS* __restrict__ coef, long long scm, long long sck, int M, int K,
           const T* __restrict__ V, long long ldv, int ncols, T* __restrict__ out, long long ldo,
           T alpha, T beta) {
  extern __shared__ __align__(16) unsigned char combo_raw[];
  T* cs = reinterpret_cast<T*>(combo_raw);   // [K][MB]
  T* red = cs + (size_t)K * MB;               // [groups][MB][33]
  const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
  const int mb0 = blockIdx.y * MB;
  const int mn = min(MB, M - mb0);
  for (int e = tid; e < K * MB; e += kComboThreads) {
    const int k = e / MB, m = e - k * MB;
    cs[e] = m < mn ? (T)coef[(long long)(mb0 + m) * scm + (long long)k * sck] : T(0);
  }
  __syncthreads();
  const int c = blockIdx.x * 32 + lane;
  T acc[MB];
#pragma unroll
  for (int m = 0; m < MB; ++m) acc[m] = T(0);
  if (c < ncols) {
#pragma unroll 2
    for (int k = g; k < K; k += kComboGroups) {
      const T v = V[(long long)k * ldv + c];
      const T* ck = cs + k * MB;
#pragma unroll
      for (int m = 0; m < MB; ++m) acc[m] = fma(ck[m], v, acc[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < MB; ++m) red[(g * MB + m) * 33 + lane] = acc[m];
  __syncthreads();
  for (int e = tid; e < MB * 32; e += kComboThreads) {
    const int m = e >> 5, l = e & 31;
    const int col = blockIdx.x * 32 + l;
    if (m >= mn || col >= ncols) continue;
    T sum = T(0);
#pragma unroll
    for (int q = 0; q < kComboGroups; ++q) sum += red[(q * MB + m) * 33 + l];
    T* o = out + (long long)(mb0 + m) * ldo + col;
    T v = alpha * sum;
    if (beta != T(0)) v = fma(beta, *o, v);
    *o = v;
  }
}

void set_smem_attr(const void* f, size_t bytes) {
  TD_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace

template <typename T>
void sk_gram(const T* A, long long lda, int M, const T* B, long long ldb, int N, int K, void* C,
             DType tc, long long ldc, double alpha, double beta, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  TD_REQUIRE(tc == DType::F32 || tc == DType::F64, TDDFT_ERR_ARG, "sk_gram: output type");
  const int tiles = ((M + kTile - 1) / kTile) * ((N + kTile - 1) / kTile);
  TD_REQUIRE((M + kTile - 1) / kTile <= 65535 && (N + kTile - 1) / kTile <= 65535, TDDFT_ERR_ARG,
             "sk_gram: too many rows");
  // about four CTAs per SM in total; chunks of 32..kcmax columns
  const int kcmax = sizeof(T) == 8 ? 128 : 256;
  const int want = std::max(1, (4 * 152 + tiles - 1) / tiles);
  int kc = std::max(1, (K + want - 1) / want);
  kc = std::min(kcmax, std::max(32, (kc + 31) / 32 * 32));
  const int S = std::max(1, (K + kc - 1) / kc);
  DevBuf part((size_t)S * M * N * sizeof(T), s);
  const size_t smem = (size_t)2 * kTile * (kc + 1) * sizeof(T);
  set_smem_attr((const void*)k_sk_gram<T>, smem);
  dim3 grid(S, (M + kTile - 1) / kTile, (N + kTile - 1) / kTile);
  if (K > 0) {
    k_sk_gram<T><<<grid, kGramThreads, smem, s>>>(A, lda, M, B, ldb, N, K, kc, part.as<T>());
    count_launch();
    TD_LAUNCH_CHECK();
  } else {
    TD_CUDA(cudaMemsetAsync(part.p, 0, (size_t)M * N * sizeof(T), s));
  }
  const long long MN = (long long)M * N;
  const unsigned rb = (unsigned)std::min<long long>((MN + 255) / 256, 4 * 152);
  if (tc == DType::F64)
    k_sk_gram_reduce<T, double><<<rb, 256, 0, s>>>(part.as<T>(), K > 0 ? S : 1, M, N, (double*)C, ldc,
                                                   alpha, beta);
  else
    k_sk_gram_reduce<T, float><<<rb, 256, 0, s>>>(part.as<T>(), K > 0 ? S : 1, M, N, (float*)C, ldc,
                                                  alpha, beta);
  count_launch();
  TD_LAUNCH_CHECK();
}
template void sk_gram<float>(const float*, long long, int, const float*, long long, int, int, void*, DType,
                             long long, double, double, cudaStream_t);
template void sk_gram<double>(const double*, long long, int, const double*, long long, int, int, void*,
                              DType, long long, double, double, cudaStream_t);

template <typename T>
void sk_combo(const void* coef, DType tcoef, long long scm, long long sck, int M, int K, const T* V,
              long long ldv, int ncols, T* out, long long ldo, double alpha, double beta,
              cudaStream_t s) {
  if (M <= 0 || ncols <= 0) return;
  TD_REQUIRE(tcoef == DType::F32 || tcoef == DType::F64, TDDFT_ERR_ARG, "sk_combo: coefficient type");
  constexpr int MB = sizeof(T) == 8 ? 16 : 32;
  const int mblocks = (M + MB - 1) / MB;
  TD_REQUIRE(mblocks <= 65535, TDDFT_ERR_ARG, "sk_combo: too many rows");
  const size_t smem = ((size_t)std::max(K, 1) * MB + (size_t)kComboGroups * MB * 33) * sizeof(T);
  TD_REQUIRE(smem <= 200 * 1024, TDDFT_ERR_ARG, "sk_combo: K too large");
  dim3 grid((ncols + 31) / 32, mblocks);
  if (tcoef == DType::F64) {
    set_smem_attr((const void*)k_sk_combo<T, double, MB>, smem);
    k_sk_combo<T, double, MB><<<grid, kComboThreads, smem, s>>>(
        static_cast<const double*>(coef), scm, sck, M, K, V, ldv, ncols, out, ldo, (T)alpha, (T)beta);
  } else {
    set_smem_attr((const void*)k_sk_combo<T, float, MB>, smem);
    k_sk_combo<T, float, MB><<<grid, kComboThreads, smem, s>>>(
        static_cast<const float*>(coef), scm, sck, M, K, V, ldv, ncols, out, ldo, (T)alpha, (T)beta);
  }
  count_launch();
  TD_LAUNCH_CHECK();
}
template void sk_combo<float>(const void*, DType, long long, long long, int, int, const float*, long long,
                              int, float*, long long, double, double, cudaStream_t);
template void sk_combo<double>(const void*, DType, long long, long long, int, int, const double*,
                               long long, int, double*, long long, double, double, cudaStream_t);

}  // namespace tddft
