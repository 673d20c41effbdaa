// Skinny products (see skinny.cuh).
#include <algorithm>
#include <type_traits>

#include "skinny.cuh"

namespace tddft {

namespace {

constexpr int kTile = 32;        // output tile of sk_gram (32 x 32, 2 x 2 per thread)
constexpr int kGramThreads = 256;
constexpr int kComboThreads = 256;
constexpr int kComboGroups = kComboThreads / 32;   // warps splitting the K sum
constexpr int kComboKc = 256;                      // K rows of coefficients staged at a time

template <typename R, typename T> __device__ __forceinline__ R cvt(T x) { return (R)x; }
template <> __device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}
template <> __device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 x) {
  return (double)__bfloat162float(x);
}

// Partial Gram matrices: CTA (chunk, mt, nt) sums k in [chunk*KC, chunk*KC + KC)
// for the output tile (mt, nt) and writes part[chunk][m][n].  The staging loads
// are fully unrolled (thread t reads column t % KC of every row it owns), so a
// thread has all of its loads in flight at once.
template <typename TA, typename TB, typename ACC, int KC>
__global__ void __launch_bounds__(kGramThreads)
k_sk_gram(const TA* __restrict__ A, long long lda, int M, const TB* __restrict__ B, long long ldb, int N,
          int K, ACC* __restrict__ part) {
  static_assert(kGramThreads % KC == 0 || KC % kGramThreads == 0, "tile mapping");
  constexpr int RSTEP = kGramThreads / KC;        // rows advanced per pass
  constexpr int PASSES = kTile / RSTEP;
  // row stride: 16-byte aligned rows for vector loads; the 4-float (2-double)
  // skew spreads the 16 B-columns of a warp over the banks
  constexpr int VW = 16 / sizeof(ACC);             // elements per 16-byte load
  constexpr int LD = KC + VW;
  extern __shared__ __align__(16) unsigned char gram_raw[];
  ACC* As = reinterpret_cast<ACC*>(gram_raw);
  ACC* Bs = As + kTile * LD;
  const int tid = threadIdx.x;
  const int k0 = blockIdx.x * KC;
  const int kn = min(KC, K - k0);
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.z * kTile;
  const int kk = tid % KC, r0 = tid / KC;
  const bool kin = kk < kn;
  ACC ra[PASSES], rb[PASSES];
#pragma unroll
  for (int p = 0; p < PASSES; ++p) {
    const int r = r0 + p * RSTEP;
    ra[p] = (kin && m0 + r < M) ? cvt<ACC>(A[(long long)(m0 + r) * lda + k0 + kk]) : ACC(0);
    rb[p] = (kin && n0 + r < N) ? cvt<ACC>(B[(long long)(n0 + r) * ldb + k0 + kk]) : ACC(0);
  }
#pragma unroll
  for (int p = 0; p < PASSES; ++p) {
    const int r = r0 + p * RSTEP;
    As[r * LD + kk] = ra[p];
    Bs[r * LD + kk] = rb[p];
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  ACC c00 = 0, c01 = 0, c10 = 0, c11 = 0;
  using V16 = typename std::conditional<sizeof(ACC) == 4, float4, double2>::type;
  const V16* a0 = reinterpret_cast<const V16*>(As + ty * LD);
  const V16* a1 = reinterpret_cast<const V16*>(As + (ty + 16) * LD);
  const V16* b0 = reinterpret_cast<const V16*>(Bs + tx * LD);
  const V16* b1 = reinterpret_cast<const V16*>(Bs + (tx + 16) * LD);
#pragma unroll 4
  for (int k = 0; k < KC / VW; ++k) {   // columns beyond kn were staged as zeros
    const V16 x0 = a0[k], x1 = a1[k], y0 = b0[k], y1 = b1[k];
    if constexpr (sizeof(ACC) == 4) {
      c00 = fma(x0.x, y0.x, c00); c00 = fma(x0.y, y0.y, c00); c00 = fma(x0.z, y0.z, c00); c00 = fma(x0.w, y0.w, c00);
      c01 = fma(x0.x, y1.x, c01); c01 = fma(x0.y, y1.y, c01); c01 = fma(x0.z, y1.z, c01); c01 = fma(x0.w, y1.w, c01);
      c10 = fma(x1.x, y0.x, c10); c10 = fma(x1.y, y0.y, c10); c10 = fma(x1.z, y0.z, c10); c10 = fma(x1.w, y0.w, c10);
      c11 = fma(x1.x, y1.x, c11); c11 = fma(x1.y, y1.y, c11); c11 = fma(x1.z, y1.z, c11); c11 = fma(x1.w, y1.w, c11);
    } else {
      c00 = fma(x0.x, y0.x, c00); c00 = fma(x0.y, y0.y, c00);
      c01 = fma(x0.x, y1.x, c01); c01 = fma(x0.y, y1.y, c01);
      c10 = fma(x1.x, y0.x, c10); c10 = fma(x1.y, y0.y, c10);
      c11 = fma(x1.x, y1.x, c11); c11 = fma(x1.y, y1.y, c11);
    }
  }
  ACC* P = part + (long long)blockIdx.x * M * N;
  const int ma = m0 + ty, mb = m0 + ty + 16, na = n0 + tx, nb = n0 + tx + 16;
  if (ma < M && na < N) P[(long long)ma * N + na] = c00;
  if (ma < M && nb < N) P[(long long)ma * N + nb] = c01;
  if (mb < M && na < N) P[(long long)mb * N + na] = c10;
  if (mb < M && nb < N) P[(long long)mb * N + nb] = c11;
}

// One warp per output element: lane l sums the chunks l, l+32, ... in order,
// then a fixed butterfly adds the lanes (deterministic).
template <typename ACC, typename TC>
__global__ void k_sk_gram_reduce(const ACC* __restrict__ part, int S, int M, int N, TC* __restrict__ C,
                                 long long ldc, double alpha, double beta) {
  const long long MN = (long long)M * N;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < MN; i += warps) {
    double acc = 0.0;
    for (int c = lane; c < S; c += 32) acc += (double)part[(long long)c * MN + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const int m = (int)(i / N), n = (int)(i - (long long)m * N);
      TC* p = C + (long long)m * ldc + n;
      double v = alpha * acc;
      if (beta != 0.0) v += beta * (double)*p;
      *p = (TC)v;
    }
  }
}

// Combination: CTA = 32 columns x kComboGroups warps; warp g sums k = g, g+8, ...
// for its lane's column and all MB rows of the block; the warps' partial sums
// are added in a fixed order through shared memory.  Coefficients are staged
// kComboKc rows of K at a time.
template <typename TS, typename TV, typename TO, typename ACC, int MB>
__global__ void __launch_bounds__(kComboThreads)
k_sk_combo(const TS* __restrict__ coef, long long scm, long long sck, int M, int K,
           const TV* __restrict__ V, long long ldv, int ncols, TO* __restrict__ out, long long ldo,
           double alpha, double beta) {
  extern __shared__ __align__(16) unsigned char combo_raw[];
  ACC* cs = reinterpret_cast<ACC*>(combo_raw);   // [kc][MB]
  ACC* red = cs + (size_t)kComboKc * MB;          // [groups][MB][33]
  const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
  const int mb0 = blockIdx.y * MB;
  const int mn = min(MB, M - mb0);
  const int c = blockIdx.x * 32 + lane;
  ACC acc[MB];
#pragma unroll
  for (int m = 0; m < MB; ++m) acc[m] = ACC(0);
  for (int k0 = 0; k0 < K; k0 += kComboKc) {
    const int kn = min(kComboKc, K - k0);
    __syncthreads();
    for (int e = tid; e < kn * MB; e += kComboThreads) {
      const int k = e / MB, m = e - k * MB;
      cs[e] = m < mn ? (ACC)coef[(long long)(mb0 + m) * scm + (long long)(k0 + k) * sck] : ACC(0);
    }
    __syncthreads();
    if (c < ncols) {
#pragma unroll 8
      for (int k = g; k < kn; k += kComboGroups) {
        const ACC v = cvt<ACC>(V[(long long)(k0 + k) * ldv + c]);
        const ACC* ck = cs + k * MB;
#pragma unroll
        for (int m = 0; m < MB; ++m) acc[m] = fma(ck[m], v, acc[m]);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < MB; ++m) red[(g * MB + m) * 33 + lane] = acc[m];
  __syncthreads();
  for (int e = tid; e < MB * 32; e += kComboThreads) {
    const int m = e >> 5, l = e & 31;
    const int col = blockIdx.x * 32 + l;
    if (m >= mn || col >= ncols) continue;
    ACC sum = ACC(0);
#pragma unroll
    for (int q = 0; q < kComboGroups; ++q) sum += red[(q * MB + m) * 33 + l];
    TO* o = out + (long long)(mb0 + m) * ldo + col;
    ACC v = (ACC)alpha * sum;
    if (beta != 0.0) v = fma((ACC)beta, (ACC)*o, v);
    *o = (TO)v;
  }
}

void set_smem_attr(const void* f, size_t bytes) {
  ensure_smem(f, bytes);
}

template <typename TA, typename TB, typename ACC>
void gram_typed(const void* A, long long lda, int M, const void* B, long long ldb, int N, int K, void* C,
                DType tc, long long ldc, double alpha, double beta, cudaStream_t s) {
  const int tiles = ((M + kTile - 1) / kTile) * ((N + kTile - 1) / kTile);
  TD_REQUIRE((M + kTile - 1) / kTile <= 65535 && (N + kTile - 1) / kTile <= 65535, TDDFT_ERR_ARG,
             "sk_gram: too many rows");
  // fixed K chunks: 256 columns (FP32 staging) or 128 (FP64)
  constexpr int KC = sizeof(ACC) == 8 ? 128 : 256;
  const int S = K > 0 ? (K + KC - 1) / KC : 1;
  (void)tiles;
  DevBuf part((size_t)S * M * N * sizeof(ACC), s);
  if (K > 0) {
    const size_t smem = (size_t)2 * kTile * (KC + 16 / sizeof(ACC)) * sizeof(ACC);
    set_smem_attr((const void*)k_sk_gram<TA, TB, ACC, KC>, smem);
    dim3 grid(S, (M + kTile - 1) / kTile, (N + kTile - 1) / kTile);
    k_sk_gram<TA, TB, ACC, KC><<<grid, kGramThreads, smem, s>>>(static_cast<const TA*>(A), lda, M,
                                                                static_cast<const TB*>(B), ldb, N, K,
                                                                part.as<ACC>());
    count_launch();
    TD_LAUNCH_CHECK();
  } else {
    TD_CUDA(cudaMemsetAsync(part.p, 0, (size_t)M * N * sizeof(ACC), s));
  }
  const long long MN = (long long)M * N;
  const unsigned rb = (unsigned)std::min<long long>((MN + 7) / 8, 16 * 152);   // 8 warps per block
  if (tc == DType::F64)
    k_sk_gram_reduce<ACC, double><<<rb, 256, 0, s>>>(part.as<ACC>(), S, M, N, (double*)C, ldc, alpha, beta);
  else
    k_sk_gram_reduce<ACC, float><<<rb, 256, 0, s>>>(part.as<ACC>(), S, M, N, (float*)C, ldc, alpha, beta);
  count_launch();
  TD_LAUNCH_CHECK();
}

// Wide combination (FP32 accumulation, FP32 or BF16 V): each lane owns four
// consecutive columns, loaded with one 16-byte (FP32) or 8-byte (BF16) access
// per V row, so a warp reads 512 or 256 contiguous bytes of a row and a thread
// keeps eight such loads in flight; a CTA covers 128 columns and kWideRows
// output rows (row blocks fastest in the grid, so the CTAs that share a stripe
// of V run together and share it through L2).  The K split over warps and the
// order of every sum are those of k_sk_combo: the results are the same bits.
constexpr int kWideRows = 8;
constexpr int kWideLd = 132;   // 128 columns + 4 (16-byte aligned rows)

__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float (&v)[4]) {
  const uint2 q = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&q.x);
  const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&q.y);
  v[0] = __low2float(a); v[1] = __high2float(a); v[2] = __low2float(b); v[3] = __high2float(b);
}

template <typename TS, typename TV, typename TO>
__global__ void __launch_bounds__(kComboThreads)
k_sk_combo_wide(const TS* __restrict__ coef, long long scm, long long sck, int M, int K,
                const TV* __restrict__ V, long long ldv, int ncols, TO* __restrict__ out, long long ldo,
                double alpha, double beta) {
  extern __shared__ __align__(16) unsigned char wide_raw[];
  float* cs = reinterpret_cast<float*>(wide_raw);        // [kComboKc][kWideRows]
  float* red = cs + (size_t)kComboKc * kWideRows;         // [groups][kWideRows][kWideLd]
  const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
  const int mb0 = blockIdx.x * kWideRows;
  const int mn = min(kWideRows, M - mb0);
  const int c0 = blockIdx.y * 128 + lane * 4;
  const bool full = c0 + 4 <= ncols;
  float acc[kWideRows][4];
#pragma unroll
  for (int m = 0; m < kWideRows; ++m)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[m][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kComboKc) {
    const int kn = min(kComboKc, K - k0);
    __syncthreads();
    for (int e = tid; e < kn * kWideRows; e += kComboThreads) {
      const int k = e / kWideRows, m = e - k * kWideRows;
      cs[e] = m < mn ? (float)coef[(long long)(mb0 + m) * scm + (long long)(k0 + k) * sck] : 0.f;
    }
    __syncthreads();
    if (c0 < ncols) {
#pragma unroll 8
      for (int k = g; k < kn; k += kComboGroups) {
        const TV* row = V + (long long)(k0 + k) * ldv + c0;
        float v[4];
        if (full) {
          load4(row, v);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) v[j] = c0 + j < ncols ? cvt<float>(row[j]) : 0.f;
        }
        const float* ck = cs + k * kWideRows;
#pragma unroll
        for (int m = 0; m < kWideRows; ++m) {
          const float cm = ck[m];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[m][j] = fmaf(cm, v[j], acc[m][j]);
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kWideRows; ++m)
    *reinterpret_cast<float4*>(red + (size_t)(g * kWideRows + m) * kWideLd + lane * 4) =
        make_float4(acc[m][0], acc[m][1], acc[m][2], acc[m][3]);
  __syncthreads();
  for (int e = tid; e < kWideRows * 128; e += kComboThreads) {
    const int m = e >> 7, l = e & 127;
    const int col = blockIdx.y * 128 + l;
    if (m >= mn || col >= ncols) continue;
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < kComboGroups; ++q) sum += red[(size_t)(q * kWideRows + m) * kWideLd + l];
    TO* o = out + (long long)(mb0 + m) * ldo + col;
    float v = (float)alpha * sum;
    if (beta != 0.0) v = fmaf((float)beta, (float)*o, v);
    *o = (TO)v;
  }
}

template <typename TS, typename TV, typename TO, typename ACC>
void combo_typed(const void* coef, long long scm, long long sck, int M, int K, const void* V, long long ldv,
                 int ncols, void* out, long long ldo, double alpha, double beta, cudaStream_t s) {
  if constexpr (std::is_same<ACC, float>::value &&
                (std::is_same<TV, float>::value || std::is_same<TV, __nv_bfloat16>::value)) {
    // wide path where every lane's four columns can be one aligned access
    const uintptr_t va = reinterpret_cast<uintptr_t>(V);
    const long long stripes = (ncols + 127) / 128;
    if (ncols >= 128 && ldv % 4 == 0 && va % (4 * sizeof(TV)) == 0 && stripes <= 65535) {
      const size_t smem = ((size_t)kComboKc * kWideRows + (size_t)kComboGroups * kWideRows * kWideLd) *
                          sizeof(float);
      dim3 grid((M + kWideRows - 1) / kWideRows, (unsigned)stripes);
      set_smem_attr((const void*)k_sk_combo_wide<TS, TV, TO>, smem);
      k_sk_combo_wide<TS, TV, TO><<<grid, kComboThreads, smem, s>>>(
          static_cast<const TS*>(coef), scm, sck, M, K, static_cast<const TV*>(V), ldv, ncols,
          static_cast<TO*>(out), ldo, alpha, beta);
      count_launch();
      TD_LAUNCH_CHECK();
      return;
    }
  }
  constexpr int MB = sizeof(ACC) == 8 ? 16 : 32;
  const int mblocks = (M + MB - 1) / MB;
  TD_REQUIRE(mblocks <= 65535, TDDFT_ERR_ARG, "sk_combo: too many rows");
  const size_t smem = ((size_t)kComboKc * MB + (size_t)kComboGroups * MB * 33) * sizeof(ACC);
  dim3 grid((ncols + 31) / 32, mblocks);
  set_smem_attr((const void*)k_sk_combo<TS, TV, TO, ACC, MB>, smem);
  k_sk_combo<TS, TV, TO, ACC, MB><<<grid, kComboThreads, smem, s>>>(
      static_cast<const TS*>(coef), scm, sck, M, K, static_cast<const TV*>(V), ldv, ncols,
      static_cast<TO*>(out), ldo, alpha, beta);
  count_launch();
  TD_LAUNCH_CHECK();
}

}  // namespace

void sk_gram(const void* A, DType ta, long long lda, int M, const void* B, DType tb, long long ldb, int N,
             int K, void* C, DType tc, long long ldc, double alpha, double beta, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  TD_REQUIRE(tc == DType::F32 || tc == DType::F64, TDDFT_ERR_ARG, "sk_gram: output type");
  if (ta == DType::F64 && tb == DType::F64)
    gram_typed<double, double, double>(A, lda, M, B, ldb, N, K, C, tc, ldc, alpha, beta, s);
  else if (ta == DType::F32 && tb == DType::F32)
    gram_typed<float, float, float>(A, lda, M, B, ldb, N, K, C, tc, ldc, alpha, beta, s);
  else if (ta == DType::BF16 && tb == DType::F32)
    gram_typed<__nv_bfloat16, float, float>(A, lda, M, B, ldb, N, K, C, tc, ldc, alpha, beta, s);
  else
    throw Error(TDDFT_ERR_ARG, "sk_gram: unsupported operand types");
}

void sk_combo(const void* coef, DType tcoef, long long scm, long long sck, int M, int K, const void* V,
              DType tv, long long ldv, int ncols, void* out, DType tout, long long ldo, double alpha,
              double beta, cudaStream_t s) {
  if (M <= 0 || ncols <= 0) return;
  TD_REQUIRE(tcoef == DType::F32 || tcoef == DType::F64, TDDFT_ERR_ARG, "sk_combo: coefficient type");
  if (tv == DType::F64 && tout == DType::F64) {
    TD_REQUIRE(tcoef == DType::F64, TDDFT_ERR_ARG, "sk_combo: FP64 vectors need FP64 coefficients");
    combo_typed<double, double, double, double>(coef, scm, sck, M, K, V, ldv, ncols, out, ldo, alpha, beta, s);
  } else if (tv == DType::F32 && tout == DType::F32) {
    if (tcoef == DType::F64)
      combo_typed<double, float, float, float>(coef, scm, sck, M, K, V, ldv, ncols, out, ldo, alpha, beta, s);
    else
      combo_typed<float, float, float, float>(coef, scm, sck, M, K, V, ldv, ncols, out, ldo, alpha, beta, s);
  } else if (tv == DType::BF16 && tout == DType::F32 && tcoef == DType::F32) {
    combo_typed<float, __nv_bfloat16, float, float>(coef, scm, sck, M, K, V, ldv, ncols, out, ldo, alpha,
                                                    beta, s);
  } else {
    throw Error(TDDFT_ERR_ARG, "sk_combo: unsupported operand types");
  }
}

}  // namespace tddft
