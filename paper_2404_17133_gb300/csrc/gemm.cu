// Strided, batched SIMT GEMM used for the FP64 (plain) and FP32 (mixed) operator
// contractions and for the skinny products of the Davidson subspace algebra
// (projection V^T (AV), Ritz vectors V x, Gram-Schmidt coefficients).
//
// Tiling: a CTA computes a BM x BN tile of C from BK-deep slabs of A and B staged
// in shared memory (the next slab is prefetched into registers while the current
// one is consumed); each thread owns a TM x TN micro-tile whose rows and columns
// are strided by BM/TM and BN/TN so that shared-memory reads are conflict-free and
// global stores of C are coalesced along n.
#include "common.cuh"

namespace tddft {

thread_local long long g_launches = 0;

template <typename T> struct ElemIO;
template <> struct ElemIO<double> {
  template <typename R> __device__ static R ld(const double* p) { return (R)__ldg(p); }
};
template <> struct ElemIO<float> {
  template <typename R> __device__ static R ld(const float* p) { return (R)__ldg(p); }
};
template <> struct ElemIO<__nv_bfloat16> {
  template <typename R> __device__ static R ld(const __nv_bfloat16* p) {
    return (R)__bfloat162float(*p);
  }
};

struct GemmArgs {
  int M, N, K;
  const void* A; long long sam, sak;
  const void* B; long long sbk, sbn;
  void* C; long long scm, scn;
  double alpha, beta;
  int nb1;
  long long sA0, sA1, sB0, sB1, sC0, sC1;
};

template <typename TA, typename TB, typename TC, typename ACC, int BM, int BN, int BK, int TM,
          int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_kernel(GemmArgs g) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int LA = (BM * BK + NT - 1) / NT;
  constexpr int LB = (BN * BK + NT - 1) / NT;
  constexpr int RS = BM / TM;  // row stride of the micro-tile
  constexpr int CS = BN / TN;  // column stride
  __shared__ ACC As[BK][BM + 1];
  __shared__ ACC Bs[BK][BN + 1];

  const int tid = threadIdx.x;
  const int tx = tid % CS, ty = tid / CS;
  const long long bz = blockIdx.z;
  const long long b0 = bz / g.nb1, b1 = bz % g.nb1;
  const TA* A = static_cast<const TA*>(g.A) + b0 * g.sA0 + b1 * g.sA1;
  const TB* B = static_cast<const TB*>(g.B) + b0 * g.sB0 + b1 * g.sB1;
  TC* C = static_cast<TC*>(g.C) + b0 * g.sC0 + b1 * g.sC1;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const bool a_kc = (g.sak == 1);   // A contiguous along k
  const bool b_nc = (g.sbn == 1);   // B contiguous along n

  ACC ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      int e = tid + l * NT;
      int mm, kk;
      if (a_kc) { mm = e / BK; kk = e % BK; } else { mm = e % BM; kk = e / BM; }
      int m = m0 + mm, k = k0 + kk;
      ra[l] = (e < BM * BK && m < g.M && k < g.K)
                  ? ElemIO<TA>::template ld<ACC>(A + (long long)m * g.sam + (long long)k * g.sak)
                  : ACC(0);
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      int e = tid + l * NT;
      int nn, kk;
      if (b_nc) { nn = e % BN; kk = e / BN; } else { nn = e / BK; kk = e % BK; }
      int n = n0 + nn, k = k0 + kk;
      rb[l] = (e < BN * BK && n < g.N && k < g.K)
                  ? ElemIO<TB>::template ld<ACC>(B + (long long)k * g.sbk + (long long)n * g.sbn)
                  : ACC(0);
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      int e = tid + l * NT;
      if (e < BM * BK) {
        int mm, kk;
        if (a_kc) { mm = e / BK; kk = e % BK; } else { mm = e % BM; kk = e / BM; }
        As[kk][mm] = ra[l];
      }
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      int e = tid + l * NT;
      if (e < BN * BK) {
        int nn, kk;
        if (b_nc) { nn = e % BN; kk = e / BN; } else { nn = e / BK; kk = e % BK; }
        Bs[kk][nn] = rb[l];
      }
    }
  };

  ACC acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = ACC(0);

  load(0);
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    __syncthreads();
    store();
    __syncthreads();
    if (k0 + BK < g.K) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      ACC a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * RS];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * CS];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int m = m0 + ty + i * RS;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int n = n0 + tx + j * CS;
      if (n >= g.N) continue;
      TC* c = C + (long long)m * g.scm + (long long)n * g.scn;
      double v = g.alpha * (double)acc[i][j];
      if (g.beta != 0.0) v += g.beta * (double)(*c);
      *c = (TC)v;
    }
  }
}

template <typename TA, typename TB, typename TC, typename ACC, int BM, int BN, int BK, int TM,
          int TN>
static void launch_cfg(const GemmDesc& d, cudaStream_t s) {
  GemmArgs g{d.M, d.N, d.K, d.A, d.sam, d.sak, d.B, d.sbk, d.sbn, d.C, d.scm, d.scn,
             d.alpha, d.beta, d.nb1, d.sA0, d.sA1, d.sB0, d.sB1, d.sC0, d.sC1};
  long long nb = (long long)d.nb0 * d.nb1;
  TD_REQUIRE(nb <= 65535, TDDFT_ERR_ARG, "gemm: batch count above 65535");
  dim3 grid((d.N + BN - 1) / BN, (d.M + BM - 1) / BM, (unsigned)nb);
  TD_REQUIRE(grid.y <= 65535, TDDFT_ERR_ARG, "gemm: M too large");
  gemm_kernel<TA, TB, TC, ACC, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, s>>>(g);
  count_launch();
  TD_LAUNCH_CHECK();
}

template <typename TA, typename TB, typename TC, typename ACC>
static void launch_shape(const GemmDesc& d, cudaStream_t s) {
  if (sizeof(ACC) == 8) {
    // FP64 is ALU-bound on this GPU: pick the tile that wastes the least padding
    if (d.M <= 16) launch_cfg<TA, TB, TC, ACC, 16, 128, 8, 1, 8>(d, s);
    else if (d.N <= 16) launch_cfg<TA, TB, TC, ACC, 128, 16, 8, 8, 1>(d, s);
    else if (d.M <= 32) launch_cfg<TA, TB, TC, ACC, 32, 128, 8, 2, 8>(d, s);
    else if (d.N <= 32) launch_cfg<TA, TB, TC, ACC, 128, 32, 8, 8, 2>(d, s);
    else launch_cfg<TA, TB, TC, ACC, 64, 64, 8, 4, 4>(d, s);
  } else {
    if (d.M <= 32) launch_cfg<TA, TB, TC, ACC, 32, 128, 8, 2, 8>(d, s);
    else if (d.M <= 64 || d.N <= 64) launch_cfg<TA, TB, TC, ACC, 64, 64, 8, 4, 4>(d, s);
    else launch_cfg<TA, TB, TC, ACC, 128, 128, 8, 8, 8>(d, s);
  }
}

template <typename TA, typename TB>
static void launch_f32(const GemmDesc& d, cudaStream_t s) {
  if (d.tc == DType::F64) launch_shape<TA, TB, double, float>(d, s);
  else if (d.tc == DType::F32) launch_shape<TA, TB, float, float>(d, s);
  else throw Error(TDDFT_ERR_ARG, "gemm: unsupported output type");
}

void gemm(const GemmDesc& d, cudaStream_t s) {
  if (d.M <= 0 || d.N <= 0 || d.nb0 <= 0 || d.nb1 <= 0) return;
  if (d.acc64) {
    TD_REQUIRE(d.ta == DType::F64 && d.tb == DType::F64 && d.tc == DType::F64, TDDFT_ERR_ARG,
               "gemm: FP64 accumulation needs FP64 operands");
    launch_shape<double, double, double, double>(d, s);
    return;
  }
  if (d.ta == DType::F32 && d.tb == DType::F32) launch_f32<float, float>(d, s);
  else if (d.ta == DType::BF16 && d.tb == DType::F32) launch_f32<__nv_bfloat16, float>(d, s);
  else if (d.ta == DType::F32 && d.tb == DType::BF16) launch_f32<float, __nv_bfloat16>(d, s);
  else if (d.ta == DType::BF16 && d.tb == DType::BF16) launch_f32<__nv_bfloat16, __nv_bfloat16>(d, s);
  else throw Error(TDDFT_ERR_ARG, "gemm: unsupported operand types for FP32 accumulation");
}

// ---------------------------------------------------------------------------
// Split-K (deterministic): partial products over K-chunks into a scratch buffer,
// then a fixed-order sum (no atomics, so results do not depend on scheduling).

template <typename TP, typename TC>
__global__ void splitk_reduce(const TP* __restrict__ part, int S, int M, int N, TC* C, long long scm,
                              long long scn, double alpha, double beta) {
  long long MN = (long long)M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < MN;
       idx += (long long)gridDim.x * blockDim.x) {
    int m = (int)(idx / N), n = (int)(idx % N);
    double acc = 0.0;
    for (int s = 0; s < S; ++s) acc += (double)part[s * MN + idx];
    TC* c = C + m * scm + n * scn;
    double v = alpha * acc;
    if (beta != 0.0) v += beta * (double)(*c);
    *c = (TC)v;
  }
}

int auto_splits(int M, int N, long long K) {
  long long tiles = (long long)((M + 63) / 64) * ((N + 63) / 64);
  long long S = K / 512;
  long long want = (2 * 152 + tiles - 1) / tiles;
  if (S > want) S = want;
  if (S > 1024) S = 1024;
  return (int)(S < 1 ? 1 : S);
}

void gemm_splitk(const GemmDesc& d0, int S, cudaStream_t s) {
  if (d0.M <= 0 || d0.N <= 0) return;
  TD_REQUIRE(d0.nb0 == 1 && d0.nb1 == 1, TDDFT_ERR_ARG, "gemm_splitk: batched input");
  if (S <= 1 || d0.K < 2 * S) { gemm(d0, s); return; }
  long long K = d0.K;
  long long kc = (K + S - 1) / S;
  S = (int)((K + kc - 1) / kc);
  const DType tp = d0.acc64 ? DType::F64 : DType::F32;
  const size_t es = dtype_size(tp);
  const long long MN = (long long)d0.M * d0.N;
  DevBuf part((size_t)S * MN * es, s);
  long long full = K / kc;
  GemmDesc d = d0;
  d.K = (int)kc;
  d.C = part.p; d.tc = tp; d.scm = d0.N; d.scn = 1; d.alpha = 1.0; d.beta = 0.0;
  d.nb0 = (int)full; d.nb1 = 1;
  d.sA0 = kc * d0.sak; d.sB0 = kc * d0.sbk; d.sC0 = MN;
  if (full > 0) gemm(d, s);
  if (full < S) {
    GemmDesc t = d;
    t.K = (int)(K - full * kc);
    t.A = (const char*)d0.A + full * kc * d0.sak * (long long)dtype_size(d0.ta);
    t.B = (const char*)d0.B + full * kc * d0.sbk * (long long)dtype_size(d0.tb);
    t.C = (char*)part.p + full * MN * es;
    t.nb0 = 1;
    gemm(t, s);
  }
  unsigned g = (unsigned)((MN + 255) / 256);
  if (g > 152 * 16) g = 152 * 16;
  if (tp == DType::F64) {
    TD_REQUIRE(d0.tc == DType::F64, TDDFT_ERR_ARG, "gemm_splitk: FP64 partials need FP64 output");
    splitk_reduce<double, double><<<g, 256, 0, s>>>(part.as<double>(), S, d0.M, d0.N, (double*)d0.C,
                                                    d0.scm, d0.scn, d0.alpha, d0.beta);
  } else if (d0.tc == DType::F32) {
    splitk_reduce<float, float><<<g, 256, 0, s>>>(part.as<float>(), S, d0.M, d0.N, (float*)d0.C,
                                                  d0.scm, d0.scn, d0.alpha, d0.beta);
  } else {
    splitk_reduce<float, double><<<g, 256, 0, s>>>(part.as<float>(), S, d0.M, d0.N, (double*)d0.C,
                                                   d0.scm, d0.scn, d0.alpha, d0.beta);
  }
  count_launch();
  TD_LAUNCH_CHECK();
}

void gemm_splitk_f64(int M, int N, long long K, const double* A, long long sam, long long sak,
                     const double* B, long long sbk, long long sbn, double* C, long long scm,
                     long long scn, double alpha, double beta, cudaStream_t s) {
  GemmDesc d;
  d.M = M; d.N = N; d.K = (int)K;
  d.A = A; d.sam = sam; d.sak = sak; d.B = B; d.sbk = sbk; d.sbn = sbn;
  d.C = C; d.scm = scm; d.scn = scn; d.alpha = alpha; d.beta = beta;
  gemm_splitk(d, auto_splits(M, N, K), s);
}

}  // namespace tddft
