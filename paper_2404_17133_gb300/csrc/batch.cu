// Batched TDA solves: many small independent problems (molecules) advanced
// together, one Davidson iteration of every problem at a time (Sec. 2.1 for
// each problem; the rid preconditioner of Sec. 3 with its inner solve).
//
// A solve of one small molecule is a long chain of small kernels; run one at a
// time (or a few on concurrent streams) the device idles between them.  Here
// every step of an iteration is one launch for all problems:
//   * grouped GEMM: a persistent kernel walks a device list of tasks (one per
//     problem and product: C = alpha A B + beta C with arbitrary strides, FP32,
//     BF16 or FP64 operands, FP32 accumulation) tile by tile; tall-K products
//     (Gram matrices) are split over K with a fixed-order FP64 reduction;
//   * row operations (combination, residuals, preconditioner, norms, copies)
//     from a device list of rows;
//   * one CTA per problem (or right-hand side) for the small matrices:
//     Jacobi eigensolver, shifted LU solves, pivot-dropping Cholesky.
// The grouped-GEMM tile shape is chosen by a measured autotune: each variant
// runs the first exchange contraction of the batch once (the variants give the
// same bits: the K order of every sum is the same) and the fastest is kept.
// The exact-operator product of an iteration (Coulomb, the P-chunked exchange
// and the combination, for every problem) runs as one captured CUDA graph
// whose task lists are rewritten in place before each replay.
//
// The exact operator's lists run on the tensor cores instead (k_ggemm_tc: the
// same tasks and tile walk, every operand split into three BF16 parts on its
// way to shared memory, six products per K step, FP32 accumulation --
// FP32-accurate), and the SIMT variants are timed on the ris lists.
//
// Precision (the batched workload's form): trial vectors, exact factors and
// products in FP32 (exact products FP32-accurate on the tensor cores), ris
// factors in BF16 with FP32 accumulation, the projected matrices and small
// solves in FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>

#include <cstdio>
#include <cstdlib>

#include "ctx.cuh"
#include "small.cuh"
#include "tc_ptx.cuh"
#include "vecops.cuh"

namespace tddft {

namespace {

using Clock = std::chrono::steady_clock;

// TDDFT_TRACE=1: one line per lockstep iteration (first problem and the worst residual)
bool btrace() {
  static int v = -1;
  if (v < 0) { const char* e = getenv("TDDFT_TRACE"); v = (e && e[0] >= '1' && e[0] <= '9') ? 1 : 0; }
  return v != 0;
}

// ============================================================================
// grouped GEMM

struct GTask {
  const void* A;
  const void* B;
  float* C;                        // FP32 result (when Cd is null)
  double* Cd;                      // FP64 result through the split reduction
  float* part;                     // [ksplit][M][N] partial sums (split or FP64 result)
  long long sam, sak, sbk, sbn;    // A(r,k) = A[r*sam + k*sak], B(k,c) = B[k*sbk + c*sbn]
  long long scm, scn, scm1;        // C(r,c) = C[(r / crin)*scm1 + (r % crin)*scm + c*scn]
  float alpha, beta;
  int M, N, K, crin;
  int ta, tb;                      // operand types: 0 FP32, 1 BF16, 2 FP64
  int tiles_m, tiles_n, ksplit, kchunk;
  int tile0, elem0;                // first global tile / reduced element of the task
};

struct GHdr {
  int ntask, total_tiles, total_elems, pad;
};

constexpr int GBK = 16;   // K step of every tile variant (fixes the summation order)

__device__ __forceinline__ float ld_el(const void* p, long long i, int t) {
  if (t == 0) return reinterpret_cast<const float*>(p)[i];
  if (t == 1) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[i]);
  return (float)reinterpret_cast<const double*>(p)[i];
}

// largest task index i with key(i) <= x (tasks sorted by key)
__device__ __forceinline__ int find_task(const GTask* __restrict__ T, int n, int x, bool elem) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int key = elem ? T[mid].elem0 : T[mid].tile0;
    if (key <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_ggemm(const GTask* __restrict__ tasks, const GHdr* __restrict__ hdr) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ float As[GBK][BM + 1];
  __shared__ float Bs[GBK][BN + 1];
  const int ntask = hdr->ntask, total = hdr->total_tiles;
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const GTask& g = tasks[find_task(tasks, ntask, t, false)];
    int lt = t - g.tile0;
    const int ks = lt % g.ksplit;
    lt /= g.ksplit;
    const int m0 = (lt / g.tiles_n) * BM, n0 = (lt % g.tiles_n) * BN;
    const int k0 = ks * g.kchunk, k1 = min(g.K, k0 + g.kchunk);
    const int M = g.M, N = g.N;
    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
    for (int kb = k0; kb < k1; kb += GBK) {
      if (g.sak == 1) {
        for (int idx = tid; idx < BM * GBK; idx += NT) {
          const int r = idx / GBK, kk = idx % GBK;
          const int gr = m0 + r, gk = kb + kk;
          As[kk][r] = (gr < M && gk < k1) ? ld_el(g.A, gr * g.sam + gk, g.ta) : 0.f;
        }
      } else {
        for (int idx = tid; idx < BM * GBK; idx += NT) {
          const int kk = idx / BM, r = idx % BM;
          const int gr = m0 + r, gk = kb + kk;
          As[kk][r] = (gr < M && gk < k1) ? ld_el(g.A, gr * g.sam + gk * g.sak, g.ta) : 0.f;
        }
      }
      if (g.sbn == 1) {
        for (int idx = tid; idx < BN * GBK; idx += NT) {
          const int kk = idx / BN, c = idx % BN;
          const int gc = n0 + c, gk = kb + kk;
          Bs[kk][c] = (gc < N && gk < k1) ? ld_el(g.B, gk * g.sbk + gc, g.tb) : 0.f;
        }
      } else {
        for (int idx = tid; idx < BN * GBK; idx += NT) {
          const int c = idx / GBK, kk = idx % GBK;
          const int gc = n0 + c, gk = kb + kk;
          Bs[kk][c] = (gc < N && gk < k1) ? ld_el(g.B, gk * g.sbk + gc * g.sbn, g.tb) : 0.f;
        }
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GBK; ++kk) {
        float a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
    const bool split = g.ksplit > 1 || g.Cd != nullptr;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int r = m0 + ty * TM + i;
      if (r >= M) continue;
      const long long roff = (long long)(r / g.crin) * g.scm1 + (long long)(r % g.crin) * g.scm;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int c = n0 + tx * TN + j;
        if (c >= N) continue;
        if (split) {
          g.part[((long long)ks * M + r) * N + c] = acc[i][j];
        } else {
          float* cp = g.C + roff + c * g.scn;
          *cp = g.alpha * acc[i][j] + (g.beta != 0.f ? g.beta * *cp : 0.f);
        }
      }
    }
  }
}

// Split reduction: the partial sums of each split task, added in a fixed order
// in FP64, into C (FP32) or Cd (FP64).
__global__ void k_gsum(const GTask* __restrict__ tasks, const GHdr* __restrict__ hdr) {
  const int ntask = hdr->ntask, total = hdr->total_elems;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const GTask& g = tasks[find_task(tasks, ntask, e, true)];
    const int le = e - g.elem0;
    const int r = le / g.N, c = le % g.N;
    double acc = 0.0;
    for (int s = 0; s < g.ksplit; ++s) acc += (double)g.part[((long long)s * g.M + r) * g.N + c];
    const long long off = (long long)(r / g.crin) * g.scm1 + (long long)(r % g.crin) * g.scm + c * g.scn;
    if (g.Cd) {
      double* cp = g.Cd + off;
      *cp = (double)g.alpha * acc + (g.beta != 0.f ? (double)g.beta * *cp : 0.0);
    } else {
      float* cp = g.C + off;
      *cp = (float)((double)g.alpha * acc + (g.beta != 0.f ? (double)g.beta * *cp : 0.0));
    }
  }
}

// ---------------------------------------------------------------------------
// Grouped tensor-core tile kernel: the task list and tile walk of k_ggemm with
// 128 x 128 tiles.  Every operand element is loaded (FP32, BF16 or FP64),
// split into three BF16 parts x = h + m + l (24 significand bits) and written
// to K-major 128-byte-swizzled shared memory; one thread issues the six
// products hh + hm + mh + hl + lh + mm per 16-element K step (kind::f16, FP32
// accumulation in tensor memory, 2^-24 of the leading term dropped): an
// FP32-accurate product at the BF16 tensor-core rate.  Two stages: the
// loads of a k-block overlap the MMAs of the one before.  A wait that times
// out sets g_batch_tc_err and ends the kernel.
constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64;
constexpr int TC_THREADS = 256;
constexpr int TC_PART = 128 * 128;            // bytes of one part tile: 128 rows x 64 BF16
constexpr int TC_STAGE = 6 * TC_PART;         // A and B, three parts each
constexpr int TC_SMEM = 2 * TC_STAGE + 1024 + 128;

__device__ int g_batch_tc_err = 0;

// byte offset of (row, k) in a part tile (128-byte rows, 16-byte chunks XORed by row % 8)
__device__ __forceinline__ uint32_t sw128(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 3) ^ (row & 7))) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ void split3_store(unsigned char* base, uint32_t off, float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
  *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(base + TC_PART + off) = m;
  *reinterpret_cast<__nv_bfloat16*>(base + 2 * TC_PART + off) = l;
}

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_f(double x) { return (float)x; }

// One 128 x 64 operand tile (rows row0.., k kbase..) into its three part
// tiles: every thread loads its 32 elements first (independent loads in
// flight together), then splits and stores them.  KC: k is the contiguous
// index of the source (consecutive threads take consecutive k), else the row.
template <typename T, bool KC>
__device__ __forceinline__ void tc_load(unsigned char* dst, const T* __restrict__ src, long long s_row,
                                        long long s_k, int row0, int rows, int kbase, int k1, int tid) {
  constexpr int PER = 128 * TC_BK / TC_THREADS;
  float x[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = tid + i * TC_THREADS;
    const int r = KC ? (idx >> 6) : (idx & 127);
    const int kk = KC ? (idx & 63) : (idx >> 7);
    const int gk = kbase + kk;
    x[i] = (r < rows && gk < k1) ? to_f(src[(long long)(row0 + r) * s_row + (long long)gk * s_k]) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = tid + i * TC_THREADS;
    const int r = KC ? (idx >> 6) : (idx & 127);
    const int kk = KC ? (idx & 63) : (idx >> 7);
    split3_store(dst, sw128(r, kk), x[i]);
  }
}

// dispatch on the element type (0 FP32, 1 BF16, 2 FP64) and the contiguous index
__device__ __forceinline__ void tc_load_any(unsigned char* dst, const void* src, int type, long long s_row,
                                            long long s_k, int row0, int rows, int kbase, int k1, int tid) {
  if (type == 0) {
    if (s_k == 1) tc_load<float, true>(dst, (const float*)src, s_row, s_k, row0, rows, kbase, k1, tid);
    else tc_load<float, false>(dst, (const float*)src, s_row, s_k, row0, rows, kbase, k1, tid);
  } else if (type == 1) {
    if (s_k == 1) tc_load<__nv_bfloat16, true>(dst, (const __nv_bfloat16*)src, s_row, s_k, row0, rows, kbase, k1, tid);
    else tc_load<__nv_bfloat16, false>(dst, (const __nv_bfloat16*)src, s_row, s_k, row0, rows, kbase, k1, tid);
  } else {
    if (s_k == 1) tc_load<double, true>(dst, (const double*)src, s_row, s_k, row0, rows, kbase, k1, tid);
    else tc_load<double, false>(dst, (const double*)src, s_row, s_k, row0, rows, kbase, k1, tid);
  }
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__global__ void __launch_bounds__(TC_THREADS, 1)
k_ggemm_tc(const GTask* __restrict__ tasks, const GHdr* __restrict__ hdr) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * TC_STAGE);   // [0], [1] stages, [2] tile done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) mbar_init(&bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  uint32_t ph[2] = {0u, 0u}, phd = 0u;
  bool pend[2] = {false, false};
  int it = 0;
  bool ok = true;
  const int ntask = hdr->ntask, total = hdr->total_tiles;
  for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
    const GTask& g = tasks[find_task(tasks, ntask, t, false)];
    int lt = t - g.tile0;
    const int ks = lt % g.ksplit;
    lt /= g.ksplit;
    const int m0 = (lt / g.tiles_n) * TC_BM, n0 = (lt % g.tiles_n) * TC_BN;
    const int k0 = ks * g.kchunk, k1 = min(g.K, k0 + g.kchunk);
    const int M = g.M, N = g.N;
    const int nb = min(TC_BN, (N - n0 + 15) & ~15);   // the MMA spans the tile's columns below N
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nb >> 3) << 17) |
                           ((uint32_t)(TC_BM >> 4) << 24);
    const int nkb = k1 > k0 ? (k1 - k0 + TC_BK - 1) / TC_BK : 0;
    for (int kb = 0; kb < nkb; ++kb, ++it) {
      const int s = it & 1;
      if (pend[s]) {   // the MMAs that last read this stage have completed
        if (!mbar_wait(&bar[s], ph[s])) ok = false;
        ph[s] ^= 1u;
        pend[s] = false;
      }
      if (!__syncthreads_and(ok)) { ok = false; break; }
      unsigned char* st = smem + s * TC_STAGE;
      unsigned char* sb = st + 3 * TC_PART;
      const int kbase = k0 + kb * TC_BK;
      tc_load_any(st, g.A, g.ta, g.sam, g.sak, m0, M - m0, kbase, k1, tid);   // A(r, k) = A[r sam + k sak]
      tc_load_any(sb, g.B, g.tb, g.sbn, g.sbk, n0, N - n0, kbase, k1, tid);   // B(k, c) = B[k sbk + c sbn]
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the stores, seen by the tensor cores
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t a0 = sdesc(st), a1 = sdesc(st + TC_PART), a2 = sdesc(st + 2 * TC_PART);
        const uint64_t b0 = sdesc(sb), b1 = sdesc(sb + TC_PART), b2 = sdesc(sb + 2 * TC_PART);
        const int rem = k1 - kbase;
        const int nks = rem >= TC_BK ? TC_BK / 16 : (rem + 15) / 16;   // zero-filled K steps issue no MMA
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          if (kk < nks) {
            const uint64_t o = (uint64_t)(kk * 32) >> 4;
            mma_bf16(tmem, a0 + o, b0 + o, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(tmem, a0 + o, b1 + o, idesc, 1u);
            mma_bf16(tmem, a1 + o, b0 + o, idesc, 1u);
            mma_bf16(tmem, a0 + o, b2 + o, idesc, 1u);
            mma_bf16(tmem, a2 + o, b0 + o, idesc, 1u);
            mma_bf16(tmem, a1 + o, b1 + o, idesc, 1u);
          }
        }
        mma_commit(&bar[s]);
      }
      pend[s] = true;
    }
    if (!ok) break;
    if (nkb > 0) {   // every MMA of the tile has completed
      if (tid == 0) mma_commit(&bar[2]);
      if (!mbar_wait(&bar[2], phd)) ok = false;
      phd ^= 1u;
      if (!__syncthreads_and(ok)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +32, columns 64 (w / 4) .. +64
    const int q = warp & 3, half = warp >> 2;
    const int r = m0 + q * 32 + lane;
    const bool split = g.ksplit > 1 || g.Cd != nullptr;
    const long long roff = r < M ? (long long)(r / g.crin) * g.scm1 + (long long)(r % g.crin) * g.scm : 0;
    for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 16) {
      if (n0 + c0 >= N) break;   // uniform over the warp
      uint32_t v[16];
      if (nkb > 0) {
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
            " [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;
      }
      if (r < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = n0 + c0 + j;
          if (c < N) {
            const float acc = __uint_as_float(v[j]);
            if (split) {
              g.part[((long long)ks * M + r) * N + c] = acc;
            } else {
              float* cp = g.C + roff + (long long)c * g.scn;
              *cp = g.alpha * acc + (g.beta != 0.f ? g.beta * *cp : 0.f);
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // the next tile's MMAs overwrite the accumulator
  }
  // the last commits have arrived before the CTA leaves
  for (int s2 = 0; s2 < 2; ++s2)
    if (pend[s2] && !mbar_wait(&bar[s2], ph[s2])) ok = false;
  if (!ok && lane == 0) atomicOr(&g_batch_tc_err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN));
}

struct Variant {
  const char* name;
  const void* fn;
  int threads;
  int bm, bn;
  int smem = 0;            // dynamic shared memory
  int ctas_per_sm = 4;     // persistent grid: ctas_per_sm x SMs
};

template <int BM, int BN, int TM, int TN>
Variant make_variant(const char* name) {
  return Variant{name, (const void*)k_ggemm<BM, BN, TM, TN>, (BM / TM) * (BN / TN), BM, BN};
}

// The exact operator's tile kernel (k_ggemm_tc).
const Variant& tc_variant() {
  static const Variant v{"tc128x128", (const void*)k_ggemm_tc, TC_THREADS, TC_BM, TC_BN, TC_SMEM, 1};
  return v;
}

// Reads and clears the tensor-core kernel's timeout flag.
void check_batch_tc(cudaStream_t s) {
  int h = 0;
  TD_CUDA(cudaMemcpyFromSymbolAsync(&h, g_batch_tc_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  TD_CUDA(cudaStreamSynchronize(s));
  if (h) {
    const int z = 0;
    TD_CUDA(cudaMemcpyToSymbolAsync(g_batch_tc_err, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    TD_CUDA(cudaStreamSynchronize(s));
    throw Error(TDDFT_ERR_CUDA, "batched tensor-core kernel wait timed out");
  }
}

const std::vector<Variant>& variants() {
  static const std::vector<Variant> v = {
      make_variant<64, 64, 4, 4>("64x64"),
      make_variant<128, 64, 8, 4>("128x64"),
      make_variant<64, 128, 4, 8>("64x128"),
      make_variant<128, 128, 8, 8>("128x128"),
      make_variant<32, 128, 2, 8>("32x128"),
  };
  return v;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  }
  return n;
}

// Pinned staging ring for the uploads of task and row lists: each upload takes
// the next slice and is copied in stream order; the stream is synchronised only
// when the ring wraps, so filling a list never waits for the device.
struct Ring {
  char* h = nullptr;
  size_t cap = 0, off = 0;
  ~Ring() { if (h) cudaFreeHost(h); }
  void upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return;
    const size_t need = (bytes + 255) & ~size_t(255);
    if (!h || need > cap) {
      TD_CUDA(cudaStreamSynchronize(s));
      if (h) cudaFreeHost(h);
      cap = std::max<size_t>(need * 4, 32u << 20);
      TD_CUDA(cudaMallocHost(&h, cap));
      off = 0;
    } else if (off + need > cap) {
      TD_CUDA(cudaStreamSynchronize(s));   // every earlier copy out of the ring is done
      off = 0;
    }
    std::memcpy(h + off, src, bytes);
    TD_CUDA(cudaMemcpyAsync(dst, h + off, bytes, cudaMemcpyHostToDevice, s));
    off += need;
  }
};

// One list of grouped-GEMM tasks: host staging (pinned), device copy, header
// and a partial-sum arena.  `run` uploads the list and launches the tile
// kernel of variant `v` (grid: a few CTAs per SM, persistent) and the split
// reduction; the launch shapes do not depend on the list, so a run can be
// captured into a graph and replayed after the list is rewritten in place.
struct GList {
  std::vector<GTask> tasks;
  GTask* h_tasks = nullptr;     // pinned
  GHdr* h_hdr = nullptr;        // pinned
  DevBuf d_tasks, d_hdr, arena;
  size_t cap_tasks = 0, arena_bytes = 0, arena_used = 0;
  int cur_bm = 64, cur_bn = 64;
  GList() = default;
  GList(const GList&) = delete;
  GList& operator=(const GList&) = delete;
  ~GList() {
    if (h_tasks) cudaFreeHost(h_tasks);
    if (h_hdr) cudaFreeHost(h_hdr);
  }
  void reset(int bm, int bn) {
    tasks.clear();
    arena_used = 0;
    cur_bm = bm;
    cur_bn = bn;
  }
  // C = alpha A B + beta C; ksplit chosen for tall-K products with few tiles
  void add(int M, int N, int K, const void* A, int ta, long long sam, long long sak, const void* B, int tb,
           long long sbk, long long sbn, float* C, double* Cd, long long scm, long long scn, float alpha,
           float beta, int crin = 0, long long scm1 = 0) {
    if (M <= 0 || N <= 0) return;
    GTask g{};
    g.A = A; g.B = B; g.C = C; g.Cd = Cd;
    g.sam = sam; g.sak = sak; g.sbk = sbk; g.sbn = sbn;
    g.scm = scm; g.scn = scn;
    g.crin = crin > 0 ? crin : (1 << 30);
    g.scm1 = scm1;
    g.alpha = alpha; g.beta = beta;
    g.M = M; g.N = N; g.K = std::max(K, 0);
    g.ta = ta; g.tb = tb;
    // tiles of the widest variant fix the split rule, so every variant splits alike
    const int tiles_big = ((M + 127) / 128) * ((N + 127) / 128);
    int ks = 1;
    if (tiles_big <= 4 && K > 2048) ks = std::min(64, K / 1024);
    g.ksplit = std::max(1, ks);
    g.kchunk = ((K + g.ksplit - 1) / g.ksplit + GBK - 1) / GBK * GBK;
    if (g.kchunk <= 0) g.kchunk = GBK;
    g.ksplit = std::max(1, (K + g.kchunk - 1) / g.kchunk);
    tasks.push_back(g);
  }
  // fill tile/element prefixes and partial-sum pointers for tile shape bm x bn
  GHdr hdr_host{};
  void finalize(int bm, int bn, cudaStream_t s) {
    // the pinned staging may still be read by the previous upload
    if (!ring) TD_CUDA(cudaStreamSynchronize(s));
    size_t need = 0;
    for (const GTask& g : tasks)
      if (g.ksplit > 1 || g.Cd) need += ((size_t)g.ksplit * g.M * g.N * 4 + 255) & ~size_t(255);
    if (need > arena_bytes) {
      arena = DevBuf(need + (need >> 2) + (1 << 20), s);
      arena_bytes = arena.bytes;
    }
    if (tasks.size() > cap_tasks) {
      if (h_tasks) cudaFreeHost(h_tasks);
      h_tasks = nullptr;
      cap_tasks = tasks.size() + tasks.size() / 2 + 64;
      if (!ring) TD_CUDA(cudaMallocHost(&h_tasks, cap_tasks * sizeof(GTask)));
      d_tasks = DevBuf(cap_tasks * sizeof(GTask), s);
    }
    if (!d_hdr.p) d_hdr = DevBuf(sizeof(GHdr), s);
    if (!ring && !h_hdr) TD_CUDA(cudaMallocHost(&h_hdr, sizeof(GHdr)));
    int tile = 0, elem = 0;
    size_t off = 0;
    for (GTask& g : tasks) {
      g.tiles_m = (g.M + bm - 1) / bm;
      g.tiles_n = (g.N + bn - 1) / bn;
      g.tile0 = tile;
      tile += g.tiles_m * g.tiles_n * g.ksplit;
      g.elem0 = elem;
      if (g.ksplit > 1 || g.Cd) {
        g.part = reinterpret_cast<float*>(static_cast<char*>(arena.p) + off);
        off += ((size_t)g.ksplit * g.M * g.N * 4 + 255) & ~size_t(255);
        elem += g.M * g.N;
      } else {
        g.part = nullptr;
      }
    }
    hdr_host.ntask = (int)tasks.size();
    hdr_host.total_tiles = tile;
    hdr_host.total_elems = elem;
    if (!ring) {
      std::memcpy(h_tasks, tasks.data(), tasks.size() * sizeof(GTask));
      *h_hdr = hdr_host;
    }
  }
  // upload + launch (finalize first)
  Ring* ring = nullptr;
  void launch(const Variant& v, cudaStream_t s) {
    if (tasks.empty()) return;
    if (ring) {
      ring->upload(d_tasks.p, tasks.data(), tasks.size() * sizeof(GTask), s);
      ring->upload(d_hdr.p, &hdr_host, sizeof(GHdr), s);
    } else {
      TD_CUDA(cudaMemcpyAsync(d_tasks.p, h_tasks, tasks.size() * sizeof(GTask), cudaMemcpyHostToDevice, s));
      TD_CUDA(cudaMemcpyAsync(d_hdr.p, h_hdr, sizeof(GHdr), cudaMemcpyHostToDevice, s));
    }
    launch_kernels(v, std::max(1, hdr_host.total_tiles), std::max(1, hdr_host.total_elems), s);
  }
  void launch_kernels(const Variant& v, int tiles, int elems, cudaStream_t s) {
    const int grid = std::max(1, std::min(tiles, num_sms() * v.ctas_per_sm));
    void* args[] = {&d_tasks.p, &d_hdr.p};
    if (v.smem > 0) ensure_smem(v.fn, (size_t)v.smem);
    TD_CUDA(cudaLaunchKernel(v.fn, dim3(grid), dim3(v.threads), args, (size_t)v.smem, s));
    count_launch();
    const int rg = std::min((elems + 255) / 256, num_sms() * 8);
    k_gsum<<<rg, 256, 0, s>>>(d_tasks.as<GTask>(), d_hdr.as<GHdr>());
    count_launch();
    TD_LAUNCH_CHECK();
  }
  void run(const Variant& v, cudaStream_t s) {
    if (tasks.empty()) return;
    finalize(v.bm, v.bn, s);
    launch(v, s);
  }
  // Launch shapes that do not depend on the list (for graph capture): the
  // whole staging capacity is copied and the grids are fixed; an empty list
  // runs as zero tasks.
  void reserve(size_t ntasks, cudaStream_t s) {
    if (ntasks <= cap_tasks && h_hdr) return;
    TD_CUDA(cudaStreamSynchronize(s));
    if (ntasks > cap_tasks) {
      if (h_tasks) cudaFreeHost(h_tasks);
      cap_tasks = ntasks;
      TD_CUDA(cudaMallocHost(&h_tasks, cap_tasks * sizeof(GTask)));
      d_tasks = DevBuf(cap_tasks * sizeof(GTask), s);
    }
    if (!h_hdr) {
      TD_CUDA(cudaMallocHost(&h_hdr, sizeof(GHdr)));
      d_hdr = DevBuf(sizeof(GHdr), s);
    }
  }
  void launch_fixed(const Variant& v, cudaStream_t s) {
    TD_CUDA(cudaMemcpyAsync(d_tasks.p, h_tasks, cap_tasks * sizeof(GTask), cudaMemcpyHostToDevice, s));
    TD_CUDA(cudaMemcpyAsync(d_hdr.p, h_hdr, sizeof(GHdr), cudaMemcpyHostToDevice, s));
    launch_kernels(v, num_sms() * v.ctas_per_sm, num_sms() * 8 * 256, s);
  }
  // the staging as seen by launch_fixed (after finalize); true if it still fits
  bool stage_fixed(const Variant& v, cudaStream_t s) {
    const size_t cap0 = cap_tasks;
    const void* d0 = d_tasks.p;
    if (tasks.empty()) {
      TD_CUDA(cudaStreamSynchronize(s));
      if (h_hdr) { h_hdr->ntask = 0; h_hdr->total_tiles = 0; h_hdr->total_elems = 0; }
      return h_hdr != nullptr;
    }
    finalize(v.bm, v.bn, s);
    return cap_tasks == cap0 && d_tasks.p == d0;
  }
};

// ============================================================================
// row operations

enum RowOpKind : int {
  R_COMBINE = 0,   // y = d*x1 + s0*x2 + s1*x3   (x2, x3 may be null)
  R_RESID = 1,     // y = x1 - lam*x2, norm      (lam = *sp)
  R_PRECOND = 2,   // y = x1 / (d - lam), guarded
  R_SRESID = 3,    // y = x1 - lam*x2 - x3, norm
  R_NORM = 4,      // norm of x1
  R_COPY = 5,      // y = x1
  R_UNIT = 6,      // y = e_(idx[s_idx])
};

struct RowOp {
  int op, n, idx;
  float* y;
  const float* x1;
  const float* x2;
  const float* x3;
  const double* d;
  const double* sp;     // device scalar (shift) or null
  const int* ord;       // R_UNIT: index table
  double* nrm;          // squared norm out (or null)
  double s0, s1;
};

__global__ void __launch_bounds__(256) k_rowops(const RowOp* __restrict__ ops, int nops) {
  __shared__ double red[8];
  for (int o = blockIdx.x; o < nops; o += gridDim.x) {
    const RowOp r = ops[o];
    const double lam = r.sp ? *r.sp : r.s0;
    double acc = 0.0;
    if (r.op == R_UNIT) {
      const int hot = r.ord[r.idx];
      for (int e = threadIdx.x; e < r.n; e += blockDim.x) r.y[e] = (e == hot) ? 1.f : 0.f;
    } else {
      for (int e = threadIdx.x; e < r.n; e += blockDim.x) {
        float v;
        switch (r.op) {
          case R_COMBINE: {
            double t = r.d[e] * (double)r.x1[e];
            if (r.x2) t += r.s0 * (double)r.x2[e];
            if (r.x3) t += r.s1 * (double)r.x3[e];
            v = (float)t;
            break;
          }
          case R_RESID: v = (float)((double)r.x1[e] - lam * (double)r.x2[e]); break;
          case R_PRECOND: {
            double den = r.d[e] - lam;
            if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
            v = (float)((double)r.x1[e] / den);
            break;
          }
          case R_SRESID: v = (float)((double)r.x1[e] - lam * (double)r.x2[e] - (double)r.x3[e]); break;
          case R_NORM: v = r.x1[e]; break;
          default: v = r.x1[e]; break;
        }
        if (r.op != R_NORM) r.y[e] = v;
        acc += (double)v * (double)v;
      }
    }
    if (r.nrm) {
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *r.nrm = t;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_combine_rows(const RowOp* __restrict__ ops, const int* __restrict__ n);

// A device list of row operations (pinned staging, like GList).
struct RList {
  std::vector<RowOp> ops;
  RowOp* h = nullptr;
  DevBuf d;
  size_t cap = 0;
  void free_stage() { if (h) cudaFreeHost(h); h = nullptr; }
  void add(const RowOp& r) { ops.push_back(r); }
  Ring* ring = nullptr;
  void run(cudaStream_t s) {
    if (ops.empty()) return;
    if (ops.size() > cap) {
      if (h) cudaFreeHost(h);
      h = nullptr;
      cap = ops.size() + ops.size() / 2 + 64;
      if (!ring) TD_CUDA(cudaMallocHost(&h, cap * sizeof(RowOp)));
      d = DevBuf(cap * sizeof(RowOp), s);
    }
    if (ring) {
      ring->upload(d.p, ops.data(), ops.size() * sizeof(RowOp), s);
    } else {
      // the pinned staging may still be read by an earlier copy: wait for the stream
      TD_CUDA(cudaStreamSynchronize(s));
      std::memcpy(h, ops.data(), ops.size() * sizeof(RowOp));
      TD_CUDA(cudaMemcpyAsync(d.p, h, ops.size() * sizeof(RowOp), cudaMemcpyHostToDevice, s));
    }
    const int grid = (int)std::min<size_t>(ops.size(), (size_t)num_sms() * 8);
    k_rowops<<<grid, 256, 0, s>>>(d.as<RowOp>(), (int)ops.size());
    count_launch();
    TD_LAUNCH_CHECK();
    ops.clear();
  }
  // graph form (R_COMBINE rows only): a fixed capacity, the count in device memory
  int* h_n = nullptr;
  DevBuf d_n;
  bool stage_fixed(size_t capacity, cudaStream_t s) {
    TD_CUDA(cudaStreamSynchronize(s));
    bool same = true;
    if (!h_n) {
      TD_CUDA(cudaMallocHost(&h_n, sizeof(int)));
      d_n = DevBuf(sizeof(int), s);
      same = false;
    }
    if (std::max(ops.size(), capacity) > cap) {
      if (h) cudaFreeHost(h);
      cap = std::max(ops.size(), capacity);
      TD_CUDA(cudaMallocHost(&h, cap * sizeof(RowOp)));
      d = DevBuf(cap * sizeof(RowOp), s);
      same = false;
    }
    if (!ops.empty()) std::memcpy(h, ops.data(), ops.size() * sizeof(RowOp));
    *h_n = (int)ops.size();
    ops.clear();
    return same;
  }
  void launch_fixed(cudaStream_t s) {
    TD_CUDA(cudaMemcpyAsync(d.p, h, cap * sizeof(RowOp), cudaMemcpyHostToDevice, s));
    TD_CUDA(cudaMemcpyAsync(d_n.p, h_n, sizeof(int), cudaMemcpyHostToDevice, s));
    k_combine_rows<<<num_sms() * 8, 256, 0, s>>>(d.as<RowOp>(), d_n.as<int>());
    count_launch();
    TD_LAUNCH_CHECK();
  }
  ~RList() {
    if (h_n) cudaFreeHost(h_n);
    free_stage();
  }
};

// R_COMBINE rows with the count read from device memory: the last step of the
// captured operator graph (the count changes between replays).
__global__ void __launch_bounds__(256) k_combine_rows(const RowOp* __restrict__ ops, const int* __restrict__ n) {
  const int nops = *n;
  for (int o = blockIdx.x; o < nops; o += gridDim.x) {
    const RowOp r = ops[o];
    for (int e = threadIdx.x; e < r.n; e += blockDim.x) {
      double t = r.d[e] * (double)r.x1[e];
      if (r.x2) t += r.s0 * (double)r.x2[e];
      if (r.x3) t += r.s1 * (double)r.x3[e];
      r.y[e] = (float)t;
    }
  }
}

RowOp rowop(int op, int n, float* y, const float* x1, const float* x2 = nullptr, const float* x3 = nullptr) {
  RowOp r{};
  r.op = op; r.n = n; r.y = y; r.x1 = x1; r.x2 = x2; r.x3 = x3;
  return r;
}

// ============================================================================
// the batch

constexpr int kCap = kBatchSmall;        // outer subspace rows per problem
constexpr int kInnerCap = kBatchSmall;   // inner (ris) subspace rows per problem
constexpr size_t kZBudget = 128ull << 20;  // exchange intermediates per problem

struct Ops {   // one operator of one problem (FP32 exact or BF16 ris factors)
  int nJ = 0, nK = 0, tf = 0;     // tf: factor element type (0 FP32, 1 BF16)
  const void* Jov = nullptr;
  const void* Koo = nullptr;
  const void* Kvv = nullptr;
};

struct Prob {
  Ctx* c = nullptr;
  int no = 0, nv = 0, ov = 0, k = 0, k0 = 0;
  tddft_opts o{};
  Ops ex, ris;
  int pc_ex = 1, pc_ris = 1, mmax = 1;
  // operator work buffers
  DevBuf t, J, K1, Z;
  // outer space
  DevBuf V, W, a, lam, xv, X, AX, R, cand, tmp, C, G, Tm, keep, nrm0, Xprev;
  int N = 0;
  bool have_prev = false;
  // inner space
  DevBuf S, TS, ti, h, y, v, Tv, res, icand;
  int Ns = 0;
  // host state
  std::vector<double> om, rr, rnorm0;
  std::vector<int> todo;
  bool done = false, converged = false;
  int n_iter = 0;
  long long mv = 0, ris_mv = 0;
  // status in the batch status buffer
  int st_off = 0;
};

struct Batch {
  std::vector<Prob> P;
  cudaStream_t s = nullptr;
  Ring ring;
  GList g;
  RList rl;
  const Variant* var = nullptr;
  std::vector<double> tune_ms;
  DevBuf status;                  // doubles: per problem [lam(kmax) | rn2(kmax) | keep(kmax)]
  double* h_status = nullptr;
  int stride = 0;                 // doubles per problem in the status buffer
  long long graph_launches = 0;
  // captured exact-operator graph: per P-chunk round the stage-1 and
  // stage-2 task lists, then the combination rows
  bool use_graph = true;
  int ex_rounds = 0;
  std::vector<std::unique_ptr<GList>> gs1, gs2;
  RList gcomb;
  size_t comb_cap = 0, s1_cap = 0, s2_cap = 0;
  cudaGraphExec_t op_exec = nullptr;
  int graph_nodes = 0, graph_captures = 0;
  ~Batch() {
    if (h_status) cudaFreeHost(h_status);
    if (op_exec) cudaGraphExecDestroy(op_exec);
  }
  double* st(Prob& p) { return status.as<double>() + p.st_off; }
  double* hst(Prob& p) { return h_status + p.st_off; }
  void pull() {
    TD_CUDA(cudaMemcpyAsync(h_status, status.p, (size_t)stride * P.size() * 8, cudaMemcpyDeviceToHost, s));
    TD_CUDA(cudaStreamSynchronize(s));
  }
};

// ---------------------------------------------------------------------------
// The operator on rows Xp[0..m) of each listed problem: Y = Delta X + c_J J(X)
// - a_x K1(X) (Eq. hessian, A alone), J and K1 as products over P-chunks.
struct OpCall {
  Prob* p;
  const float* X;
  float* Y;
  int m;
};

void add_operator_tasks(GList& g, std::vector<OpCall>& calls, bool ris, int chunk_round, bool& more) {
  more = false;
  for (OpCall& q : calls) {
    Prob& p = *q.p;
    const Ops& op = ris ? p.ris : p.ex;
    const int pc = ris ? p.pc_ris : p.pc_ex;
    const int m = q.m, no = p.no, nv = p.nv, ov = p.ov;
    if (m <= 0) continue;
    const int nch = op.nK > 0 ? (op.nK + pc - 1) / pc : 0;
    if (chunk_round == 0 && op.nJ > 0) {
      // t = Jov X^T  [nJ][m]  (tall K)
      g.add(op.nJ, m, ov, op.Jov, op.tf, ov, 1, q.X, 0, 1, ov, p.t.as<float>(), nullptr, m, 1, 1.f, 0.f);
    }
    if (chunk_round < nch) {
      const int p0 = chunk_round * pc, pn = std::min(pc, op.nK - p0);
      const size_t es = op.tf ? 2 : 4;
      // Z[n][i][P][a] = sum_j Koo[P][i][j] X[n][j][a], one task per vector n;
      // rows r = (P, i): offset (r / no)*nv + (r % no)*pc*nv
      for (int n = 0; n < m; ++n)
        g.add(pn * no, nv, no, (const char*)op.Koo + (size_t)p0 * no * no * es, op.tf, no, 1,
              q.X + (size_t)n * ov, 0, nv, 1, p.Z.as<float>() + (size_t)n * no * pc * nv, nullptr,
              (long long)pc * nv, 1, 1.f, 0.f, no, nv);
      if (chunk_round + 1 < nch) more = true;
    }
  }
}

void add_exchange_tasks(GList& g, std::vector<OpCall>& calls, bool ris, int chunk_round) {
  for (OpCall& q : calls) {
    Prob& p = *q.p;
    const Ops& op = ris ? p.ris : p.ex;
    const int pc = ris ? p.pc_ris : p.pc_ex;
    const int m = q.m, no = p.no, nv = p.nv, ov = p.ov;
    if (m <= 0) continue;
    const int nch = op.nK > 0 ? (op.nK + pc - 1) / pc : 0;
    if (chunk_round == 0 && op.nJ > 0) {
      // J = t^T Jov  [m][ov]
      g.add(m, ov, op.nJ, p.t.as<float>(), 0, 1, m, op.Jov, op.tf, ov, 1, p.J.as<float>(), nullptr, ov, 1, 1.f,
            0.f);
    }
    if (chunk_round < nch) {
      const int p0 = chunk_round * pc, pn = std::min(pc, op.nK - p0);
      const size_t es = op.tf ? 2 : 4;
      // K1[(n,i)][b] (+)= sum_(P,a) Z[(n,i)][(P,a)] Kvv[(P,a)][b]
      g.add(m * no, nv, pn * nv, p.Z.as<float>(), 0, (long long)pc * nv, 1,
            (const char*)op.Kvv + (size_t)p0 * nv * nv * es, op.tf, nv, 1, p.K1.as<float>(), nullptr, nv, 1,
            1.f, chunk_round > 0 ? 1.f : 0.f);
    }
  }
}

void operator_graph(Batch& B, std::vector<OpCall>& calls);

void operator_batch(Batch& B, std::vector<OpCall>& calls, bool ris) {
  if (calls.empty()) return;
  if (!ris && B.use_graph && B.ex_rounds > 0) {
    for (OpCall& q : calls) {
      TD_REQUIRE(q.m <= q.p->mmax, TDDFT_ERR_ARG, "batch: operator call larger than its work buffers");
      q.p->mv += q.m;
    }
    operator_graph(B, calls);
    return;
  }
  int maxch = 0;
  for (OpCall& q : calls) {
    TD_REQUIRE(q.m <= q.p->mmax, TDDFT_ERR_ARG, "batch: operator call larger than its work buffers");
    const Ops& op = ris ? q.p->ris : q.p->ex;
    const int pc = ris ? q.p->pc_ris : q.p->pc_ex;
    maxch = std::max(maxch, op.nK > 0 ? (op.nK + pc - 1) / pc : 0);
    if (ris) q.p->ris_mv += q.m; else q.p->mv += q.m;
  }
  // the exact operator on the tensor cores, the ris operator on the tuned SIMT tiles
  const Variant& v = ris ? *B.var : tc_variant();
  for (int c = 0; c < std::max(maxch, 1); ++c) {
    bool more = false;
    B.g.reset(v.bm, v.bn);
    add_operator_tasks(B.g, calls, ris, c, more);
    B.g.run(v, B.s);
    B.g.reset(v.bm, v.bn);
    add_exchange_tasks(B.g, calls, ris, c);
    B.g.run(v, B.s);
  }
  for (OpCall& q : calls) {
    Prob& p = *q.p;
    const Ops& op = ris ? p.ris : p.ex;
    const double cJ = p.c->c_J, ax = p.c->a_x;
    for (int n = 0; n < q.m; ++n) {
      RowOp r = rowop(R_COMBINE, p.ov, q.Y + (size_t)n * p.ov, q.X + (size_t)n * p.ov,
                      op.nJ > 0 ? p.J.as<float>() + (size_t)n * p.ov : nullptr,
                      op.nK > 0 ? p.K1.as<float>() + (size_t)n * p.ov : nullptr);
      r.d = p.c->delta.as<double>();
      r.s0 = cJ;
      r.s1 = -ax;
      B.rl.add(r);
    }
  }
  B.rl.run(B.s);
}

// The exact operator as one CUDA graph: the task lists of every P-chunk round
// and the combination rows are rewritten in their pinned staging, then the
// graph (uploads + persistent kernels with fixed grids) is replayed.  It is
// captured again only when a list outgrows its staging.
void operator_graph(Batch& B, std::vector<OpCall>& calls) {
  const Variant& v = tc_variant();
  cudaStream_t s = B.s;
  const int R = B.ex_rounds;
  if ((int)B.gs1.size() < R) {
    for (int r = (int)B.gs1.size(); r < R; ++r) {
      B.gs1.emplace_back(new GList());
      B.gs2.emplace_back(new GList());
      B.gs1.back()->reserve(B.s1_cap, s);
      B.gs2.back()->reserve(B.s2_cap, s);
    }
  }
  bool same = B.op_exec != nullptr;
  for (int r = 0; r < R; ++r) {
    bool more = false;
    B.gs1[r]->reset(v.bm, v.bn);
    add_operator_tasks(*B.gs1[r], calls, false, r, more);
    same = B.gs1[r]->stage_fixed(v, s) && same;
    B.gs2[r]->reset(v.bm, v.bn);
    add_exchange_tasks(*B.gs2[r], calls, false, r);
    same = B.gs2[r]->stage_fixed(v, s) && same;
  }
  for (OpCall& q : calls) {
    Prob& p = *q.p;
    for (int n = 0; n < q.m; ++n) {
      RowOp r = rowop(R_COMBINE, p.ov, q.Y + (size_t)n * p.ov, q.X + (size_t)n * p.ov,
                      p.ex.nJ > 0 ? p.J.as<float>() + (size_t)n * p.ov : nullptr,
                      p.ex.nK > 0 ? p.K1.as<float>() + (size_t)n * p.ov : nullptr);
      r.d = p.c->delta.as<double>();
      r.s0 = p.c->c_J;
      r.s1 = -p.c->a_x;
      B.gcomb.add(r);
    }
  }
  same = B.gcomb.stage_fixed(B.comb_cap, s) && same;
  if (!same) {
    if (B.op_exec) {
      cudaGraphExecDestroy(B.op_exec);
      B.op_exec = nullptr;
    }
    const long long before = g_launches;
    cudaGraph_t graph;
    TD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      for (int r = 0; r < R; ++r) {
        B.gs1[r]->launch_fixed(v, s);
        B.gs2[r]->launch_fixed(v, s);
      }
      B.gcomb.launch_fixed(s);
    } catch (...) {
      cudaStreamEndCapture(s, &graph);
      throw;
    }
    TD_CUDA(cudaStreamEndCapture(s, &graph));
    const cudaError_t e = cudaGraphInstantiate(&B.op_exec, graph, 0);
    cudaGraphDestroy(graph);
    TD_CUDA(e);
    B.graph_nodes = (int)(g_launches - before);
    g_launches = before;
    ++B.graph_captures;
  }
  TD_CUDA(cudaGraphLaunch(B.op_exec, s));
  ++B.graph_launches;
  count_launch(B.graph_nodes);
}

// Time every SIMT tile variant on the first ris exchange contraction list
// (the exact operator runs on the tensor cores; the ris products are the
// largest SIMT lists; same bits from each variant) and keep the fastest.
// TDDFT_BATCH_VARIANT=i forces variant i (after timing every variant).
int forced_variant() {
  const char* e = getenv("TDDFT_BATCH_VARIANT");
  if (!e || !*e) return -1;
  const int v = atoi(e);
  return (v >= 0 && v < (int)variants().size()) ? v : -1;
}

void autotune(Batch& B, std::vector<OpCall>& calls) {
  const auto& vs = variants();
  B.tune_ms.assign(vs.size(), -1.0);
  // one ris exchange round's tasks after its stage-1 products exist
  B.g.reset(64, 64);
  bool more = false;
  add_operator_tasks(B.g, calls, true, 0, more);
  B.g.run(vs[0], B.s);
  cudaEvent_t e0, e1;
  TD_CUDA(cudaEventCreate(&e0));
  TD_CUDA(cudaEventCreate(&e1));
  int best = 0;
  for (size_t v = 0; v < vs.size(); ++v) {
    B.g.reset(vs[v].bm, vs[v].bn);
    add_exchange_tasks(B.g, calls, true, 0);
    B.g.finalize(vs[v].bm, vs[v].bn, B.s);
    B.g.launch(vs[v], B.s);   // warm
    TD_CUDA(cudaEventRecord(e0, B.s));
    B.g.launch(vs[v], B.s);
    TD_CUDA(cudaEventRecord(e1, B.s));
    TD_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    TD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    B.tune_ms[v] = ms;
    if (ms < B.tune_ms[best]) best = (int)v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int f = forced_variant();
  B.var = &vs[f >= 0 ? f : best];
}

// ---------------------------------------------------------------------------
// Gram-Schmidt of candidate rows cand[0..nc) of each problem against its
// space S[0..N) and among themselves (two passes: projection + pivot-dropping
// Cholesky), survivors appended at S[N...].  Returns nothing; updates N.
struct OrthCall {
  Prob* p;
  float* S;        // space rows [cap][ov]
  int* N;          // rows in S (updated)
  float* cand;     // [nc][ov] candidates (overwritten)
  int nc;
  int cap;
};

void orth_append_batch(Batch& B, std::vector<OrthCall>& calls) {
  if (calls.empty()) return;
  const Variant& v = *B.var;
  // initial squared norms (drop rule of pass one)
  for (OrthCall& q : calls) {
    Prob& p = *q.p;
    for (int j = 0; j < q.nc; ++j) {
      RowOp r = rowop(R_NORM, p.ov, nullptr, q.cand + (size_t)j * p.ov);
      r.nrm = p.nrm0.as<double>() + j;
      B.rl.add(r);
    }
  }
  B.rl.run(B.s);
  int ncmax = 1;
  for (OrthCall& q : calls) ncmax = std::max(ncmax, q.nc);
  std::vector<BDrop> dd;
  DevBuf d_dd(calls.size() * sizeof(BDrop), B.s);
  for (int pass = 0; pass < 2; ++pass) {
    // C = S cand^T [N][nc] (FP64), cand -= C^T S
    B.g.reset(v.bm, v.bn);
    for (OrthCall& q : calls) {
      Prob& p = *q.p;
      if (*q.N > 0 && q.nc > 0)
        B.g.add(*q.N, q.nc, p.ov, q.S, 0, p.ov, 1, q.cand, 0, 1, p.ov, nullptr, p.C.as<double>(), q.nc, 1, 1.f, 0.f);
    }
    B.g.run(v, B.s);
    B.g.reset(v.bm, v.bn);
    for (OrthCall& q : calls) {
      Prob& p = *q.p;
      if (*q.N > 0 && q.nc > 0)
        B.g.add(q.nc, p.ov, *q.N, p.C.as<double>(), 2, 1, q.nc, q.S, 0, p.ov, 1, q.cand, nullptr, p.ov, 1, -1.f,
                1.f);
    }
    B.g.run(v, B.s);
    // G = cand cand^T (FP64), pivot-dropping Cholesky -> T, keep
    B.g.reset(v.bm, v.bn);
    for (OrthCall& q : calls) {
      Prob& p = *q.p;
      if (q.nc > 0)
        B.g.add(q.nc, q.nc, p.ov, q.cand, 0, p.ov, 1, q.cand, 0, 1, p.ov, nullptr, p.G.as<double>(), q.nc, 1, 1.f,
                0.f);
    }
    B.g.run(v, B.s);
    dd.clear();
    for (OrthCall& q : calls) {
      Prob& p = *q.p;
      dd.push_back(BDrop{p.G.as<double>(), q.nc, pass == 0 ? p.nrm0.as<double>() : nullptr, p.Tm.as<double>(),
                         p.keep.as<int>()});
    }
    TD_CUDA(cudaMemcpyAsync(d_dd.p, dd.data(), dd.size() * sizeof(BDrop), cudaMemcpyHostToDevice, B.s));
    batch_chol_drop(d_dd.as<BDrop>(), (int)dd.size(), ncmax, 1e-16, B.s);
    // cand <- T cand (into tmp, then back)
    B.g.reset(v.bm, v.bn);
    for (OrthCall& q : calls) {
      Prob& p = *q.p;
      if (q.nc > 0)
        B.g.add(q.nc, p.ov, q.nc, p.Tm.as<double>(), 2, q.nc, 1, q.cand, 0, p.ov, 1, p.tmp.as<float>(), nullptr,
                p.ov, 1, 1.f, 0.f);
    }
    B.g.run(v, B.s);
    for (OrthCall& q : calls) {
      Prob& p = *q.p;
      for (int j = 0; j < q.nc; ++j)
        B.rl.add(rowop(R_COPY, p.ov, q.cand + (size_t)j * p.ov, p.tmp.as<float>() + (size_t)j * p.ov));
    }
    B.rl.run(B.s);
  }
  // keep flags of the second pass decide; append survivors in order
  std::vector<std::vector<int>> kh(calls.size());
  for (size_t i = 0; i < calls.size(); ++i) {
    kh[i].resize(std::max(calls[i].nc, 1));
    if (calls[i].nc > 0)
      TD_CUDA(cudaMemcpyAsync(kh[i].data(), calls[i].p->keep.p, calls[i].nc * 4, cudaMemcpyDeviceToHost, B.s));
  }
  TD_CUDA(cudaStreamSynchronize(B.s));
  for (size_t i = 0; i < calls.size(); ++i) {
    OrthCall& q = calls[i];
    Prob& p = *q.p;
    for (int j = 0; j < q.nc; ++j) {
      if (!kh[i][j] || *q.N >= std::min(q.cap, p.ov)) continue;
      B.rl.add(rowop(R_COPY, p.ov, q.S + (size_t)(*q.N) * p.ov, q.cand + (size_t)j * p.ov));
      ++*q.N;
    }
  }
  B.rl.run(B.s);
}

// ---------------------------------------------------------------------------
// rid: (T - lam_j) v_j = R_j for the unconverged roots of every listed problem
// (Eq. precondition with the ris operator), block Galerkin per problem,
// diag-preconditioned expansion, stopped at |res_j| <= inner_tol |R_j| or
// inner_max_iter iterations (the same reading as the single-solve path).
void inner_rid_batch(Batch& B, std::vector<Prob*>& ps) {
  const Variant& v = *B.var;
  // R rows of the todo roots are p.R[0..nu), shifts p.lam[todo] (host values in p.om)
  std::vector<Prob*> act;
  for (Prob* p : ps) {
    p->Ns = 0;
    const int nu = (int)p->todo.size();
    if (nu == 0) continue;
    // seed: diag-preconditioned residuals
    for (int j = 0; j < nu; ++j) {
      RowOp r = rowop(R_PRECOND, p->ov, p->icand.as<float>() + (size_t)j * p->ov,
                      p->cand.as<float>() + (size_t)j * p->ov);   // cand holds the gathered residuals
      r.d = p->c->delta.as<double>();
      r.s0 = p->om[p->todo[j]];
      B.rl.add(r);
    }
    act.push_back(p);
  }
  B.rl.run(B.s);
  if (act.empty()) return;
  std::vector<OrthCall> oc;
  for (Prob* p : act) oc.push_back(OrthCall{p, p->S.as<float>(), &p->Ns, p->icand.as<float>(), (int)p->todo.size(), kInnerCap});
  orth_append_batch(B, oc);
  std::vector<OpCall> calls;
  for (Prob* p : act) calls.push_back(OpCall{p, p->S.as<float>(), p->TS.as<float>(), p->Ns});
  operator_batch(B, calls, true);
  std::vector<int> nold(act.size(), 0);
  std::vector<char> fin(act.size(), 0);
  const int maxit = act.front()->o.inner_max_iter;
  std::vector<BLu> lu;
  DevBuf d_lu(1, B.s);
  for (int it = 0; it < maxit; ++it) {
    // t = S^T TS (full, FP64), h[j][r] = R_j . S_r
    B.g.reset(v.bm, v.bn);
    for (size_t i = 0; i < act.size(); ++i) {
      if (fin[i]) continue;
      Prob& p = *act[i];
      const int nu = (int)p.todo.size();
      B.g.add(p.Ns, p.Ns, p.ov, p.S.as<float>(), 0, p.ov, 1, p.TS.as<float>(), 0, 1, p.ov, nullptr, p.ti.as<double>(),
              kInnerCap, 1, 1.f, 0.f);
      B.g.add(nu, p.Ns, p.ov, p.cand.as<float>(), 0, p.ov, 1, p.S.as<float>(), 0, 1, p.ov, nullptr, p.h.as<double>(),
              p.Ns, 1, 1.f, 0.f);
    }
    B.g.run(v, B.s);
    lu.clear();
    int nmax = 1;
    for (size_t i = 0; i < act.size(); ++i) {
      if (fin[i]) continue;
      Prob& p = *act[i];
      for (size_t j = 0; j < p.todo.size(); ++j)
        lu.push_back(BLu{p.ti.as<double>(), kInnerCap, p.Ns, p.om[p.todo[j]], p.h.as<double>() + j * p.Ns,
                         p.y.as<double>() + j * p.Ns});
      nmax = std::max(nmax, p.Ns);
    }
    if (lu.empty()) break;
    if (d_lu.bytes < lu.size() * sizeof(BLu)) d_lu = DevBuf(lu.size() * sizeof(BLu), B.s);
    TD_CUDA(cudaMemcpyAsync(d_lu.p, lu.data(), lu.size() * sizeof(BLu), cudaMemcpyHostToDevice, B.s));
    batch_lu(d_lu.as<BLu>(), (int)lu.size(), nmax, B.s);
    // v = y S, Tv = y TS, res = Tv - lam v - R
    B.g.reset(v.bm, v.bn);
    for (size_t i = 0; i < act.size(); ++i) {
      if (fin[i]) continue;
      Prob& p = *act[i];
      const int nu = (int)p.todo.size();
      B.g.add(nu, p.ov, p.Ns, p.y.as<double>(), 2, p.Ns, 1, p.S.as<float>(), 0, p.ov, 1, p.v.as<float>(), nullptr,
              p.ov, 1, 1.f, 0.f);
      B.g.add(nu, p.ov, p.Ns, p.y.as<double>(), 2, p.Ns, 1, p.TS.as<float>(), 0, p.ov, 1, p.Tv.as<float>(), nullptr,
              p.ov, 1, 1.f, 0.f);
    }
    B.g.run(v, B.s);
    for (size_t i = 0; i < act.size(); ++i) {
      if (fin[i]) continue;
      Prob& p = *act[i];
      for (size_t j = 0; j < p.todo.size(); ++j) {
        RowOp r = rowop(R_SRESID, p.ov, p.res.as<float>() + j * p.ov, p.Tv.as<float>() + j * p.ov,
                        p.v.as<float>() + j * p.ov, p.cand.as<float>() + j * p.ov);
        r.s0 = p.om[p.todo[j]];
        r.nrm = B.st(p) + 3 * p.k + j;   // scratch slots of the status block
        B.rl.add(r);
      }
    }
    B.rl.run(B.s);
    B.pull();
    // decide per problem; expand the unconverged
    std::vector<OrthCall> oc2;
    std::vector<size_t> who;
    for (size_t i = 0; i < act.size(); ++i) {
      if (fin[i]) continue;
      Prob& p = *act[i];
      const int nu = (int)p.todo.size();
      int nc = 0;
      for (int j = 0; j < nu; ++j) {
        const double rn = std::sqrt(B.hst(p)[3 * p.k + j]);
        if (!(rn <= p.o.inner_tol * p.rnorm0[j])) {
          RowOp r = rowop(R_PRECOND, p.ov, p.icand.as<float>() + (size_t)nc * p.ov, p.res.as<float>() + (size_t)j * p.ov);
          r.d = p.c->delta.as<double>();
          r.s0 = p.om[p.todo[j]];
          B.rl.add(r);
          ++nc;
        }
      }
      if (nc == 0 || it == maxit - 1 || p.Ns + nc > kInnerCap) {
        fin[i] = 1;
        B.rl.ops.resize(B.rl.ops.size() - nc);
        continue;
      }
      nold[i] = p.Ns;
      oc2.push_back(OrthCall{&p, p.S.as<float>(), &p.Ns, p.icand.as<float>(), nc, kInnerCap});
      who.push_back(i);
    }
    B.rl.run(B.s);
    if (oc2.empty()) break;
    orth_append_batch(B, oc2);
    calls.clear();
    for (size_t w = 0; w < who.size(); ++w) {
      Prob& p = *act[who[w]];
      const int n0 = nold[who[w]];
      if (p.Ns == n0) { fin[who[w]] = 1; continue; }
      calls.push_back(OpCall{&p, p.S.as<float>() + (size_t)n0 * p.ov, p.TS.as<float>() + (size_t)n0 * p.ov, p.Ns - n0});
    }
    operator_batch(B, calls, true);
  }
  // the inner solutions become the outer candidates
  for (Prob* p : act)
    for (size_t j = 0; j < p->todo.size(); ++j)
      B.rl.add(rowop(R_COPY, p->ov, p->cand.as<float>() + j * p->ov, p->v.as<float>() + j * p->ov));
  B.rl.run(B.s);
}

// ---------------------------------------------------------------------------
// One batched Davidson (TDA) on the exact (ris = false) or ris operator, with
// the rid (inner) or diagonal preconditioner.  The guess rows are in p.X
// (ng[p] rows); k_of[p] wanted states; results in p.om, p.rr and p.X.
void davidson_batch(Batch& B, std::vector<Prob*>& ps, bool ris, bool rid, const std::vector<int>& ng,
                    const std::vector<int>& k_of, const std::vector<double>& tol, int max_iter) {
  const Variant* vp = B.var;
  std::vector<OrthCall> oc;
  for (size_t i = 0; i < ps.size(); ++i) {
    Prob& p = *ps[i];
    p.N = 0;
    p.done = false;
    p.converged = false;
    p.n_iter = 0;
    p.have_prev = false;
    p.om.assign(k_of[i], 0.0);
    p.rr.assign(k_of[i], 1.0);
    // guess rows X -> cand, orthonormalised into V
    for (int j = 0; j < ng[i]; ++j)
      B.rl.add(rowop(R_COPY, p.ov, p.cand.as<float>() + (size_t)j * p.ov, p.X.as<float>() + (size_t)j * p.ov));
    oc.push_back(OrthCall{&p, p.V.as<float>(), &p.N, p.cand.as<float>(), ng[i], kCap});
  }
  B.rl.run(B.s);
  if (!vp) B.var = &variants()[0];
  orth_append_batch(B, oc);
  std::vector<OpCall> calls;
  for (Prob* p : ps) calls.push_back(OpCall{p, p->V.as<float>(), p->W.as<float>(), p->N});
  if (!vp && !ris) autotune(B, calls);
  operator_batch(B, calls, ris);
  std::vector<BEig> eg;
  DevBuf d_eg(ps.size() * sizeof(BEig), B.s);
  for (int it = 1; it <= max_iter; ++it) {
    std::vector<Prob*> act;
    for (Prob* p : ps)
      if (!p->done) act.push_back(p);
    if (act.empty()) break;
    const Variant& v = *B.var;
    // projected matrix a = V^T W (full, FP64)
    B.g.reset(v.bm, v.bn);
    for (Prob* p : act)
      B.g.add(p->N, p->N, p->ov, p->V.as<float>(), 0, p->ov, 1, p->W.as<float>(), 0, 1, p->ov, nullptr,
              p->a.as<double>(), kCap, 1, 1.f, 0.f);
    B.g.run(v, B.s);
    // lowest kk eigenpairs
    eg.clear();
    int nmax = 1;
    for (size_t i = 0; i < act.size(); ++i) {
      Prob& p = *act[i];
      const int kk = std::min((int)p.om.size(), p.N);
      eg.push_back(BEig{p.a.as<double>(), kCap, p.N, kk, B.st(p), p.xv.as<double>()});
      nmax = std::max(nmax, p.N);
      p.n_iter = it;
    }
    TD_CUDA(cudaMemcpyAsync(d_eg.p, eg.data(), eg.size() * sizeof(BEig), cudaMemcpyHostToDevice, B.s));
    batch_eig(d_eg.as<BEig>(), (int)eg.size(), nmax, B.s);
    // Ritz vectors X = x V, AX = x W; residuals R = AX - lam X
    B.g.reset(v.bm, v.bn);
    for (Prob* p : act) {
      const int kk = std::min((int)p->om.size(), p->N);
      B.g.add(kk, p->ov, p->N, p->xv.as<double>(), 2, p->N, 1, p->V.as<float>(), 0, p->ov, 1, p->X.as<float>(),
              nullptr, p->ov, 1, 1.f, 0.f);
      B.g.add(kk, p->ov, p->N, p->xv.as<double>(), 2, p->N, 1, p->W.as<float>(), 0, p->ov, 1, p->AX.as<float>(),
              nullptr, p->ov, 1, 1.f, 0.f);
    }
    B.g.run(v, B.s);
    for (Prob* p : act) {
      const int kk = std::min((int)p->om.size(), p->N);
      for (int j = 0; j < kk; ++j) {
        RowOp r = rowop(R_RESID, p->ov, p->R.as<float>() + (size_t)j * p->ov, p->AX.as<float>() + (size_t)j * p->ov,
                        p->X.as<float>() + (size_t)j * p->ov);
        r.sp = B.st(*p) + j;
        r.nrm = B.st(*p) + p->k + j;
        B.rl.add(r);
      }
    }
    B.rl.run(B.s);
    B.pull();
    // convergence and the directions to add
    std::vector<Prob*> need;
    for (size_t i = 0; i < act.size(); ++i) {
      Prob& p = *act[i];
      const int kk = std::min((int)p.om.size(), p.N);
      const double tl = tol[std::find(ps.begin(), ps.end(), &p) - ps.begin()];
      p.todo.clear();
      for (int j = 0; j < kk; ++j) {
        p.om[j] = B.hst(p)[j];
        p.rr[j] = std::sqrt(B.hst(p)[p.k + j]);
        if (!std::isfinite(p.om[j]) || !std::isfinite(p.rr[j]))
          throw Error(TDDFT_ERR_INDEFINITE, "non-finite Ritz values in a batched solve");
        if (!(p.rr[j] < tl)) p.todo.push_back(j);
      }
      if (btrace()) {
        double mr = 0.0;
        for (int j = 0; j < kk; ++j) mr = std::max(mr, p.rr[j]);
        fprintf(stderr, "[tddft-batch] %s it=%d prob=%zu/%zu ov=%d N=%d kk=%d omega0=%.10f max|r|=%.3e todo=%zu\n",
                ris ? "ris" : (rid ? "rid" : "diag"), it, i, act.size(), p.ov, p.N, kk, p.om[0], mr, p.todo.size());
      }
      if (p.todo.empty() && kk == (int)p.om.size()) { p.done = true; p.converged = true; continue; }
      if (it == max_iter) { p.done = true; continue; }
      need.push_back(&p);
    }
    if (need.empty()) break;
    // gather the residuals of the unconverged roots into cand
    for (Prob* p : need) {
      p->rnorm0.resize(p->todo.size());
      for (size_t j = 0; j < p->todo.size(); ++j) {
        B.rl.add(rowop(R_COPY, p->ov, p->cand.as<float>() + j * p->ov, p->R.as<float>() + (size_t)p->todo[j] * p->ov));
        p->rnorm0[j] = p->rr[p->todo[j]] > 0 ? p->rr[p->todo[j]] : 1.0;
      }
    }
    B.rl.run(B.s);
    if (rid) {
      inner_rid_batch(B, need);
    } else {
      for (Prob* p : need)
        for (size_t j = 0; j < p->todo.size(); ++j) {
          RowOp r = rowop(R_PRECOND, p->ov, p->cand.as<float>() + j * p->ov, p->cand.as<float>() + j * p->ov);
          r.d = p->c->delta.as<double>();
          r.s0 = p->om[p->todo[j]];
          B.rl.add(r);
        }
      B.rl.run(B.s);
    }
    // thick restart when the space would overflow: V <- the current Ritz
    // vectors and, where they fit with the new directions, those of the
    // previous iteration (their products recomputed)
    std::vector<Prob*> rst;
    for (Prob* p : need) {
      const int nu = (int)p->todo.size();
      if (p->N + nu <= std::min(kCap, p->ov)) continue;
      const int kk = std::min((int)p->om.size(), p->N);
      for (int j = 0; j < kk; ++j) {
        B.rl.add(rowop(R_COPY, p->ov, p->V.as<float>() + (size_t)j * p->ov, p->X.as<float>() + (size_t)j * p->ov));
        B.rl.add(rowop(R_COPY, p->ov, p->W.as<float>() + (size_t)j * p->ov, p->AX.as<float>() + (size_t)j * p->ov));
      }
      p->N = kk;
      if (p->have_prev && 2 * kk + nu <= std::min(kCap, p->ov)) {
        for (int j = 0; j < kk; ++j)
          B.rl.add(rowop(R_COPY, p->ov, p->tmp.as<float>() + (size_t)j * p->ov, p->Xprev.as<float>() + (size_t)j * p->ov));
        rst.push_back(p);
      }
    }
    B.rl.run(B.s);
    if (!rst.empty()) {
      // tmp is the orthonormalisation's scratch: move the previous vectors to R first
      for (Prob* p : rst) {
        const int kk = p->N;
        for (int j = 0; j < kk; ++j)
          B.rl.add(rowop(R_COPY, p->ov, p->R.as<float>() + (size_t)j * p->ov, p->tmp.as<float>() + (size_t)j * p->ov));
      }
      B.rl.run(B.s);
      std::vector<OrthCall> oc3;
      std::vector<int> n0;
      for (Prob* p : rst) {
        n0.push_back(p->N);
        oc3.push_back(OrthCall{p, p->V.as<float>(), &p->N, p->R.as<float>(), p->N, kCap});
      }
      orth_append_batch(B, oc3);
      std::vector<OpCall> rc;
      for (size_t i = 0; i < rst.size(); ++i) {
        Prob* p = rst[i];
        if (p->N > n0[i])
          rc.push_back(OpCall{p, p->V.as<float>() + (size_t)n0[i] * p->ov, p->W.as<float>() + (size_t)n0[i] * p->ov,
                              p->N - n0[i]});
      }
      operator_batch(B, rc, ris);
    }
    // the current Ritz vectors become the previous ones of the next iteration
    for (Prob* p : need) {
      const int kk = std::min((int)p->om.size(), p->N);
      for (int j = 0; j < kk; ++j)
        B.rl.add(rowop(R_COPY, p->ov, p->Xprev.as<float>() + (size_t)j * p->ov, p->X.as<float>() + (size_t)j * p->ov));
      p->have_prev = true;
    }
    B.rl.run(B.s);
    std::vector<int> nold;
    oc.clear();
    for (Prob* p : need) {
      nold.push_back(p->N);
      oc.push_back(OrthCall{p, p->V.as<float>(), &p->N, p->cand.as<float>(), (int)p->todo.size(), kCap});
    }
    orth_append_batch(B, oc);
    calls.clear();
    for (size_t i = 0; i < need.size(); ++i) {
      Prob* p = need[i];
      if (p->N == nold[i]) { p->done = true; continue; }
      calls.push_back(OpCall{p, p->V.as<float>() + (size_t)nold[i] * p->ov, p->W.as<float>() + (size_t)nold[i] * p->ov,
                             p->N - nold[i]});
    }
    operator_batch(B, calls, ris);
  }
}

}  // namespace

// ===========================================================================

tddft_status solve_tda_batch(Ctx* const* ctxs, int n, const tddft_opts* opts, double* omega, double* resid,
                             tddft_stats* stats, tddft_batch_info* info) {
  auto t0 = Clock::now();
  g_launches = 0;
  TD_REQUIRE(n >= 1 && ctxs && opts && omega, TDDFT_ERR_ARG, "batch: bad arguments");
  Batch B;
  B.s = ctxs[0]->s;
  B.g.ring = &B.ring;
  B.rl.ring = &B.ring;
  B.P.resize(n);
  int kmax = 1;
  for (int i = 0; i < n; ++i) {
    Ctx* c = ctxs[i];
    TD_REQUIRE(c != nullptr, TDDFT_ERR_ARG, "batch: null context");
    TD_REQUIRE(c->device == ctxs[0]->device, TDDFT_ERR_ARG, "batch: contexts on different devices");
    TD_REQUIRE((c->precisions & 2) != 0, TDDFT_ERR_ARG, "batch: contexts need the MIXED factor copies");
    const tddft_opts& o = opts[i];
    TD_REQUIRE(o.n_states >= 1 && o.n_states <= 32, TDDFT_ERR_ARG, "batch: n_states must be 1..32");
    TD_REQUIRE(o.precond == TDDFT_PRECOND_DIAG || o.precond == TDDFT_PRECOND_RID, TDDFT_ERR_ARG,
               "batch: unknown preconditioner");
    TD_REQUIRE(o.tol > 0 && o.inner_tol > 0 && o.guess_tol > 0 && o.max_iter >= 1 && o.inner_max_iter >= 1,
               TDDFT_ERR_ARG, "batch: tolerances / iteration limits must be positive");
    TD_REQUIRE(!c->exact(TDDFT_MIXED).has_variants(), TDDFT_ERR_ARG, "batch: variant terms are not supported");
    Prob& p = B.P[i];
    p.c = c;
    p.o = o;
    p.no = c->no; p.nv = c->nv; p.ov = c->ov;
    p.k = std::min(o.n_states, p.ov);
    const int extra = o.n_extra_guess >= 0 ? o.n_extra_guess : (o.precond == TDDFT_PRECOND_RID ? std::min(p.k, 3) : 8);
    p.k0 = std::min(p.k + extra, p.ov);
    TD_REQUIRE(std::min(p.k0 + 8, p.ov) <= c->n_order, TDDFT_ERR_ARG, "batch: too many initial guesses");
    TD_REQUIRE(2 * p.k0 <= kCap, TDDFT_ERR_ARG, "batch: too many states for the batched subspace");
    kmax = std::max(kmax, p.k0 + 8);
  }
  // status block: [lam kmax][rn2 kmax][rn2 of inner roots kmax]...
  B.stride = 4 * (kmax + 8);
  B.status = DevBuf((size_t)B.stride * n * 8, B.s);
  TD_CUDA(cudaMallocHost(&B.h_status, (size_t)B.stride * n * 8));
  cudaStream_t s = B.s;
  for (int i = 0; i < n; ++i) {
    Prob& p = B.P[i];
    Ctx& c = *p.c;
    p.st_off = i * B.stride;
    p.k = std::max(p.k, 0);
    // the status slots index by the largest k of this problem's solves
    p.k = std::max(p.k, p.k0);
    FactorSet fx = c.exact(TDDFT_MIXED), fr = c.ris(TDDFT_MIXED);
    p.ex = Ops{fx.nJ, fx.nK, 0, fx.Jov, fx.Koo, fx.Kvv};
    p.ris = Ops{fr.nJ, fr.nK, 1, fr.Jov, fr.Koo, fr.Kvv};
    // the largest operator call: the initial space (N_init + 8 rows for the
    // guess on the ris operator) or the new directions of one iteration (<= k)
    p.mmax = std::max(std::min(p.k0 + 8, p.ov), p.k);
    const size_t ov = p.ov;
    const size_t zrow = (size_t)p.mmax * p.no * p.nv * 4;
    p.pc_ex = (int)std::max<size_t>(1, std::min<size_t>(p.ex.nK > 0 ? p.ex.nK : 1, kZBudget / std::max<size_t>(zrow, 1)));
    p.pc_ris = (int)std::max<size_t>(1, std::min<size_t>(p.ris.nK > 0 ? p.ris.nK : 1, kZBudget / std::max<size_t>(zrow, 1)));
    const int pcz = std::max(p.pc_ex, p.pc_ris);
    const int mrow = p.mmax;
    p.t = DevBuf((size_t)std::max(p.ex.nJ, p.ris.nJ) * mrow * 4 + 4, s);
    p.J = DevBuf((size_t)mrow * ov * 4, s);
    p.K1 = DevBuf((size_t)mrow * ov * 4, s);
    p.Z = DevBuf((size_t)mrow * p.no * pcz * p.nv * 4, s);
    p.V = DevBuf((size_t)kCap * ov * 4, s);
    p.W = DevBuf((size_t)kCap * ov * 4, s);
    p.a = DevBuf((size_t)kCap * kCap * 8, s);
    p.xv = DevBuf((size_t)kCap * kCap * 8, s);
    p.X = DevBuf((size_t)kCap * ov * 4, s);
    p.AX = DevBuf((size_t)kCap * ov * 4, s);
    p.R = DevBuf((size_t)kCap * ov * 4, s);
    p.cand = DevBuf((size_t)kCap * ov * 4, s);
    p.tmp = DevBuf((size_t)kCap * ov * 4, s);
    p.C = DevBuf((size_t)kCap * kCap * 8, s);
    p.G = DevBuf((size_t)kCap * kCap * 8, s);
    p.Tm = DevBuf((size_t)kCap * kCap * 8, s);
    p.keep = DevBuf((size_t)kCap * 4, s);
    p.Xprev = DevBuf((size_t)kCap * ov * 4, s);
    p.nrm0 = DevBuf((size_t)kCap * 8, s);
    p.S = DevBuf((size_t)kInnerCap * ov * 4, s);
    p.TS = DevBuf((size_t)kInnerCap * ov * 4, s);
    p.ti = DevBuf((size_t)kInnerCap * kInnerCap * 8, s);
    p.h = DevBuf((size_t)kCap * kInnerCap * 8, s);
    p.y = DevBuf((size_t)kCap * kInnerCap * 8, s);
    p.v = DevBuf((size_t)kCap * ov * 4, s);
    p.Tv = DevBuf((size_t)kCap * ov * 4, s);
    p.res = DevBuf((size_t)kCap * ov * 4, s);
    p.icand = DevBuf((size_t)kCap * ov * 4, s);
  }
  for (Prob& p : B.P) {
    B.ex_rounds = std::max(B.ex_rounds, p.ex.nK > 0 ? (p.ex.nK + p.pc_ex - 1) / p.pc_ex : 1);
    B.s1_cap += p.mmax + 1;
    B.s2_cap += 2;
    B.comb_cap += p.mmax;
  }
  // initial guesses: unit vectors at the smallest Delta, then (rid) a Davidson
  // on the ris operator to guess_tol for N_init states (Sec. 3.1-3.2)
  std::vector<Prob*> all, rid_ps, diag_ps;
  for (Prob& p : B.P) {
    all.push_back(&p);
    (p.o.precond == TDDFT_PRECOND_RID ? rid_ps : diag_ps).push_back(&p);
  }
  std::vector<int> ng, kof;
  std::vector<double> tl;
  for (Prob* p : rid_ps) {
    const int kg = std::min(p->k0 + 8, p->ov);
    for (int j = 0; j < kg; ++j) {
      RowOp r = rowop(R_UNIT, p->ov, p->X.as<float>() + (size_t)j * p->ov, nullptr);
      r.idx = j;
      r.ord = p->c->order.as<int>();
      B.rl.add(r);
    }
  }
  for (Prob* p : diag_ps)
    for (int j = 0; j < p->k0; ++j) {
      RowOp r = rowop(R_UNIT, p->ov, p->X.as<float>() + (size_t)j * p->ov, nullptr);
      r.idx = j;
      r.ord = p->c->order.as<int>();
      B.rl.add(r);
    }
  B.rl.run(s);
  if (!rid_ps.empty()) {
    ng.clear(); kof.clear(); tl.clear();
    for (Prob* p : rid_ps) {
      ng.push_back(std::min(p->k0 + 8, p->ov));
      kof.push_back(p->k0);
      tl.push_back(p->o.guess_tol);
    }
    B.var = &variants()[0];
    davidson_batch(B, rid_ps, true, false, ng, kof, tl, rid_ps.front()->o.max_iter);
    B.var = nullptr;
  }
  // outer solves on the exact operator (guess rows in X)
  ng.clear(); kof.clear(); tl.clear();
  std::vector<Prob*> outer;
  for (Prob& p : B.P) {
    outer.push_back(&p);
    ng.push_back(p.k0);
    kof.push_back(std::min(p.o.n_states, p.ov));
    tl.push_back(p.o.tol);
  }
  // rid and diag problems in one lockstep pass each
  std::vector<Prob*> o_rid, o_diag;
  std::vector<int> ng_r, ng_d, k_r, k_d;
  std::vector<double> t_r, t_d;
  for (size_t i = 0; i < outer.size(); ++i) {
    if (outer[i]->o.precond == TDDFT_PRECOND_RID) { o_rid.push_back(outer[i]); ng_r.push_back(ng[i]); k_r.push_back(kof[i]); t_r.push_back(tl[i]); }
    else { o_diag.push_back(outer[i]); ng_d.push_back(ng[i]); k_d.push_back(kof[i]); t_d.push_back(tl[i]); }
  }
  int max_iter = 1;
  for (Prob& p : B.P) max_iter = std::max(max_iter, p.o.max_iter);
  if (!o_rid.empty()) davidson_batch(B, o_rid, false, true, ng_r, k_r, t_r, max_iter);
  if (!o_diag.empty()) davidson_batch(B, o_diag, false, false, ng_d, k_d, t_d, max_iter);
  TD_CUDA(cudaStreamSynchronize(s));
  // outputs
  check_batch_tc(B.s);
  size_t off = 0;
  bool all_ok = true;
  int iters = 0;
  for (int i = 0; i < n; ++i) {
    Prob& p = B.P[i];
    const int k = (int)p.om.size();
    for (int j = 0; j < k; ++j) {
      omega[off + j] = p.om[j];
      if (resid) resid[off + j] = p.rr[j];
    }
    off += k;
    all_ok = all_ok && p.converged;
    iters = std::max(iters, p.n_iter);
    if (stats) {
      tddft_stats& st = stats[i];
      std::memset(&st, 0, sizeof(st));
      st.n_iter = p.n_iter;
      st.n_matvec = (int)p.mv;
      st.n_ris_matvec = (int)p.ris_mv;
      st.converged = p.converged ? 1 : 0;
      double m = 0.0;
      for (double r : p.rr) m = std::max(m, r);
      st.max_resid = m;
      st.max_resid_certified = -1.0;   // no separate recomputation in the batched solves
      st.t_total_s = std::chrono::duration<double>(Clock::now() - t0).count();
    }
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    const auto& vs = variants();
    info->n_variants = (int)std::min<size_t>(vs.size(), 8);
    for (int v = 0; v < 8; ++v) info->autotune_ms[v] = v < (int)B.tune_ms.size() ? B.tune_ms[v] : -1.0;
    info->variant = -1;
    for (size_t v = 0; v < vs.size(); ++v)
      if (B.var == &vs[v]) info->variant = (int)v;
    info->outer_iterations = iters;
    info->launches = g_launches;
    info->graph_launches = B.graph_launches;
    info->graph_nodes = B.graph_nodes;
    info->t_total_s = std::chrono::duration<double>(Clock::now() - t0).count();
  }
  return all_ok ? TDDFT_OK : TDDFT_ERR_NOCONV;
}

}  // namespace tddft
