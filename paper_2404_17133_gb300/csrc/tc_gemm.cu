// tcgen05 tensor-core kernel for the exchange contraction of the exact operator,
//   K1[(n,i)][b] = sum_P sum_a Z[(n,i)][P][a] L^P_ab           (Eq. hessian, (ij|ab) term)
// the dominant cost of every response product (about 90% of its flops).
//
// Operands are split into BF16 hi + lo parts (x = hi + lo exactly to ~2^-17);
// each tile pair contributes hi*hi + hi*lo + lo*hi (the lo*lo term is below the
// FP32 accumulator's resolution) so the product has ~FP32 accuracy at BF16
// tensor-core rate.
//
// Layout / mapping (all K-major, so both operands stream along a):
//   A = Z  viewed as a 3-D tensor (a: nv, P: pn, row: M), row pitch pn*nvp
//   B = L  viewed as a 3-D tensor (a: nv, b: nv, P: pn); L^P is symmetric so the
//          row b of L^P read along a is the column b of the GEMM's B operand
//   K loop: for each P in the CTA's split range, a-blocks of 64 (128 bytes, one
//          128B-swizzle atom); TMA zero-fills a >= nv, b >= nv and rows >= M.
// CTA = 128 x 128 output tile, 6 warps: warp 0 issues TMA loads, warp 1 owns the
// tensor memory and one elected lane issues tcgen05.mma, warps 2-5 drain the
// FP32 accumulator from TMEM.  A 3-stage mbarrier ring connects producer and MMA;
// tcgen05.commit releases a stage when its MMAs have read it.
// Split-K: blockIdx.z takes a contiguous range of (P, a-block) steps and writes
// its own FP32 partial tile; a fixed-order reduction sums the partials.
//
// Every wait on an mbarrier is bounded: on timeout the thread records an error
// code in `err` and leaves the loop; the host turns it into TDDFT_ERR_CUDA.
#include <cuda.h>

#include "tc_gemm.cuh"
#include "vecops.cuh"

namespace tddft {

namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;                       // bf16 elements per 128-byte row
constexpr int STAGES = 3;
constexpr int A_BYTES = BM * BK * 2;          // 16 KB per hi or lo tile
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int THREADS = 192;
constexpr long long WAIT_LIMIT = 1ll << 23;

struct Params {
  int M, N;          // output rows / columns
  int nab;           // a-blocks per P
  int total;         // pn * nab steps
  int per_split;     // steps per split
  float* part;       // [splits][M][N]
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the completion of phase `parity`; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  const uint64_t addr = smem_u32(p);
  return ((addr & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, M = 128, N = BN.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__global__ void __launch_bounds__(THREADS, 1)
k1_tc_kernel(const __grid_constant__ CUtensorMap mA_hi, const __grid_constant__ CUtensorMap mA_lo,
             const __grid_constant__ CUtensorMap mB_hi, const __grid_constant__ CUtensorMap mB_lo,
             Params p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int k_begin = blockIdx.z * p.per_split;
  const int k_end = min(p.total, k_begin + p.per_split);
  const int nk = max(0, k_end - k_begin);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)), "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    bool ok = true;
    for (int i = 0; i < nk && ok; ++i) {
      const int s = i % STAGES;
      const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) { atomicOr(p.err, 1); ok = false; break; }
      const int kb = k_begin + i;
      const int P = kb / p.nab, a0 = (kb - P * p.nab) * BK;
      unsigned char* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_3d(st, &mA_hi, &full[s], a0, P, m0);
      tma_load_3d(st + A_BYTES, &mA_lo, &full[s], a0, P, m0);
      tma_load_3d(st + 2 * A_BYTES, &mB_hi, &full[s], a0, n0, P);
      tma_load_3d(st + 2 * A_BYTES + B_BYTES, &mB_lo, &full[s], a0, n0, P);
    }
    // let the copies already issued land before the CTA can exit
    for (int i = max(0, nk - STAGES); i < nk; ++i) {
      if (!mbar_wait(&full[i % STAGES], (uint32_t)(i / STAGES) & 1u)) { atomicOr(p.err, 2); break; }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    bool ok = true;
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      if (!mbar_wait(&full[s], (uint32_t)(i / STAGES) & 1u)) { atomicOr(p.err, 4); ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* st = smem + s * STAGE_BYTES;
      const uint64_t ah = sdesc(st), al = sdesc(st + A_BYTES);
      const uint64_t bh = sdesc(st + 2 * A_BYTES), bl = sdesc(st + 2 * A_BYTES + B_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t off = (uint64_t)(kk * 32) >> 4;   // 16 bf16 = 32 bytes along K
        mma_bf16(tmem, ah + off, bh + off, (i > 0 || kk > 0) ? 1u : 0u);
        mma_bf16(tmem, ah + off, bl + off, 1u);
        mma_bf16(tmem, al + off, bh + off, 1u);
      }
      mma_commit(&empty[s]);
    }
    (void)ok;
    mma_commit(done);   // fires when every MMA issued above has completed
  } else if (warp >= 2) {
    // ---- epilogue: TMEM -> registers -> FP32 partial tile
    const int q = warp & 3;                 // TMEM lane quadrant of this warp
    const int row = m0 + q * 32 + lane;
    bool have = true;
    if (nk > 0) {
      if (!mbar_wait(done, 0)) { atomicOr(p.err, 8); have = false; }
      have = __all_sync(0xffffffffu, have);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    float* out = p.part + (size_t)blockIdx.z * p.M * p.N;
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
      uint32_t v[16];
      if (nk > 0 && have) {
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c;
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
      if (row < p.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c + j;
          if (col < p.N) out[(size_t)row * p.N + col] = __uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
  }
}

// Sum the split partials into out (FP32), accumulating when asked.
__global__ void k_sum_splits(const float* __restrict__ part, int S, long long MN, float* out,
                             int accumulate) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < MN;
       t += (long long)gridDim.x * blockDim.x) {
    float acc = accumulate ? out[t] : 0.f;
    for (int s = 0; s < S; ++s) acc += part[s * MN + t];
    out[t] = acc;
  }
}

// FP32 Z [M][pn*nv] -> BF16 hi/lo [M][pn][nvp] (row pitch padded to 16 bytes, pads zero)
__global__ void k_split_pad(const float* __restrict__ Z, int M, int pn, int nv, int nvp,
                            __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const long long tot = (long long)M * pn * nvp;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t % nvp);
    const long long rp = t / nvp;   // row * pn + P
    float v = 0.f;
    if (a < nv) v = Z[rp * nv + a];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[t] = h;
    lo[t] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    TD_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
    TD_REQUIRE(f != nullptr && q == cudaDriverEntryPointSuccess, TDDFT_ERR_CUDA,
               "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<EncodeFn>(f);
  }
  return fn;
}

CUtensorMap make_map(const void* base, const cuuint64_t dims[3], const cuuint64_t strides[2],
                     const cuuint32_t box[3]) {
  TD_REQUIRE((reinterpret_cast<uintptr_t>(base) & 15) == 0, TDDFT_ERR_ARG, "TMA base not 16-byte aligned");
  TD_REQUIRE(strides[0] % 16 == 0 && strides[1] % 16 == 0, TDDFT_ERR_ARG, "TMA strides not 16-byte multiples");
  CUtensorMap m;
  const cuuint32_t es[3] = {1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  TD_REQUIRE(r == CUDA_SUCCESS, TDDFT_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

}  // namespace

int tc_pad(int nv) { return (nv + 7) & ~7; }

void tc_split_pad(const float* Z, int M, int pn, int nv, __nv_bfloat16* hi, __nv_bfloat16* lo,
                  cudaStream_t s) {
  const long long tot = (long long)M * pn * tc_pad(nv);
  long long g = (tot + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_split_pad<<<(unsigned)g, 256, 0, s>>>(Z, M, pn, nv, tc_pad(nv), hi, lo);
  count_launch();
  TD_LAUNCH_CHECK();
}

void tc_exchange_k1(const __nv_bfloat16* Zhi, const __nv_bfloat16* Zlo, int M, int pn, int nv,
                    const __nv_bfloat16* Lhi, const __nv_bfloat16* Llo, float* out, bool accumulate,
                    int* err, cudaStream_t s) {
  if (M <= 0 || pn <= 0) return;
  const int nvp = tc_pad(nv);
  const int nab = (nv + BK - 1) / BK;
  const int total = pn * nab;
  const int mt = (M + BM - 1) / BM, nt = (nv + BN - 1) / BN;
  int splits = (2 * 152 + mt * nt - 1) / (mt * nt);
  if (splits > total) splits = total;
  if (splits < 1) splits = 1;
  const int per = (total + splits - 1) / splits;
  splits = (total + per - 1) / per;

  const cuuint64_t dA[3] = {(cuuint64_t)nv, (cuuint64_t)pn, (cuuint64_t)M};
  const cuuint64_t sA[2] = {(cuuint64_t)nvp * 2, (cuuint64_t)pn * nvp * 2};
  const cuuint32_t bA[3] = {BK, 1, BM};
  const cuuint64_t dB[3] = {(cuuint64_t)nv, (cuuint64_t)nv, (cuuint64_t)pn};
  const cuuint64_t sB[2] = {(cuuint64_t)nvp * 2, (cuuint64_t)nv * nvp * 2};
  const cuuint32_t bB[3] = {BK, BN, 1};
  CUtensorMap mAh = make_map(Zhi, dA, sA, bA), mAl = make_map(Zlo, dA, sA, bA);
  CUtensorMap mBh = make_map(Lhi, dB, sB, bB), mBl = make_map(Llo, dB, sB, bB);

  DevBuf part((size_t)splits * M * nv * 4, s);
  Params p{M, nv, nab, total, per, part.as<float>(), err};
  static bool attr = false;
  if (!attr) {
    TD_CUDA(cudaFuncSetAttribute(k1_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr = true;
  }
  dim3 grid(nt, mt, splits);
  k1_tc_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(mAh, mAl, mBh, mBl, p);
  count_launch();
  TD_LAUNCH_CHECK();
  const long long MN = (long long)M * nv;
  long long g = (MN + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_sum_splits<<<(unsigned)g, 256, 0, s>>>(part.as<float>(), splits, MN, out, accumulate ? 1 : 0);
  count_launch();
  TD_LAUNCH_CHECK();
}

}  // namespace tddft
