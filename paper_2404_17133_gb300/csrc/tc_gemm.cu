// tcgen05 tensor-core contraction over the auxiliary index,
//   C[m][n] (+)= sum_P sum_k A[m][P][k] B[P][n][k],
// used for the exchange terms of the response products (Eq. hessian):
//   K1[(n,i)][b] = sum_P sum_a Z[(n,i)][P][a] L^P_ab      ((ij|ab) term, k = a)
//   K2[(n,i)][a] = sum_P sum_j Q[(n,i)][P][j] L^P_ja      ((ib|ja) term, k = j)
// K1's contraction is the dominant cost of every product (about 70-90% of flops).
//
// Exact operator: every operand is scaled by a power of two s (so that
// max |s x| <= 2^14, or below 2^15 from a Cauchy-Schwarz bound for the stage-1
// results) and split into FP16 hi + lo parts, x s = hi + lo to ~2^-22 (11
// significand bits each; s keeps the lo parts of all but the negligible
// elements above FP16's normal range); each tile pair contributes
// hi*hi + hi*lo + lo*hi (lo*lo is below 2^-22), FP32 accumulation, and the
// sum is multiplied by 1 / (s_A s_B): an FP32-accurate product at the FP16
// tensor-core rate.  ris operator: BF16 factors (no scaling), the trial
// vectors as BF16 hi + lo.
//
// Layout / mapping (all K-major, so both operands stream along k):
//   A viewed as a 3-D tensor (k: Kin, P: pn, row: M), row pitch pn*ldk
//   B viewed as a 3-D tensor (k: Kin, n: N, P: pn), rows of ldk; for K1 the
//          rows of the symmetric L^P are its columns, for K2 B is L^P_ov
//          stored transposed ([P][a][j])
//   K loop: for each P in the CTA's split range, k-blocks of 128 bytes (one
//          128B-swizzle atom per row) or, for the hi+lo x hi+lo products, of
//          64 bytes (64B swizzle); TMA zero-fills k >= Kin, n >= N and rows >= M.
// CTA = 128 x 256 output tile, 6 warps: warp 0 issues TMA loads, warp 1 owns the
// tensor memory and one elected lane issues tcgen05.mma, warps 2-5 drain the
// FP32 accumulator from TMEM.  A 3- or 4-stage mbarrier ring (~192 KB) connects
// producer and MMA; tcgen05.commit releases a stage when its MMAs have read it.
// Split-K: blockIdx.z takes a contiguous range of (P, a-block) steps and writes
// its own FP32 partial tile; a fixed-order reduction sums the partials.
//
// Every wait on an mbarrier is bounded: on timeout the thread records an error
// code in `err` and leaves the loop; the host turns it into TDDFT_ERR_CUDA.
#include <algorithm>
#include <cstdlib>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "ctx.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"
#include "vecops.cuh"

namespace tddft {

namespace {

constexpr int BM = 128;
constexpr int BN = 256;                      // 128 x 256 MMA tiles (full tcgen05 rate per CTA)
constexpr int BK = 64;                       // bf16 elements per 128-byte row
constexpr int A_BYTES = BM * 128;             // 16 KB per hi or lo tile (128-byte rows)
constexpr int B_BYTES = BN * 128;
// Operand element types of the contraction: BF16 or FP16 (kind::f16, 64
// elements per 128-byte row) or FP8 e4m3 (kind::f8f6f4, 128 elements per row).
// Either way one tcgen05.mma consumes 32 bytes of K, so the descriptors
// advance alike.
enum ElemType : int { ET_BF16 = 0, ET_F16 = 1, ET_E4M3 = 2 };
template <int ET> struct Elem {
  static constexpr int BKE = ET == ET_E4M3 ? 128 : 64;
  // instruction-descriptor A and B type fields: kind::f16 F16 = 0, BF16 = 1; kind::f8f6f4 E4M3 = 0
  static constexpr uint32_t TYPE_BITS = ET == ET_BF16 ? ((1u << 7) | (1u << 10)) : 0u;
};
constexpr int elem_of(TcElt e) { return e == TcElt::F16 ? ET_F16 : ET_BF16; }
// Operand split modes: SINGLE = one product; BOTH = A and B as hi + lo
// (hi*hi + hi*lo + lo*hi); ASPLIT = A as hi + lo, B a plain operand
// (hi*B + lo*B: exact with respect to B, e.g. FP32 vectors against BF16 ris factors).
enum SplitMode : int { SINGLE = 0, BOTH = 1, ASPLIT = 2 };
__host__ __device__ constexpr bool a_split(int m) { return m != SINGLE; }
__host__ __device__ constexpr bool b_split(int m) { return m == BOTH; }
__host__ __device__ constexpr int n_parts_a(int m) { return a_split(m) ? 2 : 1; }
__host__ __device__ constexpr int n_parts_b(int m) { return b_split(m) ? 2 : 1; }

// Ring of the contraction kernel for rows of RB bytes along K (128: one
// 128-byte swizzle atom per row; 64: half as much K per stage in a 64-byte
// swizzle, so twice as many stages fit -- the split-B products, whose hi+lo
// tiles fill 96 KB per 128-byte stage, use it for a four-deep ring).
template <int MODE, int RB = 128> struct Cfg {
  static constexpr int STAGE_BYTES = (n_parts_a(MODE) * A_BYTES + n_parts_b(MODE) * B_BYTES) * RB / 128;
  static constexpr int STAGES = (MODE == SINGLE ? 4 : (MODE == ASPLIT ? 3 : 2)) * 128 / RB;   // ~192 KB ring
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
};
constexpr int THREADS = 192;
constexpr int S1_EPI_WARPS = 16;                   // stage-1 epilogue warps (4 per TMEM lane quadrant)
constexpr int S1_THREADS = 64 + 32 * S1_EPI_WARPS;   // producer, MMA and the epilogue warps

struct Params {
  int M, N;          // output rows / columns
  int Kin;           // k extent per P (the last k-block of a P issues only the MMAs it needs)
  int nab;           // k-blocks per P
  int total;         // pn * nab steps
  int per_split;     // steps per split
  float* part;       // [splits][M][N]
  int* err;
};


__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}


// Instruction descriptor: D = F32, A and B of the same type (BF16 or FP16
// for kind::f16, E4M3 for kind::f8f6f4), both K-major, M = 128, N = nb.
template <int ET>
__host__ __device__ constexpr uint32_t idesc_of(int nb = BN) {
  return (1u << 4) | Elem<ET>::TYPE_BITS | ((uint32_t)(nb >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int ET>
__device__ __forceinline__ void mma_op(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accum,
                                       uint32_t idesc = idesc_of<ET>()) {
  if constexpr (ET == ET_E4M3) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
  }
}

// Shared-memory matrix descriptor for RB-byte rows: K-major, 128-byte (RB =
// 128) or 64-byte (RB = 64) swizzle, 8-row groups 8 RB bytes apart.
template <int RB>
__device__ __forceinline__ uint64_t sdesc_rb(const void* p) {
  if constexpr (RB == 128) return sdesc(p);
  const uint64_t addr = smem_u32(p);
  return ((addr & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)((8 * RB) >> 4) << 32) | (1ull << 46) |
         (4ull << 61);
}

// TMA load into the same shared-memory offset of every CTA in `mask` of the
// cluster, signalling each one's mbarrier at the same offset.
__device__ __forceinline__ void tma_load_3d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                               int c2, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%3, %4, %5}], [%2], %6;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "h"(mask)
      : "memory");
}

// Arrive on the mbarrier at this offset in every CTA of `mask` when the MMAs
// issued so far have completed.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}


// CL = 2: the CTAs run in clusters of two along the M tiles; both need the same
// B tile, so each loads half of its rows and multicasts them to both (halving
// each SM's B traffic), and a stage is refilled only after both CTAs' MMAs
// have read it (their commits arrive on both CTAs' `empty` barriers).
// CX = 2 (with CL = 2): clusters of 2 x 2, the two CTAs of each N pair also
// share their A tile the same way.  Cluster rank r = x + CX y: the CTAs that
// share r's A tile are those of its row y, those that share its B tile those
// of its column x; r's stage is written by both, so r's `empty` barrier counts
// the commits of all of them (CL + CX - 1).
template <int MODE, int ET, int CL = 1, int RB = 128, int CX = 1>
__global__ void __launch_bounds__(THREADS, 1)
k1_tc_kernel(const __grid_constant__ CUtensorMap mA_hi, const __grid_constant__ CUtensorMap mA_lo,
             const __grid_constant__ CUtensorMap mB_hi, const __grid_constant__ CUtensorMap mB_lo,
             Params p) {
  constexpr int STAGES = Cfg<MODE, RB>::STAGES;
  constexpr int STAGE_BYTES = Cfg<MODE, RB>::STAGE_BYTES;
  constexpr int AB = A_BYTES * RB / 128, BB = B_BYTES * RB / 128;   // one part tile
  constexpr int B_OFF = a_split(MODE) ? 2 * AB : AB;                // first B tile in a stage
  constexpr int BKE = Elem<ET>::BKE * RB / 128;                     // K elements per k-block
  constexpr int KSTEPS = RB / 32;                                   // 32-byte K steps per k-block
  constexpr int CN = CL * CX;                                       // CTAs per cluster
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

  const uint32_t crank = CN > 1 ? cluster_rank() : 0u;
  const uint32_t cx = crank % CX, cy = crank / CX;
  uint16_t mask_a = 0, mask_b = 0;   // CTAs receiving this CTA's A / B rows
#pragma unroll
  for (int x = 0; x < CX; ++x) mask_a |= (uint16_t)(1u << (x + CX * cy));
#pragma unroll
  for (int y = 0; y < CL; ++y) mask_b |= (uint16_t)(1u << (cx + CX * y));
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], CL + CX - 1); }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)), "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  if constexpr (CN > 1) cluster_sync_all();   // every barrier of the cluster initialised
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
      const int P = kb / p.nab, a0 = (kb - P * p.nab) * BKE;
      unsigned char* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      if constexpr (CX > 1) {
        // this CTA's share of the A rows, to every CTA of its row
        constexpr int HA = AB / CX;
        const int mh = m0 + (int)cx * (BM / CX);
        tma_load_3d_mc(st + cx * HA, &mA_hi, &full[s], a0, P, mh, mask_a);
        if (a_split(MODE)) tma_load_3d_mc(st + AB + cx * HA, &mA_lo, &full[s], a0, P, mh, mask_a);
      } else {
        tma_load_3d(st, &mA_hi, &full[s], a0, P, m0);
        if (a_split(MODE)) tma_load_3d(st + AB, &mA_lo, &full[s], a0, P, m0);
      }
      if constexpr (CL > 1) {
        // this CTA's share of the B rows, to every CTA of its column
        constexpr int HB = BB / CL;
        const int nh = n0 + (int)cy * (BN / CL);
        tma_load_3d_mc(st + B_OFF + cy * HB, &mB_hi, &full[s], a0, nh, P, mask_b);
        if (b_split(MODE)) tma_load_3d_mc(st + B_OFF + BB + cy * HB, &mB_lo, &full[s], a0, nh, P, mask_b);
      } else {
        tma_load_3d(st + B_OFF, &mB_hi, &full[s], a0, n0, P);
        if (b_split(MODE)) tma_load_3d(st + B_OFF + BB, &mB_lo, &full[s], a0, n0, P);
      }
    }
    // let the copies already issued land before the CTA can exit
    for (int i = max(0, nk - STAGES); i < nk; ++i) {
      if (!mbar_wait(&full[i % STAGES], (uint32_t)(i / STAGES) & 1u)) { atomicOr(p.err, 2); break; }
    }
    if constexpr (CN > 1) {
      // and the peers' last commits arrive on this CTA's `empty` barriers
      for (int i = nk; i < nk + STAGES; ++i) {
        if (!mbar_wait(&empty[i % STAGES], ((uint32_t)(i / STAGES) & 1u) ^ 1u)) { atomicOr(p.err, 2); break; }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer.  The MMA spans only the tile's columns below N
    // (rounded up to 16) and, in the last k-block of each P, only the 32-byte
    // K steps below Kin: the skipped products are of TMA's zero fill.
    const int nb_cta = max(16, min(BN, (p.N - n0 + 15) & ~15));   // >= 16: a padding tile of a cluster
    const uint32_t idesc = idesc_of<ET>(nb_cta);
    bool ok = true;
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      if (!mbar_wait(&full[s], (uint32_t)(i / STAGES) & 1u)) { atomicOr(p.err, 4); ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* st = smem + s * STAGE_BYTES;
      const uint64_t ah = sdesc_rb<RB>(st), bh = sdesc_rb<RB>(st + B_OFF);
      const int kb = k_begin + i;
      const int rem = p.Kin - (kb % p.nab) * BKE;
      const int nks = rem >= BKE ? KSTEPS : (rem * KSTEPS + BKE - 1) / BKE;
#pragma unroll
      for (int kk = 0; kk < KSTEPS; ++kk) {
        if (kk < nks) {
          const uint64_t off = (uint64_t)(kk * 32) >> 4;   // 32 bytes along K per MMA
          mma_op<ET>(tmem, ah + off, bh + off, (i > 0 || kk > 0) ? 1u : 0u, idesc);
          if (b_split(MODE)) mma_op<ET>(tmem, ah + off, sdesc_rb<RB>(st + B_OFF + BB) + off, 1u, idesc);
          if (a_split(MODE)) mma_op<ET>(tmem, sdesc_rb<RB>(st + AB) + off, bh + off, 1u, idesc);
        }
      }
      if constexpr (CN > 1) mma_commit_mc(&empty[s], (uint16_t)(mask_a | mask_b));
      else mma_commit(&empty[s]);
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
        const int col0 = n0 + c;
        float* o = out + (size_t)row * p.N + col0;
        if ((p.N & 3) == 0 && col0 + 16 <= p.N) {   // 16-byte aligned: four vector stores
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(o + j) = make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                                            __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (col0 + j < p.N) o[j] = __uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
  }
  if constexpr (CN > 1) cluster_sync_all();   // no CTA leaves while another may still signal it
}


// ---------------------------------------------------------------------------
// Stage-1 contractions of the exchange terms, batched over P:
//   C_P[r][c] = sum_(k<K) A[r][k] B_P[c][k]   (r < M, c < N <= 256)
// written as BF16 hi (+ lo) into the stage-2 operand layout
//   out[(g*N + c)][P][ri] with r = g*R + ri, row pitch pn*ldo (ldo = pad8(R)):
//   K1: A = X^T per trial vector ([(n,a)][j]), B_P = L^P_oo ([i][j]) -> Z[(n,i)][P][a]
//   K2: A = X ([(n,j)][b]),            B_P = L^P_ov ([i][b]) -> Q[(n,i)][P][j]
// Persistent over P: the CTA owns one M-tile and the P range blockIdx.y*ppc ...;
// k-blocks of A and B_P stream through a TMA/mbarrier ring; the TMEM
// accumulator is double-buffered so the epilogue of one P overlaps the MMAs of
// the next (tmem_full / tmem_empty barriers).
struct S1Params {
  int M, N, R, ldo, pn, ppc, nkb;
  int K;               // k extent (the last k-block issues only the MMAs it needs)
  int nb;              // MMA N (multiple of 16, >= N)
  int acc_cols;        // TMEM columns per accumulator buffer
  int stages, stage_bytes, a_bytes, b_bytes;
  int a_res_bytes;     // RES: the resident A tile (every k-block, every part)
  void* out_hi;        // BF16 / FP16 parts (2-byte elements) or e4m3 bytes
  void* out_lo;
  // FP16 output: the accumulator times *mul before its split; FP8 output:
  // times mu[P] (one scale per auxiliary row)
  const float* mul;
  const float* mu;
  int* err;
};

__device__ __forceinline__ unsigned char to_e4m3(float x) {
  return (unsigned char)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float from_e4m3(unsigned char q) {
  return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3)));
}

// RES: the CTA's A tile (all k-blocks) is loaded once and stays in shared
// memory while the CTA walks its P range; the ring streams B_P only.
// CL = 2: the CTAs run in clusters of two along the M tiles; both need the same
// B_P tiles, so each loads half of the rows and multicasts them to both, and
// a stage is refilled only when both CTAs' MMAs have read it.
template <int MODE, int IN, int OUT, bool RES = false, int CL = 1>
__global__ void __launch_bounds__(S1_THREADS, 1)
k_stage1_tc(const __grid_constant__ CUtensorMap mA_hi, const __grid_constant__ CUtensorMap mA_lo,
            const __grid_constant__ CUtensorMap mB_hi, const __grid_constant__ CUtensorMap mB_lo,
            S1Params p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* ares = smem;                                   // RES: resident A
  unsigned char* ring = smem + (RES ? p.a_res_bytes : 0);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + p.stages * p.stage_bytes);
  uint64_t* empty = full + p.stages;
  uint64_t* tfull = empty + p.stages;      // [2]
  uint64_t* tempty = tfull + 2;            // [2]
  uint64_t* afull = tempty + 2;            // RES: the resident A tile has landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(afull + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM;
  const int P0 = blockIdx.y * p.ppc;
  const int nP = max(0, min(p.pn, P0 + p.ppc) - P0);
  const uint32_t idesc = idesc_of<IN>(p.nb);
  const int a_part = RES ? n_parts_a(MODE) * p.a_bytes : 0;   // resident bytes per k-block
  const int b_off = RES ? 0 : n_parts_a(MODE) * p.a_bytes;     // first B tile in a stage
  const uint32_t crank = CL > 1 ? cluster_rank() : 0u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], CL); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], S1_EPI_WARPS); }
    mbar_init(afull, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)), "r"(2 * p.acc_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  if constexpr (CL > 1) cluster_sync_all();   // every barrier of the cluster initialised
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int nsteps = nP * p.nkb;

  if (warp == 0 && lane == 0) {
    if constexpr (RES) {
      if (nsteps > 0) {
        mbar_expect_tx(afull, p.a_res_bytes);
        for (int kb = 0; kb < p.nkb; ++kb) {
          tma_load_3d(ares + kb * a_part, &mA_hi, afull, kb * BK, m0, 0);
          if (a_split(MODE)) tma_load_3d(ares + kb * a_part + p.a_bytes, &mA_lo, afull, kb * BK, m0, 0);
        }
      }
    }
    for (int i = 0; i < nsteps; ++i) {
      const int s = i % p.stages;
      if (!mbar_wait(&empty[s], ((uint32_t)(i / p.stages) & 1u) ^ 1u)) { atomicOr(p.err, 16); break; }
      const int P = P0 + i / p.nkb, k0 = (i % p.nkb) * BK;
      unsigned char* st = ring + s * p.stage_bytes;
      mbar_expect_tx(&full[s], p.stage_bytes);
      if constexpr (!RES) {
        tma_load_3d(st, &mA_hi, &full[s], k0, m0, 0);
        if (a_split(MODE)) tma_load_3d(st + p.a_bytes, &mA_lo, &full[s], k0, m0, 0);
      }
      if constexpr (CL > 1) {
        // this CTA's half of the B_P rows, to both CTAs of the pair
        const int hb = p.b_bytes / 2;
        const int r0 = (int)crank * (p.nb / 2);
        tma_load_3d_mc(st + b_off + crank * hb, &mB_hi, &full[s], k0, r0, P, (uint16_t)0x3);
        if (b_split(MODE))
          tma_load_3d_mc(st + b_off + p.b_bytes + crank * hb, &mB_lo, &full[s], k0, r0, P, (uint16_t)0x3);
      } else {
        tma_load_3d(st + b_off, &mB_hi, &full[s], k0, 0, P);
        if (b_split(MODE)) tma_load_3d(st + b_off + p.b_bytes, &mB_lo, &full[s], k0, 0, P);
      }
    }
    // let the copies already issued land before the CTA can exit
    for (int i = max(0, nsteps - p.stages); i < nsteps; ++i)
      if (!mbar_wait(&full[i % p.stages], (uint32_t)(i / p.stages) & 1u)) { atomicOr(p.err, 32); break; }
    if constexpr (CL > 1) {
      // and the peer's last commits arrive on this CTA's `empty` barriers
      for (int i = nsteps; i < nsteps + p.stages; ++i)
        if (!mbar_wait(&empty[i % p.stages], ((uint32_t)(i / p.stages) & 1u) ^ 1u)) { atomicOr(p.err, 32); break; }
    }
  } else if (warp == 1 && lane == 0) {
    bool ok = true;
    if constexpr (RES) {
      if (nsteps > 0 && !mbar_wait(afull, 0)) { atomicOr(p.err, 128); ok = false; }
    }
    for (int j = 0; j < nP && ok; ++j) {
      const int buf = j & 1;
      // wait until the epilogue has drained this accumulator buffer (use j/2 - 1)
      if (!mbar_wait(&tempty[buf], ((uint32_t)(j >> 1) & 1u) ^ 1u)) { atomicOr(p.err, 64); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + (uint32_t)(buf * p.acc_cols);
      for (int kb = 0; kb < p.nkb; ++kb) {
        const int i = j * p.nkb + kb;
        const int s = i % p.stages;
        if (!mbar_wait(&full[s], (uint32_t)(i / p.stages) & 1u)) { atomicOr(p.err, 128); ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* st = ring + s * p.stage_bytes;
        unsigned char* at = RES ? ares + kb * a_part : st;
        const uint64_t ah = sdesc(at), bh = sdesc(st + b_off);
        const int rem = p.K - kb * BK;
        const int nks = rem >= BK ? BK / 16 : (rem + 15) / 16;   // the zero-filled tail issues no MMA
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          if (kk < nks) {
            const uint64_t off = (uint64_t)(kk * 32) >> 4;
            mma_op<IN>(acc, ah + off, bh + off, (kb > 0 || kk > 0) ? 1u : 0u, idesc);
            if (b_split(MODE)) mma_op<IN>(acc, ah + off, sdesc(st + b_off + p.b_bytes) + off, 1u, idesc);
            if (a_split(MODE)) mma_op<IN>(acc, sdesc(at + p.a_bytes) + off, bh + off, 1u, idesc);
          }
        }
        if constexpr (CL > 1) mma_commit_mc(&empty[s], (uint16_t)0x3);
        else mma_commit(&empty[s]);
      }
      mma_commit(&tfull[buf]);
    }
  } else if (warp >= 2) {
    // epilogue warps: TMEM lane quadrant q = warp & 3; the four warps of a
    // quadrant take the 16-column chunks part, part + 4, part + 8, ...; each
    // warp loads its next chunk from TMEM while it stores the current one
    constexpr int NPART = S1_EPI_WARPS / 4;
    const int q = warp & 3;
    const int part = (warp - 2) >> 2;
    const int r = m0 + q * 32 + lane;
    const int g = r / p.R, ri = r - (r / p.R) * p.R;
    const size_t cs = (size_t)p.pn * p.ldo;   // output stride between consecutive columns
    const float mul = OUT == ET_F16 ? *p.mul : 1.f;
    auto tmem_ld = [&](uint32_t (&v)[16], uint32_t taddr) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
          " [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
    };
    auto tmem_wait = [] { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); };
    auto store = [&](const uint32_t (&v)[16], int c0, int P) {
      if (r >= p.M) return;
      const size_t base = (((size_t)g * p.N + c0) * p.pn + P) * p.ldo + ri;
      const int nc = min(16, p.N - c0);
      if constexpr (OUT == ET_E4M3) {
        const float mu = p.mu[P];
        unsigned char* oh = static_cast<unsigned char*>(p.out_hi) + base;
        unsigned char* ol = static_cast<unsigned char*>(p.out_lo) + base;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          if (t < nc) {
            const float x = __uint_as_float(v[t]) * mu;
            const unsigned char h = to_e4m3(x);
            oh[t * cs] = h;
            ol[t * cs] = to_e4m3(x - from_e4m3(h));
          }
        }
      } else if constexpr (OUT == ET_F16) {
        __half* oh = static_cast<__half*>(p.out_hi) + base;
        __half* ol = static_cast<__half*>(p.out_lo) + base;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          if (t < nc) {
            const float x = __uint_as_float(v[t]) * mul;
            const __half h = __float2half_rn(x);
            oh[t * cs] = h;
            ol[t * cs] = __float2half_rn(x - __half2float(h));
          }
        }
      } else {
        __nv_bfloat16* oh = static_cast<__nv_bfloat16*>(p.out_hi) + base;
        __nv_bfloat16* ol = a_split(MODE) ? static_cast<__nv_bfloat16*>(p.out_lo) + base : nullptr;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          if (t < nc) {
            const float x = __uint_as_float(v[t]);
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            oh[t * cs] = h;
            if (a_split(MODE)) ol[t * cs] = __float2bfloat16_rn(x - __bfloat162float(h));
          }
        }
      }
    };
    for (int j = 0; j < nP; ++j) {
      const int buf = j & 1;
      bool ok = mbar_wait(&tfull[buf], (uint32_t)(j >> 1) & 1u);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) { if (lane == 0) atomicOr(p.err, 256); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int P = P0 + j;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * p.acc_cols);
      constexpr int STEP = 16 * NPART;
      uint32_t va[16], vb[16];
      int c0 = 16 * part;
      if (c0 < p.N) tmem_ld(va, tbase + (uint32_t)c0);
      tmem_wait();
#pragma unroll 1
      for (; c0 < p.N; c0 += 2 * STEP) {
        const int c1 = c0 + STEP;
        if (c1 < p.N) tmem_ld(vb, tbase + (uint32_t)c1);
        store(va, c0, P);
        tmem_wait();
        if (c1 >= p.N) break;
        if (c1 + STEP < p.N) tmem_ld(va, tbase + (uint32_t)(c1 + STEP));
        store(vb, c1, P);
        tmem_wait();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[buf])) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * p.acc_cols));
  }
  if constexpr (CL > 1) cluster_sync_all();   // neither CTA leaves while the other may still signal it
}

// Sum the split partials into out (FP32), accumulating when asked.
// With `scale` (device scalar), the summed partials are multiplied by *scale
// before they are added (the FP8 operands carry a scale factor).
__global__ void k_sum_splits(const float* __restrict__ part, int S, long long MN, float* out,
                             int accumulate, const float* __restrict__ scale) {
  if (!scale) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < MN;
         t += (long long)gridDim.x * blockDim.x) {
      float acc = accumulate ? out[t] : 0.f;
      for (int s = 0; s < S; ++s) acc += part[s * MN + t];
      out[t] = acc;
    }
    return;
  }
  const float f = *scale;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < MN;
       t += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < S; ++s) acc += part[s * MN + t];
    out[t] = (accumulate ? out[t] : 0.f) + f * acc;
  }
}

// Split of x (converted to FP32, times *scale when given) into two 16-bit
// parts hi = round(x), lo = round(x - hi) of the element type E (BF16 or
// FP16); lo optional.
template <typename E> __device__ __forceinline__ E to_elem(float x);
template <> __device__ __forceinline__ __nv_bfloat16 to_elem<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __half to_elem<__half>(float x) { return __float2half_rn(x); }
__device__ __forceinline__ float from_elem(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float from_elem(__half x) { return __half2float(x); }

template <typename E>
__device__ __forceinline__ void split_store(float v, long long t, E* hi, E* lo) {
  const E h = to_elem<E>(v);
  hi[t] = h;
  if (lo) lo[t] = to_elem<E>(v - from_elem(h));
}

// Transpose + split of factor rows: src [rows][n1][n2] -> dst [rows][n2][pad8(n1)]
// (dst[r][b][a] = src[r][a][b]; pads zero).  lo may be NULL (one part).
template <typename TS, typename E>
__global__ void k_transpose_split(const TS* __restrict__ src, int rows, int n1, int n2, int ld,
                                  const float* __restrict__ scale, E* hi, E* lo) {
  const long long tot = (long long)rows * n2 * ld;
  const float sc = scale ? *scale : 1.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t % ld);
    const long long rb = t / ld;
    const int b = (int)(rb % n2);
    const long long r = rb / n2;
    float v = 0.f;
    if (a < n1) v = (float)src[(r * n1 + a) * n2 + b] * sc;
    split_store<E>(v, t, hi, lo);
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

// 3-D tiled map with 128-byte swizzle over elements of type et (ET_BF16,
// ET_F16 or ET_E4M3, the last as bytes).
CUtensorMap make_map(const void* base, const cuuint64_t dims[3], const cuuint64_t strides[2],
                     const cuuint32_t box[3], int et = ET_BF16, int swizzle_bytes = 128) {
  TD_REQUIRE((reinterpret_cast<uintptr_t>(base) & 15) == 0, TDDFT_ERR_ARG, "TMA base not 16-byte aligned");
  TD_REQUIRE(strides[0] % 16 == 0 && strides[1] % 16 == 0, TDDFT_ERR_ARG, "TMA strides not 16-byte multiples");
  CUtensorMap m;
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = et == ET_E4M3 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                 : (et == ET_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  CUresult r = encode_fn()(&m, dt, 3,
                           const_cast<void*>(base), dims, strides,
                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  TD_REQUIRE(r == CUDA_SUCCESS, TDDFT_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

}  // namespace

int tc_pad(int nv) { return (nv + 7) & ~7; }
int tc_pad16(int n) { return (n + 15) & ~15; }

namespace {
template <typename E>
void transpose_split_t(const void* src, DType ts, int rows, int n1, int n2, const float* scale, E* hi, E* lo,
                       cudaStream_t s) {
  const int ld = tc_pad(n1);
  const long long tot = (long long)rows * n2 * ld;
  long long g = (tot + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (ts == DType::F32)
    k_transpose_split<float, E><<<(unsigned)g, 256, 0, s>>>((const float*)src, rows, n1, n2, ld, scale, hi, lo);
  else if (ts == DType::BF16)
    k_transpose_split<__nv_bfloat16, E><<<(unsigned)g, 256, 0, s>>>((const __nv_bfloat16*)src, rows, n1, n2, ld,
                                                                    scale, hi, lo);
  else
    k_transpose_split<double, E><<<(unsigned)g, 256, 0, s>>>((const double*)src, rows, n1, n2, ld, scale, hi, lo);
}
}  // namespace

void tc_transpose_split(const void* src, DType ts, int rows, int n1, int n2, void* hi, void* lo, TcElt et,
                        const float* scale, cudaStream_t s) {
  TD_REQUIRE(et == TcElt::F16 || scale == nullptr, TDDFT_ERR_ARG, "tc_transpose_split: BF16 parts take no scale");
  if (et == TcElt::F16)
    transpose_split_t<__half>(src, ts, rows, n1, n2, scale, (__half*)hi, (__half*)lo, s);
  else
    transpose_split_t<__nv_bfloat16>(src, ts, rows, n1, n2, scale, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, s);
  count_launch();
  TD_LAUNCH_CHECK();
}

// SMs of the current device (queried once).
int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      n = 152;
  }
  return n;
}

// Work split for a grid of `tiles` x splits CTAs, one CTA per SM, each taking
// ceil(total / splits) consecutive units: the launch lasts (number of waves) x
// (units per CTA + a fixed per-CTA cost of `overhead` units), so a last,
// nearly empty wave costs as much as a full one.  Tries the splits that fill
// one to four waves and keeps the cheapest (the fewest splits on ties).
int wave_splits(int tiles, int total, int overhead, int sms = 0) {
  if (sms <= 0) sms = sm_count();
  int best = 1;
  long long best_cost = -1;
  for (int w = 1; w <= 4; ++w) {
    int sp = std::max(1, (w * sms) / std::max(tiles, 1));
    sp = std::min(sp, std::max(total, 1));
    const int per = (total + sp - 1) / sp;
    sp = (total + per - 1) / per;
    const long long waves = ((long long)tiles * sp + sms - 1) / sms;
    const long long cost = waves * (per + overhead);
    if (best_cost < 0 || cost < best_cost || (cost == best_cost && sp < best)) {
      best_cost = cost;
      best = sp;
    }
  }
  return best;
}

namespace {
bool cluster_pairs_enabled() {
  const char* e = std::getenv("TDDFT_TC_CLUSTER");
  return !(e && e[0] == '0');
}

bool cluster_quads_enabled() {
  const char* e = std::getenv("TDDFT_TC_QUAD");
  return !(e && e[0] == '0');
}

// CTAs of the paired contraction that can be resident at once: two per
// co-resident cluster (an SM left over in a GPC takes no pair).
int pair_slots(int et) {
  static int cached[2] = {0, 0};
  int& c = cached[et == ET_F16 ? 1 : 0];
  if (c == 0) {
    const void* k = et == ET_F16 ? (const void*)k1_tc_kernel<BOTH, ET_F16, 2, 64>
                                 : (const void*)k1_tc_kernel<BOTH, ET_BF16, 2, 64>;
    const int smem = Cfg<BOTH, 64>::SMEM_BYTES;
    ensure_smem(k, smem);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = 2;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(1, 2, 1);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess || n <= 0) {
      (void)cudaGetLastError();
      n = sm_count() / 2;
    }
    c = 2 * n;
  }
  return c;
}
}  // namespace

void tc_contract(const void* Ahi, const void* Alo, int M, int pn, int Kin, const void* Bhi, const void* Blo,
                 int N, float* out, bool accumulate, TcElt elt, const float* scale, int* err, cudaStream_t s,
                 KernelProfile* prof, double prof_flops, double prof_bytes, int max_kb) {
  if (M <= 0 || pn <= 0 || N <= 0) return;
  TD_REQUIRE(Alo != nullptr || Blo == nullptr, TDDFT_ERR_ARG, "tc_contract: B split without A split");
  const int et = elem_of(elt);
  const int mode = Alo ? (Blo ? BOTH : ASPLIT) : SINGLE;
  // the split-B products run on 64-byte K rows (a four-deep ring), the others on 128-byte rows
  const int rb = mode == BOTH ? 64 : 128;
  const int bke = BK * rb / 128;
  const int ldk = tc_pad(Kin);
  const int nab = (Kin + bke - 1) / bke;
  const int total = pn * nab;
  if (max_kb > 0) max_kb = max_kb * (BK / bke);   // max_kb counts 64-element k-blocks
  const int mt0 = (M + BM - 1) / BM, nt0 = (N + BN - 1) / BN;
  // split-B products in pairs of M tiles that share each B tile through a
  // cluster multicast (TDDFT_TC_CLUSTER=0 turns this off; the results are the
  // same bits either way: every CTA issues the same MMAs on the same data)
  const bool pair = mode == BOTH && mt0 > 1 && cluster_pairs_enabled();
  const int mt = pair ? (mt0 + 1) & ~1 : mt0;
  // and, with two or more N tiles, in 2 x 2 clusters whose N pairs also share each A tile
  const int cx = pair && nt0 > 1 && cluster_quads_enabled() ? 2 : 1;
  const int nt = cx > 1 ? (nt0 + 1) & ~1 : nt0;
  // a CTA's fixed cost (barriers, TMEM, pipeline fill, 128 KB epilogue) is about
  // four 64-element k-blocks of MMA work.  The split count depends on the
  // problem only (its own tiles, the pairs' residency), not on the cluster
  // shape of the launch: every shape then forms the same sums, bit for bit.
  const bool pairable = mode == BOTH && mt0 > 1;
  int splits = wave_splits(mt0 * nt0, total, 4 * (BK / bke), pairable ? pair_slots(et) : 0);
  if (max_kb > 0) splits = std::max(splits, (total + max_kb - 1) / max_kb);   // bounded accumulation runs
  const int per = (total + splits - 1) / splits;
  splits = (total + per - 1) / per;

  const cuuint64_t dA[3] = {(cuuint64_t)Kin, (cuuint64_t)pn, (cuuint64_t)M};
  const cuuint64_t sA[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)pn * ldk * 2};
  const cuuint32_t bA[3] = {(cuuint32_t)bke, 1, (cuuint32_t)(BM / cx)};   // a quad's N pair loads half an A tile each
  const cuuint64_t dB[3] = {(cuuint64_t)Kin, (cuuint64_t)N, (cuuint64_t)pn};
  const cuuint64_t sB[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)N * ldk * 2};
  const cuuint32_t bB[3] = {(cuuint32_t)bke, (cuuint32_t)(pair ? BN / 2 : BN), 1};   // a pair loads half a B tile each
  CUtensorMap mAh = make_map(Ahi, dA, sA, bA, et, rb), mBh = make_map(Bhi, dB, sB, bB, et, rb);
  CUtensorMap mAl = Alo ? make_map(Alo, dA, sA, bA, et, rb) : mAh;
  CUtensorMap mBl = Blo ? make_map(Blo, dB, sB, bB, et, rb) : mBh;

  DevBuf part((size_t)splits * M * N * 4, s);
  Params p{M, N, Kin, nab, total, per, part.as<float>(), err};
  dim3 grid(nt, mt, splits);
  auto launch = [&](auto kernel, int smem) {
    ensure_smem((const void*)kernel, smem);
    if (prof) prof->begin(s);
    kernel<<<grid, THREADS, smem, s>>>(mAh, mAl, mBh, mBl, p);
    if (prof) prof->end(s, prof_flops, prof_bytes);
  };
  auto launch_pair = [&](auto kernel, int smem) {
    ensure_smem((const void*)kernel, smem);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cx;
    at[0].val.clusterDim.y = 2;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = grid;
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (prof) prof->begin(s);
    TD_CUDA(cudaLaunchKernelEx(&cfg, kernel, mAh, mAl, mBh, mBl, p));
    if (prof) prof->end(s, prof_flops, prof_bytes);
  };
  if (et == ET_F16) {
    if (pair && cx > 1) launch_pair(k1_tc_kernel<BOTH, ET_F16, 2, 64, 2>, Cfg<BOTH, 64>::SMEM_BYTES);
    else if (pair) launch_pair(k1_tc_kernel<BOTH, ET_F16, 2, 64>, Cfg<BOTH, 64>::SMEM_BYTES);
    else if (mode == BOTH) launch(k1_tc_kernel<BOTH, ET_F16, 1, 64>, Cfg<BOTH, 64>::SMEM_BYTES);
    else if (mode == ASPLIT) launch(k1_tc_kernel<ASPLIT, ET_F16>, Cfg<ASPLIT>::SMEM_BYTES);
    else launch(k1_tc_kernel<SINGLE, ET_F16>, Cfg<SINGLE>::SMEM_BYTES);
  } else {
    if (pair && cx > 1) launch_pair(k1_tc_kernel<BOTH, ET_BF16, 2, 64, 2>, Cfg<BOTH, 64>::SMEM_BYTES);
    else if (pair) launch_pair(k1_tc_kernel<BOTH, ET_BF16, 2, 64>, Cfg<BOTH, 64>::SMEM_BYTES);
    else if (mode == BOTH) launch(k1_tc_kernel<BOTH, ET_BF16, 1, 64>, Cfg<BOTH, 64>::SMEM_BYTES);
    else if (mode == ASPLIT) launch(k1_tc_kernel<ASPLIT, ET_BF16>, Cfg<ASPLIT>::SMEM_BYTES);
    else launch(k1_tc_kernel<SINGLE, ET_BF16>, Cfg<SINGLE>::SMEM_BYTES);
  }
  count_launch();
  TD_LAUNCH_CHECK();
  const long long MN = (long long)M * N;
  long long g = (MN + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_sum_splits<<<(unsigned)g, 256, 0, s>>>(part.as<float>(), splits, MN, out, accumulate ? 1 : 0, scale);
  count_launch();
  TD_LAUNCH_CHECK();
}

void tc_contract8(const unsigned char* Ahi, const unsigned char* Alo, int M, int pn, int Kin,
                  const unsigned char* B, int N, float* out, bool accumulate, const float* scale, int* err,
                  cudaStream_t s) {
  if (M <= 0 || pn <= 0 || N <= 0) return;
  TD_REQUIRE(Ahi && Alo && B && scale, TDDFT_ERR_ARG, "tc_contract8: operands missing");
  constexpr int BKE = Elem<ET_E4M3>::BKE;
  const int ldk = tc_pad16(Kin);
  const int nab = (Kin + BKE - 1) / BKE;
  const int total = pn * nab;
  const int mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
  int splits = wave_splits(mt * nt, total, 4);
  const int per = (total + splits - 1) / splits;
  splits = (total + per - 1) / per;
  const cuuint64_t dA[3] = {(cuuint64_t)Kin, (cuuint64_t)pn, (cuuint64_t)M};
  const cuuint64_t sA[2] = {(cuuint64_t)ldk, (cuuint64_t)pn * ldk};
  const cuuint32_t bA[3] = {(cuuint32_t)BKE, 1, BM};
  const cuuint64_t dB[3] = {(cuuint64_t)Kin, (cuuint64_t)N, (cuuint64_t)pn};
  const cuuint64_t sB[2] = {(cuuint64_t)ldk, (cuuint64_t)N * ldk};
  const cuuint32_t bB[3] = {(cuuint32_t)BKE, BN, 1};
  CUtensorMap mAh = make_map(Ahi, dA, sA, bA, ET_E4M3), mAl = make_map(Alo, dA, sA, bA, ET_E4M3);
  CUtensorMap mB = make_map(B, dB, sB, bB, ET_E4M3);
  DevBuf part((size_t)splits * M * N * 4, s);
  Params p{M, N, Kin, nab, total, per, part.as<float>(), err};
  dim3 grid(nt, mt, splits);
  ensure_smem((const void*)k1_tc_kernel<ASPLIT, ET_E4M3>, Cfg<ASPLIT>::SMEM_BYTES);
  k1_tc_kernel<ASPLIT, ET_E4M3><<<grid, THREADS, Cfg<ASPLIT>::SMEM_BYTES, s>>>(mAh, mAl, mB, mB, p);
  count_launch();
  TD_LAUNCH_CHECK();
  const long long MN = (long long)M * N;
  long long g = (MN + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_sum_splits<<<(unsigned)g, 256, 0, s>>>(part.as<float>(), splits, MN, out, accumulate ? 1 : 0, scale);
  count_launch();
  TD_LAUNCH_CHECK();
}

namespace {
// CTAs of a paired stage-1 launch that can be resident at once (two per
// co-resident cluster).
int s1_pair_slots(bool res, int smem) {
  static int cached[2] = {0, 0}, cached_smem[2] = {0, 0};
  int& c = cached[res ? 1 : 0];
  if (c == 0 || cached_smem[res ? 1 : 0] != smem) {
    cached_smem[res ? 1 : 0] = smem;
    const void* k = res ? (const void*)k_stage1_tc<BOTH, ET_F16, ET_F16, true, 2>
                        : (const void*)k_stage1_tc<BOTH, ET_F16, ET_F16, false, 2>;
    ensure_smem(k, smem);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(S1_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess || n <= 0) {
      (void)cudaGetLastError();
      n = sm_count() / 2;
    }
    c = 2 * n;
  }
  return c;
}

// out_is8: e4m3 outputs with per-P multipliers mu (A as hi + lo, B plain);
// otherwise 16-bit outputs of the inputs' element type et, FP16 ones times *mul.
void stage1_impl(const void* Ahi, const void* Alo, int M, int K, const void* Bhi, const void* Blo, int N, int pn,
                 int R, int et, bool out_is8, void* out_hi, void* out_lo, const float* mul, const float* mu, int* err,
                 cudaStream_t s) {
  if (M <= 0 || pn <= 0 || N <= 0) return;
  TD_REQUIRE(N <= 256, TDDFT_ERR_ARG, "tc_stage1: N above 256");
  TD_REQUIRE((Alo != nullptr || Blo == nullptr) &&
                 (out_is8 ? (out_lo != nullptr && mu != nullptr) : (Alo != nullptr) == (out_lo != nullptr)),
             TDDFT_ERR_ARG, "tc_stage1: hi/lo operands mismatch");
  TD_REQUIRE((et == ET_F16) == (mul != nullptr) && (!out_is8 || et == ET_BF16), TDDFT_ERR_ARG,
             "tc_stage1: FP16 outputs need a multiplier, FP8 outputs BF16 inputs");
  const int mode = Alo ? (Blo ? BOTH : ASPLIT) : SINGLE;
  const int ldk = tc_pad(K);
  const int nb = (N + 15) & ~15;
  int acc_cols = 32;
  while (acc_cols < nb) acc_cols *= 2;
  const int a_bytes = BM * BK * 2, b_bytes = nb * BK * 2;
  const int nkb = (K + BK - 1) / BK;
  const int mt0 = (M + BM - 1) / BM;
  // The FP16 exact operands (hi + lo on both sides): the A tile stays resident
  // when all its k-blocks fit beside a ring of three B stages, and pairs of M
  // tiles share each B_P tile through a cluster multicast.
  constexpr int kSmemBudget = 224 * 1024;
  const int a_res = nkb * n_parts_a(mode) * a_bytes;
  const int b_stage = n_parts_b(mode) * b_bytes;
  const bool res = et == ET_F16 && !out_is8 && a_res + 3 * b_stage + 2048 <= kSmemBudget;
  const bool pair = et == ET_F16 && !out_is8 && mt0 > 1 && cluster_pairs_enabled();
  const int mt = pair ? (mt0 + 1) & ~1 : mt0;
  const int stage_bytes = res ? b_stage : n_parts_a(mode) * a_bytes + b_stage;
  int stages = ((res ? kSmemBudget - a_res - 2048 : 200 * 1024)) / stage_bytes;
  if (stages > 6) stages = 6;
  TD_REQUIRE(stages >= 2, TDDFT_ERR_ARG, "tc_stage1: tile too large");
  const int smem = (res ? a_res : 0) + stages * stage_bytes + 1024 + 256;
  int groups = wave_splits(mt, pn, 1, pair ? s1_pair_slots(res, smem) : 0);   // units: P-rows
  const int ppc = (pn + groups - 1) / groups;
  groups = (pn + ppc - 1) / ppc;

  const cuuint64_t dA[3] = {(cuuint64_t)K, (cuuint64_t)M, 1};
  const cuuint64_t sA[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)M * ldk * 2};
  const cuuint32_t bA[3] = {BK, BM, 1};
  const cuuint64_t dB[3] = {(cuuint64_t)K, (cuuint64_t)N, (cuuint64_t)pn};
  const cuuint64_t sB[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)N * ldk * 2};
  const cuuint32_t bB[3] = {BK, (cuuint32_t)(pair ? nb / 2 : nb), 1};   // a pair loads half a B tile each
  CUtensorMap mAh = make_map(Ahi, dA, sA, bA, et), mBh = make_map(Bhi, dB, sB, bB, et);
  CUtensorMap mAl = Alo ? make_map(Alo, dA, sA, bA, et) : mAh;
  CUtensorMap mBl = Blo ? make_map(Blo, dB, sB, bB, et) : mBh;
  S1Params p{M, N, R, out_is8 ? tc_pad16(R) : tc_pad(R), pn, ppc, nkb, K, nb, acc_cols, stages,
             stage_bytes, a_bytes, b_bytes, res ? a_res : 0, out_hi, out_lo, mul, mu, err};
  dim3 grid(mt, groups, 1);
  auto launch = [&](auto kernel) {
    ensure_smem((const void*)kernel, smem);
    kernel<<<grid, S1_THREADS, smem, s>>>(mAh, mAl, mBh, mBl, p);
  };
  auto launch_pair = [&](auto kernel) {
    ensure_smem((const void*)kernel, smem);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = grid;
    cfg.blockDim = dim3(S1_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    TD_CUDA(cudaLaunchKernelEx(&cfg, kernel, mAh, mAl, mBh, mBl, p));
  };
  if (out_is8) {
    TD_REQUIRE(mode == ASPLIT, TDDFT_ERR_ARG, "tc_stage1: FP8 output needs hi+lo A and a plain B");
    launch(k_stage1_tc<ASPLIT, ET_BF16, ET_E4M3>);
  } else if (et == ET_F16) {
    TD_REQUIRE(mode == BOTH, TDDFT_ERR_ARG, "tc_stage1: FP16 operands come as hi + lo");
    if (res && pair) launch_pair(k_stage1_tc<BOTH, ET_F16, ET_F16, true, 2>);
    else if (res) launch(k_stage1_tc<BOTH, ET_F16, ET_F16, true, 1>);
    else if (pair) launch_pair(k_stage1_tc<BOTH, ET_F16, ET_F16, false, 2>);
    else launch(k_stage1_tc<BOTH, ET_F16, ET_F16>);
  } else if (mode == BOTH) launch(k_stage1_tc<BOTH, ET_BF16, ET_BF16>);
  else if (mode == ASPLIT) launch(k_stage1_tc<ASPLIT, ET_BF16, ET_BF16>);
  else launch(k_stage1_tc<SINGLE, ET_BF16, ET_BF16>);
  count_launch();
  TD_LAUNCH_CHECK();
}
}  // namespace

void tc_stage1(const void* Ahi, const void* Alo, int M, int K, const void* Bhi, const void* Blo, int N, int pn,
               int R, TcElt et, const float* mul, void* out_hi, void* out_lo, int* err, cudaStream_t s) {
  stage1_impl(Ahi, Alo, M, K, Bhi, Blo, N, pn, R, elem_of(et), false, out_hi, out_lo, mul, nullptr, err, s);
}

void tc_stage1_fp8(const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo, int M, int K, const __nv_bfloat16* B,
                   int N, int pn, int R, const float* mu, unsigned char* out_hi, unsigned char* out_lo, int* err,
                   cudaStream_t s) {
  stage1_impl(Ahi, Alo, M, K, B, nullptr, N, pn, R, ET_BF16, true, out_hi, out_lo, nullptr, mu, err, s);
}

// F64/F32/BF16 rows [rows][n] -> hi (+ lo) [rows][tc_pad(n)] (times *scale when given)
template <typename TS, typename E>
__global__ void k_pad_split(const TS* __restrict__ src, long long rows, int n, int ld,
                            const float* __restrict__ scale, E* hi, E* lo) {
  const long long tot = rows * ld;
  const float sc = scale ? *scale : 1.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t % ld);
    const long long r = t / ld;
    const float v = a < n ? (float)src[r * n + a] * sc : 0.f;
    split_store<E>(v, t, hi, lo);
  }
}

template <typename E>
void pad_split_t(const void* src, DType ts, long long rows, int n, int ld, const float* scale, E* hi, E* lo,
                 cudaStream_t s) {
  const long long tot = rows * ld;
  long long g = (tot + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (ts == DType::F64)
    k_pad_split<double, E><<<(unsigned)g, 256, 0, s>>>((const double*)src, rows, n, ld, scale, hi, lo);
  else if (ts == DType::F32)
    k_pad_split<float, E><<<(unsigned)g, 256, 0, s>>>((const float*)src, rows, n, ld, scale, hi, lo);
  else
    k_pad_split<__nv_bfloat16, E><<<(unsigned)g, 256, 0, s>>>((const __nv_bfloat16*)src, rows, n, ld, scale, hi, lo);
}

void tc_pad_split(const void* src, DType ts, long long rows, int n, void* hi, void* lo, TcElt et,
                  const float* scale, cudaStream_t s) {
  TD_REQUIRE(et == TcElt::F16 || scale == nullptr, TDDFT_ERR_ARG, "tc_pad_split: BF16 parts take no scale");
  if (et == TcElt::F16)
    pad_split_t<__half>(src, ts, rows, n, tc_pad(n), scale, (__half*)hi, (__half*)lo, s);
  else
    pad_split_t<__nv_bfloat16>(src, ts, rows, n, tc_pad(n), scale, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, s);
  count_launch();
  TD_LAUNCH_CHECK();
}


// ---------------------------------------------------------------------------
// FP8 (e4m3) operands of the ris exchange contractions, with a scale per
// auxiliary row P.  The ris factors L^P are stored as q^P = e4m3(L^P / s_P),
// s_P = max |L^P| / 448 (448 = the largest finite e4m3).  A product
// sum_P C_P L^P = sum_P (s_P C_P) q^P: the stage-1 result C_P is multiplied by
// mu_P = s_P * g before its own hi + lo e4m3 split, and the contraction's sum
// by 1/g, with g chosen from a bound so that |mu_P C_P| <= 224:
//   |C_P[(n,i)][k]| <= rho_P * kappa   (Cauchy-Schwarz), rho_P = max_i ||L^P_i,:||,
//   kappa = the largest norm of the trial-vector slices that C contracts with.
namespace {

__global__ void k_quant_e4m3_t(const __nv_bfloat16* __restrict__ src, int n1, int n2, int ld,
                               unsigned char* __restrict__ dst, float* __restrict__ scale) {
  const long long per = (long long)n1 * n2;
  const __nv_bfloat16* x = src + blockIdx.x * per;
  unsigned char* y = dst + (long long)blockIdx.x * n2 * ld;
  __shared__ float red[32];
  float m = 0.f;
  for (long long t = threadIdx.x; t < per; t += blockDim.x) m = fmaxf(m, fabsf(__bfloat162float(x[t])));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  const float sc = red[0] > 0.f ? red[0] / 448.f : 1.f;
  const float inv = 1.f / sc;
  if (threadIdx.x == 0) scale[blockIdx.x] = sc;
  const long long tot = (long long)n2 * ld;
  for (long long t = threadIdx.x; t < tot; t += blockDim.x) {   // y[b][a] = x[a][b] / s
    const int a = (int)(t % ld);
    const long long b = t / ld;
    y[t] = a < n1 ? to_e4m3(__bfloat162float(x[(long long)a * n2 + b]) * inv) : (unsigned char)0;
  }
}

__global__ void k_row_norm_max(const __nv_bfloat16* __restrict__ src, int nr, int nc, float* __restrict__ rho) {
  const __nv_bfloat16* x = src + (long long)blockIdx.x * nr * nc;
  __shared__ float red[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float m = 0.f;
  for (int i = warp; i < nr; i += nw) {
    float acc = 0.f;
    for (int c = lane; c < nc; c += 32) {
      const float v = __bfloat162float(x[(long long)i * nc + c]);
      acc += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    m = fmaxf(m, sqrtf(acc));
  }
  if (lane == 0) red[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int w = 0; w < nw; ++w) r = fmaxf(r, red[w]);
    rho[blockIdx.x] = r;
  }
}

// kappa[0] = max_(n,a) ||X[n][:][a]||, kappa[1] = max_(n,j) ||X[n][j][:]||,
// kappa[2] = max |X| (as float bits; non-negative floats order like their bit
// patterns)
template <typename T>
__global__ void k_x_norms(const T* __restrict__ X, int no, int nv, unsigned* __restrict__ kappa) {
  const T* x = X + (long long)blockIdx.x * no * nv;
  __shared__ float red[3][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float mc = 0.f, mr = 0.f, ma = 0.f;
  for (int a = threadIdx.x; a < nv; a += blockDim.x) {
    float acc = 0.f;
    for (int j = 0; j < no; ++j) {
      const float v = (float)x[(long long)j * nv + a];
      acc += v * v;
      ma = fmaxf(ma, fabsf(v));
    }
    mc = fmaxf(mc, sqrtf(acc));
  }
  for (int j = warp; j < no; j += nw) {
    float acc = 0.f;
    for (int b = lane; b < nv; b += 32) { const float v = (float)x[(long long)j * nv + b]; acc += v * v; }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    mr = fmaxf(mr, sqrtf(acc));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mc = fmaxf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
  }
  if (lane == 0) { red[0][warp] = mc; red[1][warp] = mr; red[2][warp] = ma; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float c = 0.f, r = 0.f, m = 0.f;
    for (int w = 0; w < nw; ++w) { c = fmaxf(c, red[0][w]); r = fmaxf(r, red[1][w]); m = fmaxf(m, red[2][w]); }
    atomicMax(&kappa[0], __float_as_uint(c));
    atomicMax(&kappa[1], __float_as_uint(r));
    atomicMax(&kappa[2], __float_as_uint(m));
  }
}

// 2^(top - e) for b = f 2^e, f in [0.5, 1): the largest power of two s with
// s b < 2^top (1 for b = 0).
__device__ __forceinline__ float pow2_scale(float b, int top) {
  if (!(b > 0.f)) return 1.f;
  int e = 0;
  frexpf(b, &e);
  e = max(-100, min(100, e));
  return ldexpf(1.f, top - e);
}

// st[0] = max |x| and st[1] = the largest row norm of FP32 rows [rows][n]
// (float bits); one warp per row
__global__ void k_f16_tensor_stats(const float* __restrict__ src, long long rows, int n, unsigned* __restrict__ st) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  float ma = 0.f, mr = 0.f;
  for (long long r = w0; r < rows; r += nw) {
    float acc = 0.f;
    for (int c = lane; c < n; c += 32) {
      const float v = src[r * n + c];
      acc += v * v;
      ma = fmaxf(ma, fabsf(v));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    mr = fmaxf(mr, sqrtf(acc));
  }
  for (int o = 16; o > 0; o >>= 1) ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
  if (lane == 0) {
    atomicMax(&st[0], __float_as_uint(ma));
    atomicMax(&st[1], __float_as_uint(mr));
  }
}

// sc[0] = sigma (max |sigma x| < 2^14), sc[1] = sigma * largest row norm
__global__ void k_f16_sigma(const unsigned* __restrict__ st, float* __restrict__ sc) {
  const float sg = pow2_scale(__uint_as_float(st[0]), 14);
  sc[0] = sg;
  sc[1] = sg * __uint_as_float(st[1]);
}

// Per-product scales of the FP16 exact contractions (layout in tc_gemm.cuh).
__global__ void k_f16_product_scales(const unsigned* __restrict__ kappa, const float* __restrict__ fsc,
                                     float* __restrict__ out) {
  const float kc = __uint_as_float(kappa[0]), kr = __uint_as_float(kappa[1]);
  const float sx = pow2_scale(__uint_as_float(kappa[2]), 14);
  // |Z'| <= rho_oo' ||X'[n][:][a]||, |Q'| <= ||X'[n][i][:]|| rho_ov' (Cauchy-Schwarz)
  const float mz = pow2_scale(fsc[1] * sx * kc, 15);
  const float mq = pow2_scale(fsc[5] * sx * kr, 15);
  out[0] = sx;
  out[1] = mz;
  out[2] = mq;
  out[3] = 1.f / (mz * fsc[0] * sx * fsc[2]);
  out[4] = 1.f / (mq * sx * fsc[4] * fsc[4]);
}

// out[0] = 1/g1, out[1] = 1/g2, out[2 + P] = s1_P g1, out[2 + nK + P] = s2_P g2
__global__ void k_fp8_mu(const unsigned* __restrict__ kappa, const float* __restrict__ s1,
                         const float* __restrict__ r1, const float* __restrict__ s2,
                         const float* __restrict__ r2, int nK, float* __restrict__ out) {
  __shared__ float red[2][32];
  const float kc = __uint_as_float(kappa[0]), kr = __uint_as_float(kappa[1]);
  float b1 = 0.f, b2 = 0.f;
  for (int P = threadIdx.x; P < nK; P += blockDim.x) {
    b1 = fmaxf(b1, s1[P] * r1[P] * kc);
    b2 = fmaxf(b2, s2[P] * r2[P] * kr);
  }
  for (int o = 16; o > 0; o >>= 1) {
    b1 = fmaxf(b1, __shfl_xor_sync(0xffffffffu, b1, o));
    b2 = fmaxf(b2, __shfl_xor_sync(0xffffffffu, b2, o));
  }
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][warp] = b1; red[1][warp] = b2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float x1 = 0.f, x2 = 0.f;
    for (int w = 0; w < nw; ++w) { x1 = fmaxf(x1, red[0][w]); x2 = fmaxf(x2, red[1][w]); }
    red[0][0] = x1 > 0.f ? 224.f / x1 : 1.f;
    red[1][0] = x2 > 0.f ? 224.f / x2 : 1.f;
    out[0] = 1.f / red[0][0];
    out[1] = 1.f / red[1][0];
  }
  __syncthreads();
  const float g1 = red[0][0], g2 = red[1][0];
  for (int P = threadIdx.x; P < nK; P += blockDim.x) {
    out[2 + P] = s1[P] * g1;
    out[2 + nK + P] = s2[P] * g2;
  }
}

}  // namespace

void tc_quant_e4m3(const __nv_bfloat16* src, int rows, int n1, int n2, unsigned char* dst, float* scale,
                   cudaStream_t s) {
  if (rows <= 0) return;
  k_quant_e4m3_t<<<rows, 512, 0, s>>>(src, n1, n2, tc_pad16(n1), dst, scale);
  count_launch();
  TD_LAUNCH_CHECK();
}

void tc_row_norm_max(const __nv_bfloat16* src, int rows, int nr, int nc, float* rho, cudaStream_t s) {
  if (rows <= 0) return;
  k_row_norm_max<<<rows, 256, 0, s>>>(src, nr, nc, rho);
  count_launch();
  TD_LAUNCH_CHECK();
}

void tc_fp8_scales(const void* X, DType xt, int m, int no, int nv, const float* s_vv, const float* rho_oo,
                   const float* s_vo, const float* rho_ov, int nK, float* out, unsigned* kappa,
                   cudaStream_t s) {
  TD_CUDA(cudaMemsetAsync(kappa, 0, 3 * sizeof(unsigned), s));
  if (xt == DType::F32) k_x_norms<float><<<m, 256, 0, s>>>(static_cast<const float*>(X), no, nv, kappa);
  else k_x_norms<double><<<m, 256, 0, s>>>(static_cast<const double*>(X), no, nv, kappa);
  count_launch();
  TD_LAUNCH_CHECK();
  k_fp8_mu<<<1, 256, 0, s>>>(kappa, s_vv, rho_oo, s_vo, rho_ov, nK, out);
  count_launch();
  TD_LAUNCH_CHECK();
}

void tc_f16_tensor_scale(const float* src, long long rows, int n, float* sc, unsigned* scratch, cudaStream_t s) {
  TD_CUDA(cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned), s));
  if (rows > 0 && n > 0) {
    long long g = (rows * 32 + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    k_f16_tensor_stats<<<(unsigned)g, 256, 0, s>>>(src, rows, n, scratch);
    count_launch();
    TD_LAUNCH_CHECK();
  }
  k_f16_sigma<<<1, 1, 0, s>>>(scratch, sc);
  count_launch();
  TD_LAUNCH_CHECK();
}

namespace {
__global__ void k_inv_prod(const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out) {
  out[0] = 1.f / (a[0] * b[0]);
}
}  // namespace

void tc_inv_prod(const float* a, const float* b, float* out, cudaStream_t s) {
  k_inv_prod<<<1, 1, 0, s>>>(a, b, out);
  count_launch();
  TD_LAUNCH_CHECK();
}

void tc_f16_product_scales(const void* X, DType xt, int m, int no, int nv, const float* fsc, float* out,
                           unsigned* kappa, cudaStream_t s) {
  TD_CUDA(cudaMemsetAsync(kappa, 0, 3 * sizeof(unsigned), s));
  if (xt == DType::F32) k_x_norms<float><<<m, 256, 0, s>>>(static_cast<const float*>(X), no, nv, kappa);
  else k_x_norms<double><<<m, 256, 0, s>>>(static_cast<const double*>(X), no, nv, kappa);
  count_launch();
  TD_LAUNCH_CHECK();
  k_f16_product_scales<<<1, 1, 0, s>>>(kappa, fsc, out);
  count_launch();
  TD_LAUNCH_CHECK();
}

}  // namespace tddft
