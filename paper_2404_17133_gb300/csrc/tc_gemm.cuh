// tcgen05 tensor-core contraction for the exchange term K1 (BF16 hi+lo split).
#pragma once
#include "common.cuh"

namespace tddft {

// Row pitch (elements) of the padded BF16 operands: nv rounded up to 8 so that
// every TMA stride is a multiple of 16 bytes.
int tc_pad(int nv);

// FP32 Z [M][pn][nv] -> BF16 hi + lo [M][pn][tc_pad(nv)] (pads zero).
void tc_split_pad(const float* Z, int M, int pn, int nv, __nv_bfloat16* hi, __nv_bfloat16* lo,
                  cudaStream_t s);

// K1[(n,i)][b] (+)= sum_(P,a) Z[(n,i)][P][a] Kvv[P][a][b] for one chunk of pn
// auxiliary rows, with Z and Kvv each split as hi + lo BF16 and the three
// products hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory.
//   Zhi/Zlo [M][pn][tc_pad(nv)]; Kvv_hi/lo [pn][nv][tc_pad(nv)] (symmetric in a,b);
//   out [M][nv] FP32, accumulated into when `accumulate`.  Timeouts of the
//   kernel's internal waits are reported by OR-ing a nonzero code into *err.
void tc_exchange_k1(const __nv_bfloat16* Zhi, const __nv_bfloat16* Zlo, int M, int pn, int nv,
                    const __nv_bfloat16* Kvv_hi, const __nv_bfloat16* Kvv_lo, float* out,
                    bool accumulate, int* err, cudaStream_t s);

}  // namespace tddft
