// tcgen05 tensor-core contraction for the exchange term K1 (BF16 hi+lo split).
#pragma once
#include "common.cuh"

namespace tddft {

// K1[(n,i)][b] (+)= sum_(P,a) Z[(n,i)][(P,a)] Kvv[P][a][b] for one chunk of pn
// auxiliary rows, with Z and Kvv each split as hi + lo BF16 and the three
// products hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory.
//   Zhi/Zlo [M][pn*nv] row-major; Kvv_hi/lo [pn][nv][nv] (symmetric in a,b);
//   out [M][nv] FP32, accumulated into when `accumulate`.
void tc_exchange_k1(const __nv_bfloat16* Zhi, const __nv_bfloat16* Zlo, int M, int pn, int nv,
                    const __nv_bfloat16* Kvv_hi, const __nv_bfloat16* Kvv_lo, float* out,
                    bool accumulate, cudaStream_t s);

}  // namespace tddft
