// tcgen05 tensor-core contraction for the exchange term K1 (BF16 hi+lo split).
#pragma once
#include "common.cuh"

namespace tddft {

// Row pitch (elements) of the padded BF16 operands: nv rounded up to 8 so that
// every TMA stride is a multiple of 16 bytes.
int tc_pad(int nv);
// Row pitch (elements) of the padded FP8 operands: n rounded up to 16.
int tc_pad16(int n);

// FP32 Z [M][pn][nv] -> BF16 hi (+ lo unless NULL) [M][pn][tc_pad(nv)] (pads zero).
void tc_split_pad(const float* Z, int M, int pn, int nv, __nv_bfloat16* hi, __nv_bfloat16* lo,
                  cudaStream_t s);

// Factor rows src [rows][n1][n2] (F64, F32 or BF16) -> BF16 hi (+ lo unless NULL)
// [rows][n2][tc_pad(n1)], transposed in the last two indices.
// With l2, also the third part of a three-part split (x = hi + lo + l2).
void tc_transpose_split(const void* src, DType ts, int rows, int n1, int n2, __nv_bfloat16* hi,
                        __nv_bfloat16* lo, cudaStream_t s, __nv_bfloat16* l2 = nullptr);

// C[m][n] (+)= sum_(P<pn) sum_(k<Kin) A[m][P][k] B[P][n][k] on the tcgen05 tensor
// cores.  A: [M][pn][tc_pad(Kin)] BF16, B: [pn][N][tc_pad(Kin)] BF16, C: [M][N] FP32,
// accumulated into when `accumulate`.  Operand splits: with Alo and Blo the
// three products hi*hi + hi*lo + lo*hi are formed; with Alo alone the two
// products Ahi*B + Alo*B; with neither one BF16 product (Blo without Alo is not
// allowed).  Timeouts of the kernel's internal waits are reported by OR-ing a
// nonzero code into *err.  With `cross`, only the two cross products
// Ahi*Blo + Alo*Bhi are formed (a pass of a three-part split).  With `prof`, CUDA events bracket the contraction
// kernel alone (not the split reduction) and prof_flops / prof_bytes (the
// launch's algorithmic flops and bytes) are credited to it.
struct KernelProfile;
void tc_contract(const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo, int M, int pn, int Kin,
                 const __nv_bfloat16* Bhi, const __nv_bfloat16* Blo, int N, float* out,
                 bool accumulate, int* err, cudaStream_t s, KernelProfile* prof = nullptr,
                 double prof_flops = 0.0, double prof_bytes = 0.0, bool cross = false);

// Rows src [rows][n] (F64, F32 or BF16) -> BF16 hi (+ lo unless NULL) [rows][tc_pad(n)].
void tc_pad_split(const void* src, DType ts, long long rows, int n, __nv_bfloat16* hi,
                  __nv_bfloat16* lo, cudaStream_t s, __nv_bfloat16* l2 = nullptr);

// Stage-1 exchange contraction on the tensor cores, batched over P:
//   C_P[r][c] = sum_(k<K) A[r][k] B_P[c][k],  A: [M][tc_pad(K)], B: [pn][N][tc_pad(K)],
// written as BF16 hi (+ lo) to out[(g*N + c)][P][ri] (r = g*R + ri, row pitch
// pn*tc_pad(R)) -- the A operand layout of tc_contract.  N <= 256.  With lo
// operands the three hi/lo products are formed.
void tc_stage1(const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo, int M, int K,
               const __nv_bfloat16* Bhi, const __nv_bfloat16* Blo, int N, int pn, int R,
               __nv_bfloat16* out_hi, __nv_bfloat16* out_lo, int* err, cudaStream_t s);

// ---- FP8 (e4m3) ris exchange operands with one scale per auxiliary row P.
// Factor rows src [rows][n1][n2] (BF16) -> dst [rows][n2][tc_pad16(n1)] e4m3
// (transposed in the last two indices) of src / scale[P], scale[P] =
// max |src[P]| / 448.
void tc_quant_e4m3(const __nv_bfloat16* src, int rows, int n1, int n2, unsigned char* dst, float* scale,
                   cudaStream_t s);
// rho[P] = max_i sqrt(sum_c src[P][i][c]^2), src [rows][nr][nc] BF16.
void tc_row_norm_max(const __nv_bfloat16* src, int rows, int nr, int nc, float* rho, cudaStream_t s);
// Per-product scales of the FP8 exchange contractions for trial vectors X
// [m][no][nv] (F64 or F32): out[0], out[1] = the output factors 1/g1, 1/g2 of
// K1 and K2; out[2 + P] = s_vv[P] g1 and out[2 + nK + P] = s_vo[P] g2, the
// multipliers of the stage-1 results (mu_P).  g1 = 224 / max_P(s_vv[P]
// rho_oo[P] kappa_col), g2 likewise with s_vo, rho_ov and kappa_row, where
// kappa_col = max ||X[n][:][a]|| and kappa_row = max ||X[n][j][:]||.  kappa:
// device scratch of two words.  No host synchronisation.
void tc_fp8_scales(const void* X, DType xt, int m, int no, int nv, const float* s_vv, const float* rho_oo,
                   const float* s_vo, const float* rho_ov, int nK, float* out, unsigned* kappa,
                   cudaStream_t s);
// Stage 1 with three-part BF16 operands and output (x = x0 + x1 + x2, 24
// significand bits; the six products down to 2^-18 of the leading one, FP32
// accumulation): an FP32-accurate product on the tensor cores.  Needs
// tc_stage1_3_fits(N) (the three-part tiles of a stage fit twice in shared memory).
void tc_stage1_3(const __nv_bfloat16* const A[3], int M, int K, const __nv_bfloat16* const B[3], int N, int pn,
                 int R, __nv_bfloat16* const out[3], int* err, cudaStream_t s);
bool tc_stage1_3_fits(int N);
// Stage 1 with e4m3 hi + lo output: out[(g*N + c)][P][ri] (row pitch
// pn*tc_pad16(R) bytes) = split of mu[P] * C_P[r][c]; A as BF16 hi + lo, B BF16.
void tc_stage1_fp8(const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo, int M, int K, const __nv_bfloat16* B,
                   int N, int pn, int R, const float* mu, unsigned char* out_hi, unsigned char* out_lo, int* err,
                   cudaStream_t s);
// out (+)= (*scale) * sum_P sum_k A[m][P][k] B[P][n][k] on the tensor cores
// (kind::f8f6f4, e4m3 x e4m3, FP32 accumulation): A as e4m3 hi + lo
// [M][pn][tc_pad16(Kin)], B e4m3 [pn][N][tc_pad16(Kin)]; scale a device scalar.
void tc_contract8(const unsigned char* Ahi, const unsigned char* Alo, int M, int pn, int Kin,
                  const unsigned char* B, int N, float* out, bool accumulate, const float* scale, int* err,
                  cudaStream_t s);

}  // namespace tddft
