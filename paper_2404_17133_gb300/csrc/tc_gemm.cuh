// tcgen05 tensor-core contractions of the exchange terms (FP16 or BF16 hi+lo splits, FP8 ris).
#pragma once
#include "common.cuh"

namespace tddft {

// 16-bit element types of the tensor-core operands: BF16 (ris factors and
// their trial-vector splits) or FP16 (the exact operator: every operand scaled
// by a power of two and split into FP16 hi + lo).
enum class TcElt : int { BF16 = 0, F16 = 1 };

// Row pitch (elements) of the padded 16-bit operands: nv rounded up to 8 so
// that every TMA stride is a multiple of 16 bytes.
int tc_pad(int nv);
// Row pitch (elements) of the padded FP8 operands: n rounded up to 16.
int tc_pad16(int n);

// Factor rows src [rows][n1][n2] (F64, F32 or BF16) -> hi (+ lo unless NULL)
// [rows][n2][tc_pad(n1)] of element type et, transposed in the last two
// indices; FP16 parts are of (*scale) x (scale a device scalar), BF16 parts
// take no scale (NULL).
void tc_transpose_split(const void* src, DType ts, int rows, int n1, int n2, void* hi, void* lo, TcElt et,
                        const float* scale, cudaStream_t s);

// Rows src [rows][n] (F64, F32 or BF16) -> hi (+ lo unless NULL) [rows][tc_pad(n)],
// element type and scale as for tc_transpose_split.
void tc_pad_split(const void* src, DType ts, long long rows, int n, void* hi, void* lo, TcElt et,
                  const float* scale, cudaStream_t s);

// C[m][n] (+)= s * sum_(P<pn) sum_(k<Kin) A[m][P][k] B[P][n][k] on the tcgen05
// tensor cores.  A: [M][pn][tc_pad(Kin)], B: [pn][N][tc_pad(Kin)] of element type
// et, C: [M][N] FP32, accumulated into when `accumulate`; s = *scale (a device
// scalar) or 1 when scale is NULL.  Operand splits: with Alo and Blo the three
// products hi*hi + hi*lo + lo*hi are formed; with Alo alone the two products
// Ahi*B + Alo*B; with neither one product (Blo without Alo is not allowed).
// Timeouts of the kernel's internal waits are reported by OR-ing a nonzero
// code into *err.  With `prof`, CUDA events bracket the contraction kernel
// alone (not the split reduction) and prof_flops / prof_bytes (the launch's
// algorithmic flops and bytes) are credited to it.  max_kb > 0 bounds the
// K extent one CTA accumulates in FP32 to max_kb blocks of 64 elements (more
// split-K partials, summed in a fixed order), for contractions whose K is long enough that the length of
// the accumulation run sets the rounding error.
struct KernelProfile;
void tc_contract(const void* Ahi, const void* Alo, int M, int pn, int Kin, const void* Bhi, const void* Blo,
                 int N, float* out, bool accumulate, TcElt et, const float* scale, int* err, cudaStream_t s,
                 KernelProfile* prof = nullptr, double prof_flops = 0.0, double prof_bytes = 0.0, int max_kb = 0);

// Stage-1 exchange contraction on the tensor cores, batched over P:
//   C_P[r][c] = sum_(k<K) A[r][k] B_P[c][k],  A: [M][tc_pad(K)], B: [pn][N][tc_pad(K)],
// written as hi (+ lo) parts of element type et to out[(g*N + c)][P][ri]
// (r = g*R + ri, row pitch pn*tc_pad(R)) -- the A operand layout of
// tc_contract.  N <= 256.  BF16: with lo operands the hi/lo products are
// formed, mul NULL.  FP16: A and B as hi + lo, and the parts are those of
// (*mul) C_P (mul a device scalar).
void tc_stage1(const void* Ahi, const void* Alo, int M, int K, const void* Bhi, const void* Blo, int N, int pn,
               int R, TcElt et, const float* mul, void* out_hi, void* out_lo, int* err, cudaStream_t s);

// ---- FP16 scales of the exact operator.  Factor-set scale block (8 floats):
//   [0] s_oo, [1] s_oo * max ||L^P_oo[i][:]||, [2] s_vv, [4] s_ov,
//   [5] s_ov * max ||L^P_ov[i][:]||  ([3], [6], [7] unused), each s the power
// of two with max |s L| < 2^14.
// sc[0] = s, sc[1] = s * (largest row norm) for FP32 rows [rows][n]; scratch:
// two device words.
void tc_f16_tensor_scale(const float* src, long long rows, int n, float* sc, unsigned* scratch, cudaStream_t s);
// Per-product block (5 floats) for trial vectors X [m][no][nv] (F64 or F32):
//   [0] s_x (max |s_x X| < 2^14), [1] m_z, [2] m_q: the multipliers of the
//   stage-1 accumulators (Z' = s_oo s_x Z, Q' = s_x s_ov Q) before their FP16
//   split, powers of two with |m Z'| < 2^15 by Cauchy-Schwarz;
//   [3] 1 / (m_z s_oo s_x s_vv), [4] 1 / (m_q s_x s_ov^2): the factors of the
//   K1 and K2 sums.  kappa: three device words.  No host synchronisation.
void tc_f16_product_scales(const void* X, DType xt, int m, int no, int nv, const float* fsc, float* out,
                           unsigned* kappa, cudaStream_t s);
// out[0] = 1 / (a[0] * b[0]) (device scalars): the factor that removes two scales.
void tc_inv_prod(const float* a, const float* b, float* out, cudaStream_t s);

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
// device scratch of three words.  No host synchronisation.
void tc_fp8_scales(const void* X, DType xt, int m, int no, int nv, const float* s_vv, const float* rho_oo,
                   const float* s_vo, const float* rho_ov, int nK, float* out, unsigned* kappa,
                   cudaStream_t s);
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
