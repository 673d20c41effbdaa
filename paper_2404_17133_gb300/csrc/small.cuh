// Small dense subspace algebra (projected matrices of size n <= kSmallMax).
#pragma once
#include "common.cuh"

namespace tddft {

constexpr int kSmallMax = 160;   // largest projected matrix (subspace) handled
constexpr int kWantMax = 64;     // largest number of refined eigenpairs

// FP32 eigendecomposition of a symmetric FP64 matrix H (n x n, leading dim ldh):
// eigenvalues ascending in lam32[n]; eigenvectors as rows vec32[j*n + r].
void eig32(const double* H, int ldh, int n, float* lam32, float* vec32, cudaStream_t s);

// FP64 eigenpairs (lowest k) of H refined from the FP32 decomposition:
// lam[k] ascending, vecs[i*n + r] (row i = eigenvector i, orthonormal).
// `rounds` Newton-type correction rounds, then Cholesky-QR and an FP64
// Rayleigh-Ritz on the k-dimensional space.  scratch: >= 2*k*n doubles.
void refine_lowest(const double* H, int ldh, int n, int k, const float* lam32, const float* vec32,
                   double* lam, double* vecs, double* scratch, int rounds, cudaStream_t s);

// Y[r] = (H - sigma[r] I)^-1 B[r] for r < nr (rows of length n), from the FP32
// decomposition plus `nref` FP64 residual-correction rounds (kept only while
// they reduce the residual).
void shifted_solve(const double* H, int ldh, int n, const float* lam32, const float* vec32,
                   const double* sigma, int nr, const double* B, double* Y, int nref,
                   cudaStream_t s);

// Y[r] = (H - sigma[r] I)^-1 B[r] for r < nr by Gaussian elimination with
// partial pivoting, one CTA per right-hand side; storage and compute type S
// (float or double).
template <typename S>
void lu_shift_solve(const S* H, int ldh, int n, const double* sigma, int nr, const S* B, S* Y,
                    cudaStream_t s);

// Small part of one paired Galerkin iteration, one CTA per system r < nr, with
// a- = L L^T (L lower) and H = L^T a+ L (both n x n, row stride ld):
//   z = L^-1 h-[r],  (H - s_r^2) u~ = L^T h+[r] + s_r z  (LU, partial pivoting),
//   uc[r] = L u~,  wc[r] = L^-T (z + s_r u~)      (hm NULL: z = 0).
// hp, hm, uc, wc: [nr][n]; sh: shifts s_r (device).  Type S throughout.
template <typename S>
void paired_small_solve(const S* L, const S* H, int ld, int n, const S* hp, const S* hm, const double* sh,
                        int nr, S* uc, S* wc, cudaStream_t s);

// In-place Cholesky H = L L^T (lower, zeroed above the diagonal), type S.
// info[0] = 0 on success, j+1 when pivot j is not positive / not finite.
template <typename S>
void cholesky(S* H, int ldh, int n, int* info, cudaStream_t s);

// Bordered Cholesky: rows < n0 of L (row stride ld) hold the lower factor of
// the leading n0 x n0 block; rows n0..n-1 hold rows n0..n-1 of the matrix.  On
// return rows n0..n-1 hold the factor's new rows (zero above the diagonal).
// info[0] = 0 on success, j+1 when pivot j is not positive / not finite.
template <typename S>
void cholesky_border(S* L, int ld, int n0, int n, int* info, cudaStream_t s);

// Triangular solves with the lower factor L (n x n, ldl) for nr right-hand
// sides stored as rows of B (in place): trans = 0: L x = b; 1: L^T x = b.
template <typename S>
void trsv_rows(const S* L, int ldl, int n, S* B, int nr, int trans, cudaStream_t s);

// Orthonormalisation helper for a block of candidate rows (Gram matrix
// G = C C^T given): pivot-dropping Cholesky G = R^T R over the candidates in
// order; a candidate whose remaining squared norm is below
// drop2 * norm0sq[j] is dropped (norm0sq NULL: unit norms).  Writes T (nc x nc, row-major) with
// C_new = T C orthonormal (zero rows for dropped) and keep[j] flags.
void chol_drop(const double* G, int nc, const double* norm0sq, double drop2, double* T,
               int* keep, cudaStream_t s);

// ---- batched forms for many small independent problems (device descriptor
// arrays; one CTA per entry).  Sizes up to kBatchSmall.
constexpr int kBatchSmall = 112;
struct BEig {            // lowest k eigenpairs of the symmetric part of H (n x n, row stride ld)
  const double* H; int ld, n, k;
  double* lam;           // [k] ascending
  double* vec;           // [k][n]
};
struct BLu {             // y = (H - sigma I)^-1 b (symmetric part of H)
  const double* H; int ld, n; double sigma;
  const double* b; double* y;   // [n]
};
struct BDrop {           // chol_drop of G (nc x nc) -> T, keep (norm0sq may be NULL)
  const double* G; int nc; const double* norm0sq; double* T; int* keep;
};
void batch_eig(const BEig* d, int nb, int nmax, cudaStream_t s);
void batch_lu(const BLu* d, int nr, int nmax, cudaStream_t s);
void batch_chol_drop(const BDrop* d, int nb, int ncmax, double drop2, cudaStream_t s);

}  // namespace tddft
