// Small dense subspace algebra on the GPU (the projected problems of Eq. 1-2 and
// of the inner solves of Eq. precondition).
//
// GB300 executes FP64 at about 1/64 of the FP32 SIMT rate, so the O(n^3) parts
// run in FP32 and FP64 is kept to O(n^2 k) work:
//   * eig32: parallel cyclic Jacobi (round-robin pair ordering, n/2 disjoint
//     rotations per round) in FP32, one CTA, matrix and eigenvectors in shared
//     memory;
//   * refine_lowest: for each wanted eigenpair, Newton-type corrections
//     q <- q - sum_{j != i} v_j (v_j^T r) / (lam_j - lam), r = Hq - lam q, with
//     the FP32 eigenvectors v_j (one CTA per pair), then Cholesky-QR of the k
//     vectors and an FP64 Rayleigh-Ritz (FP64 Jacobi on the k x k matrix);
//   * shifted_solve: (H - sigma)^-1 b from the FP32 decomposition plus FP64
//     residual-correction rounds (mixed-precision iterative refinement);
//   * cholesky / trsv_rows: FP64 factor of a projected A-B and triangular solves;
//   * chol_drop: pivot-dropping Cholesky of a candidate Gram matrix, the
//     in-block step of the Gram-Schmidt orthonormalisation.
#include "small.cuh"

namespace tddft {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA; every thread gets the result.  `red` has >= 33 doubles.
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

template <typename T> __device__ __forceinline__ T big_theta();
template <> __device__ __forceinline__ float big_theta<float>() { return 1e18f; }
template <> __device__ __forceinline__ double big_theta<double>() { return 1e150; }

// Parallel cyclic Jacobi on the symmetric matrix A (n x n, shared memory,
// leading dimension ld) accumulating Q <- Q G.  Each round applies n/2
// disjoint rotations (circle-method pairing); a sweep is n-1 rounds.  The
// two-sided update of a round is done block by block: the 2x2 block of rows
// (p_i, q_i) and columns (p_j, q_j) becomes R_i X R_j^T, so a round needs one
// pass over A (and Q) and two barriers.
template <typename T>
__device__ void jacobi_cta(T* A, T* Q, int n, int ld, double frob, int max_sweeps, double stop_rel,
                           int* pp, int* qq, T* cc, T* ss, unsigned* smax) {
  const int NP = (n + 1) & ~1;
  const int half = NP / 2;
  const int tid = threadIdx.x, nth = blockDim.x;
  const T stop = (T)(stop_rel * frob);
  const T skip = (T)(stop_rel * 1e-3 * frob);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *smax = 0u;
    __syncthreads();
    for (int r = 0; r < NP - 1; ++r) {
      for (int i = tid; i < half; i += nth) {
        int p, q;
        if (i == 0) { p = r; q = NP - 1; }
        else { p = (r + i) % (NP - 1); q = (r - i + NP - 1) % (NP - 1); }
        T c = 1, s = 0;
        if (p < n && q < n) {
          T apq = A[p * ld + q];
          T aa = apq < 0 ? -apq : apq;
          if (aa > skip) {
            atomicMax(smax, __float_as_uint((float)aa));
            T theta = (A[q * ld + q] - A[p * ld + p]) / (T(2) * apq);
            T at = theta < 0 ? -theta : theta;
            T t = at > big_theta<T>() ? T(0.5) / theta
                                      : (theta < 0 ? T(-1) : T(1)) / (at + sqrt(theta * theta + T(1)));
            c = T(1) / sqrt(t * t + T(1));
            s = t * c;
          }
        }
        pp[i] = p; qq[i] = q; cc[i] = c; ss[i] = s;
      }
      __syncthreads();
      // A <- G^T A G, block by block: warp w takes the row pairs w, w + nw, ...,
      // its lanes the column pairs (no index division in the loop)
      const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
      for (int bi = warp; bi < half; bi += nw) {
        const T si = ss[bi], ci = cc[bi];
        T* rp = A + pp[bi] * ld;
        T* rq = A + qq[bi] * ld;
        for (int bj = lane; bj < half; bj += 32) {
          const T sj = ss[bj];
          if (si == T(0) && sj == T(0)) continue;
          const T cj = cc[bj];
          const int pj = pp[bj], qj = qq[bj];
          const T x00 = rp[pj], x01 = rp[qj], x10 = rq[pj], x11 = rq[qj];
          // rows: R_i = [[c, -s], [s, c]]
          const T y00 = ci * x00 - si * x10, y01 = ci * x01 - si * x11;
          const T y10 = si * x00 + ci * x10, y11 = si * x01 + ci * x11;
          // columns: times [[c, s], [-s, c]]
          T z00 = cj * y00 - sj * y01, z01 = sj * y00 + cj * y01;
          T z10 = cj * y10 - sj * y11, z11 = sj * y10 + cj * y11;
          if (bi == bj) { z01 = T(0); z10 = T(0); }   // the rotation annihilates a_pq
          rp[pj] = z00; rp[qj] = z01;
          rq[pj] = z10; rq[qj] = z11;
        }
      }
      // Q <- Q G (columns p_j, q_j of every row): warp per column pair, lanes over rows
      for (int bj = warp; bj < half; bj += nw) {
        const T sj = ss[bj];
        if (sj == T(0)) continue;
        const T cj = cc[bj];
        const int pj = pp[bj], qj = qq[bj];
        for (int row = lane; row < NP; row += 32) {
          const T qp = Q[row * ld + pj], qv = Q[row * ld + qj];
          Q[row * ld + pj] = cj * qp - sj * qv;
          Q[row * ld + qj] = sj * qp + cj * qv;
        }
      }
      __syncthreads();
    }
    float m = __uint_as_float(*smax);
    __syncthreads();
    if (m <= (float)stop) break;
  }
}

// rank of diagonal entry t among the first n (ascending, ties by index)
template <typename T>
__device__ int diag_rank(const T* A, int ld, int n, int t) {
  T v = A[t * ld + t];
  int r = 0;
  for (int j = 0; j < n; ++j) {
    T u = A[j * ld + j];
    r += (u < v) || (u == v && j < t);
  }
  return r;
}

__global__ void __launch_bounds__(1024) k_eig32(const double* __restrict__ H, int ldh, int n,
                                                float* __restrict__ lam32, float* __restrict__ vec32) {
  extern __shared__ float sm32[];
  __shared__ int pp[kSmallMax / 2 + 1], qq[kSmallMax / 2 + 1];
  __shared__ float cc[kSmallMax / 2 + 1], ss[kSmallMax / 2 + 1];
  __shared__ unsigned smax;
  __shared__ double red[33];
  const int NP = (n + 1) & ~1, ld = NP + 1;
  float* A = sm32;
  float* Q = sm32 + NP * ld;
  double f2 = 0.0;
  for (int idx = threadIdx.x; idx < NP * NP; idx += blockDim.x) {
    int r = idx / NP, c = idx - r * NP;
    double v = 0.0;
    if (r < n && c < n) v = 0.5 * (H[(long long)r * ldh + c] + H[(long long)c * ldh + r]);
    f2 += v * v;
    A[r * ld + c] = (float)v;
    Q[r * ld + c] = (r == c) ? 1.f : 0.f;
  }
  double frob = sqrt(block_sum(f2, red));
  jacobi_cta<float>(A, Q, n, ld, frob, 16, 2e-7, pp, qq, cc, ss, &smax);
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    int r = diag_rank(A, ld, n, t);
    lam32[r] = A[t * ld + t];
    for (int q = 0; q < n; ++q) vec32[(long long)r * n + q] = Q[q * ld + t];
  }
}

// One CTA per wanted eigenpair i: Newton-type refinement in FP64.
__global__ void __launch_bounds__(256) k_refine(const double* __restrict__ H, int ldh, int n,
                                                const float* __restrict__ lam32,
                                                const float* __restrict__ vec32, int rounds,
                                                double* __restrict__ Qk, double* __restrict__ Yk) {
  __shared__ double q[kSmallMax], y[kSmallMax], r[kSmallMax], c[kSmallMax];
  __shared__ double red[33];
  const int i = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  float lmin = lam32[0], lmax = lam32[n - 1];
  double scale = fmax(fabs((double)lmin), fabs((double)lmax));
  double gapmin = 1e-5 * scale;
  for (int t = tid; t < n; t += blockDim.x) q[t] = vec32[(long long)i * n + t];
  __syncthreads();
  for (int it = 0; it <= rounds; ++it) {
    // y = H q  (warp per row)
    for (int row = w; row < n; row += nw) {
      double acc = 0.0;
      for (int l = lane; l < n; l += 32) acc += H[(long long)row * ldh + l] * q[l];
      acc = warp_sum(acc);
      if (lane == 0) y[row] = acc;
    }
    __syncthreads();
    double qy = 0.0, qq2 = 0.0;
    for (int t = tid; t < n; t += blockDim.x) { qy += q[t] * y[t]; qq2 += q[t] * q[t]; }
    qy = block_sum(qy, red);
    qq2 = block_sum(qq2, red);
    double lam = qy / qq2;
    if (it == rounds) break;
    for (int t = tid; t < n; t += blockDim.x) r[t] = y[t] - lam * q[t];
    __syncthreads();
    for (int j = w; j < n; j += nw) {
      double acc = 0.0;
      for (int l = lane; l < n; l += 32) acc += (double)vec32[(long long)j * n + l] * r[l];
      acc = warp_sum(acc);
      if (lane == 0) {
        double den = (double)lam32[j] - lam;
        c[j] = (j == i || fabs(den) < gapmin) ? 0.0 : acc / den;
      }
    }
    __syncthreads();
    for (int t = tid; t < n; t += blockDim.x) {
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc += (double)vec32[(long long)j * n + t] * c[j];
      q[t] -= acc;
    }
    __syncthreads();
    double nn = 0.0;
    for (int t = tid; t < n; t += blockDim.x) nn += q[t] * q[t];
    nn = block_sum(nn, red);
    double inv = 1.0 / sqrt(nn);
    for (int t = tid; t < n; t += blockDim.x) q[t] *= inv;
    __syncthreads();
  }
  for (int t = tid; t < n; t += blockDim.x) {
    Qk[(long long)i * n + t] = q[t];
    Yk[(long long)i * n + t] = y[t];
  }
}

// One CTA: Cholesky-QR of the k refined vectors (rows of Qk, with Yk = H Qk
// carried along), FP64 Rayleigh-Ritz on the k x k matrix, rotate into `vecs`.
__global__ void __launch_bounds__(1024) k_orth_rr(double* __restrict__ Qk, double* __restrict__ Yk,
                                                  int k, int n, double* __restrict__ lam,
                                                  double* __restrict__ vecs) {
  extern __shared__ double sm64[];
  __shared__ int pp[kWantMax / 2 + 1], qq[kWantMax / 2 + 1];
  __shared__ double cc[kWantMax / 2 + 1], ss[kWantMax / 2 + 1];
  __shared__ unsigned smax;
  __shared__ double red[33];
  const int KP = (k + 1) & ~1, ld = KP + 1;
  double* G = sm64;             // Gram / Rayleigh matrix
  double* Z = sm64 + KP * ld;   // rotations
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  // Gram matrix of the k vectors
  for (int pidx = w; pidx < k * k; pidx += nw) {
    int a = pidx / k, b = pidx - a * k;
    if (b < a) continue;
    double acc = 0.0;
    for (int l = lane; l < n; l += 32) acc += Qk[(long long)a * n + l] * Qk[(long long)b * n + l];
    acc = warp_sum(acc);
    if (lane == 0) { G[a * ld + b] = acc; G[b * ld + a] = acc; }
  }
  __syncthreads();
  // Cholesky G = R^T R (R upper, kept in the upper triangle of G)
  for (int j = 0; j < k; ++j) {
    if (tid == 0) G[j * ld + j] = sqrt(fmax(G[j * ld + j], 1e-300));
    __syncthreads();
    double piv = G[j * ld + j];
    for (int m = j + 1 + tid; m < k; m += blockDim.x) G[j * ld + m] /= piv;
    __syncthreads();
    for (int idx = tid; idx < (k - j - 1) * (k - j - 1); idx += blockDim.x) {
      int a = j + 1 + idx / (k - j - 1), b = j + 1 + idx % (k - j - 1);
      if (b >= a) G[a * ld + b] -= G[j * ld + a] * G[j * ld + b];
    }
    __syncthreads();
  }
  // rows j of Q' = R^-T Q (forward substitution, in place), same for Y
  for (int j = 0; j < k; ++j) {
    double inv = 1.0 / G[j * ld + j];
    for (int t = tid; t < n; t += blockDim.x) {
      double qa = Qk[(long long)j * n + t], ya = Yk[(long long)j * n + t];
      for (int l = 0; l < j; ++l) {
        double rl = G[l * ld + j];
        qa -= rl * Qk[(long long)l * n + t];
        ya -= rl * Yk[(long long)l * n + t];
      }
      Qk[(long long)j * n + t] = qa * inv;
      Yk[(long long)j * n + t] = ya * inv;
    }
    __syncthreads();
  }
  // Rayleigh matrix B = Q' Y'^T (symmetrised), Jacobi in FP64
  for (int idx = tid; idx < KP * KP; idx += blockDim.x) {
    int a = idx / KP, b = idx - a * KP;
    G[a * ld + b] = 0.0;
    Z[a * ld + b] = (a == b) ? 1.0 : 0.0;
  }
  __syncthreads();
  double f2 = 0.0;
  for (int pidx = w; pidx < k * k; pidx += nw) {
    int a = pidx / k, b = pidx - a * k;
    if (b < a) continue;
    double acc = 0.0;
    for (int l = lane; l < n; l += 32)
      acc += Qk[(long long)a * n + l] * Yk[(long long)b * n + l] +
             Qk[(long long)b * n + l] * Yk[(long long)a * n + l];
    acc = 0.5 * warp_sum(acc);
    if (lane == 0) { G[a * ld + b] = acc; G[b * ld + a] = acc; f2 += (a == b ? 1.0 : 2.0) * acc * acc; }
  }
  double frob = sqrt(block_sum(f2, red));
  jacobi_cta<double>(G, Z, k, ld, frob, 30, 1e-15, pp, qq, cc, ss, &smax);
  for (int t = tid; t < k; t += blockDim.x) lam[diag_rank(G, ld, k, t)] = G[t * ld + t];
  __syncthreads();
  // vecs[rank(t)] = sum_l Z[l][t] Q'[l]
  for (int idx = tid; idx < k * n; idx += blockDim.x) {
    int t = idx / n, e = idx - t * n;
    int r = diag_rank(G, ld, k, t);
    double acc = 0.0;
    for (int l = 0; l < k; ++l) acc += Z[l * ld + t] * Qk[(long long)l * n + e];
    vecs[(long long)r * n + e] = acc;
  }
}

__global__ void __launch_bounds__(256) k_shifted(const double* __restrict__ H, int ldh, int n,
                                                 const float* __restrict__ lam32,
                                                 const float* __restrict__ vec32,
                                                 const double* __restrict__ sigma,
                                                 const double* __restrict__ B, double* __restrict__ Y,
                                                 int nref) {
  __shared__ double b[kSmallMax], y[kSmallMax], r[kSmallMax], c[kSmallMax], best[kSmallMax];
  __shared__ double red[33];
  const int rr = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const double sg = sigma[rr];
  for (int t = tid; t < n; t += blockDim.x) { b[t] = B[(long long)rr * n + t]; y[t] = 0.0; r[t] = b[t]; }
  __syncthreads();
  double best_res = 1e300;
  for (int it = 0; it <= nref; ++it) {
    // y += V (Lam - sigma)^-1 V^T r
    for (int j = w; j < n; j += nw) {
      double acc = 0.0;
      for (int l = lane; l < n; l += 32) acc += (double)vec32[(long long)j * n + l] * r[l];
      acc = warp_sum(acc);
      if (lane == 0) {
        double den = (double)lam32[j] - sg;
        if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
        c[j] = acc / den;
      }
    }
    __syncthreads();
    for (int t = tid; t < n; t += blockDim.x) {
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc += (double)vec32[(long long)j * n + t] * c[j];
      y[t] += acc;
    }
    __syncthreads();
    if (nref == 0) { for (int t = tid; t < n; t += blockDim.x) best[t] = y[t]; break; }
    // r = b - (H - sigma) y
    for (int row = w; row < n; row += nw) {
      double acc = 0.0;
      for (int l = lane; l < n; l += 32) acc += H[(long long)row * ldh + l] * y[l];
      acc = warp_sum(acc);
      if (lane == 0) r[row] = b[row] - (acc - sg * y[row]);
    }
    __syncthreads();
    double rn = 0.0;
    for (int t = tid; t < n; t += blockDim.x) rn += r[t] * r[t];
    rn = block_sum(rn, red);
    if (rn < best_res) {
      best_res = rn;
      for (int t = tid; t < n; t += blockDim.x) best[t] = y[t];
      __syncthreads();
    } else {
      break;
    }
  }
  __syncthreads();
  for (int t = tid; t < n; t += blockDim.x) Y[(long long)rr * n + t] = best[t];
}

template <typename S>
__global__ void __launch_bounds__(1024) k_cholesky(S* __restrict__ H, int ldh, int n,
                                                   int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char chol_raw[];
  S* A = reinterpret_cast<S*>(chol_raw);
  __shared__ int bad;
  const int ld = n + 1;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    int r = idx / n, c = idx - r * n;
    A[r * ld + c] = S(0.5) * (H[(long long)r * ldh + c] + H[(long long)c * ldh + r]);
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      S d = A[j * ld + j];
      if (!(d > S(0)) || !isfinite(d)) bad = j + 1;
      else A[j * ld + j] = sqrt(d);
    }
    __syncthreads();
    if (bad) break;
    S piv = A[j * ld + j];
    for (int r = j + 1 + tid; r < n; r += blockDim.x) A[r * ld + j] /= piv;
    __syncthreads();
    const int m = n - j - 1;
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      int r = j + 1 + idx / m, c = j + 1 + idx % m;
      if (c <= r) A[r * ld + c] -= A[r * ld + j] * A[c * ld + j];
    }
    __syncthreads();
  }
  if (tid == 0) info[0] = bad;
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    int r = idx / n, c = idx - r * n;
    H[(long long)r * ldh + c] = (c <= r && !bad) ? A[r * ld + c] : S(0);
  }
}

// Bordered Cholesky: rows < n0 of L already hold the factor of the leading
// block; rows n0..n-1 hold the new rows of the matrix (all n columns).  Each new
// row is first solved against the old factor by its own warp (forward
// substitution, no block barriers), then the new diagonal block is factored
// column by column.  Entries above the diagonal in the first n columns are zeroed.
template <typename S>
__global__ void __launch_bounds__(1024) k_chol_border(S* __restrict__ Lg, int ld, int n0, int n,
                                                      int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char cb_raw[];
  S* L = reinterpret_cast<S*>(cb_raw);   // [n][n] working copy (row stride n)
  __shared__ int bad;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx - r * n;
    L[idx] = Lg[(long long)r * ld + c];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  // phase 1: L[i][j], j < n0, for every new row i
  for (int i = n0 + warp; i < n; i += nw) {
    S* Li = L + i * n;
    for (int j = 0; j < n0; ++j) {
      const S* Lj = L + j * n;
      S acc = S(0);
      for (int q = lane; q < j; q += 32) acc += Li[q] * Lj[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      const S v = (Li[j] - acc) / Lj[j];
      __syncwarp();
      if (lane == 0) Li[j] = v;
      __syncwarp();
    }
  }
  __syncthreads();
  // phase 2: the new diagonal block, column by column
  for (int j = n0; j < n; ++j) {
    S* Lj = L + j * n;
    if (warp == 0) {
      S acc = S(0);
      for (int q = lane; q < j; q += 32) acc += Lj[q] * Lj[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      const S d = Lj[j] - acc;
      __syncwarp();
      if (lane == 0) {
        if (!(d > S(0)) || !isfinite(d)) bad = j + 1;
        else Lj[j] = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) break;
    for (int i = j + 1 + warp; i < n; i += nw) {
      S* Li = L + i * n;
      S acc = S(0);
      for (int q = lane; q < j; q += 32) acc += Li[q] * Lj[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      const S v = (Li[j] - acc) / Lj[j];
      __syncwarp();
      if (lane == 0) Li[j] = v;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) info[0] = bad;
  if (bad) return;
  // write back, zero above the diagonal
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx - r * n;
    Lg[(long long)r * ld + c] = c <= r ? L[idx] : S(0);
  }
}

template <typename S>
__global__ void __launch_bounds__(256) k_trsv(const S* __restrict__ L, int ldl, int n,
                                              S* __restrict__ B, int trans) {
  __shared__ S b[kSmallMax];
  __shared__ S xj;
  S* row = B + (long long)blockIdx.x * n;
  for (int t = threadIdx.x; t < n; t += blockDim.x) b[t] = row[t];
  __syncthreads();
  if (!trans) {
    for (int j = 0; j < n; ++j) {
      if (threadIdx.x == 0) { xj = b[j] / L[(long long)j * ldl + j]; b[j] = xj; }
      __syncthreads();
      for (int r = j + 1 + threadIdx.x; r < n; r += blockDim.x) b[r] -= L[(long long)r * ldl + j] * xj;
      __syncthreads();
    }
  } else {
    for (int j = n - 1; j >= 0; --j) {
      if (threadIdx.x == 0) { xj = b[j] / L[(long long)j * ldl + j]; b[j] = xj; }
      __syncthreads();
      for (int r = threadIdx.x; r < j; r += blockDim.x) b[r] -= L[(long long)j * ldl + r] * xj;
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) row[t] = b[t];
}

constexpr int kDropMax = 112;

// Pivot-dropping Cholesky of one candidate Gram matrix by the whole CTA
// (shared memory smd >= 2 nc (nc + 1) doubles; kj / dj shared scalars).
__device__ void chol_drop_cta(const double* __restrict__ G, int nc, const double* __restrict__ norm0sq,
                              double drop2, double* __restrict__ T, int* __restrict__ keep, double* smd,
                              int& kj, double& dj) {
  const int ld = nc + 1;
  double* R = smd;                 // working Gram -> upper factor
  double* Ti = smd + nc * ld;      // T rows
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nc * nc; idx += blockDim.x) {
    int a = idx / nc, b = idx - a * nc;
    R[a * ld + b] = 0.5 * (G[a * nc + b] + G[b * nc + a]);
    Ti[a * ld + b] = 0.0;
  }
  __syncthreads();
  // right-looking: after step j the trailing block holds the Gram matrix of the
  // candidates with the kept ones among 0..j projected out
  for (int j = 0; j < nc; ++j) {
    if (tid == 0) {
      double d = R[j * ld + j];
      const double n0 = norm0sq ? norm0sq[j] : 1.0;
      kj = (isfinite(d) && d > drop2 * n0 && d > 0.0) ? 1 : 0;
      dj = kj ? sqrt(d) : 0.0;
      keep[j] = kj;
    }
    __syncthreads();
    if (kj) {
      for (int m = j + tid; m < nc; m += blockDim.x) R[j * ld + m] = (m == j) ? dj : R[j * ld + m] / dj;
      __syncthreads();
      const int m = nc - j - 1;
      for (int idx = tid; idx < m * m; idx += blockDim.x) {
        int a = j + 1 + idx / m, b = j + 1 + idx % m;
        R[a * ld + b] -= R[j * ld + a] * R[j * ld + b];
      }
    } else {
      for (int m = j + tid; m < nc; m += blockDim.x) R[j * ld + m] = 0.0;
    }
    __syncthreads();
  }
  // T = R^-T restricted to kept rows: T[j] = (e_j - sum_{l<j} R[l][j] T[l]) / R[j][j]
  for (int j = 0; j < nc; ++j) {
    if (keep[j]) {
      double inv = 1.0 / R[j * ld + j];
      for (int c = tid; c <= j; c += blockDim.x) {
        double acc = (c == j) ? 1.0 : 0.0;
        for (int l = c; l < j; ++l) acc -= R[l * ld + j] * Ti[l * ld + c];
        Ti[j * ld + c] = acc * inv;
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nc * nc; idx += blockDim.x) {
    int a = idx / nc, b = idx - a * nc;
    T[idx] = Ti[a * ld + b];
  }
}

__global__ void __launch_bounds__(1024) k_chol_drop(const double* __restrict__ G, int nc,
                                                    const double* __restrict__ norm0sq, double drop2,
                                                    double* __restrict__ T, int* __restrict__ keep) {
  extern __shared__ double smd[];
  __shared__ int kj;
  __shared__ double dj;
  chol_drop_cta(G, nc, norm0sq, drop2, T, keep, smd, kj, dj);
}

// Gaussian elimination with partial pivoting on the augmented matrix [M | b]
// held in shared memory (n rows, row stride ld >= n + 1, compute type T), then
// back substitution; the solution replaces column n (in the original row order).
// Rows are not moved: perm[] (shared, >= n ints) records the pivot order, so an
// elimination step is one pivot search (warp 0) and one update pass.  Called by
// all threads of the CTA.
template <typename T>
__device__ void lu_solve_smem(T* A, int ld, int n, int* perm, T* y) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < n; i += blockDim.x) perm[i] = i;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {   // pivot: argmax |A[perm[i]][k]|, i >= k
      T best = T(-1);
      int bi = k;
      for (int i = k + lane; i < n; i += 32) {
        T v = A[perm[i] * ld + k];
        v = v < T(0) ? -v : v;
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        T ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0 && bi != k) {
        const int t = perm[k];
        perm[k] = perm[bi];
        perm[bi] = t;
      }
    }
    __syncthreads();
    const int pk = perm[k];
    const T* prow = A + pk * ld;
    T piv = prow[k];
    if (piv == T(0)) piv = T(1e-30);
    const T inv = T(1) / piv;
    for (int i = k + 1 + warp; i < n; i += nw) {
      T* row = A + perm[i] * ld;
      const T l = row[k] * inv;
      for (int j = k + 1 + lane; j <= n; j += 32) row[j] -= l * prow[j];
    }
    __syncthreads();
  }
  // back substitution by one warp: y_k = (b_k - sum_{j>k} U_kj y_j) / U_kk
  if (warp == 0) {
    for (int k = n - 1; k >= 0; --k) {
      const T* row = A + perm[k] * ld;
      T piv = row[k];
      if (piv == T(0)) piv = T(1e-30);
      const T yk = row[n] / piv;
      __syncwarp();
      for (int i = lane; i < k; i += 32) {
        T* ri = A + perm[i] * ld;
        ri[n] -= ri[k] * yk;
      }
      if (lane == 0) y[k] = yk;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) A[i * ld + n] = y[i];
  __syncthreads();
}

// One CTA per right-hand side r: Gaussian elimination with partial pivoting on
// [(H - sigma_r I) | b_r] in shared memory (compute type T), then back substitution.
template <typename T>
__global__ void __launch_bounds__(512) k_lu_shift(const T* __restrict__ H, int ldh, int n,
                                                  const double* __restrict__ sig,
                                                  const T* __restrict__ B, T* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char lu_raw[];
  T* A = reinterpret_cast<T*>(lu_raw);
  const int ld = n + 2;
  __shared__ int perm[kSmallMax];
  __shared__ T yv[kSmallMax];
  const int r = blockIdx.x;
  const double sg = sig[r];
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int idx = tid; idx < n * (n + 1); idx += nth) {
    int i = idx / (n + 1), j = idx - i * (n + 1);
    T v;
    if (j < n) v = T(0.5) * (H[(long long)i * ldh + j] + H[(long long)j * ldh + i]) - (i == j ? T(sg) : T(0));
    else v = B[(long long)r * n + i];
    A[i * ld + j] = v;
  }
  __syncthreads();
  lu_solve_smem<T>(A, ld, n, perm, yv);
  for (int i = tid; i < n; i += nth) Y[(long long)r * n + i] = A[i * ld + n];
}

// Triangular solve by one warp on a vector b[n] in shared memory with the lower
// factor L (global, row stride ldl): trans = 0: L x = b; 1: L^T x = b.
template <typename T>
__device__ void warp_trsv(const T* __restrict__ L, int ldl, int n, T* b, int trans) {
  const int lane = threadIdx.x & 31;
  if (!trans) {
    for (int j = 0; j < n; ++j) {
      const T xj = b[j] / L[(long long)j * ldl + j];
      __syncwarp();
      if (lane == 0) b[j] = xj;
      for (int r = j + 1 + lane; r < n; r += 32) b[r] -= L[(long long)r * ldl + j] * xj;
      __syncwarp();
    }
  } else {
    for (int j = n - 1; j >= 0; --j) {
      const T xj = b[j] / L[(long long)j * ldl + j];
      __syncwarp();
      if (lane == 0) b[j] = xj;
      for (int r = lane; r < j; r += 32) b[r] -= L[(long long)j * ldl + r] * xj;
      __syncwarp();
    }
  }
}

// The small part of one paired Galerkin iteration for system r (one CTA each),
// with a- = L L^T and H = L^T a+ L:
//   z = L^-1 h-,  rhs = L^T h+ + s z,  (H - s^2) u~ = rhs,  u = L u~,
//   w = L^-T (z + s u~)          (h- absent: z = 0)
template <typename T>
__global__ void __launch_bounds__(512) k_paired_small(const T* __restrict__ Lg, const T* __restrict__ H,
                                                      int ld, int n, const T* __restrict__ hp,
                                                      const T* __restrict__ hm, const double* __restrict__ sh,
                                                      T* __restrict__ uc, T* __restrict__ wc) {
  extern __shared__ __align__(16) unsigned char ps_raw[];
  const int la = n + 2;
  T* A = reinterpret_cast<T*>(ps_raw);   // [n][n+2] augmented system
  T* z = A + (size_t)n * la;             // [n]
  T* hv = z + n;                         // [n]
  // FP32: a copy of L in shared memory (row stride n + 1, so that column walks
  // are free of bank conflicts); FP64 (too large): L read from global memory
  constexpr bool kLs = sizeof(T) == 4;
  if (kLs) {
    T* Ls = hv + n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, c = idx - r * n;
      Ls[r * (n + 1) + c] = Lg[(long long)r * ld + c];
    }
  }
  const T* L = kLs ? hv + n : Lg;
  const int ll = kLs ? n + 1 : ld;
  __shared__ int perm[kSmallMax];
  __shared__ T yv[kSmallMax];
  const int r = blockIdx.x;
  const T s = (T)sh[r];
  const T s2 = (T)(sh[r] * sh[r]);
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < n; i += nth) {
    z[i] = hm ? hm[(long long)r * n + i] : T(0);
    hv[i] = hp[(long long)r * n + i];
  }
  for (int idx = tid; idx < n * n; idx += nth) {
    int i = idx / n, j = idx - i * n;
    A[i * la + j] = T(0.5) * (H[(long long)i * ld + j] + H[(long long)j * ld + i]) - (i == j ? s2 : T(0));
  }
  __syncthreads();
  if (hm && tid < 32) warp_trsv<T>(L, ll, n, z, 0);
  __syncthreads();
  for (int i = tid; i < n; i += nth) {   // rhs_i = sum_q h+_q L[q][i] + s z_i
    T acc = s * z[i];
    for (int q = i; q < n; ++q) acc += hv[q] * L[(long long)q * ll + i];
    A[i * la + n] = acc;
  }
  __syncthreads();
  lu_solve_smem<T>(A, la, n, perm, yv);
  // u = L u~ ; z <- z + s u~
  for (int i = tid; i < n; i += nth) {
    T acc = T(0);
    for (int q = 0; q <= i; ++q) acc += L[(long long)i * ll + q] * A[q * la + n];
    uc[(long long)r * n + i] = acc;
    hv[i] = z[i] + s * A[i * la + n];
  }
  __syncthreads();
  if (tid < 32) warp_trsv<T>(L, ll, n, hv, 1);
  __syncthreads();
  for (int i = tid; i < n; i += nth) wc[(long long)r * n + i] = hv[i];
}

// ---- batched forms (one CTA per problem or per right-hand side), for many
// small independent solves advanced together

// Lowest k eigenpairs of the symmetric part of H (FP64 cyclic Jacobi in
// shared memory), ascending: lam[k], vec[k][n] (rows = eigenvectors).
__global__ void __launch_bounds__(512) k_beig(const BEig* __restrict__ d) {
  extern __shared__ double smb[];
  __shared__ int pp[kBatchSmall / 2 + 1], qq[kBatchSmall / 2 + 1];
  __shared__ double cc[kBatchSmall / 2 + 1], ss[kBatchSmall / 2 + 1];
  __shared__ unsigned smax;
  __shared__ double red[33];
  const BEig e = d[blockIdx.x];
  const int n = e.n;
  if (n <= 0) return;
  const int NP = (n + 1) & ~1, ld = NP + 1;
  double* A = smb;
  double* Q = smb + NP * ld;
  double f2 = 0.0;
  for (int idx = threadIdx.x; idx < NP * NP; idx += blockDim.x) {
    int r = idx / NP, c = idx - r * NP;
    double v = 0.0;
    if (r < n && c < n) v = 0.5 * (e.H[(long long)r * e.ld + c] + e.H[(long long)c * e.ld + r]);
    f2 += v * v;
    A[r * ld + c] = v;
    Q[r * ld + c] = (r == c) ? 1.0 : 0.0;
  }
  double frob = sqrt(block_sum(f2, red));
  jacobi_cta<double>(A, Q, n, ld, frob, 30, 1e-14, pp, qq, cc, ss, &smax);
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    int r = diag_rank(A, ld, n, t);
    if (r < e.k) {
      e.lam[r] = A[t * ld + t];
      for (int q = 0; q < n; ++q) e.vec[(long long)r * n + q] = Q[q * ld + t];
    }
  }
}

// y = (H - sigma I)^-1 b for one right-hand side per CTA (LU, partial pivoting).
__global__ void __launch_bounds__(512) k_blu(const BLu* __restrict__ d) {
  extern __shared__ __align__(16) unsigned char blu_raw[];
  double* A = reinterpret_cast<double*>(blu_raw);
  __shared__ int perm[kBatchSmall];
  __shared__ double yv[kBatchSmall];
  const BLu e = d[blockIdx.x];
  const int n = e.n;
  if (n <= 0) return;
  const int ld = n + 2;
  for (int idx = threadIdx.x; idx < n * (n + 1); idx += blockDim.x) {
    int i = idx / (n + 1), j = idx - i * (n + 1);
    double v;
    if (j < n) v = 0.5 * (e.H[(long long)i * e.ld + j] + e.H[(long long)j * e.ld + i]) - (i == j ? e.sigma : 0.0);
    else v = e.b[i];
    A[i * ld + j] = v;
  }
  __syncthreads();
  lu_solve_smem<double>(A, ld, n, perm, yv);
  for (int i = threadIdx.x; i < n; i += blockDim.x) e.y[i] = A[i * ld + n];
}

__global__ void __launch_bounds__(1024) k_bdrop(const BDrop* __restrict__ d, double drop2) {
  extern __shared__ double smd[];
  __shared__ int kj;
  __shared__ double dj;
  const BDrop e = d[blockIdx.x];
  if (e.nc <= 0) return;
  chol_drop_cta(e.G, e.nc, e.norm0sq, drop2, e.T, e.keep, smd, kj, dj);
}

void set_smem(const void* f, size_t bytes) {
  ensure_smem(f, bytes);
}

}  // namespace

void eig32(const double* H, int ldh, int n, float* lam32, float* vec32, cudaStream_t s) {
  TD_REQUIRE(n >= 1 && n <= kSmallMax, TDDFT_ERR_ARG, "eig32: size out of range");
  const int NP = (n + 1) & ~1;
  size_t smem = (size_t)2 * NP * (NP + 1) * sizeof(float);
  set_smem((const void*)k_eig32, smem);
  k_eig32<<<1, 1024, smem, s>>>(H, ldh, n, lam32, vec32);
  count_launch();
  TD_LAUNCH_CHECK();
}

void refine_lowest(const double* H, int ldh, int n, int k, const float* lam32, const float* vec32,
                   double* lam, double* vecs, double* scratch, int rounds, cudaStream_t s) {
  TD_REQUIRE(k >= 1 && k <= n && k <= kWantMax, TDDFT_ERR_ARG, "refine_lowest: bad k");
  double* Qk = scratch;
  double* Yk = scratch + (size_t)k * n;
  k_refine<<<k, 256, 0, s>>>(H, ldh, n, lam32, vec32, rounds, Qk, Yk);
  count_launch();
  TD_LAUNCH_CHECK();
  const int KP = (k + 1) & ~1;
  size_t smem = (size_t)2 * KP * (KP + 1) * sizeof(double);
  set_smem((const void*)k_orth_rr, smem);
  k_orth_rr<<<1, 1024, smem, s>>>(Qk, Yk, k, n, lam, vecs);
  count_launch();
  TD_LAUNCH_CHECK();
}

void shifted_solve(const double* H, int ldh, int n, const float* lam32, const float* vec32,
                   const double* sigma, int nr, const double* B, double* Y, int nref,
                   cudaStream_t s) {
  if (nr <= 0) return;
  k_shifted<<<nr, 256, 0, s>>>(H, ldh, n, lam32, vec32, sigma, B, Y, nref);
  count_launch();
  TD_LAUNCH_CHECK();
}

template <typename S>
void lu_shift_solve(const S* H, int ldh, int n, const double* sigma, int nr, const S* B, S* Y,
                    cudaStream_t s) {
  if (nr <= 0) return;
  TD_REQUIRE(n >= 1 && n <= kSmallMax, TDDFT_ERR_ARG, "lu_shift_solve: size out of range");
  size_t smem = (size_t)n * (n + 2) * sizeof(S);
  set_smem((const void*)k_lu_shift<S>, smem);
  k_lu_shift<S><<<nr, 512, smem, s>>>(H, ldh, n, sigma, B, Y);
  count_launch();
  TD_LAUNCH_CHECK();
}
template void lu_shift_solve<float>(const float*, int, int, const double*, int, const float*, float*,
                                    cudaStream_t);
template void lu_shift_solve<double>(const double*, int, int, const double*, int, const double*, double*,
                                     cudaStream_t);

template <typename S>
void paired_small_solve(const S* L, const S* H, int ld, int n, const S* hp, const S* hm, const double* sh,
                        int nr, S* uc, S* wc, cudaStream_t s) {
  if (nr <= 0) return;
  TD_REQUIRE(n >= 1 && n <= kSmallMax, TDDFT_ERR_ARG, "paired_small_solve: size out of range");
  size_t smem = ((size_t)n * (n + 2) + 2 * (size_t)n + (sizeof(S) == 4 ? (size_t)n * (n + 1) : 0)) * sizeof(S);
  set_smem((const void*)k_paired_small<S>, smem);
  k_paired_small<S><<<nr, 512, smem, s>>>(L, H, ld, n, hp, hm, sh, uc, wc);
  count_launch();
  TD_LAUNCH_CHECK();
}
template void paired_small_solve<float>(const float*, const float*, int, int, const float*, const float*,
                                        const double*, int, float*, float*, cudaStream_t);
template void paired_small_solve<double>(const double*, const double*, int, int, const double*,
                                         const double*, const double*, int, double*, double*, cudaStream_t);

template <typename S>
void cholesky(S* H, int ldh, int n, int* info, cudaStream_t s) {
  TD_REQUIRE(n >= 1 && n <= kSmallMax, TDDFT_ERR_ARG, "cholesky: size out of range");
  size_t smem = (size_t)n * (n + 1) * sizeof(S);
  set_smem((const void*)k_cholesky<S>, smem);
  k_cholesky<S><<<1, 1024, smem, s>>>(H, ldh, n, info);
  count_launch();
  TD_LAUNCH_CHECK();
}
template void cholesky<float>(float*, int, int, int*, cudaStream_t);

template <typename S>
void cholesky_border(S* L, int ld, int n0, int n, int* info, cudaStream_t s) {
  TD_REQUIRE(n >= 1 && n <= kSmallMax && n0 >= 0 && n0 <= n, TDDFT_ERR_ARG, "cholesky_border: bad sizes");
  const size_t smem = (size_t)n * n * sizeof(S);
  ensure_smem((const void*)k_chol_border<S>, smem);
  k_chol_border<S><<<1, 1024, smem, s>>>(L, ld, n0, n, info);
  count_launch();
  TD_LAUNCH_CHECK();
}
template void cholesky_border<float>(float*, int, int, int, int*, cudaStream_t);
template void cholesky_border<double>(double*, int, int, int, int*, cudaStream_t);
template void cholesky<double>(double*, int, int, int*, cudaStream_t);

template <typename S>
void trsv_rows(const S* L, int ldl, int n, S* B, int nr, int trans, cudaStream_t s) {
  if (nr <= 0) return;
  TD_REQUIRE(n <= kSmallMax, TDDFT_ERR_ARG, "trsv: size out of range");
  k_trsv<S><<<nr, 256, 0, s>>>(L, ldl, n, B, trans);
  count_launch();
  TD_LAUNCH_CHECK();
}
template void trsv_rows<float>(const float*, int, int, float*, int, int, cudaStream_t);
template void trsv_rows<double>(const double*, int, int, double*, int, int, cudaStream_t);

void batch_eig(const BEig* d, int nb, int nmax, cudaStream_t s) {
  if (nb <= 0) return;
  TD_REQUIRE(nmax >= 1 && nmax <= kBatchSmall, TDDFT_ERR_ARG, "batch_eig: size out of range");
  const int NP = (nmax + 1) & ~1;
  const size_t smem = (size_t)2 * NP * (NP + 1) * sizeof(double);
  set_smem((const void*)k_beig, smem);
  k_beig<<<nb, 512, smem, s>>>(d);
  count_launch();
  TD_LAUNCH_CHECK();
}

void batch_lu(const BLu* d, int nr, int nmax, cudaStream_t s) {
  if (nr <= 0) return;
  TD_REQUIRE(nmax >= 1 && nmax <= kBatchSmall, TDDFT_ERR_ARG, "batch_lu: size out of range");
  const size_t smem = (size_t)nmax * (nmax + 2) * sizeof(double);
  set_smem((const void*)k_blu, smem);
  k_blu<<<nr, 512, smem, s>>>(d);
  count_launch();
  TD_LAUNCH_CHECK();
}

void batch_chol_drop(const BDrop* d, int nb, int ncmax, double drop2, cudaStream_t s) {
  if (nb <= 0) return;
  TD_REQUIRE(ncmax >= 1 && ncmax <= kBatchSmall, TDDFT_ERR_ARG, "batch_chol_drop: size out of range");
  const size_t smem = (size_t)2 * ncmax * (ncmax + 1) * sizeof(double);
  set_smem((const void*)k_bdrop, smem);
  k_bdrop<<<nb, 1024, smem, s>>>(d, drop2);
  count_launch();
  TD_LAUNCH_CHECK();
}

void chol_drop(const double* G, int nc, const double* norm0sq, double drop2, double* T, int* keep,
               cudaStream_t s) {
  TD_REQUIRE(nc >= 1 && nc <= kDropMax, TDDFT_ERR_ARG, "chol_drop: too many candidates");
  size_t smem = (size_t)2 * nc * (nc + 1) * sizeof(double);
  set_smem((const void*)k_chol_drop, smem);
  k_chol_drop<<<1, 256, smem, s>>>(G, nc, norm0sq, drop2, T, keep);
  count_launch();
  TD_LAUNCH_CHECK();
}

}  // namespace tddft
