// Preconditioned Davidson drivers (Sec. 2.1) for the TDA eigenproblem (Eq. TDA),
// the Casida eigenproblem (Eq. Casida) and the polarizability linear systems
// (Eq. TDDFT_polar), with the diagonal and the rid preconditioners (Sec. 3).
//
// Everything the algorithm computes stays on the device; per iteration the host
// reads back only the Ritz values and residual norms (a few hundred bytes) to
// decide convergence, locking and the next launch sizes.  Each step maps to
// kernels as follows:
//   Eq. 1   projected matrix, new columns only     split-K FP64 GEMM + sym_fill
//   Eq. 2   subspace eigenproblem                  eig32 (FP32 Jacobi) + FP64 refinement
//   Eq. 3   Ritz vectors X = V x, A X = (A V) x    FP64 GEMM
//   Eq. residual                                    resid kernels + row norms
//   Eq. precondition                                diag: element-wise; rid: inner
//                                                   Galerkin solve with the ris operator
//   Gram-Schmidt + append                           block Gram-Schmidt (two passes of
//                                                   projection + pivot-dropping Cholesky)
// The Casida problem uses one subspace V for X+Y and X-Y with a+ = V^T(A+B)V,
// a- = V^T(A-B)V, solved in the symmetric form L^T a+ L y = Omega^2 y (a- = L L^T).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <functional>
#include <numeric>

#include "ctx.cuh"
#include "skinny.cuh"
#include "small.cuh"
#include "tc_gemm.cuh"
#include "vecops.cuh"

namespace tddft {

namespace {

using Clock = std::chrono::steady_clock;
inline double since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

constexpr double kDrop2 = 1e-16;   // drop a direction below 1e-8 of its norm

// TDDFT_TRACE=1 prints one line per outer iteration to stderr; TDDFT_TRACE=2
// also times solver phases (stream-synchronised, so only for diagnostics).
int trace_level() {
  static int v = -1;
  if (v < 0) { const char* e = getenv("TDDFT_TRACE"); v = (e && e[0] >= '1' && e[0] <= '9') ? e[0] - '0' : 0; }
  return v;
}
bool trace_on() { return trace_level() >= 1; }

enum Phase { PH_MV = 0, PH_RIS, PH_ORTH, PH_PROJ, PH_SMALL, PH_VEC, PH_ORTH_IN, PH_PROJ_IN, PH_SMALL_IN,
             PH_VEC_IN, PH_EIG, PH_CHOL, PH_SMM, PH_LU, PH_TRSV, PH_N };
const char* kPhaseNames[PH_N] = {"exact_mv", "ris_mv", "orth", "proj+factor", "small", "vec", "orth_in",
                                 "proj+factor_in", "small_in", "vec_in", "[eig32]", "[chol]", "[small_mm]",
                                 "[lu]", "[trsv]"};
thread_local double g_phase[PH_N];
thread_local int g_inner = 0;   // > 0 inside the ris inner solves and guesses
struct InnerScope {
  InnerScope() { ++g_inner; }
  ~InnerScope() { --g_inner; }
};
struct ScopedPhase {
  int id; cudaStream_t s; Clock::time_point t0; bool on;
  ScopedPhase(int i, cudaStream_t st) : id(i), s(st), on(trace_level() >= 2) {
    if (i >= PH_EIG && trace_level() < 3) on = false;
    if (g_inner > 0 && i >= PH_ORTH && i <= PH_VEC) id = i + (PH_ORTH_IN - PH_ORTH);
    if (on) { cudaStreamSynchronize(s); t0 = Clock::now(); }
  }
  void stop() {
    if (on) { cudaStreamSynchronize(s); g_phase[id] += since(t0); on = false; }
  }
  ~ScopedPhase() { stop(); }
};
void phase_report(const char* what) {
  if (trace_level() < 2) return;
  fprintf(stderr, "[tddft] phases %s:", what);
  for (int i = 0; i < PH_N; ++i) fprintf(stderr, " %s=%.3fs", kPhaseNames[i], g_phase[i]);
  fprintf(stderr, "\n");
  for (int i = 0; i < PH_N; ++i) g_phase[i] = 0.0;
}
void trace(const char* what, int it, int N, const std::vector<double>& om, const std::vector<double>& rr) {
  if (!trace_on()) return;
  double m = 0.0;
  for (double r : rr) m = std::max(m, r);
  fprintf(stderr, "[tddft] %s it=%d N=%d max|r|=%.3e omega0=%.8f\n", what, it, N, m, om.empty() ? 0.0 : om[0]);
}

// One line per certification gate: the loop's and the recomputed residuals, root by root.
void trace_gate(const char* what, int it, const std::vector<double>& rr, const std::vector<double>& cr) {
  if (!trace_on()) return;
  double ml = 0.0, mc = 0.0, md = 0.0;
  for (size_t j = 0; j < cr.size() && j < rr.size(); ++j) {
    ml = std::max(ml, rr[j]);
    mc = std::max(mc, cr[j]);
    md = std::max(md, std::fabs(cr[j] - rr[j]));
  }
  fprintf(stderr, "[tddft] %s gate it=%d loop max %.4e recomputed max %.4e max |diff| %.3e\n", what, it, ml, mc, md);
}

template <typename T>
std::vector<T> d2h(const T* p, size_t n, cudaStream_t s) {
  std::vector<T> h(n);
  if (n) {
    TD_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    TD_CUDA(cudaStreamSynchronize(s));
  }
  return h;
}

template <typename T>
void h2d(T* p, const std::vector<T>& h, cudaStream_t s) {
  if (!h.empty()) TD_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

struct Counters {
  long long mv = 0;      // exact operator vectors
  long long ris_mv = 0;  // ris operator vectors
  double t_mv = 0.0, t_pre = 0.0, t_guess = 0.0, t_cert = 0.0;
  int restarts = 0;
};

template <typename T> constexpr DType dt_of();
template <> constexpr DType dt_of<double>() { return DType::F64; }
template <> constexpr DType dt_of<float>() { return DType::F32; }

// Operators and preconditioners over vectors stored as T (double or float).
template <typename T> using TdaOpT = std::function<void(const T* X, int m, T* out)>;
template <typename T> using PairOpT = std::function<void(const T* X, int m, T* P, T* M)>;
// TDA preconditioner: (R [nu][ov], shifts dev/host) -> out [nu][ov]
template <typename T>
using TdaPreT = std::function<void(const T* R, const double* sh, const std::vector<double>& shh,
                                   int nu, T* out)>;
// paired preconditioner: (g+ , g-, shifts) -> (u, w) each [nu][ov]
template <typename T>
using PairPreT = std::function<void(const T* gp, const T* gm, const double* sh,
                                    const std::vector<double>& shh, int nu, T* u, T* w)>;
using TdaOp = TdaOpT<double>;
using PairOp = PairOpT<double>;
using TdaPre = TdaPreT<double>;
using PairPre = PairPreT<double>;

// ---------------------------------------------------------------------------
// Subspace helpers.  Vectors are FP64 (outer Davidson, PLAIN) or FP32 (MIXED
// inner solves); every small matrix is FP64.

// G[i][j] = A[i] . B[j]  (rows of length ov), G (type S) row stride ldg; accumulated
// in the vectors' precision
template <typename T, typename S>
void gram(const T* A, int ka, const T* B, int kb, int ov, S* G, int ldg, cudaStream_t s) {
  sk_gram<T>(A, ov, ka, B, ov, kb, ov, G, dt_of<S>(), ldg, 1.0, 0.0, s);
}

// a[r][col0 + j] = V[r] . Wn[j]  for r < N, j < k  (a of type S)
template <typename T, typename S>
void proj_cols(const T* V, int N, const T* Wn, int k, int ov, S* a, int ld, int col0, cudaStream_t s) {
  gram<T, S>(V, N, Wn, k, ov, a + col0, ld, s);
}

// out[j] = alpha * sum_r coef[j][r] V[r] + beta * out[j]   (coef compact [k][N], type S)
template <typename T, typename S>
void combo(const S* coef, int k, int N, const T* V, int ov, T* out, double alpha, double beta,
           cudaStream_t s) {
  sk_combo<T>(coef, dt_of<S>(), N, 1, k, N, V, ov, ov, out, ov, alpha, beta, s);
}

// small dense product C = A * B with general strides (type S)
template <typename S>
void small_mm(int M, int N, int K, const S* A, long long sam, long long sak, const S* B,
              long long sbk, long long sbn, S* C, long long scm, cudaStream_t s) {
  GemmDesc g;
  g.acc64 = sizeof(S) == 8;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.ta = dt_of<S>(); g.sam = sam; g.sak = sak;
  g.B = B; g.tb = dt_of<S>(); g.sbk = sbk; g.sbn = sbn;
  g.C = C; g.tc = dt_of<S>(); g.scm = scm; g.scn = 1;
  gemm(g, s);
}

// Two passes of block Gram-Schmidt of the candidate rows `cand` [nc][ov]
// against V (N orthonormal rows) and each other; the result overwrites cand and
// keep[j] (device) flags the survivors (dropped rows are zero).
template <typename T>
void orth_block(const T* V, int N, T* cand, int nc, int ov, int* keep, cudaStream_t s) {
  TD_REQUIRE(nc <= 112, TDDFT_ERR_ARG, "too many new directions in one iteration");
  DevBuf n0(nc * 8, s), G((size_t)nc * nc * 8, s), Tm((size_t)nc * nc * 8, s);
  DevBuf tmp((size_t)nc * ov * sizeof(T), s);
  DevBuf coef(N > 0 ? (size_t)N * nc * 8 : 8, s);
  row_sumsq<T>(cand, ov, nc, ov, n0.as<double>(), s);
  T* cur = cand;
  T* oth = tmp.as<T>();
  for (int pass = 0; pass < 2; ++pass) {
    if (N > 0) {
      gram<T, double>(V, N, cur, nc, ov, coef.as<double>(), nc, s);   // coef[r][j] = V[r].cur[j]
      // cur[j] -= sum_r coef[r][j] V[r]
      sk_combo<T>(coef.p, DType::F64, 1, nc, nc, N, V, ov, ov, cur, ov, -1.0, 1.0, s);
    }
    gram<T, double>(cur, nc, cur, nc, ov, G.as<double>(), nc, s);
    chol_drop(G.as<double>(), nc, pass == 0 ? n0.as<double>() : nullptr, kDrop2, Tm.as<double>(), keep, s);
    combo<T, double>(Tm.as<double>(), nc, nc, cur, ov, oth, 1.0, 0.0, s);
    std::swap(cur, oth);
  }
  // two swaps: the result is back in cand
}

// Orthonormalise `cand` against V and append the survivors at V[N...].
// Returns their number (never more than ov - N).
template <typename T>
int orth_append(T* V, int N, T* cand, int nc, int ov, cudaStream_t s) {
  if (nc <= 0) return 0;
  ScopedPhase ph(PH_ORTH, s);
  DevBuf keep(nc * 4, s);
  orth_block<T>(V, N, cand, nc, ov, keep.as<int>(), s);
  std::vector<int> kh = d2h(keep.as<int>(), nc, s);
  std::vector<int> idx;
  for (int j = 0; j < nc && N + (int)idx.size() < ov; ++j)   // never beyond the space's dimension
    if (kh[j]) idx.push_back(j);
  if (!idx.empty()) {
    DevBuf di(idx.size() * 4, s);
    h2d(di.as<int>(), idx, s);
    gather_rows<T>(cand, di.as<int>(), (int)idx.size(), ov, V + (size_t)N * ov, s);
  }
  return (int)idx.size();
}

// The same without a host round trip: the survivors are compacted, in order,
// into V[N...] (V must have room for nc rows there) and their number is left in
// count[0] on the device; the caller caps it at ov - N when it reads it.
template <typename T>
void orth_append_async(T* V, int N, T* cand, int nc, int ov, int* keep, int* count, cudaStream_t s) {
  if (nc <= 0) { TD_CUDA(cudaMemsetAsync(count, 0, sizeof(int), s)); return; }
  ScopedPhase ph(PH_ORTH, s);
  orth_block<T>(V, N, cand, nc, ov, keep, s);
  compact_rows<T>(cand, keep, nc, ov, V + (size_t)N * ov, count, s);
}

// Orthonormalise `cand` against V (N rows) and each other and compact the
// survivors, in order, into `out` without appending them; returns their number
// (at most ov - N).  Used before a thick restart, so that the new directions
// are free of the whole subspace that produced them.
template <typename T>
int orth_compact(const T* V, int N, T* cand, int nc, int ov, T* out, cudaStream_t s) {
  if (nc <= 0) return 0;
  ScopedPhase ph(PH_ORTH, s);
  DevBuf keep(nc * 4, s);
  orth_block<T>(V, N, cand, nc, ov, keep.as<int>(), s);
  std::vector<int> kh = d2h(keep.as<int>(), nc, s);
  std::vector<int> idx;
  for (int j = 0; j < nc && N + (int)idx.size() < ov; ++j)
    if (kh[j]) idx.push_back(j);
  if (!idx.empty()) {
    DevBuf di(idx.size() * 4, s);
    h2d(di.as<int>(), idx, s);
    gather_rows<T>(cand, di.as<int>(), (int)idx.size(), ov, out, s);
  }
  return (int)idx.size();
}

void check_finite_host(const std::vector<double>& v, const char* what) {
  for (double x : v)
    if (!std::isfinite(x))
      throw Error(TDDFT_ERR_INDEFINITE, std::string("non-finite values in ") + what);
}

std::vector<double> sqrt_all(const std::vector<double>& v) {
  std::vector<double> r(v.size());
  for (size_t i = 0; i < v.size(); ++i) r[i] = std::sqrt(v[i]);
  return r;
}

// ---------------------------------------------------------------------------
// TDA Davidson (Sec. 2.1) on a generic symmetric operator.

struct TdaOut {
  std::vector<double> omega, resid;
  DevBuf X;     // [k][ov] Ritz vectors
  int n_iter = 0;
  bool converged = false;
  double cert = -1.0;   // largest recomputed residual (when a gate was given)
};

// Certification gate: residual norms of the k Ritz pairs recomputed from fresh
// products of the Ritz vectors (TDA: X [k][ov], omega; Casida: U, W, Omega).
using TdaCert = std::function<std::vector<double>(const double* X, const std::vector<double>& om, int k)>;
using RpaCert = std::function<std::vector<double>(const double* U, const double* W, const std::vector<double>& om,
                                                  int k)>;

// With a gate, the solve converges only when the recomputed residuals are
// below tol as well; where one is not (the fresh products round differently
// from the accumulated A V), the loop's threshold is halved and it continues.
TdaOut davidson_tda(int ov, const TdaOp& A, const TdaPre& pre, double* guess, int ng, int k,
                    double tol, int max_iter, int cap, int rounds, Counters& cnt, bool exact_op,
                    cudaStream_t s, const TdaCert* cert = nullptr) {
  TdaOut o;
  if (!exact_op) ++g_inner;
  struct Leave { bool on; ~Leave() { if (on) --g_inner; } } leave{!exact_op};
  k = std::min(k, ov);
  cap = std::min(cap, kSmallMax);
  TD_REQUIRE(k >= 1 && k <= kWantMax, TDDFT_ERR_ARG, "n_states out of range");
  TD_REQUIRE(cap >= 2 * k, TDDFT_ERR_ARG, "max_subspace must be at least 2*n_states");
  DevBuf V((size_t)cap * ov * 8, s), W((size_t)cap * ov * 8, s);
  DevBuf a((size_t)cap * cap * 8, s), lam32(cap * 4, s), vec32((size_t)cap * cap * 4, s);
  DevBuf lam(k * 8, s), x((size_t)k * cap * 8, s), scr((size_t)2 * k * cap * 8, s);
  DevBuf X((size_t)k * ov * 8, s), AX((size_t)k * ov * 8, s), R((size_t)k * ov * 8, s);
  DevBuf rn(k * 8, s), Ru((size_t)k * ov * 8, s), omu(k * 8, s), cand((size_t)k * ov * 8, s);
  DevBuf iu(k * 4, s), Xprev((size_t)k * ov * 8, s), tmpk((size_t)k * ov * 8, s);
  bool have_prev = false;
  double* Vp = V.as<double>();
  double* Wp = W.as<double>();

  int N = orth_append(Vp, 0, guess, std::min(ng, cap), ov, s);
  TD_REQUIRE(N >= 1, TDDFT_ERR_ARG, "initial guess is empty");
  auto mv = [&](int r0, int m) {
    auto t0 = Clock::now();
    ScopedPhase ph(exact_op ? PH_MV : PH_RIS, s);
    A(Vp + (size_t)r0 * ov, m, Wp + (size_t)r0 * ov);
    TD_CUDA(cudaStreamSynchronize(s));
    if (exact_op) { cnt.mv += m; cnt.t_mv += since(t0); } else { cnt.ris_mv += m; }
  };
  mv(0, N);
  int n_proj = 0;   // leading vectors whose projections are already in `a`
  std::vector<double> om(k), rr(k);
  int kk = std::min(k, N);
  double tol_loop = tol;
  for (int it = 1; it <= max_iter; ++it) {
    o.n_iter = it;
    {
      ScopedPhase ph(PH_PROJ, s);
      proj_cols(Vp, N, Wp + (size_t)n_proj * ov, N - n_proj, ov, a.as<double>(), cap, n_proj, s);  // Eq. 1
      sym_fill(a.as<double>(), cap, n_proj, N - n_proj, s);
    }
    n_proj = N;
    kk = std::min(k, N);
    ScopedPhase ph_small(PH_SMALL, s);
    {
      ScopedPhase f(trace_level() >= 3 ? PH_EIG : PH_N - 1, s);
      eig32(a.as<double>(), cap, N, lam32.as<float>(), vec32.as<float>(), s);             // Eq. 2
    }
    refine_lowest(a.as<double>(), cap, N, kk, lam32.as<float>(), vec32.as<float>(), lam.as<double>(),
                  x.as<double>(), scr.as<double>(), rounds, s);
    ph_small.stop();
    ScopedPhase ph_vec(PH_VEC, s);
    combo<double, double>(x.as<double>(), kk, N, Vp, ov, X.as<double>(), 1.0, 0.0, s);    // Eq. 3
    combo<double, double>(x.as<double>(), kk, N, Wp, ov, AX.as<double>(), 1.0, 0.0, s);
    resid_tda(X.as<double>(), AX.as<double>(), lam.as<double>(), kk, ov, R.as<double>(), s);  // Eq. residual
    row_sumsq(R.as<double>(), ov, kk, ov, rn.as<double>(), s);
    om = d2h(lam.as<double>(), kk, s);
    rr = sqrt_all(d2h(rn.as<double>(), kk, s));
    ph_vec.stop();
    check_finite_host(om, "Ritz values");
    check_finite_host(rr, "residual norms");
    trace(exact_op ? "tda" : "tda-guess", it, N, om, rr);
    std::vector<int> todo;
    for (int j = 0; j < kk; ++j)
      if (!(rr[j] < tol_loop)) todo.push_back(j);
    if (todo.empty() && kk == k) {
      if (!cert) { o.converged = true; break; }
      const std::vector<double> cr = (*cert)(X.as<double>(), om, kk);
      trace_gate("tda", it, rr, cr);
      o.cert = 0.0;
      for (int j = 0; j < kk; ++j) {
        o.cert = std::max(o.cert, cr[j]);
        if (!(cr[j] < tol)) todo.push_back(j);
      }
      if (todo.empty()) { o.converged = true; break; }
      tol_loop *= 0.5;
    }
    if (it == max_iter) break;
    const int nu = (int)todo.size();
    std::vector<double> omh(nu);
    for (int j = 0; j < nu; ++j) omh[j] = om[todo[j]];
    h2d(iu.as<int>(), todo, s);
    gather_rows(R.as<double>(), iu.as<int>(), nu, ov, Ru.as<double>(), s);
    h2d(omu.as<double>(), omh, s);
    auto tp = Clock::now();
    pre(Ru.as<double>(), omu.as<double>(), omh, nu, cand.as<double>());                   // Eq. precondition
    TD_CUDA(cudaStreamSynchronize(s));
    cnt.t_pre += since(tp);
    double* cnew = cand.as<double>();
    int nnew = nu;
    DevBuf cfree;
    if (N + nu > cap) {
      // the new directions, orthonormalised against the full subspace first
      cfree = DevBuf((size_t)nu * ov * 8, s);
      nnew = orth_compact<double>(Vp, N, cand.as<double>(), nu, ov, cfree.as<double>(), s);
      if (nnew == 0) break;
      cnew = cfree.as<double>();
      // thick restart: current Ritz vectors + those of the previous iteration,
      // the latter only where they and the new directions fit under the cap
      TD_CUDA(cudaMemcpyAsync(Vp, X.p, (size_t)kk * ov * 8, cudaMemcpyDeviceToDevice, s));
      TD_CUDA(cudaMemcpyAsync(Wp, AX.p, (size_t)kk * ov * 8, cudaMemcpyDeviceToDevice, s));
      N = kk;
      if (have_prev && 2 * kk + nnew <= cap) {
        TD_CUDA(cudaMemcpyAsync(tmpk.p, Xprev.p, (size_t)kk * ov * 8, cudaMemcpyDeviceToDevice, s));
        int ne = orth_append(Vp, N, tmpk.as<double>(), kk, ov, s);
        mv(N, ne);
        N += ne;
      }
      n_proj = 0;
      cnt.restarts++;
    }
    TD_CUDA(cudaMemcpyAsync(Xprev.p, X.p, (size_t)kk * ov * 8, cudaMemcpyDeviceToDevice, s));
    have_prev = true;
    int nacc = orth_append(Vp, N, cnew, std::min(nnew, cap - N), ov, s);
    if (nacc == 0) break;
    mv(N, nacc);
    N += nacc;
  }
  o.omega = om;
  o.resid = rr;
  o.X = std::move(X);
  return o;
}

// ---------------------------------------------------------------------------
// Paired subspace algebra shared by the Casida eigenproblem and the paired
// linear systems: a+ = V^T P, a- = V^T M, a- = L L^T, H = L^T a+ L.  The small
// matrices have the vectors' type T: FP64 in the outer solves, FP32 in the
// MIXED inner solves (which stop at a relative residual of about 1e-2).

template <typename T, typename S = T>
struct PairedSpace {
  int ov, cap;
  cudaStream_t s;
  DevBuf V, P, M, ap, am, L, tmp, H, lam32, vec32;
  int N = 0, n_old = 0, n_new = 0;
  DevBuf info;
  // `slack` extra rows of V receive candidate directions before they are accepted
  PairedSpace(int ov_, int cap_, cudaStream_t s_, int slack = 0) : ov(ov_), cap(cap_), s(s_) {
    V = DevBuf((size_t)(cap + slack) * ov * sizeof(T), s);
    P = DevBuf((size_t)cap * ov * sizeof(T), s);
    M = DevBuf((size_t)cap * ov * sizeof(T), s);
    ap = DevBuf((size_t)cap * cap * sizeof(S), s);
    am = DevBuf((size_t)cap * cap * sizeof(S), s);
    L = DevBuf((size_t)cap * cap * sizeof(S), s);
    tmp = DevBuf((size_t)cap * cap * sizeof(S), s);
    H = DevBuf((size_t)cap * cap * sizeof(S), s);
    lam32 = DevBuf(cap * 4, s);
    vec32 = DevBuf((size_t)cap * cap * 4, s);
    info = DevBuf(4, s);
  }
  T* v() { return V.as<T>(); }
  T* p() { return P.as<T>(); }
  T* m() { return M.as<T>(); }
  // project the new vectors, factor a- = L L^T, form H = L^T a+ L (and, for the
  // eigenproblem, its FP32 decomposition)
  void update(bool eig) {
    ScopedPhase ph(PH_PROJ, s);
    proj_cols<T, S>(v(), N, p() + (size_t)n_old * ov, n_new, ov, ap.as<S>(), cap, n_old, s);
    proj_cols<T, S>(v(), N, m() + (size_t)n_old * ov, n_new, ov, am.as<S>(), cap, n_old, s);
    sym_fill<S>(ap.as<S>(), cap, n_old, n_new, s);
    sym_fill<S>(am.as<S>(), cap, n_old, n_new, s);
    // a- = L L^T: the leading n_old rows of L are kept (the basis grows by
    // bordering); the new rows of a- are copied in and factored
    TD_CUDA(cudaMemcpy2DAsync(L.as<S>() + (size_t)n_old * cap, cap * sizeof(S),
                              am.as<S>() + (size_t)n_old * cap, cap * sizeof(S), N * sizeof(S), n_new,
                              cudaMemcpyDeviceToDevice, s));
    {
      ScopedPhase f(trace_level() >= 3 ? PH_CHOL : PH_N - 1, s);
      cholesky_border<S>(L.as<S>(), cap, n_old, N, info.as<int>(), s);
    }
    {
      ScopedPhase f(trace_level() >= 3 ? PH_SMM : PH_N - 1, s);
      // tmp = a+ L ; H = L^T tmp
      small_mm<S>(N, N, N, ap.as<S>(), cap, 1, L.as<S>(), cap, 1, tmp.as<S>(), cap, s);
      small_mm<S>(N, N, N, L.as<S>(), 1, cap, tmp.as<S>(), cap, 1, H.as<S>(), cap, s);
    }
    if constexpr (sizeof(S) == 8) {
      if (eig) {
        ScopedPhase f(trace_level() >= 3 ? PH_EIG : PH_N - 1, s);
        eig32(H.as<double>(), cap, N, lam32.as<float>(), vec32.as<float>(), s);
      }
    } else {
      TD_REQUIRE(!eig, TDDFT_ERR_ARG, "FP32 paired space: no eigensolver");
    }
    n_old = N;
    n_new = 0;
  }
  void check_definite() {
    int inf = d2h(info.as<int>(), 1, s)[0];
    if (inf != 0)
      throw Error(TDDFT_ERR_INDEFINITE, "projected A-B is not positive definite (pivot " +
                                            std::to_string(inf - 1) + ")");
  }
};

// ---------------------------------------------------------------------------
// Paired Galerkin linear solve (Eq. TDDFT_polar, and the paired form of
// Eq. precondition):  T+ u - s w = g+,  T- w - s u = g-  for nr right-hand
// sides in one shared subspace.

struct PairedLinOut {
  int n_iter = 0;
  bool converged = false;
  std::vector<double> resid;
  double cert = -1.0;   // largest recomputed relative residual (when a gate was given)
};

// Certification gate of the paired linear systems: the relative residuals of
// the nr solutions (U, W) recomputed from fresh products.
template <typename T>
using LinCert = std::function<std::vector<double>(const T* U, const T* W)>;

// The small shifted systems are solved by LU per shift in the vectors' type:
// FP64 for the outer polarizability and PLAIN solves, FP32 for the MIXED inner
// solves.
template <typename T, typename S = T>
PairedLinOut paired_linear(int ov, const PairOpT<T>& op, const PairPreT<T>& pre, const T* gp,
                           const T* gm, const std::vector<double>& shifts, int nr, T* init, int ni,
                           double tol, int max_iter, int cap, bool exact_op,
                           Counters& cnt, T* Uout, T* Wout, cudaStream_t s,
                           const LinCert<T>* cert = nullptr) {
  PairedLinOut o;
  double tol_loop = tol;
  if (!exact_op) ++g_inner;
  struct Leave { bool on; ~Leave() { if (on) --g_inner; } } leave{!exact_op};
  cap = std::min(cap, kSmallMax);
  constexpr size_t es = sizeof(T);
  // Inner solves (ris operator) select, precondition and orthonormalise the new
  // directions on the device and read back one status block per iteration.
  const bool dev_select = !exact_op;
  PairedSpace<T, S> sp(ov, cap, s, dev_select ? 2 * nr : 0);
  DevBuf sh(nr * 8, s), sig2(nr * 8, s);
  std::vector<double> s2(nr);
  for (int r = 0; r < nr; ++r) s2[r] = shifts[r] * shifts[r];
  h2d(sh.as<double>(), shifts, s);
  h2d(sig2.as<double>(), s2, s);
  // h+ and h- (and u, w coefficients) share one buffer so that, when g- follows
  // g+ in memory, one Gram product forms both
  DevBuf hpm((size_t)2 * nr * cap * sizeof(S), s), ucw((size_t)2 * nr * cap * sizeof(S), s);
  DevBuf Rp((size_t)nr * ov * es, s), Rm((size_t)nr * ov * es, s), PU((size_t)nr * ov * es, s),
      MW((size_t)nr * ov * es, s);
  DevBuf gn(nr * 8, s), gn2(nr * 8, s), rn1(nr * 8, s), rn2(nr * 8, s);
  DevBuf iu(nr * 4, s), shu(nr * 8, s), gpu_(((size_t)nr) * ov * es, s), gmu((size_t)nr * ov * es, s);
  DevBuf cand((size_t)2 * nr * ov * es, s);
  DevBuf Uprev, Wprev;
  bool have_prev = false;
  if (exact_op) {
    Uprev = DevBuf((size_t)nr * ov * es, s);
    Wprev = DevBuf((size_t)nr * ov * es, s);
  }
  row_sumsq<T>(gp, ov, nr, ov, gn.as<double>(), s);
  std::vector<double> gnh = d2h(gn.as<double>(), nr, s);
  if (gm) {
    row_sumsq<T>(gm, ov, nr, ov, gn2.as<double>(), s);
    std::vector<double> t = d2h(gn2.as<double>(), nr, s);
    for (int r = 0; r < nr; ++r) gnh[r] += t[r];
  }
  for (auto& v : gnh) v = std::sqrt(v);
  // status block read once per iteration: rn1[nr], rn2[nr] (doubles), then the
  // Cholesky info and the number of accepted directions (ints)
  DevBuf stat((size_t)2 * nr * 8 + 8, s), gdev(nr * 8, s), keep(2 * nr * 4, s);
  double* rn1p = dev_select ? stat.as<double>() : rn1.as<double>();
  double* rn2p = dev_select ? stat.as<double>() + nr : rn2.as<double>();
  int* st_info = reinterpret_cast<int*>(stat.as<double>() + 2 * nr);
  int* st_count = st_info + 1;
  if (dev_select) {
    std::vector<double> g1(nr);
    for (int r = 0; r < nr; ++r) g1[r] = gnh[r] > 0 ? gnh[r] : 1.0;
    h2d(gdev.as<double>(), g1, s);
  }

  sp.N = orth_append<T>(sp.v(), 0, init, std::min(ni, cap), ov, s);
  TD_REQUIRE(sp.N >= 1, TDDFT_ERR_ARG, "paired solve: empty initial subspace");
  auto mv = [&](int r0, int m) {
    auto t0 = Clock::now();
    ScopedPhase ph(exact_op ? PH_MV : PH_RIS, s);
    op(sp.v() + (size_t)r0 * ov, m, sp.p() + (size_t)r0 * ov, sp.m() + (size_t)r0 * ov);
    if (exact_op) {
      TD_CUDA(cudaStreamSynchronize(s));
      cnt.mv += m;
      cnt.t_mv += since(t0);
    } else {
      cnt.ris_mv += m;
    }
  };
  mv(0, sp.N);
  sp.n_old = 0;
  sp.n_new = sp.N;
  std::vector<double> rr(nr, 0.0);
  for (int it = 1; it <= max_iter; ++it) {
    o.n_iter = it;
    sp.update(false);
    if (!dev_select) sp.check_definite();
    const int N = sp.N;
    S* Lp = sp.L.template as<S>();
    ScopedPhase ph_small(PH_SMALL, s);
    // h+ = V g+ , h- = V g-   ([nr][N] each, h- right after h+)
    S* hp = hpm.as<S>();
    S* hm = hp + (size_t)nr * N;
    if (gm == gp + (size_t)nr * ov) {
      gram<T, S>(gp, 2 * nr, sp.v(), N, ov, hp, N, s);
    } else {
      gram<T, S>(gp, nr, sp.v(), N, ov, hp, N, s);
      if (gm) gram<T, S>(gm, nr, sp.v(), N, ov, hm, N, s);
    }
    // per system: z- = L^-1 h-, (H - s^2) u~ = L^T h+ + s z-, u = L u~, w = L^-T (z- + s u~)
    S* uc = ucw.as<S>();
    S* wc = uc + (size_t)nr * N;
    {
      ScopedPhase f(trace_level() >= 3 ? PH_LU : PH_N - 1, s);
      paired_small_solve<S>(Lp, sp.H.template as<S>(), cap, N, hp, gm ? hm : nullptr, sh.as<double>(), nr,
                            uc, wc, s);
    }
    ph_small.stop();
    ScopedPhase ph_vec(PH_VEC, s);
    if (Wout == Uout + (size_t)nr * ov) {
      combo<T, S>(uc, 2 * nr, N, sp.v(), ov, Uout, 1.0, 0.0, s);
    } else {
      combo<T, S>(uc, nr, N, sp.v(), ov, Uout, 1.0, 0.0, s);
      combo<T, S>(wc, nr, N, sp.v(), ov, Wout, 1.0, 0.0, s);
    }
    combo<T, S>(uc, nr, N, sp.p(), ov, PU.as<T>(), 1.0, 0.0, s);
    combo<T, S>(wc, nr, N, sp.m(), ov, MW.as<T>(), 1.0, 0.0, s);
    resid_paired<T>(Uout, Wout, PU.as<T>(), MW.as<T>(), sh.as<double>(), gp, gm, nr, ov,
                    Rp.as<T>(), Rm.as<T>(), s);
    row_sumsq<T>(Rp.as<T>(), ov, nr, ov, rn1p, s);
    row_sumsq<T>(Rm.as<T>(), ov, nr, ov, rn2p, s);
    std::vector<double> a1, a2;
    int dev_count = 0;
    if (dev_select) {
      // every system's new directions, the converged ones zeroed (and so dropped)
      ph_vec.stop();
      pre(Rp.as<T>(), Rm.as<T>(), sh.as<double>(), shifts, nr, cand.as<T>(), cand.as<T>() + (size_t)nr * ov);
      zero_converged<T>(cand.as<T>(), 2 * nr, nr, ov, rn1p, rn2p, gdev.as<double>(), tol, s);
      orth_append_async<T>(sp.v(), N, cand.as<T>(), 2 * nr, ov, keep.as<int>(), st_count, s);
      TD_CUDA(cudaMemcpyAsync(st_info, sp.info.p, sizeof(int), cudaMemcpyDeviceToDevice, s));
      std::vector<double> blk = d2h(stat.as<double>(), (size_t)2 * nr + 1, s);
      int ints[2];
      std::memcpy(ints, &blk[2 * nr], sizeof(ints));
      if (ints[0] != 0)
        throw Error(TDDFT_ERR_INDEFINITE, "projected A-B is not positive definite (pivot " +
                                              std::to_string(ints[0] - 1) + ")");
      dev_count = ints[1];
      a1.assign(blk.begin(), blk.begin() + nr);
      a2.assign(blk.begin() + nr, blk.begin() + 2 * nr);
    } else {
      a1 = d2h(rn1p, nr, s);
      a2 = d2h(rn2p, nr, s);
      ph_vec.stop();
    }
    std::vector<int> todo;
    for (int r = 0; r < nr; ++r) {
      rr[r] = std::sqrt(a1[r] + a2[r]) / (gnh[r] > 0 ? gnh[r] : 1.0);
      if (!(rr[r] <= tol_loop)) todo.push_back(r);
    }
    check_finite_host(rr, "linear-system residuals");
    if (exact_op) trace("polar", it, sp.N, std::vector<double>(), rr);
    if (todo.empty()) {
      if (!cert) { o.converged = true; break; }
      // the gate of davidson_tda
      const std::vector<double> cr = (*cert)(Uout, Wout);
      trace_gate("polar", it, rr, cr);
      o.cert = 0.0;
      for (int r = 0; r < nr; ++r) {
        o.cert = std::max(o.cert, cr[r]);
        if (!(cr[r] <= tol)) todo.push_back(r);
      }
      if (todo.empty()) { o.converged = true; break; }
      tol_loop *= 0.5;
    }
    if (it == max_iter) break;
    const int nu = (int)todo.size();
    if (dev_select) {
      if (sp.N + 2 * nu > cap) break;   // inner solve: return the current approximate solution
      const int nacc = std::min(dev_count, ov - sp.N);   // already in V[N...]
      if (nacc == 0) break;
      mv(sp.N, nacc);
      sp.n_new += nacc;
      sp.N += nacc;
      continue;
    }
    std::vector<double> shh(nu);
    for (int j = 0; j < nu; ++j) shh[j] = shifts[todo[j]];
    h2d(iu.as<int>(), todo, s);
    h2d(shu.as<double>(), shh, s);
    gather_rows<T>(Rp.as<T>(), iu.as<int>(), nu, ov, gpu_.as<T>(), s);
    gather_rows<T>(Rm.as<T>(), iu.as<int>(), nu, ov, gmu.as<T>(), s);
    auto tp = Clock::now();
    pre(gpu_.as<T>(), gmu.as<T>(), shu.as<double>(), shh, nu, cand.as<T>(), cand.as<T>() + (size_t)nu * ov);
    TD_CUDA(cudaStreamSynchronize(s));
    cnt.t_pre += since(tp);
    if (sp.N + 2 * nu > cap) {
      if (!exact_op) break;   // inner solve: return the current approximate solution
      // thick restart from the current and the previous solutions of every system
      const int nprev = (have_prev && 4 * nr <= 112 && 4 * nr + 2 * nu <= cap) ? 2 * nr : 0;
      DevBuf rst((size_t)4 * nr * ov * es, s);
      TD_CUDA(cudaMemcpyAsync(rst.p, Uout, (size_t)nr * ov * es, cudaMemcpyDeviceToDevice, s));
      TD_CUDA(cudaMemcpyAsync(rst.as<T>() + (size_t)nr * ov, Wout, (size_t)nr * ov * es,
                              cudaMemcpyDeviceToDevice, s));
      if (nprev) {
        TD_CUDA(cudaMemcpyAsync(rst.as<T>() + (size_t)2 * nr * ov, Uprev.p, (size_t)nr * ov * es,
                                cudaMemcpyDeviceToDevice, s));
        TD_CUDA(cudaMemcpyAsync(rst.as<T>() + (size_t)3 * nr * ov, Wprev.p, (size_t)nr * ov * es,
                                cudaMemcpyDeviceToDevice, s));
      }
      sp.N = orth_append<T>(sp.v(), 0, rst.as<T>(), 2 * nr + nprev, ov, s);
      mv(0, sp.N);
      sp.n_old = 0;
      sp.n_new = sp.N;
      cnt.restarts++;
    }
    if (exact_op) {
      TD_CUDA(cudaMemcpyAsync(Uprev.p, Uout, (size_t)nr * ov * es, cudaMemcpyDeviceToDevice, s));
      TD_CUDA(cudaMemcpyAsync(Wprev.p, Wout, (size_t)nr * ov * es, cudaMemcpyDeviceToDevice, s));
      have_prev = true;
    }
    int nacc = orth_append<T>(sp.v(), sp.N, cand.as<T>(), std::min(2 * nu, cap - sp.N), ov, s);
    if (nacc == 0) break;
    mv(sp.N, nacc);
    sp.n_new += nacc;
    sp.N += nacc;
  }
  o.resid = rr;
  return o;
}

// ---------------------------------------------------------------------------
// Casida Davidson (paired eigenproblem).

struct RpaOut {
  std::vector<double> omega, resid;
  DevBuf U, W;
  int n_iter = 0;
  bool converged = false;
  double cert = -1.0;
};

// The gate as in davidson_tda.
RpaOut davidson_rpa(int ov, const PairOp& op, const PairPre& pre, double* guess, int ng, int k,
                    double tol, int max_iter, int cap, int rounds, Counters& cnt, bool exact_op,
                    cudaStream_t s, const RpaCert* cert = nullptr) {
  RpaOut o;
  if (!exact_op) ++g_inner;
  struct Leave { bool on; ~Leave() { if (on) --g_inner; } } leave{!exact_op};
  k = std::min(k, ov);
  cap = std::min(cap, kSmallMax);
  TD_REQUIRE(k >= 1 && k <= kWantMax, TDDFT_ERR_ARG, "n_states out of range");
  TD_REQUIRE(cap >= 4 * k, TDDFT_ERR_ARG, "max_subspace must be at least 4*n_states");
  PairedSpace<double> sp(ov, cap, s);
  DevBuf lamH(k * 8, s), y((size_t)k * cap * 8, s), scr((size_t)2 * k * cap * 8, s);
  DevBuf uc((size_t)k * cap * 8, s), wc((size_t)k * cap * 8, s), isq(k * 8, s), iom(k * 8, s),
      omd(k * 8, s);
  DevBuf U((size_t)k * ov * 8, s), W((size_t)k * ov * 8, s), PU((size_t)k * ov * 8, s),
      MW((size_t)k * ov * 8, s), Rp((size_t)k * ov * 8, s), Rm((size_t)k * ov * 8, s);
  DevBuf rn1(k * 8, s), rn2(k * 8, s), iu(k * 4, s), shu(k * 8, s);
  DevBuf gpu_((size_t)k * ov * 8, s), gmu((size_t)k * ov * 8, s), cand((size_t)2 * k * ov * 8, s);
  DevBuf rst((size_t)4 * k * ov * 8, s), Uprev((size_t)k * ov * 8, s), Wprev((size_t)k * ov * 8, s);
  bool have_prev = false;

  sp.N = orth_append(sp.v(), 0, guess, std::min(ng, cap), ov, s);
  TD_REQUIRE(sp.N >= 1, TDDFT_ERR_ARG, "initial guess is empty");
  auto mv = [&](int r0, int m) {
    auto t0 = Clock::now();
    ScopedPhase ph(exact_op ? PH_MV : PH_RIS, s);
    op(sp.v() + (size_t)r0 * ov, m, sp.p() + (size_t)r0 * ov, sp.m() + (size_t)r0 * ov);
    TD_CUDA(cudaStreamSynchronize(s));
    if (exact_op) { cnt.mv += m; cnt.t_mv += since(t0); } else { cnt.ris_mv += m; }
  };
  mv(0, sp.N);
  sp.n_old = 0;
  sp.n_new = sp.N;
  std::vector<double> om(k), rr(k);
  int kk = k;
  double tol_loop = tol;
  for (int it = 1; it <= max_iter; ++it) {
    o.n_iter = it;
    sp.update(true);
    sp.check_definite();
    const int N = sp.N;
    kk = std::min(k, N);
    double* Lp = sp.L.template as<double>();
    ScopedPhase ph_small(PH_SMALL, s);
    refine_lowest(sp.H.template as<double>(), cap, N, kk, sp.lam32.template as<float>(), sp.vec32.template as<float>(),
                  lamH.as<double>(), y.as<double>(), scr.as<double>(), rounds, s);
    ph_small.stop();
    std::vector<double> l2 = d2h(lamH.as<double>(), kk, s);
    check_finite_host(l2, "Casida Ritz values");
    if (!(l2[0] > 0.0))
      throw Error(TDDFT_ERR_INDEFINITE, "projected Casida problem has a non-positive Omega^2");
    std::vector<double> isqh(kk), iomh(kk);
    for (int j = 0; j < kk; ++j) {
      om[j] = std::sqrt(l2[j]);
      isqh[j] = 1.0 / std::sqrt(om[j]);
      iomh[j] = 1.0 / om[j];
    }
    h2d(isq.as<double>(), isqh, s);
    h2d(iom.as<double>(), iomh, s);
    h2d(omd.as<double>(), std::vector<double>(om.begin(), om.begin() + kk), s);
    // u = L y / sqrt(Omega) ; w = a+ u / Omega
    small_mm<double>(kk, N, N, y.as<double>(), N, 1, Lp, 1, cap, uc.as<double>(), N, s);
    scale_rows(uc.as<double>(), isq.as<double>(), kk, N, s);
    small_mm<double>(kk, N, N, uc.as<double>(), N, 1, sp.ap.template as<double>(), cap, 1, wc.as<double>(), N, s);
    scale_rows(wc.as<double>(), iom.as<double>(), kk, N, s);
    combo<double, double>(uc.as<double>(), kk, N, sp.v(), ov, U.as<double>(), 1.0, 0.0, s);
    combo<double, double>(wc.as<double>(), kk, N, sp.v(), ov, W.as<double>(), 1.0, 0.0, s);
    combo<double, double>(uc.as<double>(), kk, N, sp.p(), ov, PU.as<double>(), 1.0, 0.0, s);
    combo<double, double>(wc.as<double>(), kk, N, sp.m(), ov, MW.as<double>(), 1.0, 0.0, s);
    resid_paired<double>(U.as<double>(), W.as<double>(), PU.as<double>(), MW.as<double>(), omd.as<double>(),
                 nullptr, nullptr, kk, ov, Rp.as<double>(), Rm.as<double>(), s);
    row_sumsq(Rp.as<double>(), ov, kk, ov, rn1.as<double>(), s);
    row_sumsq(Rm.as<double>(), ov, kk, ov, rn2.as<double>(), s);
    std::vector<double> a1 = d2h(rn1.as<double>(), kk, s), a2 = d2h(rn2.as<double>(), kk, s);
    std::vector<int> todo;
    for (int j = 0; j < kk; ++j) {
      rr[j] = std::sqrt(a1[j] + a2[j]);
      if (!(rr[j] < tol_loop)) todo.push_back(j);
    }
    check_finite_host(rr, "Casida residual norms");
    trace(exact_op ? "rpa" : "rpa-guess", it, N, om, rr);
    if (todo.empty() && kk == k) {
      if (!cert) { o.converged = true; break; }
      const std::vector<double> cr = (*cert)(U.as<double>(), W.as<double>(), om, kk);
      trace_gate("rpa", it, rr, cr);
      o.cert = 0.0;
      for (int j = 0; j < kk; ++j) {
        o.cert = std::max(o.cert, cr[j]);
        if (!(cr[j] < tol)) todo.push_back(j);
      }
      if (todo.empty()) { o.converged = true; break; }
      tol_loop *= 0.5;
    }
    if (it == max_iter) break;
    const int nu = (int)todo.size();
    std::vector<double> shh(nu);
    for (int j = 0; j < nu; ++j) shh[j] = om[todo[j]];
    h2d(iu.as<int>(), todo, s);
    h2d(shu.as<double>(), shh, s);
    gather_rows(Rp.as<double>(), iu.as<int>(), nu, ov, gpu_.as<double>(), s);
    gather_rows(Rm.as<double>(), iu.as<int>(), nu, ov, gmu.as<double>(), s);
    auto tp = Clock::now();
    pre(gpu_.as<double>(), gmu.as<double>(), shu.as<double>(), shh, nu, cand.as<double>(),
        cand.as<double>() + (size_t)nu * ov);
    TD_CUDA(cudaStreamSynchronize(s));
    cnt.t_pre += since(tp);
    double* cnew = cand.as<double>();
    int nnew = 2 * nu;
    DevBuf cfree;
    if (sp.N + 2 * nu > cap) {
      // the new directions, orthonormalised against the full subspace first
      cfree = DevBuf((size_t)2 * nu * ov * 8, s);
      nnew = orth_compact<double>(sp.v(), sp.N, cand.as<double>(), 2 * nu, ov, cfree.as<double>(), s);
      if (nnew == 0) break;
      cnew = cfree.as<double>();
      // thick restart: X+Y and X-Y of the wanted roots, now and one iteration ago
      const int nprev = (have_prev && 4 * kk <= 112 && 4 * kk + nnew <= cap) ? 2 * kk : 0;
      TD_CUDA(cudaMemcpyAsync(rst.p, U.p, (size_t)kk * ov * 8, cudaMemcpyDeviceToDevice, s));
      TD_CUDA(cudaMemcpyAsync(rst.as<double>() + (size_t)kk * ov, W.p, (size_t)kk * ov * 8,
                              cudaMemcpyDeviceToDevice, s));
      if (nprev) {
        TD_CUDA(cudaMemcpyAsync(rst.as<double>() + (size_t)2 * kk * ov, Uprev.p, (size_t)kk * ov * 8,
                                cudaMemcpyDeviceToDevice, s));
        TD_CUDA(cudaMemcpyAsync(rst.as<double>() + (size_t)3 * kk * ov, Wprev.p, (size_t)kk * ov * 8,
                                cudaMemcpyDeviceToDevice, s));
      }
      sp.N = orth_append(sp.v(), 0, rst.as<double>(), 2 * kk + nprev, ov, s);
      mv(0, sp.N);
      sp.n_old = 0;
      sp.n_new = sp.N;
      cnt.restarts++;
    }
    TD_CUDA(cudaMemcpyAsync(Uprev.p, U.p, (size_t)kk * ov * 8, cudaMemcpyDeviceToDevice, s));
    TD_CUDA(cudaMemcpyAsync(Wprev.p, W.p, (size_t)kk * ov * 8, cudaMemcpyDeviceToDevice, s));
    have_prev = true;
    int nacc = orth_append(sp.v(), sp.N, cnew, std::min(nnew, cap - sp.N), ov, s);
    if (nacc == 0) break;
    mv(sp.N, nacc);
    sp.n_new += nacc;
    sp.N += nacc;
  }
  o.omega = om;
  o.resid = rr;
  o.U = std::move(U);
  o.W = std::move(W);
  return o;
}

// ---------------------------------------------------------------------------
// rid inner solves (Eq. precondition with the ris operator, Sec. 3.1)

// (T - s_n) v_n = R_n by one block Galerkin subspace, diag-preconditioned
// expansion, stopped at |res_n| <= tol |R_n| or max_iter iterations.  New
// directions are selected, preconditioned and orthonormalised on the device;
// the host reads one status block (residual norms, accepted count) per iteration.
template <typename T, typename S = T>
void inner_tda(int ov, const TdaOpT<T>& Top, const double* delta, const T* R, const double* sh,
               const std::vector<double>& shh, int nu, double tol, int max_iter,
               Counters& cnt, T* out, cudaStream_t s) {
  (void)shh;
  InnerScope inner_scope;
  const int cap = kSmallMax;
  constexpr size_t es = sizeof(T);
  DevBuf Sb((size_t)(cap + nu) * ov * es, s), TS((size_t)cap * ov * es, s), t((size_t)cap * cap * sizeof(S), s);
  DevBuf h((size_t)nu * cap * sizeof(S), s), y((size_t)nu * cap * sizeof(S), s);
  DevBuf Tv((size_t)nu * ov * es, s), res((size_t)nu * ov * es, s), r0(nu * 8, s);
  DevBuf cand((size_t)nu * ov * es, s), keep(nu * 4, s), stat((size_t)nu * 8 + 8, s);
  double* rn = stat.as<double>();
  int* st_count = reinterpret_cast<int*>(stat.as<double>() + nu);
  row_sumsq<T>(R, ov, nu, ov, r0.as<double>(), s);
  std::vector<double> r0h = sqrt_all(d2h(r0.as<double>(), nu, s));
  for (auto& v : r0h) v = v > 0 ? v : 1.0;
  h2d(r0.as<double>(), r0h, s);
  precond_tda<T>(R, sh, delta, nu, ov, cand.as<T>(), s);
  int N = orth_append<T>(Sb.as<T>(), 0, cand.as<T>(), nu, ov, s);
  if (N == 0) { TD_CUDA(cudaMemsetAsync(out, 0, (size_t)nu * ov * es, s)); return; }
  {
    ScopedPhase ph(PH_RIS, s);
    Top(Sb.as<T>(), N, TS.as<T>());
  }
  cnt.ris_mv += N;
  int n_old = 0, n_new = N;
  for (int it = 0; it < max_iter; ++it) {
    proj_cols<T, S>(Sb.as<T>(), N, TS.as<T>() + (size_t)n_old * ov, n_new, ov, t.as<S>(), cap, n_old, s);
    sym_fill<S>(t.as<S>(), cap, n_old, n_new, s);
    gram<T, S>(R, nu, Sb.as<T>(), N, ov, h.as<S>(), N, s);             // h[n][r] = R_n . S_r
    {
      ScopedPhase ph(PH_SMALL, s);
      lu_shift_solve<S>(t.as<S>(), cap, N, sh, nu, h.as<S>(), y.as<S>(), s);
    }
    combo<T, S>(y.as<S>(), nu, N, Sb.as<T>(), ov, out, 1.0, 0.0, s);
    combo<T, S>(y.as<S>(), nu, N, TS.as<T>(), ov, Tv.as<T>(), 1.0, 0.0, s);
    resid_shift<T>(Tv.as<T>(), out, sh, R, nu, ov, res.as<T>(), s);
    row_sumsq<T>(res.as<T>(), ov, nu, ov, rn, s);
    const bool last = it == max_iter - 1;
    if (!last) {
      precond_tda<T>(res.as<T>(), sh, delta, nu, ov, cand.as<T>(), s);
      zero_converged<T>(cand.as<T>(), nu, nu, ov, rn, nullptr, r0.as<double>(), tol, s);
      orth_append_async<T>(Sb.as<T>(), N, cand.as<T>(), nu, ov, keep.as<int>(), st_count, s);
    }
    std::vector<double> blk = d2h(stat.as<double>(), (size_t)nu + 1, s);
    int m = 0;
    for (int j = 0; j < nu; ++j)
      if (!(std::sqrt(blk[j]) / r0h[j] <= tol)) ++m;
    if (m == 0 || last) break;
    if (N + m > cap) break;
    int dev_count;
    std::memcpy(&dev_count, &blk[nu], sizeof(int));
    const int nacc = std::min(dev_count, ov - N);   // already in S[N...]
    if (nacc == 0) break;
    {
      ScopedPhase ph(PH_RIS, s);
      Top(Sb.as<T>() + (size_t)N * ov, nacc, TS.as<T>() + (size_t)N * ov);
    }
    cnt.ris_mv += nacc;
    n_old = N;
    n_new = nacc;
    N += nacc;
  }
}

struct Plan {
  int precond, k, k0, max_iter, inner_max_iter, cap, rounds, nref_inner, nref_outer;
  double tol, inner_tol, guess_tol;
  bool mixed, tc, fp8;
};

Plan make_plan(const Ctx& c, const tddft_opts& o) {
  TD_REQUIRE(o.n_states >= 1, TDDFT_ERR_ARG, "n_states must be positive");
  TD_REQUIRE(o.precond == TDDFT_PRECOND_DIAG || o.precond == TDDFT_PRECOND_RID, TDDFT_ERR_ARG,
             "unknown preconditioner");
  TD_REQUIRE(o.precision == TDDFT_PLAIN || o.precision == TDDFT_MIXED, TDDFT_ERR_ARG,
             "unknown precision");
  TD_REQUIRE(o.tol > 0 && o.inner_tol > 0 && o.guess_tol > 0 && o.max_iter >= 1 &&
                 o.inner_max_iter >= 1, TDDFT_ERR_ARG, "tolerances / iteration limits must be positive");
  const int need = o.precision == TDDFT_PLAIN ? 1 : 2;
  TD_REQUIRE((c.precisions & need) != 0, TDDFT_ERR_ARG,
             "context was created without the factor copies for this precision");
  TD_REQUIRE(!(o.tensor_cores && o.precision != TDDFT_MIXED), TDDFT_ERR_ARG,
             "tensor_cores needs the MIXED precision");
  TD_REQUIRE(!(o.ris_fp8 && !(o.tensor_cores && o.precision == TDDFT_MIXED)), TDDFT_ERR_ARG,
             "ris_fp8 needs the MIXED precision with tensor_cores");
  Plan p;
  p.precond = o.precond;
  p.k = std::min(o.n_states, c.ov);
  TD_REQUIRE(p.k <= kWantMax, TDDFT_ERR_ARG, "n_states above the supported maximum (64)");
  int extra = o.n_extra_guess >= 0 ? o.n_extra_guess
                                   : (o.precond == TDDFT_PRECOND_RID ? std::min(p.k, 3) : 8);
  p.k0 = std::min(p.k + extra, c.ov);
  p.max_iter = o.max_iter;
  p.inner_max_iter = o.inner_max_iter;
  p.cap = o.max_subspace > 0 ? std::min(o.max_subspace, kSmallMax) : kSmallMax;
  p.tol = o.tol;
  p.inner_tol = o.inner_tol;
  p.guess_tol = o.guess_tol;
  p.mixed = o.precision == TDDFT_MIXED;
  p.tc = o.tensor_cores != 0;
  p.fp8 = o.ris_fp8 != 0;
  p.rounds = 3;
  p.nref_inner = p.mixed ? 0 : 2;
  p.nref_outer = 4;
  return p;
}

void fill_stats(tddft_stats* st, int n_iter, const Counters& cnt, bool conv,
                const std::vector<double>& resid, double cert, Clock::time_point t0) {
  if (!st) return;
  st->n_iter = n_iter;
  st->n_matvec = (int)cnt.mv;
  st->n_ris_matvec = (int)cnt.ris_mv;
  st->converged = conv ? 1 : 0;
  st->n_restart = cnt.restarts;
  double m = 0.0;
  for (double r : resid) m = std::max(m, r);
  st->max_resid = m;
  st->max_resid_certified = cert;
  st->t_total_s = since(t0);
  st->t_matvec_s = cnt.t_mv;
  st->t_precond_s = cnt.t_pre;
  st->t_guess_s = cnt.t_guess;
  st->t_certify_s = cnt.t_cert;
  st->gpu_launches = (int)g_launches;
}

void copy_out(double* dst, const double* src, size_t n, bool on_device, cudaStream_t s) {
  if (!dst) return;
  TD_CUDA(cudaMemcpyAsync(dst, src, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

}  // namespace

// ===========================================================================

tddft_status run_tda(Ctx& c, const tddft_opts& o, double* omega, double* X, double* resid,
                     tddft_stats* st) {
  auto t0 = Clock::now();
  g_launches = 0;
  const Plan p = make_plan(c, o);
  const int ov = c.ov;
  cudaStream_t s = c.s;
  Counters cnt;
  const OpDims dims = c.dims();
  const FactorSet Fx = c.exact(o.precision);
  const FactorSet Fr = c.ris(o.precision, p.fp8);
  TdaOp A = [&](const double* Xi, int m, double* out) {
    apply_operator(dims, Fx, Xi, m, OpMode::TDA, out, nullptr, p.tc, s);
  };
  TdaOp T = [&](const double* Xi, int m, double* out) {
    apply_operator(dims, Fr, Xi, m, OpMode::TDA, out, nullptr, p.tc, s);
  };
  TdaPre diag = [&](const double* R, const double* sh, const std::vector<double>&, int nu, double* out) {
    precond_tda(R, sh, c.delta.as<double>(), nu, ov, out, s);
  };
  TdaOpT<float> T32 = [&](const float* Xi, int m, float* out) {
    apply_operator(dims, Fr, Xi, m, OpMode::TDA, out, nullptr, p.tc, s);
  };
  TdaPre rid = [&](const double* R, const double* sh, const std::vector<double>& shh, int nu, double* out) {
    if (p.mixed) {   // FP32 inner solve on the BF16 ris factors
      const long long n = (long long)nu * ov;
      DevBuf R32(n * 4, s), o32(n * 4, s);
      convert(R, DType::F64, R32.p, DType::F32, n, s);
      inner_tda<float, float>(ov, T32, c.delta.as<double>(), R32.as<float>(), sh, shh, nu, p.inner_tol,
                              p.inner_max_iter, cnt, o32.as<float>(), s);
      convert(o32.p, DType::F32, out, DType::F64, n, s);
    } else {
      inner_tda<double>(ov, T, c.delta.as<double>(), R, sh, shh, nu, p.inner_tol, p.inner_max_iter,
                        cnt, out, s);
    }
  };
  // initial guess (Sec. 2.1: low-lying eigenvectors of T)
  DevBuf guess;
  int ng = p.k0;
  if (p.precond == TDDFT_PRECOND_RID) {
    auto tg = Clock::now();
    const int kg = std::min(p.k0 + 8, ov);
    DevBuf unit((size_t)kg * ov * 8, s);
    TD_REQUIRE(kg <= c.n_order, TDDFT_ERR_ARG, "too many initial guesses");
    unit_rows(unit.as<double>(), kg, ov, c.order.as<int>(), s);
    TdaOut g = davidson_tda(ov, T, diag, unit.as<double>(), kg, p.k0, p.guess_tol, p.max_iter, p.cap,
                            p.rounds, cnt, false, s);
    guess = std::move(g.X);
    TD_CUDA(cudaStreamSynchronize(s));
    cnt.t_guess = since(tg);
  } else {
    TD_REQUIRE(p.k0 <= c.n_order, TDDFT_ERR_ARG, "too many initial guesses");
    guess = DevBuf((size_t)p.k0 * ov * 8, s);
    unit_rows(guess.as<double>(), p.k0, ov, c.order.as<int>(), s);
  }
  // MIXED certification: the converged residuals recomputed from fresh
  // products of the Ritz vectors with the solve's FP32-accurate operator (FP16
  // hi+lo tensor-core or FP32 SIMT contractions), FP64 norms; the solve
  // converges only when they are below tol too
  TdaCert certify = [&](const double* Xc, const std::vector<double>& omv, int k) {
    auto tc0 = Clock::now();
    DevBuf AX((size_t)k * ov * 8, s), R((size_t)k * ov * 8, s), rn(k * 8, s), om(k * 8, s);
    A(Xc, k, AX.as<double>());
    h2d(om.as<double>(), std::vector<double>(omv.begin(), omv.begin() + k), s);
    resid_tda(Xc, AX.as<double>(), om.as<double>(), k, ov, R.as<double>(), s);
    row_sumsq(R.as<double>(), ov, k, ov, rn.as<double>(), s);
    std::vector<double> v = sqrt_all(d2h(rn.as<double>(), k, s));
    cnt.t_cert += since(tc0);
    return v;
  };
  TdaOut r = davidson_tda(ov, A, p.precond == TDDFT_PRECOND_RID ? rid : diag, guess.as<double>(), ng,
                          p.k, p.tol, p.max_iter, p.cap, p.rounds, cnt, true, s, p.mixed ? &certify : nullptr);
  double cert = r.cert;
  if (p.mixed && cert < 0.0)   // not converged: report the re-checked residuals of the last Ritz pairs
    for (double v : certify(r.X.as<double>(), r.omega, (int)r.omega.size())) cert = std::max(cert, v);
  const bool dev = o.outputs_on_device != 0;
  if (omega) {
    if (dev) { DevBuf t(p.k * 8, s); h2d(t.as<double>(), r.omega, s); copy_out(omega, t.as<double>(), p.k, true, s); TD_CUDA(cudaStreamSynchronize(s)); }
    else std::copy(r.omega.begin(), r.omega.end(), omega);
  }
  if (resid) {
    if (dev) { DevBuf t(p.k * 8, s); h2d(t.as<double>(), r.resid, s); copy_out(resid, t.as<double>(), p.k, true, s); TD_CUDA(cudaStreamSynchronize(s)); }
    else std::copy(r.resid.begin(), r.resid.end(), resid);
  }
  copy_out(X, r.X.as<double>(), (size_t)p.k * ov, dev, s);
  TD_CUDA(cudaStreamSynchronize(s));
  check_tc_error(c);
  phase_report("solve");
  fill_stats(st, r.n_iter, cnt, r.converged, r.resid, cert, t0);
  return r.converged ? TDDFT_OK : TDDFT_ERR_NOCONV;
}

namespace {
PairOp make_pair_op(const OpDims& dims, const FactorSet& F, bool tc, cudaStream_t s) {
  return [dims, F, tc, s](const double* Xi, int m, double* P, double* M) {
    apply_operator(dims, F, Xi, m, OpMode::PAIRED, P, M, tc, s);
  };
}
PairOpT<float> make_pair_op32(const OpDims& dims, const FactorSet& F, bool tc, cudaStream_t s) {
  return [dims, F, tc, s](const float* Xi, int m, float* P, float* M) {
    apply_operator(dims, F, Xi, m, OpMode::PAIRED, P, M, tc, s);
  };
}

// The rid preconditioner for the paired systems: the ris system T+ u - s w = g+,
// T- w - s u = g- solved to inner_tol; FP32 vectors on the BF16 ris factors in
// MIXED solves, FP64 in PLAIN solves.
void rid_paired(int ov, const Plan& p, const PairOp& T, const PairPre& diag, const PairOpT<float>& T32,
                const PairPreT<float>& diag32, const double* dl, const double* gp, const double* gm,
                const double* sh, const std::vector<double>& shh, int nu, Counters& cnt, double* u,
                double* w, cudaStream_t s) {
  const long long n = (long long)nu * ov;
  if (p.mixed) {
    DevBuf g32((size_t)2 * n * 4, s), init((size_t)2 * n * 4, s), uw((size_t)2 * n * 4, s);
    convert(gp, DType::F64, g32.p, DType::F32, n, s);
    convert(gm, DType::F64, g32.as<float>() + n, DType::F32, n, s);
    precond_paired<float>(g32.as<float>(), g32.as<float>() + n, sh, dl, nu, ov, init.as<float>(),
                          init.as<float>() + n, s);
    paired_linear<float, float>(ov, T32, diag32, g32.as<float>(), g32.as<float>() + n, shh, nu, init.as<float>(),
                         2 * nu, p.inner_tol, p.inner_max_iter, kSmallMax, false, cnt,
                         uw.as<float>(), uw.as<float>() + n, s);
    convert(uw.p, DType::F32, u, DType::F64, n, s);
    convert(uw.as<float>() + n, DType::F32, w, DType::F64, n, s);
  } else {
    DevBuf init((size_t)2 * n * 8, s);
    precond_paired<double>(gp, gm, sh, dl, nu, ov, init.as<double>(), init.as<double>() + n, s);
    paired_linear<double>(ov, T, diag, gp, gm, shh, nu, init.as<double>(), 2 * nu, p.inner_tol,
                          p.inner_max_iter, kSmallMax, false, cnt, u, w, s);
  }
}
}  // namespace

tddft_status run_rpa(Ctx& c, const tddft_opts& o, double* omega, double* X, double* Y,
                     double* resid, tddft_stats* st) {
  auto t0 = Clock::now();
  g_launches = 0;
  const Plan p = make_plan(c, o);
  const int ov = c.ov;
  cudaStream_t s = c.s;
  Counters cnt;
  const OpDims dims = c.dims();
  PairOp A = make_pair_op(dims, c.exact(o.precision), p.tc, s);
  PairOp T = make_pair_op(dims, c.ris(o.precision, p.fp8), p.tc, s);
  const double* dl = c.delta.as<double>();
  PairPre diag = [&](const double* gp, const double* gm, const double* sh, const std::vector<double>&,
                     int nu, double* u, double* w) { precond_paired(gp, gm, sh, dl, nu, ov, u, w, s); };
  PairOpT<float> T32 = make_pair_op32(dims, c.ris(o.precision, p.fp8), p.tc, s);
  PairPreT<float> diag32 = [&](const float* gp, const float* gm, const double* sh,
                               const std::vector<double>&, int nu, float* u, float* w) {
    precond_paired<float>(gp, gm, sh, dl, nu, ov, u, w, s);
  };
  PairPre rid = [&](const double* gp, const double* gm, const double* sh,
                    const std::vector<double>& shh, int nu, double* u, double* w) {
    rid_paired(ov, p, T, diag, T32, diag32, dl, gp, gm, sh, shh, nu, cnt, u, w, s);
  };
  DevBuf guess;
  int ng = p.k0;
  if (p.precond == TDDFT_PRECOND_RID) {
    auto tg = Clock::now();
    const int kg = std::min(p.k0 + 8, ov);
    TD_REQUIRE(kg <= c.n_order, TDDFT_ERR_ARG, "too many initial guesses");
    DevBuf unit((size_t)kg * ov * 8, s);
    unit_rows(unit.as<double>(), kg, ov, c.order.as<int>(), s);
    RpaOut g = davidson_rpa(ov, T, diag, unit.as<double>(), kg, p.k0, p.guess_tol, p.max_iter, p.cap,
                            p.rounds, cnt, false, s);
    guess = DevBuf((size_t)2 * p.k0 * ov * 8, s);
    TD_CUDA(cudaMemcpyAsync(guess.p, g.U.p, (size_t)p.k0 * ov * 8, cudaMemcpyDeviceToDevice, s));
    TD_CUDA(cudaMemcpyAsync(guess.as<double>() + (size_t)p.k0 * ov, g.W.p, (size_t)p.k0 * ov * 8,
                            cudaMemcpyDeviceToDevice, s));
    ng = 2 * p.k0;
    TD_CUDA(cudaStreamSynchronize(s));
    cnt.t_guess = since(tg);
  } else {
    TD_REQUIRE(p.k0 <= c.n_order, TDDFT_ERR_ARG, "too many initial guesses");
    guess = DevBuf((size_t)p.k0 * ov * 8, s);
    unit_rows(guess.as<double>(), p.k0, ov, c.order.as<int>(), s);
  }
  // MIXED certification as in run_tda
  RpaCert certify = [&](const double* Uc, const double* Wc, const std::vector<double>& omv, int k) {
    auto tc0 = Clock::now();
    DevBuf PU((size_t)k * ov * 8, s), MU((size_t)k * ov * 8, s), PW((size_t)k * ov * 8, s),
        MW((size_t)k * ov * 8, s), Rp((size_t)k * ov * 8, s), Rm((size_t)k * ov * 8, s);
    DevBuf a1(k * 8, s), a2(k * 8, s), om(k * 8, s);
    A(Uc, k, PU.as<double>(), MU.as<double>());
    A(Wc, k, PW.as<double>(), MW.as<double>());
    h2d(om.as<double>(), std::vector<double>(omv.begin(), omv.begin() + k), s);
    resid_paired<double>(Uc, Wc, PU.as<double>(), MW.as<double>(), om.as<double>(), nullptr, nullptr, k, ov,
                         Rp.as<double>(), Rm.as<double>(), s);
    row_sumsq(Rp.as<double>(), ov, k, ov, a1.as<double>(), s);
    row_sumsq(Rm.as<double>(), ov, k, ov, a2.as<double>(), s);
    auto h1 = d2h(a1.as<double>(), k, s), h2 = d2h(a2.as<double>(), k, s);
    std::vector<double> v(k);
    for (int j = 0; j < k; ++j) v[j] = std::sqrt(h1[j] + h2[j]);
    cnt.t_cert += since(tc0);
    return v;
  };
  RpaOut r = davidson_rpa(ov, A, p.precond == TDDFT_PRECOND_RID ? rid : diag, guess.as<double>(), ng,
                          p.k, p.tol, p.max_iter, p.cap, p.rounds, cnt, true, s, p.mixed ? &certify : nullptr);
  double cert = r.cert;
  if (p.mixed && cert < 0.0)
    for (double v : certify(r.U.as<double>(), r.W.as<double>(), r.omega, (int)r.omega.size())) cert = std::max(cert, v);
  const bool dev = o.outputs_on_device != 0;
  if (omega) {
    if (dev) { DevBuf t(p.k * 8, s); h2d(t.as<double>(), r.omega, s); copy_out(omega, t.as<double>(), p.k, true, s); TD_CUDA(cudaStreamSynchronize(s)); }
    else std::copy(r.omega.begin(), r.omega.end(), omega);
  }
  if (resid) {
    if (dev) { DevBuf t(p.k * 8, s); h2d(t.as<double>(), r.resid, s); copy_out(resid, t.as<double>(), p.k, true, s); TD_CUDA(cudaStreamSynchronize(s)); }
    else std::copy(r.resid.begin(), r.resid.end(), resid);
  }
  if (X || Y) {
    DevBuf Xd((size_t)p.k * ov * 8, s), Yd((size_t)p.k * ov * 8, s);
    half_sum_diff(r.U.as<double>(), r.W.as<double>(), (long long)p.k * ov, Xd.as<double>(), Yd.as<double>(), s);
    copy_out(X, Xd.as<double>(), (size_t)p.k * ov, dev, s);
    copy_out(Y, Yd.as<double>(), (size_t)p.k * ov, dev, s);
    TD_CUDA(cudaStreamSynchronize(s));
  }
  TD_CUDA(cudaStreamSynchronize(s));
  check_tc_error(c);
  phase_report("solve");
  fill_stats(st, r.n_iter, cnt, r.converged, r.resid, cert, t0);
  return r.converged ? TDDFT_OK : TDDFT_ERR_NOCONV;
}

tddft_status run_polar(Ctx& c, const tddft_opts& o, const double* mu, int n_dip,
                       const double* freqs, int n_freq, double* alpha, tddft_stats* st) {
  auto t0 = Clock::now();
  g_launches = 0;
  tddft_opts oo = o;
  if (oo.n_states < 1) oo.n_states = 1;
  const Plan p = make_plan(c, oo);
  TD_REQUIRE(n_dip >= 1 && n_freq >= 1 && mu && freqs, TDDFT_ERR_ARG, "polar: need dipoles and frequencies");
  const int nr = n_dip * n_freq;
  TD_REQUIRE(2 * nr <= 112, TDDFT_ERR_ARG, "polar: too many right-hand sides");
  TD_REQUIRE(4 * nr <= p.cap, TDDFT_ERR_ARG, "polar: max_subspace must be at least 4*n_dip*n_freq");
  const int ov = c.ov;
  cudaStream_t s = c.s;
  Counters cnt;
  const OpDims dims = c.dims();
  PairOp A = make_pair_op(dims, c.exact(o.precision), p.tc, s);
  PairOp T = make_pair_op(dims, c.ris(o.precision, p.fp8), p.tc, s);
  const double* dl = c.delta.as<double>();
  const bool dev = o.outputs_on_device != 0;
  // right-hand sides 2 mu for every (omega_f, mu_u): row f*n_dip + u
  DevBuf mud((size_t)n_dip * ov * 8, s), b((size_t)nr * ov * 8, s);
  TD_CUDA(cudaMemcpyAsync(mud.p, mu, (size_t)n_dip * ov * 8, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  std::vector<double> fh(n_freq);
  if (dev) fh = d2h(freqs, n_freq, s);
  else fh.assign(freqs, freqs + n_freq);
  std::vector<double> sh(nr), two(nr, 2.0);
  DevBuf twod(nr * 8, s), shd(nr * 8, s);
  for (int f = 0; f < n_freq; ++f)
    for (int u = 0; u < n_dip; ++u) sh[f * n_dip + u] = fh[f];
  TD_CUDA(cudaMemsetAsync(b.p, 0, (size_t)nr * ov * 8, s));
  h2d(twod.as<double>(), two, s);
  h2d(shd.as<double>(), sh, s);
  for (int f = 0; f < n_freq; ++f)
    axpy_rows(b.as<double>() + (size_t)f * n_dip * ov, mud.as<double>(), twod.as<double>(), n_dip, ov, s);
  PairPre diag = [&](const double* gp, const double* gm, const double* shv, const std::vector<double>&,
                     int nu, double* u, double* w) { precond_paired(gp, gm, shv, dl, nu, ov, u, w, s); };
  PairOpT<float> T32 = make_pair_op32(dims, c.ris(o.precision, p.fp8), p.tc, s);
  PairPreT<float> diag32 = [&](const float* gp, const float* gm, const double* shv,
                               const std::vector<double>&, int nu, float* u, float* w) {
    precond_paired<float>(gp, gm, shv, dl, nu, ov, u, w, s);
  };
  PairPre rid = [&](const double* gp, const double* gm, const double* shv,
                    const std::vector<double>& shh, int nu, double* u, double* w) {
    rid_paired(ov, p, T, diag, T32, diag32, dl, gp, gm, shv, shh, nu, cnt, u, w, s);
  };
  // initial directions
  DevBuf init((size_t)2 * nr * ov * 8, s);
  double* iu = init.as<double>();
  double* iw = iu + (size_t)nr * ov;
  if (p.precond == TDDFT_PRECOND_RID) {
    // initial guess: the ris system solved to the guess tolerance (Sec. 3.1)
    if (p.mixed) {
      const long long n = (long long)nr * ov;
      DevBuf b32(n * 4, s), d0((size_t)2 * n * 4, s), uw((size_t)2 * n * 4, s);
      convert(b.p, DType::F64, b32.p, DType::F32, n, s);
      precond_paired<float>(b32.as<float>(), nullptr, shd.as<double>(), dl, nr, ov, d0.as<float>(),
                            d0.as<float>() + n, s);
      paired_linear<float, float>(ov, T32, diag32, b32.as<float>(), nullptr, sh, nr, d0.as<float>(), 2 * nr,
                           p.guess_tol, p.max_iter, kSmallMax, false, cnt, uw.as<float>(),
                           uw.as<float>() + n, s);
      convert(uw.p, DType::F32, iu, DType::F64, 2 * n, s);
    } else {
      DevBuf d0((size_t)2 * nr * ov * 8, s);
      precond_paired<double>(b.as<double>(), nullptr, shd.as<double>(), dl, nr, ov, d0.as<double>(),
                             d0.as<double>() + (size_t)nr * ov, s);
      paired_linear<double>(ov, T, diag, b.as<double>(), nullptr, sh, nr, d0.as<double>(), 2 * nr,
                            p.guess_tol, p.max_iter, kSmallMax, false, cnt, iu, iw, s);
    }
  } else {
    precond_paired<double>(b.as<double>(), nullptr, shd.as<double>(), dl, nr, ov, iu, iw, s);
  }
  DevBuf U((size_t)nr * ov * 8, s), W((size_t)nr * ov * 8, s);
  // MIXED certification as in run_tda (relative residuals)
  DevBuf rhs_norm(nr * 8, s);
  row_sumsq(b.as<double>(), ov, nr, ov, rhs_norm.as<double>(), s);
  const std::vector<double> bn = sqrt_all(d2h(rhs_norm.as<double>(), nr, s));
  LinCert<double> certify = [&](const double* Uc, const double* Wc) {
    auto tc0 = Clock::now();
    DevBuf PU((size_t)nr * ov * 8, s), MU((size_t)nr * ov * 8, s), PW((size_t)nr * ov * 8, s),
        MW((size_t)nr * ov * 8, s), Rp((size_t)nr * ov * 8, s), Rm((size_t)nr * ov * 8, s);
    DevBuf a1(nr * 8, s), a2(nr * 8, s);
    A(Uc, nr, PU.as<double>(), MU.as<double>());
    A(Wc, nr, PW.as<double>(), MW.as<double>());
    resid_paired<double>(Uc, Wc, PU.as<double>(), MW.as<double>(), shd.as<double>(), b.as<double>(), nullptr, nr,
                         ov, Rp.as<double>(), Rm.as<double>(), s);
    row_sumsq(Rp.as<double>(), ov, nr, ov, a1.as<double>(), s);
    row_sumsq(Rm.as<double>(), ov, nr, ov, a2.as<double>(), s);
    auto h1 = d2h(a1.as<double>(), nr, s), h2 = d2h(a2.as<double>(), nr, s);
    std::vector<double> v(nr);
    for (int j = 0; j < nr; ++j) v[j] = std::sqrt(h1[j] + h2[j]) / (bn[j] > 0 ? bn[j] : 1.0);
    cnt.t_cert += since(tc0);
    return v;
  };
  PairedLinOut r = paired_linear<double>(ov, A, p.precond == TDDFT_PRECOND_RID ? rid : diag,
                                         b.as<double>(), nullptr, sh, nr, iu, 2 * nr, p.tol, p.max_iter,
                                         p.cap, true, cnt, U.as<double>(), W.as<double>(), s,
                                         p.mixed ? &certify : nullptr);
  double cert = r.cert;
  if (p.mixed && cert < 0.0)
    for (double v : certify(U.as<double>(), W.as<double>())) cert = std::max(cert, v);
  // alpha[f][v][u] = mu_v . U[f*n_dip + u]
  DevBuf G((size_t)n_dip * nr * 8, s);
  gram(mud.as<double>(), n_dip, U.as<double>(), nr, ov, G.as<double>(), nr, s);
  std::vector<double> gh = d2h(G.as<double>(), (size_t)n_dip * nr, s);
  std::vector<double> al((size_t)n_freq * n_dip * n_dip);
  for (int f = 0; f < n_freq; ++f)
    for (int v = 0; v < n_dip; ++v)
      for (int u = 0; u < n_dip; ++u) al[((size_t)f * n_dip + v) * n_dip + u] = gh[(size_t)v * nr + f * n_dip + u];
  if (alpha) {
    if (dev) { DevBuf t(al.size() * 8, s); h2d(t.as<double>(), al, s); copy_out(alpha, t.as<double>(), al.size(), true, s); }
    else std::copy(al.begin(), al.end(), alpha);
  }
  TD_CUDA(cudaStreamSynchronize(s));
  check_tc_error(c);
  phase_report("solve");
  fill_stats(st, r.n_iter, cnt, r.converged, r.resid, cert, t0);
  return r.converged ? TDDFT_OK : TDDFT_ERR_NOCONV;
}

}  // namespace tddft
