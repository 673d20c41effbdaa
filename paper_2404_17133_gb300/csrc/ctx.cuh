// Solver context: resident factor copies, orbital data and the request queue.
#pragma once
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace tddft {

// One operator's factors in one element type.
//   Coulomb   J(X)_ia  = sum_P Jov[P][ia] sum_jb Jov[P][jb] X_jb            (nJ rows)
//   exchange  K1(X)_ib = sum_P sum_j Koo[P][i][j] sum_a X_ja Kvv[P][a][b]      (nK rows)
//             K2(X)_ia = sum_P sum_j (sum_b Kov[P][i][b] X_jb) Kov[P][j][a]
struct FactorSet {
  DType dt = DType::F64;
  int nJ = 0, nK = 0;
  const void* Jov = nullptr;
  const void* Koo = nullptr;
  const void* Kvv = nullptr;
  const void* Kov = nullptr;
  // Tensor-core operands (rows padded to tc_pad): Kvv as [P][b][a] and Kov
  // transposed as [P][a][j]; for the exact operator FP16 hi + lo parts of the
  // factors times the powers of two in tc_scale (tc_f16_tensor_scale), for the
  // ris operator hi only (plain BF16).
  TcElt tc_elt = TcElt::BF16;
  const float* tc_scale = nullptr;   // FP16: the factor-set scale block (8 floats)
  const void* Kvv_hi = nullptr;
  const void* Kvv_lo = nullptr;
  const void* Kvo_hi = nullptr;
  const void* Kvo_lo = nullptr;
  // stage-1 operands: Koo as [P][i][pad(j)], Kov as [P][i][pad(b)]
  const void* Koo_hi = nullptr;
  const void* Koo_lo = nullptr;
  const void* Kovp_hi = nullptr;
  const void* Kovp_lo = nullptr;
  // FP16 exact sets that carry the Coulomb term: s_ov L_ov transposed
  // ([ov][tc_pad(nJ)], hi + lo), the B operand of J = t^T L_ov; with Kovp (the
  // same rows as [P][ov]) both Coulomb contractions run on the tensor cores
  const void* JovT_hi = nullptr;
  const void* JovT_lo = nullptr;
  // Variant terms of the exact operator (Eq. hessian for other functionals):
  // a second exchange factor set entering with weight b_x, and a low-rank
  // kernel sum_g w_g F^g_ia F^g_jb added to the Coulomb term, its rows stored
  // scaled by sqrt|w_g| and split by the sign of w_g (element type dt).
  const FactorSet* lr = nullptr;
  double b_x = 0.0;
  // FP8 e4m3 copies of the (BF16) ris exchange rows with one scale per row P,
  // used by the tensor-core path when fp8 is set: Kvv8 as [P][b][tc_pad16(a)],
  // Kvo8 (L_ov transposed) as [P][a][tc_pad16(j)]; s_vv / s_vo the scales,
  // rho_oo / rho_ov the largest row norms of L^P_oo and L^P_ov (bounds of the
  // stage-1 results)
  bool fp8 = false;
  const unsigned char* Kvv8 = nullptr;
  const unsigned char* Kvo8 = nullptr;
  const float* s_vv = nullptr;
  const float* s_vo = nullptr;
  const float* rho_oo = nullptr;
  const float* rho_ov = nullptr;
  const void* Fpos = nullptr;
  const void* Fneg = nullptr;
  int nFpos = 0, nFneg = 0;
  bool has_variants() const { return (lr && b_x != 0.0) || nFpos > 0 || nFneg > 0; }
};

// Device copies of one exact factor set (L_oo, L_ov, L_vv with n rows) in the
// precisions a context keeps.
struct ExactCopies {
  int n = 0;
  DevBuf f64_oo, f64_ov, f64_vv;  // PLAIN
  DevBuf f32_oo, f32_ov, f32_vv;  // MIXED: SIMT operands
  DevBuf vv_hi, vv_lo;            // [n][nv][tc_pad(nv)] FP16 split of s_vv L_vv
  DevBuf vo_hi, vo_lo;            // [n][nv][tc_pad(no)] FP16 split of s_ov L_ov transposed
  DevBuf oo_hi, oo_lo;            // [n][no][tc_pad(no)] (s_oo L_oo)
  DevBuf ov_hi, ov_lo;            // [n][no][tc_pad(nv)] (s_ov L_ov)
  DevBuf ovT_hi, ovT_lo;          // [ov][tc_pad(n)] (s_ov L_ov transposed; sets with the Coulomb term)
  DevBuf tc_scale;                // the scale block of tc_f16_tensor_scale (8 floats)
  // Exchange operands of `precision` into f (and the Coulomb block when coulomb).
  void fill(FactorSet& f, int precision, bool coulomb) const;
};

// Event-based timing of one kernel family (the dominant contraction).
struct KernelProfile {
  bool on = false;
  std::vector<cudaEvent_t> ev;      // pairs (start, stop)
  std::vector<cudaEvent_t> spare;   // events already created, reused by later launches
  std::vector<double> pend_flops, pend_bytes;   // per launch, until collected
  long long launches = 0;
  double flops = 0.0, ms = 0.0;
  // collected per-launch records (the first kMaxRecords launches)
  static constexpr size_t kMaxRecords = 1u << 17;
  std::vector<double> rec_ms, rec_flops, rec_bytes;
  void begin(cudaStream_t s);
  // launch_flops / launch_bytes: the launch's algorithmic flops and bytes
  // (operands read once, result written once)
  void end(cudaStream_t s, double launch_flops, double launch_bytes = 0.0);
  void reserve(size_t n_events);    // create events ahead of the launches they will time
  void collect();                   // fold recorded pairs into ms (synchronises)
  void reset();
  ~KernelProfile();
};

struct OpDims {
  int no = 0, nv = 0, ov = 0;
  double a_x = 0.0, c_J = 2.0;
  const double* delta = nullptr;  // device [ov]
  KernelProfile* prof = nullptr;       // optional timing of the K1 contraction (tcgen05)
  KernelProfile* prof_simt = nullptr;  // the same for the SIMT contraction
  int* tc_err = nullptr;          // device flag set by the tensor-core kernel
};

enum class OpMode { TDA, PAIRED };

// out0 = A X (TDA) or (A+B) X and out1 = (A-B) X (PAIRED); X, out FP64 [m][ov].
// tc: 0 SIMT contractions; nonzero the exchange contractions on tcgen05
// (exact factor sets: FP16 hi+lo operands with power-of-two scales, three
// products, FP32-accurate; ris factor sets: trial vectors as BF16 hi+lo
// against the plain BF16 rows, or the FP8 rows when the set has them).
void apply_operator(const OpDims& d, const FactorSet& f, const double* X, int m, OpMode mode,
                    double* out0, double* out1, int tc, cudaStream_t s);
// FP32 vectors (FP32 or BF16 factor sets only): the ris products of the inner solves.
void apply_operator(const OpDims& d, const FactorSet& f, const float* X, int m, OpMode mode,
                    float* out0, float* out1, int tc, cudaStream_t s);

struct Request {
  int kind = 0;
  tddft_request* req = nullptr;
  tddft_status status = TDDFT_PENDING;
  bool done = false;
};

// Device bytes of the factor copies tddft_create makes for `d` (both
// precisions as selected by d.precisions).
unsigned long long factor_copy_bytes(const tddft_desc& d, bool coulomb = true);

struct Ctx {
  cudaStream_t s = nullptr;
  bool own_stream = false;
  int device = 0;
  int no = 0, nv = 0, ov = 0, naux = 0, nJ = 0, nK = 0;
  double a_x = 0.25, c_J = 2.0, t_cut = 0.0;
  int precisions = 3;
  // orbital data
  DevBuf eps_o, eps_v, delta;
  DevBuf order;                   // int32 indices of Delta ascending (first n_order)
  int n_order = 0;
  // exact factors
  ExactCopies x;
  // variant terms (tddft_add_exchange, tddft_add_kernel)
  ExactCopies lrx;                // second exchange set, n = 0 if none
  double b_x = 0.0;
  FactorSet lr_set[2];            // PLAIN and MIXED views of lrx
  DevBuf ker64[2], ker32[2];      // kernel rows scaled by sqrt|w|: w > 0, w < 0
  int n_ker[2] = {0, 0};
  DevBuf tc_err;                  // int flag, see OpDims::tc_err
  // ris factors: Coulomb ov (all rows), exchange oo/vv/ov (s rows, windowed)
  DevBuf r64_J, r64_Koo, r64_Kvv, r64_Kov;
  DevBuf r16_J, r16_Koo, r16_Kvv, r16_Kov;
  DevBuf r16_vvp, r16_vo, r16_oop, r16_ovp;   // tensor-core copies of the ris exchange rows
  DevBuf r8_vvp, r8_vo;           // FP8 e4m3 copies of the ris exchange rows (FactorSet::Kvv8, Kvo8)
  DevBuf r8_aux;                  // float [4][n_K]: s_vv, s_vo, rho_oo, rho_ov
  tddft_desc desc{};              // as given to tddft_create
  unsigned long long device_bytes = 0;
  std::string err;
  // request queue
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<unsigned long long> queue;
  std::map<unsigned long long, Request> requests;
  unsigned long long next_ticket = 1;
  std::thread worker;
  bool stopping = false;
  std::mutex run_mu;  // one solve at a time on the context's stream
  KernelProfile prof, prof_simt;

  OpDims dims() const {
    OpDims d;
    d.no = no; d.nv = nv; d.ov = ov; d.a_x = a_x; d.c_J = c_J;
    d.delta = delta.as<double>();
    d.prof = const_cast<KernelProfile*>(&prof);
    d.prof_simt = const_cast<KernelProfile*>(&prof_simt);
    d.tc_err = tc_err.as<int>();
    return d;
  }
  FactorSet exact(int precision) const;  // PLAIN -> FP64, MIXED -> FP32 (+ BF16 split)
  FactorSet ris(int precision, bool fp8 = false) const;  // PLAIN -> FP64, MIXED -> BF16 (+ FP8)
};

// Throw if the tensor-core kernel reported a timeout since the last check.
void check_tc_error(Ctx& c);

tddft_status run_tda(Ctx& c, const tddft_opts& o, double* omega, double* X, double* resid,
                     tddft_stats* st);
tddft_status run_rpa(Ctx& c, const tddft_opts& o, double* omega, double* X, double* Y,
                     double* resid, tddft_stats* st);
tddft_status run_polar(Ctx& c, const tddft_opts& o, const double* mu, int n_dip,
                       const double* freqs, int n_freq, double* alpha, tddft_stats* st);
tddft_status solve_tda_batch(Ctx* const* ctxs, int n, const tddft_opts* opts, double* omega, double* resid,
                             tddft_stats* stats, tddft_batch_info* info);

}  // namespace tddft
