// On-the-fly response products over density-fitted factors (Eq. hessian with
// (pq|rs) = sum_P L^P_pq L^P_rs, Eq. pqrs_approx):
//   A X     = Delta X + c_J J(X) - a_x K1(X)                      (Eq. TDA)
//   (A+B) X = Delta X + 2 c_J J(X) - a_x (K1(X) + K2(X))
//   (A-B) X = Delta X + a_x (K2(X) - K1(X))
// with J(X)_ia = sum_jb (ia|jb) X_jb, K1(X)_ib = sum_ja (ij|ab) X_ja,
// K2(X)_ia = sum_jb (ib|ja) X_jb.  The four-index integrals are never formed;
// each term is a pair of contractions over P:
//   J : t[P][n] = sum_ia L_ov[P][ia] X[n][ia];  J[n][ia] = sum_P t[P][n] L_ov[P][ia]
//   K1: Z[n][i][P][a] = sum_j L_oo[P][i][j] X[n][j][a]   (batched over P, n)
//       K1[(n,i)][b] = sum_(P,a) Z[(n,i)][(P,a)] L_vv[P][a][b]   (one tall-K GEMM)
//   K2: Q[n][i][P][j] = sum_b L_ov[P][i][b] X[n][j][b]
//       K2[(n,i)][a] = sum_(P,j) Q[(n,i)][(P,j)] L_ov[P][j][a]
// P is processed in chunks so the intermediates stay within a bounded
// workspace; the second contractions of K1 and K2 (most of the flops) run on the
// tcgen05 tensor cores when asked (MIXED precision).
#include "ctx.cuh"
#include "skinny.cuh"
#include "tc_gemm.cuh"
#include "vecops.cuh"

namespace tddft {

namespace {
cudaEvent_t take_event(std::vector<cudaEvent_t>& spare) {
  cudaEvent_t e;
  if (!spare.empty()) {
    e = spare.back();
    spare.pop_back();
  } else {
    TD_CUDA(cudaEventCreate(&e));
  }
  return e;
}
}  // namespace

void KernelProfile::begin(cudaStream_t s) {
  cudaEvent_t a = take_event(spare);
  ev.push_back(a);
  TD_CUDA(cudaEventRecord(a, s));
}
void KernelProfile::end(cudaStream_t s, double launch_flops, double launch_bytes) {
  cudaEvent_t b = take_event(spare);
  ev.push_back(b);
  TD_CUDA(cudaEventRecord(b, s));
  pend_flops.push_back(launch_flops);
  pend_bytes.push_back(launch_bytes);
  launches++;
  flops += launch_flops;
}
void KernelProfile::reserve(size_t n_events) {
  while (spare.size() < n_events) {
    cudaEvent_t e;
    TD_CUDA(cudaEventCreate(&e));
    spare.push_back(e);
  }
}
void KernelProfile::collect() {
  for (size_t i = 0; i + 1 < ev.size(); i += 2) {
    TD_CUDA(cudaEventSynchronize(ev[i + 1]));
    float t = 0.f;
    TD_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
    ms += t;
    if (rec_ms.size() < kMaxRecords) {
      rec_ms.push_back(t);
      rec_flops.push_back(pend_flops[i / 2]);
      rec_bytes.push_back(pend_bytes[i / 2]);
    }
  }
  spare.insert(spare.end(), ev.begin(), ev.end());   // recorded and waited on: reusable
  ev.clear();
  pend_flops.clear();
  pend_bytes.clear();
}
void KernelProfile::reset() {
  for (auto e : ev) cudaEventDestroy(e);   // possibly still pending: not reused
  ev.clear();
  pend_flops.clear();
  pend_bytes.clear();
  rec_ms.clear();
  rec_flops.clear();
  rec_bytes.clear();
  launches = 0;
  flops = 0.0;
  ms = 0.0;
}
KernelProfile::~KernelProfile() {
  for (auto e : spare) cudaEventDestroy(e);
  for (auto e : ev) cudaEventDestroy(e);
}

namespace {
// Exchange intermediates of one P-chunk: SIMT contractions keep them within
// 512 MB; the tensor-core path takes 4 GB, so that a contraction launch covers
// many auxiliary rows (longer K loops per CTA, fewer launches and pipeline fills).
constexpr size_t kChunkBytes = 512ull << 20;
constexpr size_t kChunkBytesTC = 4ull << 30;
// k-blocks one CTA accumulates in FP32 before its split-K partial is summed
// (fixed order) with the others: the rounding of an FP32 run grows with its
// length, and runs over a whole P-chunk of the exchange contraction (~1e4 MMA
// steps) left the large Casida solve's recomputed residuals 3e-6 above the
// loop's.  Exchange: 256 k-blocks (16384 terms); the Coulomb term's J = t^T
// L_ov (K = n_aux): 16.
constexpr int kExchangeKb = 256;
constexpr int kCoulombKb = 16;

int chunk_rows(int nrows, long long per_row_bytes, int m, size_t budget = kChunkBytes) {
  long long pc = (long long)(budget / (per_row_bytes > 0 ? per_row_bytes : 1));
  if (pc < 1) pc = 1;
  if (pc > nrows) pc = nrows;
  long long bmax = 65535 / (m > 0 ? m : 1);
  if (pc > bmax) pc = bmax;
  return (int)(pc < 1 ? 1 : pc);
}
}  // namespace

void check_tc_error(Ctx& c) {
  int h = 0;
  TD_CUDA(cudaMemcpyAsync(&h, c.tc_err.p, 4, cudaMemcpyDeviceToHost, c.s));
  TD_CUDA(cudaStreamSynchronize(c.s));
  if (h != 0) {
    TD_CUDA(cudaMemsetAsync(c.tc_err.p, 0, 4, c.s));
    throw Error(TDDFT_ERR_CUDA, "tensor-core kernel wait timed out (code " + std::to_string(h) + ")");
  }
}

template <typename TX>
static void apply_operator_t(const OpDims& d, const FactorSet& f, const TX* X, int m, OpMode mode,
                             TX* out0, TX* out1, int tc, cudaStream_t s) {
  const bool tensor_cores = tc != 0;
  if (m <= 0) return;
  const int no = d.no, nv = d.nv, ov = d.ov;
  const bool f64 = (f.dt == DType::F64);
  const DType tw = f64 ? DType::F64 : DType::F32;  // working / accumulation type
  const size_t ew = dtype_size(tw);
  const long long mov = (long long)m * ov;
  constexpr bool x32 = sizeof(TX) == 4;
  TD_REQUIRE(!(x32 && f64), TDDFT_ERR_ARG, "FP32 vectors need FP32/BF16 factors");

  const void* Xw = X;
  DevBuf xbuf;
  if (!f64 && !x32) {
    xbuf = DevBuf(mov * 4, s);
    cast_f64_to_f32(reinterpret_cast<const double*>(X), xbuf.as<float>(), mov, s);
    Xw = xbuf.p;
  }

  // ---- Coulomb (and the low-rank kernel term, which enters with the same prefactor)
  DevBuf Jb;
  bool have_J = false;
  if (f.nJ > 0 && d.c_J != 0.0) {
    // t[P][n] = sum_ia L_ov[P][ia] X[n][ia];  J[n][ia] = sum_P t[P][n] L_ov[P][ia]
    Jb = DevBuf(mov * ew, s);
    if (tensor_cores && f.tc_elt == TcElt::F16 && f.JovT_hi && !f64) {
      // t = L_ov X^T on the SIMT path (K = ov: its FP32 reduction tree keeps t
      // at ~1e-7; one tensor-core accumulation run per 4096 terms left the
      // Coulomb products at ~2e-6), then J = t^T L_ov on the tensor cores,
      // streaming the FP16 hi+lo copy of s_ov L_ov transposed once, with t as
      // FP16 parts of s_t t
      DevBuf t((size_t)f.nJ * m * 4, s), sct(2 * 4, s), scr(8, s), fac(4, s);
      sk_gram(f.Jov, f.dt, ov, f.nJ, Xw, tw, ov, m, ov, t.p, tw, m, 1.0, 0.0, s);
      tc_f16_tensor_scale(t.as<float>(), f.nJ, m, sct.as<float>(), scr.as<unsigned>(), s);
      const int nJp = tc_pad(f.nJ);
      DevBuf th((size_t)m * nJp * 2, s), tl((size_t)m * nJp * 2, s);
      tc_transpose_split(t.p, DType::F32, 1, f.nJ, m, th.p, tl.p, TcElt::F16, sct.as<float>(), s);
      tc_inv_prod(sct.as<float>(), f.tc_scale + 4, fac.as<float>(), s);      // 1 / (s_t s_ov)
      tc_contract(th.p, tl.p, m, 1, f.nJ, f.JovT_hi, f.JovT_lo, ov, Jb.as<float>(), false, TcElt::F16,
                  fac.as<float>(), d.tc_err, s, nullptr, 0.0, 0.0, kCoulombKb);
    } else {
      DevBuf t((size_t)f.nJ * m * ew, s);
      sk_gram(f.Jov, f.dt, ov, f.nJ, Xw, tw, ov, m, ov, t.p, tw, m, 1.0, 0.0, s);
      sk_combo(t.p, tw, 1, m, m, f.nJ, f.Jov, f.dt, ov, ov, Jb.p, tw, ov, 1.0, 0.0, s);
    }
    have_J = true;
  }
  if (d.c_J != 0.0) {
    // sum_g w_g F^g_ia (F^g . X): rows stored as sqrt|w_g| F^g, one pass per sign
    const void* Fr[2] = {f.Fpos, f.Fneg};
    const int nr[2] = {f.nFpos, f.nFneg};
    for (int k = 0; k < 2; ++k) {
      if (nr[k] <= 0) continue;
      if (!have_J) Jb = DevBuf(mov * ew, s);
      DevBuf t((size_t)nr[k] * m * ew, s);
      sk_gram(Fr[k], f.dt, ov, nr[k], Xw, tw, ov, m, ov, t.p, tw, m, 1.0, 0.0, s);
      sk_combo(t.p, tw, 1, m, m, nr[k], Fr[k], f.dt, ov, ov, Jb.p, tw, ov, k == 0 ? 1.0 : -1.0,
               have_J ? 1.0 : 0.0, s);
      have_J = true;
    }
  }

  // ---- exchange: K1 (and K2 for the paired products) of one factor set
  const bool need_k2 = (mode == OpMode::PAIRED);
  auto exchange = [&](const FactorSet& f, DevBuf& K1b, DevBuf& K2b) {
    K1b = DevBuf(mov * ew, s);
    if (need_k2) K2b = DevBuf(mov * ew, s);
    const bool use_tc = tensor_cores && !f64 && f.Kvv_hi && f.Kvo_hi && f.Koo_hi && f.Kovp_hi;
    TD_REQUIRE(!tensor_cores || f64 || use_tc, TDDFT_ERR_ARG, "tensor-core factor copies missing");
    const int pc = chunk_rows(f.nK, (long long)m * ov * (long long)ew, m, use_tc ? kChunkBytesTC : kChunkBytes);
    const size_t es = dtype_size(f.dt);
    // 16-bit tensor-core operand pointer at element offset o
    auto at16 = [](const void* b, size_t o) { return static_cast<const void*>(static_cast<const uint16_t*>(b) + o); };
    if (use_tc && f.fp8) {
      // ris exchange rows in FP8 e4m3 (one scale per row P): the stage-1
      // products Z = L_oo X and Q = L_ov X^T run as for BF16 (trial vectors as
      // BF16 hi + lo against the BF16 rows) and leave their results as e4m3
      // hi + lo, multiplied by mu_P; the second contractions run as
      // kind::f8f6f4 (two products: hi and lo against the e4m3 rows) and the
      // sums are multiplied back by 1/g (tc_fp8_scales).
      TD_REQUIRE(f.Kvv8 && f.Kvo8 && f.s_vv, TDDFT_ERR_ARG, "FP8 ris copies missing");
      const int nvp = tc_pad(nv), nop = tc_pad(no), nv16 = tc_pad16(nv), no16 = tc_pad16(no);
      const DType xt = x32 ? DType::F32 : DType::F64;
      DevBuf sc((size_t)(2 + 2 * f.nK) * 4, s), kap(16, s);
      tc_fp8_scales(X, xt, m, no, nv, f.s_vv, f.rho_oo, f.s_vo, f.rho_ov, f.nK, sc.as<float>(), kap.as<unsigned>(), s);
      const float* inv1 = sc.as<float>();
      const float* inv2 = inv1 + 1;
      const float* mu1 = inv1 + 2;
      const float* mu2 = mu1 + f.nK;
      DevBuf Xt_hi((size_t)m * nv * nop * 2, s), Xt_lo((size_t)m * nv * nop * 2, s), Xs_hi, Xs_lo;
      tc_transpose_split(X, xt, m, no, nv, Xt_hi.p, Xt_lo.p, TcElt::BF16, nullptr, s);
      if (need_k2) {
        Xs_hi = DevBuf((size_t)m * no * nvp * 2, s);
        Xs_lo = DevBuf((size_t)m * no * nvp * 2, s);
        tc_pad_split(X, xt, (long long)m * no, nv, Xs_hi.p, Xs_lo.p, TcElt::BF16, nullptr, s);
      }
      DevBuf Zhi((size_t)m * no * pc * nv16, s), Zlo((size_t)m * no * pc * nv16, s), Qhi, Qlo;
      if (need_k2) {
        Qhi = DevBuf((size_t)m * no * pc * no16, s);
        Qlo = DevBuf((size_t)m * no * pc * no16, s);
      }
      const int Mz = m * no;
      for (int p0 = 0; p0 < f.nK; p0 += pc) {
        const int pn = (f.nK - p0 < pc) ? f.nK - p0 : pc;
        tc_stage1_fp8(Xt_hi.as<__nv_bfloat16>(), Xt_lo.as<__nv_bfloat16>(), m * nv, no,
                      static_cast<const __nv_bfloat16*>(f.Koo_hi) + (size_t)p0 * no * nop, no, pn, nv, mu1 + p0,
                      Zhi.as<unsigned char>(),
                      Zlo.as<unsigned char>(), d.tc_err, s);
        tc_contract8(Zhi.as<unsigned char>(), Zlo.as<unsigned char>(), Mz, pn, nv,
                     f.Kvv8 + (size_t)p0 * nv * nv16, nv, K1b.as<float>(), p0 > 0, inv1, d.tc_err, s);
        if (need_k2) {
          tc_stage1_fp8(Xs_hi.as<__nv_bfloat16>(), Xs_lo.as<__nv_bfloat16>(), m * no, nv,
                        static_cast<const __nv_bfloat16*>(f.Kovp_hi) + (size_t)p0 * no * nvp, no, pn, no, mu2 + p0,
                        Qhi.as<unsigned char>(),
                        Qlo.as<unsigned char>(), d.tc_err, s);
          tc_contract8(Qhi.as<unsigned char>(), Qlo.as<unsigned char>(), Mz, pn, no,
                       f.Kvo8 + (size_t)p0 * nv * no16, nv, K2b.as<float>(), p0 > 0, inv2, d.tc_err, s);
        }
      }
    } else if (use_tc) {
      // Both contractions of K1 and of K2 on the tensor cores.  The trial block
      // enters twice: transposed per vector ([(n,a)][j]) for Z = L_oo X and as is
      // ([(n,j)][b]) for Q = L_ov X^T, always as hi + lo (so Z and Q are too).
      // Exact factor sets (FP16): the factors are split hi + lo as well (three
      // products); every operand carries a power of two (tc_f16_product_scales)
      // that the contractions' sums remove.  ris factor sets (BF16): the
      // factors are used as they are (two products, exact with respect to them).
      const bool f16 = f.tc_elt == TcElt::F16;
      TD_REQUIRE(!f16 || (f.Kvv_lo && f.Kvo_lo && f.Koo_lo && f.Kovp_lo && f.tc_scale), TDDFT_ERR_ARG,
                 "FP16 factor parts missing");
      const TcElt et = f.tc_elt;
      const int nvp = tc_pad(nv), nop = tc_pad(no);
      const DType xt = x32 ? DType::F32 : DType::F64;
      DevBuf sc, kap;
      const float* sx = nullptr;
      const float *mz = nullptr, *mq = nullptr, *f1 = nullptr, *f2 = nullptr;
      if (f16) {
        sc = DevBuf(8 * 4, s);
        kap = DevBuf(16, s);
        tc_f16_product_scales(X, xt, m, no, nv, f.tc_scale, sc.as<float>(), kap.as<unsigned>(), s);
        sx = sc.as<float>();
        mz = sx + 1; mq = sx + 2; f1 = sx + 3; f2 = sx + 4;
      }
      DevBuf Xt_hi((size_t)m * nv * nop * 2, s), Xt_lo((size_t)m * nv * nop * 2, s), Xs_hi, Xs_lo;
      tc_transpose_split(X, xt, m, no, nv, Xt_hi.p, Xt_lo.p, et, sx, s);
      if (need_k2) {
        Xs_hi = DevBuf((size_t)m * no * nvp * 2, s);
        Xs_lo = DevBuf((size_t)m * no * nvp * 2, s);
        tc_pad_split(X, xt, (long long)m * no, nv, Xs_hi.p, Xs_lo.p, et, sx, s);
      }
      DevBuf Zhi((size_t)m * no * pc * nvp * 2, s), Zlo((size_t)m * no * pc * nvp * 2, s), Qhi, Qlo;
      if (need_k2) {
        Qhi = DevBuf((size_t)m * no * pc * nop * 2, s);
        Qlo = DevBuf((size_t)m * no * pc * nop * 2, s);
      }
      const int Mz = m * no;
      for (int p0 = 0; p0 < f.nK; p0 += pc) {
        const int pn = (f.nK - p0 < pc) ? f.nK - p0 : pc;
        tc_stage1(Xt_hi.p, Xt_lo.p, m * nv, no, at16(f.Koo_hi, (size_t)p0 * no * nop),
                  f16 ? at16(f.Koo_lo, (size_t)p0 * no * nop) : nullptr, no, pn, nv, et, mz, Zhi.p, Zlo.p,
                  d.tc_err, s);
        const bool timed = d.prof && d.prof->on && f16;
        tc_contract(Zhi.p, Zlo.p, Mz, pn, nv, at16(f.Kvv_hi, (size_t)p0 * nv * nvp),
                    f16 ? at16(f.Kvv_lo, (size_t)p0 * nv * nvp) : nullptr, nv, K1b.as<float>(), p0 > 0, et, f1,
                    d.tc_err, s, timed ? d.prof : nullptr, 2.0 * Mz * (double)nv * (double)pn * nv,
                    // Z hi+lo [Mz][pn*nv], L_vv chunk [pn*nv][nv] (hi+lo for FP16), K1 FP32
                    // written (and read back when accumulating)
                    4.0 * Mz * (double)pn * nv + (f16 ? 4.0 : 2.0) * (double)pn * nv * nv +
                        4.0 * Mz * (double)nv * (p0 > 0 ? 2.0 : 1.0),
                    f16 ? kExchangeKb : 0);
        if (need_k2) {
          tc_stage1(Xs_hi.p, Xs_lo.p, m * no, nv, at16(f.Kovp_hi, (size_t)p0 * no * nvp),
                    f16 ? at16(f.Kovp_lo, (size_t)p0 * no * nvp) : nullptr, no, pn, no, et, mq, Qhi.p, Qlo.p,
                    d.tc_err, s);
          tc_contract(Qhi.p, Qlo.p, Mz, pn, no, at16(f.Kvo_hi, (size_t)p0 * nv * nop),
                      f16 ? at16(f.Kvo_lo, (size_t)p0 * nv * nop) : nullptr, nv, K2b.as<float>(), p0 > 0, et, f2,
                      d.tc_err, s, nullptr, 0.0, 0.0, f16 ? kExchangeKb : 0);
        }
      }
    } else {
      DevBuf Zb((size_t)m * no * pc * nv * ew, s);
      DevBuf Qb;
      if (need_k2) Qb = DevBuf((size_t)m * no * pc * no * ew, s);
      for (int p0 = 0; p0 < f.nK; p0 += pc) {
        const int pn = (f.nK - p0 < pc) ? f.nK - p0 : pc;
        // Z[n][i][P][a] = sum_j Koo[P][i][j] X[n][j][a]
        GemmDesc z;
        z.acc64 = f64;
        z.M = no; z.N = nv; z.K = no;
        z.A = (const char*)f.Koo + (size_t)p0 * no * no * es; z.ta = f.dt; z.sam = no; z.sak = 1;
        z.B = Xw; z.tb = tw; z.sbk = nv; z.sbn = 1;
        z.C = Zb.p; z.tc = tw; z.scm = (long long)pn * nv; z.scn = 1;
        z.nb0 = pn; z.nb1 = m;
        z.sA0 = (long long)no * no; z.sB0 = 0; z.sC0 = nv;
        z.sA1 = 0; z.sB1 = ov; z.sC1 = (long long)no * pn * nv;
        gemm(z, s);
        const int Mz = m * no;
        const long long Kz = (long long)pn * nv;
        const bool timed = d.prof_simt && d.prof_simt->on && f.dt != DType::BF16;
        if (timed) d.prof_simt->begin(s);
        GemmDesc k;
        k.acc64 = f64;
        k.M = Mz; k.N = nv; k.K = (int)Kz;
        k.A = Zb.p; k.ta = tw; k.sam = Kz; k.sak = 1;
        k.B = (const char*)f.Kvv + (size_t)p0 * nv * nv * es; k.tb = f.dt; k.sbk = nv; k.sbn = 1;
        k.C = K1b.p; k.tc = tw; k.scm = nv; k.scn = 1;
        k.beta = (p0 > 0) ? 1.0 : 0.0;
        gemm_splitk(k, auto_splits(k.M, k.N, k.K), s);
        if (timed)
          d.prof_simt->end(s, 2.0 * Mz * (double)nv * (double)Kz,
                           (double)ew * Mz * (double)Kz + (double)es * Kz * nv +
                               (double)ew * Mz * nv * (p0 > 0 ? 2.0 : 1.0));
        if (need_k2) {
          // Q[n][i][P][j] = sum_b Kov[P][i][b] X[n][j][b]
          GemmDesc q;
          q.acc64 = f64;
          q.M = no; q.N = no; q.K = nv;
          q.A = (const char*)f.Kov + (size_t)p0 * ov * es; q.ta = f.dt; q.sam = nv; q.sak = 1;
          q.B = Xw; q.tb = tw; q.sbk = 1; q.sbn = nv;
          q.C = Qb.p; q.tc = tw; q.scm = (long long)pn * no; q.scn = 1;
          q.nb0 = pn; q.nb1 = m;
          q.sA0 = ov; q.sB0 = 0; q.sC0 = no;
          q.sA1 = 0; q.sB1 = ov; q.sC1 = (long long)no * pn * no;
          gemm(q, s);
          GemmDesc k2;
          k2.acc64 = f64;
          k2.M = m * no; k2.N = nv; k2.K = pn * no;
          k2.A = Qb.p; k2.ta = tw; k2.sam = (long long)pn * no; k2.sak = 1;
          k2.B = (const char*)f.Kov + (size_t)p0 * ov * es; k2.tb = f.dt; k2.sbk = nv; k2.sbn = 1;
          k2.C = K2b.p; k2.tc = tw; k2.scm = nv; k2.scn = 1;
          k2.beta = (p0 > 0) ? 1.0 : 0.0;
          gemm_splitk(k2, auto_splits(k2.M, k2.N, k2.K), s);
        }
      }
    }
  };
  DevBuf K1b, K2b;
  double kx = d.a_x;   // weight of the exchange parts in the final combination
  if (f.nK > 0 && d.a_x != 0.0) exchange(f, K1b, K2b);
  if (f.lr && f.b_x != 0.0 && f.lr->nK > 0) {
    // second exchange set: K = a_x K[L] + b_x K[M], combined with weight 1
    DevBuf L1, L2;
    exchange(*f.lr, L1, L2);
    const bool have = K1b.p != nullptr;
    if (!have) {
      K1b = DevBuf(mov * ew, s);
      if (need_k2) K2b = DevBuf(mov * ew, s);
    }
    axpby(K1b.p, L1.p, tw, have ? d.a_x : 0.0, f.b_x, mov, s);
    if (need_k2) axpby(K2b.p, L2.p, tw, have ? d.a_x : 0.0, f.b_x, mov, s);
    kx = 1.0;
  }

  const void* J = Jb.p;
  const void* K1 = K1b.p;
  const void* K2 = K2b.p;
  if constexpr (x32) {
    const float* Jf = static_cast<const float*>(J);
    const float* K1f = static_cast<const float*>(K1);
    const float* K2f = static_cast<const float*>(K2);
    if (mode == OpMode::TDA) {
      combine_f32(X, d.delta, Jf, K1f, nullptr, d.c_J, -kx, 0.0, m, ov, out0, s);
    } else {
      combine_f32(X, d.delta, Jf, K1f, K2f, 2.0 * d.c_J, -kx, -kx, m, ov, out0, s);
      combine_f32(X, d.delta, nullptr, K1f, K2f, 0.0, -kx, kx, m, ov, out1, s);
    }
  } else {
    if (mode == OpMode::TDA) {
      combine(X, d.delta, J, K1, nullptr, tw, d.c_J, -kx, 0.0, m, ov, out0, s);
    } else {
      combine(X, d.delta, J, K1, K2, tw, 2.0 * d.c_J, -kx, -kx, m, ov, out0, s);
      combine(X, d.delta, nullptr, K1, K2, tw, 0.0, -kx, kx, m, ov, out1, s);
    }
  }
}

void apply_operator(const OpDims& d, const FactorSet& f, const double* X, int m, OpMode mode,
                    double* out0, double* out1, int tc, cudaStream_t s) {
  apply_operator_t<double>(d, f, X, m, mode, out0, out1, tc, s);
}

void apply_operator(const OpDims& d, const FactorSet& f, const float* X, int m, OpMode mode,
                    float* out0, float* out1, int tc, cudaStream_t s) {
  apply_operator_t<float>(d, f, X, m, mode, out0, out1, tc, s);
}

}  // namespace tddft
