// C ABI (include/tddft.h): argument checking, factor staging, the request
// queue, and the translation of internal errors into status codes.  No call
// lets a C++ exception or a CUDA error escape; each returns a tddft_status.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

#include "ctx.cuh"
#include "tc_gemm.cuh"
#include "vecops.cuh"

using namespace tddft;

namespace {

thread_local std::string g_create_error;

tddft_status fail(Ctx* c, const std::exception& e, tddft_status st) {
  if (c) c->err = e.what();
  else g_create_error = e.what();
  return st;
}

// Copy `rows` rows of `row_elems` elements from a host or device array of type
// `tin` into device copies, chunk by chunk (bounded staging memory).
struct StageTarget {
  void* dst;        // device
  DType tout;       // F64, F32 or BF16
};

void stage_rows(const void* src, DType tin, bool on_device, long long rows, long long row_elems,
                const std::vector<StageTarget>& targets, cudaStream_t s) {
  if (rows == 0 || targets.empty()) return;
  const size_t es = dtype_size(tin);
  const long long total = rows * row_elems;
  long long chunk = (256ll << 20) / (long long)es;   // elements per staging chunk
  if (chunk > total) chunk = total;
  DevBuf stage;
  if (!on_device) stage = DevBuf((size_t)chunk * es, s);
  for (long long off = 0; off < total; off += chunk) {
    long long n = std::min(chunk, total - off);
    const void* in;
    if (on_device) {
      in = (const char*)src + off * es;
    } else {
      TD_CUDA(cudaMemcpyAsync(stage.p, (const char*)src + off * es, (size_t)n * es,
                              cudaMemcpyHostToDevice, s));
      in = stage.p;
    }
    for (const auto& t : targets) {
      convert(in, tin, (char*)t.dst + off * dtype_size(t.tout), t.tout, n, s);
    }
    if (!on_device) TD_CUDA(cudaStreamSynchronize(s));  // staging buffer reused
  }
}

// Device copies of one exact factor set: FP64 (PLAIN) and/or FP32 + FP16 hi/lo
// tensor-core operands (of the factors times a power of two per tensor) with
// rows padded for the TMA strides (MIXED).
void stage_exact(ExactCopies& e, const void* L_oo, const void* L_ov, const void* L_vv, long long A,
                 DType tin, bool dev, int no, int nv, bool p64, bool pmx, cudaStream_t s, bool coulomb = false) {
  const long long ov = (long long)no * nv;
  e.n = (int)A;
  if (p64) {
    e.f64_oo = DevBuf(A * no * no * 8, s);
    e.f64_ov = DevBuf(A * ov * 8, s);
    e.f64_vv = DevBuf(A * nv * nv * 8, s);
  }
  if (pmx) {
    e.f32_oo = DevBuf(A * no * no * 4, s);
    e.f32_ov = DevBuf(A * ov * 4, s);
    e.f32_vv = DevBuf(A * nv * nv * 4, s);
  }
  auto targets = [&](DevBuf& t64, DevBuf& t32) {
    std::vector<StageTarget> v;
    if (p64) v.push_back({t64.p, DType::F64});
    if (pmx) v.push_back({t32.p, DType::F32});
    return v;
  };
  stage_rows(L_oo, tin, dev, A, (long long)no * no, targets(e.f64_oo, e.f32_oo), s);
  stage_rows(L_ov, tin, dev, A, ov, targets(e.f64_ov, e.f32_ov), s);
  stage_rows(L_vv, tin, dev, A, (long long)nv * nv, targets(e.f64_vv, e.f32_vv), s);
  if (pmx) {
    // scale block: s_oo and the scaled largest L_oo row norm, s_vv, s_ov and the
    // scaled largest L_ov row norm (tc_f16_tensor_scale)
    e.tc_scale = DevBuf(8 * 4, s);
    TD_CUDA(cudaMemsetAsync(e.tc_scale.p, 0, 8 * 4, s));
    DevBuf scratch(8, s);
    float* sc = e.tc_scale.as<float>();
    tc_f16_tensor_scale(e.f32_oo.as<float>(), A * no, no, sc + 0, scratch.as<unsigned>(), s);
    tc_f16_tensor_scale(e.f32_vv.as<float>(), A * nv, nv, sc + 2, scratch.as<unsigned>(), s);
    tc_f16_tensor_scale(e.f32_ov.as<float>(), A * no, nv, sc + 4, scratch.as<unsigned>(), s);
    auto parts = [&](DevBuf& hi, DevBuf& lo, long long elems) {
      hi = DevBuf(elems * 2, s);
      lo = DevBuf(elems * 2, s);
    };
    parts(e.vv_hi, e.vv_lo, A * nv * tc_pad(nv));
    tc_pad_split(e.f32_vv.p, DType::F32, A * nv, nv, e.vv_hi.p, e.vv_lo.p, TcElt::F16, sc + 2, s);
    parts(e.vo_hi, e.vo_lo, A * nv * tc_pad(no));
    tc_transpose_split(e.f32_ov.p, DType::F32, (int)A, no, nv, e.vo_hi.p, e.vo_lo.p, TcElt::F16, sc + 4, s);
    parts(e.oo_hi, e.oo_lo, A * no * tc_pad(no));
    tc_pad_split(e.f32_oo.p, DType::F32, A * no, no, e.oo_hi.p, e.oo_lo.p, TcElt::F16, sc + 0, s);
    parts(e.ov_hi, e.ov_lo, A * no * tc_pad(nv));
    tc_pad_split(e.f32_ov.p, DType::F32, A * no, nv, e.ov_hi.p, e.ov_lo.p, TcElt::F16, sc + 4, s);
    if (coulomb) {   // L_ov transposed for the Coulomb term's second contraction
      parts(e.ovT_hi, e.ovT_lo, ov * tc_pad((int)A));
      tc_transpose_split(e.f32_ov.p, DType::F32, 1, (int)A, (int)ov, e.ovT_hi.p, e.ovT_lo.p, TcElt::F16, sc + 4, s);
    }
  }
}

// true when every element of the set's widest copy is finite
bool exact_finite(const ExactCopies& e, int no, int nv, bool p64, cudaStream_t s) {
  const long long A = e.n, ov = (long long)no * nv;
  DevBuf flag(4, s);
  TD_CUDA(cudaMemsetAsync(flag.p, 0, 4, s));
  if (p64) {
    check_finite(e.f64_ov.p, DType::F64, A * ov, flag.as<int>(), s);
    check_finite(e.f64_oo.p, DType::F64, A * no * no, flag.as<int>(), s);
    check_finite(e.f64_vv.p, DType::F64, A * nv * nv, flag.as<int>(), s);
  } else {
    check_finite(e.f32_ov.p, DType::F32, A * ov, flag.as<int>(), s);
    check_finite(e.f32_oo.p, DType::F32, A * no * no, flag.as<int>(), s);
    check_finite(e.f32_vv.p, DType::F32, A * nv * nv, flag.as<int>(), s);
  }
  int fh = 0;
  TD_CUDA(cudaMemcpyAsync(&fh, flag.p, 4, cudaMemcpyDeviceToHost, s));
  TD_CUDA(cudaStreamSynchronize(s));
  return fh == 0;
}

void worker_loop(Ctx* c) {
  cudaSetDevice(c->device);
  for (;;) {
    unsigned long long t;
    Request* r;
    {
      std::unique_lock<std::mutex> lk(c->mu);
      c->cv_work.wait(lk, [&] { return c->stopping || !c->queue.empty(); });
      if (c->stopping && c->queue.empty()) return;
      t = c->queue.front();
      c->queue.pop_front();
      r = &c->requests[t];
    }
    tddft_status st;
    try {
      tddft_request* q = r->req;
      std::lock_guard<std::mutex> run(c->run_mu);
      if (r->kind == 0) st = run_tda(*c, q->opts, q->omega, q->X, q->resid, &q->stats);
      else if (r->kind == 1) st = run_rpa(*c, q->opts, q->omega, q->X, q->Y, q->resid, &q->stats);
      else st = run_polar(*c, q->opts, q->mu, q->n_dip, q->freqs, q->n_freq, q->alpha, &q->stats);
    } catch (const Error& e) {
      std::lock_guard<std::mutex> lk(c->mu);
      c->err = e.what();
      st = e.status;
    } catch (const std::exception& e) {
      std::lock_guard<std::mutex> lk(c->mu);
      c->err = e.what();
      st = TDDFT_ERR_CUDA;
    }
    {
      std::lock_guard<std::mutex> lk(c->mu);
      r->status = st;
      r->done = true;
    }
    c->cv_done.notify_all();
  }
}

}  // namespace

namespace tddft {

unsigned long long factor_copy_bytes(const tddft_desc& d, bool coulomb) {
  const bool p64 = d.precisions & 1, pmx = d.precisions & 2;
  const double no = d.n_occ, nv = d.n_vir, ov = no * nv;
  const double nvv = (double)d.n_aux * nv * nv, noo = (double)d.n_aux * no * no, nov = (double)d.n_aux * ov;
  const double nr = (double)d.n_aux_ris_J * ov + (double)d.n_aux_ris_K * (no * no + nv * nv + ov);
  const double padded = nv * (tc_pad(d.n_vir) + tc_pad(d.n_occ)) + no * (tc_pad(d.n_occ) + tc_pad(d.n_vir));
  double bytes = 0.0;
  if (p64) bytes += 8.0 * (nvv + noo + nov + nr);
  // FP8 copies of the ris exchange rows: vv and ov^T padded to 16, four floats per row
  const double fp8 = (double)d.n_aux_ris_K * (nv * (tc_pad16(d.n_vir) + tc_pad16(d.n_occ)) + 16.0);
  // MIXED: FP32 copies, two FP16 parts of every padded exact operand (and of L_ov
  // transposed for the Coulomb term), BF16 ris rows and their padded copies
  if (pmx) bytes += 4.0 * (nvv + noo + nov) + 4.0 * (double)d.n_aux * padded +
                    (coulomb ? 4.0 * ov * tc_pad(d.n_aux) : 0.0) + 2.0 * nr +
                    2.0 * (double)d.n_aux_ris_K * padded + fp8;
  return (unsigned long long)bytes;
}

void ExactCopies::fill(FactorSet& f, int precision, bool coulomb) const {
  if (precision == TDDFT_PLAIN) {
    f.dt = DType::F64;
    if (coulomb) f.Jov = f64_ov.p;
    f.Koo = f64_oo.p; f.Kvv = f64_vv.p; f.Kov = f64_ov.p;
  } else {
    f.dt = DType::F32;
    if (coulomb) f.Jov = f32_ov.p;
    f.Koo = f32_oo.p; f.Kvv = f32_vv.p; f.Kov = f32_ov.p;
    f.tc_elt = TcElt::F16;
    f.tc_scale = tc_scale.as<float>();
    f.Kvv_hi = vv_hi.p;
    f.Kvv_lo = vv_lo.p;
    f.Kvo_hi = vo_hi.p;
    f.Kvo_lo = vo_lo.p;
    f.Koo_hi = oo_hi.p;
    f.Koo_lo = oo_lo.p;
    f.Kovp_hi = ov_hi.p;
    f.Kovp_lo = ov_lo.p;
    if (coulomb) {
      f.JovT_hi = ovT_hi.p;
      f.JovT_lo = ovT_lo.p;
    }
  }
}

FactorSet Ctx::exact(int precision) const {
  FactorSet f;
  f.nJ = naux;
  f.nK = naux;
  x.fill(f, precision, true);
  const int k = precision == TDDFT_PLAIN ? 0 : 1;
  if (lrx.n > 0 && b_x != 0.0) {
    f.lr = &lr_set[k];
    f.b_x = b_x;
  }
  const DevBuf* ker = precision == TDDFT_PLAIN ? ker64 : ker32;
  f.Fpos = ker[0].p; f.nFpos = n_ker[0];
  f.Fneg = ker[1].p; f.nFneg = n_ker[1];
  return f;
}

FactorSet Ctx::ris(int precision, bool fp8) const {
  FactorSet f;
  f.nJ = nJ;
  f.nK = nK;
  if (precision == TDDFT_PLAIN) {
    f.dt = DType::F64;
    f.Jov = r64_J.p; f.Koo = r64_Koo.p; f.Kvv = r64_Kvv.p; f.Kov = r64_Kov.p;
  } else {
    f.dt = DType::BF16;
    f.Jov = r16_J.p; f.Koo = r16_Koo.p; f.Kvv = r16_Kvv.p; f.Kov = r16_Kov.p;
    f.tc_elt = TcElt::BF16;
    f.Kvv_hi = r16_vvp.p;
    f.Kvo_hi = r16_vo.p;
    f.Koo_hi = r16_oop.p;
    f.Kovp_hi = r16_ovp.p;
    if (fp8 && nK > 0 && r8_vvp.p) {
      f.fp8 = true;
      f.Kvv8 = r8_vvp.as<unsigned char>();
      f.Kvo8 = r8_vo.as<unsigned char>();
      f.s_vv = r8_aux.as<float>();
      f.s_vo = f.s_vv + nK;
      f.rho_oo = f.s_vv + 2 * nK;
      f.rho_ov = f.s_vv + 3 * nK;
    }
  }
  return f;
}

}  // namespace tddft

extern "C" {

void tddft_default_opts(tddft_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precond = TDDFT_PRECOND_RID;
  o->n_states = 5;
  o->n_extra_guess = -1;
  o->tol = 1e-5;
  o->inner_tol = 1e-2;
  o->guess_tol = 1e-3;
  o->max_iter = 50;
  o->inner_max_iter = 20;
  o->max_subspace = 0;
  o->precision = TDDFT_PLAIN;
  o->tensor_cores = 0;
  o->outputs_on_device = 0;
  o->ris_fp8 = 0;
}

void tddft_default_desc(tddft_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->a_x = 0.25;
  d->coulomb_factor = 2.0;
  d->t_cut_ha = 40.0 / 27.211386245988;
  d->precisions = 3;
  d->hbm_budget_gb = 0.0;
}

tddft_status tddft_create(const tddft_desc* desc, const double* eps_occ, const double* eps_vir,
                          const void* L_oo, const void* L_ov, const void* L_vv, const void* Lr_oo,
                          const void* Lr_ov, const void* Lr_vv, const int* ris_K_index,
                          tddft_dtype dtype, int inputs_on_device, void* cuda_stream,
                          tddft_ctx** out) {
  Ctx* c = nullptr;
  try {
    TD_REQUIRE(out != nullptr && desc != nullptr, TDDFT_ERR_ARG, "null desc or out pointer");
    *out = nullptr;
    const tddft_desc& d = *desc;
    TD_REQUIRE(d.n_occ >= 1 && d.n_vir >= 1 && d.n_aux >= 1 && d.n_aux_ris_J >= 0 &&
                   d.n_aux_ris_K >= 0 && d.n_aux_ris_K <= d.n_aux_ris_J,
               TDDFT_ERR_ARG, "bad sizes in tddft_desc");
    TD_REQUIRE((long long)d.n_occ * d.n_vir < (1ll << 31), TDDFT_ERR_ARG, "n_occ*n_vir too large");
    TD_REQUIRE(eps_occ && eps_vir && L_oo && L_ov && L_vv, TDDFT_ERR_ARG, "null exact-factor input");
    TD_REQUIRE(d.n_aux_ris_J == 0 || Lr_ov, TDDFT_ERR_ARG, "null ris Coulomb factors");
    TD_REQUIRE(d.n_aux_ris_K == 0 || (Lr_oo && Lr_vv && ris_K_index), TDDFT_ERR_ARG,
               "null ris exchange factors");
    TD_REQUIRE(dtype == TDDFT_F64 || dtype == TDDFT_F32, TDDFT_ERR_ARG, "unknown dtype");
    TD_REQUIRE((d.precisions & 3) != 0, TDDFT_ERR_ARG, "precisions must keep at least one copy");
    TD_REQUIRE(std::isfinite(d.a_x) && std::isfinite(d.coulomb_factor) && std::isfinite(d.t_cut_ha),
               TDDFT_ERR_ARG, "non-finite a_x / coulomb_factor / t_cut");

    c = new Ctx();
    TD_CUDA(cudaGetDevice(&c->device));
    {
      // Solves allocate and free many small stream-ordered work buffers; keep the
      // device pool's memory mapped across synchronisations instead of returning
      // it to the driver at every sync (the default threshold of 0).
      cudaMemPool_t pool;
      TD_CUDA(cudaDeviceGetDefaultMemPool(&pool, c->device));
      uint64_t keep = ~0ull;
      TD_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    if (cuda_stream) {
      c->s = (cudaStream_t)cuda_stream;
    } else {
      TD_CUDA(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    cudaStream_t s = c->s;
    c->no = d.n_occ; c->nv = d.n_vir; c->ov = d.n_occ * d.n_vir;
    c->naux = d.n_aux; c->nJ = d.n_aux_ris_J; c->nK = d.n_aux_ris_K;
    c->a_x = d.a_x; c->c_J = d.coulomb_factor; c->t_cut = d.t_cut_ha;
    c->precisions = d.precisions & 3;
    const int no = c->no, nv = c->nv, ov = c->ov;
    const DType tin = dtype == TDDFT_F64 ? DType::F64 : DType::F32;
    const bool dev = inputs_on_device != 0;

    if (dev) {
      // device inputs written by work queued on the legacy default stream (as
      // PyTorch's default stream is) are read only after that work
      cudaEvent_t e;
      TD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      cudaError_t er = cudaEventRecord(e, cudaStreamLegacy);
      if (er == cudaSuccess) er = cudaStreamWaitEvent(s, e, 0);
      cudaEventDestroy(e);
      TD_CUDA(er);
    }

    // orbital energies (host copy for the window and the guess order)
    std::vector<double> eo(no), ev(nv);
    cudaMemcpyKind k = dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    // on the context's stream: no wait on work that other contexts queued
    TD_CUDA(cudaMemcpyAsync(eo.data(), eps_occ, no * 8, k, s));
    TD_CUDA(cudaMemcpyAsync(ev.data(), eps_vir, nv * 8, k, s));
    TD_CUDA(cudaStreamSynchronize(s));
    for (double x : eo) TD_REQUIRE(std::isfinite(x), TDDFT_ERR_ARG, "non-finite orbital energy");
    for (double x : ev) TD_REQUIRE(std::isfinite(x), TDDFT_ERR_ARG, "non-finite orbital energy");
    TD_REQUIRE(std::is_sorted(eo.begin(), eo.end()) && std::is_sorted(ev.begin(), ev.end()),
               TDDFT_ERR_ARG, "orbital energies must be ascending");
    std::vector<int> kidx;
    if (d.n_aux_ris_K > 0) {
      kidx.resize(d.n_aux_ris_K);
      TD_CUDA(cudaMemcpyAsync(kidx.data(), ris_K_index, kidx.size() * 4, k, s));
      TD_CUDA(cudaStreamSynchronize(s));
      for (int r : kidx) TD_REQUIRE(r >= 0 && r < d.n_aux_ris_J, TDDFT_ERR_ARG, "ris_K_index out of range");
    }

    // memory admission
    const bool p64 = c->precisions & 1, pmx = c->precisions & 2;
    c->desc = d;
    const double bytes = (double)factor_copy_bytes(d);
    size_t fr = 0, tot = 0;
    TD_CUDA(cudaMemGetInfo(&fr, &tot));
    double budget = d.hbm_budget_gb > 0 ? d.hbm_budget_gb * 1e9 : (double)fr - 2e9;
    if (bytes > budget) {
      throw Error(TDDFT_ERR_OOM, "factor copies need " + std::to_string(bytes / 1e9) +
                                     " GB, budget " + std::to_string(budget / 1e9) + " GB");
    }
    c->device_bytes = (unsigned long long)bytes;

    c->tc_err = DevBuf(4, s);
    TD_CUDA(cudaMemsetAsync(c->tc_err.p, 0, 4, s));
    c->eps_o = DevBuf(no * 8, s);
    c->eps_v = DevBuf(nv * 8, s);
    c->delta = DevBuf((size_t)ov * 8, s);
    TD_CUDA(cudaMemcpyAsync(c->eps_o.p, eo.data(), no * 8, cudaMemcpyHostToDevice, s));
    TD_CUDA(cudaMemcpyAsync(c->eps_v.p, ev.data(), nv * 8, cudaMemcpyHostToDevice, s));
    delta_kernel(c->eps_o.as<double>(), c->eps_v.as<double>(), no, nv, c->delta.as<double>(), s);
    {
      // order of Delta ascending (ties by index), for the unit-vector guesses
      std::vector<double> dl(ov);
      for (int i = 0; i < no; ++i)
        for (int a = 0; a < nv; ++a) dl[(size_t)i * nv + a] = ev[a] - eo[i];
      std::vector<int> ord(ov);
      std::iota(ord.begin(), ord.end(), 0);
      c->n_order = std::min(ov, 4096);
      std::partial_sort(ord.begin(), ord.begin() + c->n_order, ord.end(), [&](int x, int y) {
        return dl[x] < dl[y] || (dl[x] == dl[y] && x < y);
      });
      c->order = DevBuf(c->n_order * 4, s);
      TD_CUDA(cudaMemcpyAsync(c->order.p, ord.data(), c->n_order * 4, cudaMemcpyHostToDevice, s));
      TD_CUDA(cudaStreamSynchronize(s));
    }

    // exact factors
    const long long A = d.n_aux;
    stage_exact(c->x, L_oo, L_ov, L_vv, A, tin, dev, no, nv, p64, pmx, s, true);

    // ris factors (Coulomb rows all; exchange rows windowed, Sec. 3.1)
    const long long RJ = d.n_aux_ris_J, RK = d.n_aux_ris_K;
    if (RJ > 0) {
      if (p64) c->r64_J = DevBuf(RJ * ov * 8, s);
      if (pmx) c->r16_J = DevBuf(RJ * ov * 2, s);
      std::vector<StageTarget> v;
      if (p64) v.push_back({c->r64_J.p, DType::F64});
      if (pmx) v.push_back({c->r16_J.p, DType::BF16});
      stage_rows(Lr_ov, tin, dev, RJ, ov, v, s);
    }
    if (RK > 0) {
      std::vector<unsigned char> mo(no), mv(nv);
      for (int i = 0; i < no; ++i) mo[i] = eo[i] >= ev[0] - d.t_cut_ha;
      for (int a = 0; a < nv; ++a) mv[a] = ev[a] <= eo[no - 1] + d.t_cut_ha;
      DevBuf dmo(no, s), dmv(nv, s);
      TD_CUDA(cudaMemcpyAsync(dmo.p, mo.data(), no, cudaMemcpyHostToDevice, s));
      TD_CUDA(cudaMemcpyAsync(dmv.p, mv.data(), nv, cudaMemcpyHostToDevice, s));
      if (p64) {
        c->r64_Koo = DevBuf(RK * no * no * 8, s);
        c->r64_Kvv = DevBuf(RK * nv * nv * 8, s);
        c->r64_Kov = DevBuf(RK * ov * 8, s);
      }
      if (pmx) {
        c->r16_Koo = DevBuf(RK * no * no * 2, s);
        c->r16_Kvv = DevBuf(RK * nv * nv * 2, s);
        c->r16_Kov = DevBuf(RK * ov * 2, s);
      }
      std::vector<StageTarget> voo, vvv;
      if (p64) { voo.push_back({c->r64_Koo.p, DType::F64}); vvv.push_back({c->r64_Kvv.p, DType::F64}); }
      if (pmx) { voo.push_back({c->r16_Koo.p, DType::BF16}); vvv.push_back({c->r16_Kvv.p, DType::BF16}); }
      stage_rows(Lr_oo, tin, dev, RK, (long long)no * no, voo, s);
      stage_rows(Lr_vv, tin, dev, RK, (long long)nv * nv, vvv, s);
      for (long long r = 0; r < RK; ++r) {
        if (p64)
          TD_CUDA(cudaMemcpyAsync(c->r64_Kov.as<double>() + r * ov, c->r64_J.as<double>() + (long long)kidx[r] * ov,
                                  (size_t)ov * 8, cudaMemcpyDeviceToDevice, s));
        if (pmx)
          TD_CUDA(cudaMemcpyAsync(c->r16_Kov.as<__nv_bfloat16>() + r * ov,
                                  c->r16_J.as<__nv_bfloat16>() + (long long)kidx[r] * ov, (size_t)ov * 2,
                                  cudaMemcpyDeviceToDevice, s));
      }
      if (p64) {
        mask_block(c->r64_Koo.p, DType::F64, (int)RK, no, no, dmo.as<unsigned char>(), dmo.as<unsigned char>(), s);
        mask_block(c->r64_Kvv.p, DType::F64, (int)RK, nv, nv, dmv.as<unsigned char>(), dmv.as<unsigned char>(), s);
        mask_block(c->r64_Kov.p, DType::F64, (int)RK, no, nv, dmo.as<unsigned char>(), dmv.as<unsigned char>(), s);
      }
      if (pmx) {
        mask_block(c->r16_Koo.p, DType::BF16, (int)RK, no, no, dmo.as<unsigned char>(), dmo.as<unsigned char>(), s);
        mask_block(c->r16_Kvv.p, DType::BF16, (int)RK, nv, nv, dmv.as<unsigned char>(), dmv.as<unsigned char>(), s);
        mask_block(c->r16_Kov.p, DType::BF16, (int)RK, no, nv, dmo.as<unsigned char>(), dmv.as<unsigned char>(), s);
        // padded tensor-core copies (vv is symmetric, so its transpose is itself)
        c->r16_vvp = DevBuf(RK * nv * tc_pad(nv) * 2, s);
        c->r16_vo = DevBuf(RK * nv * tc_pad(no) * 2, s);
        tc_transpose_split(c->r16_Kvv.p, DType::BF16, (int)RK, nv, nv, c->r16_vvp.p, nullptr, TcElt::BF16,
                           nullptr, s);
        tc_transpose_split(c->r16_Kov.p, DType::BF16, (int)RK, no, nv, c->r16_vo.p, nullptr, TcElt::BF16,
                           nullptr, s);
        c->r16_oop = DevBuf(RK * no * tc_pad(no) * 2, s);
        c->r16_ovp = DevBuf(RK * no * tc_pad(nv) * 2, s);
        tc_pad_split(c->r16_Koo.p, DType::BF16, RK * no, no, c->r16_oop.p, nullptr, TcElt::BF16, nullptr, s);
        tc_pad_split(c->r16_Kov.p, DType::BF16, RK * no, nv, c->r16_ovp.p, nullptr, TcElt::BF16, nullptr, s);
        // FP8 e4m3 copies with a scale per row (opts.ris_fp8), from the windowed BF16 rows
        c->r8_vvp = DevBuf(RK * nv * tc_pad16(nv), s);
        c->r8_vo = DevBuf(RK * nv * tc_pad16(no), s);
        c->r8_aux = DevBuf(RK * 4 * 4, s);
        float* aux = c->r8_aux.as<float>();
        tc_quant_e4m3(c->r16_Kvv.as<__nv_bfloat16>(), (int)RK, nv, nv, c->r8_vvp.as<unsigned char>(), aux, s);
        tc_quant_e4m3(c->r16_Kov.as<__nv_bfloat16>(), (int)RK, no, nv, c->r8_vo.as<unsigned char>(), aux + RK, s);
        tc_row_norm_max(c->r16_Koo.as<__nv_bfloat16>(), (int)RK, no, no, aux + 2 * RK, s);
        tc_row_norm_max(c->r16_Kov.as<__nv_bfloat16>(), (int)RK, no, nv, aux + 3 * RK, s);
      }
      TD_CUDA(cudaStreamSynchronize(s));
    }
    // reject non-finite factors
    {
      DevBuf flag(4, s);
      TD_CUDA(cudaMemsetAsync(flag.p, 0, 4, s));
      TD_REQUIRE(exact_finite(c->x, no, nv, p64, s), TDDFT_ERR_INDEFINITE, "non-finite values in the factors");
    }
    c->worker = std::thread(worker_loop, c);
    *out = reinterpret_cast<tddft_ctx*>(c);
    return TDDFT_OK;
  } catch (const Error& e) {
    tddft_status st = e.status;
    g_create_error = e.what();
    if (c) tddft_destroy(reinterpret_cast<tddft_ctx*>(c));
    return st;
  } catch (const std::exception& e) {
    g_create_error = e.what();
    if (c) tddft_destroy(reinterpret_cast<tddft_ctx*>(c));
    return TDDFT_ERR_CUDA;
  }
}

#define TD_API_BODY(ctxp, ...)                                                           \
  Ctx* c = reinterpret_cast<Ctx*>(ctxp);                                                  \
  if (!c) return TDDFT_ERR_ARG;                                                           \
  try {                                                                                   \
    __VA_ARGS__;                                                                          \
  } catch (const Error& e) {                                                              \
    return fail(c, e, e.status);                                                          \
  } catch (const std::exception& e) {                                                     \
    return fail(c, e, TDDFT_ERR_CUDA);                                                    \
  }

tddft_status tddft_solve_tda(tddft_ctx* ctx, const tddft_opts* opts, double* omega, double* X,
                             double* resid, tddft_stats* stats) {
  TD_API_BODY(ctx, {
    TD_REQUIRE(opts != nullptr, TDDFT_ERR_ARG, "null opts");
    std::lock_guard<std::mutex> run(c->run_mu);
    return run_tda(*c, *opts, omega, X, resid, stats);
  })
}

tddft_status tddft_solve_rpa(tddft_ctx* ctx, const tddft_opts* opts, double* omega, double* X,
                             double* Y, double* resid, tddft_stats* stats) {
  TD_API_BODY(ctx, {
    TD_REQUIRE(opts != nullptr, TDDFT_ERR_ARG, "null opts");
    std::lock_guard<std::mutex> run(c->run_mu);
    return run_rpa(*c, *opts, omega, X, Y, resid, stats);
  })
}

tddft_status tddft_solve_polar(tddft_ctx* ctx, const tddft_opts* opts, const double* mu, int n_dip,
                               const double* omega, int n_freq, double* alpha, tddft_stats* stats) {
  TD_API_BODY(ctx, {
    TD_REQUIRE(opts != nullptr, TDDFT_ERR_ARG, "null opts");
    std::lock_guard<std::mutex> run(c->run_mu);
    return run_polar(*c, *opts, mu, n_dip, omega, n_freq, alpha, stats);
  })
}

tddft_status tddft_apply(tddft_ctx* ctx, int kind, int precision, int tensor_cores, const double* X,
                         int m, double* out0, double* out1, int on_device) {
  TD_API_BODY(ctx, {
    TD_REQUIRE(kind >= 0 && kind <= 3, TDDFT_ERR_ARG, "kind must be 0..3");
    TD_REQUIRE(precision == TDDFT_PLAIN || precision == TDDFT_MIXED, TDDFT_ERR_ARG, "bad precision");
    TD_REQUIRE((c->precisions & (precision == TDDFT_PLAIN ? 1 : 2)) != 0, TDDFT_ERR_ARG,
               "context lacks the factor copies for this precision");
    TD_REQUIRE(!(tensor_cores && precision != TDDFT_MIXED), TDDFT_ERR_ARG, "tensor_cores needs MIXED");
    TD_REQUIRE(m >= 0 && X && out0 && ((kind & 1) == 0 || out1), TDDFT_ERR_ARG, "bad buffers");
    if (m == 0) return TDDFT_OK;
    std::lock_guard<std::mutex> run(c->run_mu);
    cudaStream_t s = c->s;
    const size_t n = (size_t)m * c->ov;
    const bool ris = kind >= 2;
    const bool paired = kind & 1;
    TD_REQUIRE(tensor_cores >= 0 && tensor_cores <= 2, TDDFT_ERR_ARG, "tensor_cores must be 0..2");
    FactorSet f = ris ? c->ris(precision, tensor_cores == 2) : c->exact(precision);
    DevBuf xb, o0, o1;
    const double* Xd = X;
    double* d0 = out0;
    double* d1 = out1;
    if (!on_device) {
      xb = DevBuf(n * 8, s);
      TD_CUDA(cudaMemcpyAsync(xb.p, X, n * 8, cudaMemcpyHostToDevice, s));
      Xd = xb.as<double>();
      o0 = DevBuf(n * 8, s);
      d0 = o0.as<double>();
      if (paired) { o1 = DevBuf(n * 8, s); d1 = o1.as<double>(); }
    }
    g_launches = 0;
    apply_operator(c->dims(), f, Xd, m, paired ? OpMode::PAIRED : OpMode::TDA, d0, paired ? d1 : nullptr,
                   tensor_cores != 0 ? 1 : 0, s);
    if (!on_device) {
      TD_CUDA(cudaMemcpyAsync(out0, d0, n * 8, cudaMemcpyDeviceToHost, s));
      if (paired) TD_CUDA(cudaMemcpyAsync(out1, d1, n * 8, cudaMemcpyDeviceToHost, s));
    }
    TD_CUDA(cudaStreamSynchronize(s));
    check_tc_error(*c);
    return TDDFT_OK;
  })
}

tddft_status tddft_submit(tddft_ctx* ctx, int kind, tddft_request* req, unsigned long long* ticket) {
  TD_API_BODY(ctx, {
    TD_REQUIRE(req && ticket && kind >= 0 && kind <= 2, TDDFT_ERR_ARG, "bad request");
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->queue.size() >= 4096) return TDDFT_ERR_BUSY;
    unsigned long long t = c->next_ticket++;
    Request r;
    r.kind = kind;
    r.req = req;
    c->requests[t] = r;
    c->queue.push_back(t);
    *ticket = t;
    c->cv_work.notify_one();
    return TDDFT_OK;
  })
}

tddft_status tddft_poll(tddft_ctx* ctx, unsigned long long ticket, int timeout_ms) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return TDDFT_ERR_ARG;
  std::unique_lock<std::mutex> lk(c->mu);
  auto it = c->requests.find(ticket);
  if (it == c->requests.end()) return TDDFT_ERR_ARG;
  if (!it->second.done && timeout_ms > 0) {
    c->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
      auto j = c->requests.find(ticket);
      return j != c->requests.end() && j->second.done;
    });
    it = c->requests.find(ticket);
  }
  if (!it->second.done) return timeout_ms > 0 ? TDDFT_ERR_TIMEOUT : TDDFT_PENDING;
  tddft_status st = it->second.status;
  c->requests.erase(it);
  return st;
}

void tddft_destroy(tddft_ctx* ctx) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    c->stopping = true;
  }
  c->cv_work.notify_all();
  if (c->worker.joinable()) c->worker.join();
  if (c->s) cudaStreamSynchronize(c->s);
  cudaStream_t s = c->s;
  bool own = c->own_stream;
  delete c;  // DevBuf destructors free on the stream
  if (s) pool_trim(s);
  if (s) cudaStreamSynchronize(s);
  if (own && s) cudaStreamDestroy(s);
}

const char* tddft_last_error(const tddft_ctx* ctx) {
  const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

tddft_status tddft_profile(tddft_ctx* ctx, int enable) {
  TD_API_BODY(ctx, {
    std::lock_guard<std::mutex> run(c->run_mu);
    c->prof.reset();
    c->prof_simt.reset();
    c->prof.on = c->prof_simt.on = enable != 0;
    if (enable) {   // event creation stays out of the timed launches
      c->prof.reserve(8192);
      c->prof_simt.reserve(1024);
    }
    return TDDFT_OK;
  })
}

tddft_status tddft_profile_read(const tddft_ctx* ctx, int which, long long* launches, double* ms,
                                double* flops) {
  TD_API_BODY(const_cast<tddft_ctx*>(ctx), {
    TD_REQUIRE(which == 0 || which == 1, TDDFT_ERR_ARG, "which must be 0 or 1");
    std::lock_guard<std::mutex> run(c->run_mu);
    KernelProfile& kp = which == 0 ? c->prof : c->prof_simt;
    kp.collect();
    if (launches) *launches = kp.launches;
    if (ms) *ms = kp.ms;
    if (flops) *flops = kp.flops;
    return TDDFT_OK;
  })
}

tddft_status tddft_add_exchange(tddft_ctx* ctx, double b_x, int n_aux_lr, const void* M_oo, const void* M_ov,
                                const void* M_vv, tddft_dtype dtype, int inputs_on_device) {
  TD_API_BODY(ctx, {
    TD_REQUIRE(n_aux_lr >= 1 && M_oo && M_ov && M_vv, TDDFT_ERR_ARG, "bad second exchange set");
    TD_REQUIRE(std::isfinite(b_x), TDDFT_ERR_ARG, "non-finite b_x");
    TD_REQUIRE(dtype == TDDFT_F64 || dtype == TDDFT_F32, TDDFT_ERR_ARG, "unknown dtype");
    std::lock_guard<std::mutex> run(c->run_mu);
    TD_REQUIRE(c->lrx.n == 0, TDDFT_ERR_ARG, "the context already has a second exchange set");
    cudaStream_t s = c->s;
    const bool p64 = c->precisions & 1, pmx = c->precisions & 2;
    ExactCopies e;
    stage_exact(e, M_oo, M_ov, M_vv, n_aux_lr, dtype == TDDFT_F64 ? DType::F64 : DType::F32,
                inputs_on_device != 0, c->no, c->nv, p64, pmx, s);
    TD_REQUIRE(exact_finite(e, c->no, c->nv, p64, s), TDDFT_ERR_INDEFINITE,
               "non-finite values in the second exchange set");
    c->lrx = std::move(e);
    c->b_x = b_x;
    for (int k = 0; k < 2; ++k) {
      FactorSet f;
      f.nJ = 0;
      f.nK = n_aux_lr;
      if ((k == 0 && p64) || (k == 1 && pmx)) c->lrx.fill(f, k == 0 ? TDDFT_PLAIN : TDDFT_MIXED, false);
      c->lr_set[k] = f;
    }
    tddft_desc dl = c->desc;
    dl.n_aux = n_aux_lr;
    dl.n_aux_ris_J = dl.n_aux_ris_K = 0;
    c->device_bytes += factor_copy_bytes(dl, false);
    return TDDFT_OK;
  })
}

tddft_status tddft_add_kernel(tddft_ctx* ctx, int n_g, const double* w, const void* F_ov, tddft_dtype dtype,
                              int inputs_on_device) {
  TD_API_BODY(ctx, {
    TD_REQUIRE(n_g >= 1 && w && F_ov, TDDFT_ERR_ARG, "bad kernel term");
    TD_REQUIRE(dtype == TDDFT_F64 || dtype == TDDFT_F32, TDDFT_ERR_ARG, "unknown dtype");
    std::lock_guard<std::mutex> run(c->run_mu);
    TD_REQUIRE(c->n_ker[0] + c->n_ker[1] == 0, TDDFT_ERR_ARG, "the context already has a kernel term");
    cudaStream_t s = c->s;
    const long long ov = c->ov;
    std::vector<double> wh(n_g);
    if (inputs_on_device) {
      TD_CUDA(cudaMemcpyAsync(wh.data(), w, (size_t)n_g * 8, cudaMemcpyDeviceToHost, s));
      TD_CUDA(cudaStreamSynchronize(s));
    } else {
      std::memcpy(wh.data(), w, (size_t)n_g * 8);
    }
    for (double x : wh) TD_REQUIRE(std::isfinite(x), TDDFT_ERR_ARG, "non-finite kernel weight");
    // every row in FP64, then per sign: gather, scale by sqrt|w|, keep the copies
    DevBuf all((size_t)n_g * ov * 8, s);
    stage_rows(F_ov, dtype == TDDFT_F64 ? DType::F64 : DType::F32, inputs_on_device != 0, n_g, ov,
               {{all.p, DType::F64}}, s);
    {
      DevBuf flag(4, s);
      TD_CUDA(cudaMemsetAsync(flag.p, 0, 4, s));
      check_finite(all.p, DType::F64, (long long)n_g * ov, flag.as<int>(), s);
      int fh = 0;
      TD_CUDA(cudaMemcpyAsync(&fh, flag.p, 4, cudaMemcpyDeviceToHost, s));
      TD_CUDA(cudaStreamSynchronize(s));
      TD_REQUIRE(fh == 0, TDDFT_ERR_INDEFINITE, "non-finite values in the kernel rows");
    }
    const bool p64 = c->precisions & 1, pmx = c->precisions & 2;
    unsigned long long bytes = 0;
    for (int k = 0; k < 2; ++k) {
      std::vector<int> idx;
      std::vector<double> sc;
      for (int g = 0; g < n_g; ++g)
        if (k == 0 ? wh[g] > 0.0 : wh[g] < 0.0) {
          idx.push_back(g);
          sc.push_back(std::sqrt(std::fabs(wh[g])));
        }
      const int n = (int)idx.size();
      if (n == 0) continue;
      DevBuf di(n * 4, s), ds(n * 8, s), rows((size_t)n * ov * 8, s);
      TD_CUDA(cudaMemcpyAsync(di.p, idx.data(), n * 4, cudaMemcpyHostToDevice, s));
      TD_CUDA(cudaMemcpyAsync(ds.p, sc.data(), n * 8, cudaMemcpyHostToDevice, s));
      gather_rows(all.as<double>(), di.as<int>(), n, (int)ov, rows.as<double>(), s);
      scale_rows(rows.as<double>(), ds.as<double>(), n, (int)ov, s);
      if (pmx) {
        c->ker32[k] = DevBuf((size_t)n * ov * 4, s);
        convert(rows.p, DType::F64, c->ker32[k].p, DType::F32, (long long)n * ov, s);
        bytes += (unsigned long long)n * ov * 4;
      }
      if (p64) {
        c->ker64[k] = std::move(rows);
        bytes += (unsigned long long)n * ov * 8;
      }
      TD_CUDA(cudaStreamSynchronize(s));   // the host vectors above are copied from
      c->n_ker[k] = n;
    }
    c->device_bytes += bytes;
    return TDDFT_OK;
  })
}

tddft_status tddft_ctx_desc(const tddft_ctx* ctx, tddft_desc* desc) {
  const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
  if (!c || !desc) return TDDFT_ERR_ARG;
  *desc = c->desc;
  return TDDFT_OK;
}

tddft_status tddft_profile_records(const tddft_ctx* ctx, int which, int max_records, double* ms, double* flops,
                                   double* bytes, int* count) {
  TD_API_BODY(const_cast<tddft_ctx*>(ctx), {
    TD_REQUIRE(which == 0 || which == 1, TDDFT_ERR_ARG, "which must be 0 or 1");
    TD_REQUIRE(max_records >= 0 && count && (max_records == 0 || (ms && flops && bytes)), TDDFT_ERR_ARG,
               "bad record buffers");
    std::lock_guard<std::mutex> run(c->run_mu);
    KernelProfile& kp = which == 0 ? c->prof : c->prof_simt;
    kp.collect();
    const int n = (int)kp.rec_ms.size();
    const int k = std::min(n, max_records);
    for (int i = 0; i < k; ++i) {
      ms[i] = kp.rec_ms[i];
      flops[i] = kp.rec_flops[i];
      bytes[i] = kp.rec_bytes[i];
    }
    *count = n;
    return TDDFT_OK;
  })
}

unsigned long long tddft_device_bytes(const tddft_ctx* ctx) {
  const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
  return c ? c->device_bytes : 0ull;
}

tddft_status tddft_solve_tda_batch(tddft_ctx* const* ctxs, int n, const tddft_opts* opts, double* omega,
                                   double* resid, tddft_stats* stats, tddft_batch_info* info) {
  if (!ctxs || n < 1 || !ctxs[0] || !opts || !omega) return TDDFT_ERR_ARG;
  Ctx* c0 = reinterpret_cast<Ctx*>(ctxs[0]);
  try {
    std::vector<Ctx*> cs(n);
    for (int i = 0; i < n; ++i) {
      cs[i] = reinterpret_cast<Ctx*>(ctxs[i]);
      TD_REQUIRE(cs[i] != nullptr, TDDFT_ERR_ARG, "batch: null context");
    }
    std::vector<Ctx*> uniq(cs);
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    std::vector<std::unique_lock<std::mutex>> locks;   // one solve at a time per context
    for (Ctx* u : uniq) locks.emplace_back(u->run_mu);
    return solve_tda_batch(cs.data(), n, opts, omega, resid, stats, info);
  } catch (const Error& e) {
    return fail(c0, e, e.status);
  } catch (const std::exception& e) {
    return fail(c0, e, TDDFT_ERR_CUDA);
  }
}

tddft_status tddft_pool_usage(int device, unsigned long long* used_current,
                              unsigned long long* used_high, int reset_high) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return TDDFT_ERR_ARG;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) != cudaSuccess) return TDDFT_ERR_CUDA;
  uint64_t cur = 0, high = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &cur) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high) != cudaSuccess)
    return TDDFT_ERR_CUDA;
  if (used_current) *used_current = cur;
  if (used_high) *used_high = high;
  if (reset_high) {
    uint64_t zero = 0;   // restarts the high-water mark at the current use
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess) return TDDFT_ERR_CUDA;
  }
  return TDDFT_OK;
}

}  // extern "C"
