// tddft_apply_noalloc: the response-operator product of tddft_apply for callers
// that may not allocate device memory at call time -- code that runs while
// another runtime owns the whole device pool, real-time loops that cannot take
// the latency or the failure modes of an allocation, and contexts where
// allocation calls are not permitted.  Every intermediate of the product lives
// in one file-scope device array; nothing here calls cudaMalloc, cudaFree or an
// allocating library routine.
#include <algorithm>
#include <mutex>

#include "ctx.cuh"
#include "vecops.cuh"

namespace tddft {

namespace {

// Size of the shared scratch array.  Every GPU that loads the library holds
// this much device memory for the lifetime of the process.
constexpr size_t kScratchBytes = 64ull << 20;   // 64 MiB

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, so the address is looked up with the
// device current.  The lookup is repeated on every call whose stream is not
// being captured (it allocates nothing): after cudaDeviceReset, or under another
// CUDA context, the module is loaded again and an address cached from before
// would point at freed or foreign memory.  While the stream is being captured
// the address of the last uncaptured call on this device is used, so the first
// call on a device has to come before any capture.
void* scratch_address(int dev, cudaStream_t s) {
  TD_REQUIRE(dev >= 0 && dev < kMaxDevices, TDDFT_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TD_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) {
    TD_REQUIRE(g_scratch_addr[dev] != nullptr, TDDFT_ERR_ARG,
               "tddft_apply_noalloc: first call on this device made during stream capture");
    return g_scratch_addr[dev];
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess || p == nullptr)
    throw Error(TDDFT_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch) failed: ") +
                                    cudaGetErrorString(e));
  g_scratch_addr[dev] = p;
  return p;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

// Same arithmetic as apply_operator's SIMT path (FP64 for PLAIN, FP32 for MIXED),
// with unsplit GEMMs and every buffer carved from the static scratch array.
static void apply_operator_static(const OpDims& d, const FactorSet& f, const double* X, int m,
                                  OpMode mode, double* out0, double* out1, unsigned char* base,
                                  cudaStream_t s) {
  const int no = d.no, nv = d.nv, ov = d.ov;
  const bool f64 = (f.dt == DType::F64);
  const DType tw = f64 ? DType::F64 : DType::F32;
  const size_t ew = dtype_size(tw);
  const size_t mov = (size_t)m * ov;
  const bool need_k2 = (mode == OpMode::PAIRED);
  const bool do_j = f.nJ > 0 && d.c_J != 0.0;
  const bool do_k = f.nK > 0 && d.a_x != 0.0;

  size_t fixed = (f64 ? 0 : up256(mov * 4)) + (do_j ? up256((size_t)f.nJ * m * ew) + up256(mov * ew) : 0) +
                 (do_k ? up256(mov * ew) * (need_k2 ? 2 : 1) : 0);
  const size_t per_row = (size_t)m * no * nv * ew + (need_k2 ? (size_t)m * no * no * ew : 0);
  TD_REQUIRE(fixed + (do_k ? up256(per_row) + 256 : 0) <= kScratchBytes, TDDFT_ERR_ARG,
             "tddft_apply_noalloc: problem needs more than the 64 MiB static scratch "
             "(reduce m or use tddft_apply)");
  size_t off = 0;
  auto take = [&](size_t bytes) { void* p = base + off; off += up256(bytes); return p; };

  const void* Xw = X;
  if (!f64) {
    float* xb = static_cast<float*>(take(mov * 4));
    cast_f64_to_f32(X, xb, (long long)mov, s);
    Xw = xb;
  }
  void* Jb = nullptr;
  if (do_j) {
    void* t = take((size_t)f.nJ * m * ew);
    Jb = take(mov * ew);
    GemmDesc g;
    g.acc64 = f64;
    g.M = f.nJ; g.N = m; g.K = ov;
    g.A = f.Jov; g.ta = f.dt; g.sam = ov; g.sak = 1;
    g.B = Xw; g.tb = tw; g.sbk = 1; g.sbn = ov;
    g.C = t; g.tc = tw; g.scm = m; g.scn = 1;
    gemm(g, s);
    GemmDesc h;
    h.acc64 = f64;
    h.M = m; h.N = ov; h.K = f.nJ;
    h.A = t; h.ta = tw; h.sam = 1; h.sak = m;
    h.B = f.Jov; h.tb = f.dt; h.sbk = ov; h.sbn = 1;
    h.C = Jb; h.tc = tw; h.scm = ov; h.scn = 1;
    gemm(h, s);
  }
  void* K1b = nullptr;
  void* K2b = nullptr;
  if (do_k) {
    K1b = take(mov * ew);
    if (need_k2) K2b = take(mov * ew);
    long long pc = (long long)((kScratchBytes - off - 512) / (per_row + 512));
    if (pc > f.nK) pc = f.nK;
    if (pc * m > 65535) pc = 65535 / m;
    TD_REQUIRE(pc >= 1, TDDFT_ERR_ARG, "tddft_apply_noalloc: static scratch too small");
    void* Zb = take((size_t)m * no * pc * nv * ew);
    void* Qb = need_k2 ? take((size_t)m * no * pc * no * ew) : nullptr;
    const size_t es = dtype_size(f.dt);
    for (int p0 = 0; p0 < f.nK; p0 += (int)pc) {
      const int pn = (int)std::min<long long>(pc, f.nK - p0);
      GemmDesc z;
      z.acc64 = f64;
      z.M = no; z.N = nv; z.K = no;
      z.A = (const char*)f.Koo + (size_t)p0 * no * no * es; z.ta = f.dt; z.sam = no; z.sak = 1;
      z.B = Xw; z.tb = tw; z.sbk = nv; z.sbn = 1;
      z.C = Zb; z.tc = tw; z.scm = (long long)pn * nv; z.scn = 1;
      z.nb0 = pn; z.nb1 = m;
      z.sA0 = (long long)no * no; z.sC0 = nv;
      z.sB1 = ov; z.sC1 = (long long)no * pn * nv;
      gemm(z, s);
      GemmDesc k;
      k.acc64 = f64;
      k.M = m * no; k.N = nv; k.K = pn * nv;
      k.A = Zb; k.ta = tw; k.sam = (long long)pn * nv; k.sak = 1;
      k.B = (const char*)f.Kvv + (size_t)p0 * nv * nv * es; k.tb = f.dt; k.sbk = nv; k.sbn = 1;
      k.C = K1b; k.tc = tw; k.scm = nv; k.scn = 1;
      k.beta = p0 > 0 ? 1.0 : 0.0;   // the first chunk overwrites what the last call left
      gemm(k, s);
      if (need_k2) {
        GemmDesc q;
        q.acc64 = f64;
        q.M = no; q.N = no; q.K = nv;
        q.A = (const char*)f.Kov + (size_t)p0 * ov * es; q.ta = f.dt; q.sam = nv; q.sak = 1;
        q.B = Xw; q.tb = tw; q.sbk = 1; q.sbn = nv;
        q.C = Qb; q.tc = tw; q.scm = (long long)pn * no; q.scn = 1;
        q.nb0 = pn; q.nb1 = m;
        q.sA0 = ov; q.sC0 = no;
        q.sB1 = ov; q.sC1 = (long long)no * pn * no;
        gemm(q, s);
        GemmDesc k2;
        k2.acc64 = f64;
        k2.M = m * no; k2.N = nv; k2.K = pn * no;
        k2.A = Qb; k2.ta = tw; k2.sam = (long long)pn * no; k2.sak = 1;
        k2.B = (const char*)f.Kov + (size_t)p0 * ov * es; k2.tb = f.dt; k2.sbk = nv; k2.sbn = 1;
        k2.C = K2b; k2.tc = tw; k2.scm = nv; k2.scn = 1;
        k2.beta = p0 > 0 ? 1.0 : 0.0;
        gemm(k2, s);
      }
    }
  }
  if (mode == OpMode::TDA) {
    combine(X, d.delta, Jb, K1b, nullptr, tw, d.c_J, -d.a_x, 0.0, m, ov, out0, s);
  } else {
    combine(X, d.delta, Jb, K1b, K2b, tw, 2.0 * d.c_J, -d.a_x, -d.a_x, m, ov, out0, s);
    combine(X, d.delta, nullptr, K1b, K2b, tw, 0.0, -d.a_x, d.a_x, m, ov, out1, s);
  }
}

}  // namespace tddft

using namespace tddft;

extern "C" tddft_status tddft_apply_noalloc(tddft_ctx* ctx, int kind, int precision, const double* X,
                                            int m, double* out0, double* out1) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return TDDFT_ERR_ARG;
  int prev = -1;
  try {
    TD_REQUIRE(kind >= 0 && kind <= 3, TDDFT_ERR_ARG, "kind must be 0..3");
    TD_REQUIRE(precision == TDDFT_PLAIN || precision == TDDFT_MIXED, TDDFT_ERR_ARG, "bad precision");
    TD_REQUIRE((c->precisions & (precision == TDDFT_PLAIN ? 1 : 2)) != 0, TDDFT_ERR_ARG,
               "context lacks the factor copies for this precision");
    TD_REQUIRE(m >= 0 && X && out0 && ((kind & 1) == 0 || out1), TDDFT_ERR_ARG, "bad buffers");
    if (m == 0) return TDDFT_OK;
    std::lock_guard<std::mutex> run(c->run_mu);
    TD_CUDA(cudaGetDevice(&prev));
    if (prev != c->device) TD_CUDA(cudaSetDevice(c->device));
    unsigned char* base = static_cast<unsigned char*>(scratch_address(c->device, c->s));
    const bool ris = kind >= 2;
    const bool paired = (kind & 1) != 0;
    FactorSet f = ris ? c->ris(precision) : c->exact(precision);
    TD_REQUIRE(!f.has_variants(), TDDFT_ERR_ARG,
               "tddft_apply_noalloc does not apply a second exchange set or a kernel term");
    apply_operator_static(c->dims(), f, X, m, paired ? OpMode::PAIRED : OpMode::TDA, out0,
                          paired ? out1 : nullptr, base, c->s);
    if (prev != c->device) TD_CUDA(cudaSetDevice(prev));
    return TDDFT_OK;
  } catch (const Error& e) {
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    c->err = e.what();
    return e.status;
  } catch (const std::exception& e) {
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    c->err = e.what();
    return TDDFT_ERR_CUDA;
  }
}
