// Shared declarations of the CUDA library (internal, not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <stdexcept>
#include <vector>

#include "../../include/tddft.h"

namespace tddft {

// Error carried from deep inside the host driver up to the C ABI boundary,
// where it becomes a tddft_status and a message; never escapes extern "C".
struct Error : std::runtime_error {
  tddft_status status;
  Error(tddft_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define TD_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw ::tddft::Error(e_ == cudaErrorMemoryAllocation ? TDDFT_ERR_OOM : TDDFT_ERR_CUDA, \
                           std::string(#call " failed: ") + cudaGetErrorString(e_));     \
  } while (0)

#define TD_LAUNCH_CHECK() TD_CUDA(cudaGetLastError())

#define TD_REQUIRE(cond, status, msg)                                                    \
  do {                                                                                   \
    if (!(cond)) throw ::tddft::Error(status, msg);                                      \
  } while (0)

// Element types that the contraction kernels read.
enum class DType : int { F64 = 0, F32 = 1, BF16 = 2 };

inline size_t dtype_size(DType t) { return t == DType::F64 ? 8 : (t == DType::F32 ? 4 : 2); }

// Counts kernel launches so a solve can report them (host side, per thread).
extern thread_local long long g_launches;
inline void count_launch(int n = 1) { g_launches += n; }

// --------------------------------------------------------------------------
// Stream-ordered work buffers.  Blocks up to 64 MiB are cached per stream after
// release and handed out again to later requests of the same size class on the
// same stream (stream order makes the reuse safe), so the many small buffers
// of an iterative solve cost no allocator calls; larger blocks go straight to
// cudaMallocAsync / cudaFreeAsync.  pool_trim returns a stream's cached blocks.
void* pool_get(size_t bytes, cudaStream_t s);
void pool_put(void* p, size_t bytes, cudaStream_t s);
void pool_trim(cudaStream_t s);

// Raise a kernel's dynamic shared-memory limit (once per kernel, size and device).
void ensure_smem(const void* kernel, size_t bytes);

// Device buffer owned by host code (stream-ordered allocation).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(size_t n, cudaStream_t st) : bytes(n), s(st) {
    if (n) p = pool_get(n, st);
  }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes; s = o.s;
      o.p = nullptr; o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) pool_put(p, bytes, s);
    p = nullptr; bytes = 0;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

// --------------------------------------------------------------------------
// Generic strided, batched SIMT GEMM:
//   C[b](m,n) = alpha * sum_k A[b](m,k) * B[b](k,n) + beta * C[b](m,n)
// A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn], C(m,n) = C[m*scm + n*scn];
// batch index b = b0*nb1 + b1 with per-index offsets (in elements).
struct GemmDesc {
  int M = 0, N = 0, K = 0;
  const void* A = nullptr; DType ta = DType::F64; long long sam = 0, sak = 0;
  const void* B = nullptr; DType tb = DType::F64; long long sbk = 0, sbn = 0;
  void* C = nullptr; DType tc = DType::F64; long long scm = 0, scn = 0;
  double alpha = 1.0, beta = 0.0;
  int nb0 = 1, nb1 = 1;
  long long sA0 = 0, sA1 = 0, sB0 = 0, sB1 = 0, sC0 = 0, sC1 = 0;
  bool acc64 = true;  // accumulate in FP64 (else FP32)
};
void gemm(const GemmDesc& d, cudaStream_t s);

// Split-K GEMM (nb0 = nb1 = 1): K cut into S chunks, partials summed in a fixed
// order.  auto_splits picks S to give ~2 CTAs per SM.
int auto_splits(int M, int N, long long K);
void gemm_splitk(const GemmDesc& d, int S, cudaStream_t s);

// Split-K GEMM for tall reductions: C(m,n) = alpha * sum_k A(m,k)B(k,n) + beta*C,
// partials summed in a fixed order (deterministic).  FP64.
void gemm_splitk_f64(int M, int N, long long K, const double* A, long long sam, long long sak,
                     const double* B, long long sbk, long long sbn, double* C, long long scm,
                     long long scn, double alpha, double beta, cudaStream_t s);

}  // namespace tddft
