// eig_gemm_noalloc: the FP64 split-K GEMM of eig_gemm for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// fully reserved by another allocator's pool (a framework caching allocator
// that owns every free byte), or a latency-critical loop that cannot afford
// the implicit device synchronisation a cudaMalloc / cudaFree pair brings.
// eig_gemm takes its split-K scratch from the handle workspace, which the
// library grows with cudaMalloc; this variant instead keeps the scratch in a
// file-scope device array that exists for as long as the library is loaded
// (every GPU that loads the library holds it until the process exits).
//
// In host code g_gemm_scratch names a host-side stand-in, not a device
// address, so the kernels are given the address cudaGetSymbolAddress returns
// for the current device; it is looked up once per device, on that device's
// first call, which therefore should come before any stream capture.  The
// cached address outlives nothing but the device's primary context: after a
// device reset the entry point must not be called on that device again.
//
// Every call shares the array and it keeps the contents of the last call.
// Nothing in it needs to start at zero: each K-chunk partial a call reads is
// written by the same call first.  Calls that overlap on the GPU (different
// streams, or different host threads without ordering) race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/eigdc.h"
#include "internal.h"

namespace {

constexpr size_t kScratchDoubles = size_t(1) << 20;   // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_gemm_scratch[kScratchDoubles];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up on the
// first call per device).  Returns nullptr on failure.
double* scratch_for_device(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_gemm_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" int eig_gemm_noalloc(void* stream, int ta, int tb, int m, int n, int k, double alpha,
                                const double* dA, int lda, const double* dB, int ldb, double beta,
                                double* dC, int ldc) {
  if (m < 0 || n < 0 || k < 0 || dC == nullptr || ldc < (m > 1 ? m : 1)) return EIG_ERR_ARG;
  const int arows = ta ? k : m;
  const int brows = tb ? n : k;
  if (m > 0 && n > 0 && k > 0) {
    if (dA == nullptr || dB == nullptr) return EIG_ERR_ARG;
    if (lda < (arows > 1 ? arows : 1) || ldb < (brows > 1 ? brows : 1)) return EIG_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return EIG_ERR_CUDA;
  }
  const int splits = eigdc::gemm_choose_splits(m, n, k);
  double* scratch = nullptr;
  if (splits > 1) {
    if ((size_t)splits * (size_t)m * (size_t)n > kScratchDoubles) return EIG_ERR_SCRATCH;
    scratch = scratch_for_device(dev);
    if (scratch == nullptr) return EIG_ERR_CUDA;
  }
  const cudaError_t e = eigdc::gemm(static_cast<cudaStream_t>(stream), ta != 0, tb != 0, m, n, k,
                                    alpha, dA, lda, dB, ldb, beta, dC, ldc, splits, scratch);
  return e == cudaSuccess ? EIG_OK : EIG_ERR_CUDA;
}
