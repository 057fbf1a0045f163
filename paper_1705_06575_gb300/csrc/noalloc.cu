// noalloc.cu — a solve entry point that allocates no memory.
//
// sym_solve_multi needs a work block of n * nrhs doubles for the permuted right-hand sides; it
// allocates that block with cudaMalloc on first use and whenever nrhs grows. Some callers cannot
// allow that: a caller whose device memory is owned by its own pool or caching allocator (so a
// raw cudaMalloc may fail or fragment it), or a latency-critical loop where the implicit device
// synchronization of cudaMalloc/cudaFree is unacceptable. sym_solve_multi_noalloc runs the same
// kernels with the work block taken from a fixed array in the library's device memory instead.
#include <cuda_runtime.h>

#include <mutex>

#include "sym.h"

namespace sym {
int check_solve_ready(sym_handle h);
int solve_with_work(sym_handle h, int32_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
                    double *work);
int set_error(int code, const char *msg);
int64_t plan_n(sym_handle h);
}  // namespace sym

namespace {

// The shared work block: SYM_NOALLOC_MAX_WORK doubles (8 MiB) in every device's memory that
// loads this library, held until the process exits.
static __device__ __align__(256) double g_noalloc_work[SYM_NOALLOC_MAX_WORK];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_work_ptr[kMaxDevices] = {};  // device address of g_noalloc_work, per device

// The host-side name g_noalloc_work is not a device address; look up the real address once per
// device, with that device current.
int work_address(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return sym::set_error(SYM_ERR_CUDA, "sym_solve_multi_noalloc: no usable current device");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_work_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_work);
    if (e != cudaSuccess || !p)
      return sym::set_error(SYM_ERR_CUDA, "sym_solve_multi_noalloc: cudaGetSymbolAddress failed");
    g_work_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_work_ptr[dev];
  return SYM_OK;
}

}  // namespace

extern "C" int sym_solve_multi_noalloc(sym_handle h, int32_t nrhs, const double *B, int64_t ldb,
                                       double *X, int64_t ldx) {
  if (!h) return sym::set_error(SYM_ERR_INVALID, "null handle");
  const int64_t n = sym::plan_n(h);
  if (nrhs < 0) return sym::set_error(SYM_ERR_INVALID, "bad solve arguments");
  if (n * (int64_t)nrhs > (int64_t)SYM_NOALLOC_MAX_WORK)
    return sym::set_error(SYM_ERR_LIMIT, "sym_solve_multi_noalloc: n * nrhs exceeds SYM_NOALLOC_MAX_WORK");
  // the handle and its device are checked before the array's address is looked up, so a call
  // refused for a wrong current device does not touch that device
  int rc = sym::check_solve_ready(h);
  if (rc) return rc;
  double *work = nullptr;
  rc = work_address(&work);
  if (rc) return rc;
  return sym::solve_with_work(h, nrhs, B, ldb, X, ldx, work);
}
