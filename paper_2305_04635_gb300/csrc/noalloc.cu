// noalloc.cu -- bchol_factor_noalloc: the band factorization for callers that
// cannot allocate GPU memory.
//
// Some callers are not allowed to call cudaMalloc at all: code that runs
// inside a memory pool or arena it does not own, real-time or embedded hosts
// that forbid allocation after start-up, or plugins whose host application
// owns every device allocation.  For them this entry point runs the same
// persistent factor kernel as bchol_factor, but takes its scratch memory (the
// task ticket, the abort word and the per-tile ready counters) from one fixed
// array in the library's own device memory instead of a handle workspace.
//
// The array is a file-scope __device__ variable of kScratchBytes (1 MiB).
// Every GPU that loads the library holds it until the process exits.  It is
// shared by every call on that device and keeps the last call's contents, so
// each call clears the part it uses before launching.  Two calls that run at
// the same time on one device (for instance on two streams) use the same
// array and race: callers must order them.
//
// Host code cannot pass the array's name to a kernel: on the host that name
// stands for a host-side shadow, not a device address.  The first call on
// each device therefore looks up the device address with
// cudaGetSymbolAddress, with that device current, and keeps it.  Make that
// first call before any stream capture.
#include <mutex>

#include "../../include/bchol.h"
#include "bchol_internal.h"

namespace bchol {

constexpr size_t kScratchBytes = size_t(1) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once).
static cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// Tile size and CTAs per SM for half-bandwidth k; the same rule bchol_factor uses by default.
static int noalloc_tile(int k) { return k <= 640 ? 16 : 32; }
static int noalloc_ctas_per_sm(int k) { return k <= 256 ? 1 : 2; }

}  // namespace bchol

using namespace bchol;

extern "C" bchol_status_t bchol_factor_noalloc(void* stream, int n, int k, double* ab, int ldab, int* info_dev,
                                               int* status_dev) {
  if (n < 0 || k < 0 || ldab < k + 1 || !info_dev || !status_dev || (n > 0 && !ab)) return BCHOL_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int kk = (n > 0 && k > n - 1) ? n - 1 : k;
  const FactorPlan P = make_factor_plan(n, kk, noalloc_tile(kk));
  if (n > 0 && factor_workspace_bytes(P) > kScratchBytes) return BCHOL_ERR_UNSUPPORTED;
  if (cudaMemsetAsync(status_dev, 0, sizeof(int), st) != cudaSuccess) return BCHOL_ERR_CUDA;
  if (n == 0) return cudaMemsetAsync(info_dev, 0, sizeof(int), st) == cudaSuccess ? BCHOL_OK : BCHOL_ERR_CUDA;
  void* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return BCHOL_ERR_CUDA;
  }
  // launch_factor clears the ticket, abort word and ready counters it uses.
  cudaError_t e = launch_factor(P, ab, ldab, info_dev, scratch, status_dev, 2000ull * 1000000ull,
                                noalloc_ctas_per_sm(kk), -1, -1, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BCHOL_ERR_CUDA;
  }
  return BCHOL_OK;
}
