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
// stands for a host-side shadow, not a device address.  The first call in
// each CUDA context therefore looks up the device address with
// cudaGetSymbolAddress, with that context current, and keeps it, keyed by the
// context's unique ID (a context made after cudaDeviceReset, or a context of
// the caller's own, gets its own lookup).  Make that first call before any
// stream capture, and again after a cudaDeviceReset.
#include <cuda.h>

#include <mutex>

#include "../../include/bchol.h"
#include "bchol_internal.h"

namespace bchol {

constexpr size_t kScratchBytes = size_t(1) << 20;
constexpr int kMaxContexts = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static std::mutex g_noalloc_mutex;
static unsigned long long g_ctx_id[kMaxContexts] = {};
static void* g_ctx_ptr[kMaxContexts] = {};
static int g_ctx_count = 0;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique ID of the current CUDA context (0 if none is current or the driver
// does not say), through the runtime's driver entry points.
static unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx != nullptr &&
      get_id(ctx, &id) == CUDA_SUCCESS)
    return id;
  return 0;
}

// Device address of g_noalloc_scratch in the current context: looked up once
// per context and kept (contexts beyond the table's size are looked up on
// every call).
static cudaError_t noalloc_scratch(void** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  unsigned long long id = current_context_id();
  for (int i = 0; id != 0 && i < g_ctx_count; ++i) {
    if (g_ctx_id[i] == id) {
      *out = g_ctx_ptr[i];
      return cudaSuccess;
    }
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the device's context current if needed
  if (e != cudaSuccess) return e;
  if (id == 0) id = current_context_id();
  if (id != 0 && g_ctx_count < kMaxContexts) {
    g_ctx_id[g_ctx_count] = id;
    g_ctx_ptr[g_ctx_count] = p;
    ++g_ctx_count;
  }
  *out = p;
  return cudaSuccess;
}

}  // namespace bchol

using namespace bchol;

extern "C" bchol_status_t bchol_factor_noalloc(void* stream, int n, int k, double* ab, int ldab, int* info_dev,
                                               int* status_dev) {
  if (n < 0 || k < 0 || ldab < k + 1 || !info_dev || !status_dev || (n > 0 && !ab)) return BCHOL_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int kk = (n > 0 && k > n - 1) ? n - 1 : k;
  const FactorPlan P = make_factor_plan(n, kk, auto_tile(kk));
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
                                auto_ctas_per_sm(kk), -1, -1, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BCHOL_ERR_CUDA;
  }
  return BCHOL_OK;
}
