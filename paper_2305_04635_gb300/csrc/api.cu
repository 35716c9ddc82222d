// api.cu -- the C ABI of libbchol (declared in include/bchol.h): handle,
// workspace management, argument checks and launches.
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/bchol.h"
#include "bchol_internal.h"
#include "schedule.cuh"

namespace bchol {

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
  return n;
}

// Workspace layout: [0, 256) status words (timeout record), then the region
// used by one call (factor flags and control block, or inverted blocks).
constexpr size_t kStatusBytes = 256;

}  // namespace bchol

struct bchol_handle_s {
  cudaStream_t stream = nullptr;
  void* ws_own = nullptr;
  size_t ws_own_bytes = 0;
  void* ws_lent = nullptr;
  size_t ws_lent_bytes = 0;
  int tile = 0;
  int wait_ms = 2000;
  int ctas_per_sm = 0;
  int last_launches = 0;
  int stall_I = -1, stall_J = -1;
  int* last_status = nullptr;  // status word of the workspace used last
  bchol_batch_t batch = nullptr;  // bchol_factor_batched's own plan
  int precision = BCHOL_FP64;
  int max_refine = 10;
  double tol = 1e-10;
  // BCHOL_FP32_UPDATE: the factorization that the next bchol_solve refines against
  bool mixed_ready = false;
  int mixed_n = 0, mixed_k = 0, mixed_ldab = 0;
  const double* mixed_ab = nullptr;
  const char* mixed_ws = nullptr;
  const int* mixed_info = nullptr;
  int last_iters = 0;
  double last_resid = 0.0, last_corr = 0.0;
  int solve_path = 0;  // 0 automatic, 1 cluster, 2 partitioned, 3 cluster without far clusters
  int tma = 1;         // the chain's tile copies: 0 plain loads, 1 TMA where possible (measured no slower)
  int last_tma = 0;    // whether the last factorization's chain used TMA
};

using namespace bchol;

// Does a precision mode run the split updates on the tensor cores?
static bool split_mode(int precision) { return precision == BCHOL_FP64_SPLIT; }

// Right-hand sides refined together by a BCHOL_FP32_UPDATE solve (its
// workspace holds a copy of that many columns and their residuals).
constexpr int kMixedChunk = 16;

static size_t call_bytes(bchol_handle_t h, int n, int k) {
  const int kk = (n > 0 && k > n - 1) ? n - 1 : k;
  const int b = h->tile ? h->tile : auto_tile(kk);
  if (h->precision == BCHOL_FP32_UPDATE && n > 0) return kStatusBytes + mixed_workspace_bytes(n, kk, kMixedChunk, b);
  const FactorPlan P = make_factor_plan(n, kk, b);
  size_t f = factor_workspace_bytes(P), s = solve_workspace_bytes(n, kk);
  return kStatusBytes + (f > s ? f : s);
}

// Workspace of at least `bytes`: the lent buffer, or the handle's own one
// (grown with cudaMalloc; its status words are zeroed when it is created).
static bchol_status_t get_workspace(bchol_handle_t h, size_t bytes, char** ws) {
  if (h->ws_lent) {
    if (h->ws_lent_bytes < bytes) return BCHOL_ERR_ALLOC;
    *ws = static_cast<char*>(h->ws_lent);
    return BCHOL_OK;
  }
  if (h->ws_own_bytes < bytes) {
    if (h->ws_own) {
      if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BCHOL_ERR_CUDA;
      cudaFree(h->ws_own);
      h->ws_own = nullptr;
      h->ws_own_bytes = 0;
      h->last_status = nullptr;
      h->mixed_ready = false;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return BCHOL_ERR_ALLOC;
    }
    if (cudaMemsetAsync(p, 0, kStatusBytes, h->stream) != cudaSuccess) {
      cudaFree(p);
      return BCHOL_ERR_CUDA;
    }
    h->ws_own = p;
    h->ws_own_bytes = bytes;
  }
  *ws = static_cast<char*>(h->ws_own);
  return BCHOL_OK;
}

// bchol_solve in the BCHOL_FP32_UPDATE mode: the factor of S A S that the last
// bchol_factor left in the workspace, and refinement against A (ab still holds
// A in this mode), kMixedChunk right-hand sides at a time; B is overwritten by X.
static bchol_status_t solve_fp32_update(bchol_handle_t h, int n, int k, int nrhs, const double* ab, int ldab,
                                        double* b, int ldb) {
  const int kk = (n > 0 && k > n - 1) ? n - 1 : k;
  const char* cur = h->ws_lent ? static_cast<const char*>(h->ws_lent) : static_cast<const char*>(h->ws_own);
  if (!h->mixed_ready || h->mixed_n != n || h->mixed_k != kk || h->mixed_ab != ab || h->mixed_ldab != ldab ||
      h->mixed_ws != cur)
    return BCHOL_ERR_ARG;  // no matching bchol_factor on this handle
  int info = 0;
  if (cudaMemcpyAsync(&info, h->mixed_info, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return BCHOL_ERR_CUDA;
  if (info != 0) return BCHOL_ERR_NOT_SPD;
  char* ws = const_cast<char*>(cur) + kStatusBytes;
  const int tile = h->tile ? h->tile : auto_tile(kk);
  double* b0 = mixed_rhs_copy(ws, n, kk, kMixedChunk, tile);
  int launches = 0, iters = 0;
  double resid = 0.0, corr = 0.0;
  for (int c0 = 0; c0 < nrhs; c0 += kMixedChunk) {
    const int nc = nrhs - c0 < kMixedChunk ? nrhs - c0 : kMixedChunk;
    double* bc = b + (long long)c0 * ldb;
    if (cudaMemcpy2DAsync(b0, sizeof(double) * n, bc, sizeof(double) * ldb, sizeof(double) * n, nc,
                          cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return BCHOL_ERR_CUDA;
    int it = 0, l = 0;
    double rs = 0.0, cr = 0.0;
    const int r = mixed_refine(n, kk, nc, ab, ldab, b0, n, bc, ldb, h->max_refine, h->tol, tile, ws, kMixedChunk,
                               h->stream, &it, &rs, &cr, &l, nullptr);
    if (r != BCHOL_OK) {
      cudaGetLastError();
      return static_cast<bchol_status_t>(r);
    }
    launches += l + 1;
    iters = iters > it ? iters : it;
    resid = resid > rs ? resid : rs;
    corr = corr > cr ? corr : cr;
  }
  h->last_iters = iters;
  h->last_resid = resid;
  h->last_corr = corr;
  h->last_launches = launches;
  return BCHOL_OK;
}

extern "C" {

bchol_status_t bchol_last_refinement(bchol_handle_t h, int* iters, double* resid, double* corr) {
  if (!h || !iters || !resid || !corr) return BCHOL_ERR_ARG;
  *iters = h->last_iters;
  *resid = h->last_resid;
  *corr = h->last_corr;
  return BCHOL_OK;
}

bchol_status_t bchol_create(bchol_handle_t* handle, void* stream) {
  if (!handle) return BCHOL_ERR_ARG;
  bchol_handle_t h = new (std::nothrow) bchol_handle_s();
  if (!h) return BCHOL_ERR_ALLOC;
  h->stream = static_cast<cudaStream_t>(stream);
  *handle = h;
  return BCHOL_OK;
}

bchol_status_t bchol_destroy(bchol_handle_t h) {
  if (!h) return BCHOL_ERR_ARG;
  bchol_status_t rc = BCHOL_OK;
  if (h->batch) bchol_batch_destroy(h->batch);
  if (h->ws_own) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = BCHOL_ERR_CUDA;
    cudaFree(h->ws_own);
  }
  delete h;
  return rc;
}

bchol_status_t bchol_set_stream(bchol_handle_t h, void* stream) {
  if (!h) return BCHOL_ERR_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return BCHOL_OK;
}

bchol_status_t bchol_set_workspace(bchol_handle_t h, void* ptr, size_t bytes) {
  if (!h) return BCHOL_ERR_ARG;
  h->mixed_ready = false;
  if (ptr == nullptr || bytes == 0) {
    h->ws_lent = nullptr;
    h->ws_lent_bytes = 0;
    h->last_status = nullptr;
    return BCHOL_OK;
  }
  if ((reinterpret_cast<uintptr_t>(ptr) & 15u) != 0 || bytes < kStatusBytes) return BCHOL_ERR_ARG;
  if (cudaMemsetAsync(ptr, 0, kStatusBytes, h->stream) != cudaSuccess) return BCHOL_ERR_CUDA;
  h->ws_lent = ptr;
  h->ws_lent_bytes = bytes;
  h->last_status = nullptr;
  return BCHOL_OK;
}

size_t bchol_workspace_size(bchol_handle_t h, int n, int k) {
  if (!h || n < 0 || k < 0) return 0;
  return call_bytes(h, n, k);
}

bchol_status_t bchol_set_tile(bchol_handle_t h, int tile) {
  if (!h || !(tile == 0 || tile == 16 || tile == 32 || tile == 64)) return BCHOL_ERR_ARG;
  h->tile = tile;
  return BCHOL_OK;
}

bchol_status_t bchol_set_precision(bchol_handle_t h, bchol_precision_t precision, int max_refine, double tol) {
  if (!h || max_refine < 0 || !(tol >= 0.0)) return BCHOL_ERR_ARG;
  switch (precision) {
    case BCHOL_FP64:
    case BCHOL_FP64_SPLIT:
    case BCHOL_FP32_UPDATE:
      break;
    case BCHOL_TF32_UPDATE:
      return BCHOL_ERR_UNSUPPORTED;
    default:
      return BCHOL_ERR_ARG;
  }
  if (precision != h->precision) h->mixed_ready = false;
  h->precision = precision;
  h->max_refine = max_refine;
  h->tol = tol;
  return BCHOL_OK;
}

bchol_status_t bchol_set_tile_staging(bchol_handle_t h, int tma) {
  if (!h || (tma != 0 && tma != 1)) return BCHOL_ERR_ARG;
  h->tma = tma;
  return BCHOL_OK;
}

int bchol_last_tile_staging(bchol_handle_t h) { return h ? h->last_tma : -1; }

bchol_status_t bchol_set_solve_path(bchol_handle_t h, int path) {
  if (!h || path < 0 || path > 3) return BCHOL_ERR_ARG;
  h->solve_path = path;
  return BCHOL_OK;
}

bchol_status_t bchol_set_wait_limit_ms(bchol_handle_t h, int ms) {
  if (!h || ms < 1) return BCHOL_ERR_ARG;
  h->wait_ms = ms;
  return BCHOL_OK;
}

bchol_status_t bchol_set_ctas_per_sm(bchol_handle_t h, int c) {
  if (!h || c < 0 || c > 32) return BCHOL_ERR_ARG;
  h->ctas_per_sm = c;
  return BCHOL_OK;
}

bchol_status_t bchol_set_stall_tile(bchol_handle_t h, int I, int J) {
  if (!h || I < -1 || J < -1 || (I >= 0) != (J >= 0) || (I >= 0 && J > I)) return BCHOL_ERR_ARG;
  h->stall_I = I;
  h->stall_J = J;
  return BCHOL_OK;
}

long long bchol_plan_task_count(int n, int k, int tile) {
  return bchol_plan_task_count_ex(n, k, tile, BCHOL_FP64);
}

bchol_status_t bchol_plan_task(int n, int k, int tile, long long ticket, int* type, int* s, int* I, int* J) {
  return bchol_plan_task_ex(n, k, tile, BCHOL_FP64, ticket, type, s, I, J);
}

long long bchol_plan_task_count_ex(int n, int k, int tile, int precision) {
  if (n < 0 || k < 0 || !(tile == 16 || tile == 32 || tile == 64) || precision < 0 || precision > 3) return -1;
  return plan_task_count(make_factor_plan(n, k, tile, split_mode(precision)));
}

bchol_status_t bchol_plan_task_ex(int n, int k, int tile, int precision, long long ticket, int* type, int* s, int* I,
                                  int* J) {
  if (n < 0 || k < 0 || !(tile == 16 || tile == 32 || tile == 64) || precision < 0 || precision > 3 || !type || !s ||
      !I || !J)
    return BCHOL_ERR_ARG;
  const FactorPlan P = make_factor_plan(n, k, tile, split_mode(precision));
  if (ticket < 0 || ticket >= plan_task_count(P)) return BCHOL_ERR_ARG;
  plan_task(P, ticket, *type, *s, *I, *J);
  return BCHOL_OK;
}

long long bchol_adjoint_plan_task_count(int n, int k, int tile) {
  if (n < 0 || k < 0 || !(tile == 16 || tile == 32 || tile == 64)) return -1;
  const int kk = (n > 0 && k > n - 1) ? n - 1 : k;
  return adjoint_plan_count(n, kk, tile);
}

bchol_status_t bchol_adjoint_plan_task(int n, int k, int tile, long long ticket, int* type, int* J, int* I, int* g) {
  if (n < 0 || k < 0 || !(tile == 16 || tile == 32 || tile == 64) || !type || !J || !I || !g) return BCHOL_ERR_ARG;
  const int kk = (n > 0 && k > n - 1) ? n - 1 : k;
  if (ticket < 0 || ticket >= adjoint_plan_count(n, kk, tile)) return BCHOL_ERR_ARG;
  adjoint_plan_task(n, kk, tile, ticket, type, J, I, g);
  return BCHOL_OK;
}

bchol_status_t bchol_check_pivot_rcp(bchol_handle_t h, const double* x, double* y, int n) {
  if (!h || n < 0 || (n > 0 && (!x || !y))) return BCHOL_ERR_ARG;
  if (launch_pivot_rcp(x, y, n, h->stream) != cudaSuccess) {
    cudaGetLastError();
    return BCHOL_ERR_CUDA;
  }
  return BCHOL_OK;
}

bchol_status_t bchol_check_split_product(bchol_handle_t h, int m, int n, const double* A, int lda, const double* B,
                                         int ldb, double* C, int ldc) {
  if (!h || m < 0 || n < 0 || lda < (m > 1 ? m : 1) || ldb < (n > 1 ? n : 1) || ldc < (m > 1 ? m : 1))
    return BCHOL_ERR_ARG;
  if (m > 0 && n > 0 && (!A || !B || !C)) return BCHOL_ERR_ARG;
  h->last_launches = 0;
  if (m == 0 || n == 0) return BCHOL_OK;
  char* ws = nullptr;
  bchol_status_t rc = get_workspace(h, kStatusBytes, &ws);
  if (rc != BCHOL_OK) return rc;
  int* status = reinterpret_cast<int*>(ws);
  h->last_status = status;
  if (cudaMemsetAsync(status + 1, 0, sizeof(int), h->stream) != cudaSuccess) return BCHOL_ERR_CUDA;
  if (launch_split_check(m, n, A, lda, B, ldb, C, ldc, status, status + 1, (uint64_t)h->wait_ms * 1000000ull,
                         h->stream) != cudaSuccess) {
    cudaGetLastError();
    return BCHOL_ERR_CUDA;
  }
  h->last_launches = 1;
  return BCHOL_OK;
}

bchol_status_t bchol_probe_rate(bchol_handle_t h, int kind, int iters, double* tflops) {
  if (!h || kind < 0 || kind > 3 || iters < 1 || !tflops) return BCHOL_ERR_ARG;
  char* ws = nullptr;
  bchol_status_t rc = get_workspace(h, kStatusBytes, &ws);
  if (rc != BCHOL_OK) return rc;
  int* status = reinterpret_cast<int*>(ws);
  h->last_status = status;
  if (probe_rate(kind, iters, tflops, status, (uint64_t)h->wait_ms * 1000000ull, h->stream) != cudaSuccess) {
    cudaGetLastError();
    return BCHOL_ERR_CUDA;
  }
  int st = 0;
  if (cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return BCHOL_ERR_CUDA;
  return st != 0 ? BCHOL_ERR_TIMEOUT : BCHOL_OK;
}

int bchol_last_launch_count(bchol_handle_t h) { return h ? h->last_launches : 0; }

const char* bchol_version(void) { return "bchol 0.1.0 (sm_103a)"; }

bchol_status_t bchol_factor(bchol_handle_t h, int n, int k, double* ab, int ldab, int* info_dev) {
  if (!h || n < 0 || k < 0 || ldab < k + 1 || !info_dev || (n > 0 && !ab)) return BCHOL_ERR_ARG;
  h->last_launches = 0;
  const int kk = (n > 0 && k > n - 1) ? n - 1 : k;
  if (n == 0) return cudaMemsetAsync(info_dev, 0, sizeof(int), h->stream) == cudaSuccess ? BCHOL_OK : BCHOL_ERR_CUDA;
  char* ws = nullptr;
  bchol_status_t rc = get_workspace(h, call_bytes(h, n, k), &ws);
  if (rc != BCHOL_OK) return rc;
  const int b = h->tile ? h->tile : auto_tile(kk);
  int* status = reinterpret_cast<int*>(ws);
  h->last_status = status;
  if (h->precision == BCHOL_FP32_UPDATE) {
    h->mixed_ready = false;
    int launches = 0;
    const int r = mixed_factor(n, kk, ab, ldab, info_dev, b, h->ctas_per_sm ? h->ctas_per_sm : auto_ctas_per_sm(kk),
                               ws + kStatusBytes, kMixedChunk, status, (uint64_t)h->wait_ms * 1000000ull, h->stream,
                               &launches);
    if (r != BCHOL_OK) {
      cudaGetLastError();
      return static_cast<bchol_status_t>(r);
    }
    h->mixed_ready = true;
    h->mixed_n = n;
    h->mixed_k = kk;
    h->mixed_ab = ab;
    h->mixed_ldab = ldab;
    h->mixed_ws = ws;
    h->mixed_info = info_dev;
    h->last_launches = launches;
    return BCHOL_OK;
  }
  // With the automatic tile the split updates run where that tile is 32 (k > 640):
  // below, the diagonal chain bounds the factorization and the FP64 updates of
  // 16-tiles are faster (measured); a tile set with bchol_set_tile is taken as is.
  const bool split = split_mode(h->precision) && (h->tile != 0 || b == 32);
  const FactorPlan P = make_factor_plan(n, kk, b, split);
  cudaError_t e = launch_factor(P, ab, ldab, info_dev, ws + kStatusBytes, status,
                                (uint64_t)h->wait_ms * 1000000ull, h->ctas_per_sm ? h->ctas_per_sm : auto_ctas_per_sm(kk),
                                h->stall_I, h->stall_J, h->stream, h->tma, &h->last_tma);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BCHOL_ERR_CUDA;
  }
  h->last_launches = 1;
  return BCHOL_OK;
}

bchol_status_t bchol_solve(bchol_handle_t h, int n, int k, int nrhs, const double* ab, int ldab, double* b,
                           int ldb) {
  if (!h || n < 0 || k < 0 || nrhs < 0 || ldab < k + 1 || ldb < (n > 1 ? n : 1)) return BCHOL_ERR_ARG;
  if (n > 0 && nrhs > 0 && (!ab || !b)) return BCHOL_ERR_ARG;
  h->last_launches = 0;
  if (n == 0 || nrhs == 0) return BCHOL_OK;
  if (h->precision == BCHOL_FP32_UPDATE) return solve_fp32_update(h, n, k, nrhs, ab, ldab, b, ldb);
  char* ws = nullptr;
  bchol_status_t rc = get_workspace(h, call_bytes(h, n, k), &ws);
  if (rc != BCHOL_OK) return rc;
  h->last_status = reinterpret_cast<int*>(ws);
  int launches = 0;
  cudaError_t e = launch_solve(n, k, nrhs, ab, ldab, b, ldb, ws + kStatusBytes, &launches, h->stream, h->solve_path,
                               h->last_status, (uint64_t)h->wait_ms * 1000000ull);
  h->last_launches = launches;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BCHOL_ERR_CUDA;
  }
  return BCHOL_OK;
}

bchol_status_t bchol_logdet(bchol_handle_t h, int n, const double* ab, int ldab, double* out_dev) {
  if (!h || n < 1 || ldab < 1 || !ab || !out_dev) return BCHOL_ERR_ARG;
  h->last_launches = 0;
  if (launch_logdet(ab, ldab, n, out_dev, h->stream) != cudaSuccess) {
    cudaGetLastError();
    return BCHOL_ERR_CUDA;
  }
  h->last_launches = 1;
  return BCHOL_OK;
}

bchol_status_t bchol_backward(bchol_handle_t h, int n, int k, const double* ab, int ldab, const double* x,
                              const double* xbar, double ldbar, double* abar, int ldabar, double* bbar) {
  if (!h || n < 1 || k < 0 || ldab < k + 1 || ldabar < k + 1 || !ab || !abar) return BCHOL_ERR_ARG;
  if ((xbar != nullptr) && (!x || !bbar)) return BCHOL_ERR_ARG;
  h->last_launches = 0;
  const int kk = k > n - 1 ? n - 1 : k;
  const int b = h->tile ? h->tile : auto_tile(kk);
  size_t need = call_bytes(h, n, k);
  const size_t sel = kStatusBytes + selinv_workspace_bytes(n, kk, b);
  if (sel > need) need = sel;
  char* ws = nullptr;
  bchol_status_t rc = get_workspace(h, need, &ws);
  if (rc != BCHOL_OK) return rc;
  int* status = reinterpret_cast<int*>(ws);
  h->last_status = status;
  int launches = 0;
  if (xbar) {
    // bbar = A^{-1} xbar by the two substitution sweeps on the factor
    if (cudaMemcpyAsync(bbar, xbar, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return BCHOL_ERR_CUDA;
    int l2 = 0;
    if (launch_solve(n, kk, 1, ab, ldab, bbar, n, ws + kStatusBytes, &l2, h->stream, 0, status,
                     (uint64_t)h->wait_ms * 1000000ull) != cudaSuccess) {
      cudaGetLastError();
      return BCHOL_ERR_CUDA;
    }
    launches += l2;
  }
  if (launch_backward(n, kk, b, ab, ldab, xbar ? x : nullptr, xbar ? bbar : nullptr, ldbar, abar, ldabar,
                      ws + kStatusBytes, status, (uint64_t)h->wait_ms * 1000000ull,
                      h->ctas_per_sm ? h->ctas_per_sm : auto_ctas_per_sm(kk), h->stream) != cudaSuccess) {
    cudaGetLastError();
    return BCHOL_ERR_CUDA;
  }
  h->last_launches = launches + 3;
  return BCHOL_OK;
}

bchol_status_t bchol_solve_mixed(bchol_handle_t h, int n, int k, int nrhs, const double* ab, int ldab,
                                 const double* b, int ldb, double* x, int ldx, int max_iter, double tol,
                                 int* info_dev, int* iters, double* resid, double* corr) {
  if (!h || n < 1 || k < 0 || nrhs < 1 || ldab < k + 1 || ldb < n || ldx < n || !ab || !b || !x || !info_dev ||
      max_iter < 0 || !(tol >= 0.0) || !iters || !resid || !corr)
    return BCHOL_ERR_ARG;
  h->last_launches = 0;
  const int kk = k > n - 1 ? n - 1 : k;
  const int tile = h->tile ? h->tile : auto_tile(kk);
  char* ws = nullptr;
  bchol_status_t rc = get_workspace(h, kStatusBytes + mixed_workspace_bytes(n, kk, nrhs, tile), &ws);
  if (rc != BCHOL_OK) return rc;
  int* status = reinterpret_cast<int*>(ws);
  h->last_status = status;
  int launches = 0;
  const int r = mixed_solve(n, kk, nrhs, ab, ldab, b, ldb, x, ldx, max_iter, tol, info_dev, tile,
                            h->ctas_per_sm ? h->ctas_per_sm : auto_ctas_per_sm(kk), ws + kStatusBytes, status,
                            (uint64_t)h->wait_ms * 1000000ull, h->stream, iters, resid, corr, &launches);
  h->last_launches = launches;
  if (r != BCHOL_OK) cudaGetLastError();
  int st = 0;
  if (r == BCHOL_OK && cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && st != 0)
    return BCHOL_ERR_TIMEOUT;
  return static_cast<bchol_status_t>(r);
}

bchol_status_t bchol_batch_run(bchol_handle_t h, bchol_batch_t batch) {
  if (!h || !batch) return BCHOL_ERR_ARG;
  h->last_launches = 0;
  char* ws = nullptr;
  bchol_status_t rc = get_workspace(h, kStatusBytes, &ws);
  if (rc != BCHOL_OK) return rc;
  int* status = reinterpret_cast<int*>(ws);
  h->last_status = status;
  int launches = 0;
  const int r = batch_run(batch, status, (uint64_t)h->wait_ms * 1000000ull, h->stream, &launches);
  h->last_launches = launches;
  if (r != BCHOL_OK) cudaGetLastError();
  return static_cast<bchol_status_t>(r);
}

bchol_status_t bchol_factor_batched(bchol_handle_t h, int count, const int* n, const int* k, double* const* ab,
                                    const int* ldab, int* info_dev, const int* nrhs, double* const* b,
                                    const int* ldb) {
  if (!h) return BCHOL_ERR_ARG;
  if (!h->batch) {
    bchol_status_t rc = bchol_batch_create(&h->batch);
    if (rc != BCHOL_OK) return rc;
  }
  bchol_status_t rc = bchol_batch_set_precision(h->batch, split_mode(h->precision) ? BCHOL_FP64_SPLIT : BCHOL_FP64);
  if (rc != BCHOL_OK) return rc;
  rc = bchol_batch_plan(h->batch, count, n, k, ab, ldab, info_dev, nrhs, b, ldb, h->tile, h->ctas_per_sm);
  if (rc != BCHOL_OK) return rc;
  return bchol_batch_run(h, h->batch);
}

bchol_status_t bchol_get_info(bchol_handle_t h, const int* info_dev, int count, int* info_host) {
  if (!h || count < 0 || (count > 0 && (!info_dev || !info_host))) return BCHOL_ERR_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BCHOL_ERR_CUDA;
  if (count > 0 && cudaMemcpy(info_host, info_dev, sizeof(int) * (size_t)count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return BCHOL_ERR_CUDA;
  int status = 0;
  if (h->last_status) {
    if (cudaMemcpy(&status, h->last_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return BCHOL_ERR_CUDA;
    if (status != 0 && cudaMemset(h->last_status, 0, sizeof(int)) != cudaSuccess) return BCHOL_ERR_CUDA;
  }
  if (status == kStatusTimeout) return BCHOL_ERR_TIMEOUT;
  for (int i = 0; i < count; ++i)
    if (info_host[i] > 0) return BCHOL_ERR_NOT_SPD;
  return BCHOL_OK;
}

}  // extern "C"
