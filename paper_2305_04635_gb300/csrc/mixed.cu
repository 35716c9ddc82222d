// mixed.cu -- mixed-precision factor + solve with FP64 iterative refinement.
//
// A copy of A is equilibrated, Ã = S A S with S = diag(A)^{-1/2}, and factored
// with the tile algorithm of the paper (Algorithm 1) in which the trailing
// SYRK/GEMM updates accumulate in FP32 and the panel TRSMs run in FP32 (the
// diagonal POTRF stays FP64; the factor is stored in FP64).  The solution is
// then refined in FP64:
//     x_0 = S Ã^{-1} S b,     r_i = b - A x_i  (FP64),
//     d_i = S Ã^{-1} S r_i    (the correction solve, FP32 arithmetic),
//     x_{i+1} = x_i + d_i     (FP64),
// until the relative residual max_c ||r_c|| / ||b_c|| falls to `tol`, stops
// shrinking, or `max_iter` corrections have been made.  The paper's method is FP64 throughout;
// this form trades the FP64 trailing update, which dominates the flop count
// (Sec. 3.2), for FP32 arithmetic that GB300 runs 73 times faster.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/bchol.h"
#include "bchol_device.cuh"
#include "bchol_internal.h"

namespace bchol {

// s_j = A_jj^{-1/2} (1 where A_jj is not positive: the factorization reports it).
__global__ void equil_scale_kernel(const double* __restrict__ ab, long long ldab, int n, double* __restrict__ s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double a = ab[(long long)j * ldab];
  s[j] = (a > 0.0) ? rsqrt(a) : 1.0;
}

// F(d, j) = s_{j+d} A(d, j) s_j over the band (one thread per band entry).
__global__ void equil_copy_kernel(const double* __restrict__ ab, long long ldab, int n, int k,
                                  const double* __restrict__ s, double* __restrict__ f, long long ldf) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)(k + 1) * n;
  if (idx >= total) return;
  const int j = (int)(idx / (k + 1)), d = (int)(idx % (k + 1));
  if (j + d >= n) return;
  f[d + (long long)j * ldf] = s[j + d] * ab[d + (long long)j * ldab] * s[j];
}

// x(i, c) *= s_i
__global__ void scale_rows_kernel(double* __restrict__ x, long long ldx, int n, int nrhs, const double* __restrict__ s) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * nrhs) return;
  const int i = (int)(idx % n), c = (int)(idx / n);
  x[i + (long long)c * ldx] *= s[i];
}

// r = b - A x for the symmetric band A (lower band stored), one thread per row,
// and nrm[c] += ||r_c||^2.  FP64.
constexpr int kResRhs = 16;
__global__ void __launch_bounds__(128) residual_kernel(const double* __restrict__ ab, long long ldab, int n, int k,
                                                       const double* __restrict__ b, long long ldb,
                                                       const double* __restrict__ x, long long ldx,
                                                       double* __restrict__ r, long long ldr, int c0, int nr,
                                                       double* __restrict__ nrm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[kResRhs];
#pragma unroll
  for (int c = 0; c < kResRhs; ++c) acc[c] = 0.0;
  if (i < n) {
    // A(i, j) for j <= i is band[i-j, j]; for j > i it is band[j-i, i].
    const int jlo = max(0, i - k), jhi = min(n - 1, i + k);
    for (int j = jlo; j <= jhi; ++j) {
      const double a = (j <= i) ? __ldg(ab + (i - j) + (long long)j * ldab) : __ldg(ab + (j - i) + (long long)i * ldab);
#pragma unroll
      for (int c = 0; c < kResRhs; ++c)
        if (c < nr) acc[c] = fma(a, __ldg(x + j + (long long)(c0 + c) * ldx), acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kResRhs; ++c)
      if (c < nr) {
        const double v = b[i + (long long)(c0 + c) * ldb] - acc[c];
        r[i + (long long)(c0 + c) * ldr] = v;
        acc[c] = v * v;
      }
  }
  // block sums of ||r||^2 per right-hand side
  __shared__ double red[kResRhs][128 / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < kResRhs; ++c) {
    if (c < nr) {
      double v = (i < n) ? acc[c] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[c][w] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < nr) {
    double v = 0.0;
    for (int ww = 0; ww < 128 / 32; ++ww) v += red[threadIdx.x][ww];
    atomicAdd(nrm + c0 + threadIdx.x, v);
  }
}

// x += d; nrm_d[c] += ||d_c||^2, nrm_x[c] += ||x_c||^2 (after the update).
__global__ void __launch_bounds__(256) update_kernel(double* __restrict__ x, long long ldx, const double* __restrict__ d,
                                                     long long ldd, int n, int c, double* __restrict__ nrm_d,
                                                     double* __restrict__ nrm_x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double dv = 0.0, xv = 0.0;
  if (i < n) {
    dv = d[i + (long long)c * ldd];
    xv = x[i + (long long)c * ldx] + dv;
    x[i + (long long)c * ldx] = xv;
  }
  double a = dv * dv, bsum = xv * xv;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(nrm_d + c, a);
    atomicAdd(nrm_x + c, bsum);
  }
}

// ||b_c||^2
__global__ void __launch_bounds__(256) colnorm_kernel(const double* __restrict__ b, long long ldb, int n, int c,
                                                      double* __restrict__ nrm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = (i < n) ? b[i + (long long)c * ldb] : 0.0;
  v *= v;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(nrm + c, v);
}

}  // namespace bchol

using namespace bchol;

namespace bchol {

// Workspace of the mixed path, in this order: the equilibrated copy F of the
// band, the scale vector s, a copy B0 of up to nrhs right-hand sides (used when
// the solution overwrites them), the residual block R, the norms, and the
// factor/solve scratch.  The factorization writes F and s only, so a later
// solve with the same (n, k) finds them in place.
struct MixedWs {
  double* F;
  double* s;
  double* B0;
  double* R;
  double* nrm;
  void* fws;
  void* sws;
};

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

static MixedWs mixed_layout(void* wsp, int n, int k, int nrhs, int tile) {
  char* ws = static_cast<char*>(wsp);
  MixedWs m;
  m.F = reinterpret_cast<double*>(ws);
  ws += up256(sizeof(double) * (size_t)(k + 1) * n);
  m.s = reinterpret_cast<double*>(ws);
  ws += up256(sizeof(double) * n);
  m.B0 = reinterpret_cast<double*>(ws);
  ws += up256(sizeof(double) * (size_t)n * nrhs);
  m.R = reinterpret_cast<double*>(ws);
  ws += up256(sizeof(double) * (size_t)n * nrhs);
  m.nrm = reinterpret_cast<double*>(ws);  // [0,nrhs): ||b||^2, then ||r||^2, ||d||^2, ||x||^2
  ws += up256(sizeof(double) * 4 * (size_t)nrhs);
  m.fws = ws;
  ws += up256(factor_workspace_bytes(make_factor_plan(n, k, tile)));
  m.sws = ws;
  return m;
}

double* mixed_rhs_copy(void* ws, int n, int k, int nrhs_max, int tile) {
  return mixed_layout(ws, n, k, nrhs_max, tile).B0;
}

size_t mixed_workspace_bytes(int n, int k, int nrhs, int tile) {
  const FactorPlan P = make_factor_plan(n, k, tile);
  return up256(sizeof(double) * (size_t)(k + 1) * n) + up256(sizeof(double) * n) +
         2 * up256(sizeof(double) * (size_t)n * nrhs) + up256(sizeof(double) * 4 * (size_t)nrhs) +
         up256(factor_workspace_bytes(P)) + up256(solve_workspace_bytes(n, k));
}

// Equilibrate A into F and factor F with FP32-accumulated updates (asynchronous:
// info_dev is written by the kernel).
int mixed_factor(int n, int k, const double* ab, long long ldab, int* info_dev, int tile, int ctas_per_sm, void* wsp,
                 int nrhs_max, int* status, uint64_t wait_ns, cudaStream_t st, int* launches_out) {
  const MixedWs m = mixed_layout(wsp, n, k, nrhs_max, tile);
  FactorPlan P = make_factor_plan(n, k, tile);
  P.f32_update = true;
  const int T = 256;
  const unsigned gn = (unsigned)((n + T - 1) / T);
  equil_scale_kernel<<<gn, T, 0, st>>>(ab, ldab, n, m.s);
  const long long nb = (long long)(k + 1) * n;
  equil_copy_kernel<<<(unsigned)((nb + T - 1) / T), T, 0, st>>>(ab, ldab, n, k, m.s, m.F, k + 1);
  if (cudaGetLastError() != cudaSuccess) return BCHOL_ERR_CUDA;
  if (launch_factor(P, m.F, k + 1, info_dev, m.fws, status, wait_ns, ctas_per_sm, -1, -1, st) != cudaSuccess)
    return BCHOL_ERR_CUDA;
  *launches_out = 3;
  return BCHOL_OK;
}

// x from b by the factor in the workspace and FP64 refinement against A.
// nrhs <= the nrhs_max the workspace was laid out for.  Synchronises.
int mixed_refine(int n, int k, int nrhs, const double* ab, long long ldab, const double* b, long long ldb, double* x,
                 long long ldx, int max_iter, double tol, int tile, void* wsp, int nrhs_max, cudaStream_t st,
                 int* iters_out, double* resid_out, double* corr_out, int* launches_out, double* phase_ms) {
  const MixedWs m = mixed_layout(wsp, n, k, nrhs_max, tile);
  double* R = m.R;
  double* nrm = m.nrm;
  const long long ldf = k + 1;
  int launches = 0;
  const int T = 256;
  const unsigned gn = (unsigned)((n + T - 1) / T);
  std::vector<double> h(4 * (size_t)nrhs);
  cudaError_t e;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (phase_ms) {
    for (auto& v : ev) cudaEventCreate(&v);
    phase_ms[0] = phase_ms[1] = 0.0;
  }
  auto tic = [&]() { if (phase_ms) cudaEventRecord(ev[0], st); };
  auto toc = [&](int which) {
    if (!phase_ms) return;
    cudaEventRecord(ev[1], st);
    cudaEventSynchronize(ev[1]);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    phase_ms[which] += ms;
  };
#define BCHOL_CK(call)              \
  do {                              \
    e = (call);                     \
    if (e != cudaSuccess) return BCHOL_ERR_CUDA; \
  } while (0)
  // ||b||^2 and x_0 = S F^{-1} S b
  tic();
  BCHOL_CK(cudaMemsetAsync(nrm, 0, sizeof(double) * 4 * nrhs, st));
  for (int c = 0; c < nrhs; ++c) colnorm_kernel<<<gn, T, 0, st>>>(b, ldb, n, c, nrm);
  BCHOL_CK(cudaMemcpy2DAsync(x, sizeof(double) * ldx, b, sizeof(double) * ldb, sizeof(double) * n, nrhs,
                             cudaMemcpyDeviceToDevice, st));
  const unsigned gx = (unsigned)(((long long)n * nrhs + T - 1) / T);
  scale_rows_kernel<<<gx, T, 0, st>>>(x, ldx, n, nrhs, m.s);
  int l2 = 0;
  BCHOL_CK(launch_solve_f32(n, k, nrhs, m.F, ldf, x, ldx, m.sws, &l2, st));
  scale_rows_kernel<<<gx, T, 0, st>>>(x, ldx, n, nrhs, m.s);
  BCHOL_CK(cudaGetLastError());
  launches += nrhs + 2 + l2;
  toc(0);
  // Refinement: r = b - A x (FP64); stop when max_c ||r_c|| / ||b_c|| <= tol, when the
  // residual stops shrinking, or after max_iter corrections d = S F^{-1} S r, x += d.
  double corr = 0.0, res = 0.0, prev = 1e300;
  int it = 0;
  while (true) {
    tic();
    BCHOL_CK(cudaMemsetAsync(nrm + nrhs, 0, sizeof(double) * 3 * nrhs, st));
    for (int c0 = 0; c0 < nrhs; c0 += kResRhs) {
      const int nr = std::min(kResRhs, nrhs - c0);
      residual_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(ab, ldab, n, k, b, ldb, x, ldx, R, n, c0, nr,
                                                                  nrm + nrhs);
      ++launches;
    }
    BCHOL_CK(cudaGetLastError());
    BCHOL_CK(cudaMemcpyAsync(h.data(), nrm, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
    BCHOL_CK(cudaStreamSynchronize(st));
    toc(1);
    res = 0.0;
    for (int c = 0; c < nrhs; ++c) res = std::max(res, std::sqrt(h[nrhs + c] / std::max(h[c], 1e-300)));
    if (!(res > tol) || it >= max_iter || res > 0.5 * prev) break;
    prev = res;
    tic();
    scale_rows_kernel<<<gx, T, 0, st>>>(R, n, n, nrhs, m.s);
    BCHOL_CK(launch_solve_f32(n, k, nrhs, m.F, ldf, R, n, m.sws, &l2, st));
    scale_rows_kernel<<<gx, T, 0, st>>>(R, n, n, nrhs, m.s);
    for (int c = 0; c < nrhs; ++c) update_kernel<<<gn, T, 0, st>>>(x, ldx, R, n, n, c, nrm + 2 * nrhs, nrm + 3 * nrhs);
    BCHOL_CK(cudaGetLastError());
    launches += 2 + l2 + nrhs;
    BCHOL_CK(cudaMemcpyAsync(h.data() + 2 * nrhs, nrm + 2 * nrhs, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost,
                             st));
    BCHOL_CK(cudaStreamSynchronize(st));
    toc(0);
    corr = 0.0;
    for (int c = 0; c < nrhs; ++c)
      corr = std::max(corr, std::sqrt(h[2 * nrhs + c] / std::max(h[3 * nrhs + c], 1e-300)));
    ++it;
  }
#undef BCHOL_CK
  if (phase_ms)
    for (auto& v : ev) cudaEventDestroy(v);
  *iters_out = it;
  *resid_out = res;
  *corr_out = corr;
  *launches_out = launches;
  return BCHOL_OK;
}

// The whole mixed solve (bchol_solve_mixed): factor, check info, refine.
int mixed_solve(int n, int k, int nrhs, const double* ab, long long ldab, const double* b, long long ldb, double* x,
                long long ldx, int max_iter, double tol, int* info_dev, int tile, int ctas_per_sm, void* wsp,
                int* status, uint64_t wait_ns, cudaStream_t st, int* iters_out, double* resid_out,
                double* corr_out, int* launches_out) {
  int l1 = 0, l2 = 0;
  int r = mixed_factor(n, k, ab, ldab, info_dev, tile, ctas_per_sm, wsp, nrhs, status, wait_ns, st, &l1);
  if (r != BCHOL_OK) return r;
  int info = 0;
  if (cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return BCHOL_ERR_CUDA;
  if (info != 0) {
    *launches_out = l1;
    return BCHOL_ERR_NOT_SPD;
  }
  r = mixed_refine(n, k, nrhs, ab, ldab, b, ldb, x, ldx, max_iter, tol, tile, wsp, nrhs, st, iters_out, resid_out,
                   corr_out, &l2, nullptr);
  *launches_out = l1 + l2;
  return r;
}

}  // namespace bchol
