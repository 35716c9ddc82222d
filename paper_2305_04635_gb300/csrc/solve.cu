// solve.cu -- X = A^{-1} B from the band Cholesky factor (LAPACK pbtrs
// semantics): forward substitution L Y = B, then back substitution L^T X = Y.
// The paper factors only; the solve is the use it motivates (Sec. 1, Sec. 2).
//
// Rows are taken in blocks of 32.  With y_I the I-th block of Y,
//     y_I = L_II^{-1} (b_I - sum_{J=I-P}^{I-1} L_IJ y_J),     P = ceil(k/32),
//     x_I = L_II^{-T} (y_I - sum_{J=I+1}^{I+P} L_JI^T x_J).
// The chain over I is sequential.  To keep it short, the diagonal blocks are
// inverted first, all at once (inv_diag_kernel), so each chain step is two
// small matrix-vector products instead of a 32-step substitution.  The sweep
// runs on one thread-block cluster: CTA 0 (the leader) owns the chain and the
// nearest block L_{I,I-1}; the other CTAs compute the far contributions
// (J <= I-2) one block ahead and write their partial sums straight into the
// leader's shared memory (distributed shared memory).  One cluster barrier
// separates two chain steps.
#include <cooperative_groups.h>

#include "bchol_device.cuh"
#include "bchol_internal.h"

namespace cg = cooperative_groups;

namespace bchol {

constexpr int kSB = 32;        // solve block
constexpr int kNRC = 8;        // right-hand sides per pass
constexpr int kSThreads = 256;
constexpr int kSWarps = kSThreads / 32;

int solve_block(int) { return kSB; }

size_t solve_workspace_bytes(int n, int) {
  const size_t S = (size_t)((n + kSB - 1) / kSB);
  return S * kSB * kSB * sizeof(double);
}

// L_II^{-1} of every diagonal block, column-major per block.  Thread c forms
// column c by forward substitution on the unit vector e_c.  Rows past n are
// padded with the identity.
__global__ void __launch_bounds__(32) inv_diag_kernel(const double* __restrict__ ab, long long ldab, int n, int k,
                                                      double* __restrict__ linv) {
  __shared__ double sL[kSB * kSB];
  __shared__ double rinv[kSB];
  const int I = blockIdx.x, c = threadIdx.x;
  const int gi = I * kSB + c;
#pragma unroll 4
  for (int j = 0; j < kSB; ++j) {
    const int gj = I * kSB + j, d = gi - gj;
    sL[j * kSB + c] = (gi < n && d >= 0 && d <= k) ? ab[d + (long long)gj * ldab] : 0.0;
  }
  __syncwarp();
  rinv[c] = (gi < n) ? 1.0 / sL[c * kSB + c] : 1.0;
  __syncwarp();
  double x[kSB];
#pragma unroll
  for (int i = 0; i < kSB; ++i) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < i; ++l) s = fma(sL[l * kSB + i], x[l], s);
    x[i] = (i < c) ? 0.0 : ((i == c) ? rinv[i] : -s * rinv[i]);
  }
  double* out = linv + (size_t)I * kSB * kSB + (size_t)c * kSB;
#pragma unroll
  for (int i = 0; i < kSB; ++i) out[i] = x[i];
}

struct SolveArgs {
  const double* ab;
  long long ldab;
  int n, k, S, P;
  double* b;
  long long ldb;
  int nrhs;
  const double* linv;
};

// Band entry L(gi, gj) (zero outside the band or the matrix).
__device__ __forceinline__ double lband(const SolveArgs& a, int gi, int gj) {
  const int d = gi - gj;
  return (gi < a.n && gj >= 0 && d >= 0 && d <= a.k) ? __ldg(a.ab + d + (long long)gj * a.ldab) : 0.0;
}

// acc[rhs] += sum over this warp's columns l = w, w+8, .. of M(i, l) v[rhs][l]
// then reduce the warps' sums through shared memory into out[rhs][i].
__device__ __forceinline__ void reduce_rows(double (&acc)[kNRC], double* red, int nr, double* out) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int r = 0; r < kNRC; ++r) red[(w * kNRC + r) * kSB + lane] = acc[r];
  __syncthreads();
  if (tid < nr * kSB) {
    const int r = tid / kSB, i = tid % kSB;
    double s = 0.0;
#pragma unroll
    for (int ww = 0; ww < kSWarps; ++ww) s += red[(ww * kNRC + r) * kSB + i];
    out[r * kSB + i] = s;
  }
  __syncthreads();
}

template <int CL>
__global__ void __launch_bounds__(kSThreads, 1) solve_kernel(SolveArgs a) {
  constexpr int NW = CL - 1;
  extern __shared__ __align__(16) double smem[];
  double* part = smem;                          // [2][NW][kNRC][kSB], written by the workers
  double* red = part + 2 * NW * kNRC * kSB;     // [kSWarps][kNRC][kSB]
  double* tmp = red + kSWarps * kNRC * kSB;     // [kNRC][kSB]
  double* ycur = tmp + kNRC * kSB;              // [kNRC][kSB]: the last block of the chain
  double* sum = ycur + kNRC * kSB;              // [kNRC][kSB]
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  double* part_leader = cluster.map_shared_rank(part, 0);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;

  for (int c0 = 0; c0 < a.nrhs; c0 += kNRC) {
    const int nr = min(kNRC, a.nrhs - c0);
    double* bc = a.b + (long long)c0 * a.ldb;
    for (int sweep = 0; sweep < 2; ++sweep) {
      const bool fwd = (sweep == 0);
      if (rank == 0)
        for (int idx = tid; idx < 2 * NW * kNRC * kSB; idx += kSThreads) part[idx] = 0.0;
      cluster.sync();
      for (int step = 0; step < a.S; ++step) {
        const int I = fwd ? step : a.S - 1 - step;
        if (rank == 0) {
          // near block: L_{I,I-1} y_{I-1} (forward) or L_{I+1,I}^T x_{I+1} (backward)
          double acc[kNRC];
#pragma unroll
          for (int r = 0; r < kNRC; ++r) acc[r] = 0.0;
          const int Jn = fwd ? I - 1 : I + 1;
          if (Jn >= 0 && Jn < a.S) {
#pragma unroll
            for (int q = 0; q < kSB / kSWarps; ++q) {
              const int l = w + kSWarps * q;
              const double m = fwd ? lband(a, I * kSB + lane, Jn * kSB + l) : lband(a, Jn * kSB + l, I * kSB + lane);
#pragma unroll
              for (int r = 0; r < kNRC; ++r) acc[r] = fma(m, ycur[r * kSB + l], acc[r]);
            }
          }
          reduce_rows(acc, red, nr, sum);
          if (tid < nr * kSB) {
            const int r = tid / kSB, i = tid % kSB, gi = I * kSB + i;
            double v = (gi < a.n) ? bc[gi + (long long)r * a.ldb] : 0.0;
            v -= sum[r * kSB + i];
            const double* pp = part + (size_t)(I & 1) * NW * kNRC * kSB;
#pragma unroll 1
            for (int ww = 0; ww < NW; ++ww) v -= pp[(ww * kNRC + r) * kSB + i];
            tmp[r * kSB + i] = v;
          }
          __syncthreads();
          // y_I = L_II^{-1} tmp   or   x_I = L_II^{-T} tmp
          const double* li = a.linv + (size_t)I * kSB * kSB;
#pragma unroll
          for (int r = 0; r < kNRC; ++r) acc[r] = 0.0;
#pragma unroll
          for (int q = 0; q < kSB / kSWarps; ++q) {
            const int l = w + kSWarps * q;
            const double m = fwd ? li[l * kSB + lane] : li[lane * kSB + l];
#pragma unroll
            for (int r = 0; r < kNRC; ++r) acc[r] = fma(m, tmp[r * kSB + l], acc[r]);
          }
          reduce_rows(acc, red, nr, ycur);
          if (tid < nr * kSB) {
            const int r = tid / kSB, i = tid % kSB, gi = I * kSB + i;
            if (gi < a.n) bc[gi + (long long)r * a.ldb] = ycur[r * kSB + i];
          }
        } else {
          // far blocks of the next chain step, this worker's share
          const int T = fwd ? I + 1 : I - 1;
          if (T >= 0 && T < a.S) {
            double acc[kNRC];
#pragma unroll
            for (int r = 0; r < kNRC; ++r) acc[r] = 0.0;
            const int jlo = fwd ? max(0, T - a.P) : T + 2;
            const int jhi = fwd ? T - 2 : min(a.S - 1, T + a.P);
            int j0 = jlo + ((rank - 1) - (jlo % NW) + NW) % NW;
            for (int J = j0; J <= jhi; J += NW) {
#pragma unroll
              for (int q = 0; q < kSB / kSWarps; ++q) {
                const int l = w + kSWarps * q;
                const int gl = J * kSB + l;
                const double m = fwd ? lband(a, T * kSB + lane, gl) : lband(a, gl, T * kSB + lane);
                if (gl < a.n) {
#pragma unroll
                  for (int r = 0; r < kNRC; ++r)
                    if (r < nr) acc[r] = fma(m, __ldcg(bc + gl + (long long)r * a.ldb), acc[r]);
                }
              }
            }
            reduce_rows(acc, red, nr, sum);
            if (tid < nr * kSB) {
              const int r = tid / kSB, i = tid % kSB;
              part_leader[((size_t)(T & 1) * NW + (rank - 1)) * kNRC * kSB + r * kSB + i] = sum[r * kSB + i];
            }
          }
        }
        cluster.sync();
      }
    }
  }
}

template <int CL>
static cudaError_t launch_cluster(const SolveArgs& a, cudaStream_t stream, bool* fits) {
  const size_t smem = sizeof(double) * (size_t)(2 * (CL - 1) * kNRC * kSB + kSWarps * kNRC * kSB + 3 * kNRC * kSB);
  cudaError_t e = cudaFuncSetAttribute(solve_kernel<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (CL > 8) {
    e = cudaFuncSetAttribute(solve_kernel<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *fits = false;
      return cudaSuccess;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(kSThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&clusters, solve_kernel<CL>, &cfg);
  if (e != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    *fits = false;
    return cudaSuccess;
  }
  *fits = true;
  return cudaLaunchKernelEx(&cfg, solve_kernel<CL>, a);
}

cudaError_t launch_solve(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb, void* ws,
                         int* launches, cudaStream_t stream) {
  *launches = 0;
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (k > n - 1) k = n - 1;
  const int S = (n + kSB - 1) / kSB;
  int P = (k + kSB - 1) / kSB;
  if (P > S - 1) P = S - 1;
  double* linv = static_cast<double*>(ws);
  inv_diag_kernel<<<S, 32, 0, stream>>>(ab, ldab, n, k, linv);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  *launches = 1;
  SolveArgs a{ab, ldab, n, k, S, P, b, ldb, nrhs, linv};
  bool fits = false;
  e = launch_cluster<16>(a, stream, &fits);
  if (e == cudaSuccess && !fits) e = launch_cluster<8>(a, stream, &fits);
  if (e == cudaSuccess && !fits) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess) *launches = 2;
  return e;
}

}  // namespace bchol
