// solve.cu -- X = A^{-1} B from the band Cholesky factor (LAPACK pbtrs
// semantics): forward substitution L Y = B, then back substitution L^T X = Y.
// The paper factors only; the solve is the use it motivates (Sec. 1, Sec. 2).
//
// Rows are taken in blocks of 32.  With P = ceil(k/32) and blocks y_I, x_I:
//     y_I = L_II^{-1} b_I - M_I y_{I-1} - L_II^{-1} sum_{J=I-P}^{I-2} L_IJ y_J,   M_I = L_II^{-1} L_{I,I-1}
//     x_I = L_II^{-T} y_I - N_I x_{I+1} - L_II^{-T} sum_{J=I+2}^{I+P} L_JI^T x_J, N_I = (L_{I+1,I} L_II^{-1})^T
// solve_prep_kernel forms L_II^{-1}, M_I and N_I for all blocks at once.
// The sequential chain then costs one 32 x 32 matrix-vector product per block.
//
// The sweeps run on one thread-block cluster (16 CTAs, or 8 when 16 cannot
// be scheduled).  CTA 0, the leader, runs the chain.  The other CTAs (the
// workers) own the far blocks J = w-1 (mod CL-1).  One round ahead of the
// leader they form their share L_II^{-1} sum_J L_IJ y_J (worker 1 also folds
// in the L_II^{-1} b_I term) and write it into the leader's shared memory.
// The leader pushes each new block y_I into the shared memory of the worker
// that owns block I.  The workers prefetch next round's band tiles into
// registers, so no global-memory latency sits on the chain.  One cluster
// barrier separates two rounds.
#include <cooperative_groups.h>

#include <algorithm>

#include "bchol_device.cuh"
#include "bchol_internal.h"

namespace cg = cooperative_groups;

namespace bchol {

constexpr int kSB = 32;        // solve block
constexpr int kSThreads = 256;
constexpr int kSWarps = kSThreads / 32;
constexpr int kQ = kSB / kSWarps;   // columns per warp in a 32 x 32 product
constexpr int kMaxT = 6;            // far tiles per worker per round prefetched into shared memory
constexpr int kRing = kMaxT + 1;    // pushed solution blocks kept per worker
constexpr int kLd = kSB + 1;        // row pitch of a 32 x 32 block staged in shared memory
constexpr size_t kBlk = (size_t)kSB * kSB;

int solve_block(int) { return kSB; }

size_t solve_workspace_bytes(int n, int k) {
  const size_t S = (size_t)((n + kSB - 1) / kSB);
  return std::max(3 * S * kBlk * sizeof(double), psolve_workspace_bytes(n, k));
}

// Band entry L(gi, gj) (zero outside the band or the matrix).
__device__ __forceinline__ double lband(const double* __restrict__ ab, long long ldab, int n, int k, int gi, int gj) {
  const int d = gi - gj;
  return (gi < n && gj >= 0 && d >= 0 && d <= k) ? __ldg(ab + d + (long long)gj * ldab) : 0.0;
}

// Per block I: L_II^{-1}, M_I = L_II^{-1} L_{I,I-1} and N_I = (L_{I+1,I} L_II^{-1})^T,
// each 32 x 32 column-major.  Rows past n are padded with the identity.
__global__ void __launch_bounds__(256) solve_prep_kernel(const double* __restrict__ ab, long long ldab, int n, int k,
                                                         int S, double* __restrict__ linv, double* __restrict__ mfw,
                                                         double* __restrict__ nbw) {
  __shared__ double sL[kSB][kSB + 1];
  __shared__ double sInv[kSB][kSB + 1];
  __shared__ double sC[kSB][kSB + 1];
  __shared__ double rinv[kSB];
  const int I = blockIdx.x, tid = threadIdx.x;
  for (int idx = tid; idx < kSB * kSB; idx += 256) {
    const int i = idx % kSB, j = idx / kSB;
    const int gi = I * kSB + i, gj = I * kSB + j;
    double v = lband(ab, ldab, n, k, gi, gj);
    if (gi >= n && i == j) v = 1.0;
    sL[i][j] = v;
  }
  __syncthreads();
  if (tid < kSB) rinv[tid] = 1.0 / sL[tid][tid];
  __syncthreads();
  if (tid < kSB) {
    // column c of L^{-1} by forward substitution on e_c
    const int c = tid;
    double x[kSB];
#pragma unroll
    for (int i = 0; i < kSB; ++i) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < i; ++l) s = fma(sL[i][l], x[l], s);
      x[i] = (i < c) ? 0.0 : ((i == c) ? rinv[i] : -s * rinv[i]);
    }
#pragma unroll
    for (int i = 0; i < kSB; ++i) sInv[i][c] = x[i];
  }
  __syncthreads();
  double* li = linv + (size_t)I * kBlk;
  for (int idx = tid; idx < kSB * kSB; idx += 256) li[idx] = sInv[idx % kSB][idx / kSB];
  if (I >= 1) {
    for (int idx = tid; idx < kSB * kSB; idx += 256) {
      const int i = idx % kSB, j = idx / kSB;
      sC[i][j] = lband(ab, ldab, n, k, I * kSB + i, (I - 1) * kSB + j);
    }
    __syncthreads();
    double* m = mfw + (size_t)I * kBlk;
    for (int idx = tid; idx < kSB * kSB; idx += 256) {
      const int i = idx % kSB, j = idx / kSB;
      double s = 0.0;
      for (int l = 0; l <= i; ++l) s = fma(sInv[i][l], sC[l][j], s);
      m[j * kSB + i] = s;
    }
    __syncthreads();
  }
  if (I + 1 < S) {
    for (int idx = tid; idx < kSB * kSB; idx += 256) {
      const int l = idx % kSB, m = idx / kSB;
      sC[l][m] = lband(ab, ldab, n, k, (I + 1) * kSB + l, I * kSB + m);
    }
    __syncthreads();
    double* nb = nbw + (size_t)I * kBlk;
    for (int idx = tid; idx < kSB * kSB; idx += 256) {
      const int l = idx % kSB, i = idx / kSB;     // G = L_{I+1,I} L_II^{-1}; N(i,l) = G(l,i) at [l*32+i]
      double s = 0.0;
      for (int m = i; m < kSB; ++m) s = fma(sC[l][m], sInv[m][i], s);
      nb[l * kSB + i] = s;
    }
  }
}

struct SolveArgs {
  const double* ab;
  long long ldab;
  int n, k, S, P;
  double* b;
  long long ldb;
  int nrhs;
  const double* linv;
  const double* mfw;
  const double* nbw;
  int use_ring;   // far solution blocks come from the pushed ring (else from global memory)
  int rhs_per;    // right-hand-side columns per cluster (clusters split the columns)
};

// Shared-memory layout (doubles).  The leader and the workers use different
// parts of the union.  pfs/lvs hold 32 x 32 blocks, double-buffered by chain
// position, filled with cp.async: unlike plain loads, these copies do not hold
// up the release of the cluster barrier at the end of a round.  Entry (i, c)
// of a product's matrix (i the output row, c the column) sits at c * kLd + i:
// the consumer (lane = i) reads a row of consecutive words, and a copy whose
// lanes run down a band column (the backward sweep's transposed tiles) writes
// with a pitch of 33 words, so neither side has bank conflicts and every
// global read is coalesced.
// T is the arithmetic type of the sweeps: double for bchol_solve, float for
// the correction solves of the mixed-precision refinement.  Band tiles and
// the prepared blocks are always read as FP64 and rounded to T when used.
template <int NW, typename T, int NRC>
struct SolveSmem {
  union {
    T part[2][NW][NRC][kSB];             // leader: workers' shares for the next two blocks
    struct {
      double pfs[2][kMaxT][kSB * kLd];    // worker: far band tiles
      T ring[kRing][NRC][kSB];             // worker: solution blocks pushed by the leader
    } w;
  } u;
  double lvs[2][kSB * kLd];               // L_TT^{-1} (worker) or M_T / N_T (leader)
  double bpre[2][NRC][kSB];               // worker 1: the block's right-hand side (b, or y backward)
  T red[kSWarps][NRC][kSB];
  T vec[NRC][kSB];                       // leader: last chain block; worker: its partial sum
};

__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ void cp_async8(double* dst, const double* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int sz = valid ? 8 : 0;   // 0: nothing is read and the slot is zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Balanced-tree sum of N values p[0], p[stride], ... (short dependency chains).
template <int N, typename T>
__device__ __forceinline__ T tree_sum(const T* p, int stride) {
  if constexpr (N == 1) {
    return p[0];
  } else {
    constexpr int H = N / 2;
    return tree_sum<H, T>(p, stride) + tree_sum<N - H, T>(p + H * stride, stride);
  }
}

// Cross-warp sum: each warp's per-lane values acc[r] (r < nr) -> out[r][lane] (32*nr threads write).
template <int NW, typename T, int NRC>
__device__ __forceinline__ void warp_sum_rows(const T (&acc)[NRC], int nr, SolveSmem<NW, T, NRC>& sm, int w, int lane) {
#pragma unroll
  for (int r = 0; r < NRC; ++r)
    if (r < nr) sm.red[w][r][lane] = acc[r];
  __syncthreads();
}

// Band tile entry for the 32 x 32 products of the sweeps, laid out so that lane = output row i
// and column c = w + 8q: forward uses L_TJ(i, c), backward uses L_JT(c, i) (the transpose).
__device__ __forceinline__ double tile_entry(const SolveArgs& a, bool fwd, int T, int J, int i, int c) {
  return fwd ? lband(a.ab, a.ldab, a.n, a.k, T * kSB + i, J * kSB + c)
             : lband(a.ab, a.ldab, a.n, a.k, J * kSB + c, T * kSB + i);
}

// Address and validity of the same entry, for cp.async.
__device__ __forceinline__ const double* tile_addr(const SolveArgs& a, bool fwd, int T, int J, int i, int c, bool* ok) {
  const int gi = fwd ? T * kSB + i : J * kSB + c;   // row
  const int gj = fwd ? J * kSB + c : T * kSB + i;   // column
  const int d = gi - gj;
  *ok = (gi < a.n && gj >= 0 && d >= 0 && d <= a.k);
  return *ok ? a.ab + d + (long long)gj * a.ldab : a.ab;
}

template <int CL, typename VT, int NRC>
__global__ void __launch_bounds__(kSThreads, 1) solve_kernel(SolveArgs a) {
  constexpr int NW = CL - 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SolveSmem<NW, VT, NRC>& sm = *reinterpret_cast<SolveSmem<NW, VT, NRC>*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  SolveSmem<NW, VT, NRC>* leader = cluster.map_shared_rank(&sm, 0);

  // Clusters split the right-hand sides: cluster blockIdx.x / CL takes columns
  // [cid * rhs_per, (cid + 1) * rhs_per); the clusters run side by side.
  const int cid = blockIdx.x / CL;
  const int cbeg = cid * a.rhs_per, cend = min(a.nrhs, cbeg + a.rhs_per);
  for (int c0 = cbeg; c0 < cend; c0 += NRC) {
    const int nr = min(NRC, cend - c0);
    double* bc = a.b + (long long)c0 * a.ldb;
    for (int sweep = 0; sweep < 2; ++sweep) {
      const bool fwd = (sweep == 0);
      for (int idx = tid; idx < NRC * kSB; idx += kSThreads) (&sm.vec[0][0])[idx] = VT(0);
      // Registers prefetched one round ahead: the worker's far tiles and L_TT^{-1} (or its
      // transpose), or the leader's coupling block M_T / N_T.  Lane = output row i, column
      // c = w + 8q of the 32 x 32 product.
      auto prefetch = [&](int pos) {
        if (pos >= a.S) return;
        const int T = fwd ? pos : a.S - 1 - pos;
        const int buf = pos & 1;
        if (rank == 0) {
          const bool has = fwd ? (T >= 1) : (T + 1 < a.S);
          const double* cb = (fwd ? a.mfw : a.nbw) + (size_t)T * kBlk;
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const int c = w + kSWarps * q;
            cp_async8(&sm.lvs[buf][c * kLd + lane], has ? cb + c * kSB + lane : a.ab, has);
          }
          cp_async_commit();
          return;
        }
        if (rank == 1) {   // the block's b (y in the backward sweep): read before the leader overwrites it
          for (int idx = tid; idx < nr * kSB; idx += kSThreads) {
            const int r = idx / kSB, gi = T * kSB + idx % kSB;
            cp_async8(&sm.bpre[buf][r][idx % kSB], gi < a.n ? bc + gi + (long long)r * a.ldb : a.ab, gi < a.n);
          }
        }
        const double* li = a.linv + (size_t)T * kBlk;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          // the word at [x*32 + lane]: forward Linv(i = lane, c = x), backward Linv(c = lane, i = x)
          const int x = w + kSWarps * q;
          cp_async8(&sm.lvs[buf][fwd ? x * kLd + lane : lane * kLd + x], li + x * kSB + lane, true);
        }
        const int jlo = fwd ? max(0, T - a.P) : T + 2;
        const int jhi = fwd ? T - 2 : min(a.S - 1, T + a.P);
        int J = jlo + ((rank - 1) - (jlo % NW) + NW) % NW;
        for (int t = 0; t < kMaxT && J <= jhi; ++t, J += NW) {
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            // lanes run down a band column: forward i = lane, backward c = lane
            const int x = w + kSWarps * q;
            const int i = fwd ? lane : x, c = fwd ? x : lane;
            bool ok;
            const double* src = tile_addr(a, fwd, T, J, i, c, &ok);
            cp_async8(&sm.u.w.pfs[buf][t][c * kLd + i], src, ok);
          }
        }
        cp_async_commit();
      };
      // Worker: its share of chain block T (at position pos), into the leader's part slot:
      //   forward  L_TT^{-1} (sum_J L_TJ y_J  [- b_T for worker 1])
      //   backward L_TT^{-T} (sum_J L_JT^T x_J [- y_T for worker 1])
      auto worker_step = [&](int pos) {
        const int T = fwd ? pos : a.S - 1 - pos;
        const int jlo = fwd ? max(0, T - a.P) : T + 2;
        const int jhi = fwd ? T - 2 : min(a.S - 1, T + a.P);
        VT acc[NRC];
#pragma unroll
        for (int r = 0; r < NRC; ++r) acc[r] = VT(0);
        const int buf = pos & 1;
        int J = jlo + ((rank - 1) - (jlo % NW) + NW) % NW;
        for (int t = 0; J <= jhi; ++t, J += NW) {
          const VT* ring = &sm.u.w.ring[(J / NW) % kRing][0][0];
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const int c = w + kSWarps * q;
            const VT m = (VT)((t < kMaxT) ? sm.u.w.pfs[buf][t][c * kLd + lane] : tile_entry(a, fwd, T, J, lane, c));
            const int gc = J * kSB + c;
#pragma unroll
            for (int r = 0; r < NRC; ++r) {
              if (r < nr) {
                const VT v = a.use_ring ? ring[r * kSB + c]
                                       : (VT)(gc < a.n ? __ldcg(bc + gc + (long long)r * a.ldb) : 0.0);
                acc[r] = fmat(m, v, acc[r]);
              }
            }
          }
        }
        warp_sum_rows<NW, VT, NRC>(acc, nr, sm, w, lane);
        for (int idx = tid; idx < nr * kSB; idx += kSThreads) {
          const int r = idx / kSB, i = idx % kSB;
          VT s = tree_sum<kSWarps, VT>(&sm.red[0][r][i], NRC * kSB);
          if (rank == 1) s -= (VT)sm.bpre[buf][r][i];
          sm.vec[r][i] = s;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < NRC; ++r) {
          acc[r] = VT(0);
          if (r < nr) {
#pragma unroll
            for (int q = 0; q < kQ; ++q) acc[r] = fmat((VT)sm.lvs[buf][(w + kSWarps * q) * kLd + lane], sm.vec[r][w + kSWarps * q], acc[r]);
          }
        }
        warp_sum_rows<NW, VT, NRC>(acc, nr, sm, w, lane);
        for (int idx = tid; idx < nr * kSB; idx += kSThreads) {
          const int r = idx / kSB, i = idx % kSB;
          leader->u.part[T & 1][rank - 1][r][i] = tree_sum<kSWarps, VT>(&sm.red[0][r][i], NRC * kSB);
        }
      };

      // round -1: the workers' shares for the first chain block
      // Prefetches are issued one round before they are used, at the start of a
      // round, so that the HBM latency overlaps a whole round.
      prefetch(0);
      if (rank != 0) {
        cp_async_wait_all();
        prefetch(1);
        worker_step(0);
      }
      cluster.sync();
      for (int pos = 0; pos < a.S; ++pos) {
        const int T = fwd ? pos : a.S - 1 - pos;
        if (rank == 0) {
          // block T = -(M_T or N_T) * previous block - sum of the workers' shares
          const int buf = pos & 1;
          cp_async_wait_all();
          prefetch(pos + 1);
          VT acc[NRC];
#pragma unroll
          for (int r = 0; r < NRC; ++r) {
            acc[r] = VT(0);
            if (r < nr) {
#pragma unroll
              for (int q = 0; q < kQ; ++q) acc[r] = fmat((VT)sm.lvs[buf][(w + kSWarps * q) * kLd + lane], sm.vec[r][w + kSWarps * q], acc[r]);
            }
          }
          warp_sum_rows<NW, VT, NRC>(acc, nr, sm, w, lane);
          for (int idx = tid; idx < nr * kSB; idx += kSThreads) {
            const int r = idx / kSB, i = idx % kSB, gi = T * kSB + i;
            const VT y = -(tree_sum<kSWarps, VT>(&sm.red[0][r][i], NRC * kSB) +
                           tree_sum<NW, VT>(&sm.u.part[T & 1][0][r][i], NRC * kSB));
            sm.vec[r][i] = y;
            if (gi < a.n) bc[gi + (long long)r * a.ldb] = (double)y;
            if (a.use_ring) {
              SolveSmem<NW, VT, NRC>* owner = cluster.map_shared_rank(&sm, (T % NW) + 1);
              owner->u.w.ring[(T / NW) % kRing][r][i] = y;
            }
          }
        } else if (pos + 1 < a.S) {
          cp_async_wait_all();
          prefetch(pos + 2);
          worker_step(pos + 1);
        }
        cluster.sync();
      }
    }
  }
}

// Sets the launch attributes of one instantiation; false if its cluster size is refused.
template <int CL, typename VT, int NRC>
static cudaError_t prepare_kernel(bool* ok) {
  *ok = true;
  const size_t smem = sizeof(SolveSmem<CL - 1, VT, NRC>);
  cudaError_t e = cudaFuncSetAttribute(solve_kernel<CL, VT, NRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (CL > 8) {
    e = cudaFuncSetAttribute(solve_kernel<CL, VT, NRC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *ok = false;
    }
  }
  return cudaSuccess;
}

template <int CL, typename VT, int NRC>
static cudaError_t launch_columns(cudaLaunchConfig_t cfg, const SolveArgs& a) {
  bool ok = false;
  cudaError_t e = prepare_kernel<CL, VT, NRC>(&ok);
  if (e != cudaSuccess) return e;
  if (!ok) return cudaErrorInvalidConfiguration;
  cfg.dynamicSmemBytes = sizeof(SolveSmem<CL - 1, VT, NRC>);
  return cudaLaunchKernelEx(&cfg, solve_kernel<CL, VT, NRC>, a);
}

// The cluster count comes from the 8-column instantiation (the largest shared
// memory); the launch then takes the instantiation whose columns per pass
// (1, 2, 4, 8) are the fewest that hold a cluster's share, so no product or
// reduction loops over columns that are not there.
template <int CL, typename VT>
static cudaError_t launch_cluster(const SolveArgs& a0, cudaStream_t stream, bool* fits, bool need_all) {
  constexpr int NRC = 8;
  SolveArgs a = a0;
  a.use_ring = (a.P <= (CL - 1) * (kRing - 1)) ? 1 : 0;
  bool ok = false;
  cudaError_t e = prepare_kernel<CL, VT, NRC>(&ok);
  if (e != cudaSuccess) return e;
  if (!ok) {
    *fits = false;
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(kSThreads);
  cfg.dynamicSmemBytes = sizeof(SolveSmem<CL - 1, VT, NRC>);
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&clusters, solve_kernel<CL, VT, NRC>, &cfg);
  if (e != cudaSuccess || clusters < 1 || (need_all && clusters < a.nrhs)) {
    cudaGetLastError();
    *fits = false;
    return cudaSuccess;
  }
  // as many clusters as fit at once, each with an equal share of the columns
  a.rhs_per = (a.nrhs + clusters - 1) / clusters;
  const int groups = (a.nrhs + a.rhs_per - 1) / a.rhs_per;
  cfg.gridDim = dim3(CL * groups);
  *fits = true;
  if (a.rhs_per == 1) return launch_columns<CL, VT, 1>(cfg, a);
  if (a.rhs_per == 2) return launch_columns<CL, VT, 2>(cfg, a);
  if (a.rhs_per <= 4) return launch_columns<CL, VT, 4>(cfg, a);
  return launch_columns<CL, VT, NRC>(cfg, a);
}

template <typename VT>
static cudaError_t launch_solve_t(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb,
                                  void* ws, int* launches, cudaStream_t stream) {
  *launches = 0;
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (k > n - 1) k = n - 1;
  const int S = (n + kSB - 1) / kSB;
  int P = (k + kSB - 1) / kSB;
  if (P > S - 1) P = S - 1;
  double* linv = static_cast<double*>(ws);
  double* mfw = linv + (size_t)S * kBlk;
  double* nbw = mfw + (size_t)S * kBlk;
  solve_prep_kernel<<<S, 256, 0, stream>>>(ab, ldab, n, k, S, linv, mfw, nbw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  *launches = 1;
  SolveArgs a{ab, ldab, n, k, S, P, b, ldb, nrhs, linv, mfw, nbw, 1, nrhs};
  bool fits = false;
  // One column per cluster when 16-CTA clusters can cover all of them; else 8-CTA
  // clusters (more of them fit); else 16-CTA clusters with several columns each.
  e = launch_cluster<16, VT>(a, stream, &fits, true);
  if (e == cudaSuccess && !fits) e = launch_cluster<8, VT>(a, stream, &fits, true);
  if (e == cudaSuccess && !fits) e = launch_cluster<16, VT>(a, stream, &fits, false);
  if (e == cudaSuccess && !fits) e = launch_cluster<8, VT>(a, stream, &fits, false);
  if (e == cudaSuccess && !fits) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess) *launches = 2;
  return e;
}

// Path of the FP64 solve: the partitioned chunk solve (psolve.cu) for
// 1 <= k <= psolve_max_k() and at least eight chunks, where the cluster chain's
// per-block latency dominates; the cluster solve otherwise.  path: 0 automatic,
// 1 cluster, 2 partitioned (where it applies).
cudaError_t launch_solve(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb, void* ws,
                         int* launches, cudaStream_t stream, int path, int* status, uint64_t wait_ns) {
  const int kk = (n > 0 && k > n - 1) ? n - 1 : k;
  const bool part_ok = kk >= 1 && kk <= psolve_max_k() && status != nullptr;
  const bool part = part_ok && (path == 2 || (path == 0 && n >= 8 * 256));
  if (part) return launch_psolve(n, kk, nrhs, ab, ldab, b, ldb, ws, status, wait_ns, launches, stream);
  return launch_solve_t<double>(n, k, nrhs, ab, ldab, b, ldb, ws, launches, stream);
}

cudaError_t launch_solve_f32(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb,
                             void* ws, int* launches, cudaStream_t stream) {
  return launch_solve_t<float>(n, k, nrhs, ab, ldab, b, ldb, ws, launches, stream);
}

}  // namespace bchol
