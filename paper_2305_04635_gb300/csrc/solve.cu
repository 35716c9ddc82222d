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
#include <type_traits>

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
// Far clusters (one-column solves with more than 16 blocks of band below the
// diagonal, 16-CTA clusters): the group's own cluster keeps the block
// distances 2 .. 16 (one tile per worker) and up to kMaxF more clusters take
// the distances beyond.
constexpr int kMaxF = 6;            // far clusters per column group
constexpr int kFarRing = 32;        // slots of the far partial sums (>= the near distances + 2)
constexpr size_t kFarCtlBytes = 256;  // [0] positions published by the group, [1] abort, [8 + f] targets of far cluster f
constexpr size_t kBlk = (size_t)kSB * kSB;

int solve_block(int) { return kSB; }

size_t solve_workspace_bytes(int n, int k) {
  const size_t S = (size_t)((n + kSB - 1) / kSB);
  const size_t cluster = 3 * S * kBlk * sizeof(double) + kFarCtlBytes + (size_t)kMaxF * kFarRing * kSB * sizeof(double);
  return std::max(cluster, psolve_workspace_bytes(n, k));
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
  int far;        // far clusters per column group (0: none; only with one column per group)
  int dnear;      // block distances 2 .. dnear on the group's own cluster (P without far clusters)
  int* fctl;      // far-cluster control words (kFarCtlBytes, zeroed before the launch)
  double* fsum;   // far partial sums: [far][kFarRing][kSB]
  int* status;    // set to the timeout status if a bounded wait runs out
  unsigned long long wait_ns;
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
  alignas(16) double fpre[2][kMaxF][kSB];  // worker 1: the far clusters' sums for the block
  T fpart[2][NW + 1][kSB];                 // far cluster rank 0: the CTAs' partial sums of a target
  int fseen;                               // worker 1: smallest far-cluster count seen so far
};

__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ void cp_async8(double* dst, const double* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int sz = valid ? 8 : 0;   // 0: nothing is read and the slot is zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
}
// 16-byte copy through L2 only (the far sums are rewritten by other clusters; no stale L1 line).
__device__ __forceinline__ void cp_async16_cg(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
// One thread: wait until *flag >= target.  False when the group is aborted or
// the wait runs out; a timeout sets the status word and the abort word, and the
// caller goes on without waiting again (every CTA still takes all of its
// cluster barriers, so nothing hangs; the result is then wrong and the status
// says so).
__device__ __forceinline__ bool far_wait(const SolveArgs& a, const int* flag, int target) {
  if (ld_acquire(flag) >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (ld_acquire(flag) >= target) return true;
    if (ld_relaxed(&a.fctl[1]) != 0) return false;
    if (globaltimer_ns() - t0 > a.wait_ns) {
      atomicExch(a.status, kStatusTimeout);
      atomicExch(&a.fctl[1], 1);
      return false;
    }
  }
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

// A far cluster of a one-column group: for every target block T of both
// sweeps, the sum over its block distances d = D0 + e, D0 + e + stride, ...
// (D0 = dnear + 1, e = this CTA's index among the far clusters' CTAs) of
//   forward  L_{T,T-d} y_{T-d},   backward  L_{T+d,T}^T x_{T+d},
// summed over the cluster's CTAs through rank 0's shared memory and written to
// slot g % kFarRing of the cluster's far sums; its count (the targets done)
// goes out with the next target, and after the sweep's last one.  The
// solved blocks come from the column itself (the leader stores each block
// there) once the group's published count covers them; the band tiles come
// one target ahead through cp.async.  Targets at positions below D0 have no
// far terms.  Every CTA takes the same cluster barriers whatever happens to
// its waits, so an abort ends in a wrong result and the status word, not a hang.
// The cluster runs behind the chain's count in steady state, so it keeps the
// last count it acquired and polls only when that falls short, and loads the
// next target's blocks into registers while the current one is multiplied
// (L2 loads: the column is rewritten between the sweeps).  Not inlined: the
// chain cluster's code stays as compact as without far clusters.
template <int CL, typename VT, int NRC>
__device__ __noinline__ void far_cluster(const SolveArgs& a, SolveSmem<CL - 1, VT, NRC>& sm, cg::cluster_group& cluster, int f,
                            int cbeg, int cend) {
  constexpr int NW = CL - 1;
  __shared__ int s_ok, s_seen;
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  SolveSmem<NW, VT, NRC>* root = cluster.map_shared_rank(&sm, 0);
  const int D0 = a.dnear + 1, e = f * CL + rank, stride = a.far * CL;
  bool alive = true;
  if (tid == 0) s_seen = 0;
  for (int c0 = cbeg; c0 < cend; c0 += NRC) {
    const double* bc = a.b + (long long)c0 * a.ldb;
    for (int sweep = 0; sweep < 2; ++sweep) {
      const bool fwd = (sweep == 0);
      const long long base = ((long long)((c0 - cbeg) / NRC) * 2 + sweep) * a.S;
      auto tiles_at = [&](int pos) {   // this CTA's far tiles of the target at position pos
        int nt = 0;
        while (nt < kMaxT && D0 + e + nt * stride <= min(a.P, pos)) ++nt;
        return nt;
      };
      auto prefetch = [&](int pos) {
        if (pos >= a.S) return;
        const int T = fwd ? pos : a.S - 1 - pos;
        const int buf = pos & 1, nt = tiles_at(pos);
        for (int t = 0; t < nt; ++t) {
          const int d = D0 + e + t * stride, J = fwd ? T - d : T + d;
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const int x = w + kSWarps * q;
            const int i = fwd ? lane : x, c = fwd ? x : lane;
            bool ok;
            const double* src = tile_addr(a, fwd, T, J, i, c, &ok);
            cp_async8(&sm.u.w.pfs[buf][t][c * kLd + i], src, ok);
          }
        }
        cp_async_commit();
      };
      // thread idx < nt * kSB holds block entry (t, c) = (idx / kSB, idx % kSB) of a target
      auto yload = [&](int pos, int idx) {
        const int T = fwd ? pos : a.S - 1 - pos;
        const int t = idx / kSB, c = idx % kSB;
        const int d = D0 + e + t * stride, gc = (fwd ? T - d : T + d) * kSB + c;
        return gc < a.n ? __ldcg(bc + gc) : 0.0;
      };
      double ynext = 0.0;
      bool have_next = false;
      prefetch(D0);
      for (int pos = D0; pos < a.S; ++pos) {
        const int buf = pos & 1, nt = tiles_at(pos);
        const long long g = base + pos;
        cp_async_wait_all();
        prefetch(pos + 1);
        // the newest block read, at position pos - D0, is published once the count passes
        // it.  Every CTA waits, tiles or not: the wait also keeps the cluster from writing
        // slot g % kFarRing before worker 1 has copied the target kFarRing steps back.
        if (tid == 0) {
          int ok = alive ? 1 : 0;
          if (ok && s_seen < (int)(g - D0 + 1)) {
            ok = far_wait(a, &a.fctl[0], (int)(g - D0 + 1));
            s_seen = ld_acquire(&a.fctl[0]);   // an acquire: the cached count covers later reads too
          }
          s_ok = ok;
        }
        __syncthreads();
        alive = alive && s_ok;
        if (tid < nt * kSB) sm.u.w.ring[tid / kSB][0][tid % kSB] = (VT)(have_next ? ynext : yload(pos, tid));
        // the next target's blocks, if the count acquired so far covers them
        have_next = pos + 1 < a.S && s_seen >= (int)(g + 1 - D0 + 1);
        if (have_next && tid < tiles_at(pos + 1) * kSB) ynext = yload(pos + 1, tid);
        __syncthreads();
        VT acc = VT(0);
        for (int t = 0; t < nt; ++t) {
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const int c = w + kSWarps * q;
            acc = fmat((VT)sm.u.w.pfs[buf][t][c * kLd + lane], sm.u.w.ring[t][0][c], acc);
          }
        }
        sm.red[w][0][lane] = acc;
        __syncthreads();
        if (tid < kSB) root->fpart[pos & 1][rank][tid] = tree_sum<kSWarps, VT>(&sm.red[0][0][tid], NRC * kSB);
        cluster.sync();
        if (rank == 0 && tid < kSB) {
          // the count of the targets before this one goes out first: their sums were stored a
          // target ago, so the fence has nothing left to wait for and stays off the path
          if (tid == 0 && pos > D0) {
            __threadfence();   // then the count: the release pattern (warp 0 stored the sums)
            st_relaxed(&a.fctl[8 + f], (int)g);
          }
          a.fsum[((size_t)f * kFarRing + (size_t)(g % kFarRing)) * kSB + tid] =
              (double)tree_sum<CL, VT>(&sm.fpart[pos & 1][0][tid], kSB);
        }
      }
      if (rank == 0 && a.S > D0) {   // the sweep's last target
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          st_relaxed(&a.fctl[8 + f], (int)(base + a.S));
        }
      }
    }
  }
  cp_async_wait_all();
}

// FAR: the instantiation with the far-cluster roles (16-CTA clusters, FP64, one
// column); the others carry none of that code.
template <int CL, typename VT, int NRC, bool FAR = false>
__global__ void __launch_bounds__(kSThreads, 1) solve_kernel(SolveArgs a) {
  constexpr int NW = CL - 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SolveSmem<NW, VT, NRC>& sm = *reinterpret_cast<SolveSmem<NW, VT, NRC>*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  SolveSmem<NW, VT, NRC>* leader = cluster.map_shared_rank(&sm, 0);

  // Clusters split the right-hand sides: group grp = cluster / (1 + far) takes
  // columns [grp * rhs_per, (grp + 1) * rhs_per); the groups run side by side.
  // Within a group, cluster 0 runs the chain (the leader and its workers) and
  // clusters 1 .. far the far distances (far > 0 only with one column a group).
  const int ncl = FAR ? 1 + a.far : 1;
  const int cid = blockIdx.x / CL, fidx = cid % ncl, grp = cid / ncl;
  const int cbeg = grp * a.rhs_per, cend = min(a.nrhs, cbeg + a.rhs_per);
  if constexpr (FAR) {
    if (fidx > 0) {
      far_cluster<CL, VT, NRC>(a, sm, cluster, fidx - 1, cbeg, cend);
      return;
    }
  }
  constexpr bool far_on = FAR;
  const int pn = far_on ? a.dnear : a.P;   // the largest block distance this cluster's workers take
  if (rank == 1 && tid == 0) sm.fseen = 0;
  for (int c0 = cbeg; c0 < cend; c0 += NRC) {
    const int nr = min(NRC, cend - c0);
    double* bc = a.b + (long long)c0 * a.ldb;
    for (int sweep = 0; sweep < 2; ++sweep) {
      const bool fwd = (sweep == 0);
      const long long base = ((long long)((c0 - cbeg) / NRC) * 2 + sweep) * a.S;
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
          if (far_on && pos > a.dnear && w == 0) {
            // the far clusters' sums for this block: each lane acquires the counts itself
            // (bounded), unless an earlier look already saw them past this target
            const int g = (int)(base + pos);
            if (sm.fseen < g + 1) {
              int seen = 0x7fffffff;
              for (int f = 0; f < a.far; ++f) {
                far_wait(a, &a.fctl[8 + f], g + 1);
                seen = min(seen, ld_acquire(&a.fctl[8 + f]));   // acquired: later targets read under it
              }
              __syncwarp();
              if (lane == 0) sm.fseen = seen;
              __syncwarp();
            }
            for (int idx = lane; idx < a.far * (kSB / 2); idx += 32) {
              const int f = idx / (kSB / 2), h = 2 * (idx % (kSB / 2));
              cp_async16_cg(&sm.fpre[buf][f][h], a.fsum + ((size_t)f * kFarRing + (size_t)(g % kFarRing)) * kSB + h);
            }
          }
        }
        const double* li = a.linv + (size_t)T * kBlk;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          // the word at [x*32 + lane]: forward Linv(i = lane, c = x), backward Linv(c = lane, i = x)
          const int x = w + kSWarps * q;
          cp_async8(&sm.lvs[buf][fwd ? x * kLd + lane : lane * kLd + x], li + x * kSB + lane, true);
        }
        const int jlo = fwd ? max(0, T - pn) : T + 2;
        const int jhi = fwd ? T - 2 : min(a.S - 1, T + pn);
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
        const int jlo = fwd ? max(0, T - pn) : T + 2;
        const int jhi = fwd ? T - 2 : min(a.S - 1, T + pn);
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
          if (rank == 1) {
            s -= (VT)sm.bpre[buf][r][i];
            if (far_on && pos > a.dnear)
              for (int f = 0; f < a.far; ++f) s += (VT)sm.fpre[buf][f][i];
          }
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
        // the blocks of positions < pos are in the column (the leader stored them
        // before the last cluster barrier): one worker thread publishes that count
        // for the far clusters, up to the last position they read
        if (far_on && rank == NW && tid == kSThreads - 32 && pos >= 1 && pos <= a.S - 1 - a.dnear) {
          __threadfence();
          st_relaxed(&a.fctl[0], (int)(base + pos));
        }
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
  if constexpr (CL == 16 && NRC == 1 && std::is_same<VT, double>::value) {
    if (a.far > 0) {
      e = cudaFuncSetAttribute(solve_kernel<CL, VT, NRC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)cfg.dynamicSmemBytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(solve_kernel<CL, VT, NRC, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
      return cudaLaunchKernelEx(&cfg, solve_kernel<CL, VT, NRC, true>, a);
    }
  }
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
  // One column, 16-CTA clusters and block distances past 16: far clusters take
  // the distances 17 .. P, one tile per CTA where the resident clusters allow
  // (every cluster of the launch must be resident at once: the group's
  // clusters wait on one another, with bounded waits).
  if (CL == 16 && a.nrhs == 1 && a.fctl != nullptr && a.P > CL) {
    const int nf = a.P - CL;   // distances CL + 1 .. P
    int F = std::min((nf + CL - 1) / CL, std::min(kMaxF, clusters - 1));
    if (F >= 1 && (nf + F * CL - 1) / (F * CL) <= kMaxT) {
      e = cudaMemsetAsync(a.fctl, 0, kFarCtlBytes, stream);
      if (e != cudaSuccess) return e;
      a.far = F;
      a.dnear = CL;
      cfg.gridDim = dim3(CL * (1 + F));
    }
  }
  *fits = true;
  if (a.rhs_per == 1) return launch_columns<CL, VT, 1>(cfg, a);
  if (a.rhs_per == 2) return launch_columns<CL, VT, 2>(cfg, a);
  if (a.rhs_per <= 4) return launch_columns<CL, VT, 4>(cfg, a);
  return launch_columns<CL, VT, NRC>(cfg, a);
}

// status / wait_ns: the status word and the wait limit of the far clusters'
// bounded waits (status == nullptr: no far clusters).
template <typename VT>
static cudaError_t launch_solve_t(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb,
                                  void* ws, int* launches, cudaStream_t stream, int* status, uint64_t wait_ns) {
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
  a.dnear = P;
  if (status) {
    a.fctl = reinterpret_cast<int*>(nbw + (size_t)S * kBlk);
    a.fsum = reinterpret_cast<double*>(reinterpret_cast<char*>(a.fctl) + kFarCtlBytes);
    a.status = status;
    a.wait_ns = wait_ns;
  }
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
// 1 cluster, 2 partitioned (where it applies), 3 cluster without far clusters.
cudaError_t launch_solve(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb, void* ws,
                         int* launches, cudaStream_t stream, int path, int* status, uint64_t wait_ns) {
  const int kk = (n > 0 && k > n - 1) ? n - 1 : k;
  const bool part_ok = kk >= 1 && kk <= psolve_max_k() && status != nullptr;
  const bool part = part_ok && (path == 2 || (path == 0 && n >= 8 * 256));
  if (part) return launch_psolve(n, kk, nrhs, ab, ldab, b, ldb, ws, status, wait_ns, launches, stream);
  return launch_solve_t<double>(n, k, nrhs, ab, ldab, b, ldb, ws, launches, stream, path == 3 ? nullptr : status,
                                wait_ns);
}

cudaError_t launch_solve_f32(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb,
                             void* ws, int* launches, cudaStream_t stream) {
  return launch_solve_t<float>(n, k, nrhs, ab, ldab, b, ldb, ws, launches, stream, nullptr, 0);
}

}  // namespace bchol
