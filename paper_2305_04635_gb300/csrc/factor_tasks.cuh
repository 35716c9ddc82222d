// factor_tasks.cuh -- the tile tasks of the band factorization (POTRF, TRSM,
// UPD), shared by the single-matrix and the batched persistent kernels.
// The method and the ready-counter protocol are described in factor.cu.
#pragma once
#include "bchol_device.cuh"
#include "bchol_internal.h"
#include "schedule.cuh"

namespace bchol {

struct FactorArgs {
  double* ab;
  long long ldab;
  int n, k, S, p;
  long long Sreg, Treg;
  unsigned long long total;
  int* flags;
  Control* ctl;
  int* status;
  int* info;
  uint64_t wait_ns;
  int stall;  // flag index whose waits never succeed (failure-path test hook), or -1
  int H;      // strip height of the ticket order (1: one tile per update task)
  int tma = 0;  // the chain's prefetch warps copy A(s, s), A(s, s-1) with TMA (the kernel's tensor map)
};

__device__ __forceinline__ int fidx(const FactorArgs& a, int I, int J) { return J * (a.p + 1) + (I - J); }
__device__ __forceinline__ int first_step(const FactorArgs& a, int I) { return I - a.p > 0 ? I - a.p : 0; }

// Wait (one thread) until the ready counter of tile (I,J) reaches `target`.
__device__ __forceinline__ bool wait_tile(const FactorArgs& a, int I, int J, int target) {
  const int f = fidx(a, I, J);
  if (f == a.stall) target = 0x7fffffff;
  return wait_flag_geq(&a.flags[f], target, a.ctl, a.status, a.wait_ns);
}

// Wait (one thread) until each of the cnt ready counters f[q] (flag indices)
// reaches t[q].  From three counters on (the strips), they are read with
// relaxed loads, all in flight together, and one acquire fence follows when
// every target is met: one L2 round trip where acquire loads one after another
// would take cnt (an acquire load holds back the memory operations after it).
// Otherwise (one or two counters, where the GPU-scope fence costs about what it
// saves), and for the test hook's stalled counter, the bounded waits of
// wait_tile, one at a time.
template <int N>
__device__ __forceinline__ bool wait_tiles(const FactorArgs& a, const int (&f)[N], const int (&t)[N], int cnt) {
  if (cnt <= 2) {
    for (int q = 0; q < cnt; ++q) {
      const int target = f[q] == a.stall ? 0x7fffffff : t[q];
      if (!wait_flag_geq(&a.flags[f[q]], target, a.ctl, a.status, a.wait_ns)) return false;
    }
    return true;
  }
  int v[N];
#pragma unroll
  for (int q = 0; q < N; ++q) v[q] = q < cnt ? ld_relaxed(&a.flags[f[q]]) : 0;
  bool met = true;
#pragma unroll
  for (int q = 0; q < N; ++q)
    if (q < cnt && (v[q] < t[q] || f[q] == a.stall)) met = false;
  if (met) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return true;
  }
  for (int q = 0; q < cnt; ++q) {
    const int target = f[q] == a.stall ? 0x7fffffff : t[q];
    if (!wait_flag_geq(&a.flags[f[q]], target, a.ctl, a.status, a.wait_ns)) return false;
  }
  return true;
}

constexpr int kThreads = 256;

template <int B>
struct Smem {
  double t0[B * B];
  double t1[B * B];
};

// Publish: every thread's stores are done (barrier), then one fence and a
// relaxed store of the counter (the release pattern, with a single fence).
__device__ __forceinline__ void publish(int* flag, int value) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_relaxed(flag, value);
  }
}

// ---------------------------------------------------------------- POTRF(s)
// Right-looking Cholesky of the diagonal tile in shared memory, one column
// per barrier.  TPR threads share a row; the thread that updates the next
// pivot computes its reciprocal square root right away, so the pivot is ready
// when the barrier opens.  A pivot that is not > 0 (NaN included) stops the
// launch and sets info to its 1-based global column (LAPACK convention).
template <int B>
__device__ bool task_potrf(const FactorArgs& a, int s, Smem<B>& sm, int* s_flag) {
  constexpr int TPR = kThreads / B;
  __shared__ double s_rinv[B], s_ljj[B];
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  const int s0 = first_step(a, s);
  if (tid == 0) *s_flag = wait_tile(a, s, s, s - s0);
  __syncthreads();
  if (!*s_flag) return false;
  double* sA = sm.t0;
  double* sL = sm.t1;
  load_tile<B, kThreads>(a.ab, a.ldab, a.n, a.k, s, s, sA);
  for (int idx = tid; idx < B * B; idx += kThreads) sL[idx] = 0.0;
  const int jmax = min(B, a.n - s * B);
  __syncthreads();
  if (tid == 0) {
    s_fail = 0;
    const double d = sA[0];
    if (!(d > 0.0)) {
      s_fail = 1;
    } else {
      const double r = rsqrt(d);
      s_rinv[0] = r;
      s_ljj[0] = d * r;
    }
  }
  __syncthreads();
  const int i = tid / TPR, sub = tid % TPR;
  for (int j = 0; j < jmax; ++j) {
    if (s_fail) break;
    const double r = s_rinv[j];
    if (i > j && i < jmax) {
      const double x = sA[j * B + i] * r;  // L(i,j)
      const double y = x * r;              // A(i,j) / A(j,j)
      if (sub == 0) sL[j * B + i] = x;
      for (int l = j + 1 + sub; l <= i; l += TPR) {
        const double v = fma(-y, sA[j * B + l], sA[l * B + i]);
        sA[l * B + i] = v;
        if (l == i && i == j + 1) {  // the next pivot
          if (!(v > 0.0)) {
            s_fail = j + 2;
          } else {
            const double rr = rsqrt(v);
            s_rinv[j + 1] = rr;
            s_ljj[j + 1] = v * rr;
          }
        }
      }
    }
    if (tid == 0) sL[j * B + j] = s_ljj[j];
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) {
      atomicCAS(a.info, 0, s * B + s_fail);
      atomicExch(&a.ctl->abort, 1);
    }
    return false;
  }
  store_tile<B, kThreads>(a.ab, a.ldab, a.n, a.k, s, s, sL);
  publish(&a.flags[fidx(a, s, s)], s - s0 + 1);
  return true;
}

// ---------------------------------------------------------------- TRSM(I,s)
// X = A_Is L_ss^{-T}, row by row: TPR threads own a row, thread `sub` keeps
// the columns l = sub (mod TPR) in registers; column j's value, final when the
// sweep reaches it, is shuffled to the row group.  No block barriers in the
// loop, and no division or scaling on its chain (the unit lower form below).
template <int B>
__device__ bool task_trsm(const FactorArgs& a, int I, int s, Smem<B>& sm, int* s_flag) {
  constexpr int TPR = kThreads / B;
  constexpr int R = B / TPR;
  __shared__ double s_rinv[B];
  const int tid = threadIdx.x;
  if (tid == 0) {
    const int f[2] = {fidx(a, s, s), fidx(a, I, s)};
    const int t[2] = {s - first_step(a, s) + 1, s - first_step(a, I)};
    bool ok = wait_tiles(a, f, t, 2);
    *s_flag = ok;
  }
  __syncthreads();
  if (!*s_flag) return false;
  double* sX = sm.t0;
  double* sL = sm.t1;
  load_tile2<B, kThreads>(a.ab, a.ldab, a.n, a.k, I, s, sX, s, s, sL);
  __syncthreads();
  const int jmax = min(B, a.n - s * B);
  if (tid < B) s_rinv[tid] = (tid < jmax) ? 1.0 / sL[tid * B + tid] : 0.0;
  __syncthreads();
  // X L^T = A with L = U diag(L_jj), U unit lower: the rows of Z = X diag(L_jj)
  // solve Z U^T = A, one shuffle and one DFMA per step (no scaling on the
  // chain), and X = Z diag(1 / L_jj) at the end.
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int l = idx % B, j = idx / B;
    if (l > j) sL[idx] *= s_rinv[j];
  }
  const int i = tid / TPR, sub = tid % TPR;
  double acc[R];
#pragma unroll
  for (int q = 0; q < R; ++q) acc[q] = sX[(sub + q * TPR) * B + i];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < B - 1; ++j) {
    const int owner = j % TPR, qj = j / TPR;
    const double z = __shfl_sync(0xffffffffu, acc[qj], owner, TPR);
#pragma unroll
    for (int q = qj; q < R; ++q) {
      const int l = sub + q * TPR;
      if (l > j) acc[q] = fma(-z, sL[j * B + l], acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < R; ++q) sX[(sub + q * TPR) * B + i] = acc[q] * s_rinv[sub + q * TPR];
  __syncthreads();
  store_tile<B, kThreads>(a.ab, a.ldab, a.n, a.k, I, s, sX);
  publish(&a.flags[fidx(a, I, s)], s - first_step(a, I) + 1);
  return true;
}

// ---------------------------------------------------------------- UPD(I,J,s)
// A_IJ -= L_Is L_Js^T: the two panel tiles are staged in shared memory, the
// updated tile stays in registers (an R x R block per thread, rows ty+16r and
// columns tx+16c).  On a diagonal tile (the DSYRK case) the blocks that lie
// wholly above the diagonal are skipped.
// With lis_in_smem, L_Is is already in sm.t0 (the same CTA has just solved it
// with task_trsm, which leaves its result there) and is neither waited for nor
// read again.
template <int B>
__device__ bool task_upd(const FactorArgs& a, int I, int J, int s, Smem<B>& sm, int* s_flag,
                         bool lis_in_smem = false) {
  constexpr int R = B / 16;
  const int tid = threadIdx.x;
  const int s0I = first_step(a, I);
  // L_Is and A_IJ are usually final first; L_Js of the next block column comes
  // last (for UPD(I, s+1, s) it is the diagonal chain's TRSM), so it is waited
  // for and loaded after the others are already in flight.
  if (tid == 0) {
    const int f[2] = {fidx(a, I, J), fidx(a, I, s)};
    const int t[2] = {s - s0I, s - s0I + 1};
    bool ok = wait_tiles(a, f, t, lis_in_smem ? 1 : 2);
    *s_flag = ok;
  }
  __syncthreads();
  if (!*s_flag) return false;
  double* sA = sm.t0;
  double* sB = sm.t1;
  // Both L tiles go through registers and reach shared memory together, so
  // that the loads of L_Is are still in flight while L_Js is waited for.
  constexpr int E = B * B / kThreads;
  double li[E], lj[E];
  if (!lis_in_smem) {
#pragma unroll
    for (int e = 0; e < E; ++e) li[e] = tile_elem(a.ab, a.ldab, a.n, a.k, I, s, tid + e * kThreads, B);
  }
  const int ty = tid / 16, tx = tid % 16;
  const bool diag = (I == J);
  double acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int gi = I * B + ty + 16 * r, gj = J * B + tx + 16 * c;
      const int d = gi - gj;
      acc[r][c] = (gi < a.n && d >= 0 && d <= a.k) ? __ldcg(a.ab + d + (long long)gj * a.ldab) : 0.0;
    }
  if (J != I) {
    __shared__ int s_ok_j;  // not s_flag: other threads may still be reading that one
    if (tid == 0) s_ok_j = wait_tile(a, J, s, s - first_step(a, J) + 1);
    __syncthreads();
    if (!s_ok_j) return false;
#pragma unroll
    for (int e = 0; e < E; ++e) lj[e] = tile_elem(a.ab, a.ldab, a.n, a.k, J, s, tid + e * kThreads, B);
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = tid + e * kThreads;
    if (!lis_in_smem) sA[idx] = li[e];
    if (J != I) sB[idx] = lj[e];
  }
  const double* sBr = (J != I) ? sB : sA;
  __syncthreads();
#pragma unroll 4
  for (int l = 0; l < B; ++l) {
    double av[R], bv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) av[r] = sA[l * B + ty + 16 * r];
#pragma unroll
    for (int c = 0; c < R; ++c) bv[c] = sBr[l * B + tx + 16 * c];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c)
        if (!(diag && r < c)) acc[r][c] = fma(-av[r], bv[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int gi = I * B + ty + 16 * r, gj = J * B + tx + 16 * c;
      const int d = gi - gj;
      if (gi < a.n && d >= 0 && d <= a.k) a.ab[d + (long long)gj * a.ldab] = acc[r][c];
    }
  publish(&a.flags[fidx(a, I, J)], s - s0I + 1);
  return true;
}

// ------------------------------------------------------------ TRSM, FP32
// The mixed-precision form of TRSM: X = A_Is L_ss^{-T} with both tiles
// rounded to FP32 and the substitution in FP32; the result is stored in the
// FP64 band.  (The diagonal POTRF stays FP64; refinement of the solve
// recovers FP64 accuracy.)
template <int B>
__device__ bool task_trsm_f32(const FactorArgs& a, int I, int s, Smem<B>& sm, int* s_flag) {
  constexpr int TPR = kThreads / B;
  constexpr int R = B / TPR;
  __shared__ float s_rinv32[B];
  const int tid = threadIdx.x;
  if (tid == 0) {
    const int f[2] = {fidx(a, s, s), fidx(a, I, s)};
    const int t[2] = {s - first_step(a, s) + 1, s - first_step(a, I)};
    bool ok = wait_tiles(a, f, t, 2);
    *s_flag = ok;
  }
  __syncthreads();
  if (!*s_flag) return false;
  float* fX = reinterpret_cast<float*>(sm.t0);
  float* fL = reinterpret_cast<float*>(sm.t1);
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int i = idx % B, j = idx / B;
    int gi = I * B + i, gj = s * B + j, d = gi - gj;
    fX[j * B + i] = (gi < a.n && d >= 0 && d <= a.k) ? (float)__ldcg(a.ab + d + (long long)gj * a.ldab) : 0.0f;
    gi = s * B + i;
    d = gi - gj;
    fL[j * B + i] = (gi < a.n && d >= 0 && d <= a.k) ? (float)__ldcg(a.ab + d + (long long)gj * a.ldab) : 0.0f;
  }
  __syncthreads();
  const int jmax = min(B, a.n - s * B);
  if (tid < B) s_rinv32[tid] = (tid < jmax) ? 1.0f / fL[tid * B + tid] : 0.0f;
  const int i = tid / TPR, sub = tid % TPR;
  float acc[R];
#pragma unroll
  for (int q = 0; q < R; ++q) acc[q] = fX[(sub + q * TPR) * B + i];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < B; ++j) {
    const int owner = j % TPR, qj = j / TPR;
    float x = 0.0f;
    if (sub == owner) {
      x = acc[qj] * s_rinv32[j];
      acc[qj] = x;
    }
    x = __shfl_sync(0xffffffffu, x, owner, TPR);
#pragma unroll
    for (int q = qj; q < R; ++q) {
      const int l = sub + q * TPR;
      if (l > j) acc[q] = fmaf(-x, fL[j * B + l], acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int gi = I * B + i, gj = s * B + sub + q * TPR, d = gi - gj;
    if (gi < a.n && d >= 0 && d <= a.k) a.ab[d + (long long)gj * a.ldab] = (double)acc[q];
  }
  publish(&a.flags[fidx(a, I, s)], s - first_step(a, I) + 1);
  return true;
}

// ------------------------------------------------------------ UPD, FP32 update
// The mixed-precision form of UPD: the two panel tiles are rounded to FP32,
// their product L_Is L_Js^T is accumulated in FP32 (FFMA), and the FP64 tile
// is updated by that product, A_IJ -= (double) P.  POTRF and TRSM stay FP64.
template <int B>
__device__ bool task_upd_f32(const FactorArgs& a, int I, int J, int s, Smem<B>& sm, int* s_flag) {
  constexpr int R = B / 16;
  constexpr int E = B * B / kThreads;
  const int tid = threadIdx.x;
  const int s0I = first_step(a, I);
  // As in task_upd: L_Is and A_IJ first, with their loads in flight while
  // L_Js is waited for; A_IJ goes straight to registers.
  if (tid == 0) {
    const int f[2] = {fidx(a, I, s), fidx(a, I, J)};
    const int t[2] = {s - s0I + 1, s - s0I};
    bool ok = wait_tiles(a, f, t, 2);
    *s_flag = ok;
  }
  __syncthreads();
  if (!*s_flag) return false;
  float* fA = reinterpret_cast<float*>(sm.t0);
  float* fB = reinterpret_cast<float*>(sm.t1);
  double li[E], lj[E];
#pragma unroll
  for (int e = 0; e < E; ++e) li[e] = tile_elem(a.ab, a.ldab, a.n, a.k, I, s, tid + e * kThreads, B);
  const int ty = tid / 16, tx = tid % 16;
  const bool diag = (I == J);
  double aij[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int gi = I * B + ty + 16 * r, gj = J * B + tx + 16 * c;
      const int d = gi - gj;
      aij[r][c] = (gi < a.n && d >= 0 && d <= a.k) ? __ldcg(a.ab + d + (long long)gj * a.ldab) : 0.0;
    }
  if (J != I) {
    __shared__ int s_ok_j32;  // not s_flag: other threads may still be reading that one
    if (tid == 0) s_ok_j32 = wait_tile(a, J, s, s - first_step(a, J) + 1);
    __syncthreads();
    if (!s_ok_j32) return false;
#pragma unroll
    for (int e = 0; e < E; ++e) lj[e] = tile_elem(a.ab, a.ldab, a.n, a.k, J, s, tid + e * kThreads, B);
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = tid + e * kThreads;
    fA[idx] = (float)li[e];
    if (J != I) fB[idx] = (float)lj[e];
  }
  const float* fBr = (J != I) ? fB : fA;
  float acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = 0.0f;
  __syncthreads();
#pragma unroll 4
  for (int l = 0; l < B; ++l) {
    float av[R], bv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) av[r] = fA[l * B + ty + 16 * r];
#pragma unroll
    for (int c = 0; c < R; ++c) bv[c] = fBr[l * B + tx + 16 * c];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c)
        if (!(diag && r < c)) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int gi = I * B + ty + 16 * r, gj = J * B + tx + 16 * c;
      const int d = gi - gj;
      if (gi < a.n && d >= 0 && d <= a.k) a.ab[d + (long long)gj * a.ldab] = aij[r][c] - (double)acc[r][c];
    }
  publish(&a.flags[fidx(a, I, J)], s - s0I + 1);
  return true;
}

}  // namespace bchol
