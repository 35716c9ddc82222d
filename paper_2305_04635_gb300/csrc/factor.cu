// factor.cu -- the persistent band Cholesky kernel.
//
// Method (Sec. 3 of Liu, Fredriksson, Markidis, arXiv 2305.04635): the active
// window of the band is cut into b x b tiles.  Step s of the factorization
// (one "outer iteration" of Algorithm 1) is
//     POTRF(s)       L_ss L_ss^T = A_ss                         (dense Cholesky)
//     TRSM(I,s)      L_Is = A_Is L_ss^{-T},        I = s+1..s+p (DTRSM)
//     UPD(I,J,s)     A_IJ -= L_Is L_Js^T,  s < J <= I <= s+p    (DGEMM; DSYRK when I == J)
// with p = ceil(k/b) panel tiles below the diagonal tile.  The tiles of the
// last panel row are cut by the band; they are masked on load and store
// instead of going through the paper's zeroed work array.
//
// Scheduling replaces the paper's OpenMP task graph (Sec. 3.1) with one
// persistent launch.  Each CTA claims tasks from a monotone ticket counter in
// a topological order with one step of lookahead (schedule.cuh): the update
// of the next panel column and the next panel come before the rest of the
// current step's trailing update.  Every tile position (I,J) carries a
// ready counter in global memory, which is the paper's cross-iteration
// overlap (Sec. 3): the tile of step s+1 that overlaps tile (I+1,J+1) of step
// s waits for that tile's update, not for a barrier.  The counter of tile
// (I,J) holds how many of its updates (steps s0(I) = max(0, I-p) .. J-1) are
// done; it reaches J - s0(I) + 1 when the tile is final (POTRF or TRSM done).
// A task waits only for tasks with smaller tickets, which are running or
// finished, so the walk cannot deadlock; every wait is bounded in time.
#include <cstdio>

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
};

__device__ __forceinline__ int fidx(const FactorArgs& a, int I, int J) { return J * (a.p + 1) + (I - J); }
__device__ __forceinline__ int first_step(const FactorArgs& a, int I) { return I - a.p > 0 ? I - a.p : 0; }

// Wait (one thread) until the ready counter of tile (I,J) reaches `target`.
__device__ __forceinline__ bool wait_tile(const FactorArgs& a, int I, int J, int target) {
  const int f = fidx(a, I, J);
  if (f == a.stall) target = 0x7fffffff;
  return wait_flag_geq(&a.flags[f], target, a.ctl, a.status, a.wait_ns);
}

constexpr int kThreads = 256;

template <int B>
struct Smem {
  double t0[B * B];
  double t1[B * B];
};

// Publish: every thread's stores are done (barrier), then one release store.
__device__ __forceinline__ void publish(int* flag, int value) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(flag, value);
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
// the columns l = sub (mod TPR) in registers; column j's value is formed by
// its owner and shuffled to the row group.  No block barriers in the loop.
template <int B>
__device__ bool task_trsm(const FactorArgs& a, int I, int s, Smem<B>& sm, int* s_flag) {
  constexpr int TPR = kThreads / B;
  constexpr int R = B / TPR;
  __shared__ double s_rinv[B];
  const int tid = threadIdx.x;
  if (tid == 0) {
    bool ok = wait_tile(a, s, s, s - first_step(a, s) + 1);
    if (ok) ok = wait_tile(a, I, s, s - first_step(a, I));
    *s_flag = ok;
  }
  __syncthreads();
  if (!*s_flag) return false;
  double* sX = sm.t0;
  double* sL = sm.t1;
  load_tile<B, kThreads>(a.ab, a.ldab, a.n, a.k, I, s, sX);
  load_tile<B, kThreads>(a.ab, a.ldab, a.n, a.k, s, s, sL);
  __syncthreads();
  const int jmax = min(B, a.n - s * B);
  if (tid < B) s_rinv[tid] = (tid < jmax) ? 1.0 / sL[tid * B + tid] : 0.0;
  const int i = tid / TPR, sub = tid % TPR;
  double acc[R];
#pragma unroll
  for (int q = 0; q < R; ++q) acc[q] = sX[(sub + q * TPR) * B + i];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < B; ++j) {
    const int owner = j % TPR, qj = j / TPR;
    double x = 0.0;
    if (sub == owner) {
      x = acc[qj] * s_rinv[j];
      acc[qj] = x;
    }
    x = __shfl_sync(0xffffffffu, x, owner, TPR);
#pragma unroll
    for (int q = qj; q < R; ++q) {
      const int l = sub + q * TPR;
      if (l > j) acc[q] = fma(-x, sL[j * B + l], acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < R; ++q) sX[(sub + q * TPR) * B + i] = acc[q];
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
template <int B>
__device__ bool task_upd(const FactorArgs& a, int I, int J, int s, Smem<B>& sm, int* s_flag) {
  constexpr int R = B / 16;
  const int tid = threadIdx.x;
  const int s0I = first_step(a, I);
  if (tid == 0) {
    bool ok = wait_tile(a, I, s, s - s0I + 1);
    if (ok && J != I) ok = wait_tile(a, J, s, s - first_step(a, J) + 1);
    if (ok) ok = wait_tile(a, I, J, s - s0I);
    *s_flag = ok;
  }
  __syncthreads();
  if (!*s_flag) return false;
  double* sA = sm.t0;
  double* sB = sm.t1;
  load_tile<B, kThreads>(a.ab, a.ldab, a.n, a.k, I, s, sA);
  if (J != I) load_tile<B, kThreads>(a.ab, a.ldab, a.n, a.k, J, s, sB);
  const double* sBr = (J != I) ? sB : sA;
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

template <int B>
__global__ void __launch_bounds__(kThreads, 2) factor_kernel(FactorArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<B>& sm = *reinterpret_cast<Smem<B>*>(smem_raw);
  __shared__ long long s_task;
  __shared__ int s_flag;
  unsigned long long next = 0;
  if (threadIdx.x == 0) next = atomicAdd(&a.ctl->ticket, 1ULL);
  while (true) {
    if (threadIdx.x == 0) s_task = (long long)next;
    __syncthreads();
    const long long t = s_task;
    if (t >= (long long)a.total) break;
    if (threadIdx.x == 0) next = atomicAdd(&a.ctl->ticket, 1ULL);  // claim the next task early
    int type, s, I, J;
    decode_task(Schedule{a.S, a.p, a.Sreg, a.Treg}, t, type, s, I, J);
    bool ok;
    if (type == kPotrf)
      ok = task_potrf<B>(a, s, sm, &s_flag);
    else if (type == kTrsm)
      ok = task_trsm<B>(a, I, s, sm, &s_flag);
    else
      ok = task_upd<B>(a, I, J, s, sm, &s_flag);
    if (!ok) break;
  }
}

FactorPlan make_factor_plan(int n, int k, int b) {
  FactorPlan P;
  P.n = n;
  P.k = (n > 0 && k > n - 1) ? n - 1 : k;
  P.b = b;
  if (n <= 0) return P;
  P.S = (n + b - 1) / b;
  P.p = (P.k + b - 1) / b;
  if (P.p > P.S - 1) P.p = P.S - 1;
  P.Sreg = (P.S - 1 - P.p > 0) ? P.S - 1 - P.p : 0;
  P.Treg = 2LL * P.p + 1 + (long long)P.p * (P.p - 1) / 2;
  const Schedule sc{P.S, P.p, P.Sreg, P.Treg};
  unsigned long long total = 1 + (unsigned long long)sched_m(sc, 0);
  total += (unsigned long long)P.Sreg * (unsigned long long)P.Treg;
  for (int s = (int)P.Sreg; s < P.S; ++s) total += (unsigned long long)sched_block_size(sc, s);
  P.total = total;
  P.flag_count = (size_t)P.S * (size_t)(P.p + 1);
  return P;
}

size_t factor_workspace_bytes(const FactorPlan& P) { return 256 + P.flag_count * sizeof(int); }

template <int B>
static cudaError_t launch_b(const FactorArgs& a, int ctas_per_sm, cudaStream_t stream) {
  const size_t smem = sizeof(Smem<B>);
  cudaError_t e = cudaFuncSetAttribute(factor_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, factor_kernel<B>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  long long grid = (long long)per_sm * num_sms();
  if ((unsigned long long)grid > a.total) grid = (long long)a.total;
  factor_kernel<B><<<(unsigned)grid, kThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_factor(const FactorPlan& P, double* ab, long long ldab, int* info, void* ws, int* status,
                          uint64_t wait_ns, int ctas_per_sm, int stall_I, int stall_J, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int), stream);
  if (e != cudaSuccess || P.n <= 0) return e;
  e = cudaMemsetAsync(ws, 0, factor_workspace_bytes(P), stream);
  if (e != cudaSuccess) return e;
  FactorArgs a;
  a.ab = ab;
  a.ldab = ldab;
  a.n = P.n;
  a.k = P.k;
  a.S = P.S;
  a.p = P.p;
  a.Sreg = P.Sreg;
  a.Treg = P.Treg;
  a.total = P.total;
  a.ctl = reinterpret_cast<Control*>(ws);
  a.flags = reinterpret_cast<int*>(static_cast<char*>(ws) + 256);
  a.status = status;
  a.info = info;
  a.wait_ns = wait_ns;
  a.stall = -1;
  if (stall_I >= 0 && stall_J >= 0 && stall_I < P.S && stall_J <= stall_I && stall_I - stall_J <= P.p)
    a.stall = stall_J * (P.p + 1) + (stall_I - stall_J);
  switch (P.b) {
    case 16: return launch_b<16>(a, ctas_per_sm, stream);
    case 32: return launch_b<32>(a, ctas_per_sm, stream);
    case 64: return launch_b<64>(a, ctas_per_sm, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bchol
