// batched.cu -- many independent band systems of uneven n and k in one
// persistent factor launch plus one solve launch (the batched form of the
// paper's factorization; the paper itself factors one matrix at a time).
//
// Factor: every matrix keeps its own tile schedule (schedule.cuh), ready
// counters and ticket counter.  A CTA does not block on one matrix: warp 0
// probes the next ticket of 32 matrices at once, checks whether that task's
// inputs are already final (acquire loads of its ready counters), and claims
// the first ready one with a compare-and-swap on that matrix's ticket.  The
// task then runs with the same code as the single-matrix kernel; its waits
// return at once.  Since no CTA ever waits for a task that has not started,
// the launch cannot deadlock; a CTA that finds no ready task for longer than
// the wait limit records a timeout and stops.  While one matrix's step chain
// is busy, the CTAs work on the others, which hides the latency of the chain.
// With the split updates (BCHOL_FP64_SPLIT, tiles of 16 or 32) each matrix's
// trailing updates are strips of 128 / b tiles (decode_st_task), run as split
// products on the tensor cores (strip_task.cuh); every CTA then holds 256
// (tiles of 32) or 128 (tiles of 16) tensor-memory columns for its lifetime.
//
// Solve: one CTA per matrix, largest first, forward then back substitution
// in blocks of 32 rows (batched_solve.cuh: the chain on four warps, one per
// SM sub-partition, the far terms and the next block's tiles one block ahead
// on the other four).
#include <algorithm>
#include <vector>

#include "../../include/bchol.h"
#include "batched_solve.cuh"
#include "bchol_internal.h"
#include "strip_task.cuh"

namespace bchol {

struct BatchMat {
  double* ab;
  long long ldab;
  int n, k, S, p;
  long long Sreg, Treg;
  unsigned long long total;
  long long flag_off;   // offset (ints) of this matrix's ready counters in the pool
  int* info;
  double* b;
  long long ldb;
  int nrhs;
  int H;                // strip height of the updates (1: one tile per update task)
  long long part_off;   // solve: offset (doubles) of this system's worker partial sums in the pool
  int W;                // solve: worker CTAs of this system (batched_solve.cuh)
  int pad2;
};

struct BatchArgs {
  const BatchMat* mats;
  Control* ctl;         // per matrix: ticket, abort word, retired mark
  int* flags;
  int count;
  int* retired;         // number of matrices with no task left to claim
  unsigned long long* progress;   // tasks claimed so far (all CTAs)
  int* status;
  uint64_t wait_ns;
};

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void decode_mat_task(const FactorArgs& a, long long t, int& type, int& s, int& I, int& J) {
  const Schedule sc{a.S, a.p, a.Sreg, a.Treg, a.H};
  if (a.H > 1)
    decode_st_task(sc, t, type, s, I, J);
  else
    decode_task(sc, t, type, s, I, J);
}

__device__ __forceinline__ FactorArgs matrix_args(const BatchArgs& g, int m) {
  const BatchMat& M = g.mats[m];
  FactorArgs a;
  a.ab = M.ab;
  a.ldab = M.ldab;
  a.n = M.n;
  a.k = M.k;
  a.S = M.S;
  a.p = M.p;
  a.Sreg = M.Sreg;
  a.Treg = M.Treg;
  a.total = M.total;
  a.flags = g.flags + M.flag_off;
  a.ctl = g.ctl + m;
  a.status = g.status;
  a.info = M.info;
  a.wait_ns = g.wait_ns;
  a.stall = -1;
  a.H = M.H;
  return a;
}

// Are the inputs of task (type, s, I, J) final?  The same targets as the waits
// in the tasks.  A probe only: relaxed loads, all in flight together (the task
// itself then waits with acquire ordering, and finds them met).
__device__ __forceinline__ bool task_ready(const FactorArgs& a, int type, int s, int I, int J) {
  if (type == kStrip) {  // STRIP(I, J, s): every tile's panel tile and previous update, and L_Js
    const int h = strip_rows(a.H, s, min(a.p, a.S - 1 - s), I);
    int v[2 * 8 + 1], t[2 * 8 + 1];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool on = q < h;
      const int Ii = I + (on ? q : 0), s0 = first_step(a, Ii);
      v[2 * q] = on ? ld_relaxed(&a.flags[fidx(a, Ii, s)]) : 0;
      t[2 * q] = on ? s - s0 + 1 : 0;
      v[2 * q + 1] = on ? ld_relaxed(&a.flags[fidx(a, Ii, J)]) : 0;
      t[2 * q + 1] = on ? s - s0 : 0;
    }
    const bool own = J >= I && J < I + h;
    v[16] = own ? 0 : ld_relaxed(&a.flags[fidx(a, J, s)]);
    t[16] = own ? 0 : s - first_step(a, J) + 1;
    bool ready = true;
#pragma unroll
    for (int q = 0; q < 17; ++q) ready = ready && v[q] >= t[q];
    return ready;
  }
  if (type == kPotrf) return ld_relaxed(&a.flags[fidx(a, s, s)]) >= s - first_step(a, s);
  if (type == kTrsm) {
    const int v0 = ld_relaxed(&a.flags[fidx(a, s, s)]), v1 = ld_relaxed(&a.flags[fidx(a, I, s)]);
    return v0 >= s - first_step(a, s) + 1 && v1 >= s - first_step(a, I);
  }
  const int v0 = ld_relaxed(&a.flags[fidx(a, I, s)]), v1 = ld_relaxed(&a.flags[fidx(a, J, s)]),
            v2 = ld_relaxed(&a.flags[fidx(a, I, J)]);
  return v0 >= s - first_step(a, I) + 1 && v1 >= s - first_step(a, J) + 1 && v2 >= s - first_step(a, I);
}

template <int B, bool TC>
__global__ void __launch_bounds__(kThreads, 2) factor_batched_kernel(BatchArgs g) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<B>& sm = *reinterpret_cast<Smem<B>*>(smem_raw);
  __shared__ int s_m, s_go, s_flag;
  __shared__ long long s_t;
  __shared__ unsigned long long s_mbar;
  __shared__ uint32_t s_tmem;
  split::Ctx cx{};
  if constexpr (TC) cx = split::ctx_begin<B>(&s_mbar, &s_tmem);
  const int tid = threadIdx.x, lane = tid & 31;
  int m0 = blockIdx.x % g.count;   // where this CTA's search starts
  uint64_t idle_since = 0;
  unsigned long long seen = 0;
  if (tid == 0) idle_since = globaltimer_ns();
  while (true) {
    if (tid < 32) {
      int go = 0, mm_won = -1;
      long long t_won = 0;
      const int rounds = (g.count + 31) / 32;
      for (int rd = 0; rd < rounds && !go; ++rd) {
        const int mm = (m0 + rd * 32 + lane) % g.count;
        bool ready = false;
        unsigned long long t = 0;
        if (rd * 32 + lane < g.count) {
          Control* c = g.ctl + mm;
          const int retired = ld_relaxed(&c->retired);   // the three words in one round trip
          t = ld_relaxed_u64(&c->ticket);
          const int aborted = ld_relaxed(&c->abort);
          if (retired == 0) {
            const FactorArgs a = matrix_args(g, mm);
            if (t >= a.total || aborted != 0) {
              if (atomicCAS(&c->retired, 0, 1) == 0) atomicAdd(g.retired, 1);
            } else {
              int type, s, I, J;
              decode_mat_task(a, (long long)t, type, s, I, J);
              ready = task_ready(a, type, s, I, J);
            }
          }
        }
        unsigned ballot = __ballot_sync(0xffffffffu, ready);
        while (ballot && !go) {
          const int f = __ffs(ballot) - 1;
          int won = 0;
          if (lane == f) won = (atomicCAS(&g.ctl[mm].ticket, t, t + 1) == t);
          won = __shfl_sync(0xffffffffu, won, f);
          if (won) {
            go = 1;
            mm_won = __shfl_sync(0xffffffffu, mm, f);
            t_won = (long long)__shfl_sync(0xffffffffu, (unsigned long long)t, f);
          }
          ballot &= ballot - 1;
        }
      }
      if (lane == 0) {
        if (go) {
          s_go = 1;
          s_m = mm_won;
          s_t = t_won;
          m0 = mm_won;   // prefer the same matrix next time: its next ticket is often ready
          atomicAdd(g.progress, 1ULL);
          idle_since = globaltimer_ns();
        } else if (ld_relaxed(g.retired) >= g.count) {
          s_go = -1;
        } else {
          s_go = 0;
          m0 = (m0 + 32) % g.count;
          // a stall only if no CTA has claimed a task for the whole wait limit
          const unsigned long long now_seen = ld_relaxed_u64(g.progress);
          const uint64_t now = globaltimer_ns();
          if (now_seen != seen) {
            seen = now_seen;
            idle_since = now;
          } else if (now - idle_since > g.wait_ns) {
            atomicExch(g.status, kStatusTimeout);
            s_go = -1;
          }
        }
      }
      m0 = __shfl_sync(0xffffffffu, m0, 0);
    }
    __syncthreads();
    const int go = s_go;
    if (go < 0) break;
    if (go == 0) {
      if (tid == 0) __nanosleep(200);
      __syncthreads();
      continue;
    }
    const FactorArgs a = matrix_args(g, s_m);
    int type, s, I, J;
    decode_mat_task(a, s_t, type, s, I, J);
    if constexpr (TC) {
      if (type == kStrip) {
        // a product that did not complete leaves this CTA's barrier phase unknown: stop
        if (!task_strip<B>(a, I, J, s, *reinterpret_cast<split::Smem<B>*>(smem_raw), cx, &s_flag)) break;
        __syncthreads();
        continue;
      }
    }
    if (type == kPotrf)
      task_potrf<B>(a, s, sm, &s_flag);
    else if (type == kTrsm)
      task_trsm<B>(a, I, s, sm, &s_flag);
    else
      task_upd<B>(a, I, J, s, sm, &s_flag);
    __syncthreads();
  }
  if constexpr (TC) split::ctx_end<B>(cx);
}

// ------------------------------------------------------------------ solve
// CTAs take roles from a queue, largest system first: role 0 of a system is
// its leader (the chain and the near far terms), roles 1..W its workers (the
// other far terms; batched_solve.cuh).  A system's roles are consecutive in
// the queue and every CTA of the launch is resident, so a leader never waits
// on a role that no CTA will take: the systems ahead of it in the queue have
// all their roles running and finish.
struct SolveArgs {
  const BatchMat* mats;
  const int* entries;   // (system << 4) | role
  int nent;
  unsigned* queue;
  int* ctl;             // kCtlInts per system
  double* part;
  int* status;
  uint64_t wait_ns;
};

__global__ void __launch_bounds__(bsolve::kThreads, 2) solve_batched_kernel(SolveArgs sa) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  bsolve::Smem& sm = *reinterpret_cast<bsolve::Smem*>(smem_raw);
  bsolve::WSmem& ws = *reinterpret_cast<bsolve::WSmem*>(smem_raw);
  __shared__ int s_e;
  const int tid = threadIdx.x;
  while (true) {
    if (tid == 0) {
      const unsigned q = atomicAdd(sa.queue, 1u);
      s_e = (q < (unsigned)sa.nent) ? sa.entries[q] : -1;
    }
    __syncthreads();
    const int e = s_e;
    __syncthreads();
    if (e < 0) break;
    const int mi = e >> 4, role = e & 15;
    const BatchMat& M = sa.mats[mi];
    const int nrhs = M.nrhs, n = M.n;
    if (nrhs <= 0 || n <= 0 || __ldcg(M.info) != 0) continue;
    bsolve::Sys sy;
    sy.ab = M.ab;
    sy.ldab = M.ldab;
    sy.n = n;
    sy.k = M.k;
    sy.S = (n + bsolve::kB - 1) / bsolve::kB;
    sy.P = min((M.k + bsolve::kB - 1) / bsolve::kB, sy.S - 1);
    bsolve::Group G;
    G.W = M.W;
    G.span = bsolve::worker_span(sy.P, G.W);
    G.ctl = sa.ctl + (size_t)mi * bsolve::kCtlInts;
    G.part = sa.part + M.part_off;
    G.status = sa.status;
    G.wait_ns = sa.wait_ns;
    double* const b = M.b;
    const long long ldb = M.ldb;
    for (int c0 = 0, pass = 0; c0 < nrhs; c0 += bsolve::kR, ++pass) {
      const int nr = min(bsolve::kR, nrhs - c0);
      double* bc = b + (long long)c0 * ldb;
      const long long base = 2LL * pass * sy.S;
      if (role == 0) {
        bsolve::sweep<true>(sm, sy, bc, ldb, nr, G, base);
        bsolve::sweep<false>(sm, sy, bc, ldb, nr, G, base + sy.S);
      } else if (!bsolve::worker_sweep_nr<true>(ws, sy, bc, ldb, nr, G, role, base) ||
                 !bsolve::worker_sweep_nr<false>(ws, sy, bc, ldb, nr, G, role, base + sy.S)) {
        break;
      }
    }
    __syncthreads();
  }
}

}  // namespace bchol

// ------------------------------------------------------------------ host side
using namespace bchol;

// Resident CTAs of the solve launch (its grid when it has that many roles).
static cudaError_t solve_capacity(int* cap) {
  const size_t smem = sizeof(bsolve::Smem);
  cudaError_t e = cudaFuncSetAttribute(solve_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(solve_batched_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_batched_kernel, bsolve::kThreads, smem);
  if (e != cudaSuccess) return e;
  *cap = std::max(1, per_sm) * num_sms();
  return cudaSuccess;
}

// Tickets of one system's strip order (decode_st_task).
static unsigned long long st_total(const FactorPlan& P) {
  const Schedule sc{P.S, P.p, P.Sreg, st_treg(P.p, P.H), P.H};
  unsigned long long total = 1 + (unsigned long long)sched_m(sc, 0);
  total += (unsigned long long)sc.Sreg * (unsigned long long)sc.Treg;
  for (int s = (int)sc.Sreg; s < sc.S; ++s) total += (unsigned long long)st_block_size(sc, s);
  return total;
}

static bool batch_query_args(int n, int k, int tile, int precision) {
  return n >= 1 && k >= 0 && (tile == 16 || tile == 32 || tile == 64) &&
         (precision == BCHOL_FP64 || precision == BCHOL_FP64_SPLIT);
}

extern "C" bchol_status_t bchol_batch_solve_group(int n, int k, int ctas, int* workers, int* span, int* slots) {
  if (n < 1 || k < 0 || !workers || !span || !slots) return BCHOL_ERR_ARG;
  const int S = (n + bsolve::kB - 1) / bsolve::kB;
  const int P = std::min((std::min(k, n - 1) + bsolve::kB - 1) / bsolve::kB, S - 1);
  *workers = bsolve::workers_for(P, ctas);
  *span = bsolve::worker_span(P, *workers);
  *slots = bsolve::kSlots;
  return BCHOL_OK;
}

extern "C" long long bchol_batch_plan_task_count(int n, int k, int tile, int precision) {
  if (!batch_query_args(n, k, tile, precision)) return -1;
  const FactorPlan P = make_factor_plan(n, std::min(k, n - 1), tile, precision == BCHOL_FP64_SPLIT);
  return (long long)(P.H > 1 ? st_total(P) : P.total);
}

extern "C" bchol_status_t bchol_batch_plan_task(int n, int k, int tile, int precision, long long ticket, int* type,
                                                int* s, int* I, int* J) {
  if (!batch_query_args(n, k, tile, precision) || !type || !s || !I || !J) return BCHOL_ERR_ARG;
  const FactorPlan P = make_factor_plan(n, std::min(k, n - 1), tile, precision == BCHOL_FP64_SPLIT);
  const unsigned long long total = P.H > 1 ? st_total(P) : P.total;
  if (ticket < 0 || (unsigned long long)ticket >= total) return BCHOL_ERR_ARG;
  const Schedule sc{P.S, P.p, P.Sreg, P.H > 1 ? st_treg(P.p, P.H) : P.Treg, P.H};
  if (P.H > 1)
    decode_st_task(sc, ticket, *type, *s, *I, *J);
  else
    decode_task(sc, ticket, *type, *s, *I, *J);
  return BCHOL_OK;
}

struct bchol_batch_s {
  int count = 0;
  int b = 32;
  int ctas_per_sm = 1;
  int precision = BCHOL_FP64;   // BCHOL_FP64_SPLIT: updates as split products (tiles of 16 and 32)
  std::vector<int> member_precision;   // per-system modes for the next plan (empty: `precision` for all)
  bool split = false;           // some system of the planned batch runs the split updates
  bool any_rhs = false;
  int* info_dev = nullptr;
  size_t bytes = 0;
  void* dev = nullptr;          // descriptors | solve roles | control | flags | counters | solve control | partial sums
  size_t ctl_off = 0, flags_off = 0, cnt_off = 0, order_off = 0, sctl_off = 0, part_off = 0, clear_bytes = 0;
  int nent = 0;                 // solve roles
};

extern "C" bchol_status_t bchol_batch_create(bchol_batch_t* batch) {
  if (!batch) return BCHOL_ERR_ARG;
  *batch = new (std::nothrow) bchol_batch_s();
  return *batch ? BCHOL_OK : BCHOL_ERR_ALLOC;
}

extern "C" bchol_status_t bchol_batch_destroy(bchol_batch_t batch) {
  if (!batch) return BCHOL_ERR_ARG;
  if (batch->dev) cudaFree(batch->dev);
  delete batch;
  return BCHOL_OK;
}

extern "C" bchol_status_t bchol_batch_set_precision(bchol_batch_t batch, int precision) {
  if (!batch) return BCHOL_ERR_ARG;
  if (precision == BCHOL_FP32_UPDATE || precision == BCHOL_TF32_UPDATE) return BCHOL_ERR_UNSUPPORTED;
  if (precision != BCHOL_FP64 && precision != BCHOL_FP64_SPLIT) return BCHOL_ERR_ARG;
  batch->precision = precision;
  return BCHOL_OK;
}

extern "C" bchol_status_t bchol_batch_set_member_precision(bchol_batch_t batch, int count, const int* precision) {
  if (!batch || count < 0 || (count > 0 && !precision)) return BCHOL_ERR_ARG;
  for (int m = 0; m < count; ++m) {
    if (precision[m] == BCHOL_FP32_UPDATE || precision[m] == BCHOL_TF32_UPDATE) return BCHOL_ERR_UNSUPPORTED;
    if (precision[m] != BCHOL_FP64 && precision[m] != BCHOL_FP64_SPLIT) return BCHOL_ERR_ARG;
  }
  batch->member_precision.assign(precision, precision + count);
  return BCHOL_OK;
}

extern "C" bchol_status_t bchol_batch_plan(bchol_batch_t batch, int count, const int* n, const int* k, double* const* ab,
                                           const int* ldab, int* info_dev, const int* nrhs, double* const* b,
                                           const int* ldb, int tile, int ctas_per_sm) {
  if (!batch || count <= 0 || !n || !k || !ab || !ldab || !info_dev) return BCHOL_ERR_ARG;
  if (!(tile == 0 || tile == 16 || tile == 32 || tile == 64) || ctas_per_sm < 0 || ctas_per_sm > 8) return BCHOL_ERR_ARG;
  for (int m = 0; m < count; ++m) {
    if (n[m] < 1 || k[m] < 0 || ldab[m] < k[m] + 1 || !ab[m]) return BCHOL_ERR_ARG;
    const int r = nrhs ? nrhs[m] : 0;
    if (r < 0 || (r > 0 && (!b || !b[m] || !ldb || ldb[m] < n[m]))) return BCHOL_ERR_ARG;
  }
  // automatic tile: 32 (tiles of 16 quadruple the tasks, and per-task latency bounds this launch)
  const int bt = tile ? tile : 32;
  if (!batch->member_precision.empty() && (int)batch->member_precision.size() != count) return BCHOL_ERR_ARG;
  auto split_of = [&](int m) {
    const int pm = batch->member_precision.empty() ? batch->precision : batch->member_precision[m];
    return pm == BCHOL_FP64_SPLIT && (bt == 16 || bt == 32);
  };
  bool split = false;
  std::vector<BatchMat> mats(count);
  std::vector<double> work(count);
  size_t flag_total = 0;
  bool any_rhs = false;
  for (int m = 0; m < count; ++m) {
    const int kk = std::min(k[m], n[m] - 1);
    const FactorPlan P = make_factor_plan(n[m], kk, bt, split_of(m));
    split = split || P.H > 1;
    BatchMat& M = mats[m];
    M.ab = ab[m];
    M.ldab = ldab[m];
    M.n = n[m];
    M.k = kk;
    M.S = P.S;
    M.p = P.p;
    M.Sreg = P.Sreg;
    M.Treg = P.Treg;
    M.total = P.total;
    M.H = P.H;
    if (P.H > 1) {  // the ticket-only order with strips (decode_st_task)
      M.Treg = st_treg(P.p, P.H);
      M.total = st_total(P);
    }
    M.flag_off = (long long)flag_total;
    M.info = info_dev + m;
    M.nrhs = nrhs ? nrhs[m] : 0;
    M.b = M.nrhs ? b[m] : nullptr;
    M.ldb = M.nrhs ? ldb[m] : 1;
    flag_total += P.flag_count;
    any_rhs = any_rhs || M.nrhs > 0;
    work[m] = (double)n[m] * (kk + 1.0) * (kk + 4.0);
  }
  // largest matrices first: both kernels take them in this order
  std::vector<int> order(count);
  for (int m = 0; m < count; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  std::vector<BatchMat> sorted(count);
  for (int q = 0; q < count; ++q) sorted[q] = mats[order[q]];
  // solve roles: each system with right-hand sides, its leader then its
  // workers; no group larger than the CTAs the solve launch keeps resident
  int cap = 0;
  if (any_rhs && solve_capacity(&cap) != cudaSuccess) return BCHOL_ERR_CUDA;
  std::vector<int> roles;
  long long part_total = 0;
  for (int q = 0; q < count; ++q) {
    BatchMat& M = sorted[q];
    M.part_off = part_total;
    M.W = 0;
    M.pad2 = 0;
    if (M.nrhs <= 0) continue;
    const int S = (M.n + bsolve::kB - 1) / bsolve::kB;
    const int P = std::min((M.k + bsolve::kB - 1) / bsolve::kB, S - 1);
    const int W = bsolve::workers_for(P, cap);
    M.W = W;
    for (int r = 0; r <= W; ++r) roles.push_back((q << 4) | r);
    part_total += (long long)W * bsolve::kSlots * bsolve::kR * bsolve::kB;
  }
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t desc_b = up(sizeof(BatchMat) * count);
  const size_t order_b = up(sizeof(int) * std::max<size_t>(roles.size(), 1));
  const size_t ctl_b = up(sizeof(Control) * count);
  const size_t flags_b = up(sizeof(int) * flag_total);
  const size_t cnt_b = 256;
  const size_t sctl_b = up(sizeof(int) * bsolve::kCtlInts * count);
  const size_t part_b = up(sizeof(double) * (size_t)part_total);
  const size_t need = desc_b + order_b + ctl_b + flags_b + cnt_b + sctl_b + part_b;
  if (batch->bytes < need) {
    if (batch->dev) {
      cudaDeviceSynchronize();
      cudaFree(batch->dev);
      batch->dev = nullptr;
      batch->bytes = 0;
    }
    if (cudaMalloc(&batch->dev, need) != cudaSuccess) {
      cudaGetLastError();
      return BCHOL_ERR_ALLOC;
    }
    batch->bytes = need;
  }
  char* base = static_cast<char*>(batch->dev);
  batch->order_off = desc_b;
  batch->ctl_off = desc_b + order_b;
  batch->flags_off = batch->ctl_off + ctl_b;
  batch->cnt_off = batch->flags_off + flags_b;
  batch->sctl_off = batch->cnt_off + cnt_b;
  batch->part_off = batch->sctl_off + sctl_b;
  batch->clear_bytes = ctl_b + flags_b + cnt_b + sctl_b;   // control, flags, counters, solve control: contiguous
  batch->nent = (int)roles.size();
  if (cudaMemcpy(base, sorted.data(), sizeof(BatchMat) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
      (!roles.empty() &&
       cudaMemcpy(base + batch->order_off, roles.data(), sizeof(int) * roles.size(), cudaMemcpyHostToDevice) !=
           cudaSuccess))
    return BCHOL_ERR_CUDA;
  batch->count = count;
  batch->b = bt;
  batch->split = split;
  batch->ctas_per_sm = ctas_per_sm ? ctas_per_sm : 2;   // automatic: two (more hide more of the per-task latency)
  batch->any_rhs = any_rhs;
  batch->info_dev = info_dev;
  return BCHOL_OK;
}

template <int B, bool TC = false>
static cudaError_t launch_batched_factor(const BatchArgs& g, int ctas_per_sm, cudaStream_t st) {
  auto kern = factor_batched_kernel<B, TC>;
  size_t smem = sizeof(Smem<B>);
  if constexpr (TC) smem = std::max(smem, sizeof(split::Smem<B>));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if constexpr (TC) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    e = tc_ctas_per_sm(reinterpret_cast<const void*>(kern), smem, split::tmem_cols<B>(), kThreads, &per_sm);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  }
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  kern<<<per_sm * num_sms(), kThreads, smem, st>>>(g);
  return cudaGetLastError();
}

// Launches for a planned batch (capturable in a CUDA graph): clear the
// control words, factor every matrix, then solve those with right-hand sides.
namespace bchol {
int batch_run(bchol_batch_s* batch, int* status, uint64_t wait_ns, cudaStream_t st, int* launches) {
  *launches = 0;
  if (!batch || batch->count <= 0 || !batch->dev) return BCHOL_ERR_ARG;
  char* base = static_cast<char*>(batch->dev);
  if (cudaMemsetAsync(base + batch->ctl_off, 0, batch->clear_bytes, st) != cudaSuccess ||
      cudaMemsetAsync(batch->info_dev, 0, sizeof(int) * batch->count, st) != cudaSuccess)
    return BCHOL_ERR_CUDA;
  BatchArgs g;
  g.mats = reinterpret_cast<const BatchMat*>(base);
  g.ctl = reinterpret_cast<Control*>(base + batch->ctl_off);
  g.flags = reinterpret_cast<int*>(base + batch->flags_off);
  g.count = batch->count;
  g.retired = reinterpret_cast<int*>(base + batch->cnt_off);
  g.progress = reinterpret_cast<unsigned long long*>(base + batch->cnt_off + 128);
  g.status = status;
  g.wait_ns = wait_ns;
  cudaError_t e;
  if (batch->split)
    e = batch->b == 16 ? launch_batched_factor<16, true>(g, batch->ctas_per_sm, st)
                       : launch_batched_factor<32, true>(g, batch->ctas_per_sm, st);
  else switch (batch->b) {
    case 16: e = launch_batched_factor<16>(g, batch->ctas_per_sm, st); break;
    case 32: e = launch_batched_factor<32>(g, batch->ctas_per_sm, st); break;
    default: e = launch_batched_factor<64>(g, batch->ctas_per_sm, st); break;
  }
  if (e != cudaSuccess) return BCHOL_ERR_CUDA;
  *launches = 1;
  if (batch->any_rhs && batch->nent > 0) {
    SolveArgs sa;
    sa.mats = g.mats;
    sa.entries = reinterpret_cast<const int*>(base + batch->order_off);
    sa.nent = batch->nent;
    sa.queue = reinterpret_cast<unsigned*>(base + batch->cnt_off + 64);
    sa.ctl = reinterpret_cast<int*>(base + batch->sctl_off);
    sa.part = reinterpret_cast<double*>(base + batch->part_off);
    sa.status = status;
    sa.wait_ns = wait_ns;
    const size_t smem = sizeof(bsolve::Smem);
    int cap = 0;
    if (solve_capacity(&cap) != cudaSuccess) return BCHOL_ERR_CUDA;
    // every CTA resident at once, and no group larger than the grid (the plan's cap)
    const int grid = std::min(batch->nent, cap);
    solve_batched_kernel<<<grid, bsolve::kThreads, smem, st>>>(sa);
    if (cudaGetLastError() != cudaSuccess) return BCHOL_ERR_CUDA;
    *launches = 2;
  }
  return BCHOL_OK;
}
}  // namespace bchol
