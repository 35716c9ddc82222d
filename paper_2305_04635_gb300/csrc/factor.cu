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
//
// With tiles of 16 or 32 the first CTA of the launch runs the diagonal chain
// instead (diag_chain.cuh): every task of the diagonal and the first
// sub-diagonal, fused per step, and the other CTAs take the rest by ticket in
// the order of decode_cp_ticket.  When the band holds two or more tiles below
// the diagonal, CTAs 1 and 2 are helpers that run the three tasks of each step
// at distance two from the diagonal in a fixed order (the tasks the chain's
// next inputs hang on, so that they never queue behind other tickets; two
// CTAs, because one SM's FP64 rate does not fit the three into a chain step),
// and the tickets follow decode_hp_ticket.  All CTAs of the launch are resident at
// once (the grid is sized from the occupancy), and every task the chain or a
// helper waits for precedes, in the combined order, every task that waits for
// it, so this walk cannot deadlock either.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "diag_chain.cuh"
#include "strip_task.cuh"

namespace bchol {

template <int B, bool F32>
__device__ __forceinline__ bool run_task(const FactorArgs& a, int type, int s, int I, int J, Smem<B>& sm, int* s_flag) {
  if (type == kPotrf) return task_potrf<B>(a, s, sm, s_flag);
  if (type == kTrsm && F32) return task_trsm_f32<B>(a, I, s, sm, s_flag);
  if (type == kTrsm) return task_trsm<B>(a, I, s, sm, s_flag);
  if (F32) return task_upd_f32<B>(a, I, J, s, sm, s_flag);
  return task_upd<B>(a, I, J, s, sm, s_flag);
}

// Helper CTA `role` (1 or 2) of the chain mode with helpers: the tasks at
// distance two from the diagonal, in step order (schedule.cuh).  Helper 2
// solves L(t, t-2) and applies it to A(t, t-1) once the chain's L(t-1, t-2) is
// in (A(t, t-1) is the chain's later input), using the solved tile straight
// from its shared memory; helper 1 applies L(t, t-2) to A(t, t).
template <int B, bool F32>
__device__ void factor_helper(const FactorArgs& a, Smem<B>& sm, int* s_flag, int role) {
  for (int t = 2; t < a.S; ++t) {
    bool ok;
    if (role == 1) {
      ok = run_task<B, F32>(a, kUpd, t - 2, t, t, sm, s_flag);
    } else if constexpr (F32) {
      ok = run_task<B, F32>(a, kTrsm, t - 2, t, t - 2, sm, s_flag) &&
           run_task<B, F32>(a, kUpd, t - 2, t, t - 1, sm, s_flag);
    } else {
      ok = task_trsm<B>(a, t, t - 2, sm, s_flag) && task_upd<B>(a, t, t - 1, t - 2, sm, s_flag, true);
    }
    if (!ok) return;
  }
}

// MODE 0: tickets only; 1: the diagonal chain (CTA 0) and tickets; 2: the chain,
// two helpers (CTAs 1 and 2) and tickets.  TC: the update tickets are strips,
// split products on the tensor cores (strip_task.cuh); each ticket CTA holds
// 256 (tiles of 32) or 128 (tiles of 16) columns of tensor memory for its
// lifetime.
template <int B, bool F32, int MODE, bool TC>
__global__ void __launch_bounds__(kThreads, 2) factor_kernel(FactorArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long s_task;
  __shared__ int s_flag;
  __shared__ unsigned long long s_mbar;
  __shared__ uint32_t s_tmem;
  if constexpr (MODE >= 1) {
    if (blockIdx.x == 0) {
      if (threadIdx.x == 0) st_release(&a.ctl->chain_sm, sm_id() + 1);
      diag_chain<B, F32>(a, *reinterpret_cast<DiagSmem<B, F32>*>(smem_raw), &tmap);
      return;
    }
    if constexpr (MODE == 2) {
      if (blockIdx.x <= 2) {
        if (threadIdx.x == 0) st_release(&a.ctl->helper_sm[blockIdx.x - 1], sm_id() + 1);
        factor_helper<B, F32>(a, *reinterpret_cast<Smem<B>*>(smem_raw), &s_flag, (int)blockIdx.x);
        return;
      }
    }
    // A ticket CTA on the SM of the chain CTA (or of a helper) leaves: their
    // FP64 work is the critical path and each SM sub-partition's FP64 unit is
    // shared.  (All CTAs are resident at once, so those CTAs publish their SMs
    // promptly; the wait is bounded and a CTA that gives up simply stays.)
    if (threadIdx.x == 0) {
      const int me = sm_id() + 1;
      const uint64_t t0 = globaltimer_ns();
      int c = ld_acquire(&a.ctl->chain_sm);
      while (c == 0 && globaltimer_ns() - t0 < 200000ull) c = ld_acquire(&a.ctl->chain_sm);
      bool leave = (c == me);
      if constexpr (MODE == 2) {
        for (int h = 0; h < 2 && !leave; ++h) {
          int hs = ld_acquire(&a.ctl->helper_sm[h]);
          while (hs == 0 && globaltimer_ns() - t0 < 200000ull) hs = ld_acquire(&a.ctl->helper_sm[h]);
          leave = (hs == me);
        }
      }
      s_flag = leave;
    }
    __syncthreads();
    if (s_flag) return;
  }
  Smem<B>& sm = *reinterpret_cast<Smem<B>*>(smem_raw);
  split::Ctx cx{};
  if constexpr (TC) cx = split::ctx_begin<B>(&s_mbar, &s_tmem);
  unsigned long long next = 0;
  if (threadIdx.x == 0) next = atomicAdd(&a.ctl->ticket, 1ULL);
  while (true) {
    if (threadIdx.x == 0) s_task = (long long)next;
    __syncthreads();
    const long long t = s_task;
    if (t >= (long long)a.total) break;
    if (threadIdx.x == 0) next = atomicAdd(&a.ctl->ticket, 1ULL);  // claim the next task early
    int type, s, I, J;
    if constexpr (MODE == 2)
      decode_hp_ticket(Schedule{a.S, a.p, a.Sreg, a.Treg, a.H}, t, type, s, I, J);
    else if constexpr (MODE == 1)
      decode_cp_ticket(Schedule{a.S, a.p, a.Sreg, a.Treg, a.H}, t, type, s, I, J);
    else
      decode_task(Schedule{a.S, a.p, a.Sreg, a.Treg}, t, type, s, I, J);
    if constexpr (TC) {
      if (type == kStrip) {
        if (!task_strip<B>(a, I, J, s, *reinterpret_cast<split::Smem<B>*>(smem_raw), cx, &s_flag)) break;
        continue;
      }
    }
    if (!run_task<B, F32>(a, type, s, I, J, sm, &s_flag)) break;
  }
  if constexpr (TC) split::ctx_end<B>(cx);
}

__global__ void pivot_rcp_kernel(const double* x, double* y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = pivot_rcp(x[i]);
}

cudaError_t launch_pivot_rcp(const double* x, double* y, int n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  pivot_rcp_kernel<<<(n + 255) / 256, 256, 0, stream>>>(x, y, n);
  return cudaGetLastError();
}

FactorPlan make_factor_plan(int n, int k, int b, bool split) {
  FactorPlan P;
  P.H = (split && (b == 16 || b == 32)) ? split::kRowsA / b : 1;
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
  P.Treg_cp = cp_treg(P.p, P.H);
  const Schedule cs{P.S, P.p, P.Sreg, P.Treg_cp, P.H};
  unsigned long long tickets = (unsigned long long)cp_panel0(cs);
  tickets += (unsigned long long)P.Sreg * (unsigned long long)P.Treg_cp;
  for (int s = (int)P.Sreg; s < P.S; ++s) tickets += (unsigned long long)cp_block_size(cs, s);
  P.total_cp = tickets;
  // Helpers pay off while the chain bounds the launch; with many tiles per
  // panel (k = 2000 at b = 32) and FP64 updates the two CTAs are worth more
  // as ticket CTAs.
  // With the split updates the trailing update is cheap at every k, so the
  // chain's inputs always get the helpers.
  P.helper = (b <= 32 && P.p >= 2 && (P.p <= 40 || P.H > 1));
  P.Treg_hp = hp_treg(P.p, P.H);
  const Schedule hs{P.S, P.p, P.Sreg, P.Treg_hp, P.H};
  tickets = (unsigned long long)hp_panel0(hs);
  tickets += (unsigned long long)P.Sreg * (unsigned long long)P.Treg_hp;
  for (int s = (int)P.Sreg; s < P.S; ++s) tickets += (unsigned long long)hp_block_size(hs, s);
  P.total_hp = tickets;
  return P;
}

size_t factor_workspace_bytes(const FactorPlan& P) { return 256 + P.flag_count * sizeof(int); }

// CTAs per SM of a kernel that allocates tensor memory.  The occupancy query
// answers 1 for any such kernel, whatever it allocates; the SM runs as many
// CTAs as its registers, shared memory and threads allow, and tcgen05.alloc
// waits for columns, so the count comes from those resources and from the
// SM's 512 tensor-memory columns.
cudaError_t tc_ctas_per_sm(const void* func, size_t dyn_smem, int tmem_cols, int threads, int* per_sm) {
  cudaFuncAttributes fa;
  int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e != cudaSuccess) return e;
  const int regs_cta = (fa.numRegs + 7) / 8 * 8 * threads;
  const int smem_cta = (int)(dyn_smem + fa.sharedSizeBytes) + reserved;
  int fit = std::min(regs_sm / std::max(regs_cta, 1), smem_sm / std::max(smem_cta, 1));
  fit = std::min({fit, 2048 / threads, 512 / std::max(tmem_cols, 1)});
  *per_sm = std::max(1, fit);
  return cudaSuccess;
}

template <int B, bool F32, int MODE, bool TC = false>
static cudaError_t launch_b(const FactorArgs& a, const CUtensorMap& tmap, int ctas_per_sm, cudaStream_t stream) {
  size_t smem = sizeof(Smem<B>);
  if constexpr (MODE >= 1) smem = std::max(smem, sizeof(DiagSmem<B, F32>));
  if constexpr (TC) smem = std::max(smem, sizeof(split::Smem<B>));
  cudaError_t e =
      cudaFuncSetAttribute(factor_kernel<B, F32, MODE, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // The split products' 72 KB per CTA fit two CTAs per SM only with the
  // largest shared-memory carveout; ask for it, or the occupancy (and the
  // grid) is computed for a smaller one.
  if constexpr (TC) {
    e = cudaFuncSetAttribute(factor_kernel<B, F32, MODE, TC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, factor_kernel<B, F32, MODE, TC>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  // The split kernels size their grid from the SM's resources (tc_ctas_per_sm):
  // each ticket CTA holds 256 (tiles of 32) or 128 (tiles of 16) of the SM's
  // 512 tensor-memory columns.
  if constexpr (TC) {
    int fit = 0;
    e = tc_ctas_per_sm(reinterpret_cast<const void*>(factor_kernel<B, F32, MODE, TC>), smem, split::tmem_cols<B>(),
                       kThreads, &fit);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, ctas_per_sm > 0 ? std::min(fit, ctas_per_sm) : fit);
  }
  long long grid = (long long)per_sm * num_sms();
  const unsigned long long need = a.total + (MODE == 2 ? 3 : MODE == 1 ? 1 : 0);  // tickets + chain (+ helpers)
  if ((unsigned long long)grid > need) grid = (long long)need;
  if (grid < 1) grid = 1;
  factor_kernel<B, F32, MODE, TC><<<(unsigned)grid, kThreads, smem, stream>>>(a, tmap);
  return cudaGetLastError();
}

// The band as the 2-D tensor of the chain's TMA copies (diag_chain.cuh): element
// (gi, gj) at ab + gi + gj (ldab - 1), dims (n, n), boxes of b x b.  False when
// the tensor-map rules exclude it (stride (ldab - 1) * 8 not a multiple of 16,
// a base not 16-byte aligned) or the driver declines the encoding.
static bool encode_band_map(CUtensorMap* m, const double* ab, int n, long long ldab, int b) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<Encode>(f);
    else
      cudaGetLastError();
  }
  if (!fn || ldab < 2 || ((ldab - 1) * 8) % 16 != 0 || (reinterpret_cast<uintptr_t>(ab) & 15) != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)(ldab - 1) * 8};
  const cuuint32_t box[2] = {(cuuint32_t)b, (cuuint32_t)b};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(ab), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_factor(const FactorPlan& P, double* ab, long long ldab, int* info, void* ws, int* status,
                          uint64_t wait_ns, int ctas_per_sm, int stall_I, int stall_J, cudaStream_t stream,
                          int tma, int* tma_used) {
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
  a.H = P.H;
  if (stall_I >= 0 && stall_J >= 0 && stall_I < P.S && stall_J <= stall_I && stall_I - stall_J <= P.p)
    a.stall = stall_J * (P.p + 1) + (stall_I - stall_J);
  if (P.b <= 32) {  // diagonal chain (+ helpers) + tickets
    a.Treg = P.helper ? P.Treg_hp : P.Treg_cp;
    a.total = P.helper ? P.total_hp : P.total_cp;
  }
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  a.tma = (tma && P.b <= 32 && encode_band_map(&tmap, ab, P.n, ldab, P.b)) ? 1 : 0;
  if (tma_used) *tma_used = a.tma;
  const bool h = P.helper;
  if (P.f32_update) {
    switch (P.b) {
      case 16: return h ? launch_b<16, true, 2>(a, tmap, ctas_per_sm, stream) : launch_b<16, true, 1>(a, tmap, ctas_per_sm, stream);
      case 32: return h ? launch_b<32, true, 2>(a, tmap, ctas_per_sm, stream) : launch_b<32, true, 1>(a, tmap, ctas_per_sm, stream);
      case 64: return launch_b<64, true, 0>(a, tmap, ctas_per_sm, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  if (P.b == 32 && P.H > 1)
    return h ? launch_b<32, false, 2, true>(a, tmap, ctas_per_sm, stream) : launch_b<32, false, 1, true>(a, tmap, ctas_per_sm, stream);
  if (P.b == 16 && P.H > 1)
    return h ? launch_b<16, false, 2, true>(a, tmap, ctas_per_sm, stream) : launch_b<16, false, 1, true>(a, tmap, ctas_per_sm, stream);
  switch (P.b) {
    case 16: return h ? launch_b<16, false, 2>(a, tmap, ctas_per_sm, stream) : launch_b<16, false, 1>(a, tmap, ctas_per_sm, stream);
    case 32: return h ? launch_b<32, false, 2>(a, tmap, ctas_per_sm, stream) : launch_b<32, false, 1>(a, tmap, ctas_per_sm, stream);
    case 64: return launch_b<64, false, 0>(a, tmap, ctas_per_sm, stream);
    default: return cudaErrorInvalidValue;
  }
}

// Tasks in the combined order: all tasks of the tiled factorization with one
// update per tile, fewer when the updates run as strips.
long long plan_task_count(const FactorPlan& P) {
  if (P.b > 32 || P.H == 1 || P.n <= 0) return (long long)P.total;
  const long long nd = P.p >= 1 ? 3 : 1;
  long long c = 1 + (long long)(P.S - 1) * nd;
  if (P.helper && P.S > 2) c += 3LL * (P.S - 2);
  return c + (long long)(P.helper ? P.total_hp : P.total_cp);
}

// The combined task order of one factorization (host side): for tiles of 16
// and 32, the diagonal chain's (and the helpers') tasks at their places among
// the tickets; for 64, the ticket order itself.
void plan_task(const FactorPlan& P, long long t, int& type, int& s, int& I, int& J) {
  if (P.b > 32) {
    decode_task(Schedule{P.S, P.p, P.Sreg, P.Treg}, t, type, s, I, J);
    return;
  }
  const Schedule cs{P.S, P.p, P.Sreg, P.helper ? P.Treg_hp : P.Treg_cp, P.H};
  auto ticket = [&](long long u) {
    if (P.helper)
      decode_hp_ticket(cs, u, type, s, I, J);
    else
      decode_cp_ticket(cs, u, type, s, I, J);
  };
  const long long nd = P.p >= 1 ? 3 : 1;
  auto diag = [&](int st, long long r) {
    if (st == 0 || P.p == 0 || r == 2) {
      type = kPotrf;
      s = I = J = st;
    } else if (r == 0) {
      type = kTrsm;
      s = J = st - 1;
      I = st;
    } else {
      type = kUpd;
      s = st - 1;
      I = J = st;
    }
  };
  if (t == 0) {
    diag(0, 0);
    return;
  }
  t -= 1;
  long long base = P.helper ? hp_panel0(cs) : cp_panel0(cs);
  if (t < base) {
    ticket(t);
    return;
  }
  t -= base;
  for (int st = 0; st + 1 < P.S; ++st) {
    if (t < nd) {
      diag(st + 1, t);
      return;
    }
    t -= nd;
    if (P.helper && st + 2 < P.S) {  // H(st+2): TRSM(st+2, st), UPD(st+2, st+2, st), UPD(st+2, st+1, st)
      if (t < 3) {
        s = st;
        I = st + 2;
        type = t == 0 ? kTrsm : kUpd;
        J = t == 0 ? st : t == 1 ? st + 2 : st + 1;
        return;
      }
      t -= 3;
    }
    const long long bs = P.helper ? hp_block_size(cs, st) : cp_block_size(cs, st);
    if (t < bs) {
      ticket(base + t);
      return;
    }
    t -= bs;
    base += bs;
  }
  type = -1;
  s = I = J = -1;
}

}  // namespace bchol
