// batched_solve.cuh -- the solve launch of the batched path: X = A^{-1} B for
// every system of a batch, from its band Cholesky factor (forward substitution
// L Y = B, then back substitution L^T X = Y; LAPACK pbtrs semantics).  The
// paper factors only; the solve is the use it motivates (Sec. 1, Sec. 2).
//
// One CTA per system, largest first; right-hand sides in passes of four.
// Rows go in blocks of 32.  With P = ceil(k/32), the block of step I is
//     fwd:  y_I = L_II^{-1} (b_I - L_{I,I-1} y_{I-1} - sum_{J=I-P}^{I-2} L_IJ y_J)
//     bwd:  x_I = L_II^{-T} (y_I - L_{I+1,I}^T x_{I+1} - sum_{J=I+2}^{I+P} L_JI^T x_J)
// On GB300 an SM sub-partition issues one FP64 warp instruction per 64 cycles
// whatever the number of active lanes, so the layout is chosen by instruction
// count and by which sub-partition issues it:
//   - warps 0-3 (one per sub-partition) run the chain.  Lane (i, r) holds row
//     8w + i of the block for right-hand side r, so one instruction serves
//     8 rows x 4 right-hand sides.  The 32 x 32 triangle is solved as four
//     8 x 8 triangles in sweep order; warp c solves its triangle with one
//     shuffle and one FMA per column (the column entries come pre-scaled by
//     the pivot's reciprocal, so no multiply sits on the chain), publishes its
//     eight values in shared memory, and the warps still to come subtract
//     their products with them.  The same published values feed the near
//     term of the next block (L_{I+1,I} y_I, or L_{I,I-1}^T x_I), accumulated
//     in registers while the rest of the triangle is solved.
//   - warps 4-7 work one block ahead: the far terms of the next block (lane =
//     row, 32 rows per instruction, columns split over the four warps),
//     b minus those terms into shared memory, and the next block's diagonal
//     and near tiles staged into shared memory with the reciprocals of the
//     pivots (refined hardware reciprocal) and the pre-scaled triangles.
//     Their global reads are asynchronous copies streamed through a ring in
//     shared memory (far_step).
// One CTA barrier closes each step; the chain warps also meet at a named
// barrier after each 8 x 8 triangle.
#pragma once
#include "diag_chain.cuh"

namespace bchol {
namespace bsolve {

constexpr int kB = 32;        // rows per block
constexpr int kR = 4;         // right-hand sides per pass
constexpr int kThreads = 256;
constexpr int kTP = kB + 1;   // pitch of a staged tile row (doubles)
constexpr int kXP = kB + 1;   // pitch of the published block (doubles)
constexpr int kBarChain = 1;  // warps 0-3
constexpr int kBarFar = 2;    // warps 4-7
constexpr int kDepth = 4;     // far blocks in the asynchronous-copy ring (a power of two)
// Worker CTAs (systems with P >= kMinPW): worker w = 1..W owns the far
// distances 3 + (w-1) span .. + span - 1 of every target block.  The plan caps
// W below the launch's resident CTAs, so that every group can be staffed.
constexpr int kMinPW = 5;
constexpr int kMaxW = 15;
constexpr int kWD = 2;        // far distances per worker when the count allows
constexpr int kSlots = 8;     // ring slots of a worker's partial sums (global memory)
constexpr int kMaxD = 4;      // far blocks per worker pass over shared memory
constexpr int kCtlInts = 64;  // per system: [0] blocks solved by the leader, [1] abort, [32 + w] targets done by worker w

__host__ __device__ inline int worker_span(int P, int W) { return W > 0 ? (P - 2 + W - 1) / W : 0; }
// Workers of a system with P far blocks on a launch of `cap` resident CTAs
// (cap <= 0: no limit): kWD distances each, at most kMaxW and cap - 1, then
// as few as cover the distances 3..P at the resulting span (none idle).
__host__ __device__ inline int workers_for(int P, int cap = 0) {
  if (P < kMinPW) return 0;
  int w = (P - 2 + kWD - 1) / kWD;
  if (w > kMaxW) w = kMaxW;
  if (cap > 0 && w > cap - 1) w = cap - 1;
  if (w <= 0) return 0;
  const int span = worker_span(P, w);
  return (P - 2 + span - 1) / span;
}

struct Smem {
  double T[2][2][kB][kTP];   // [slot][0: diagonal tile, 1: near tile][row][col]
  double rinv[2][kB];        // reciprocals of the diagonal tile's pivots
  double U[2][kR][kB];       // b of the block minus its far terms
  double red[4][kR][kB];     // far-warp partial sums
  double xs[kR][kXP];        // the block being solved, as its triangles complete
  double bpre[kR][kB];       // b of the far warps' block
  double ring[kDepth][128][kB / 4];   // per far thread: its 8 band entries of each block in flight
  double ys[kDepth][kB][kR];         // the solved values of each block in flight (column, rhs)
};

struct Sys {
  const double* ab;
  long long ldab;
  int n, k, S, P;
};

// A system's leader / worker group: control words, the workers' partial sums
// (part[((w-1) kSlots + slot) kR kB + r kB + row]), the launch status word.
struct Group {
  int W, span;
  int* ctl;
  double* part;
  int* status;
  uint64_t wait_ns;
};

// Shared memory of a worker CTA (aliases Smem).
struct WSmem {
  double ys[kMaxD][kB][kR];   // solved values of the blocks of one pass (column, rhs)
  double red[8][kR][kB];      // per-warp partial sums
};

// One thread: wait until *flag >= target.  False when the group is aborted or
// the wait runs out (then the launch status records a timeout and the abort
// word stops the group's other waits).
__device__ __forceinline__ bool gwait(const Group& G, const int* flag, int target) {
  if (ld_acquire(flag) >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (ld_acquire(flag) >= target) return true;
    if (ld_relaxed(&G.ctl[1]) != 0) return false;
    if (globaltimer_ns() - t0 > G.wait_ns) {
      atomicExch(G.status, kStatusTimeout);
      atomicExch(&G.ctl[1], 1);
      return false;
    }
  }
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Address of L(gi, gj), or null outside the band or the matrix.  The factor
// is read-only here (written by an earlier launch).
__device__ __forceinline__ const double* laddr(const Sys& m, int gi, int gj) {
  const int d = gi - gj;
  return (gi < m.n && gj >= 0 && d >= 0 && d <= m.k) ? m.ab + d + (long long)gj * m.ldab : nullptr;
}

// Warps 4-7 (fw = warp - 4, lane p), one block ahead of the chain: for block
// It, into `slot`,
//   - the diagonal tile L_II (identity past n) with its pivots' reciprocals
//     and its four 8 x 8 triangles pre-scaled (fwd: entry (p, q) by 1/L_qq;
//     bwd: by 1/L_pp), and the near tile (fwd: L_{I+1,I}; bwd: L_{I,I-1});
//   - U = b - the far terms (fwd: sum_{J=It-P}^{It-2} L_{It,J} y_J; bwd:
//     sum_{J=It+2}^{It+P} L_{J,It}^T x_J), lane = row, the columns of each
//     block J split over the four warps.
// Every global read is an asynchronous 8-byte copy into shared memory issued
// by the thread that later reads it: the tiles and b in one group, then the
// far blocks through a ring of kDepth slots, kDepth - 1 blocks in flight, so
// the band's latency overlaps the FMAs instead of preceding each block.
template <bool FWD, int NR>
__device__ __forceinline__ void far_step(Smem& sm, const Sys& m, const double* bc, long long ldb, int nr, int slot,
                                         int It, int fw, int p, const Group& G, long long g, int tt) {
  const int ft = fw * 32 + p;
  const int g0 = It * kB, gp = g0 + p;
#pragma unroll
  for (int u = 0; u < kB / 4; ++u) {
    const int q = fw + 4 * u;
    const double* s0 = laddr(m, g0 + p, g0 + q);
    double* d0 = &sm.T[slot][0][p][q];
    if (s0) cp_async8(d0, s0); else *d0 = (p == q) ? 1.0 : 0.0;
    const double* s1 = FWD ? laddr(m, g0 + kB + p, g0 + q) : laddr(m, g0 + p, g0 - kB + q);
    double* d1 = &sm.T[slot][1][p][q];
    if (s1) cp_async8(d1, s1); else *d1 = 0.0;
  }
  {
    const int r = fw;   // four far warps, four right-hand sides
    double* d = &sm.bpre[r][p];
    if (r < nr && gp < m.n) cp_async8(d, bc + gp + (long long)r * ldb); else *d = 0.0;
  }
  cp_commit();
  const int dmax = G.W > 0 ? 2 : m.P;   // with workers this CTA keeps distance 2 only
  const int jlo = FWD ? max(0, It - dmax) : It + 2;
  const int jhi = FWD ? It - 2 : min(m.S - 1, It + dmax);
  const int ycol = ft >> 2, yr = ft & 3;   // the solved value this thread fetches for each block
  auto issue = [&](int J) {
    const int sl = (J - jlo) & (kDepth - 1);
    double* dst = sm.ring[sl][ft];
#pragma unroll
    for (int u = 0; u < kB / 4; ++u) {
      const int gq = J * kB + fw + 4 * u;
      const double* src = FWD ? laddr(m, gp, gq) : laddr(m, gq, gp);
      if (src) cp_async8(dst + u, src); else dst[u] = 0.0;
    }
    const int gq = J * kB + ycol;
    double* yd = &sm.ys[sl][ycol][yr];
    if (yr < nr && gq < m.n) cp_async8(yd, bc + gq + (long long)yr * ldb); else *yd = 0.0;
  };
  // kDepth - 1 groups before the loop and one per iteration (empty ones
  // included).  Iteration J waits for its own group (the two after it may
  // still be in flight), meets the other far warps (their solved values are
  // in), and only then reuses the slot that every warp finished reading in
  // the previous iteration.
#pragma unroll
  for (int d = 0; d < kDepth - 1; ++d) {
    if (jlo + d <= jhi) issue(jlo + d);
    cp_commit();
  }
  double acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = 0.0;
  for (int J = jlo; J <= jhi; ++J) {
    cp_wait<kDepth - 2>();
    bar_sync(kBarFar, 128);
    if (J + kDepth - 1 <= jhi) issue(J + kDepth - 1);
    cp_commit();
    const int sl = (J - jlo) & (kDepth - 1);
    const double* src = sm.ring[sl][ft];
#pragma unroll
    for (int u = 0; u < kB / 4; ++u) {
      const double lv = src[u];
      const double* y = sm.ys[sl][fw + 4 * u];
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[r] = fma(lv, y[r], acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < kR; ++r) sm.red[fw][r][p] = r < NR ? acc[r < NR ? r : 0] : 0.0;
  cp_wait<0>();
  if (G.W > 0 && fw == 0 && p == 0) {   // the workers' partial sums of this target (step tt, global index g)
    for (int w = 1; w <= G.W; ++w) {
      const int dlo = 3 + (w - 1) * G.span;
      if (dlo <= m.P && dlo <= tt) gwait(G, &G.ctl[32 + w], (int)(g + 1));
    }
  }
  bar_sync(kBarFar, 128);   // tiles, b, partial sums of all four warps and of the workers are in
  if (fw == 0) sm.rinv[slot][p] = pivot_rcp(sm.T[slot][0][p][p]);
  {
    const int r = fw;
    double ext = 0.0;
    for (int w = 1; w <= G.W; ++w) {
      const int dlo = 3 + (w - 1) * G.span;
      if (dlo <= m.P && dlo <= tt)
        ext += __ldcg(G.part + ((size_t)((w - 1) * kSlots + (int)(g % kSlots)) * kR + r) * kB + p);
    }
    sm.U[slot][r][p] =
        sm.bpre[r][p] - ((sm.red[0][r][p] + sm.red[1][r][p]) + (sm.red[2][r][p] + sm.red[3][r][p]) + ext);
  }
  bar_sync(kBarFar, 128);
#pragma unroll
  for (int u = 0; u < kB / 4; ++u) {
    const int q = fw + 4 * u;
    if (p > q && (p >> 3) == (q >> 3)) sm.T[slot][0][p][q] *= sm.rinv[slot][FWD ? q : p];
  }
}

// Warps 0-3: solve the block of step t (block I, tiles in slot s) for the
// pass's columns at bc; nacc carries the near term of the next block.
template <bool FWD>
__device__ __forceinline__ void chain_step(Smem& sm, const Sys& m, double* bc, long long ldb, int nr, int s, int I,
                                           int a, int i, int r, double& nacc) {
  const int row = 8 * a + i;
  const unsigned full = 0xffffffffu;
  double v = sm.U[s][r][row] - nacc;
  nacc = 0.0;
  const double(*D)[kTP] = sm.T[s][0];
  const double(*N)[kTP] = sm.T[s][1];
  auto near_terms = [&](int c) {   // next block's near term from triangle c of this block
    double n0 = 0.0, n1 = 0.0;
#pragma unroll
    for (int jj = 0; jj < 8; jj += 2) {
      const int c0 = 8 * c + jj;
      n0 = fma(FWD ? N[row][c0] : N[c0][row], sm.xs[r][c0], n0);
      n1 = fma(FWD ? N[row][c0 + 1] : N[c0 + 1][row], sm.xs[r][c0 + 1], n1);
    }
    nacc += n0 + n1;
  };
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    const int c = FWD ? cc : 3 - cc;
    if (a == c) {
#pragma unroll
      for (int j8 = 0; j8 < 8; ++j8) {
        const int jj = FWD ? j8 : 7 - j8;
        const double tv = __shfl_sync(full, v, jj + 8 * r);
        if (FWD ? (i > jj) : (i < jj)) v = fma(FWD ? -D[row][8 * a + jj] : -D[8 * a + jj][row], tv, v);
      }
      v *= sm.rinv[s][row];
      sm.xs[r][row] = v;
      const int gi = I * kB + row;
      if (r < nr && gi < m.n) bc[gi + (long long)r * ldb] = v;
    }
    bar_sync(kBarChain, 128);
    if (FWD ? (a > c) : (a < c)) {   // this warp's triangle comes later: subtract triangle c's products
      double g0 = 0.0, g1 = 0.0;
#pragma unroll
      for (int jj = 0; jj < 8; jj += 2) {
        const int c0 = 8 * c + jj;
        g0 = fma(FWD ? D[row][c0] : D[c0][row], sm.xs[r][c0], g0);
        g1 = fma(FWD ? D[row][c0 + 1] : D[c0 + 1][row], sm.xs[r][c0 + 1], g1);
      }
      v -= g0 + g1;
    } else if (a == c) {             // own triangle done: the near terms of every triangle so far
#pragma unroll
      for (int c2 = 0; c2 < 4; ++c2)
        if (FWD ? (c2 <= c) : (c2 >= c)) near_terms(c2);
    } else {
      near_terms(c);
    }
  }
}

// Leader: one sweep (steps base .. base + S - 1 in the group's global step count).
template <bool FWD>
__device__ __forceinline__ void sweep(Smem& sm, const Sys& m, double* bc, long long ldb, int nr, const Group& G,
                                      long long base) {
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const bool chain = w < 4;
  const int fw = w - 4;
  const int I0 = FWD ? 0 : m.S - 1;
  auto far = [&](int slot, int It, int tt) {   // the right-hand-side count as a template argument: no idle FMAs
    const long long g = base + tt;
    switch (nr) {
      case 1: far_step<FWD, 1>(sm, m, bc, ldb, nr, slot, It, fw, lane, G, g, tt); break;
      case 2: far_step<FWD, 2>(sm, m, bc, ldb, nr, slot, It, fw, lane, G, g, tt); break;
      case 3: far_step<FWD, 3>(sm, m, bc, ldb, nr, slot, It, fw, lane, G, g, tt); break;
      default: far_step<FWD, 4>(sm, m, bc, ldb, nr, slot, It, fw, lane, G, g, tt); break;
    }
  };
  if (!chain) far(0, I0, 0);   // the first block has no far terms
  __syncthreads();
  double nacc = 0.0;
  for (int t = 0; t < m.S; ++t) {
    const int I = FWD ? t : m.S - 1 - t;
    if (chain) {
      chain_step<FWD>(sm, m, bc, ldb, nr, t & 1, I, w, lane & 7, lane >> 3, nacc);
    } else if (t + 1 < m.S) {
      far((t + 1) & 1, FWD ? I + 1 : I - 1, t + 1);
    }
    __syncthreads();
    if (G.W > 0 && tid == 128) {   // publish block I (all of its stores precede the barrier)
      __threadfence();
      st_relaxed(&G.ctl[0], (int)(base + t + 1));   // after the fence: the release pattern
    }
  }
}

// Worker w: for every target block of the sweep that has blocks at its far
// distances, once the leader has solved them, the partial sum over those
// blocks (lane = row, the 32 columns of a block over the 8 warps) into ring
// slot g % kSlots, then its done count.  It never runs more than kSlots
// targets ahead of the leader's reads.  Returns false when the group aborts.
template <bool FWD, int NR>
__device__ bool worker_sweep(WSmem& ws, const Sys& m, const double* bc, long long ldb, int nr, const Group& G, int w,
                             long long base) {
  const int dlo = 3 + (w - 1) * G.span, dhi = min(m.P, dlo + G.span - 1);
  if (dlo > dhi) return true;
  const int tid = threadIdx.x, w8 = tid >> 5, p = tid & 31;
  __shared__ int s_ok;
  for (int t = dlo; t < m.S; ++t) {
    const int It = FWD ? t : m.S - 1 - t;
    const long long g = base + t;
    const int dtop = min(dhi, t);
    if (tid == 0) s_ok = gwait(G, &G.ctl[0], (int)max(g - dlo + 1, g - kSlots));
    __syncthreads();
    if (!s_ok) return false;
    double acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0.0;
    for (int d0 = dlo; d0 <= dtop; d0 += kMaxD) {
      const int nd = min(kMaxD, dtop - d0 + 1);
      for (int e = tid; e < nd * kB * kR; e += kThreads) {
        const int dd = e / (kB * kR), col = (e / kR) % kB, r = e % kR;
        const int J = FWD ? It - (d0 + dd) : It + (d0 + dd);
        const int gq = J * kB + col;
        ws.ys[dd][col][r] = (r < nr && gq < m.n) ? __ldcg(bc + gq + (long long)r * ldb) : 0.0;
      }
      double lv[kMaxD][kB / 8];
#pragma unroll
      for (int dd = 0; dd < kMaxD; ++dd) {
        const int J = FWD ? It - (d0 + dd) : It + (d0 + dd);
#pragma unroll
        for (int u = 0; u < kB / 8; ++u) {
          const int gq = J * kB + w8 + 8 * u;
          const double* src = dd < nd ? (FWD ? laddr(m, It * kB + p, gq) : laddr(m, gq, It * kB + p)) : nullptr;
          lv[dd][u] = src ? __ldg(src) : 0.0;
        }
      }
      __syncthreads();
#pragma unroll
      for (int dd = 0; dd < kMaxD; ++dd)
        if (dd < nd) {
#pragma unroll
          for (int u = 0; u < kB / 8; ++u) {
            const double* y = ws.ys[dd][w8 + 8 * u];
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] = fma(lv[dd][u], y[r], acc[r]);
          }
        }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < kR; ++r) ws.red[w8][r][p] = r < NR ? acc[r < NR ? r : 0] : 0.0;
    __syncthreads();
    if (tid < kR * kB) {
      const int r = tid >> 5, row = tid & 31;
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) v += ws.red[q][r][row];
      G.part[((size_t)((w - 1) * kSlots + (int)(g % kSlots)) * kR + r) * kB + row] = v;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_relaxed(&G.ctl[32 + w], (int)(g + 1));   // after the fence: the release pattern
    }
  }
  return true;
}

template <bool FWD>
__device__ bool worker_sweep_nr(WSmem& ws, const Sys& m, const double* bc, long long ldb, int nr, const Group& G,
                                int w, long long base) {
  switch (nr) {
    case 1: return worker_sweep<FWD, 1>(ws, m, bc, ldb, nr, G, w, base);
    case 2: return worker_sweep<FWD, 2>(ws, m, bc, ldb, nr, G, w, base);
    case 3: return worker_sweep<FWD, 3>(ws, m, bc, ldb, nr, G, w, base);
    default: return worker_sweep<FWD, 4>(ws, m, bc, ldb, nr, G, w, base);
  }
}

}  // namespace bsolve
}  // namespace bchol
