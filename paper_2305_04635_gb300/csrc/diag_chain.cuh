// diag_chain.cuh -- the diagonal chain of the single-matrix factor kernel.
//
// One CTA of the persistent launch runs, for s = 0, 1, ..., S-1,
//     DIAG(s) = TRSM(s, s-1), UPD(s, s, s-1) (the DSYRK), POTRF(s)
// i.e. the whole critical path of Algorithm 1, with the factor of the
// previous diagonal tile (as its unit lower part and 1/diag) kept in shared
// memory between steps.  L(s, s-1) is published as soon as it is
// solved (the updates UPD(I, s, s-1) of the other CTAs need it), before the
// DSYRK and the POTRF run.
//
// Each SM sub-partition's FP64 unit accepts one warp instruction every 64
// cycles whatever the number of active lanes, and a dependent FP64 operation
// waits about that long (rsqrt about 360 cycles).  So the chain is laid out by
// sub-partition: four compute warps (0-3, one per sub-partition) carry the
// FP64 work; in POTRF warp 0 runs the pivot recurrence alone on its
// sub-partition while warps 1-3 apply the rank-1 updates one column behind.
// The other warps issue no FP64 at all: warp 4 publishes ready counters (so
// no compute warp stalls on a release), warps 5-7 wait for the next step's
// input tiles and copy them into a second buffer while the current step runs.
#pragma once
#include <cuda.h>

#include <type_traits>

#include "factor_tasks.cuh"

namespace bchol {

// 1/d for the pivot recurrence: the hardware seed rcp.approx.ftz.f64 (relative
// error below 2^-20, measured) refined by one step of the cubic Newton-type
// iteration y1 = y0 (1 + e + e^2), e = 1 - d y0, whose error is e^3 (below
// 2^-60) plus the rounding of the three FMAs.  Three dependent FP64
// operations instead of a full division on the chain.  d > 0 in use; other
// inputs give a non-finite or meaningless result, and the caller has already
// flagged the pivot.
__device__ __forceinline__ double pivot_rcp(double d) {
  double y0;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(d));
  const double e = fma(-d, y0, 1.0);
  const double p = fma(e, e, e);
  return fma(y0, p, y0);
}

// Named barriers (whole warps only: the warp is reconverged first).
__device__ __forceinline__ void bar_sync(int id, int count) {
  __syncwarp();
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count) {
  __syncwarp();
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void st_release_cta(int* p, int v) {
  asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v)
               : "memory");
}
__device__ __forceinline__ int ld_acquire_cta(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared.b32 %0, [%1];"
               : "=r"(v)
               : "r"((unsigned)__cvta_generic_to_shared(p))
               : "memory");
  return v;
}

// Named barriers of the chain CTA (0 is __syncthreads, unused there).
constexpr int kBarC = 1;     // compute warps 0-3 (128 threads)
constexpr int kBarP = 2;     // 2, 3 by parity of j: pivot j is ready (warp 0 arrives, warps 1-3 wait)
constexpr int kBarU = 4;     // 4, 5 by parity of j: column j's updates are done (warps 1-3 arrive, warp 0 waits)
constexpr int kBarW = 6;     // update warps 1-3 (96 threads)
constexpr int kBarInit = 7;  // the whole CTA (256 threads)
constexpr int kBarPF = 8;    // prefetch warps 5-7 (96 threads)

template <int B, bool F32>
struct DiagSmem {
  double X[2][B * B];  // A(s, s-1) in, L(s, s-1) out; buffer s & 1
  double D[2][B * B];  // A(s, s); buffer s & 1
  double U[B * B];     // unit lower factor of L(s, s): U(i, j) = L(i, j) / L(j, j), kept for the next TRSM
  float Xf[F32 ? B * B : 1];
  float Uf[F32 ? B * B : 1];
  float rf[F32 ? B : 1];
  double d[B];    // pivots d_j of the Schur recurrence
  double inv[B];  // 1 / d_j
  double r[B];    // 1 / sqrt(d_j) = 1 / L(j, j)
  double q[B];    // q_{j+1} = D(j+1, j)^2 after the updates of columns < j
  unsigned short tri[B * (B + 1) / 2];  // lower-triangle entries (l << 8 | i), last column first
  int in_ready;   // prefetcher: the inputs of steps < in_ready are in place
  int consumed;   // compute: steps < consumed are finished (their buffers are free)
  int pub;        // compute: publish requests issued so far
  int stop;       // any role: stop now
  int fail;       // POTRF: first non-positive pivot (1-based column in the tile), or 0
  int ok;         // compute: broadcast of a wait result
  int pf_ok_d;    // prefetch: broadcast of the wait for A(s, s) and A(s, s-1)
  unsigned long long pf_mbar;   // prefetch with TMA: completion of the two tile copies of a step
};

constexpr unsigned kPollNs = 64;  // back-off of the service warps' polls

// Bounded wait (one thread) until *p >= target in shared memory.
__device__ __forceinline__ bool wait_smem_geq(const int* p, int target, const int* stop, Control* ctl,
                                              int* status, uint64_t limit_ns) {
  if (ld_acquire_cta(p) >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    __nanosleep(kPollNs);  // keep the poll off the compute warps' shared-memory pipe
    if (ld_acquire_cta(p) >= target) return true;
    if (*(volatile const int*)stop) return false;
    if (ld_relaxed(&ctl->abort) != 0) return false;
    if (globaltimer_ns() - t0 > limit_ns) {
      atomicExch(status, kStatusTimeout);
      atomicExch(&ctl->abort, 1);
      return false;
    }
  }
}

// wait_tile with a back-off between polls (the chain CTA's prefetch warp).
__device__ __forceinline__ bool wait_tile_poll(const FactorArgs& a, int I, int J, int target) {
  const int f = fidx(a, I, J);
  if (f == a.stall) target = 0x7fffffff;
  const int* flag = &a.flags[f];
  if (ld_acquire(flag) >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    __nanosleep(kPollNs);
    if (ld_acquire(flag) >= target) return true;
    if (ld_relaxed(&a.ctl->abort) != 0) return false;
    if (globaltimer_ns() - t0 > a.wait_ns) {
      atomicExch(a.status, kStatusTimeout);
      atomicExch(&a.ctl->abort, 1);
      return false;
    }
  }
}

// Tiles A(s, s) and A(s, s-1) together (96 threads): every load of both is in
// flight before the first store into shared memory.
template <int B>
__device__ __forceinline__ void load_tiles_group(const FactorArgs& a, int s, double* D, double* X, bool has_x,
                                                 int pt) {
  constexpr int E = (B * B + 95) / 96;
  double vd[E], vx[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = pt + 96 * e;
    const int i = idx % B, j = idx / B;
    const int gi = s * B + i, gd = s * B + j, gx = (s - 1) * B + j;
    const bool in = idx < B * B && gi < a.n;
    vd[e] = (in && gi - gd >= 0 && gi - gd <= a.k) ? __ldcg(a.ab + (gi - gd) + (long long)gd * a.ldab) : 0.0;
    vx[e] = (has_x && in && gi - gx <= a.k) ? __ldcg(a.ab + (gi - gx) + (long long)gx * a.ldab) : 0.0;
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = pt + 96 * e;
    if (idx < B * B) {
      D[idx] = vd[e];
      if (has_x) X[idx] = vx[e];
    }
  }
}

template <int B>
__device__ __forceinline__ void store_tile_compute(const FactorArgs& a, int I, int J, const double* s, int tid) {
  for (int idx = tid; idx < B * B; idx += 128) {
    const int i = idx % B, j = idx / B;
    const int gi = I * B + i, gj = J * B + j, d = gi - gj;
    if (gi < a.n && d >= 0 && d <= a.k) a.ab[d + (long long)gj * a.ldab] = s[j * B + i];
  }
}

// ------------------------------------------------------------ publisher (warp 4)
// Releases, in order, the ready counter of L(s, s-1) (final value s - s0(s))
// and of L(s, s) (final value s - s0(s) + 1) once the compute warps have
// stored the tile and posted the request.
template <int B, bool F32>
__device__ void diag_publisher(const FactorArgs& a, DiagSmem<B, F32>& sm, int lane) {
  if (lane != 0) return;
  const uint64_t limit = 4 * a.wait_ns;
  int ev = 0;
  for (int s = 0; s < a.S; ++s) {
    const int s0 = first_step(a, s);
    if (s >= 1 && a.p >= 1) {
      if (!wait_smem_geq(&sm.pub, ev + 1, &sm.stop, a.ctl, a.status, limit)) return;
      ++ev;
      st_release(&a.flags[fidx(a, s, s - 1)], s - s0);
    }
    if (!wait_smem_geq(&sm.pub, ev + 1, &sm.stop, a.ctl, a.status, limit)) return;
    ++ev;
    st_release(&a.flags[fidx(a, s, s)], s - s0 + 1);
  }
}

// ------------------------------------------------ TMA copies of the two tiles
// The band as a 2-D tensor: element (gi, gj) at ab + gi + gj (ldab - 1) (the
// skewed tile view of bchol_device.cuh), dims (n, n), so that tile (I, J) is
// the box at (I b, J b).  The whole view lies inside the n x ldab array; boxes
// past n are zero-filled, slots outside the band are masked after the copy.
// Used when (ldab - 1) * 8 is a multiple of 16 (ldab odd), the tensor-map rule.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void pf_mbar_init(unsigned long long* mb) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mb)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void pf_expect(unsigned long long* mb, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void pf_tma_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* mb) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(mb))
      : "memory");
}
__device__ __forceinline__ bool pf_try_wait(unsigned long long* mb, unsigned parity) {
  unsigned done;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(smem_u32(mb)), "r"(parity)
      : "memory");
  return done != 0;
}

// ------------------------------------------------------- prefetcher (warps 5-7)
// For step s: waits until the other CTAs have applied every update of A(s, s)
// and A(s, s-1) except the step s-1 DSYRK (steps s0(s) .. s-2), and copies both
// tiles into buffer s & 1 (free once step s-2 is finished).  One thread waits
// for both (A(s, s-1) is the later one); the three warps copy both tiles with
// all loads in flight at once.
// With a.tma the copies are two TMA box loads onto an mbarrier (thread 0 of
// the prefetcher issues them after the waits, the three warps wait for the
// barrier with a bound, then zero the slots outside the band).
template <int B, bool F32>
__device__ void diag_prefetcher(const FactorArgs& a, DiagSmem<B, F32>& sm, int pt, const CUtensorMap* tmap) {
  const uint64_t limit = 4 * a.wait_ns;
  bool failed = false;
  if (a.tma && pt == 0) pf_mbar_init(&sm.pf_mbar);
  bar_sync(kBarPF, 96);
  for (int s = 0; s < a.S; ++s) {
    const int cur = s & 1;
    const int s0 = first_step(a, s);
    const bool has_x = s >= 1 && a.p >= 1;
    if (pt == 0) {
      int ok = 1;
      if (s >= 2) ok = wait_smem_geq(&sm.consumed, s - 1, &sm.stop, a.ctl, a.status, limit);
      if (ok) ok = wait_tile_poll(a, s, s, has_x ? s - 1 - s0 : s - s0);
      if (ok && has_x) ok = wait_tile_poll(a, s, s - 1, s - 1 - s0);
      sm.pf_ok_d = ok;
    }
    bar_sync(kBarPF, 96);
    if (!sm.pf_ok_d) {
      failed = true;
      break;
    }
    if (a.tma) {
      if (pt == 0) {
        // the buffer's previous contents were read (and masked) through the generic proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        pf_expect(&sm.pf_mbar, (has_x ? 2u : 1u) * B * B * 8u);
        pf_tma_2d(sm.D[cur], tmap, s * B, s * B, &sm.pf_mbar);
        if (has_x) pf_tma_2d(sm.X[cur], tmap, s * B, (s - 1) * B, &sm.pf_mbar);
      }
      const uint64_t t0 = globaltimer_ns();
      bool ok;
      while (!(ok = pf_try_wait(&sm.pf_mbar, (unsigned)(s & 1))) && globaltimer_ns() - t0 < limit) {
      }
      if (!ok) {   // a copy that never completes: record it and stop the chain (after a second bounded wait)
        if (pt == 0) {
          atomicExch(a.status, kStatusTimeout);
          atomicExch(&a.ctl->abort, 1);
          const uint64_t t1 = globaltimer_ns();
          while (!pf_try_wait(&sm.pf_mbar, (unsigned)(s & 1)) && globaltimer_ns() - t1 < limit) {
          }
        }
        failed = true;
        break;
      }
      constexpr int E = (B * B + 95) / 96;
#pragma unroll
      for (int e = 0; e < E; ++e) {   // the slots outside the band (and above the diagonal) read as zero
        const int idx = pt + 96 * e;
        if (idx < B * B) {
          const int i = idx % B, j = idx / B;
          const int dd = i - j;
          if (dd < 0 || dd > a.k) sm.D[cur][idx] = 0.0;
          if (has_x && B + dd > a.k) sm.X[cur][idx] = 0.0;
        }
      }
    } else {
      load_tiles_group<B>(a, s, sm.D[cur], sm.X[cur], has_x, pt);
    }
    bar_sync(kBarPF, 96);
    if (pt == 0) st_release_cta(&sm.in_ready, s + 1);
  }
  // a failed wait (timeout or abort) ends the chain
  if (failed && pt == 0) *(volatile int*)&sm.stop = 1;
}

// --------------------------------------------------------------------- TRSM
// X := X L^{-T} with L = L(s-1, s-1) = U diag(1/r): the rows of Z = X diag(1/r)
// solve the unit lower system Z U^T = A by substitution without divisions,
// and X = Z diag(r) at the end.  Warp w owns rows w*B/4 ..; G lanes share a
// row, lane g keeps columns g, g+G, ... in registers; column j, final when the
// sweep reaches it, is shuffled to the row group.  Each step of the chain is
// one shuffle and one DFMA.  (A product with an explicit L^{-1} would drop the
// chain altogether, but forming L^{-1} inside POTRF costs the chain CTA more
// than it saves here.)
template <int B, typename VT, bool F32>
__device__ __forceinline__ void diag_trsm(DiagSmem<B, F32>& sm, double* X, int tid) {
  constexpr int RPW = B / 4, G = 32 / RPW, C = B / G;
  const int warp = tid >> 5, lane = tid & 31;
  const int i = warp * RPW + lane / G, g = lane % G;
  const VT* Um;
  if constexpr (F32) Um = sm.Uf; else Um = sm.U;
  VT acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = (VT)X[(g + G * c) * B + i];
#pragma unroll
  for (int j = 0; j < B - 1; ++j) {
    const int go = j % G, co = j / G;
    const VT z = __shfl_sync(0xffffffffu, acc[co], go, G);
#pragma unroll
    for (int c = co; c < C; ++c) {
      const int l = g + G * c;
      if (l > j) {
        if constexpr (F32) acc[c] = fmaf(-z, Um[j * B + l], acc[c]);
        else acc[c] = fma(-z, Um[j * B + l], acc[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int l = g + G * c;
    VT v;
    if constexpr (F32) v = acc[c] * sm.rf[l]; else v = acc[c] * sm.r[l];
    X[l * B + i] = (double)v;
    if constexpr (F32) sm.Xf[l * B + i] = (float)v;
  }
}

// --------------------------------------------------------------------- DSYRK
// D -= X X^T on the lower triangle (FP32 products and sums in the mixed form).
// 128 threads: full passes of one entry per thread, then the R left-over
// entries split by terms over 128/R lanes each and summed by shuffles, so the
// four sub-partitions get the same number of FP64 instructions.
template <int B, typename VT, bool F32>
__device__ __forceinline__ void diag_syrk(DiagSmem<B, F32>& sm, const double* X, double* D, int tid) {
  constexpr int NT = B * (B + 1) / 2, PASSES = NT / 128, R = NT - 128 * PASSES;
  constexpr int TPE = 128 / R, TERMS = B / TPE;
  static_assert(R > 0 && 128 % R == 0 && B % TPE == 0 && TPE <= 32, "DSYRK split");
  const VT* Xm;
  if constexpr (F32) Xm = sm.Xf; else Xm = X;
  for (int ps = 0; ps < PASSES; ++ps) {
    const int code = sm.tri[tid + 128 * ps];
    const int i = code & 0xff, l = code >> 8;
    if constexpr (F32) {
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < B; ++m) acc = fmaf(Xm[m * B + i], Xm[m * B + l], acc);
      D[l * B + i] -= (double)acc;
    } else {
      double acc = D[l * B + i];
#pragma unroll
      for (int m = 0; m < B; ++m) acc = fma(-Xm[m * B + i], Xm[m * B + l], acc);
      D[l * B + i] = acc;
    }
  }
  const int code = sm.tri[128 * PASSES + tid / TPE], part = tid % TPE;
  const int i = code & 0xff, l = code >> 8;
  VT acc = 0;
#pragma unroll
  for (int m = part * TERMS; m < (part + 1) * TERMS; ++m) {
    if constexpr (F32) acc = fmaf(Xm[m * B + i], Xm[m * B + l], acc);
    else acc = fma(Xm[m * B + i], Xm[m * B + l], acc);
  }
#pragma unroll
  for (int off = TPE / 2; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (part == 0) D[l * B + i] -= (double)acc;
}

// -------------------------------------------------------------------- POTRF
// Cholesky of D (jmax valid columns) by the Schur recurrence without square
// roots on the chain: with d_j the j-th pivot and U(i, j) = D(i, j) / d_j,
//     D(i, l) -= U(i, j) D(l, j)   (j < l <= i),   d_{j+1} = D(j+1, j+1) - D(j+1, j)^2 / d_j,
// and L(i, j) = D(i, j) r_j with r_j = 1/sqrt(d_j) afterwards (all square
// roots in one batch once the chain is done).  Warp 0 lane 0 runs only the
// pivot recurrence (one DFMA and one reciprocal per column), alone on its
// sub-partition; warps 1-3 form column j of U and apply the rank-1 update one
// column behind (two entries per thread at a time, so their loads and FMAs
// overlap).  D(j+1, j+1) and q_{j+1} = D(j+1, j)^2 reach the recurrence through
// shared memory; the recurrence's own entry D(j+1, j+1) is left out of column
// j's update.  U is kept for the next step's TRSM.  (Posting the next pivot's
// two entries ahead of the rest of the column was measured slower: the update
// warps, not the recurrence, then set the pace.  So was forming the products
// D(i, j) D(l, j) before 1/d_j arrives, with the entries kept in registers:
// the product pass lengthened the update warps' step by more than the
// DMUL it took off the path.)
template <int B, bool F32>
__device__ __forceinline__ void diag_potrf(DiagSmem<B, F32>& sm, double* D, int jmax, int tid) {
  const int warp = tid >> 5, lane = tid & 31;
  double* U = sm.U;
  if (warp == 0) {
    double inv = 0.0;
    if (lane == 0) {
      const double d = D[0];
      if (jmax >= 2) sm.q[1] = D[1] * D[1];
      sm.d[0] = d;
      inv = pivot_rcp(d);
      sm.inv[0] = inv;
    }
    bar_arrive(kBarP, 128);
    for (int j = 0; j + 1 < jmax; ++j) {
      if (j >= 1) bar_sync(kBarU + ((j - 1) & 1), 128);
      if (lane == 0) {
        const double d = fma(-sm.q[j + 1], inv, D[(j + 1) * B + j + 1]);
        sm.d[j + 1] = d;
        inv = pivot_rcp(d);
        sm.inv[j + 1] = inv;
      }
      bar_arrive(kBarP + ((j + 1) & 1), 128);
    }
    if (jmax >= 2) bar_sync(kBarU + ((jmax - 2) & 1), 128);
    // The first pivot that is not positive, found once the recurrence is done
    // (one pivot per lane): a bad pivot only spoils the columns after it, and
    // the step is then abandoned, so the recurrence itself carries no test.
    for (int j0 = 0; j0 < jmax; j0 += 32) {
      const unsigned bad = __ballot_sync(0xffffffffu, j0 + lane < jmax && !(sm.d[j0 + lane] > 0.0));
      if (bad) {
        if (lane == 0) sm.fail = j0 + __ffs(bad);
        break;
      }
      if (lane == 0) sm.fail = 0;
    }
  } else {
    const int u = tid - 32;
    for (int j = 0; j < jmax; ++j) {
      bar_sync(kBarP + (j & 1), 128);
      if (j + 1 < jmax) {
        const double inv = sm.inv[j];
        for (int i = j + 1 + u; i < jmax; i += 96) U[j * B + i] = D[j * B + i] * inv;
        bar_sync(kBarW, 96);
        const int T = (B - 1 - j) * (B - j) / 2;
        for (int e = u; e < T; e += 192) {
          const int e2 = e + 96;
          const int c1 = sm.tri[e], c2 = e2 < T ? (int)sm.tri[e2] : 0;
          const int i1 = c1 & 0xff, l1 = c1 >> 8, i2 = c2 & 0xff, l2 = c2 >> 8;
          const bool ok1 = i1 < jmax && !(i1 == j + 1 && l1 == j + 1);
          const bool ok2 = e2 < T && i2 < jmax && !(i2 == j + 1 && l2 == j + 1);
          const double a1 = D[l1 * B + i1], x1 = D[j * B + l1], y1 = U[j * B + i1];
          const double a2 = D[l2 * B + i2], x2 = D[j * B + l2], y2 = U[j * B + i2];
          const double v1 = fma(-y1, x1, a1);
          const double v2 = fma(-y2, x2, a2);
          if (ok1) {
            D[l1 * B + i1] = v1;
            if (i1 == j + 2 && l1 == j + 1) sm.q[j + 2] = v1 * v1;
          }
          if (ok2) {
            D[l2 * B + i2] = v2;
            if (i2 == j + 2 && l2 == j + 1) sm.q[j + 2] = v2 * v2;
          }
        }
        bar_arrive(kBarU + (j & 1), 128);
      }
    }
  }
}

// ------------------------------------------------------------ compute warps 0-3
template <int B, bool F32>
__device__ void diag_compute(const FactorArgs& a, DiagSmem<B, F32>& sm, int tid) {
  using VT = typename std::conditional<F32, float, double>::type;
  const uint64_t limit = 4 * a.wait_ns;
  int pub = 0;
  for (int s = 0; s < a.S; ++s) {
    const int cur = s & 1;
    if (tid == 0) sm.ok = wait_smem_geq(&sm.in_ready, s + 1, &sm.stop, a.ctl, a.status, limit);
    bar_sync(kBarC, 128);
    if (!sm.ok) return;
    double* X = sm.X[cur];
    double* D = sm.D[cur];
    if (s >= 1 && a.p >= 1) {
      diag_trsm<B, VT, F32>(sm, X, tid);
      bar_sync(kBarC, 128);
      store_tile_compute<B>(a, s, s - 1, X, tid);
      bar_sync(kBarC, 128);
      if (tid == 0) st_release_cta(&sm.pub, ++pub);
      diag_syrk<B, VT, F32>(sm, X, D, tid);
    }
    bar_sync(kBarC, 128);
    const int jmax = min(B, a.n - s * B);
    diag_potrf<B, F32>(sm, D, jmax, tid);
    bar_sync(kBarC, 128);
    if (sm.fail) {
      if (tid == 0) {
        atomicCAS(a.info, 0, s * B + sm.fail);
        atomicExch(&a.ctl->abort, 1);
        *(volatile int*)&sm.stop = 1;
      }
      return;
    }
    if (tid < jmax) sm.r[tid] = rsqrt(sm.d[tid]);
    bar_sync(kBarC, 128);
    if constexpr (F32) {
      if (tid < B) sm.rf[tid] = (float)sm.r[tid];
    }
    // L(i, j) = D(i, j) r_j and L(j, j) = d_j r_j, formed as they are stored
    for (int idx = tid; idx < B * B; idx += 128) {
      const int i = idx % B, j = idx / B;
      if (i >= j && i < jmax) {
        const double rj = sm.r[j];
        const int gi = s * B + i, gj = s * B + j, dd = gi - gj;
        if (dd <= a.k) a.ab[dd + (long long)gj * a.ldab] = (i == j) ? sm.d[j] * rj : D[idx] * rj;
        if constexpr (F32) sm.Uf[idx] = (float)sm.U[idx];
      }
    }
    bar_sync(kBarC, 128);
    if (tid == 0) {
      st_release_cta(&sm.pub, ++pub);
      st_release_cta(&sm.consumed, s + 1);
    }
  }
}

// Entry of the chain CTA (all kThreads threads).
template <int B, bool F32>
__device__ void diag_chain(const FactorArgs& a, DiagSmem<B, F32>& sm, const CUtensorMap* tmap) {
  static_assert(B == 16 || B == 32, "the diagonal chain supports tiles of 16 and 32");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    sm.in_ready = 0;
    sm.consumed = 0;
    sm.pub = 0;
    sm.stop = 0;
    sm.fail = 0;
  }
  // triangle table: column l holds B - l entries, columns ordered B-1, B-2, ..., 0
  for (int e = tid; e < B * (B + 1) / 2; e += kThreads) {
    int l = B - 1, off = 0;
    while (e >= off + (B - l)) {
      off += B - l;
      --l;
    }
    const int i = l + (e - off);
    sm.tri[e] = (unsigned short)((l << 8) | i);
  }
  bar_sync(kBarInit, kThreads);
  if (warp == 4) {
    diag_publisher<B, F32>(a, sm, lane);
  } else if (warp >= 5) {
    diag_prefetcher<B, F32>(a, sm, tid - 160, tmap);
  } else {
    diag_compute<B, F32>(a, sm, tid);
  }
}

}  // namespace bchol
