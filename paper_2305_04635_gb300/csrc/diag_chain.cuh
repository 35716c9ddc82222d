// diag_chain.cuh -- the diagonal chain of the single-matrix factor kernel.
//
// One CTA of the persistent launch runs, for s = 0, 1, ..., S-1,
//     DIAG(s) = TRSM(s, s-1), UPD(s, s, s-1) (the DSYRK), POTRF(s)
// i.e. the whole critical path of Algorithm 1, with L(s-1, s-1) kept in
// shared memory between steps.  L(s, s-1) is published as soon as it is
// solved (the updates UPD(I, s, s-1) of the other CTAs need it), before the
// DSYRK and the POTRF run.
//
// Each SM sub-partition's FP64 unit accepts one warp instruction every 64
// cycles whatever the number of active lanes, and a dependent FP64 operation
// waits about that long (rsqrt about 360 cycles).  So the chain is laid out by
// sub-partition: four compute warps (0-3, one per sub-partition) carry the
// FP64 work; in POTRF warp 0 runs the pivot recurrence alone on its
// sub-partition while warps 1-3 apply the rank-1 updates one column behind.
// Two more warps issue no FP64 at all: warp 4 publishes ready counters (so no
// compute warp stalls on a release), warp 5 waits for the next step's input
// tiles and copies them into a second buffer while the current step runs.
#pragma once
#include <type_traits>

#include "factor_tasks.cuh"

namespace bchol {

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
constexpr int kBarInit = 7;  // warps 0-5 (192 threads)

template <int B, bool F32>
struct DiagSmem {
  double X[2][B * B];  // A(s, s-1) in, L(s, s-1) out; buffer s & 1
  double D[2][B * B];  // A(s, s); buffer s & 1
  double L[B * B];     // L(s, s), kept for the next step's TRSM
  float Xf[F32 ? B * B : 1];
  float Lf[F32 ? B * B : 1];
  double r[B];    // 1 / L(j, j): the reciprocal square roots of the last POTRF's pivots
  float rf[F32 ? B : 1];
  double lj[B];   // L(j, j)
  double col[B];  // column j of L while POTRF runs
  unsigned short tri[B * (B + 1) / 2];  // lower-triangle entries (l << 8 | i), last column first
  int in_ready;   // prefetcher: the inputs of steps < in_ready are in place
  int consumed;   // compute: steps < consumed are finished (their buffers are free)
  int pub;        // compute: publish requests issued so far
  int stop;       // any role: stop now
  int fail;       // POTRF: first non-positive pivot (1-based column in the tile), or 0
  int ok;         // compute: broadcast of a wait result
};

// Bounded wait (one thread) until *p >= target in shared memory.
__device__ __forceinline__ bool wait_smem_geq(const int* p, int target, const int* stop, Control* ctl,
                                              int* status, uint64_t limit_ns) {
  if (ld_acquire_cta(p) >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
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

template <int B>
__device__ __forceinline__ void load_tile_lanes(const FactorArgs& a, int I, int J, double* s, int lane) {
#pragma unroll 8
  for (int idx = lane; idx < B * B; idx += 32) {
    const int i = idx % B, j = idx / B;
    const int gi = I * B + i, gj = J * B + j, d = gi - gj;
    s[j * B + i] = (gi < a.n && d >= 0 && d <= a.k) ? __ldcg(a.ab + d + (long long)gj * a.ldab) : 0.0;
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

// ----------------------------------------------------------- prefetcher (warp 5)
// For step s: waits until the other CTAs have applied every update of A(s, s-1)
// and A(s, s) except the step s-1 DSYRK (steps s0(s) .. s-2), and copies both
// tiles into buffer s & 1 (free once step s-2 is finished).
template <int B, bool F32>
__device__ void diag_prefetcher(const FactorArgs& a, DiagSmem<B, F32>& sm, int lane) {
  const uint64_t limit = 4 * a.wait_ns;
  for (int s = 0; s < a.S; ++s) {
    const int cur = s & 1;
    const int s0 = first_step(a, s);
    const bool has_x = s >= 1 && a.p >= 1;
    int ok = 1;
    if (lane == 0) {
      if (s >= 2) ok = wait_smem_geq(&sm.consumed, s - 1, &sm.stop, a.ctl, a.status, limit);
      if (ok && has_x) ok = wait_tile(a, s, s - 1, s - 1 - s0);
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    if (!ok) break;
    if (has_x) load_tile_lanes<B>(a, s, s - 1, sm.X[cur], lane);
    if (lane == 0) ok = wait_tile(a, s, s, has_x ? s - 1 - s0 : s - s0);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    if (!ok) break;
    load_tile_lanes<B>(a, s, s, sm.D[cur], lane);
    __syncwarp();
    if (lane == 0) st_release_cta(&sm.in_ready, s + 1);
  }
  if (lane == 0) {
    // a failed wait (timeout or abort) ends the chain
    if (ld_acquire_cta(&sm.in_ready) < a.S) *(volatile int*)&sm.stop = 1;
  }
}

// --------------------------------------------------------------------- TRSM
// X := X L^{-T} with L = L(s-1, s-1) and r = 1/diag(L), in place.  Warp w owns
// rows w*B/4 ..; G lanes share a row, lane g keeps columns g, g+G, ... in
// registers; column j is finished by its owner and shuffled to the row group.
template <int B, typename VT, bool F32>
__device__ __forceinline__ void diag_trsm(DiagSmem<B, F32>& sm, double* X, int tid) {
  constexpr int RPW = B / 4, G = 32 / RPW, C = B / G;
  const int warp = tid >> 5, lane = tid & 31;
  const int i = warp * RPW + lane / G, g = lane % G;
  const VT* Lm;
  if constexpr (F32) Lm = sm.Lf; else Lm = sm.L;
  VT acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = (VT)X[(g + G * c) * B + i];
#pragma unroll
  for (int j = 0; j < B; ++j) {
    const int go = j % G, co = j / G;
    if constexpr (F32) {
      if (g == go) acc[co] *= sm.rf[j];
    } else {
      if (g == go) acc[co] *= sm.r[j];
    }
    const VT x = __shfl_sync(0xffffffffu, acc[co], go, G);
#pragma unroll
    for (int c = co; c < C; ++c) {
      const int l = g + G * c;
      if (l > j) {
        if constexpr (F32) acc[c] = fmaf(-x, Lm[j * B + l], acc[c]);
        else acc[c] = fma(-x, Lm[j * B + l], acc[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < C; ++c) {
    X[(g + G * c) * B + i] = (double)acc[c];
    if constexpr (F32) sm.Xf[(g + G * c) * B + i] = (float)acc[c];
  }
}

// --------------------------------------------------------------------- DSYRK
// D -= X X^T on the lower triangle (FP32 products and sums in the mixed form).
template <int B, typename VT, bool F32>
__device__ __forceinline__ void diag_syrk(DiagSmem<B, F32>& sm, const double* X, double* D, int tid) {
  constexpr int NT = B * (B + 1) / 2;
  const VT* Xm;
  if constexpr (F32) Xm = sm.Xf; else Xm = X;
  for (int e = tid; e < NT; e += 128) {
    const int code = sm.tri[e];
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
}

// -------------------------------------------------------------------- POTRF
// Right-looking Cholesky of D (jmax valid columns) into sm.L.  Warp 0 lane 0
// runs the pivot recurrence  x = D(j+1,j) r_j,  d_{j+1} = D(j+1,j+1) - x^2,
// r_{j+1} = rsqrt(d_{j+1}); warps 1-3 then form column j of L and apply its
// rank-1 update to the trailing triangle (all but D(j+1,j+1), which the
// recurrence owns).  Warp 0 needs column j-1's updates before pivot j+1, so
// the updates run one column behind the recurrence.
template <int B, bool F32>
__device__ __forceinline__ void diag_potrf(DiagSmem<B, F32>& sm, double* D, int jmax, int tid) {
  const int warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    double r = 0.0;
    if (lane == 0) {
      const double d = D[0];
      if (!(d > 0.0)) sm.fail = 1;
      r = rsqrt(d);
      sm.r[0] = r;
      sm.lj[0] = d * r;
    }
    __syncwarp();
    bar_arrive(kBarP, 128);
    for (int j = 0; j + 1 < jmax; ++j) {
      if (j >= 1) bar_sync(kBarU + ((j - 1) & 1), 128);
      if (lane == 0) {
        const double x = D[j * B + j + 1] * r;
        const double v = fma(-x, x, D[(j + 1) * B + j + 1]);
        if (!(v > 0.0) && sm.fail == 0) sm.fail = j + 2;
        r = rsqrt(v);
        sm.r[j + 1] = r;
        sm.lj[j + 1] = v * r;
      }
      __syncwarp();
      bar_arrive(kBarP + ((j + 1) & 1), 128);
    }
    if (jmax >= 2) bar_sync(kBarU + ((jmax - 2) & 1), 128);
  } else {
    const int u = tid - 32;
    for (int j = 0; j < jmax; ++j) {
      bar_sync(kBarP + (j & 1), 128);
      const double r = sm.r[j];
      for (int i = j + 1 + u; i < jmax; i += 96) {
        const double lc = D[j * B + i] * r;
        sm.col[i] = lc;
        sm.L[j * B + i] = lc;
      }
      if (u == 0) sm.L[j * B + j] = sm.lj[j];
      if (j + 1 < jmax) {
        __syncwarp();
        bar_sync(kBarW, 96);
        const int T = (B - 1 - j) * (B - j) / 2;
        for (int e = u; e < T; e += 96) {
          const int code = sm.tri[e];
          const int i = code & 0xff, l = code >> 8;
          if (i < jmax && !(i == j + 1 && l == j + 1)) D[l * B + i] = fma(-sm.col[i], sm.col[l], D[l * B + i]);
        }
        __syncwarp();
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
      bar_sync(kBarC, 128);
    }
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
    store_tile_compute<B>(a, s, s, sm.L, tid);
    if constexpr (F32) {
      for (int idx = tid; idx < B * B; idx += 128) sm.Lf[idx] = (float)sm.L[idx];
      if (tid < B) sm.rf[tid] = (float)sm.r[tid];
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
__device__ void diag_chain(const FactorArgs& a, DiagSmem<B, F32>& sm) {
  static_assert(B == 16 || B == 32, "the diagonal chain supports tiles of 16 and 32");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp >= 6) return;
  if (tid == 0) {
    sm.in_ready = 0;
    sm.consumed = 0;
    sm.pub = 0;
    sm.stop = 0;
    sm.fail = 0;
  }
  // triangle table: column l holds B - l entries, columns ordered B-1, B-2, ..., 0
  for (int e = tid; e < B * (B + 1) / 2; e += 192) {
    int l = B - 1, off = 0;
    while (e >= off + (B - l)) {
      off += B - l;
      --l;
    }
    const int i = l + (e - off);
    sm.tri[e] = (unsigned short)((l << 8) | i);
  }
  bar_sync(kBarInit, 192);
  if (warp == 4) {
    diag_publisher<B, F32>(a, sm, lane);
  } else if (warp == 5) {
    diag_prefetcher<B, F32>(a, sm, lane);
  } else {
    diag_compute<B, F32>(a, sm, tid);
  }
}

}  // namespace bchol
