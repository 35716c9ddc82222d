// bchol_device.cuh -- device-side helpers shared by the factor and solve kernels.
//
// Band storage (Sec. 3 of the paper keeps the LAPACK band layout): A(i,j),
// 0 <= i-j <= k, lives at ab[(i-j) + j*ldab].  A b x b tile (I,J) of the
// matrix is therefore a skewed view of `ab`: element (i,j) of the tile sits
// at ab + (I*b+i) + (J*b+j)*(ldab-1).  Slots outside the band alias other
// entries or run past the array, so every tile load masks them to zero and
// every tile store skips them (this plays the part of the paper's zeroed work
// array for the cut-off corner block, Sec. 2.1 / Algorithm 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bchol_internal.h"

namespace bchol {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// A relaxed store: after a fence (__threadfence) it completes the release
// pattern, so several counters published together share one fence instead of
// a release store (an implied fence) each.
__device__ __forceinline__ void st_relaxed(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Control block shared by all CTAs of one launch (zeroed before each launch).
struct Control {
  unsigned long long ticket;  // next task ticket
  int abort;                  // != 0: stop (a pivot failed or a wait ran out)
  int chain_sm;               // 1 + the SM of the diagonal-chain CTA, 0 until it is known
  int retired;                // batched launch: every ticket of this matrix is taken
  int helper_sm[2];           // 1 + the SMs of the two helper CTAs, 0 until known (or without helpers)
};

__device__ __forceinline__ int sm_id() {
  int v;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
  return v;
}

// Spin (one thread) until *flag >= target.  Returns false when the launch is
// aborted or the wait exceeds wait_ns; a timeout is recorded in *status and
// raises the abort word so that every other CTA stops too.
__device__ __forceinline__ bool wait_flag_geq(const int* flag, int target, Control* ctl, int* status,
                                              uint64_t wait_ns) {
  if (ld_acquire(flag) >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (ld_acquire(flag) >= target) return true;
    if (ld_relaxed(&ctl->abort) != 0) return false;
    if (globaltimer_ns() - t0 > wait_ns) {
      atomicExch(status, kStatusTimeout);
      atomicExch(&ctl->abort, 1);
      return false;
    }
  }
}

// Band tile (I,J) of size B x B into shared memory, column-major (s[j*B + i]);
// out-of-band and out-of-matrix elements read as zero.  L2-only loads: the
// tile may have been written by another CTA of the same launch.
template <int B, int NT>
__device__ __forceinline__ void load_tile(const double* __restrict__ ab, long long ldab, int n, int k, int I,
                                          int J, double* s) {
  for (int idx = threadIdx.x; idx < B * B; idx += NT) {
    const int i = idx % B, j = idx / B;
    const int gi = I * B + i, gj = J * B + j;
    const int d = gi - gj;
    double v = 0.0;
    if (gi < n && gj < n && d >= 0 && d <= k) v = __ldcg(ab + d + (long long)gj * ldab);
    s[j * B + i] = v;
  }
}

// Element idx (column-major: i = idx % B, j = idx / B) of band tile (I,J), as load_tile reads it.
__device__ __forceinline__ double tile_elem(const double* __restrict__ ab, long long ldab, int n, int k, int I, int J,
                                            int idx, int B) {
  const int i = idx % B, j = idx / B;
  const int gi = I * B + i, gj = J * B + j;
  const int d = gi - gj;
  return (gi < n && gj < n && d >= 0 && d <= k) ? __ldcg(ab + d + (long long)gj * ldab) : 0.0;
}

// Two band tiles at once (every load of both is issued before any store).
template <int B, int NT>
__device__ __forceinline__ void load_tile2(const double* __restrict__ ab, long long ldab, int n, int k, int I1, int J1,
                                           double* s1, int I2, int J2, double* s2) {
  static_assert((B * B) % NT == 0, "whole passes");
  constexpr int E = B * B / NT;
  double v1[E], v2[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    v1[e] = tile_elem(ab, ldab, n, k, I1, J1, threadIdx.x + e * NT, B);
    v2[e] = tile_elem(ab, ldab, n, k, I2, J2, threadIdx.x + e * NT, B);
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    s1[threadIdx.x + e * NT] = v1[e];
    s2[threadIdx.x + e * NT] = v2[e];
  }
}

// Store the in-band, in-matrix elements of a column-major shared tile.
template <int B, int NT>
__device__ __forceinline__ void store_tile(double* __restrict__ ab, long long ldab, int n, int k, int I, int J,
                                           const double* s) {
  for (int idx = threadIdx.x; idx < B * B; idx += NT) {
    const int i = idx % B, j = idx / B;
    const int gi = I * B + i, gj = J * B + j;
    const int d = gi - gj;
    if (gi < n && gj < n && d >= 0 && d <= k) ab[d + (long long)gj * ldab] = s[j * B + i];
  }
}

}  // namespace bchol
