// strip_task.cuh -- the trailing update of the FP64_SPLIT factorization:
// STRIP(I0, J, s) applies UPD(I, J, s), A_IJ -= L_Is L_Js^T (Algorithm 1), to
// the h tiles I = I0 .. I0+h-1 of block column J (tiles of b = 16 or 32,
// h <= 128 / b) as one split product on the tensor cores (split_update.cuh):
// the h panel tiles L_Is are the b h rows of A, L_Js the b rows of B and the
// strip of A_IJ is C.  The
// ready-counter protocol is the per-tile one of factor.cu: the strip waits for
// each tile's previous update and its panel tiles, and releases each tile's
// counter after its stores.
#pragma once
#include "factor_tasks.cuh"
#include "split_update.cuh"

namespace bchol {

template <int B>
__device__ bool task_strip(const FactorArgs& a, int I0, int J, int s, split::Smem<B>& sm, split::Ctx& cx,
                           int* s_flag) {
  const int ms = min(a.p, a.S - 1 - s);
  const int h = strip_rows(a.H, s, ms, I0);
  if (threadIdx.x == 0) {
    // every tile's panel tile and previous update, and L_Js (one of the strip's own
    // panel tiles when the strip starts on the diagonal), read together
    constexpr int N = 2 * (split::kRowsA / B) + 1;
    int f[N], tg[N], cnt = 0;
#pragma unroll
    for (int t = 0; t < split::kRowsA / B; ++t) {
      if (t < h) {
        const int I = I0 + t, s0 = first_step(a, I);
        f[cnt] = fidx(a, I, s);
        tg[cnt++] = s - s0 + 1;
        f[cnt] = fidx(a, I, J);
        tg[cnt++] = s - s0;
      }
    }
    if (!(J >= I0 && J < I0 + h)) {
      f[cnt] = fidx(a, J, s);
      tg[cnt++] = s - first_step(a, J) + 1;
    }
    *s_flag = wait_tiles(a, f, tg, cnt);
  }
  __syncthreads();
  if (!*s_flag) return false;
  const int rows = B * h;
  auto band = [&](int gi, int gj) -> double {
    const int d = gi - gj;
    return (gi < a.n && d >= 0 && d <= a.k) ? __ldcg(a.ab + d + (long long)gj * a.ldab) : 0.0;
  };
  auto la = [&](int r, int k) { return r < rows ? band(I0 * B + r, s * B + k) : 0.0; };
  auto lb = [&](int j, int k) { return band(J * B + j, s * B + k); };
  auto ldc = [&](int r, int j) { return r < rows ? band(I0 * B + r, J * B + j) : 0.0; };
  auto stc = [&](int r, int j, double v) {
    const int gi = I0 * B + r, gj = J * B + j, d = gi - gj;
    if (r < rows && gi < a.n && d >= 0 && d <= a.k) a.ab[d + (long long)gj * a.ldab] = v;
  };
  if (!split::product<B>(sm, cx, la, lb, ldc, stc, a.wait_ns, a.status, &a.ctl->abort)) return false;
  __syncthreads();
  if (threadIdx.x == 0) {   // one fence, then the tiles' counters (the release pattern)
    __threadfence();
    for (int t = 0; t < h; ++t) {
      const int I = I0 + t;
      st_relaxed(&a.flags[fidx(a, I, J)], s - first_step(a, I) + 1);
    }
  }
  return true;
}

}  // namespace bchol
