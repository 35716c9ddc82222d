// psolve.cu -- the banded triangular solves for small half-bandwidths as
// independent chunk solves plus a short sequential pass over chunk boundaries.
//
// bchol_solve (LAPACK pbtrs semantics; the use the paper's interior-point
// setting motivates, Sec. 1, Sec. 2) runs L Y = B, then L^T X = Y.  Row by row
// both sweeps are a chain of n dependent steps; the cluster solve (solve.cu)
// walks it in 32-row blocks, one ~2.3 us round per block, so at small k it
// spends most of its time waiting on the chain.  For small k this file cuts the
// rows into chunks of m = 256 rows, c = 0, 1, ..., and uses linearity:
//
//   forward, chunk c (rows R_c):   L_cc y_c = b_c - L_{c,c-1} t_{c-1},
//   where t_{c-1} is the last k entries of y_{c-1} (the band couples nothing
//   else), so y_c = u_c + G_c t_{c-1} with u_c = L_cc^{-1} b_c and the "spikes"
//   G_c = -L_cc^{-1} L_{c,c-1} (m x k).  With H_c, v_c the last k rows of G_c
//   and u_c,
//       t_c = v_c + H_c t_{c-1},  t_0 = v_0,
//   a recurrence of n/m steps of k x k products, and then y_c = u_c + G_c t_{c-1}
//   for every chunk at once.
//   backward: the same from the last chunk down, with L^T, the first k
//   entries of each chunk and s_c = v'_c + H'_c s_{c+1}.
//
// The spike pass keeps the previous k solution rows of each column in a ring
// in shared memory, initialised with the coupling block: spike column j starts
// from the unit vector e_j and a zero right-hand side, a right-hand-side
// column from zeros; it writes G_c and overwrites b_c with u_c.  The boundary
// recurrence runs on one CTA and stages each chunk's k x k block H_c by a bulk
// (TMA) copy two steps ahead.  Work: n (k + nrhs) k multiply-adds per sweep
// for the spikes, so this form pays off only for small k.
#include <algorithm>

#include "bchol_device.cuh"
#include "bchol_internal.h"

namespace bchol {

constexpr int kPM = 256;         // rows per chunk
constexpr int kPThreads = 256;
constexpr int kPLanes = 4;       // lanes that share one column's dot product
constexpr int kPMaxK = 112;      // largest half-bandwidth this solve takes
constexpr int kPRhs = 8;         // right-hand sides per pass

int psolve_max_k() { return kPMaxK; }

// Row stride of the spike blocks: k rounded up to even, so that every k-row
// block starts on a 16-byte boundary (bulk copies need it).
__host__ __device__ inline int pstride(int k) { return (k + 1) & ~1; }

struct PArgs {
  const double* ab;
  long long ldab;
  int n, k, C;          // C chunks
  double* b;            // n x nrhs, ldb; u_c after the spike pass, the solution after the last one
  long long ldb;
  int c0, nr;           // right-hand-side columns c0 .. c0+nr-1 of this pass
  double* G;            // per chunk kPM x pstride(k), row-major: the spikes G_c
  double* V;            // per chunk k x kPRhs: the coupling rows of u_c
  double* T;            // per chunk k x kPRhs: the boundary values t_c (forward) or s_c (backward)
  int* status;          // set to the timeout status if a bounded wait runs out
  uint64_t wait_ns;
};

__device__ __forceinline__ double lb(const PArgs& a, int i, int j) {  // L(i, j), i >= j, zero outside
  const int d = i - j;
  return (i < a.n && j >= 0 && d >= 0 && d <= a.k) ? __ldg(a.ab + d + (long long)j * a.ldab) : 0.0;
}

// Dynamic shared memory of the spike kernel: the ring of k + 1 solution rows
// of up to k + kPRhs columns.
size_t psolve_ring_bytes(int k) { return sizeof(double) * (size_t)(k + 1) * (k + kPRhs); }

// The spike pass of one chunk (all threads).  FWD: rows r0 .. r1-1 ascending
// with L; else descending with L^T.  A coupled chunk (every chunk but the
// first of the order) carries k spike columns before the right-hand sides;
// their rows go to G, the right-hand sides' solution u_c overwrites b, and the
// coupling rows of u_c (the last k forward, the first k backward) go to V.
template <bool FWD>
__global__ void __launch_bounds__(kPThreads) psolve_spike_kernel(PArgs a) {
  extern __shared__ __align__(16) double ring_raw[];  // solution rows, row r at slot r mod (k+1)
  __shared__ double lrow[2][kPMaxK];                   // L entries of the current and the next row
  __shared__ double rdiag[2];
  const int c = blockIdx.x, tid = threadIdx.x;
  const int k = a.k, K1 = k + 1, RW = k + kPRhs, ks = pstride(k);
  auto ring = [&](int slot) -> double* { return ring_raw + (size_t)slot * RW; };
  const int r0 = c * kPM, r1 = min(a.n, r0 + kPM), m = r1 - r0;
  const bool coupled = FWD ? (c > 0) : (c + 1 < a.C);
  const int ns = coupled ? k : 0;  // spike columns
  const int nc = ns + a.nr;
  double* Gc = a.G + (size_t)c * kPM * ks;
  // coupling block: rows r0-k .. r0-1 (forward) or r1 .. r1+k-1 (backward)
  for (int idx = tid; idx < k * nc; idx += kPThreads) {
    const int jj = idx % k, col = idx / k;
    const int row = FWD ? r0 - k + jj : r1 + jj;
    ring(((row % K1) + K1) % K1)[col] = (col < ns && jj == col) ? 1.0 : 0.0;
  }
  // coupling rows a short last chunk does not reach stay zero
  for (int idx = tid; idx < k * kPRhs; idx += kPThreads) a.V[(size_t)c * k * kPRhs + idx] = 0.0;
  // the L entries of row i: forward L(i, i-k+t), t < k; backward L(i+k-t, i), t < k.
  // Thread t < k fetches entry t and thread k the diagonal, two rows ahead in a
  // register, so that the global load's latency overlaps a row of the chain.
  auto fetch = [&](int i) -> double {
    const int ii = r0 + i;
    if (i < 0 || i >= m) return 1.0;
    if (tid < k) return FWD ? lb(a, ii, ii - k + tid) : lb(a, ii + k - tid, ii);
    if (tid == k) return lb(a, ii, ii);
    return 0.0;
  };
  auto put = [&](double v, int buf) {
    if (tid < k) lrow[buf][tid] = v;
    else if (tid == k) rdiag[buf] = 1.0 / v;
  };
  put(fetch(FWD ? 0 : m - 1), 0);
  double ahead = fetch(FWD ? 1 : m - 2);  // the row after the first
  __syncthreads();
  const int lane = tid & 31, part = lane % kPLanes;
  const int colw = (tid / 32) * (32 / kPLanes) + lane / kPLanes;  // column of this thread, pass 0
  constexpr int kColsPerPass = kPThreads / kPLanes;               // 64
  for (int step = 0; step < m; ++step) {
    const int i = FWD ? step : m - 1 - step;
    const int buf = step & 1;
    if (step + 1 < m) {
      put(ahead, buf ^ 1);
      ahead = fetch(FWD ? i + 2 : i - 2);
    }
    const int row = r0 + i;
    const int rslot = row % K1;
    // ring slot of the row of term t = part: row - k + part (forward), row + k - part
    // (backward), modulo k + 1; later terms step it by 4 (forward) or -4 (backward)
    const int slot0 = FWD ? ((row - k + part) % K1 + K1) % K1 : ((row + k - part) % K1 + K1) % K1;
    for (int col = colw; col - lane / kPLanes < nc; col += kColsPerPass) {
      double s0 = 0.0, s1 = 0.0;
      if (col < nc) {
        // terms t = part, part + 4, ...: rows row-k+t (forward) or row+k-t (backward)
        int t = part, sa = slot0;
        for (; t + kPLanes < k; t += 2 * kPLanes) {
          int sb = FWD ? sa + kPLanes : sa - kPLanes;  // k >= 5 here, so one wrap suffices
          if (FWD && sb >= K1) sb -= K1;
          if (!FWD && sb < 0) sb += K1;
          s0 = fma(lrow[buf][t], ring(sa)[col], s0);
          s1 = fma(lrow[buf][t + kPLanes], ring(sb)[col], s1);
          sa = FWD ? sb + kPLanes : sb - kPLanes;
          if (FWD && sa >= K1) sa -= K1;
          if (!FWD && sa < 0) sa += K1;
        }
        if (t < k) s0 = fma(lrow[buf][t], ring(sa)[col], s0);
      }
      double s = s0 + s1;
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (col < nc && part == 0) {
        double* bp = a.b + row + (long long)(a.c0 + col - ns) * a.ldb;
        const double rhs = (col < ns) ? 0.0 : *bp;
        const double y = (rhs - s) * rdiag[buf];
        ring(rslot)[col] = y;
        if (col < ns) {
          Gc[(size_t)i * ks + col] = y;
        } else {
          *bp = y;
          const int jj = FWD ? i - (m - k) : i;  // coupling rows of the chunk
          if (jj >= 0 && jj < k) a.V[((size_t)c * k + jj) * kPRhs + (col - ns)] = y;
        }
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ uint32_t psmem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t pnow() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Dynamic shared memory of the boundary kernel: two buffers of one chunk's
// H block (k x pstride(k)) and V block (k x kPRhs).
size_t psolve_boundary_bytes(int k) {
  return sizeof(double) * 2 * ((size_t)k * pstride(k) + (size_t)k * kPRhs);
}

// The boundary recurrence over the chunks (one CTA): forward t_c = v_c + H_c
// t_{c-1} from c = 0, backward s_c = v'_c + H'_c s_{c+1} from the last chunk;
// the first chunk of the order has no coupling (t = v).  H_c is a k-row block
// of G_c (its last k rows forward, first k backward), contiguous in memory;
// thread 0 stages it and V_c into shared memory by bulk copies two steps
// ahead (an mbarrier per buffer, bounded waits).  A last chunk shorter than k
// rows: forward its t is never used; backward it is the first of the order
// (no H), its missing V rows are zero, and the band entries that would use
// them are zero too.
template <bool FWD>
__global__ void __launch_bounds__(kPThreads) psolve_boundary_kernel(PArgs a) {
  extern __shared__ __align__(16) double bsm[];
  __shared__ double tcur[kPMaxK][kPRhs];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ int s_ok;
  const int k = a.k, tid = threadIdx.x, lane = tid & 31, ks = pstride(k);
  double* Hs[2] = {bsm, bsm + (size_t)k * ks};
  double* Vs[2] = {bsm + 2 * (size_t)k * ks, bsm + 2 * (size_t)k * ks + (size_t)k * kPRhs};
  const uint32_t hbytes = (uint32_t)(sizeof(double) * k * ks), vbytes = (uint32_t)(sizeof(double) * k * kPRhs);
  // G lanes share one output entry (jj, r) and its k-term dot product
  const int outs = k * a.nr;
  int G = 1;
  while (G < 32 && G * 2 * outs <= kPThreads) G *= 2;
  const int per_pass = kPThreads / G;
  const int g = lane % G;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(psmem(&mbar[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
  }
  __syncthreads();
  auto issue = [&](int q) {  // thread 0: the blocks of step q into buffer q & 1
    if (q >= a.C) return;
    const int c = FWD ? q : a.C - 1 - q, buf = q & 1;
    const int r0 = c * kPM, m = min(a.n, r0 + kPM) - r0;
    int hrow = FWD ? m - k : 0;
    if (hrow < 0) hrow = 0;  // a short last chunk (forward): its t is never used
    const double* h = a.G + ((size_t)c * kPM + hrow) * ks;
    const double* v = a.V + (size_t)c * k * kPRhs;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(psmem(&mbar[buf])),
                 "r"(hbytes + vbytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     psmem(Hs[buf])),
                 "l"(h), "r"(hbytes), "r"(psmem(&mbar[buf]))
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     psmem(Vs[buf])),
                 "l"(v), "r"(vbytes), "r"(psmem(&mbar[buf]))
                 : "memory");
  };
  auto wait = [&](int buf, uint32_t parity) -> bool {
    uint32_t ok = 0;
    const uint64_t t0 = pnow();
    while (true) {
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(psmem(&mbar[buf])), "r"(parity)
          : "memory");
      if (ok) return true;
      if (pnow() - t0 > a.wait_ns) return false;
    }
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  for (int q = 0; q < a.C; ++q) {
    const int c = FWD ? q : a.C - 1 - q;
    const int buf = q & 1;
    if (tid == 0 && !wait(buf, (q >> 1) & 1)) {
      atomicExch(a.status, kStatusTimeout);
      s_ok = 0;
    }
    __syncthreads();
    if (!s_ok) break;
    const double* h = Hs[buf];
    const double* v = Vs[buf];
    double out[(kPMaxK * kPRhs + 31) / 32];
    int np = 0;
    for (int base = 0; base < outs; base += per_pass, ++np) {
      const int idx = base + tid / G;
      double acc0 = 0.0, acc1 = 0.0;
      if (idx < outs && q > 0) {
        const int jj = idx % k, r = idx / k;
        int l = g;
        for (; l + G < k; l += 2 * G) {
          acc0 = fma(h[(size_t)jj * ks + l], tcur[l][r], acc0);
          acc1 = fma(h[(size_t)jj * ks + l + G], tcur[l + G][r], acc1);
        }
        if (l < k) acc0 = fma(h[(size_t)jj * ks + l], tcur[l][r], acc0);
      }
      double s = acc0 + acc1;
      for (int o = 1; o < G; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      out[np] = (idx < outs) ? s + v[(idx % k) * kPRhs + idx / k] : 0.0;
    }
    __syncthreads();  // every thread has read buffer buf and tcur
    np = 0;
    for (int base = 0; base < outs; base += per_pass, ++np) {
      const int idx = base + tid / G;
      if (idx < outs && g == 0) {
        const int jj = idx % k, r = idx / k;
        tcur[jj][r] = out[np];
        a.T[((size_t)c * k + jj) * kPRhs + r] = out[np];
      }
    }
    if (tid == 0) issue(q + 2);
    __syncthreads();  // tcur is complete
  }
  // a copy still in flight (after a timeout) lands before the CTA exits
  if (tid == 0 && !s_ok) {
    for (int b = 0; b < 2; ++b) wait(b, 0), wait(b, 1);
  }
}

// The coupled chunks' final values, all chunks at once: y_c = u_c + G_c t_{c-1}
// (forward) or x_c = u'_c + G'_c s_{c+1} (backward), in place in b.  One CTA
// per chunk, a thread per (row, right-hand side).
template <bool FWD>
__global__ void __launch_bounds__(kPThreads) psolve_apply_kernel(PArgs a) {
  __shared__ double tprev[kPMaxK][kPRhs];
  const int c = blockIdx.x, tid = threadIdx.x, k = a.k, ks = pstride(k);
  const bool coupled = FWD ? (c > 0) : (c + 1 < a.C);
  if (!coupled) return;
  const int nb = FWD ? c - 1 : c + 1;
  for (int idx = tid; idx < k * kPRhs; idx += kPThreads) (&tprev[0][0])[idx] = a.T[(size_t)nb * k * kPRhs + idx];
  __syncthreads();
  const int r0 = c * kPM, m = min(a.n, r0 + kPM) - r0;
  const double* Gc = a.G + (size_t)c * kPM * ks;
  for (int idx = tid; idx < m * a.nr; idx += kPThreads) {
    const int i = idx % m, r = idx / m;
    const double* grow = Gc + (size_t)i * ks;
    double s0 = 0.0, s1 = 0.0;
    int j = 0;
    for (; j + 1 < k; j += 2) {
      s0 = fma(grow[j], tprev[j][r], s0);
      s1 = fma(grow[j + 1], tprev[j + 1][r], s1);
    }
    if (j < k) s0 = fma(grow[j], tprev[j][r], s0);
    a.b[r0 + i + (long long)(a.c0 + r) * a.ldb] += s0 + s1;
  }
}

size_t psolve_workspace_bytes(int n, int k) {
  if (k > kPMaxK || n <= 0) return 0;
  const size_t C = (size_t)((n + kPM - 1) / kPM);
  return sizeof(double) * C * ((size_t)kPM * pstride(k) + 2 * (size_t)k * kPRhs);
}

// Both sweeps for nrhs columns, kPRhs at a time: per sweep the spike pass, the
// boundary recurrence and the final update.  Requires 1 <= k <= psolve_max_k()
// and n >= k + 1; ws holds psolve_workspace_bytes(n, k), 16-byte aligned.
cudaError_t launch_psolve(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb,
                          void* ws, int* status, uint64_t wait_ns, int* launches, cudaStream_t stream) {
  *launches = 0;
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (k > n - 1) k = n - 1;
  if (k < 1 || k > kPMaxK || !status) return cudaErrorInvalidValue;
  const int C = (n + kPM - 1) / kPM;
  PArgs a{};
  a.ab = ab;
  a.ldab = ldab;
  a.n = n;
  a.k = k;
  a.C = C;
  a.b = b;
  a.ldb = ldb;
  a.G = static_cast<double*>(ws);
  a.V = a.G + (size_t)C * kPM * pstride(k);
  a.T = a.V + (size_t)C * k * kPRhs;
  a.status = status;
  a.wait_ns = wait_ns;
  const size_t rb = psolve_ring_bytes(k), bb = psolve_boundary_bytes(k);
  cudaError_t e = cudaFuncSetAttribute(psolve_boundary_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bb);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(psolve_boundary_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bb);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(psolve_spike_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rb);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(psolve_spike_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rb);
  if (e != cudaSuccess) return e;
  for (int c0 = 0; c0 < nrhs; c0 += kPRhs) {
    a.c0 = c0;
    a.nr = std::min(kPRhs, nrhs - c0);
    psolve_spike_kernel<true><<<C, kPThreads, rb, stream>>>(a);
    psolve_boundary_kernel<true><<<1, kPThreads, bb, stream>>>(a);
    psolve_apply_kernel<true><<<C, kPThreads, 0, stream>>>(a);
    psolve_spike_kernel<false><<<C, kPThreads, rb, stream>>>(a);
    psolve_boundary_kernel<false><<<1, kPThreads, bb, stream>>>(a);
    psolve_apply_kernel<false><<<C, kPThreads, 0, stream>>>(a);
    *launches += 6;
  }
  return cudaGetLastError();
}

}  // namespace bchol
