// selinv.cu -- the adjoint of the band factor + solve: the band of
// Sigma = A^{-1} by selected inversion, and the gradient with respect to the
// stored band entries of A.
//
// The paper motivates the banded solver by interior-point optimisation
// (Sec. 1, Sec. 2), whose gradients need x = A^{-1} b and log det A to be
// differentiable.  For f(x, log det A) with xbar = df/dx and ldbar =
// df/dlogdet, bbar = A^{-1} xbar, the gradient with respect to a stored
// entry ab(i-j, j), which moves both A(i,j) and A(j,i), is
//     abar(i,j) = 2 ldbar Sigma(i,j) - (bbar_i x_j + bbar_j x_i)    (i > j)
//     abar(i,i) =   ldbar Sigma(i,i) -  bbar_i x_i.
// Only the band of Sigma is needed.  It follows from Sigma L = L^{-T} (the
// Takahashi recurrences), walked over b x b tiles from the last block column
// to the first; every quantity below stays inside the band.  For block column
// J with m = min(p, S-1-J) tiles below the diagonal:
//     P_IJ   = sum_{M=J+1..J+m} Sigma_IM L_MJ           (I = J+1..J+m)
//     Sigma_IJ = -P_IJ L_JJ^{-1}                         (back substitution on L_JJ)
//     E_J    = sum_{I=J+1..J+m} Sigma_IJ^T L_IJ          (lower triangle)
//     the diagonal tile, column by column from the right:
//       Sigma_ij = -(E_ij + sum_{l in tile, l>j} L_lj Sigma_il) / L_jj   (i > j)
//       Sigma_jj = (1/L_jj - E_jj - sum_{i in tile, i>j} L_ij Sigma_ij) / L_jj
// Tasks (a persistent launch with the factorization's ticket / ready-counter
// protocol):
//     FAR(I,J,g)  the terms M = J+2.. of P_IJ, in groups of kFarGroup (of one
//                 term for the row I = J+1, whose NEAR is on the chain: its
//                 terms then run side by side), each into its own partial
//                 tile (no chain between the groups).
//                 For I >= J+2 they read only block columns >= J+2, so they
//                 are ordered a column early; for I = J+1 they wait for
//                 column J+1.
//     NEAR(I,J)   P_IJ = Sigma_{I,J+1} L_{J+1,J} + the partials, Sigma_IJ, and
//                 its share Sigma_IJ^T L_IJ of E_J into a partial tile.
//     DIAG(J)     E_J = sum of the shares, then the diagonal tile.
// So one block column costs three dependent tasks (FAR of row J+1, NEAR,
// DIAG) instead of accumulation chains of m tasks.  Of these, NEAR(J+1,J) and
// DIAG(J) form the critical path from column to column (NEAR(J+1,J) reads
// DIAG(J+1)'s tile, DIAG(J) reads NEAR(J+1,J)'s share), so CTA 0 of the launch
// runs them itself, back to back, as the chain (no ticket claim and no flag
// hop between them), and the tickets carry the rest: per column
//     FAR(J+1, J, g), NEAR(J+2..J+m, J), then FAR(I, J-2, g) (the early far terms),
// with the chain's NEAR(J+1,J), DIAG(J) between the NEARs and the early far
// terms in the combined order (sel_combined).  Partial tiles live in a
// scratch ring of four block columns; a task of column J writes its slot only
// once DIAG(J+4) is done, which implies that every reader of the slot's
// previous contents (the NEAR tasks and DIAG of column J+4) has finished --
// the NEAR tasks of far rows of column J need not otherwise wait for it.
#include "../../include/bchol.h"
#include "factor_tasks.cuh"

namespace bchol {

constexpr int kFarGroup = 4;       // terms of P_IJ per FAR task
constexpr int kFarGroupNear = 4;   // the same for the row J+1

struct SelArgs {
  const double* L;   // factor band
  long long ldl;
  double* sig;       // output band: Sigma
  long long lds;
  int n, k, S, p;
  int ngmax;         // FAR groups per tile at m = p (rows below J+1)
  int rz;            // FAR partial slots of the row J+1 (one per term)
  long long cstride; // partial tiles per column slot: rz + (p - 1) ngmax
  unsigned long long total;
  int* flags;        // [tiles: Sigma final] [tiles: FAR partials done] [columns: E shares done]
  double* part;      // FAR partials: [4 columns][p rows][ngmax][b*b]
  double* wsh;       // E shares:     [4 columns][p rows][b*b]
  Control* ctl;
  int* status;
  uint64_t wait_ns;
  int chain;         // 1: CTA 0 runs NEAR(J+1,J) and DIAG(J) (the tickets omit them)
};

enum SelType { kFar = 0, kNear = 1, kDiag = 2 };

__host__ __device__ inline int sel_m(int S, int p, int J) { return (p < S - 1 - J) ? p : S - 1 - J; }
__host__ __device__ inline int sel_ng(int m) { return m >= 2 ? (m - 1 + kFarGroup - 1) / kFarGroup : 0; }
// FAR groups of tile row I = J+1+r of a column with m tiles: one term each for r = 0.
__host__ __device__ inline int sel_ngr(int m, int r) { return r == 0 ? (m >= 2 ? (m - 1 + kFarGroupNear - 1) / kFarGroupNear : 0) : sel_ng(m); }
__host__ __device__ inline int sel_gs(int r) { return r == 0 ? kFarGroupNear : kFarGroup; }

// Tickets of block column J, in processing order:
//   FAR(J+1, J, g) (g < ng(m_J)), NEAR(J+1..J+m_J, J), DIAG(J),
//   then FAR(I, J-2, g) for I = J..J-2+m_{J-2} (the early far terms of column J-2).
__host__ __device__ inline long long sel_bsize(int S, int p, int J, int chain = 0) {
  const int m = sel_m(S, p, J);
  long long sz = chain ? sel_ngr(m, 0) + (m >= 1 ? m - 1 : 0) : sel_ngr(m, 0) + m + 1;
  if (J >= 2) {
    const int m2 = sel_m(S, p, J - 2);
    if (m2 >= 2) sz += (long long)(m2 - 1) * sel_ng(m2);
  }
  return sz;
}

// Ticket -> (type, J, I, g).  Columns J = S-1 .. 0; the columns with m_J = p and
// m_{J-2} = p (2 <= J <= S-1-p) all have the same block size.
__host__ __device__ inline void sel_decode(int S, int p, long long t, int& type, int& J, int& I, int& g,
                                           int chain = 0) {
  J = S - 1;
  const int jreg_hi = S - 1 - p;  // regular columns: 2 .. jreg_hi
  while (J > jreg_hi && J >= 0) {  // head: m_J < p
    const long long bs = sel_bsize(S, p, J, chain);
    if (t < bs) break;
    t -= bs;
    --J;
  }
  if (J <= jreg_hi && J >= 2) {
    const long long breg = sel_bsize(S, p, jreg_hi, chain);
    const long long nreg = (long long)jreg_hi - 1;  // columns jreg_hi .. 2
    const long long d = t / breg;
    if (d < nreg) {
      J = jreg_hi - (int)d;
      t -= d * breg;
    } else {
      t -= nreg * breg;
      J = 1;
    }
  }
  while (J < 2 && J >= 0) {  // tail: columns 1 and 0 (when not in the head)
    const long long bs = sel_bsize(S, p, J, chain);
    if (t < bs) break;
    t -= bs;
    --J;
  }
  const int m = sel_m(S, p, J), ng = sel_ngr(m, 0);
  if (t < ng) {
    type = kFar;
    I = J + 1;
    g = (int)t;
    return;
  }
  t -= ng;
  const int nn = chain ? (m >= 1 ? m - 1 : 0) : m;   // the chain runs NEAR(J+1, J) itself
  if (t < nn) {
    type = kNear;
    I = J + 1 + (chain ? 1 : 0) + (int)t;
    g = 0;
    return;
  }
  t -= nn;
  if (!chain) {
    if (t == 0) {
      type = kDiag;
      I = J;
      g = 0;
      return;
    }
    t -= 1;
  }
  const int J2 = J - 2, ng2 = sel_ng(sel_m(S, p, J2));
  type = kFar;
  I = J2 + 2 + (int)(t / ng2);
  g = (int)(t % ng2);
  J = J2;
}

unsigned long long sel_total(int S, int p, int chain = 0) {
  unsigned long long t = 0;
  for (int J = S - 1; J >= 0; --J) t += (unsigned long long)sel_bsize(S, p, J, chain);
  return t;
}

__device__ __forceinline__ int sfidx(const SelArgs& a, int I, int J) { return J * (a.p + 1) + (I - J); }
__device__ __forceinline__ int* sig_flag(const SelArgs& a, int I, int J) { return &a.flags[sfidx(a, I, J)]; }
__device__ __forceinline__ int* far_flag(const SelArgs& a, int I, int J) {
  return &a.flags[a.S * (a.p + 1) + sfidx(a, I, J)];
}
__device__ __forceinline__ int* w_flag(const SelArgs& a, int J) { return &a.flags[2 * a.S * (a.p + 1) + J]; }

// Partial tiles of a column slot: the row J+1's rz, then ngmax per row below.
template <int B>
__device__ __forceinline__ double* part_tile(const SelArgs& a, int I, int J, int g) {
  const int r = I - J - 1;
  const long long t = (long long)(J & 3) * a.cstride + (r == 0 ? g : a.rz + (long long)(r - 1) * a.ngmax + g);
  return a.part + (size_t)t * B * B;
}
template <int B>
__device__ __forceinline__ double* w_tile(const SelArgs& a, int I, int J) {
  return a.wsh + (((size_t)(J & 3) * a.p + (I - J - 1)) * B * B);
}

// Band element (gi, gj), gi >= gj, of an array (zero outside the band/matrix).
__device__ __forceinline__ double bget(const double* x, long long ld, int n, int k, int gi, int gj, bool cg) {
  const int d = gi - gj;
  if (gi >= n || gj < 0 || d < 0 || d > k) return 0.0;
  return cg ? __ldcg(x + d + (long long)gj * ld) : __ldg(x + d + (long long)gj * ld);
}
// Symmetric access: Sigma(gi, gj) for any order of the indices.
__device__ __forceinline__ double sget(const SelArgs& a, int gi, int gj) {
  return gi >= gj ? bget(a.sig, a.lds, a.n, a.k, gi, gj, true) : bget(a.sig, a.lds, a.n, a.k, gj, gi, true);
}
__device__ __forceinline__ void sput(const SelArgs& a, int gi, int gj, double v) {
  const int d = gi - gj;
  if (gi < a.n && d >= 0 && d <= a.k) a.sig[d + (long long)gj * a.lds] = v;
}

// Release a counter after a CTA's stores: barrier, fence, one atomic add.
__device__ __forceinline__ void publish_add(int* counter) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1);
  }
}

// acc (R x R per thread: rows ty+16r, columns tx+16c) += X Y with X, Y staged as
// sX[l*B+i] = X(i, l), sY[l*B+j] = Y(l, j).
template <int B>
__device__ __forceinline__ void tile_mma(const double* sX, const double* sY, double (&acc)[B / 16][B / 16], int ty,
                                         int tx) {
  constexpr int R = B / 16;
#pragma unroll 4
  for (int l = 0; l < B; ++l) {
    double xv[R], yv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) xv[r] = sX[l * B + ty + 16 * r];
#pragma unroll
    for (int c = 0; c < R; ++c) yv[c] = sY[l * B + tx + 16 * c];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c) acc[r][c] = fma(xv[r], yv[c], acc[r][c]);
  }
}

// FAR(I,J,g): partial = sum over M in group g of Sigma_IM L_MJ.
template <int B>
__device__ bool sel_far(const SelArgs& a, int I, int J, int g, Smem<B>& sm, int* s_flag) {
  constexpr int R = B / 16;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int m = sel_m(a.S, a.p, J);
  const int gs = sel_gs(I - J - 1);
  const int mlo = J + 2 + g * gs, mhi = min(J + 1 + (g + 1) * gs, J + m);
  double acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = 0.0;
  double* sX = sm.t0;
  double* sY = sm.t1;
  for (int M = mlo; M <= mhi; ++M) {
    if (tid == 0) *s_flag = wait_flag_geq(sig_flag(a, max(I, M), min(I, M)), 1, a.ctl, a.status, a.wait_ns);
    __syncthreads();
    if (!*s_flag) return false;
    for (int idx = tid; idx < B * B; idx += kThreads) {
      const int i = idx % B, l = idx / B;
      sX[l * B + i] = sget(a, I * B + i, M * B + l);
      sY[l * B + i] = bget(a.L, a.ldl, a.n, a.k, M * B + l, J * B + i, false);   // (l, j = i)
    }
    __syncthreads();
    tile_mma<B>(sX, sY, acc, ty, tx);
    __syncthreads();
  }
  if (J + 4 < a.S) {  // the scratch slot's previous column is finished
    if (tid == 0) *s_flag = wait_flag_geq(sig_flag(a, J + 4, J + 4), 1, a.ctl, a.status, a.wait_ns);
    __syncthreads();
    if (!*s_flag) return false;
  }
  double* out = part_tile<B>(a, I, J, g);
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) out[(tx + 16 * c) * B + ty + 16 * r] = acc[r][c];
  publish_add(far_flag(a, I, J));
  return true;
}

// NEAR(I,J): Sigma_IJ = -(Sigma_{I,J+1} L_{J+1,J} + FAR partials) L_JJ^{-1}, then
// its share Sigma_IJ^T L_IJ (lower triangle) of E_J.
// CHAIN (the chain CTA's NEAR(J+1, J)): Sigma_{J+1,J+1} is the chain's own
// last DIAG, still in sm.t0 (as sS[l*B + i] = Sigma(i, l), both triangles), so
// it is neither waited for nor loaded; nor is the scratch slot's previous
// column (the chain's own DIAG(J+4)).
template <int B, bool CHAIN = false>
__device__ bool sel_near(const SelArgs& a, int I, int J, Smem<B>& sm, int* s_flag) {
  constexpr int R = B / 16;
  constexpr int TPR = kThreads / B;
  constexpr int RS = B / TPR;
  __shared__ double sP[B * B];
  __shared__ double s_rinv[B];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int m = sel_m(a.S, a.p, J), ng = sel_ngr(m, I - J - 1);
  // L_JJ, L_IJ and L_{J+1,J} (final: the factor is done) are read before the
  // waits, into registers, so that their loads overlap the waits and the first
  // product instead of following them
  constexpr int E = B * B / kThreads;
  double rjj[E], rij[E], rjn[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = tid + e * kThreads, l = idx % B, j = idx / B;
    rjj[e] = bget(a.L, a.ldl, a.n, a.k, J * B + l, J * B + j, false);        // -> sY[j*B + l]
    rij[e] = bget(a.L, a.ldl, a.n, a.k, I * B + l, J * B + j, false);        // -> sY[l*B + j]
    rjn[e] = bget(a.L, a.ldl, a.n, a.k, (J + 1) * B + j, J * B + l, false);  // L_{J+1,J}(j, l) -> sY[j*B + l]
  }
  if (tid == 0) {
    bool ok = wait_flag_geq(far_flag(a, I, J), ng, a.ctl, a.status, a.wait_ns);
    if (!CHAIN) {
      if (ok) ok = wait_flag_geq(sig_flag(a, I, J + 1), 1, a.ctl, a.status, a.wait_ns);
      // the share's scratch slot: its previous column is finished
      if (ok && J + 4 < a.S) ok = wait_flag_geq(sig_flag(a, J + 4, J + 4), 1, a.ctl, a.status, a.wait_ns);
    }
    *s_flag = ok;
  }
  __syncthreads();
  if (!*s_flag) return false;
  double* sX = sm.t0;
  double* sY = sm.t1;
#pragma unroll
  for (int e = 0; e < E; ++e) sY[tid + e * kThreads] = rjn[e];   // sY[l*B + i] = L_{J+1,J}(l, i)
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int i = idx % B, l = idx / B;
    if (CHAIN) {   // the band slots of DIAG(J+1)'s tile, as sget would read them
      const int d = i > l ? i - l : l - i;
      if (d > a.k) sX[l * B + i] = 0.0;
    } else {
      sX[l * B + i] = sget(a, I * B + i, (J + 1) * B + l);   // Sigma_{I,J+1} (symmetric when I = J+1)
    }
  }
  double acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int off = (tx + 16 * c) * B + ty + 16 * r;
      double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;   // the partials' loads issued four at a time
      int gg = 0;
      for (; gg + 3 < ng; gg += 4) {
        v0 += __ldcg(part_tile<B>(a, I, J, gg) + off);
        v1 += __ldcg(part_tile<B>(a, I, J, gg + 1) + off);
        v2 += __ldcg(part_tile<B>(a, I, J, gg + 2) + off);
        v3 += __ldcg(part_tile<B>(a, I, J, gg + 3) + off);
      }
      for (; gg < ng; ++gg) v0 += __ldcg(part_tile<B>(a, I, J, gg) + off);
      acc[r][c] = (v0 + v1) + (v2 + v3);
    }
  __syncthreads();
  tile_mma<B>(sX, sY, acc, ty, tx);
  // P -> shared memory (sP[j*B + i]); L_JJ -> sY (sY[j*B + l] = L(J*B+l, J*B+j))
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) sP[(tx + 16 * c) * B + ty + 16 * r] = acc[r][c];
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = tid + e * kThreads;
    sY[(idx / B) * B + idx % B] = rjj[e];
  }
  __syncthreads();
  // Sigma_IJ = -P L_JJ^{-1}, row by row: back substitution over the columns,
  // right to left, on the rows of L_JJ scaled by 1 / L_jj (no division or
  // scaling on the chain; the result is scaled at the end)
  const int jmax = min(B, a.n - J * B);
  if (tid < B) s_rinv[tid] = (tid < jmax) ? 1.0 / sY[tid * B + tid] : 0.0;
  __syncthreads();
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int j = idx % B, l = idx / B;
    if (j > l) sY[idx] *= s_rinv[j];   // sY[l*B + j] = L(j, l) / L(j, j)
  }
  const int i = tid / TPR, sub = tid % TPR;
  double sacc[RS];
#pragma unroll
  for (int qq = 0; qq < RS; ++qq) sacc[qq] = -sP[(sub + qq * TPR) * B + i];
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < B - 1; ++jj) {
    const int j = B - 1 - jj;
    const int owner = j % TPR, qj = j / TPR;
    const double z = __shfl_sync(0xffffffffu, sacc[qj], owner, TPR);
#pragma unroll
    for (int qq = 0; qq <= qj; ++qq) {
      const int l = sub + qq * TPR;
      if (l < j) sacc[qq] = fma(-z, sY[l * B + j], sacc[qq]);
    }
  }
#pragma unroll
  for (int qq = 0; qq < RS; ++qq) sacc[qq] *= s_rinv[sub + qq * TPR];
  __syncthreads();   // every warp is done with L_JJ in sY before it is overwritten below
  // store Sigma_IJ (band slots only) and keep the stored values (zero off the band) for the share
#pragma unroll
  for (int qq = 0; qq < RS; ++qq) {
    const int gi = I * B + i, gj = J * B + sub + qq * TPR, d = gi - gj;
    const bool in = gi < a.n && d >= 0 && d <= a.k;
    if (in) a.sig[d + (long long)gj * a.lds] = sacc[qq];
    sX[i * B + sub + qq * TPR] = in ? sacc[qq] : 0.0;   // sX[l*B + c] = Sigma_IJ(l, c)
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = tid + e * kThreads;
    sY[(idx % B) * B + idx / B] = rij[e];   // sY[l*B + j] = L_IJ(l, j)
  }
  __syncthreads();
  // share(c, j) = sum_l Sigma_IJ(l, c) L_IJ(l, j), lower triangle c >= j
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = 0.0;
  tile_mma<B>(sX, sY, acc, ty, tx);
  double* out = w_tile<B>(a, I, J);
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) out[(tx + 16 * c) * B + ty + 16 * r] = (ty + 16 * r >= tx + 16 * c) ? acc[r][c] : 0.0;
  __syncthreads();
  if (tid == 0) {
    __threadfence();   // then both counters (the release pattern, one fence)
    st_relaxed(sig_flag(a, I, J), 1);
    atomicAdd(w_flag(a, J), 1);
  }
  return true;
}

// DIAG(J): E_J from the shares, then the diagonal tile by the scalar recurrence,
// columns from right to left.  sS holds Sigma of the tile (full square, both
// triangles); sE holds E_J; sL the factor tile.
template <int B>
__device__ bool sel_diag(const SelArgs& a, int J, Smem<B>& sm, int* s_flag) {
  __shared__ double sE[B * B];
  __shared__ double s_rl[B];
  const int tid = threadIdx.x;
  const int m = sel_m(a.S, a.p, J);
  // L_JJ (final: the factor is done) is read before the wait for the shares
  constexpr int E = (B * B + kThreads - 1) / kThreads;
  double lj[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = tid + e * kThreads;
    lj[e] = idx < B * B ? bget(a.L, a.ldl, a.n, a.k, J * B + idx % B, J * B + idx / B, false) : 0.0;
  }
  if (tid == 0) *s_flag = wait_flag_geq(w_flag(a, J), m, a.ctl, a.status, a.wait_ns);
  __syncthreads();
  if (!*s_flag) return false;
  double* sS = sm.t0;   // sS[j*B + i] = Sigma(i, j), symmetric
  double* sL = sm.t1;   // sL[j*B + i] = L(i, j)
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int idx = tid + e * kThreads;
    if (idx < B * B) sL[idx] = lj[e];
  }
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int i = idx % B, j = idx / B;
    double e0 = 0.0, e1 = 0.0, e2 = 0.0, e3 = 0.0;   // the shares' loads issued four at a time
    if (i >= j) {
      int ii = J + 1;
      for (; ii + 3 <= J + m; ii += 4) {
        e0 += __ldcg(w_tile<B>(a, ii, J) + idx);
        e1 += __ldcg(w_tile<B>(a, ii + 1, J) + idx);
        e2 += __ldcg(w_tile<B>(a, ii + 2, J) + idx);
        e3 += __ldcg(w_tile<B>(a, ii + 3, J) + idx);
      }
      for (; ii <= J + m; ++ii) e0 += __ldcg(w_tile<B>(a, ii, J) + idx);
    }
    sE[j * B + i] = (e0 + e1) + (e2 + e3);
    sS[j * B + i] = 0.0;
  }
  __syncthreads();
  const int jmax = min(B, a.n - J * B);
  if (tid < B) s_rl[tid] = (tid < jmax) ? 1.0 / sL[tid * B + tid] : 0.0;   // every reciprocal at once
  __syncthreads();
  // The recurrence is warp 0's alone, so warp barriers order it; the other
  // warps wait at the block barrier below.  Tiles of 16: row i = lane % 16,
  // and the two half-warps take alternate terms of each row's dot product
  // (half the FP64 instructions: GB300 issues one per 64 cycles per
  // sub-partition whatever the active lanes), fully unrolled so that the
  // shared-memory operands load ahead of the FMAs.  Larger tiles: rows
  // i = lane, lane + 32, ...
  if constexpr (B == 16) {
    if (tid < 32) {
      const int lane = tid, i = lane & 15, h = lane >> 4;
#pragma unroll
      for (int j = B - 1; j >= 0; --j) {
        if (j < jmax) {
          const double rl = s_rl[j];
          double sp = 0.0;
#pragma unroll
          for (int mm = j + 1 + h; mm < B; mm += 2) sp = fma(sL[j * B + mm], sS[mm * B + i], sp);   // L(mm,j) Sigma(i,mm)
          sp += __shfl_xor_sync(0xffffffffu, sp, 16);
          double part = 0.0;
          if (i > j && i < jmax) {   // Sigma_ij for i > j
            const double v = -(sE[j * B + i] + sp) * rl;
            if (h == 0) {
              sS[j * B + i] = v;
              sS[i * B + j] = v;   // symmetric copy (row j)
              part = sL[j * B + i] * v;   // L(i,j) Sigma(i,j)
            }
          }
#pragma unroll
          for (int off = 8; off >= 1; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
          if (lane == 0) sS[j * B + j] = (rl - (sE[j * B + j] + part)) * rl;
          __syncwarp();
        }
      }
    }
  } else if (tid < 32) {
    const int lane = tid;
    for (int j = jmax - 1; j >= 0; --j) {
      const double rl = s_rl[j];
      double part = 0.0;
      for (int i = lane; i < jmax; i += 32) {
        if (i > j) {   // Sigma_ij for i > j
          double s = sE[j * B + i];
          for (int mm = j + 1; mm < jmax; ++mm) s = fma(sL[j * B + mm], sS[mm * B + i], s);   // L(mm,j) Sigma(i,mm)
          const double v = -s * rl;
          sS[j * B + i] = v;
          part = fma(sL[j * B + i], v, part);   // L(i,j) Sigma(i,j)
        }
      }
#pragma unroll
      for (int off = (B < 32 ? B : 32) / 2; off >= 1; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
      if (lane == 0) sS[j * B + j] = (rl - (sE[j * B + j] + part)) * rl;
      for (int i = lane; i < jmax; i += 32)
        if (i > j) sS[i * B + j] = sS[j * B + i];   // symmetric copy (row j)
      __syncwarp();
    }
  }
  __syncthreads();
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int i = idx % B, j = idx / B;
    if (i >= j && i < jmax) sput(a, J * B + i, J * B + j, sS[j * B + i]);
  }
  publish(sig_flag(a, J, J), 1);
  return true;
}

template <int B>
__global__ void __launch_bounds__(kThreads, 2) selinv_kernel(SelArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<B>& sm = *reinterpret_cast<Smem<B>*>(smem_raw);
  __shared__ long long s_task;
  __shared__ int s_flag;
  if (a.chain) {
    if (blockIdx.x == 0) {   // the chain: NEAR(J+1, J) and DIAG(J), column by column from the last
      if (threadIdx.x == 0) st_release(&a.ctl->chain_sm, sm_id() + 1);
      for (int J = a.S - 1; J >= 0; --J) {
        if (sel_m(a.S, a.p, J) >= 1 && !sel_near<B, true>(a, J + 1, J, sm, &s_flag)) return;
        if (!sel_diag<B>(a, J, sm, &s_flag)) return;
      }
      return;
    }
    // A ticket CTA on the chain's SM leaves: the chain's FP64 work is the
    // critical path and the SM's FP64 units are shared.  (All CTAs are
    // resident at once, so the chain publishes its SM promptly; the wait is
    // bounded and a CTA that gives up simply stays.)
    if (threadIdx.x == 0) {
      const uint64_t t0 = globaltimer_ns();
      int c = ld_acquire(&a.ctl->chain_sm);
      while (c == 0 && globaltimer_ns() - t0 < 200000ull) c = ld_acquire(&a.ctl->chain_sm);
      s_flag = (c == sm_id() + 1);
    }
    __syncthreads();
    if (s_flag) return;
  }
  unsigned long long next = 0;
  if (threadIdx.x == 0) next = atomicAdd(&a.ctl->ticket, 1ULL);
  while (true) {
    if (threadIdx.x == 0) s_task = (long long)next;
    __syncthreads();
    const long long t = s_task;
    if (t >= (long long)a.total) break;
    if (threadIdx.x == 0) next = atomicAdd(&a.ctl->ticket, 1ULL);
    int type, J, I, g;
    sel_decode(a.S, a.p, t, type, J, I, g, a.chain);
    bool ok;
    if (type == kFar)
      ok = sel_far<B>(a, I, J, g, sm, &s_flag);
    else if (type == kNear)
      ok = sel_near<B>(a, I, J, sm, &s_flag);
    else
      ok = sel_diag<B>(a, J, sm, &s_flag);
    if (!ok) break;
  }
}

// abar from Sigma in place: 2 ldbar Sigma_ij - (bbar_i x_j + bbar_j x_i) off the diagonal,
// ldbar Sigma_ii - bbar_i x_i on it (bbar, x may be null: then only the log det part).
__global__ void grad_from_sigma_kernel(double* __restrict__ g, long long ldg, int n, int k, const double* __restrict__ x,
                                       const double* __restrict__ bbar, double ldbar) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)(k + 1) * n) return;
  const int j = (int)(idx / (k + 1)), d = (int)(idx % (k + 1));
  const int i = j + d;
  if (i >= n) return;
  double* p = g + d + (long long)j * ldg;
  const double sig = *p;
  double v;
  if (d == 0) {
    v = ldbar * sig - ((x && bbar) ? bbar[i] * x[i] : 0.0);
  } else {
    v = 2.0 * ldbar * sig - ((x && bbar) ? (bbar[i] * x[j] + bbar[j] * x[i]) : 0.0);
  }
  *p = v;
}

// Zero the matrix slots of a band array (slots outside the matrix are left alone).
__global__ void zero_band_kernel(double* __restrict__ g, long long ldg, int n, int k) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)(k + 1) * n) return;
  const int j = (int)(idx / (k + 1)), d = (int)(idx % (k + 1));
  if (j + d < n) g[d + (long long)j * ldg] = 0.0;
}

// log det A = 2 sum_i log L_ii (one block, tree reduction).
__global__ void __launch_bounds__(1024) logdet_kernel(const double* __restrict__ ab, long long ldab, int n,
                                                      double* __restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) s += log(ab[(long long)i * ldab]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 2.0 * red[0];
}

static int sel_ngmax(int p) { return p >= 2 ? (p - 1 + kFarGroup - 1) / kFarGroup : 1; }
static int sel_rz(int p) { return p >= 2 ? (p - 1 + kFarGroupNear - 1) / kFarGroupNear : 1; }
static long long sel_cstride(int p) { return sel_rz(p) + (long long)(p - 1) * sel_ngmax(p); }

// control block | flags (2 S (p+1) + S ints, rounded to 256 B) | FAR partials | E shares
static size_t sel_flag_bytes(int S, int p) {
  const size_t f = sizeof(int) * ((size_t)2 * S * (p + 1) + S);
  return (f + 255) / 256 * 256;
}

size_t selinv_workspace_bytes(int n, int k, int b) {
  const int S = (n + b - 1) / b;
  int p = (k + b - 1) / b;
  if (p > S - 1) p = S - 1;
  if (p < 1) p = 1;
  const size_t tile = sizeof(double) * (size_t)b * b;
  return 256 + sel_flag_bytes(S, p) + (size_t)4 * sel_cstride(p) * tile + (size_t)4 * p * tile;
}

template <int B>
static cudaError_t launch_sel_b(const SelArgs& a, int ctas_per_sm, cudaStream_t st) {
  const size_t smem = sizeof(Smem<B>);
  cudaError_t e = cudaFuncSetAttribute(selinv_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, selinv_kernel<B>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  long long grid = (long long)per_sm * num_sms();
  const unsigned long long need = a.total + (a.chain ? 1 : 0);   // tickets (+ the chain CTA)
  if ((unsigned long long)grid > need) grid = (long long)need;
  if (grid < 1) grid = 1;
  selinv_kernel<B><<<(unsigned)grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

// Band of Sigma = A^{-1} into `sig` (ld lds) from the factor in L; then the gradient transform.
cudaError_t launch_backward(int n, int k, int b, const double* L, long long ldl, const double* x, const double* bbar,
                            double ldbar, double* g, long long ldg, void* ws, int* status, uint64_t wait_ns,
                            int ctas_per_sm, cudaStream_t st) {
  const int S = (n + b - 1) / b;
  int p = (k + b - 1) / b;
  if (p > S - 1) p = S - 1;
  const int pw = p < 1 ? 1 : p;   // scratch sizing (p = 0 has no off-diagonal tiles)
  cudaError_t e = cudaMemsetAsync(ws, 0, 256 + sel_flag_bytes(S, pw), st);   // control + flags (not the scratch)
  if (e != cudaSuccess) return e;
  const long long nb0 = (long long)(k + 1) * n;
  zero_band_kernel<<<(unsigned)((nb0 + 255) / 256), 256, 0, st>>>(g, ldg, n, k);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  SelArgs a;
  a.L = L;
  a.ldl = ldl;
  a.sig = g;
  a.lds = ldg;
  a.n = n;
  a.k = k;
  a.S = S;
  a.p = p;
  a.chain = 1;
  a.total = sel_total(S, p, a.chain);
  a.ngmax = sel_ngmax(pw);
  a.rz = sel_rz(pw);
  a.cstride = sel_cstride(pw);
  a.ctl = reinterpret_cast<Control*>(ws);
  a.flags = reinterpret_cast<int*>(static_cast<char*>(ws) + 256);
  a.part = reinterpret_cast<double*>(static_cast<char*>(ws) + 256 + sel_flag_bytes(S, pw));
  a.wsh = a.part + (size_t)4 * a.cstride * b * b;
  a.status = status;
  a.wait_ns = wait_ns;
  switch (b) {
    case 16: e = launch_sel_b<16>(a, ctas_per_sm, st); break;
    case 32: e = launch_sel_b<32>(a, ctas_per_sm, st); break;
    default: e = launch_sel_b<64>(a, ctas_per_sm, st); break;
  }
  if (e != cudaSuccess) return e;
  const long long nb = (long long)(k + 1) * n;
  grad_from_sigma_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(g, ldg, n, k, x, bbar, ldbar);
  return cudaGetLastError();
}

// The combined order of the launch (host side, for tests): the tickets, with
// the chain's NEAR(J+1, J) and DIAG(J) placed after column J's NEAR tickets
// and before its early far terms, FAR(I, J-2, g) (which read Sigma_JJ).
// Every task comes after the tasks it reads, so a CTA (the chain included)
// only ever waits for tasks that are running or done.
static void sel_combined(int S, int p, long long t, int& type, int& J, int& I, int& g) {
  long long base = 0;
  for (int c = S - 1; c >= 0; --c) {
    const int m = sel_m(S, p, c);
    const long long head = sel_ngr(m, 0) + (m >= 1 ? m - 1 : 0);   // FAR(c+1, c, .), NEAR(c+2.., c)
    const long long nchain = (m >= 1 ? 1 : 0) + 1;
    const long long tail = sel_bsize(S, p, c, 1) - head;        // early far terms of column c-2
    if (t < head) {
      sel_decode(S, p, base + t, type, J, I, g, 1);
      return;
    }
    t -= head;
    if (t < nchain) {
      J = c;
      g = 0;
      if (m >= 1 && t == 0) {
        type = kNear;
        I = c + 1;
      } else {
        type = kDiag;
        I = c;
      }
      return;
    }
    t -= nchain;
    if (t < tail) {
      sel_decode(S, p, base + head + t, type, J, I, g, 1);
      return;
    }
    t -= tail;
    base += head + tail;
  }
  type = -1;
  J = I = g = -1;
}

long long adjoint_plan_count(int n, int k, int b) {
  const int S = (n + b - 1) / b;
  int p = (k + b - 1) / b;
  if (p > S - 1) p = S - 1;
  if (n <= 0) return 0;
  return (long long)sel_total(S, p, 1) + 2LL * S - (p >= 1 ? 1 : S);   // tickets + NEAR(J+1,J) + DIAG(J)
}

void adjoint_plan_task(int n, int k, int b, long long t, int* type, int* J, int* I, int* g) {
  const int S = (n + b - 1) / b;
  int p = (k + b - 1) / b;
  if (p > S - 1) p = S - 1;
  sel_combined(S, p, t, *type, *J, *I, *g);
}

cudaError_t launch_logdet(const double* ab, long long ldab, int n, double* out, cudaStream_t st) {
  logdet_kernel<<<1, 1024, 0, st>>>(ab, ldab, n, out);
  return cudaGetLastError();
}

}  // namespace bchol
