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
// to the first; every quantity below stays inside the band:
//     SACC(I,J,M)  P_IJ += Sigma_IM L_MJ          (M = J+m .. J+1, descending)
//     SFIN(I,J)    Sigma_IJ = -P_IJ L_JJ^{-1}      (back substitution on L_JJ)
//     DACC(J,M)    E_J  += Sigma_MJ^T L_MJ         (lower triangle, M descending)
//     DFIN(J)      the diagonal tile, column by column from the right:
//                  Sigma_ij = -(E_ij + sum_{m in tile, m>j} L_mj Sigma_im) / L_jj   (i > j)
//                  Sigma_jj = (1/L_jj - E_jj - sum_{i in tile, i>j} L_ij Sigma_ij) / L_jj
// P_IJ and E_J accumulate in the output band array itself (its tile slots),
// so no extra storage is needed.  The walk is a persistent kernel with the
// same ticket / ready-counter protocol as the factorization.
#include "../../include/bchol.h"
#include "factor_tasks.cuh"

namespace bchol {

struct SelArgs {
  const double* L;   // factor band
  long long ldl;
  double* sig;       // output band: Sigma (accumulators first)
  long long lds;
  int n, k, S, p;
  unsigned long long total;
  int* flags;
  Control* ctl;
  int* status;
  uint64_t wait_ns;
};

enum SelType { kSacc = 0, kSfin = 1, kDacc = 2, kDfin = 3 };

__host__ __device__ inline int sel_m(int S, int p, int J) { return (p < S - 1 - J) ? p : S - 1 - J; }

// Ticket -> task.  Block column J = S-1, S-2, ..., 0 has m = sel_m(J) and
// (m+1)^2 tasks: m*m SACC (M-major, M descending), m SFIN, m DACC, 1 DFIN.
__host__ __device__ inline void sel_decode(int S, int p, long long t, int& type, int& J, int& I, int& M) {
  int jb = 0;
  const int head = (p < S) ? p : S;   // leading blocks with m = jb < p
  long long r = t;
  while (jb < head) {
    const long long sz = (long long)(jb + 1) * (jb + 1);
    if (r < sz) break;
    r -= sz;
    ++jb;
  }
  if (jb == head) {
    const long long sz = (long long)(p + 1) * (p + 1);
    jb += (int)(r / sz);
    r %= sz;
  }
  J = S - 1 - jb;
  const int m = sel_m(S, p, J);
  if (r < (long long)m * m) {
    type = kSacc;
    const int q = (int)(r / m);
    M = J + m - q;
    I = J + 1 + (int)(r % m);
    return;
  }
  r -= (long long)m * m;
  if (r < m) {
    type = kSfin;
    I = J + 1 + (int)r;
    M = 0;
    return;
  }
  r -= m;
  if (r < m) {
    type = kDacc;
    M = J + m - (int)r;
    I = J;
    return;
  }
  type = kDfin;
  I = J;
  M = 0;
}

unsigned long long sel_total(int S, int p) {
  unsigned long long t = 0;
  for (int J = S - 1; J >= 0; --J) {
    const unsigned long long m = (unsigned long long)sel_m(S, p, J);
    t += (m + 1) * (m + 1);
  }
  return t;
}

__device__ __forceinline__ int sfidx(const SelArgs& a, int I, int J) { return J * (a.p + 1) + (I - J); }

__device__ __forceinline__ bool sel_wait(const SelArgs& a, int I, int J, int target) {
  return wait_flag_geq(&a.flags[sfidx(a, I, J)], target, a.ctl, a.status, a.wait_ns);
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

// SACC(I,J,M): P_IJ += Sigma_IM L_MJ.  sX[l*B+i] = Sigma(I*B+i, M*B+l), sY[l*B+j] = L(M*B+l, J*B+j).
template <int B>
__device__ bool sel_sacc(const SelArgs& a, int I, int J, int M, Smem<B>& sm, int* s_flag) {
  constexpr int R = B / 16;
  const int tid = threadIdx.x;
  const int m = sel_m(a.S, a.p, J);
  const int q = J + m - M;   // position of M in the descending order
  if (tid == 0) {
    const int hi = I > M ? I : M, lo = I > M ? M : I;
    bool ok = sel_wait(a, hi, lo, sel_m(a.S, a.p, lo) + 1);
    if (ok) ok = sel_wait(a, I, J, q);
    *s_flag = ok;
  }
  __syncthreads();
  if (!*s_flag) return false;
  double* sX = sm.t0;
  double* sY = sm.t1;
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int i = idx % B, l = idx / B;
    sX[l * B + i] = sget(a, I * B + i, M * B + l);
    sY[l * B + i] = bget(a.L, a.ldl, a.n, a.k, M * B + l, J * B + i, false);   // (l, j = i)
  }
  const int ty = tid / 16, tx = tid % 16;
  double acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = bget(a.sig, a.lds, a.n, a.k, I * B + ty + 16 * r, J * B + tx + 16 * c, true);
  __syncthreads();
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
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) sput(a, I * B + ty + 16 * r, J * B + tx + 16 * c, acc[r][c]);
  publish(&a.flags[sfidx(a, I, J)], q + 1);
  return true;
}

// SFIN(I,J): Sigma_IJ = -P_IJ L_JJ^{-1}, row by row (back substitution over columns, right to left).
template <int B>
__device__ bool sel_sfin(const SelArgs& a, int I, int J, Smem<B>& sm, int* s_flag) {
  constexpr int TPR = kThreads / B;
  constexpr int R = B / TPR;
  __shared__ double s_rinv[B];
  const int tid = threadIdx.x;
  const int m = sel_m(a.S, a.p, J);
  if (tid == 0) *s_flag = sel_wait(a, I, J, m);
  __syncthreads();
  if (!*s_flag) return false;
  double* sL = sm.t1;   // sL[j*B + l] = L(J*B+l, J*B+j)
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int l = idx % B, j = idx / B;
    sL[j * B + l] = bget(a.L, a.ldl, a.n, a.k, J * B + l, J * B + j, false);
  }
  __syncthreads();
  const int jmax = min(B, a.n - J * B);
  if (tid < B) s_rinv[tid] = (tid < jmax) ? 1.0 / sL[tid * B + tid] : 0.0;
  const int i = tid / TPR, sub = tid % TPR;
  double acc[R];
#pragma unroll
  for (int qq = 0; qq < R; ++qq) acc[qq] = -bget(a.sig, a.lds, a.n, a.k, I * B + i, J * B + sub + qq * TPR, true);
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < B; ++jj) {
    const int j = B - 1 - jj;
    const int owner = j % TPR, qj = j / TPR;
    double x = 0.0;
    if (sub == owner) {
      x = acc[qj] * s_rinv[j];
      acc[qj] = x;
    }
    x = __shfl_sync(0xffffffffu, x, owner, TPR);
#pragma unroll
    for (int qq = 0; qq <= qj; ++qq) {
      const int l = sub + qq * TPR;
      if (l < j) acc[qq] = fma(-x, sL[l * B + j], acc[qq]);   // L(j, l)
    }
  }
#pragma unroll
  for (int qq = 0; qq < R; ++qq) sput(a, I * B + i, J * B + sub + qq * TPR, acc[qq]);
  publish(&a.flags[sfidx(a, I, J)], m + 1);
  return true;
}

// DACC(J,M): E_J += Sigma_MJ^T L_MJ (lower triangle).  sX[l*B+i] = Sigma(M*B+l, J*B+i), sY[l*B+j] = L(M*B+l, J*B+j).
template <int B>
__device__ bool sel_dacc(const SelArgs& a, int J, int M, Smem<B>& sm, int* s_flag) {
  constexpr int R = B / 16;
  const int tid = threadIdx.x;
  const int m = sel_m(a.S, a.p, J);
  const int q = J + m - M;
  if (tid == 0) {
    bool ok = sel_wait(a, M, J, m + 1);
    if (ok) ok = sel_wait(a, J, J, q);
    *s_flag = ok;
  }
  __syncthreads();
  if (!*s_flag) return false;
  double* sX = sm.t0;
  double* sY = sm.t1;
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int i = idx % B, l = idx / B;
    sX[l * B + i] = bget(a.sig, a.lds, a.n, a.k, M * B + l, J * B + i, true);
    sY[l * B + i] = bget(a.L, a.ldl, a.n, a.k, M * B + l, J * B + i, false);
  }
  const int ty = tid / 16, tx = tid % 16;
  double acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = bget(a.sig, a.lds, a.n, a.k, J * B + ty + 16 * r, J * B + tx + 16 * c, true);
  __syncthreads();
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
      for (int c = 0; c < R; ++c)
        if (r >= c) acc[r][c] = fma(xv[r], yv[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) sput(a, J * B + ty + 16 * r, J * B + tx + 16 * c, acc[r][c]);
  publish(&a.flags[sfidx(a, J, J)], q + 1);
  return true;
}

// DFIN(J): the diagonal tile by the scalar recurrence, columns from right to left.
// sS holds Sigma of the tile (full square, both triangles); sE holds E_J; sL the factor tile.
template <int B>
__device__ bool sel_dfin(const SelArgs& a, int J, Smem<B>& sm, int* s_flag) {
  __shared__ double sE[B * B];
  __shared__ double s_part[B];
  const int tid = threadIdx.x;
  const int m = sel_m(a.S, a.p, J);
  if (tid == 0) *s_flag = sel_wait(a, J, J, m);
  __syncthreads();
  if (!*s_flag) return false;
  double* sS = sm.t0;   // sS[j*B + i] = Sigma(i, j), symmetric
  double* sL = sm.t1;   // sL[j*B + i] = L(i, j)
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int i = idx % B, j = idx / B;
    sL[j * B + i] = bget(a.L, a.ldl, a.n, a.k, J * B + i, J * B + j, false);
    sE[j * B + i] = (i >= j) ? bget(a.sig, a.lds, a.n, a.k, J * B + i, J * B + j, true) : 0.0;
    sS[j * B + i] = 0.0;
  }
  __syncthreads();
  const int jmax = min(B, a.n - J * B);
  for (int j = jmax - 1; j >= 0; --j) {
    const double rl = 1.0 / sL[j * B + j];
    // Sigma_ij for i > j (one thread per row)
    if (tid < B && tid > j && tid < jmax) {
      const int i = tid;
      double s = sE[j * B + i];
      for (int mm = j + 1; mm < jmax; ++mm) s = fma(sL[j * B + mm], sS[mm * B + i], s);   // L(mm,j) Sigma(i,mm)
      const double v = -s * rl;
      sS[j * B + i] = v;
      s_part[i] = sL[j * B + i] * v;   // L(i,j) Sigma(i,j)
    }
    __syncthreads();
    if (tid == 0) {
      double t = sE[j * B + j];
      for (int i = j + 1; i < jmax; ++i) t += s_part[i];
      sS[j * B + j] = (rl - t) * rl;
    }
    __syncthreads();
    if (tid < B && tid > j && tid < jmax) sS[tid * B + j] = sS[j * B + tid];   // symmetric copy (row j)
    __syncthreads();
  }
  for (int idx = tid; idx < B * B; idx += kThreads) {
    const int i = idx % B, j = idx / B;
    if (i >= j && i < jmax) sput(a, J * B + i, J * B + j, sS[j * B + i]);
  }
  publish(&a.flags[sfidx(a, J, J)], m + 1);
  return true;
}

template <int B>
__global__ void __launch_bounds__(kThreads, 2) selinv_kernel(SelArgs a) {
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
    if (threadIdx.x == 0) next = atomicAdd(&a.ctl->ticket, 1ULL);
    int type, J, I, M;
    sel_decode(a.S, a.p, t, type, J, I, M);
    bool ok;
    if (type == kSacc)
      ok = sel_sacc<B>(a, I, J, M, sm, &s_flag);
    else if (type == kSfin)
      ok = sel_sfin<B>(a, I, J, sm, &s_flag);
    else if (type == kDacc)
      ok = sel_dacc<B>(a, J, M, sm, &s_flag);
    else
      ok = sel_dfin<B>(a, J, sm, &s_flag);
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

size_t selinv_workspace_bytes(int n, int k, int b) {
  const int S = (n + b - 1) / b;
  int p = (k + b - 1) / b;
  if (p > S - 1) p = S - 1;
  return 256 + sizeof(int) * (size_t)S * (size_t)(p + 1);
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
  if ((unsigned long long)grid > a.total) grid = (long long)a.total;
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
  cudaError_t e = cudaMemsetAsync(ws, 0, selinv_workspace_bytes(n, k, b), st);
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
  a.total = sel_total(S, p);
  a.ctl = reinterpret_cast<Control*>(ws);
  a.flags = reinterpret_cast<int*>(static_cast<char*>(ws) + 256);
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

cudaError_t launch_logdet(const double* ab, long long ldab, int n, double* out, cudaStream_t st) {
  logdet_kernel<<<1, 1024, 0, st>>>(ab, ldab, n, out);
  return cudaGetLastError();
}

}  // namespace bchol
