// split_update.cuh -- FP64-accurate tile products C -= A B^T on the tensor
// cores (tcgen05), by splitting each FP64 operand into signed 8-bit digits.
//
// The trailing update A_IJ -= L_Is L_Js^T of Algorithm 1 (the O(n k^2) part
// of the flop count, Sec. 3.2, Eq. (1)) is a dense product with inner
// dimension b.  GB300 runs FP64 FMA at 1.25 TFLOP/s, but bf16 products with
// FP32 accumulation at ~2 PFLOP/s.  The error-free splitting of Ozaki, Ogita,
// Oishi and Rump (2012) turns one FP64 product into a few low-precision
// products that are each computed exactly:
//
//  * Every row r of an operand (K entries: the inner dimension, one tile column
//    of b = K = 16 or 32) is
//    scaled by its own power of two 2^{-E_r}, |x| < 2^{E_r}, and cut into a
//    55-bit fixed-point integer F = |x| 2^{55 - E_r} (truncated).  F is written
//    in base 256 with seven balanced digits s_a in [-128, 128]:
//        x ~= sign(x) 2^{E_r - 55} sum_{a=0..6} s_a 2^{48 - 8a}.
//    (Adding 0x80 to every byte of F and subtracting 128 from every byte
//    afterwards gives the balanced form without a carry chain.)  Each digit
//    is an integer of at most 8 significant bits, exact in bf16.
//  * For digit matrices A_a (rows of A) and B_b (rows of B), the product
//    A_a B_b^T has entries sum_k s t with |s t| <= 2^14 and K <= 32 terms, so
//    every partial sum is an integer below 2^19 and the FP32 accumulation of
//    the tensor core is exact.  Level c collects the pairs a + b = c in one
//    FP32 accumulator, P_c = sum_{a+b=c} A_a B_b^T, still exact (< 7 * 2^19 <
//    2^22).  Levels c <= 6 are kept (28 pairs); the pairs dropped weigh
//    below 2^{-56} relative to the rows' scales.
//  * In the epilogue, each P_c is read from tensor memory, turned into an
//    integer exactly (|P_c| < 2^22), and the levels are summed in 64-bit fixed
//    point, acc = sum_{c<=5} P_c 2^{40-8c} + floor(P_6 / 2^8), so that
//        (A B^T)_{rj} ~= acc * 2^{E_r + E_j - 54}.
//    One int-to-double conversion and one FP64 FMA per entry apply it to C.
//
// Error: the digits carry 55 bits of each row's scale, so each product is
// accurate to about K 2^{-54} max_k|a_rk| max_k|b_jk|, the same form and size
// as the rounding bound of an FP64 dot product (K u sum_k |a_rk b_jk|, u = 2^-53)
// for rows of comparable entries.  Rows whose entries differ by many orders of
// magnitude lose the digits of their small entries below 2^{E_r - 55}.
//
// One product covers 128 rows of A (the MMA's M: 128 / b tiles of a block
// column) and the b rows of one tile of B (N = b).
//
// Layout of one operand in shared memory (K-major, no swizzle, as tcgen05
// reads it): 8 x 8 "core matrices" of bf16, 128 contiguous bytes each (8 rows
// of 16 bytes); core matrices adjacent along K are 128 bytes apart, row groups
// of 8 are 16 K bytes apart (K / 8 core matrices per row group).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bchol {
namespace split {

constexpr int kDigits = 7;      // balanced base-256 digits per operand entry
constexpr int kRowsA = 128;     // rows of A per product: the MMA's M
constexpr int kLevels = 7;      // levels c = a + b = 0..6 kept

// Tensor-memory columns for K-wide level accumulators: 7 K, rounded up to a power of two.
template <int K>
__host__ __device__ constexpr uint32_t tmem_cols() { return K == 32 ? 256u : 128u; }

// Shared memory of one split product with inner dimension K (B has K rows):
// about 72 KB for K = 32, 32 KB for K = 16.  The completion barrier and the
// tensor-memory address live outside it (see Ctx), so that other tasks of a
// persistent CTA may reuse this region between products.
template <int K>
struct Smem {
  static_assert(K == 16 || K == 32, "inner dimension 16 or 32");
  uint4 a[kDigits][kRowsA * K / 8];  // digit matrices of A
  uint4 b[kDigits][K * K / 8];       // digit matrices of B
  int ea[kRowsA];  // largest exponent field among the entries of each row of A (row_scale gives E_r)
  int eb[K];       // the same for the rows of B
};

// Per-CTA state that outlives one product: the MMA completion barrier (in
// shared memory), the tensor-memory base address and the barrier's parity.
struct Ctx {
  unsigned long long* mbar;
  uint32_t tmem;
  uint32_t phase;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of row r, K-group kg (8 consecutive k) in one digit matrix.
template <int K>
__device__ __forceinline__ uint32_t op_off(int r, int kg) {
  return (uint32_t)((r >> 3) * (16 * K) + kg * 128 + (r & 7) * 16);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (K-direction core-matrix stride, 128 B), stride byte offset
// (row-group stride, 16 K bytes), descriptor version 1, no swizzle.
template <int K>
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint32_t a = smem_u32(p);
  return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((16u * K) >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: bf16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ------------------------------------------------------------ tcgen05 wrappers
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {  // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // one whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t globaltimer_now() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// D (+)= A B^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on mbar once every MMA this thread has issued is complete.
__device__ __forceinline__ void mma_commit(unsigned long long* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

// 8 consecutive FP32 columns of this thread's tensor-memory lane (the warp
// reads the 32 lanes of its quadrant).  The registers are valid only after
// tmem_wait8 on them.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
// Wait for this thread's tensor-memory loads; the registers of one load are
// tied to the wait so that no use of them moves above it (a second wait after
// the first returns at once).
__device__ __forceinline__ void tmem_wait8(uint32_t (&v)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
               :
               : "memory");
}

// ------------------------------------------------------------------ digits
__device__ __forceinline__ int exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// The seven balanced digits of x for a row whose scale has biased exponent
// field Eb (|x| < 2^{Eb - 1023}): d[a] holds s_a (without the sign of x) as
// FP32 bits, exact, whose upper half is its bf16 pattern; *neg is the sign of
// x.  Subnormal entries are flushed to zero.
__device__ __forceinline__ void digits_of(double x, int Eb, uint32_t (&d)[kDigits], bool* neg) {
  const uint32_t lo0 = (uint32_t)__double2loint(x), hi0 = (uint32_t)__double2hiint(x);
  const int e = (int)((hi0 >> 20) & 0x7FF);
  const unsigned long long m =
      e ? (((unsigned long long)((hi0 & 0xFFFFFu) | 0x100000u) << 32) | lo0) : 0ull;
  const int sh = e - Eb + 3;  // <= 2, so F < 2^55
  unsigned long long F;
  if (sh >= 0)
    F = m << sh;
  else
    F = (sh > -64) ? (m >> (-sh)) : 0ull;
  const unsigned long long G = F + 0x80808080808080ull;  // +128 in each of the seven bytes
  const uint32_t lo = (uint32_t)G, hi = (uint32_t)(G >> 32);
  // digit a sits in bits 48-8a .. 55-8a of G (the top one may carry into bit 56)
  const uint32_t byte[kDigits] = {hi >> 16, (hi >> 8) & 0xFFu, hi & 0xFFu, lo >> 24,
                                  (lo >> 16) & 0xFFu, (lo >> 8) & 0xFFu, lo & 0xFFu};
#pragma unroll
  for (int a = 0; a < kDigits; ++a)  // (byte - 128) as a float, exact: 1.5 * 2^23 + (byte - 128) - 1.5 * 2^23
    d[a] = __float_as_uint(__int_as_float((int)(0x4B3FFF80u + byte[a])) - 12582912.0f);
  *neg = (hi0 >> 31) != 0;
}

// Write the digits of 8 consecutive entries x[0..7] (one K-group kg of row r)
// into the seven digit matrices starting at `base` (stride `slice_bytes`):
// two entries' bf16 digits per 32-bit word, the sign of each entry applied to
// its digits.
template <int K>
__device__ __forceinline__ void store_digits8(const double (&x)[8], int Eb, unsigned char* base, uint32_t slice_bytes,
                                              int r, int kg) {
  uint32_t w[kDigits][4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    uint32_t d0[kDigits], d1[kDigits];
    bool n0, n1;
    digits_of(x[e], Eb, d0, &n0);
    digits_of(x[e + 1], Eb, d1, &n1);
    const uint32_t sgn = (n0 ? 0x8000u : 0u) | (n1 ? 0x80000000u : 0u);
#pragma unroll
    for (int a = 0; a < kDigits; ++a) w[a][e >> 1] = __byte_perm(d0[a], d1[a], 0x7632) ^ sgn;
  }
  const uint32_t off = op_off<K>(r, kg);
#pragma unroll
  for (int a = 0; a < kDigits; ++a)
    *reinterpret_cast<uint4*>(base + a * slice_bytes + off) = make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
}

// Exponent field of the row scale from the largest exponent field among the
// row's entries: 2^E just above every |x|; -1 marks a non-finite entry.
__device__ __forceinline__ int row_scale(int max_e) { return max_e >= 0x7FF ? -1 : max_e + 1; }

// Issue the 28 digit products of one 128 x K (x K) product into the seven
// level accumulators (columns K c .. K c + K-1 of tensor memory), then commit
// to mbar.  One thread.  The digit matrices of B lie back to back, so
// [B_0; ...; B_{6-a}] is one operand of N = K (7 - a) rows; one MMA per digit
// a of A adds A_a B_b^T to the accumulator of level a + b for every b at once
// by writing D from column K a on.  K = 32 takes two MMAs of K = 16 per a (the
// second starts two core matrices, 256 bytes, later).
template <int K>
__device__ __forceinline__ void issue_products(Smem<K>& sm, uint32_t tmem, unsigned long long* mbar) {
  const uint64_t bd = smem_desc<K>(&sm.b[0][0]);
#pragma unroll
  for (int a = 0; a < kDigits; ++a) {
    const uint32_t idesc = idesc_bf16(kRowsA, K * (kDigits - a));
    const uint64_t ad = smem_desc<K>(&sm.a[a][0]);
    mma_bf16(tmem + (uint32_t)(K * a), ad, bd, idesc, a > 0 ? 1u : 0u);
    if constexpr (K == 32) mma_bf16(tmem + (uint32_t)(K * a), ad + (256u >> 4), bd + (256u >> 4), idesc, 1u);
  }
  mma_commit(mbar);
}

// 2^e as a double for -1022 <= e <= 1023.
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// acc * 2^ex, with the rare scales outside the normal range applied in two steps.
__device__ __forceinline__ double scaled(long long acc, int ex) {
  const double v = (double)acc;
  if (ex >= -1022 && ex <= 1023) return v * pow2(ex);
  if (ex < -1022) return ex < -2100 ? 0.0 * v : (v * pow2(ex + 600)) * pow2(-600);
  return (v * pow2(ex - 600)) * pow2(600);
}

// Sum the seven levels of 8 consecutive output columns (col0 .. col0+7) of
// this thread's row into 64-bit fixed point (see the header comment): all
// seven loads are in flight before the first wait.
template <int K>
__device__ __forceinline__ void combine_levels8(uint32_t tmem_row, int col0, long long (&acc)[8]) {
  uint32_t v[kLevels][8];
#pragma unroll
  for (int c = 0; c < kLevels; ++c) tmem_ld8(tmem_row + (uint32_t)(K * c + col0), v[c]);
#pragma unroll
  for (int c = 0; c < kLevels; ++c) tmem_wait8(v[c]);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int p[kLevels];
#pragma unroll
    for (int c = 0; c < kLevels; ++c)  // exact: |P_c| <= (c + 1) 2^19 < 2^22
      p[c] = __float_as_int(__uint_as_float(v[c][j]) + 12582912.0f) - 0x4B400000;
    // acc = P_0 2^40 + P_1 2^32 + P_2 2^24 + P_3 2^16 + P_4 2^8 + P_5 + floor(P_6 / 2^8),
    // with the pairs summed in 32 bits first (each below 2^30 in magnitude)
    const int hi = p[0] * 256 + p[1], mid = p[2] * 256 + p[3], lo = p[4] * 256 + p[5] + (p[6] >> 8);
    acc[j] = ((long long)hi << 32) + ((long long)mid << 16) + (long long)lo;
  }
}

// Set-up of a CTA that runs split products with inner dimension K (all
// threads): warp 0 allocates the tensor memory, thread 0 initialises the barrier.
template <int K>
__device__ __forceinline__ Ctx ctx_begin(unsigned long long* mbar, uint32_t* tmem_slot) {
  if ((threadIdx.x >> 5) == 0) tmem_alloc(tmem_slot, tmem_cols<K>());
  if (threadIdx.x == 0) mbar_init(mbar, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return Ctx{mbar, *tmem_slot, 0u};
}
// Tear-down (all threads, after the last product): warp 0 frees the tensor memory.
template <int K>
__device__ __forceinline__ void ctx_end(const Ctx& cx) {
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(cx.tmem, tmem_cols<K>());
  }
}

// One split update C -= A B^T of a 128-row block of A and a K-row block of B
// with inner dimension K, by all 256 threads of the CTA:
//   la(r, k), lb(j, k)  the entries of A and B (zero outside the operands);
//   ldc(r, j)  the entry of C before the update (0 outside C), read while the
//              MMAs run;  stc(r, j, v)  stores the updated entry (NaN when row r
//              of A or row j of B holds a non-finite entry);
//   cx  the CTA's barrier, tensor memory and barrier parity (advanced here).
// Warp w updates rows 32 (w % 4) .. + 31 (its tensor-memory lane quadrant),
// columns (K / 2)(w / 4) .. + K/2 - 1.
// Returns false (with *status = timeout and the abort word raised) if the
// MMAs do not complete within wait_ns; the caller then stops.
template <int K, class LA, class LB, class LC, class SC>
__device__ __forceinline__ bool product(Smem<K>& sm, Ctx& cx, LA la, LB lb, LC ldc, SC stc, uint64_t wait_ns,
                                        int* status, int* abort_word) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int KG = K / 8;                                // K-groups per row
  constexpr int kUnits = (kRowsA + K) * KG;                // (row, K-group) units: A first, then B
  constexpr int kPer = (kUnits + 255) / 256;
  constexpr int HC = K / 2;                                // output columns per thread
  if (tid < kRowsA) sm.ea[tid] = 0;
  if (tid < K) sm.eb[tid] = 0;
  __syncthreads();
  double x[kPer][8];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int u = tid + 256 * i;
    if (u < kUnits) {
      int emax = 0;
      if (u < kRowsA * KG) {
        const int r = u & (kRowsA - 1), kg = u / kRowsA;
#pragma unroll
        for (int e = 0; e < 8; ++e) x[i][e] = la(r, 8 * kg + e);
#pragma unroll
        for (int e = 0; e < 8; ++e) emax = max(emax, exp_field(x[i][e]));
        atomicMax(&sm.ea[r], emax);
      } else {
        const int v = u - kRowsA * KG, j = v % K, kg = v / K;
#pragma unroll
        for (int e = 0; e < 8; ++e) x[i][e] = lb(j, 8 * kg + e);
#pragma unroll
        for (int e = 0; e < 8; ++e) emax = max(emax, exp_field(x[i][e]));
        atomicMax(&sm.eb[j], emax);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int u = tid + 256 * i;
    if (u < kUnits) {
      if (u < kRowsA * KG) {
        const int r = u & (kRowsA - 1), kg = u / kRowsA;
        store_digits8<K>(x[i], row_scale(sm.ea[r]), reinterpret_cast<unsigned char*>(&sm.a[0][0]),
                         (uint32_t)sizeof(sm.a[0]), r, kg);
      } else {
        const int v = u - kRowsA * KG, j = v % K, kg = v / K;
        store_digits8<K>(x[i], row_scale(sm.eb[j]), reinterpret_cast<unsigned char*>(&sm.b[0][0]),
                         (uint32_t)sizeof(sm.b[0]), j, kg);
      }
    }
  }
  fence_async_smem();  // the digits, written by ordinary stores, are read by the tensor core
  __shared__ int s_done;
  __syncthreads();
  if (tid == 0) {
    tc_fence_after();
    issue_products<K>(sm, cx.tmem, cx.mbar);
  }
  // C is read while the MMAs run.
  const int q = warp & 3, h = warp >> 2, r = 32 * q + lane;
  double cold[HC];
#pragma unroll
  for (int jj = 0; jj < HC; ++jj) cold[jj] = ldc(r, HC * h + jj);
  if (tid == 0) {
    bool ok = mbar_try_wait(cx.mbar, cx.phase);
    if (!ok) {
      const uint64_t t0 = globaltimer_now();
      while (!(ok = mbar_try_wait(cx.mbar, cx.phase))) {
        if (globaltimer_now() - t0 > wait_ns) break;
      }
      if (!ok) {  // record, then give the MMAs a second bounded wait before the caller frees tensor memory
        atomicExch(status, 2);
        atomicExch(abort_word, 1);
        const uint64_t t1 = globaltimer_now();
        while (!mbar_try_wait(cx.mbar, cx.phase) && globaltimer_now() - t1 < wait_ns) {
        }
      }
    }
    s_done = ok;
  }
  __syncthreads();
  cx.phase ^= 1u;
  if (!s_done) return false;
  tc_fence_after();
  const int er = row_scale(sm.ea[r]);
#pragma unroll
  for (int half = 0; half < HC / 8; ++half) {
    long long acc[8];
    combine_levels8<K>(cx.tmem + ((uint32_t)(32 * q) << 16), HC * h + 8 * half, acc);
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = HC * h + 8 * half + jj;
      const int ej = row_scale(sm.eb[j]);
      const int ex = er + ej - 2100;  // (E_r - 1023) + (E_j - 1023) - 54
      double v;
      if (er < 0 || ej < 0)
        v = __longlong_as_double(0x7FF8000000000000ll);
      else if (ex >= -1022 && ex <= 1023)
        v = fma(-(double)acc[jj], pow2(ex), cold[8 * half + jj]);
      else
        v = cold[8 * half + jj] - scaled(acc[jj], ex);
      stc(r, j, v);
    }
  }
  tc_fence_before();
  __syncthreads();  // tensor memory is read before the next product overwrites it
  return true;
}

}  // namespace split
}  // namespace bchol
