// split.cu -- the tensor-core split product on its own, for tests:
// C := C - A B^T with inner dimension 32, computed exactly as the trailing
// updates of the FP64_SPLIT factorization compute it (split_update.cuh).
#include "../../include/bchol.h"
#include "bchol_internal.h"
#include "split_update.cuh"

namespace bchol {

struct SplitCheckArgs {
  const double* A;
  const double* B;
  double* C;
  long long lda, ldb, ldc;
  int m, n;
  int* status;
  int* abort_word;
  uint64_t wait_ns;
};

// One CTA per 128 x 32 block of C.
__global__ void __launch_bounds__(256, 1) split_check_kernel(SplitCheckArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ unsigned long long s_mbar;
  __shared__ uint32_t s_tmem;
  constexpr int K = 32;
  split::Smem<K>& sm = *reinterpret_cast<split::Smem<K>*>(smem_raw);
  split::Ctx cx = split::ctx_begin<K>(&s_mbar, &s_tmem);
  const int r0 = blockIdx.x * split::kRowsA, j0 = blockIdx.y * K;
  auto la = [&](int r, int k) { return r0 + r < a.m ? a.A[(r0 + r) + (long long)k * a.lda] : 0.0; };
  auto lb = [&](int j, int k) { return j0 + j < a.n ? a.B[(j0 + j) + (long long)k * a.ldb] : 0.0; };
  auto ldc = [&](int r, int j) {
    return (r0 + r < a.m && j0 + j < a.n) ? a.C[(r0 + r) + (long long)(j0 + j) * a.ldc] : 0.0;
  };
  auto stc = [&](int r, int j, double v) {
    if (r0 + r < a.m && j0 + j < a.n) a.C[(r0 + r) + (long long)(j0 + j) * a.ldc] = v;
  };
  split::product<K>(sm, cx, la, lb, ldc, stc, a.wait_ns, a.status, a.abort_word);
  split::ctx_end<K>(cx);
}

cudaError_t launch_split_check(int m, int n, const double* A, long long lda, const double* B, long long ldb,
                               double* C, long long ldc, int* status, int* abort_word, uint64_t wait_ns,
                               cudaStream_t stream) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const size_t smem = sizeof(split::Smem<32>);
  cudaError_t e = cudaFuncSetAttribute(split_check_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(split_check_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  SplitCheckArgs a{A, B, C, lda, ldb, ldc, m, n, status, abort_word, wait_ns};
  dim3 grid((m + split::kRowsA - 1) / split::kRowsA, (n + 31) / 32);
  split_check_kernel<<<grid, 256, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace bchol
