// bchol_internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace bchol {

// Values of the status word that records how the last launch ended.
constexpr int kStatusOk = 0;
constexpr int kStatusTimeout = 2;

// Automatic tile size and CTAs per SM, from the n = 1e5 sweep on GB300:
// b = 16 wins while the factorization is bound by its diagonal chain (whose
// step time grows with b^3 on one SM) up to k of about 640; b = 32 wins above,
// where the trailing updates dominate.  One CTA per SM while the ticket work
// is small (k <= 256); two per SM above, to overlap the tasks' load and flag
// latencies.  bchol_factor and bchol_factor_noalloc both use this rule.
inline int auto_tile(int k) { return k <= 640 ? 16 : 32; }
inline int auto_ctas_per_sm(int k) { return k <= 256 ? 1 : 2; }

// Tile geometry of one factorization: S = ceil(n/b) tile rows, p = ceil(k/b)
// sub-diagonal tiles per panel (clamped to S-1).
struct FactorPlan {
  int n = 0, k = 0, b = 32, S = 0, p = 0;
  long long Sreg = 0;          // leading ticket blocks of full size (see schedule.cuh)
  long long Treg = 0;          // tasks per such block: 2p + 1 + p(p-1)/2
  long long Treg_cp = 0;       // tickets per such block with the diagonal chain: 2(p-1) + p(p-1)/2
  unsigned long long total_cp = 0;  // tickets with the diagonal chain (tiles of 16 and 32)
  long long Treg_hp = 0;       // tickets per such block with the chain and two helper CTAs: 2(p-2) + p(p-1)/2 - 1
  unsigned long long total_hp = 0;  // tickets with the chain and the helpers
  bool helper = false;         // tiles of 16 and 32 with 2 <= p <= 40: the chain plus two helper CTAs
  unsigned long long total = 0;  // tasks of the whole factorization
  size_t flag_count = 0;       // ints of ready flags: S*(p+1)
  bool f32_update = false;     // mixed precision: trailing updates accumulated in FP32
  int H = 1;                   // > 1: the updates run as strips of H = 128 / b tiles, split products on the tensor cores
};

// Plan of one factorization with tiles of b; `split` selects the tensor-core
// split updates (tiles of 16 and 32; tiles of 64 ignore it).
FactorPlan make_factor_plan(int n, int k, int b, bool split = false);
// Task t (0-based) of the combined order that one factorization runs, and the
// number of tasks in that order.
void plan_task(const FactorPlan& P, long long t, int& type, int& s, int& I, int& J);
long long plan_task_count(const FactorPlan& P);

// Device workspace needed by one factorization (control block + flags).
size_t factor_workspace_bytes(const FactorPlan& plan);

// CTAs per SM of a kernel that allocates tmem_cols tensor-memory columns per
// CTA, from its registers, shared memory (dyn_smem dynamic bytes) and threads.
cudaError_t tc_ctas_per_sm(const void* func, size_t dyn_smem, int tmem_cols, int threads, int* per_sm);

// Launch the persistent factor kernel.  `ws` holds factor_workspace_bytes()
// bytes; `status` is a device int that outlives the call (timeout record).
cudaError_t launch_pivot_rcp(const double* x, double* y, int n, cudaStream_t stream);
// tma: the chain's prefetch warps copy their tiles with TMA where the band's
// tensor map can be encoded (ldab odd); *tma_used (if given) reports whether they do.
cudaError_t launch_factor(const FactorPlan& plan, double* ab, long long ldab, int* info, void* ws, int* status,
                          uint64_t wait_ns, int ctas_per_sm, int stall_I, int stall_J, cudaStream_t stream,
                          int tma = 0, int* tma_used = nullptr);

// Solve: block size and workspace of the inverted diagonal blocks.
int solve_block(int k);
size_t solve_workspace_bytes(int n, int k);
// path: 0 automatic, 1 cluster, 2 partitioned; status (timeout record) and
// wait_ns bound the partitioned solve's waits (without status it is not used).
cudaError_t launch_solve(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb,
                         void* ws, int* launches, cudaStream_t stream, int path = 0, int* status = nullptr,
                         uint64_t wait_ns = 2000000000ull);
// The partitioned chunk solve for small k (psolve.cu).
int psolve_max_k();
size_t psolve_workspace_bytes(int n, int k);
cudaError_t launch_psolve(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb,
                          void* ws, int* status, uint64_t wait_ns, int* launches, cudaStream_t stream);
// The same sweeps with FP32 arithmetic (FP64 band and right-hand sides in memory).
cudaError_t launch_solve_f32(int n, int k, int nrhs, const double* ab, long long ldab, double* b, long long ldb,
                             void* ws, int* launches, cudaStream_t stream);

int num_sms();

// Throughput probes of the roofline denominators (probe.cu): TFLOP/s of kind
// 0 DFMA, 1 DMMA, 2 FFMA, 3 tcgen05 bf16 MMA, over `iters` iterations per chain.
cudaError_t probe_rate(int kind, int iters, double* tflops, int* status, uint64_t wait_ns, cudaStream_t stream);

// The tensor-core split product alone (split.cu): C := C - A B^T, inner dimension 32.
cudaError_t launch_split_check(int m, int n, const double* A, long long lda, const double* B, long long ldb,
                               double* C, long long ldc, int* status, int* abort_word, uint64_t wait_ns,
                               cudaStream_t stream);

// Adjoint (selinv.cu): band of A^{-1} by selected inversion and the band gradient.
size_t selinv_workspace_bytes(int n, int k, int b);
long long adjoint_plan_count(int n, int k, int b);
void adjoint_plan_task(int n, int k, int b, long long t, int* type, int* J, int* I, int* g);
cudaError_t launch_backward(int n, int k, int b, const double* L, long long ldl, const double* x, const double* bbar,
                            double ldbar, double* g, long long ldg, void* ws, int* status, uint64_t wait_ns,
                            int ctas_per_sm, cudaStream_t stream);
cudaError_t launch_logdet(const double* ab, long long ldab, int n, double* out, cudaStream_t stream);

// Mixed-precision factor + FP64 iterative refinement (mixed.cu).
size_t mixed_workspace_bytes(int n, int k, int nrhs, int tile);
// The workspace's copy of up to nrhs_max right-hand sides (mixed_layout's B0).
double* mixed_rhs_copy(void* ws, int n, int k, int nrhs_max, int tile);
int mixed_factor(int n, int k, const double* ab, long long ldab, int* info_dev, int tile, int ctas_per_sm, void* ws,
                 int nrhs_max, int* status, uint64_t wait_ns, cudaStream_t stream, int* launches_out);
int mixed_refine(int n, int k, int nrhs, const double* ab, long long ldab, const double* b, long long ldb, double* x,
                 long long ldx, int max_iter, double tol, int tile, void* ws, int nrhs_max, cudaStream_t stream,
                 int* iters_out, double* resid_out, double* corr_out, int* launches_out, double* phase_ms);
int mixed_solve(int n, int k, int nrhs, const double* ab, long long ldab, const double* b, long long ldb, double* x,
                long long ldx, int max_iter, double tol, int* info_dev, int tile, int ctas_per_sm, void* ws,
                int* status, uint64_t wait_ns, cudaStream_t stream, int* iters_out, double* resid_out,
                double* corr_out, int* launches_out);

}  // namespace bchol

struct bchol_batch_s;
namespace bchol {
// Enqueue the launches of a planned batch (batched.cu).
int batch_run(bchol_batch_s* batch, int* status, uint64_t wait_ns, cudaStream_t stream, int* launches);

}  // namespace bchol
