/*
 * bchol.h -- C ABI of the GB300 banded Cholesky library (libbchol.so).
 *
 * Method: F. Liu, A. Fredriksson, S. Markidis, "Parallel Cholesky
 * Factorization for Banded Matrices using OpenMP Tasks" (arXiv 2305.04635).
 * The library factors a symmetric positive-definite band matrix A = L L^T
 * (Sec. 2.1, Sec. 3, Algorithm 1) and solves A X = B with the factor.
 *
 * Storage (Sec. 3: the standard LAPACK band format, kept to avoid any format
 * conversion): A of order n with half-bandwidth k ("number of super- and
 * sub-diagonals", Sec. 1 and Sec. 3.1) is held by its lower band in a
 * column-major array `ab` with leading dimension ldab >= k+1:
 *     A(i,j) = ab[(i-j) + j*ldab]      for 0 <= j <= i <= min(n-1, j+k).
 * Rows d >= k+1 of the array (when ldab > k+1) and the slots (d, j) with
 * j + d >= n hold no matrix entry; the library never reads or writes them.
 * k >= n is accepted and treated as k = n-1 (a dense lower triangle).
 *
 * Conventions shared by every entry point:
 *  - All matrix and vector pointers are DEVICE pointers owned by the caller.
 *    The library never frees or keeps them past the call.
 *  - Every call is asynchronous on the handle's CUDA stream.  Argument errors
 *    are found on the host before any launch and return BCHOL_ERR_ARG with
 *    nothing launched.  A CUDA launch or copy failure returns BCHOL_ERR_CUDA.
 *  - Numerical failure (a pivot that is not > 0, NaN included) is reported the
 *    LAPACK way through a device-resident `info`; the call itself still
 *    returns BCHOL_OK.  bchol_get_info synchronises and reads it.
 *  - Every wait inside a kernel is bounded in time.  A wait that runs out
 *    stops the kernel cleanly and records BCHOL_ERR_TIMEOUT in the handle;
 *    bchol_get_info reports it.
 *  - The handle owns internal device workspace (ready flags, a task counter,
 *    inverted diagonal blocks).  It is taken from a buffer the caller lends
 *    with bchol_set_workspace, else allocated with cudaMalloc on first use and
 *    kept until bchol_destroy.  Calls on one handle must not overlap.
 */
#ifndef BCHOL_H
#define BCHOL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bchol_handle_s* bchol_handle_t;

typedef enum {
  BCHOL_OK = 0,
  BCHOL_ERR_ARG = -1,      /* invalid argument; nothing was launched */
  BCHOL_ERR_NOT_SPD = 1,   /* some info > 0: a leading minor is not positive definite */
  BCHOL_ERR_TIMEOUT = 2,   /* a bounded in-kernel wait ran out; results are unspecified */
  BCHOL_ERR_CUDA = 3,      /* a CUDA runtime call failed */
  BCHOL_ERR_ALLOC = 4,     /* workspace allocation failed, or the lent workspace is too small */
  BCHOL_ERR_UNSUPPORTED = 5
} bchol_status_t;

/* Arithmetic of the factorization's trailing SYRK/GEMM updates (the O(n k^2)
 * part of Algorithm 1, Sec. 3.2 and Eq. (1)), set per handle with
 * bchol_set_precision.  POTRF and TRSM of the tiles are FP64 in every mode.
 *   BCHOL_FP64         FP64 fused multiply-adds (the default; the paper's arithmetic).
 *   BCHOL_FP32_UPDATE  updates accumulated in FP32 from FP32-rounded tiles (and
 *                      FP32 panel TRSMs), and FP64 iterative refinement in the
 *                      solve: bchol_factor then leaves ab holding A and keeps the
 *                      mixed factor in the handle, and bchol_solve refines
 *                      against that A (see bchol_set_precision).
 *   BCHOL_TF32_UPDATE  not built; bchol_set_precision returns BCHOL_ERR_UNSUPPORTED.
 *   BCHOL_FP64_SPLIT   FP64-accurate updates from exact bf16 digit products on the
 *                      tensor cores (bchol_check_split_product), with tiles of 16
 *                      and 32; with tiles of 64 the updates are FP64 FMA.  With
 *                      the automatic tile they run where that tile is 32
 *                      (k > 640); for smaller k the diagonal chain bounds the
 *                      factorization and the FP64 updates are kept.  L agrees
 *                      with the FP64 mode to rounding. */
typedef enum {
  BCHOL_FP64 = 0,
  BCHOL_FP32_UPDATE = 1,
  BCHOL_TF32_UPDATE = 2,
  BCHOL_FP64_SPLIT = 3
} bchol_precision_t;

/* Create a handle bound to `stream` (a cudaStream_t; NULL = the legacy default
 * stream) on the current device.  No device memory is allocated here. */
bchol_status_t bchol_create(bchol_handle_t* handle, void* stream);

/* Release the handle and any workspace it allocated itself. */
bchol_status_t bchol_destroy(bchol_handle_t handle);

/* Rebind the handle to another stream. */
bchol_status_t bchol_set_stream(bchol_handle_t handle, void* stream);

/* Lend the handle a device buffer (16-byte aligned) for its workspace, or
 * pass NULL/0 to go back to self-allocated workspace.  The buffer must stay
 * valid while calls that use it may be running. */
bchol_status_t bchol_set_workspace(bchol_handle_t handle, void* dev_ptr, size_t bytes);

/* Bytes of workspace that bchol_factor / bchol_solve need for order n and
 * half-bandwidth k with the handle's current settings. */
size_t bchol_workspace_size(bchol_handle_t handle, int n, int k);

/*
 * bchol_factor -- A = L L^T in place (Algorithm 1 and its cross-iteration
 * overlap, Sec. 3; the factor is the unique one of Sec. 2.1).
 *   n, k      order and half-bandwidth, n >= 0, k >= 0
 *   ab        device, the lower band of A as above; overwritten by L
 *   ldab      leading dimension, ldab >= k+1
 *   info_dev  device int, written by the kernel: 0 on success, or j > 0 when
 *             the leading minor of order j is not positive definite (LAPACK
 *             pbtrf convention).  When j > 0 the contents of ab are unspecified.
 * The whole factorization is one persistent kernel launch (plus one memset
 * of the ready flags).  Tiles are b x b with b chosen from k (16 up to
 * k = 640, else 32) unless bchol_set_tile fixes it.
 */
bchol_status_t bchol_factor(bchol_handle_t handle, int n, int k, double* ab, int ldab, int* info_dev);

/*
 * bchol_factor_noalloc -- bchol_factor for callers that may not allocate GPU
 * memory.  The paper has no counterpart: this exists for code that must not
 * call cudaMalloc, such as allocators or arenas that own all device memory,
 * real-time hosts that forbid allocation after start-up, or plugins whose
 * host application owns every allocation.  It takes no handle and allocates
 * nothing.  The factor kernel's scratch (task ticket, abort word, per-tile
 * ready flags) lives in one fixed 1 MiB array in the library's device memory,
 * which every GPU that loads the library holds until the process exits.
 *   stream      cudaStream_t to launch on (NULL = legacy default stream)
 *   n, k, ab, ldab, info_dev   as for bchol_factor; the kernel, and so the
 *               result, is that of bchol_factor with the default settings
 *               (automatic tile, FP64 precision mode)
 *   status_dev  device int owned by the caller: set to 0, then to
 *               BCHOL_ERR_TIMEOUT (2) if a bounded in-kernel wait ran out
 * Returns BCHOL_ERR_UNSUPPORTED, with nothing launched, when the problem needs
 * more scratch than the array holds: 256 bytes plus 4 bytes per tile ready
 * flag, ceil(n/b) * (ceil(k/b) + 1) flags with b = 16 for k <= 640, else 32.
 * At n = 1e5 every k up to 2624 fits (k = 2625 does not); at n = 1e6, k up to
 * 48.  All calls on a device share the array, so calls that overlap on the
 * GPU race; order them.  The first call in each CUDA context looks up the
 * array's device address: make it before any stream capture, and again after
 * a cudaDeviceReset (which starts a new context).
 */
bchol_status_t bchol_factor_noalloc(void* stream, int n, int k, double* ab, int ldab, int* info_dev,
                                    int* status_dev);

/*
 * bchol_solve -- X = A^{-1} B from the factor that bchol_factor left in ab
 * (LAPACK pbtrs semantics, lower): L Y = B by forward substitution, then
 * L^T X = Y by back substitution.  The paper solves no systems itself; its
 * motivation is the repeated banded solves of an interior-point method
 * (Sec. 1 and Sec. 2).
 *   ab, ldab  device, the factor L in band storage (read only)
 *   b, ldb    device, B is n x nrhs column-major with ldb >= max(1,n);
 *             overwritten by X
 */
bchol_status_t bchol_solve(bchol_handle_t handle, int n, int k, int nrhs, const double* ab, int ldab,
                           double* b, int ldb);

/*
 * bchol_logdet -- log det A = 2 sum_i log L_ii from the factor in ab, written
 * to the device double out_dev (asynchronous).
 */
bchol_status_t bchol_logdet(bchol_handle_t handle, int n, const double* ab, int ldab, double* out_dev);

/*
 * bchol_backward -- the adjoint of x = A^{-1} b and log det A with respect to
 * the stored band of A (the interior-point use the paper names, Sec. 1-2).
 * For a scalar loss f(x, log det A) with xbar = df/dx and ldbar = df/dlogdet:
 *   bbar = A^{-1} xbar   (df/db)
 *   abar(i,j) = 2 ldbar Sigma(i,j) - (bbar_i x_j + bbar_j x_i)   for i > j
 *   abar(i,i) =   ldbar Sigma(i,i) -  bbar_i x_i
 * where Sigma = A^{-1}; each stored off-diagonal entry ab(i-j, j) stands for
 * both A(i,j) and A(j,i), hence the factor 2 and the symmetric term.  Only the
 * band of Sigma is formed, by selected inversion (the Takahashi recurrences
 * Sigma L = L^{-T}) in one persistent kernel over the factor's tiles, walked
 * from the last block column to the first.
 *   ab, ldab      device, the factor L from bchol_factor (read only)
 *   x             device, the solution x = A^{-1} b (n doubles; may be NULL if xbar is NULL)
 *   xbar          device, df/dx (n doubles), or NULL for a loss of log det A alone
 *   ldbar         df/dlogdet
 *   abar, ldabar  device, output band (ldabar >= k+1): df/d ab
 *   bbar          device, output df/db (n doubles; may be NULL if xbar is NULL)
 */
bchol_status_t bchol_backward(bchol_handle_t handle, int n, int k, const double* ab, int ldab, const double* x,
                              const double* xbar, double ldbar, double* abar, int ldabar, double* bbar);

/*
 * bchol_solve_mixed -- X = A^{-1} B by a mixed-precision factorization with
 * FP64 iterative refinement.  The paper's method is FP64 throughout; this
 * form runs the trailing SYRK/GEMM updates of Algorithm 1 (the O(n k^2) part,
 * Sec. 3.2) with FP32 accumulation, keeps POTRF and TRSM of the tiles in FP64,
 * and recovers FP64 accuracy by refinement:
 *   Ã = S A S, S = diag(A)^{-1/2} (equilibration of a copy of A; A is not changed)
 *   Ã ~ L L^T (FP32-accumulated updates); x_0 = S (L L^T)^{-1} S b
 *   repeat: r = b - A x (FP64); stop when max_c ||r_c|| / ||b_c|| <= tol, when the
 *   residual stops shrinking or after max_iter corrections; else d = S (L L^T)^{-1} S r
 *   (FP32 solve) and x += d (FP64).
 *   ab, ldab      device, lower band of A (read only)
 *   b, ldb        device, n x nrhs right-hand sides (read only)
 *   x, ldx        device, n x nrhs solution (output)
 *   info_dev      device int: info of the factorization of Ã (LAPACK convention)
 *   iters, resid, corr   host outputs: corrections made, final max_c ||b_c - A x_c|| / ||b_c||,
 *                 and the last relative correction max_c ||d_c|| / ||x_c|| (0 if none)
 * Returns BCHOL_ERR_NOT_SPD (with info_dev set) if Ã is not positive definite.
 * Synchronises the handle's stream (the loop reads the norms on the host).
 * Workspace: a copy of the band, n x nrhs doubles and the factor/solve scratch.
 */
bchol_status_t bchol_solve_mixed(bchol_handle_t handle, int n, int k, int nrhs, const double* ab, int ldab,
                                 const double* b, int ldb, double* x, int ldx, int max_iter, double tol,
                                 int* info_dev, int* iters, double* resid, double* corr);

/*
 * Batched factorization and solve.  Many independent SPD band systems of
 * uneven n and k are factored by one persistent launch (the paper factors one
 * matrix at a time; this is the batched form of the same tile algorithm) and,
 * for the systems that have right-hand sides, solved by a second launch.
 * A batch object holds the plan (per-system descriptors, ticket counters and
 * ready flags, sorted largest system first) in device memory that it
 * allocates with cudaMalloc when it is planned.
 *   count            number of systems (>= 1)
 *   n, k, ldab       HOST arrays of count ints: order, half-bandwidth, leading dimension
 *   ab               HOST array of count DEVICE pointers: band storage of each A (in place -> L)
 *   info_dev         DEVICE array of count ints: per-system info (LAPACK convention)
 *   nrhs, b, ldb     optional (NULL = no solve): HOST arrays; b holds DEVICE pointers to
 *                    n x nrhs column-major blocks, overwritten by X = A^{-1} B
 *   tile             16, 32 or 64 (0 = automatic: 32); ctas_per_sm 0 = automatic (2, or fewer
 *                    where the SM's resources allow fewer)
 * bchol_batch_plan synchronises (it copies the descriptors to the device).
 * bchol_batch_run only enqueues a memset and two kernels on the handle's
 * stream, so it can be captured in a CUDA graph and replayed; the pointed-to
 * matrices must then stay at the planned addresses.
 */
typedef struct bchol_batch_s* bchol_batch_t;
bchol_status_t bchol_batch_create(bchol_batch_t* batch);
bchol_status_t bchol_batch_destroy(bchol_batch_t batch);
bchol_status_t bchol_batch_plan(bchol_batch_t batch, int count, const int* n, const int* k, double* const* ab,
                                const int* ldab, int* info_dev, const int* nrhs, double* const* b, const int* ldb,
                                int tile, int ctas_per_sm);
bchol_status_t bchol_batch_run(bchol_handle_t handle, bchol_batch_t batch);

/* bchol_batch_set_precision -- the precision of the batch's next plan:
 * BCHOL_FP64 (default) or BCHOL_FP64_SPLIT, which, with tiles of 16 or 32,
 * runs every system's trailing updates as split products on the tensor cores
 * in strips of 128 / b tiles (same accuracy contract as for bchol_factor;
 * with tiles of 64 it plans the FP64 updates).  Takes effect at the next
 * bchol_batch_plan.  BCHOL_ERR_UNSUPPORTED for BCHOL_FP32_UPDATE and
 * BCHOL_TF32_UPDATE, BCHOL_ERR_ARG for an unknown mode.
 * bchol_factor_batched plans with the handle's precision (FP64 when the
 * handle's mode is BCHOL_FP32_UPDATE). */
bchol_status_t bchol_batch_set_precision(bchol_batch_t batch, int precision);

/* bchol_batch_set_member_precision -- per-system precision modes for the next
 * bchol_batch_plan (which then needs the same count): precision[m] is
 * BCHOL_FP64 or BCHOL_FP64_SPLIT for system m (HOST array); count = 0 clears
 * the override, and the batch's bchol_batch_set_precision mode applies to
 * every system again.  One launch runs both kinds of systems.  For tuning the
 * mode per class of systems (paper_2305_04635_gb300.autotune.tune_batch_classes).
 * BCHOL_ERR_UNSUPPORTED for the FP32/TF32 modes, BCHOL_ERR_ARG otherwise. */
bchol_status_t bchol_batch_set_member_precision(bchol_batch_t batch, int count, const int* precision);

/* Schedule query of one system of a batch (host only): the batched kernel
 * walks each system's tasks in the ticket order of bchol_plan_task with tile
 * 64 (no diagonal chain), claiming whichever system's next task is ready.
 * With BCHOL_FP64_SPLIT and tile 16 or 32 the updates of each block column
 * are strips, type 3 = STRIP(I, J, s) of the tiles I .. min(I+H-1, s+m),
 * H = 128/tile, each at the place of its first tile.  Count: -1 on bad
 * arguments (n >= 1, k >= 0, tile 16/32/64, precision FP64 or FP64_SPLIT). */
/* The batched solve's group for one system (host only): with P = ceil(k/32)
 * blocks of 32 rows below each diagonal block (at most ceil(n/32) - 1), a
 * leader CTA runs the substitution chain and the far terms at block distance
 * 2, and `workers` extra CTAs (0 when P < 5) take the distances >= 3, worker
 * w = 1..workers the distances 3 + (w-1) span .. min(P, 2 + w span).  Each
 * worker passes its partial sums through a ring of `slots` slots.  ctas > 0:
 * the CTAs the solve launch keeps resident; no group is planned larger than
 * that (bchol_batch_plan uses the device's count).  BCHOL_ERR_ARG for n < 1,
 * k < 0 or a null pointer. */
bchol_status_t bchol_batch_solve_group(int n, int k, int ctas, int* workers, int* span, int* slots);

long long bchol_batch_plan_task_count(int n, int k, int tile, int precision);
bchol_status_t bchol_batch_plan_task(int n, int k, int tile, int precision, long long ticket, int* type, int* s,
                                     int* I, int* J);

/* bchol_factor_batched -- plan + run in one call with the handle's own batch
 * object and its tile / CTA settings (arguments as for bchol_batch_plan). */
bchol_status_t bchol_factor_batched(bchol_handle_t handle, int count, const int* n, const int* k, double* const* ab,
                                    const int* ldab, int* info_dev, const int* nrhs, double* const* b,
                                    const int* ldb);

/* Wait for the handle's stream, copy `count` device info words to
 * info_host, and return BCHOL_ERR_TIMEOUT if a bounded wait ran out since the
 * last call, else BCHOL_ERR_NOT_SPD if any info > 0, else BCHOL_OK.  Clears
 * the timeout record. */
bchol_status_t bchol_get_info(bchol_handle_t handle, const int* info_dev, int count, int* info_host);

/* Settings.  tile: 0 = automatic, else 16, 32 or 64.  wait_limit_ms: the time
 * budget of one in-kernel wait (default 2000 ms).  ctas_per_sm: persistent
 * CTAs per SM for the factor kernel (0 = automatic). */
bchol_status_t bchol_set_tile(bchol_handle_t handle, int tile);

/* Precision mode of the handle's factorizations (bchol_precision_t above).
 * max_refine (>= 0) and tol (>= 0) bound the iterative refinement of
 * BCHOL_FP32_UPDATE solves: corrections stop when the relative residual
 * max_c ||b_c - A x_c|| / ||b_c|| is <= tol, stops shrinking, or after
 * max_refine corrections; the other modes ignore them.  Returns BCHOL_ERR_ARG
 * for an unknown mode or bad bounds, BCHOL_ERR_UNSUPPORTED for
 * BCHOL_TF32_UPDATE (the mode is then unchanged).
 * In the BCHOL_FP32_UPDATE mode (the steps of bchol_solve_mixed, split in two):
 *   bchol_factor  equilibrates a copy of A in the handle's workspace,
 *                 S A S with S = diag(A)^{-1/2}, and factors the copy with
 *                 FP32-accumulated updates; ab is read, not overwritten, and
 *                 info_dev is that factorization's info;
 *   bchol_solve   must then be called with the same n, k, ab and ldab (ab
 *                 still holding A) on the same handle, before any other
 *                 factorization on it, else it returns BCHOL_ERR_ARG; it
 *                 returns BCHOL_ERR_NOT_SPD if that factorization failed.  It
 *                 overwrites B with X, refined in FP64 against A, 16 columns
 *                 at a time, and synchronises the stream (the refinement
 *                 reads residual norms on the host).
 * The workspace of this mode holds the copy of the band besides the usual
 * scratch (bchol_workspace_size accounts for it). */
bchol_status_t bchol_set_precision(bchol_handle_t handle, bchol_precision_t precision, int max_refine, double tol);

/* Refinement record of the last BCHOL_FP32_UPDATE bchol_solve on the handle:
 * corrections made (the largest over its 16-column groups), final relative
 * residual max_c ||b_c - A x_c|| / ||b_c|| and last relative correction
 * max_c ||d_c|| / ||x_c||. */
bchol_status_t bchol_last_refinement(bchol_handle_t handle, int* iters, double* resid, double* corr);
bchol_status_t bchol_set_wait_limit_ms(bchol_handle_t handle, int wait_limit_ms);
bchol_status_t bchol_set_ctas_per_sm(bchol_handle_t handle, int ctas_per_sm);

/* Algorithm of bchol_solve's FP64 sweeps (the result is the same to rounding):
 *   0  automatic (the default): partitioned for 1 <= k <= 112 and n >= 2048, else cluster
 *   1  cluster: the 32-row block chain on one thread-block cluster per group of
 *      right-hand sides, far blocks on the cluster's worker CTAs.  A one-column
 *      solve with more than 16 blocks of band below the diagonal (k > 512) adds
 *      up to 6 more 16-CTA clusters that take the block distances past 16 and
 *      hand their sums over through the workspace, with waits bounded by the
 *      handle's wait limit (a wait that runs out is reported by bchol_get_info
 *      as BCHOL_ERR_TIMEOUT, and the solution is then not valid)
 *   2  partitioned (for 1 <= k <= 112; other k use the cluster path): chunks of
 *      256 rows solved independently, with k "spike" columns L_cc^{-1} L_{c,c-1}
 *      per chunk, a sequential pass over the chunks' k boundary values, and a
 *      second independent pass; n (k + nrhs) k multiply-adds per sweep
 *   3  cluster as in 1, always on one cluster per group (no far clusters)
 * Returns BCHOL_ERR_ARG for other values. */
bchol_status_t bchol_set_solve_path(bchol_handle_t handle, int path);

/* bchol_set_tile_staging -- how the diagonal chain's prefetch warps copy the
 * tiles A(s, s) and A(s, s-1) of each step into shared memory (tiles of 16
 * and 32): 0 plain coalesced loads; 1 (default) TMA (cp.async.bulk.tensor box
 * copies over the band viewed as a 2-D tensor with column stride ldab - 1, on
 * an mbarrier), used where ldab is odd and > 1 and the driver encodes the
 * tensor map, else the plain loads.  bchol_last_tile_staging returns 1 if the last
 * bchol_factor's chain used TMA, 0 if not, -1 for a null handle.
 * BCHOL_ERR_ARG for other values. */
bchol_status_t bchol_set_tile_staging(bchol_handle_t handle, int tma);
int bchol_last_tile_staging(bchol_handle_t handle);

/* Test hook for the failure path.  While set to a tile (I, J) >= 0, the
 * factor kernel's waits on the ready flag of tile (I, J) (b x b tiles, block
 * row I, block column J, 0 <= I-J <= ceil(k/b)) get a target that is never
 * reached, so the first such wait runs out after the wait limit: the kernel
 * stops cleanly and bchol_get_info reports BCHOL_ERR_TIMEOUT.  (-1, -1)
 * turns it off (the default). */
bchol_status_t bchol_set_stall_tile(bchol_handle_t handle, int I, int J);

/* Schedule query (host only, no GPU needed).  The factor kernel walks the
 * tasks of the tiled factorization in ticket order.  Step s (one outer
 * iteration of Algorithm 1, Sec. 3) has POTRF(s) (type 0), TRSM(I, s) for the
 * panel rows I = s+1..s+m (type 1) and the updates UPD(I, J, s),
 * A_IJ -= L_Is L_Js^T, for s < J <= I <= s+m (type 2), with
 * m = min(ceil(k/tile), ceil(n/tile)-1-s).  Tickets run with one step of
 * lookahead: panel 0, then per step s the updates of column s+1, the panel of
 * step s+1, then the other updates of step s.  bchol_plan_task_count returns
 * the number of tasks (or -1 on bad arguments); bchol_plan_task decodes one
 * ticket into (type, s, I, J) in tile units.  tile is 16, 32 or 64. */
long long bchol_plan_task_count(int n, int k, int tile);
bchol_status_t bchol_plan_task(int n, int k, int tile, long long ticket, int* type, int* s, int* I, int* J);
/* The same for a precision mode: with BCHOL_FP64_SPLIT and tile 16 or 32 the
 * updates of each block column run as strips, type 3 = STRIP(I, J, s): the
 * updates UPD(I', J, s) of the tiles I' = I .. min(I+H-1, s+m), H = 128/tile. */
long long bchol_plan_task_count_ex(int n, int k, int tile, int precision);
bchol_status_t bchol_plan_task_ex(int n, int k, int tile, int precision, long long ticket, int* type, int* s, int* I,
                                  int* J);

/* The task order of the adjoint's selected inversion (bchol_backward), for
 * tests: the number of tasks for (n, k, tile) (or -1 on bad arguments), and
 * ticket -> (type, J, I, g) in tile units: type 0 = FAR(I, J, group g) (far
 * terms of P_IJ = sum_M Sigma_IM L_MJ), 1 = NEAR(I, J) (Sigma_IJ and its share of
 * E_J), 2 = DIAG(J) (the diagonal tile); block columns J run from last to first
 * (the Takahashi recurrences of the inverse's band; the paper's interior-point
 * motivation, Sec. 1).  The order is the launch's combined order: CTA 0 runs
 * NEAR(J+1, J) and DIAG(J) of every column itself (the chain), placed after the
 * column's other NEAR tasks and before the far terms that read DIAG(J); the
 * other tasks are tickets.  tile is 16, 32 or 64. */
long long bchol_adjoint_plan_task_count(int n, int k, int tile);
bchol_status_t bchol_adjoint_plan_task(int n, int k, int tile, long long ticket, int* type, int* J, int* I, int* g);

/* Self-check of the reciprocal the diagonal POTRF's pivot recurrence uses
 * (d_{j+1} = A(j+1,j+1) - A(j+1,j)^2 / d_j, the Schur complement of Sec. 3's
 * POTRF step): y[i] = 1/x[i] by that routine, for n device doubles x (n >= 0;
 * x and y device pointers, caller-owned, may not overlap).  Asynchronous on
 * the handle's stream.  For positive normal x the relative error is a few
 * units in the last place; tests compare it with IEEE division.  Returns
 * BCHOL_ERR_ARG on a null handle or pointer with n > 0. */
bchol_status_t bchol_check_pivot_rcp(bchol_handle_t handle, const double* x, double* y, int n);

/* Self-check of the tensor-core split product that the BCHOL_FP64_SPLIT
 * precision mode uses for the trailing updates A_IJ -= L_Is L_Js^T of
 * Algorithm 1 (Sec. 3; the O(n k^2) part of Eq. (1)):
 *     C := C - A B^T,  A m x 32, B n x 32, C m x n,
 * all column-major device doubles owned by the caller (lda >= max(1,m),
 * ldb >= max(1,n), ldc >= max(1,m); C may not overlap A or B).  Each FP64
 * entry is cut into seven balanced 8-bit digits under a per-row power-of-two
 * scale (Ozaki-style error-free splitting); the 28 digit products that carry
 * FP64 precision run as exact bf16 MMAs with FP32 accumulation in tensor
 * memory, and their sum is formed in 64-bit fixed point.  Each result is
 * accurate to about 32 * 2^-54 * max_k |A(i,k)| * max_k |B(j,k)| plus the
 * rounding of the FP64 update; integer-valued inputs whose products and sums
 * fit in 53 bits give exact results.  A non-finite entry in row i of A or row j
 * of B makes C(i,j) NaN.  Asynchronous on the handle's stream; a bounded
 * in-kernel wait that runs out is reported by bchol_get_info as
 * BCHOL_ERR_TIMEOUT.  Returns BCHOL_ERR_ARG on bad sizes or null pointers. */
bchol_status_t bchol_check_split_product(bchol_handle_t handle, int m, int n, const double* A, int lda,
                                         const double* B, int ldb, double* C, int ldc);

/* Throughput probe for the roofline denominators (not part of the paper's
 * method): runs, on every SM, a loop of one instruction kind with independent
 * accumulators and returns the delivered rate in TFLOP/s (synchronises):
 *   kind 0  FP64 FMA (the unit of POTRF, TRSM and the FP64 updates)
 *   kind 1  FP64 MMA, mma.sync m8n8k4 .f64 (shares the FP64 unit)
 *   kind 2  FP32 FMA (the FP32_UPDATE mode's updates)
 *   kind 3  bf16 tensor-core MMA, tcgen05.mma M = 128, N = 256, K = 16 with FP32
 *           accumulators in tensor memory (the split updates' instruction)
 * iters >= 1 sets the loop length (tens of milliseconds: 20000 for kinds 0-1,
 * 500000 for 2-3).  Allocates a small scratch buffer with cudaMalloc.  Returns
 * BCHOL_ERR_ARG on bad arguments, BCHOL_ERR_TIMEOUT if the tensor-core wait ran out. */
bchol_status_t bchol_probe_rate(bchol_handle_t handle, int kind, int iters, double* tflops);

/* Number of factor-kernel and solve-kernel launches made by the last call on
 * this handle (for launch accounting). */
int bchol_last_launch_count(bchol_handle_t handle);

/* Library version string. */
const char* bchol_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BCHOL_H */
