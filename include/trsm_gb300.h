/*
 * trsm_gb300.h — C ABI of a single-GPU (GB300, sm_103a) triangular solver
 * with many right-hand sides by selective diagonal-block inversion, after
 * Wicky, Solomonik & Hoefler, "Communication-Avoiding Parallel Algorithms for
 * Solving Triangular Systems of Linear Equations", arXiv:1612.01855.
 *
 * Problem (Section 1): L X = B with L n x n lower-triangular, B and X n x k
 * dense.  Left side, lower, not transposed, non-unit diagonal: the only case
 * the paper treats.
 *
 * Conventions shared by every call:
 *   - FP64 matrices are column-major: element (i, j) of M with leading
 *     dimension ld is M[j*ld + i]; ld >= max(1, rows).  Only the lower
 *     triangle of L (diagonal included) is read; its strict upper triangle
 *     is never touched.
 *   - Pointers named *_dev are device pointers of the current CUDA device;
 *     *_host are host pointers (pinned or pageable).  The library never
 *     retains a caller pointer beyond the call unless stated.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it; calls marked "synchronous"
 *     wait for their own work before returning.
 *   - Return value: TRSM_SUCCESS (0) or a negative TRSM_E* code.  A failing
 *     call leaves outputs unspecified and frees what it allocated.
 */
#ifndef TRSM_GB300_H
#define TRSM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define TRSM_SUCCESS 0
#define TRSM_EINVAL (-1)     /* bad size, leading dimension, pointer or option   */
#define TRSM_ESINGULAR (-2)  /* a diagonal entry of L is zero, Inf or NaN        */
#define TRSM_ENOMEM (-3)     /* device or host allocation failed                 */
#define TRSM_ECUDA (-4)      /* a CUDA runtime call failed (see trsm_last_cuda)  */
#define TRSM_ETIMEOUT (-5)   /* a device-side dependency wait hit its time limit */
#define TRSM_ENOSCRATCH (-6) /* trsm_solve_noalloc: workspace exceeds its fixed scratch */
#define TRSM_ENOCONV (-7)    /* trsm_solve_mixed: refinement did not converge        */

/* Low-precision formats of the mixed-precision solve (tensor-core updates). */
#define TRSM_INNER_BF16 1
#define TRSM_INNER_TF32 2
/* split bf16: every operand is hi + lo bf16 planes and the update takes the
 * three products hi*hi + hi*lo + lo*hi (about 16 significant bits per factor
 * at 1.5x the tensor work of tf32): the inner solve contracts the error far
 * faster on ill-conditioned systems */
#define TRSM_INNER_BF16X3 3
/* split fp16: hi + lo fp16 planes, three products (about 22 significant bits
 * per factor); the panels and each block row of the correction are scaled by
 * powers of two into fp16's range and the update undoes both */
#define TRSM_INNER_FP16X3 4
/* Residual of the mixed-precision solve. */
#define TRSM_RESIDUAL_SLICED 0   /* FP64-class, bf16 tensor cores, 7 integer digit planes */
#define TRSM_RESIDUAL_FP64 1     /* FP64 fused multiply-add                                */
#define TRSM_RESIDUAL_SLICED8 2  /* as SLICED with 8 digit planes: ~2^-49 instead of ~2^-43 */
#define TRSM_RESIDUAL_ADAPTIVE 3 /* SLICED until the updates stagnate above tol or their contraction
                                    stalls (an update ten times above the last contraction's
                                    prediction), then SLICED8 */
/* As ADAPTIVE, but an early residual takes 5 or 6 digit planes (15 or 21
 * plane products instead of 28; about 2^-31 and 2^-37 of |B| + |L||X|)
 * while the iterate's error, estimated from the last update and its
 * contraction, is far above what they resolve; 7 planes after that, 8 once
 * the updates stagnate. */
#define TRSM_RESIDUAL_PROGRESSIVE 4
/* Flag or-ed into `residual`: apply the FP64 inverses of the diagonal blocks
 * in FP32 arithmetic inside the inner solve (default: FP64 arithmetic). */
#define TRSM_SOLVE_S_FP32 0x100
/* Flag or-ed into `residual` (not with TRSM_SOLVE_S_FP32): apply them on the
 * tensor cores: the inverse and W_i are each cut into three tf32 planes and
 * the six plane products of weight 2^-22 and above are summed in FP32
 * (FP32-class, about 2^-24 per product). */
#define TRSM_SOLVE_S_TC 0x200
/* As TRSM_SOLVE_S_TC with two tf32 planes per factor and the three products
 * of weight 2^-11 and above (hi hi, hi mid, mid hi: about 2^-21 per product,
 * the accuracy of the split-fp16 and split-bf16 updates), or with the hi
 * planes alone (tf32, about 2^-11: the accuracy of the tf32 and bf16
 * updates).  At most one of the three tensor-core flags. */
#define TRSM_SOLVE_S_TC2 0x400
#define TRSM_SOLVE_S_TC1 0x800

/* Opaque plan: the paper's L~ (Algorithm Diagonal-Inverter, Section 6.1) —
 * a device copy of L whose n0 x n0 diagonal blocks are replaced by their
 * inverses — plus sizes.  It owns its device memory. */
typedef struct trsm_plan_s* trsm_handle_t;

/* trsm_plan — Algorithm Diagonal-Inverter (Section 6.1) with Algorithm
 * RecTriInv (Section 5.1) for every diagonal block.
 *   L_dev  : device, n x n column-major, leading dimension ldl >= n.  Read
 *            only; the caller may free it once trsm_plan has returned.
 *   n      : order of L, n >= 1.
 *   n0     : diagonal block size, 1 <= n0 (n0 >= n means one block, the full
 *            inversion; a last block shorter than n0 is allowed).
 *   out    : receives the handle (NULL on failure).
 * Synchronous: waits for the inversion so that a singular L is reported as
 * TRSM_ESINGULAR (trsm_singular_index gives the row).  Errors: TRSM_EINVAL,
 * TRSM_ESINGULAR, TRSM_ENOMEM, TRSM_ECUDA. */
int trsm_plan(const double* L_dev, int64_t n, int64_t ldl, int64_t n0, void* stream,
              trsm_handle_t* out);

/* trsm_solve — Algorithm It-Inv-TRSM (Section 6.2) with the plan's L~:
 * for every block row i, X_i = L~_ii (B_i - L_{i,<i} X_{<i}).
 *   B_dev : device, n x k, leading dimension ldb >= n; read only.
 *   X_dev : device, n x k, leading dimension ldx >= n; written.  X_dev may
 *           equal B_dev with ldx == ldb (in place); other overlaps are
 *           undefined.
 *   k     : number of right-hand sides, k >= 0 (k == 0 is a no-op).
 * Asynchronous on `stream`; it allocates its workspace (n x k doubles plus
 * dependency counters) stream-ordered and frees it stream-ordered.  A
 * device-side wait that times out is reported by trsm_sync_status.
 * Errors (immediate): TRSM_EINVAL, TRSM_ENOMEM, TRSM_ECUDA. */
int trsm_solve(trsm_handle_t h, const double* B_dev, int64_t k, int64_t ldb, double* X_dev,
               int64_t ldx, void* stream);

/* trsm_solve_schedule — trsm_solve with a chosen schedule of the same
 * arithmetic (all read the plan's L~; results agree to rounding):
 *   TRSM_SCHED_DAG            the default: one persistent kernel, tile tasks
 *                             ordered by dependency counters (trsm_solve);
 *   TRSM_SCHED_RIGHT_LOOKING  Algorithm It-Inv-TRSM (Section 6.2) as
 *                             written, with the update accumulator B~ and the
 *                             subtraction of one block row per step; the next
 *                             block row's update runs first, the rest of the
 *                             trailing update on a second stream (look-ahead);
 *   TRSM_SCHED_RECURSIVE      Algorithm Rec-TRSM (Section 4): halve on block
 *                             boundaries, X1 = Rec(L11,B1), B2 -= L21 X1,
 *                             X2 = Rec(L22,B2); the base case X = L^-1 B uses
 *                             the plan's inverted diagonal block.
 *   TRSM_SCHED_SLICED         It-Inv-TRSM in its right-looking order with
 *                             both matrix multiplies, X_i = L~_ii W_i and
 *                             W(T_{i+1}) -= L(T_{i+1}, S_i) X_i, on the BF16
 *                             tensor cores: each factor is split into eight
 *                             6-bit integer digit planes with a power-of-two
 *                             exponent per row (per row and block column for
 *                             L), the 36 plane pairs of weight >= 2^-42 are
 *                             multiplied with exact FP32 sums, and the
 *                             results are combined and applied in FP64.
 *                             Each product carries about 2^-49 of |A| |B|
 *                             (an FP64-class result, not FP64 rounding).
 *                             Needs trsm_plan_sliced on the plan first
 *                             (else TRSM_EINVAL) and k <= 5242800; X_dev
 *                             may equal B_dev with ldx == ldb.
 * B_dev must not alias X_dev for RIGHT_LOOKING and RECURSIVE.  Asynchronous;
 * allocates its workspace stream-ordered.  Errors as trsm_solve. */
#define TRSM_SCHED_DAG 0
#define TRSM_SCHED_RIGHT_LOOKING 1
#define TRSM_SCHED_RECURSIVE 2
#define TRSM_SCHED_SLICED 3
int trsm_solve_schedule(trsm_handle_t h, const double* B_dev, int64_t k, int64_t ldb, double* X_dev,
                        int64_t ldx, int schedule, void* stream);

/* trsm_plan_sliced — adds the data of TRSM_SCHED_SLICED to a plan (no
 * counterpart in the paper, which assumes exact arithmetic: this is the
 * digit splitting of Ozaki, Ogita, Oishi & Rump, 2012, applied to the two
 * matrix multiplies of It-Inv-TRSM, Section 6.2).  From the plan's L~ it
 * makes eight bf16 digit planes of L off the diagonal blocks (16 n^2 bytes)
 * and of the rows of the inverted diagonal blocks (16 n n0 bytes), counted
 * by trsm_plan_device_bytes and freed by trsm_destroy.  The block order must
 * be a multiple of 64 and at most 2048, or the plan a single block (n0 >= n)
 * of order at most 2048 (else TRSM_EINVAL).  A second call is a no-op.
 * Synchronous.  Errors: TRSM_EINVAL, TRSM_ENOMEM, TRSM_ECUDA. */
int trsm_plan_sliced(trsm_handle_t h, void* stream);

/* Workspace-explicit form of trsm_solve: the caller passes device memory
 * `ws_dev` of at least trsm_solve_workspace_size(h, k) bytes (256-byte
 * aligned); nothing is allocated.  Concurrent calls must not share ws_dev. */
int trsm_solve_workspace_size(trsm_handle_t h, int64_t k, size_t* bytes);
int trsm_solve_ws(trsm_handle_t h, const double* B_dev, int64_t k, int64_t ldb, double* X_dev,
                  int64_t ldx, void* ws_dev, size_t ws_bytes, void* stream);

/* trsm_solve_noalloc — trsm_solve that allocates nothing.  The paper has no
 * counterpart: this exists for callers that may not allocate device memory
 * while solving (an application or server that owns all GPU memory through
 * its own arena, or a latency-critical loop that cannot afford an
 * allocation's device synchronisation or pool growth).
 *   Same arguments, result and layout rules as trsm_solve; the current device
 *   must be the plan's device (else TRSM_EINVAL).
 *   Workspace: a fixed 64 MiB device array compiled into the library (held on
 *   every GPU that loads it until the process exits).  If
 *   trsm_solve_workspace_size(h, k) exceeds 64 MiB the call returns
 *   TRSM_ENOSCRATCH before any device work.
 *   All calls on a device share that array and find the previous call's data
 *   there; each call resets what must start at zero.  Calls whose device work
 *   overlaps (other streams, other host threads) race: serialise them.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it together
 *   with the id of the CUDA context it belongs to; make it before any stream
 *   capture begins.  After a cudaDeviceReset the next call sees a new
 *   context and looks the address up again (so it, too, belongs before any
 *   capture).
 * Asynchronous on `stream`.  Errors: TRSM_EINVAL, TRSM_ENOSCRATCH,
 * TRSM_ECUDA. */
int trsm_solve_noalloc(trsm_handle_t h, const double* B_dev, int64_t k, int64_t ldb,
                       double* X_dev, int64_t ldx, void* stream);

/* trsm_plan_mixed — adds the data of the mixed-precision solve to a plan
 * (no counterpart in the paper, which works in exact arithmetic; the block
 * structure is its Algorithm It-Inv-TRSM):
 *   - the off-diagonal block columns L(T_{i+1}, S_i) in `inner` precision
 *     (TRSM_INNER_BF16, TRSM_INNER_TF32, TRSM_INNER_BF16X3 or
 *     TRSM_INNER_FP16X3), for the tensor-core updates;
 *   - the original diagonal blocks and diagonal of L in FP64;
 *   - FP32 copies of the plan's inverted diagonal blocks L~_ii (n x n0
 *     floats), for the FP32 diagonal-block multiply, and three tf32 planes
 *     of them (3 n x n0 floats), for the tensor-core one;
 *   - eight 6-bit integer digit planes of the strictly lower L, for the
 *     FP64-class residual.
 *   L_dev : the same matrix the plan was made from (n x n, ldl >= n).
 * Synchronous.  Errors: TRSM_EINVAL, TRSM_ENOMEM, TRSM_ECUDA. */
int trsm_plan_mixed(trsm_handle_t h, const double* L_dev, int64_t ldl, int inner, void* stream);

/* trsm_solve_mixed — X = L^-1 B by iterative refinement around a
 * low-precision solve: X = 0, R = B; repeat D = inner_solve(R), X += D,
 * R = B - L X, until max|D| <= tol * max|X| or the updates stagnate (an
 * update larger than half the previous one: the residual's accuracy floor
 * is reached; accepted when max|D|/max|X| <= 1e-10).  inner_solve follows
 * It-Inv-TRSM (Section 6.2) in its right-looking order: per block row,
 * D_i = L~_ii W_i with the FP64 inverse (FP64 arithmetic), then the trailing
 * update W(T_{i+1}) -= L(T_{i+1}, S_i) D_i as one tcgen05 GEMM in the plan's
 * inner precision with FP32 accumulation (W is the FP32 copy of R).
 *   residual : TRSM_RESIDUAL_SLICED, _SLICED8, _ADAPTIVE, _PROGRESSIVE or _FP64 (the
 *              latter needs n0 a multiple of 32 when there is more than one
 *              block), optionally or-ed with TRSM_SOLVE_S_FP32 or
 *              one of TRSM_SOLVE_S_TC, _TC2, _TC1.  The
 *              residual's accuracy sets the attainable error: about
 *              cond * 2^-43 (SLICED), cond * 2^-49 (SLICED8), cond * 2^-53
 *              (FP64), with cond the componentwise condition of the system
 *              (the sliced residuals are componentwise only within a
 *              2048-row chunk of X: a solution whose entries span many
 *              orders of magnitude inside a chunk sees a normwise bound).
 *   max_iter : >= 1 inner solves at most; tol >= 0.
 *   iters, last_update (may be NULL): inner solves done, and the last
 *              max|D| / max|X|.
 *   B_dev must not alias X_dev.  Requires trsm_plan_mixed.  Synchronous.
 * Errors: TRSM_EINVAL, TRSM_ENOMEM, TRSM_ECUDA, TRSM_ETIMEOUT, and
 * TRSM_ENOCONV when the updates stop shrinking, turn non-finite or the
 * iteration limit is reached (X then holds the last iterate). */
int trsm_solve_mixed(trsm_handle_t h, const double* B_dev, int64_t k, int64_t ldb, double* X_dev,
                     int64_t ldx, int residual, int max_iter, double tol, int* iters,
                     double* last_update, void* stream);

/* ---- Many independent systems in one persistent launch ----
 * Each item is Algorithm It-Inv-TRSM (Section 6.2) on its own system; the
 * systems may differ in n, k and block size.  An item either carries a
 * resident plan (its inverted blocks are reused: no inversion work) or its
 * own L, whose n0 x n0 diagonal blocks (n0 = 32 or 64) are inverted inside
 * the same launch by Algorithm RecTriInv (Section 5.1, one level).  An
 * FP64 run is one memset and one persistent kernel of dependent tile tasks;
 * an FP32 run is one memset and two kernels (every diagonal block inverted
 * once, then one CTA per system and column chunk).  Either can be captured
 * in a CUDA graph, and the results do not depend on which other items share
 * the launch (every output's sums are taken in a fixed order). */
#define TRSM_F64 0
#define TRSM_F32 1

typedef struct trsm_batch_item {
  const void* L;        /* device, n x n column-major (ignored when plan != NULL) */
  int64_t ldl;
  trsm_handle_t plan;   /* resident plan for this L (FP64 batches only), or NULL */
  const void* B;        /* device, n x k, read only; must not alias X          */
  int64_t ldb;
  void* X;              /* device, n x k, written                              */
  int64_t ldx;
  int64_t n, k;
  int64_t n0;           /* 32 or 64 when plan == NULL (ignored otherwise)      */
  int64_t tile_cols;    /* columns per output tile: FP64 1 to 3 or a
                           multiple of 4 up to 32, FP32 (per CTA) 8, 16 or
                           32; 0 = fitted
                           to k (the narrowest width that holds k <= 32, else
                           32-wide tiles and, when 32 does not divide k, one
                           fitted tile for the remainder; results are the
                           same bits either way) */
} trsm_batch_item;

typedef struct trsm_batch_s* trsm_batch_t;

/* Validates the items, lays out the workspace (working copies of B, the
 * inverted blocks of plan-less items, dependency counters) and uploads the
 * task table.  Pointers in the items are retained by the batch: they must
 * stay valid while it is run.  dtype: TRSM_F64 (double data) or TRSM_F32
 * (float data; plan-less items only).  Errors: TRSM_EINVAL, TRSM_ENOMEM,
 * TRSM_ECUDA. */
int trsm_batch_create(const trsm_batch_item* items, int count, int dtype, trsm_batch_t* out);

/* Allocation-free form for a caller-managed arena (e.g. a server that
 * admits work against a memory budget): trsm_batch_workspace_size gives the
 * bytes the items need (task tables included); trsm_batch_create_ws lays
 * the batch out in ws_dev (256-byte aligned, >= that size, owned by the
 * caller and not freed by trsm_batch_destroy) and uploads its tables on
 * `stream`.  A batch made this way must run on the same stream (or after
 * it).  Same errors as trsm_batch_create. */
int trsm_batch_workspace_size(const trsm_batch_item* items, int count, int dtype, size_t* bytes);
int trsm_batch_create_ws(const trsm_batch_item* items, int count, int dtype, void* ws_dev, size_t ws_bytes,
                         void* stream, trsm_batch_t* out);

/* Enqueues one solve of every item (asynchronous). */
int trsm_batch_run(trsm_batch_t b, void* stream);

/* Records trsm_batch_run into a CUDA graph held by the batch (on a private
 * stream; `stream` is unused and may be NULL); trsm_batch_launch_graph
 * replays it on `stream`. */
int trsm_batch_capture(trsm_batch_t b, void* stream);
int trsm_batch_launch_graph(trsm_batch_t b, void* stream);

/* Waits for `stream`; returns TRSM_SUCCESS, TRSM_ETIMEOUT (a device wait ran
 * out) or TRSM_ESINGULAR with the first failing item and its row. */
int trsm_batch_status(trsm_batch_t b, void* stream, int* first_bad_item, int64_t* singular_row);

void trsm_batch_destroy(trsm_batch_t b);

/* Device bytes the batch holds. */
size_t trsm_batch_workspace_bytes(trsm_batch_t b);

/* trsm_host — the whole method (trsm_plan + trsm_solve) on HOST buffers:
 * copies L and B to the device, plans, solves, copies X back and waits.
 * Only the lower trapezoid of each n0-wide block column of L is copied
 * (about half of L), straight into the plan's L~.  When B and X are large
 * against the number of block rows (16 n k bytes above 2.5e8 per block row,
 * k >= 4096) the columns of B go in four chunks: the solve of one chunk
 * overlaps the copy of the next one in and of the previous one out (two
 * extra streams).
 *   L_host (n x n, ldl), B_host (n x k, ldb), X_host (n x k, ldx), all
 *   column-major host memory; pinned memory makes the copies asynchronous
 *   and lets them overlap.  X_host may alias B_host (same ld).
 * Synchronous.  Errors as trsm_plan and trsm_solve. */
int trsm_host(const double* L_host, int64_t n, int64_t ldl, int64_t n0, const double* B_host,
              int64_t k, int64_t ldb, double* X_host, int64_t ldx, void* stream);

/* trtri_blocks — Algorithm Diagonal-Inverter's output in packed form: the
 * inverses of the N = ceil(n/n0) diagonal blocks L(S_b, S_b),
 * S_b = [b*n0, min((b+1)*n0, n)), each by RecTriInv (Section 5.1).
 *   Linv_dev : device, N*n0*n0 doubles, caller-owned; block b is the n0 x n0
 *              column-major matrix at Linv_dev + b*n0*n0 (leading dimension
 *              n0).  Its strict upper triangle is written as zero; a short
 *              last block occupies its leading m x m corner, the rest zero.
 * Synchronous.  Errors: TRSM_EINVAL, TRSM_ESINGULAR, TRSM_ENOMEM, TRSM_ECUDA. */
int trtri_blocks(const double* L_dev, int64_t n, int64_t ldl, int64_t n0, double* Linv_dev,
                 void* stream);

/* Releases the plan's device memory (after the work queued on it). */
void trsm_destroy(trsm_handle_t h);

/* Plan accessors.  trsm_plan_lt returns the device pointer of L~ (n x n,
 * leading dimension *ldt), owned by the plan: its diagonal blocks hold the
 * inverses, below them L itself, above the diagonal zeros. */
int trsm_plan_sizes(trsm_handle_t h, int64_t* n, int64_t* n0, int64_t* nblocks);
const double* trsm_plan_lt(trsm_handle_t h, int64_t* ldt);

/* Device bytes the plan holds: L~ and, after trsm_plan_mixed, the
 * mixed-precision data (panels, digit planes, diagonal blocks).  0 for a
 * null handle.  No counterpart in the paper: memory accounting for callers
 * that admit work against an HBM budget. */
size_t trsm_plan_device_bytes(trsm_handle_t h);

/* Workspace memory.  The per-call scratch of every solve, plan and batch
 * run (working copy of B, digit planes, counters) comes from a
 * stream-ordered memory pool the library owns, one per device.  Memory a
 * call frees stays reserved in the pool for the next call (the device's
 * default pool would unmap it at each synchronisation and the next call
 * would map it again, about 1 ms per GB), and is not handed to another
 * stream before its free has completed there.  No counterpart in the paper.
 *   trsm_workspace_trim: returns the current device's idle pool memory to
 *     the system until at most keep_bytes stay reserved (memory of calls
 *     still in flight stays).  TRSM_SUCCESS, also when the pool was never
 *     used; TRSM_ECUDA without a usable device.  An allocation the pool
 *     cannot satisfy trims the pool itself and retries once.
 *   trsm_workspace_reserved_bytes: bytes the current device's pool holds
 *     mapped (in use or idle); 0 without a device or before the first call. */
int trsm_workspace_trim(size_t keep_bytes);
size_t trsm_workspace_reserved_bytes(void);

/* Waits for `stream` and returns the device status of the last solve
 * enqueued with this plan: TRSM_SUCCESS or TRSM_ETIMEOUT. */
int trsm_sync_status(trsm_handle_t h, void* stream);

/* Row of the first zero or non-finite diagonal entry met by the last plan
 * or trtri_blocks on this thread, or -1. */
int64_t trsm_singular_index(void);

/* Last CUDA runtime error code seen by the library on this thread (0 if none). */
int trsm_last_cuda(void);

/* Human-readable text of a TRSM_* code (static storage). */
const char* trsm_error_string(int code);

/* Number of kernel launches the library enqueued on this thread since the
 * counter was last reset (for launch accounting around a timed region). */
int64_t trsm_launch_count(int reset);

/* Measures the device's FP64 fused-multiply-add throughput (no counterpart
 * in the paper: a roofline denominator).  Runs a DFMA-only kernel for about
 * `iters` x 8 x 2 flops per thread on every SM and writes TFLOP/s to
 * *tflops.  Synchronous. */
int trsm_fp64_peak(int iters, double* tflops, void* stream);

/* FP32 counterpart of trsm_fp64_peak (no counterpart in the paper: the
 * roofline denominator of the FP32 batches): an FFMA-only kernel, eight
 * independent chains per thread, 32 warps per SM, `iters` x 8 x 2 flops per
 * thread; writes TFLOP/s to *tflops.  Synchronous. */
int trsm_fp32_peak(int iters, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TRSM_GB300_H */
