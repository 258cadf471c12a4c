/*
 * mpcg.h -- C ABI of libmpcg: restarted mixed-precision conjugate gradient
 * for sparse SPD systems on NVIDIA GB300 (sm_103a).
 *
 * Method: Prolubnikov, "Parameter Optimization for Restarted Mixed-Precision
 * Iterative Sparse Solver" (arXiv 2412.08059).
 *   - Algorithm I (Sec. 1): CG (Sec. 3) on float32(A), float32(b) from x = 0
 *     until the residual reaches eps1; x0 = float64(x~); CG in double from
 *     x0, with r0 = b - A x0 recomputed in double, until eps2.
 *   - Algorithm II (Sec. 9): the first k0 single-precision iterations give
 *     the mean residual-decay ratio v (Eq. 13); with n, m and the 2BFS
 *     pseudo-diameter (Sec. 6) it forms chi = (n, m, l~, v); a
 *     distance-weighted kNN vote over a labelled sample (Sec. 11, Eq. 23)
 *     picks eps1 = 10^-t; the single-precision stage continues from
 *     iterate k0.
 *
 * Conventions (all entry points):
 *   - Every array argument is DEVICE memory owned by the caller unless the
 *     parameter says otherwise.  The library never allocates device memory:
 *     it carves the caller's workspace `ws` (size from mpcg_workspace_bytes).
 *   - Calls are stream-ordered on `stream` and never synchronise the host,
 *     except mpcg_batch_tune, which times batches.  The descriptor tables of
 *     mpcg_solve_batch and mpcg_batch_step travel inside kernel parameters,
 *     so the host buffers they are built in are free when the call returns.
 *     The workspace, the outputs and the inputs must stay valid until the
 *     stream reaches the end of the call's work.  Two calls that share a
 *     workspace must not overlap on the GPU.
 *   - The return value reports argument and launch errors found on the host
 *     (MPCG_ERR_INVALID_ARG, MPCG_ERR_WORKSPACE, MPCG_ERR_CUDA).  Numerical
 *     outcomes (convergence, breakdown, NaN, timeouts of device-side waits)
 *     are written to the device-side result record and are valid after the
 *     stream has synchronised.  Negative = error, positive = warning.
 *   - CSR input: row_ptr int32[n+1] (row_ptr[0] = 0, non-decreasing,
 *     row_ptr[n] = nnz), col int32[nnz] (0 <= col < n, sorted within each
 *     row, diagonal stored), val float64[nnz].  The matrix is assumed
 *     symmetric positive definite; the sparsity graph of Sec. 4 uses the
 *     stored off-diagonal entries.  A CSR that violates the index rules is
 *     reported as MPCG_ERR_INVALID_ARG in the result record (the device
 *     check skips the work, it never faults).
 *
 * Numerics of the single-precision stage (readings of the paper): SpMV sums
 * each row in stored order with single-precision fused multiply-adds; dot
 * products and norms are accumulated with at least double accuracy (Remark 3
 * of Sec. 9); alpha and beta are rounded once to float.  The stop test uses
 * the recursively updated residual, relative to ||b|| by default.
 */
#ifndef MPCG_H
#define MPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; 0 is the legacy default stream. */
struct CUstream_st;
typedef struct CUstream_st* mpcg_stream_t;

typedef enum {
  MPCG_OK = 0,
  MPCG_WARN_EPS1_NOT_REACHED = 1,     /* stage 1 stopped by its cap or a breakdown; switched anyway */
  MPCG_WARN_TRUE_RESID_RESTARTED = 2, /* recursive residual met eps2, true one did not: FP64 restarted */
  MPCG_ERR_INVALID_ARG = -1,
  MPCG_ERR_WORKSPACE = -2,            /* ws NULL, misaligned (256 B) or smaller than required */
  MPCG_ERR_BREAKDOWN = -3,            /* d^T A d <= 0 in the FP64 stage: A is not SPD */
  MPCG_ERR_NAN = -4,                  /* non-finite value in b, A or an iterate */
  MPCG_ERR_NOT_CONVERGED = -5,        /* FP64 stage reached max_it_fp64, or its true residual
                                         still missed eps2 after max_true_restarts restarts */
  MPCG_ERR_TIMEOUT = -6,              /* a device-side wait exceeded timeout_ms */
  MPCG_ERR_CUDA = -7,                 /* a CUDA launch or runtime call failed */
  MPCG_ERR_CANCELLED = -8,            /* the caller set the options' cancel word */
  MPCG_ERR_UNIMPLEMENTED = -9
} mpcg_status_t;

/* Sparse SPD matrix, CSR, device pointers, caller-owned (see conventions). */
typedef struct {
  int32_t n;
  int32_t nnz;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
} mpcg_csr_t;

/* Feature vector chi = (n, m, l~, v) of Sec. 4; m = stored nnz. */
typedef struct {
  double n, m, pdiam, v;
  int32_t k0_done; /* single-precision iterations that entered v */
  int32_t status;
} mpcg_features_t;

/* Labelled kNN sample S of Sec. 11: feat = raw features [count][4]
 * (device, float64, row-major), cls = class t per row (device, int8,
 * eps1 = 10^-t, 0 <= t <= 15), fmin/fmax = per-component min-max scaling
 * (host values, copied at call time).  count <= MPCG_KNN_MAX_SAMPLE. */
#define MPCG_KNN_MAX_SAMPLE 65536
#define MPCG_KNN_MAX_K 64
typedef struct {
  const double* feat;
  const int8_t* cls;
  int32_t count;
  double fmin[4], fmax[4];
} mpcg_sample_t;

typedef struct {
  double eps1;               /* > 0: Algorithm I with this eps1; <= 0: Algorithm II */
  double eps2;               /* final tolerance (default 1e-10) */
  int32_t k0;                /* iterations that define v (default 10) */
  int32_t knn_k;             /* neighbours (default 5, <= MPCG_KNN_MAX_K) */
  int32_t weighted;          /* 1: Eq. (23) vote (default); 0: Eq. (22) */
  int32_t tol_relative;      /* 1: ||r||/||b|| <= eps (default); 0: ||r|| <= eps */
  int32_t max_it_fp32;       /* cap on N1 including k0 (<= 0: n) */
  int32_t max_it_fp64;       /* cap on N2 (<= 0: 10 n) */
  int32_t max_true_restarts; /* extra FP64 restarts if the true residual misses eps2 (default 2);
                                if it still misses eps2 after the last one, the status is
                                MPCG_ERR_NOT_CONVERGED (x holds the last iterate) */
  uint32_t feat_mask;        /* bit c: feature c enters the distance (default 0xF) */
  int32_t fp64_only;         /* 1: pure FP64 CG from x0 = 0 (the baseline); no stage 1 */
  int32_t grid_blocks;       /* persistent grid size; 0 = one full wave of the device */
  int32_t timeout_ms;        /* limit of every device-side wait (default 20000) */
  int32_t stage1_only;       /* 1: stop after the single-precision stage; x = float64(x~) */
  int32_t team_rows;         /* batch and server: target rows per block of a team, which sets
                                the team size of each system (<= 0: 16384) */
  int32_t serve_split;       /* server, mixed precision: 1 = two launches per step (set-up,
                                features and the single-precision stage with its SpMV staged in
                                shared memory; then the FP64 stage); 0 = one launch (default) */
  int32_t bfs_starts;        /* 2BFS runs for l~ (the repeated 2BFS of Sec. 6: run r >= 1 starts
                                from floor(r n / R); l~ = the largest); <= 1: one run (default).
                                mpcg_solve and mpcg_features only: the batched solve and the
                                server refuse Algorithm II with bfs_starts > 1
                                (MPCG_ERR_UNIMPLEMENTED) */
  int32_t precond;           /* 1: Jacobi-preconditioned CG (M = diag A, the PCG form of Sec. 5)
                                in both stages; 0: plain CG (default).  mpcg_solve and
                                mpcg_features only (the batched solve and the server refuse it:
                                MPCG_ERR_UNIMPLEMENTED); Algorithm II then runs its steps as
                                separate launches in the paper's order.  The workspace grows by
                                16 n bytes: size it with these options */
  int32_t stop_true_residual; /* 1: every stop test on ||b - A x|| of the current iterate, the
                                loop test of the CG procedure as Sec. 3 prints it (in the
                                single-precision stage b~ - A~ x~ rounded in single precision;
                                one more pass over the matrix per iteration; the FP64 stage then
                                needs no true-residual restart); 0: on the recursively updated
                                r (default).  A stage whose recursive r has fallen 1e3 times
                                below ||b - A x|| has stagnated and ends as at its iteration
                                cap.  v (Eq. 13) stays on the recursive r.  mpcg_solve
                                and mpcg_features only (MPCG_ERR_UNIMPLEMENTED in the batched
                                solve and the server); Algorithm II then runs its steps as
                                separate launches in the paper's order */
  const volatile int32_t* cancel; /* NULL (default), or a word the GPU can read -- mapped pinned
                                host memory (cudaHostAlloc with cudaHostAllocMapped) or device
                                memory -- that the caller sets to non-zero to cancel the call
                                while its work runs.  mpcg_solve, mpcg_solve_static and
                                mpcg_features poll it at every CG iteration and in every
                                device-side wait; once they see it set, the call's work ends
                                with MPCG_ERR_CANCELLED in the result record (x then holds a
                                partial iterate).  A set word also cancels later calls that
                                pass it.  The batched solve and the server do not poll it
                                (the server cancels a system by retiring it between steps) */
  int32_t acc32;             /* 1: every inner product of the single-precision stage (r^T r,
                                d^T q, ||b~||) is summed in float: each thread sums its rows in
                                order, then a butterfly over the warp's lanes, the warps of a
                                block in index order, and the blocks in index order, every
                                add rounded to float.  0 (default): the same tree carried in
                                float-float and the blocks summed in double, the reading of
                                Sec. 9, Remark 3 (norms of the single-precision stage computed
                                in double).  The FP64 stage is the same either way */
  int32_t spmv_variant;      /* column format of the sliced SpMV layout (the only access to A
                                in the CG stages): 0 (default) = chosen per system at set-up:
                                16-bit offsets from the row when every entry kept in the
                                slices lies within 32767 columns of its row, 32-bit columns
                                otherwise; 1 = 32-bit columns always.  The single-system
                                kernels read the chosen format in both stages; the batched
                                solve and the server read it in the single-precision SpMV
                                that stages its pairs in shared memory (the batch's stage 1,
                                the server's split mode) and 32-bit columns elsewhere.  Both
                                formats sum the same entries in the same order, so x and every
                                count are bit-identical; 16-bit offsets move 6 instead of 8
                                bytes a stored entry in single precision, 10 instead of 12 in
                                double */
  const int32_t* team_rows_sys; /* batched solve only: NULL (default), or a host array of one
                                entry per system of the call, each that system's target rows
                                per block (its team size, as team_rows sets it for all; an
                                entry <= 0 takes team_rows).  mpcg_batch_tune writes one.  Read
                                during the call only */
} mpcg_options_t;

/* Result record, written by the device at the end of the call's work into
 * memory the device can write (device memory or mapped pinned host memory). */
typedef struct {
  int32_t status;
  int32_t n1;                /* single-precision iterations, k0 included */
  int32_t n2;                /* double-precision iterations, restarts included */
  int32_t cls;               /* kNN class t (-1 under Algorithm I) */
  int32_t k0_done;
  int32_t restarts;          /* extra FP64 restarts taken */
  double eps1;
  double true_rel_resid;     /* ||b - A x||_2 / ||b||_2 in FP64 */
  double pdiam;              /* 2BFS pseudo-diameter (Algorithm II) */
  double v;                  /* Eq. (13) */
  double res_fp32;           /* stop measure at the end of stage 1 */
  double res_fp64;           /* stop measure at the end of stage 2 */
  /* Device clock marks (ns): call start; eps1 known (features and kNN done;
   * in Algorithm II they run alongside stage 1); end of stage 1; end of
   * stage 2; result written; end of the set-up (demotion, sliced layout,
   * ||b||). */
  uint64_t t_start_ns, t_features_ns, t_fp32_ns, t_fp64_ns, t_end_ns, t_prep_ns;
  uint64_t t_stage2_ns;      /* start of the double-precision stage (the batched solve starts
                                it in its second launch; elsewhere the end of stage 1) */
  int32_t spmv_cols;         /* bits of a stored column that the single-precision SpMV read:
                                16 (offsets from the row) or 32 (option spmv_variant); 0 if the
                                set-up did not build the layout */
  int32_t team_blocks;       /* batched solve and server: blocks of the team that solved the
                                system (its tile shape); 0 in the single-system calls */
} mpcg_result_t;

mpcg_options_t mpcg_options_default(void);
const char* mpcg_status_string(int32_t status);

/* Device workspace bytes for an n x n matrix with nnz stored entries.  The
 * bound holds for every sparsity pattern with those counts.  0 on invalid
 * sizes.  Base pointers must be 256-byte aligned. */
size_t mpcg_workspace_bytes(int32_t n, int32_t nnz, const mpcg_options_t* opts);

/* Features of Algorithm II (Sec. 9 steps 1-3; Sec. 6 for l~): converts A and
 * b to float32, runs k0 single-precision CG iterations from x = 0 for v
 * (Eq. 13) and the 2BFS pseudo-diameter.  out: device mpcg_features_t. */
int32_t mpcg_features(const mpcg_csr_t* A, const double* b, const mpcg_options_t* opts,
                      void* ws, size_t ws_bytes, mpcg_features_t* out, mpcg_stream_t stream);

/* kNN choice of eps1 (Sec. 11): min-max scales f with the sample's
 * fmin/fmax, selects the k nearest by (squared distance, index), votes by
 * Eq. (23) or Eq. (22); a zero distance votes by count among the
 * zero-distance neighbours; vote ties go to the smallest t.  f: device
 * features; eps1_out (double) and cls_out (int32): device, nullable. */
int32_t mpcg_choose_eps1(const mpcg_features_t* f, const mpcg_sample_t* sample,
                         const mpcg_options_t* opts, double* eps1_out, int32_t* cls_out,
                         mpcg_stream_t stream);

/* The same kNN vote for many queries in one launch (classifying the test set
 * of the evaluation protocol of Sec. 12), one warp per query.  chi: device,
 * double[count][4], raw feature vectors (n, m, l~, v) as mpcg_features_t
 * gives them; cls_out: device int32[count], class t of each query, or -1 for
 * an invalid query (a non-finite selected feature).  nbr_out: device
 * int32[count][opts->knn_k], nullable: the indices of the query's nearest
 * sample points in selection order ((squared distance, index) ascending),
 * -1 past the sample's size -- what the localization measure of Sec. 11.4
 * counts.  count = 0 launches nothing.  MPCG_ERR_INVALID_ARG on a bad sample,
 * options or pointer. */
int32_t mpcg_knn_batch(const mpcg_sample_t* sample, const double* chi, int32_t count,
                       const mpcg_options_t* opts, int32_t* cls_out, int32_t* nbr_out,
                       mpcg_stream_t stream);

/* The method (Algorithm II, or Algorithm I when opts->eps1 > 0, or pure FP64
 * CG when opts->fp64_only): x (device, float64[n]) receives the solution;
 * its input value is ignored (x0 = 0).  sample: required by Algorithm II,
 * ignored otherwise.  res: device-writable result record.  In Algorithm II
 * the 2BFS and the kNN run alongside the single-precision iterations, which
 * keep going past k0 and keep the iterate at every candidate eps1; N1 and x~
 * are those of the paper's sequential order (k0 iterations, features, kNN,
 * CG from iterate k0 to eps1). */
int32_t mpcg_solve(const mpcg_csr_t* A, const double* b, double* x, const mpcg_sample_t* sample,
                   const mpcg_options_t* opts, void* ws, size_t ws_bytes, mpcg_result_t* res,
                   mpcg_stream_t stream);

/* Independent systems solved together in one persistent launch (a batching
 * pattern; the paper solves one system at a time).  A: host array of nsys
 * CSR descriptors (device pointers); b, x: host arrays of nsys device
 * pointers; res: device array of nsys records.  Every system gets its own
 * features, eps1 (Algorithm II when opts->eps1 <= 0, with `sample`) and
 * result record, with the same options (fp64_only: pure FP64 CG for every
 * system; stage1_only is refused with MPCG_ERR_UNIMPLEMENTED).  The grid is
 * split into teams of 1..128 blocks; each team takes systems from size-class
 * queues (largest
 * first) and runs the whole method on each, so systems of uneven size run
 * concurrently.  Workspace: mpcg_batch_workspace_bytes (a descriptor table,
 * then one region per system).  The descriptor table is copied from host
 * memory on `stream`; that copy may wait for earlier work on the stream.
 * Errors of one system (invalid CSR, NaN, breakdown) go to its own record;
 * a device-side wait that times out ends the launch, and the records of the
 * systems not finished stay as they were. */
size_t mpcg_batch_workspace_bytes(int32_t nsys, const int32_t* n, const int32_t* nnz,
                                  const mpcg_options_t* opts);
int32_t mpcg_solve_batch(int32_t nsys, const mpcg_csr_t* A, const double* const* b,
                         double* const* x, const mpcg_sample_t* sample,
                         const mpcg_options_t* opts, void* ws, size_t ws_bytes,
                         mpcg_result_t* res, mpcg_stream_t stream);

/* Plan of the batched solve (not in the paper; host only when grid_blocks > 0):
 * the team size (blocks) the planner of mpcg_solve_batch gives each system,
 * from n and nnz and the options' team_rows and team_rows_sys, for a grid of
 * grid_blocks blocks (0: the grid mpcg_solve_batch would launch with these
 * options on the current device).  A system goes to the smallest team (1, 2,
 * 4, ..., 128 blocks) with at most its rows per block; while one team of
 * every size present does not fit in the grid, the largest size present is
 * halved.  At run time a larger team may also take a system from a smaller
 * size's queue when its own is empty.  team_blocks_out: host int32[nsys].
 * MPCG_ERR_INVALID_ARG on bad arguments, MPCG_ERR_CUDA if grid_blocks is 0
 * and the device cannot be queried. */
int32_t mpcg_batch_plan(int32_t nsys, const int32_t* n, const int32_t* nnz,
                        const mpcg_options_t* opts, int32_t grid_blocks,
                        int32_t* team_blocks_out);

/* Autotuner of the batched solve (not in the paper): the tile shape of every
 * system, i.e. its team size.  Times mpcg_solve_batch with the given arguments
 * at each of MPCG_TUNE_CANDIDATES team granularities (opts->team_rows =
 * 8192, 16384, 32768, 65536 rows per block for every system; a system's team
 * is the smallest with at most that many rows per block) and writes the
 * fastest to *team_rows_out (host).  With team_rows_sys_out (host int32[nsys],
 * nullable) it then picks a granularity per system from those runs' device
 * clock marks: each system's busy time and block-time (team blocks x busy
 * time) under every candidate.  A host simulation of the launch (the
 * planner's teams taking systems from their class queues, then from the
 * smaller classes, as the kernel does) estimates the batch; starting from
 * the best uniform candidate, the systems with the largest block-time (at
 * most 256) each move to another candidate when that shortens the
 * simulated batch.  One more timed call with that choice
 * (opts->team_rows_sys) decides: if it is faster than the best uniform
 * candidate the per-system choice is written, else the uniform best for
 * every system.  ms_out (host float[MPCG_TUNE_RUNS], nullable): each
 * candidate's milliseconds, then the per-system call's (-1 if not run).
 * Pass the results in opts->team_rows and opts->team_rows_sys to later batch
 * calls over the same systems.  The column format of each system's SpMV is
 * its own set-up choice (option spmv_variant).  Unlike the other entry
 * points this call synchronises the host with `stream` (once per timed
 * call).  x and res hold the last call's results. */
#define MPCG_TUNE_CANDIDATES 4
#define MPCG_TUNE_RUNS (MPCG_TUNE_CANDIDATES + 1)
int32_t mpcg_batch_tune(int32_t nsys, const mpcg_csr_t* A, const double* const* b,
                        double* const* x, const mpcg_sample_t* sample,
                        const mpcg_options_t* opts, void* ws, size_t ws_bytes,
                        mpcg_result_t* res, mpcg_stream_t stream, int32_t* team_rows_out,
                        int32_t* team_rows_sys_out, float* ms_out);

/* ---- serving: continuous batching over a slot table (not in the paper) ----
 *
 * A server admits systems into slots and keeps each admitted system's
 * workspace (sliced matrix, Krylov vectors, control block) resident in a
 * device pool carved from the caller's workspace.  mpcg_batch_step advances
 * every admitted system in one persistent launch by at most max_iters CG
 * iterations per stage, through the phases below; systems in different
 * phases (set-up and features, single precision, double precision) run side
 * by side.  Between steps the host retires finished systems and admits new
 * ones.  Each system's result record, x and status are those of the same
 * method as mpcg_solve (Algorithm II with `sample` when opts->eps1 <= 0,
 * Algorithm I otherwise; fp64_only gives pure FP64 CG); its own eps2 is
 * given at admission.  The server handle is host memory and is not
 * thread-safe; all steps of one server go to one stream. */
typedef struct mpcg_server mpcg_server_t;

enum {
  MPCG_PHASE_NEW = 0,      /* admitted, nothing run yet */
  MPCG_PHASE_STAGE1 = 1,   /* single-precision stage under way */
  MPCG_PHASE_STAGE2 = 2,   /* double-precision stage next */
  MPCG_PHASE_STAGE2_RUN = 3, /* double-precision stage under way */
  MPCG_PHASE_DONE = 4      /* result record, x and status written */
};

/* Workspace for a server of max_slots slots and a pool of pool_bytes (each
 * admitted system takes mpcg_workspace_bytes(n, nnz) of it, rounded up to
 * 256 bytes).  0 if max_slots <= 0. */
size_t mpcg_server_workspace_bytes(int32_t max_slots, size_t pool_bytes);

/* Create a server on the caller's device workspace (256-byte aligned, size
 * from mpcg_server_workspace_bytes).  `sample` (device arrays, kept alive
 * by the caller) and `opts` apply to every system; stage1_only is refused.
 * *out: host handle, freed by mpcg_server_destroy. */
int32_t mpcg_server_create(void* ws, size_t ws_bytes, int32_t max_slots,
                           const mpcg_sample_t* sample, const mpcg_options_t* opts,
                           mpcg_server_t** out);
void mpcg_server_destroy(mpcg_server_t* srv);

/* Admit one system: A, b, x, res as for mpcg_solve (device memory kept
 * valid until the system is retired), final tolerance eps2.  *slot receives
 * its slot.  MPCG_ERR_WORKSPACE when no slot is free or the pool has no
 * contiguous block of the system's workspace size (the caller retries after
 * retiring).  Host only; the system starts at the next step. */
int32_t mpcg_server_admit(mpcg_server_t* srv, const mpcg_csr_t* A, const double* b, double* x,
                          double eps2, mpcg_result_t* res, int32_t* slot);

/* One step on `stream`: copies the slot tables, advances every admitted
 * system by at most max_iters iterations per stage, then copies the phase
 * of every slot (int32[max_slots], MPCG_PHASE_*) to slot_phase (host memory,
 * pinned for an asynchronous copy; may be NULL), valid after the stream has
 * synchronised (a pageable slot_phase makes that copy, and so the call,
 * wait for the step).  Entries of slots that are not admitted are
 * meaningless. */
int32_t mpcg_batch_step(mpcg_server_t* srv, int32_t max_iters, int32_t* slot_phase,
                        mpcg_stream_t stream);

/* Kernel launches that one mpcg_batch_step makes while a system is admitted:
 * the table staging launches, the step kernel (two with serve_split) and the
 * abort check.  -1 for a NULL handle.  Host only. */
int32_t mpcg_batch_step_launches(const mpcg_server_t* srv);

/* Free the slot and the pool block of an admitted system (after its phase
 * is MPCG_PHASE_DONE, or to cancel it between steps). */
int32_t mpcg_server_retire(mpcg_server_t* srv, int32_t slot);

/* Size of the library's fixed scratch array used by mpcg_solve_static. */
#define MPCG_STATIC_WS_BYTES (64u << 20) /* 64 MiB */

/* mpcg_solve without a caller workspace and without any allocation.  The
 * paper has no counterpart: this is a deployment variant of mpcg_solve for
 * callers that must not allocate device memory.  Same arguments, results
 * and status codes as mpcg_solve, minus ws and ws_bytes; the scratch is a
 * fixed array of MPCG_STATIC_WS_BYTES bytes in the library's device code,
 * one per device.  Every call looks up the array's device address in the
 * calling thread's current context (a host-side name of the array is not a
 * device address), so the call also works after cudaDeviceReset and under
 * a context the caller created.
 *   Limit: systems whose mpcg_workspace_bytes(n, nnz, opts) exceeds
 *   MPCG_STATIC_WS_BYTES are rejected with MPCG_ERR_WORKSPACE before
 *   anything is launched (about n <= 200000 for a 7-point stencil).
 *   The control block is cleared on `stream` at the start of every call.
 *   Overlapping calls race: two calls on the same device whose work may run
 *   at the same time (different streams, or host threads) share the one
 *   array and corrupt each other's results.  Issue the calls of one device
 *   on one stream, or order them.
 * Errors: as mpcg_solve (argument and option checks first); MPCG_ERR_CUDA
 * if the array's address cannot be obtained in the current context (the
 * failed lookup leaves no pending CUDA error behind). */
int32_t mpcg_solve_static(const mpcg_csr_t* A, const double* b, double* x,
                          const mpcg_sample_t* sample, const mpcg_options_t* opts,
                          mpcg_result_t* res, mpcg_stream_t stream);

/* ---- building blocks exposed for verification (same kernels as above) ---- */

/* y = A x through the library's SpMV (single or double precision, chosen by
 * `fp32`); x, y device float32[n] or float64[n].  Uses ws for the sliced
 * layout built from A (same layout as the solver). */
int32_t mpcg_spmv(const mpcg_csr_t* A, int32_t fp32, const void* x, void* y, void* ws,
                  size_t ws_bytes, mpcg_stream_t stream);

/* Breadth-first distances from src over the sparsity graph (Sec. 6):
 * dist device int32[n], -1 for unreached vertices. */
int32_t mpcg_bfs(const mpcg_csr_t* A, int32_t src, int32_t* dist, void* ws, size_t ws_bytes,
                 mpcg_stream_t stream);

/* 2BFS pseudo-diameter with the per-component rule (Sec. 6); out: device
 * int32[2] = {l~, t} where t is the farthest vertex found from vertex 0. */
int32_t mpcg_pseudo_diameter(const mpcg_csr_t* A, int32_t* out, void* ws, size_t ws_bytes,
                             mpcg_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MPCG_H */
