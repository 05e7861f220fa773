/*
 * fw_seg.h -- C ABI of the GB300 Greedy Frank-Wolfe graph-segmentation library.
 *
 * The library minimises the penalised graph Ginzburg-Landau energy
 *
 *     E(U) = 1/2 tr(U^T L_s U) + 1/eps tr(U (1 - U^T)) + 1/2 ||D_w^{1/2} (U_hat - U)||_F^2
 *
 * (Sec. 2.1, eqs. gl_vv2 / gradgl_vv2) over Sigma, the product of the n unit
 * simplices of R^K (eq. fs), with the Greedy Frank-Wolfe method (Sec. 4,
 * Alg. 3): S_k = GLMO(grad E(U_k)), D_k = S_k - U_k, U_{k+1} = U_k + a_k D_k.
 * The step a_k is the exact minimiser of the quadratic E along D_k (E has the
 * constant Hessian I_K (x) (L_s + D_w - 2/eps I), App. C); the paper's Armijo
 * rule (eqs. eta, Armijo, Sec. 5.1) is available as an option.
 *
 * Conventions shared by every call:
 *  - Pointers named *_host are host memory; they are read (or written) during
 *    the call only, and the caller keeps ownership.  Pointers named *_dev are
 *    device memory on the current CUDA device.
 *  - A handle owns all device memory it allocates until its destroy call.
 *    A handle is not thread-safe; different handles are independent.
 *  - Every call returns an fw_status; negative values are errors, and
 *    fw_seg_last_error() then gives a message (per calling thread).  No call
 *    throws or aborts.
 *  - All work of a handle runs on the stream given in its options (or on a
 *    stream the handle creates); calls that return host data synchronise it.
 *  - Graph input: a symmetric weighted adjacency matrix W in CSR form with
 *    int32 row_ptr[n+1] (row_ptr[0] = 0) and col[nnz], strictly increasing
 *    column indices within each row, no self loops, finite weights w >= 0 and
 *    w_ij == w_ji exactly.  Every node needs a positive degree (the paper
 *    assumes a connected graph, Sec. 1).  Violations give FW_ERR_GRAPH or
 *    FW_ERR_ISOLATED.  Supported sizes: 2 <= K <= 32, n >= 1, and padded
 *    nnz < 2^31.
 */
#ifndef FW_SEG_H
#define FW_SEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fw_status {
    FW_OK = 0,               /* solve stopped on the gap test or at a stationary point */
    FW_NOT_CONVERGED = 1,    /* iteration cap reached; the iterate is valid */
    FW_PENDING = 2,          /* serving: request admitted or queued, not finished */
    FW_ERR_INVALID_ARG = -1, /* bad pointer, size, option or state */
    FW_ERR_GRAPH = -2,       /* CSR not symmetric / self loop / column out of range /
                                columns not increasing / weight negative or not finite */
    FW_ERR_ISOLATED = -3,    /* a node has degree 0 */
    FW_ERR_NO_MEMORY = -4,   /* device allocation failed, or serving budget exceeded */
    FW_ERR_CUDA = -5,        /* a CUDA runtime call failed (message has the CUDA error) */
    FW_ERR_NUMERIC = -6,     /* NaN or Inf in the gap or curvature */
    FW_ERR_TIMEOUT = -7,     /* a device-side wait ran out of its budget */
    FW_ERR_UNSUPPORTED = -8  /* valid request outside the supported sizes */
} fw_status;

/* Storage precision of the normalised weights, and of the iterate. */
enum { FW_WEIGHTS_F32 = 0,   /* FP32 weights, FP32 U / L U, FP32 accumulation */
       FW_WEIGHTS_BF16 = 1,  /* BF16 weights, FP32 U / L U, FP32 accumulation */
       FW_WEIGHTS_F64 = 2 }; /* FP64 weights and FP64 iterate (small problems, checks) */
/* Laplacian (Sec. 1): L_s = I - D^-1/2 W D^-1/2 (the paper's) or L = D - W. */
enum { FW_LAPLACIAN_SYM = 0, FW_LAPLACIAN_COMB = 1 };
/* Stop test: g_k <= gap_tol (absolute) or g_k <= gap_tol * g_0 (relative). */
enum { FW_TOL_ABS = 0, FW_TOL_REL = 1 };
/* Linear oracle: greedy rule of Alg. 3 (eq. eq:LMOpr) or the full LMO of Alg. 2. */
enum { FW_ORACLE_GREEDY = 0, FW_ORACLE_FULL = 1 };
/* Step: exact line search on the quadratic E, or Armijo (delta 0.5, gamma 1e-6). */
enum { FW_STEP_EXACT = 0, FW_STEP_ARMIJO = 1 };

typedef struct fw_seg_opts {
    double eps;               /* penalty parameter eps > 0; +INFINITY drops the penalty */
    double omega0;            /* fidelity weight omega_0 >= 0 on labelled nodes (Sec. 2) */
    double gap_tol;           /* stop threshold for the FW gap (see tol_mode) */
    int32_t max_iters;        /* iteration cap (>= 0) */
    int32_t tol_mode;         /* FW_TOL_* */
    int32_t weight_dtype;     /* FW_WEIGHTS_* */
    int32_t laplacian;        /* FW_LAPLACIAN_* */
    int32_t oracle;           /* FW_ORACLE_* */
    int32_t step_rule;        /* FW_STEP_* */
    int32_t refresh_every;    /* recompute L U from scratch every R iterations (0: never) */
    int32_t iters_per_launch; /* iterations captured in one CUDA graph launch (>= 1) */
    int32_t lanes_per_row;    /* lanes per CSR row in the sparse passes: 0 (auto) or 1,2,4,..,32 */
    int32_t index_width;      /* stored column indices: 0 (auto: 16-bit offsets j - i when every
                                 |j - i| < 2^15, as in pixel grids; else 32-bit) or 32 */
    int32_t class_table;      /* FW_TABLE_*: pass B reads the 4-bit classes from a copy in
                                 shared memory (same results; see below) */
    int32_t reserved;         /* 0 */
    void *cuda_stream;        /* cudaStream_t for all work; NULL: the handle makes one */
} fw_seg_opts;

typedef struct fw_seg_stats {
    int32_t iters;        /* updates applied since create / set_U */
    int32_t status;       /* fw_status of the solve (FW_PENDING while running) */
    int32_t active_rows;  /* |I_k|, rows the oracle moved at the last evaluation */
    int32_t launches;     /* kernels launched by the call */
    double gap;           /* FW gap g_k at the last evaluated iterate */
    double gap0;          /* g_0 */
    double q;             /* <D_k, H D_k> of the last step */
    double alpha;         /* last step a_k */
    double objective;     /* E(U_k), kept by the exact quadratic recurrence */
    double ms;            /* device time of the call in milliseconds */
} fw_seg_stats;

typedef struct fw_seg fw_seg;

/* Pass B forms (fw_seg_opts::class_table).  Pass B gathers the class of
 * every column it reads.  With FW_TABLE_ON, and under FW_TABLE_AUTO for graphs
 * whose columns are not banded and that have at least one 256-row tile per
 * SM, it instead runs one 1024-thread block per SM that first copies the
 * problem's 4-bit class array ((n + 1) / 2 bytes) into shared memory; this
 * needs an FP32 iterate, K <= 16, 1, 2 or 4 lanes per row, n <= 311,296 and
 * the array plus the bins within one block's shared memory (n <= 280,574
 * for 8 < K <= 10 with 2 lanes), else the direct form runs.  Both forms give the
 * same bits.  FW_TABLE_OFF always runs the direct form. */
enum { FW_TABLE_AUTO = 0, FW_TABLE_OFF = 1, FW_TABLE_ON = 2 };

/* Fill *opts with defaults: eps 50, omega0 1000 (the paper's network values,
 * Sec. 5.2), gap_tol 0, FW_TOL_ABS, max_iters 500, FP32 weights, L_s, greedy
 * oracle, exact step, refresh_every 0, iters_per_launch 32, lanes auto,
 * index width auto, class table auto. */
fw_status fw_seg_default_opts(fw_seg_opts *opts);

/* Device bytes a handle needs for a graph of n nodes, nnz stored entries and
 * K classes (peak during create), for admission control. */
size_t fw_seg_footprint(int64_t n, int64_t nnz, int32_t K, int32_t weight_dtype);

/* Create a solver for one graph (Sec. 1 graph, Sec. 2 fidelity data).
 * row_ptr_host[n+1], col_host[nnz], w_host[nnz]: the CSR of W (see top).
 * labels_host[n]: class in [0,K) of each fidelity node, -1 elsewhere; fidelity
 * nodes get omega_i = omega_0 and u_hat_i = e_class, the others omega_i = 0.
 * The handle builds D, L_s (or L), the start U_0 = U_hat with unlabelled rows
 * at 1/K (Sec. 5.1) and L U_0.  opts may be NULL (defaults).
 * Errors: FW_ERR_INVALID_ARG, FW_ERR_GRAPH, FW_ERR_ISOLATED, FW_ERR_NO_MEMORY,
 * FW_ERR_UNSUPPORTED, FW_ERR_CUDA; *out is NULL on error. */
fw_status fw_seg_create(fw_seg **out, int64_t n, const int32_t *row_ptr_host,
                        const int32_t *col_host, const double *w_host, int32_t K,
                        const int32_t *labels_host, const fw_seg_opts *opts);

/* Run GFW iterations (Alg. 3) until the stop rule holds: no active row or
 * g_k <= 0 (stationary, FW_OK), g_k <= tolerance (FW_OK), or max_iters updates
 * (FW_NOT_CONVERGED).  The test is made before the update, as in step 4 of
 * Alg. 3.  stats may be NULL.  Errors: FW_ERR_NUMERIC, FW_ERR_CUDA.
 * Execution: iterations run as a CUDA graph of iters_per_launch iterations
 * (2 kernels each, the step decision of each iteration taken at the start of
 * the next one, one finishing kernel per graph), launched repeatedly with one
 * launch queued ahead of the host's state check; fewer than iters_per_launch
 * remaining iterations run as direct launches of the same kernels.  With
 * refresh_every > 0, or on a stream that cannot be captured, the host checks
 * the state after every launch.  The stream is synchronised on return. */
fw_status fw_seg_solve(fw_seg *h, fw_seg_stats *stats);

/* Run at most `iters` iterations (fewer if the stop rule holds first) and
 * leave the updated iterate in place; used for lockstep checks. */
fw_status fw_seg_step(fw_seg *h, int32_t iters, fw_seg_stats *stats);

/* Segmentation: labels_host[i] = argmax_k u_ik (lowest index on ties). */
fw_status fw_seg_labels(fw_seg *h, int32_t *labels_host);

/* One-Shot Frank-Wolfe (Alg. 4): U_1 = S_0 = GLMO(grad E(U_0)) from the start
 * point U_0 = U_hat (Sec. 5.1), i.e. label_i = s_i, the class the (G)LMO picks
 * for row i at U_hat (the handle's oracle option: greedy GLMO or full LMO).
 * One fused pass over the CSR forms L U_hat from the fidelity data, the
 * gradient and the argmin; the handle's iterate is neither read nor changed.
 * The labels are bitwise the choices the iteration makes at U_0.  For eps
 * below the bound of Cor. nonconvb2, GFW stops after this one step and the two
 * coincide.  labels_host (n entries) may be NULL: the labels then stay on the
 * device.  ms (nullable) receives the kernel's device time in milliseconds. */
fw_status fw_seg_oneshot(fw_seg *h, int32_t *labels_host, double *ms);

/* Copy U (n x K, row-major, widened to double) to the host. */
fw_status fw_seg_get_U(fw_seg *h, double *U_host);

/* Replace U by U_host (n x K row-major, rounded to the iterate precision),
 * recompute L U from scratch and restart the iteration count (warm start,
 * Sec. 4 last paragraph; lockstep checks). Rows must lie in the simplex. */
fw_status fw_seg_set_U(fw_seg *h, const double *U_host);

/* At the current iterate, the gradient without its constant 1/eps term,
 * G' = L U - (2/eps) U + D_w (U - U_hat) (eq. gradgl_vv2g minus (1/eps) 1),
 * as the kernels compute it, plus the (G)LMO choice and the active flag of
 * every row.  Any output pointer may be NULL.  G_host is n x K row-major. */
fw_status fw_seg_get_grad(fw_seg *h, double *G_host, int32_t *choice_host,
                          uint8_t *active_host);

/* E(U) at the current iterate, evaluated directly (fresh L U product). */
fw_status fw_seg_objective(fw_seg *h, double *E);

/* Diagnostic: the classic Frank-Wolfe gap of the full LMO (Alg. 2) at the
 * current iterate, sum_i sum_k u_ik (G_ik - min_j G_ij) with G = grad E(U)
 * from a fresh L U product.  It is 0 exactly at a stationary point of E over
 * Sigma and never below the GLMO gap g_k of the iteration (which is 0 at any
 * binary point, stationary or not).  FP64 sum of per-block partials in a
 * fixed order. */
fw_status fw_seg_lmo_gap(fw_seg *h, double *gap);

/* Recompute L U from scratch (drift control for the recurrence). */
fw_status fw_seg_refresh(fw_seg *h);

/* Restart from U_0 = U_hat on the device (no host copy): same state as right
 * after fw_seg_create.  Used to time repeated solves of one resident graph. */
fw_status fw_seg_reset(fw_seg *h);

/* Measurement of the iteration kernels in the form fw_seg_solve runs them
 * (each time is taken with two CUDA events on the handle's stream around one
 * captured graph, so no event sits between kernels):
 *   *ms_per_iter  a graph of `iters` (1..4096) fused iterations (pass A with
 *                 the previous iteration's step decision, pass B) and one
 *                 finishing kernel, divided by iters;
 *   *ms_row_pass  a graph of `iters` launches of the fused pass A (update,
 *                 step decision, gradient, GLMO, gap pieces), per launch;
 *   *ms_csr_pass  a graph of `iters` launches of pass B (one-hot L S,
 *                 <D, L S>), per launch;
 *   *ms_finish    one finishing kernel (exact totals, stop test, line
 *                 search), launched directly.
 * The repeated passes run on a copy of the problem's mutable arrays taken
 * before and put back after, so they do not change the iterate.  *in_graph
 * is 1; on a stream that cannot be captured the same launches are enqueued
 * directly and *in_graph is 0.  Outputs may be NULL.  The handle must not
 * have stopped (reset first); afterwards the iterate has advanced by
 * iters + 1 iterations, exactly as fw_seg_step(h, iters + 1) would have
 * advanced it (FW_ERR_INVALID_ARG if the stop rule holds on the way). */
fw_status fw_seg_profile(fw_seg *h, int32_t iters, double *ms_row_pass, double *ms_csr_pass,
                         double *ms_finish, double *ms_per_iter, int32_t *in_graph);

/* Statistics of the handle's current state. */
fw_status fw_seg_get_stats(fw_seg *h, fw_seg_stats *stats);

/* The kernel forms create chose for the handle (host data only, no device
 * call): they change no result, only the speed.  FW_ERR_INVALID_ARG when h or
 * forms is NULL. */
typedef struct fw_seg_forms {
    int32_t lanes_per_row;   /* lanes per CSR row of the sparse passes */
    int32_t index_width;     /* 16: columns stored as offsets j - i; 32: as indices */
    int32_t class_table;     /* 1: pass B reads the 4-bit classes from shared memory */
    int32_t table_blocks;    /* blocks of that pass B (0 without it) */
    int32_t tiles;           /* row tiles of the row passes */
    int32_t tile_rows;       /* rows per tile (a multiple of 256) */
    int32_t kmax;            /* class bound the kernels were compiled for (>= K) */
    int32_t reserved;
} fw_seg_forms;
fw_status fw_seg_get_forms(fw_seg *h, fw_seg_forms *forms);

/* Release the handle (NULL is a no-op).  Waits for the handle's stream; the
 * device arrays go back, stream-ordered, to the library's per-device memory
 * pool, which keeps up to 4 GiB of freed memory mapped so that a later create
 * maps nothing new (create / destroy per request stays cheap). */
void fw_seg_destroy(fw_seg *h);

/* ------------------------------------------------------------------------
 * Batched solves: many independent problems iterated together.
 *
 * All problems of a batch live in one contiguous device pool (each at its own
 * offsets) and iterate together, from a captured CUDA graph, in one of two
 * schedules (FW_SCHED_*): per-item launches, where each iteration is one
 * launch of pass A over the row tiles of every live problem and one of pass B
 * (the kernel boundaries are the barriers); or a cooperative persistent
 * kernel: phase A, grid barrier, phase B, grid barrier, per iteration.  Each
 * problem keeps its own tile partition and reduction order, so its iterates
 * are bitwise the same as when it is solved alone (by fw_seg_* or in any
 * other batch) with the same lanes per row.  Each problem stops on its own
 * stop rule; later launches skip it.  Waits at the persistent kernel's grid
 * barrier are bounded by spin_budget_ms: a wait that runs out ends the launch
 * with FW_ERR_TIMEOUT instead of hanging.
 * ---------------------------------------------------------------------- */

/* A graph on the host (see fw_seg_create for the CSR conventions). */
typedef struct fw_graph {
    int64_t n;
    const int32_t *row_ptr_host;
    const int32_t *col_host;
    const double *w_host;
    int32_t K;
    int32_t reserved;
    const int32_t *labels_host;
} fw_graph;

/* Schedules of a batch: the persistent cooperative kernel with a static grid
 * stride or an atomic work counter over the (problem, tile) items, or
 * per-item launches (each iteration one launch of the single-problem pass A
 * over all items and one of pass B, kernel boundaries as the barriers). */
enum { FW_SCHED_AUTO = 0, FW_SCHED_STATIC = 1, FW_SCHED_DYNAMIC = 2, FW_SCHED_ITEMS = 3 };
/* How a persistent launch is issued: directly; from a captured CUDA graph,
 * with a failed capture an error (FW_ERR_CUDA); or from a captured graph when
 * the stream can be captured, else directly (fw_batch_info says which). */
enum { FW_GRAPH_OFF = 0, FW_GRAPH_REQUIRED = 1, FW_GRAPH_PREFERRED = 2 };

typedef struct fw_batch_opts {
    int32_t weight_dtype;      /* FW_WEIGHTS_*, shared by every problem */
    int32_t blocks_per_sm;     /* 0: autotune (cached) */
    int32_t schedule;          /* FW_SCHED_* (AUTO: autotuned) */
    int32_t iters_per_launch;  /* -1: autotune; 0: every iteration in one launch */
    int32_t use_graph;         /* FW_GRAPH_* (default FW_GRAPH_REQUIRED) */
    int32_t spin_budget_ms;    /* bound on one grid-barrier wait */
    int32_t test_barrier_extra;/* test hook, keep 0: the barrier also waits for this many
                                  blocks that never arrive, so every wait runs out */
    int32_t lanes_per_row;     /* -1: autotune; 0: each problem's own count (from its
                                  options, else its mean degree); else 1,2,4,..,32 for
                                  every problem */
    const char *tune_cache;    /* autotune cache file; NULL: $FW_TUNE_CACHE or none */
    void *cuda_stream;         /* cudaStream_t; NULL: the batch makes one */
} fw_batch_opts;

typedef struct fw_batch_info {
    int32_t grid;              /* blocks of the persistent launch */
    int32_t blocks_per_sm;
    int32_t schedule;          /* FW_SCHED_STATIC, FW_SCHED_DYNAMIC or FW_SCHED_ITEMS */
    int32_t graph_captured;    /* 1 if the last launch ran from a captured CUDA graph */
    int32_t tuned;             /* 0 set by the caller, 1 measured now, 2 from the cache */
    int32_t kmax;              /* class bound of the persistent kernel (>= the largest K) */
    int32_t lanes_per_row;     /* lanes per CSR row of every problem; 0: each problem's
                                  own count from its mean degree */
    int32_t iters_per_launch;  /* 0: every iteration in one launch */
    int32_t graph_error;       /* cudaError_t of the last failed capture, 0 if none */
    int32_t reserved;
    double tune_ms;            /* time spent autotuning */
    size_t pool_bytes;         /* device bytes of the problem pool */
} fw_batch_info;

typedef struct fw_batch fw_batch;

/* Defaults: FP32 weights; blocks per SM, schedule, lanes per row and
 * iterations per launch autotuned; FW_GRAPH_REQUIRED; 2000 ms barrier budget.
 *
 * Autotuning (at create, when any of those four is left to it) times a few
 * iterations of the batch itself, from U_0, for each candidate, one
 * dimension after the other: the schedule (per-item launches, or the
 * persistent kernel static or dynamic at each blocks-per-SM count); then lanes per CSR
 * row (each problem's own count, or 1, 2, 4, 8 for all); then the class
 * bound the persistent kernel is compiled for (the smallest one that holds
 * the batch's largest K, or the next); then iterations per launch (all, 64
 * or 16).  The schedule, the class bound and the launch length change no
 * result; the lanes per row change the order in which a row's entries are
 * summed, so a batch equals single solves bit for bit when those use the
 * same lanes_per_row (fw_batch_info reports it).  The choice is cached in
 * tune_cache under a signature of the device and the batch's sizes. */
fw_status fw_batch_default_opts(fw_batch_opts *opts);

/* Create a batch of P problems.  graphs[P] are host graphs, opts[P] their
 * solver options (eps, omega0, stop rule, ... may differ per problem; the
 * weight dtype comes from bopts).  bopts may be NULL (defaults). */
fw_status fw_batch_create(fw_batch **out, int32_t P, const fw_graph *graphs,
                          const fw_seg_opts *opts, const fw_batch_opts *bopts);

/* Iterate every problem to its stop rule.  stats[P] may be NULL. */
fw_status fw_batch_solve(fw_batch *b, fw_seg_stats *stats);

/* Restart every problem at U_0 on the device. */
fw_status fw_batch_reset(fw_batch *b);

fw_status fw_batch_labels(fw_batch *b, int32_t p, int32_t *labels_host);
fw_status fw_batch_get_U(fw_batch *b, int32_t p, double *U_host);
fw_status fw_batch_get_info(fw_batch *b, fw_batch_info *info);
void fw_batch_destroy(fw_batch *b);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of segmentation requests.
 *
 * A worker thread owns a device pool of hbm_budget_bytes.  Submitted requests
 * wait in a FIFO queue; a request is admitted when a slot is free and its
 * device footprint fits in the free pool, uploaded and assembled on a side
 * stream while the current epoch runs, and joins the next epoch.  An epoch is
 * iters_per_epoch iterations of every resident request (four times as many
 * while no request waits for admission): the single-problem kernels of
 * fw_seg_solve for one request -- the only resident one, the oldest when it
 * has at least 131,072 rows (enough to fill the GPU), first in, first out, or
 * the only resident below that size -- or else one batched epoch over the
 * residents below that size (a large one waits until it is the oldest):
 * per-item launches (the default) or the persistent kernel
 * (FW_SCHED_STATIC / FW_SCHED_DYNAMIC).
 * Lone-request epochs run from a captured graph, two kept in flight ahead of
 * the worker thread.
 * Requests that meet their stop rule are harvested
 * (labels copied to the host) and their memory is reused.  Results are
 * bitwise the same as when the request is solved alone.
 * ---------------------------------------------------------------------- */

typedef struct fw_srv_opts {
    size_t hbm_budget_bytes;   /* device pool for resident requests */
    int32_t max_slots;         /* requests resident at once */
    int32_t max_K;             /* largest K accepted (kernel class bound) */
    int32_t weight_dtype;      /* FW_WEIGHTS_*, shared by all requests */
    int32_t iters_per_epoch;
    int32_t blocks_per_sm;     /* 0: largest co-resident grid */
    int32_t schedule;          /* FW_SCHED_* (default and AUTO: per-item launches) */
    int32_t spin_budget_ms;
    int32_t reserved;
    void *cuda_stream;         /* stream of the epochs; NULL: the server makes one */
} fw_srv_opts;

typedef struct fw_srv_info {
    uint64_t submitted, admitted, rejected, completed, failed, epochs;
    int32_t resident;          /* requests on the device now */
    int32_t queued;            /* requests waiting for admission */
    size_t pool_bytes, pool_used;
} fw_srv_info;

typedef struct fw_srv fw_srv;

fw_status fw_srv_default_opts(fw_srv_opts *opts);
fw_status fw_srv_create(fw_srv **out, const fw_srv_opts *opts);

/* Queue a request; the graph is copied, so the caller's arrays may be reused
 * at once.  FW_PENDING and a ticket on success; FW_ERR_NO_MEMORY when the
 * request can never fit the pool (rejected); FW_ERR_UNSUPPORTED for K above
 * max_K; other errors as fw_seg_create. */
fw_status fw_srv_submit(fw_srv *s, const fw_graph *g, const fw_seg_opts *opts, uint64_t *ticket);

/* FW_PENDING while queued or running; the request's final status once done,
 * with labels_host[n] (nullable) and stats (nullable) filled.  A finished
 * ticket is forgotten after it has been returned once. */
fw_status fw_srv_poll(fw_srv *s, uint64_t ticket, int32_t *labels_host, fw_seg_stats *stats);

/* As fw_srv_poll, blocking up to timeout_ms (negative: no limit). */
fw_status fw_srv_wait(fw_srv *s, uint64_t ticket, int32_t timeout_ms, int32_t *labels_host,
                      fw_seg_stats *stats);

/* Block up to timeout_ms (negative: no limit) until some request has
 * finished whose result has not been returned yet; FW_OK with its ticket
 * (fetch the result with fw_srv_poll), or FW_PENDING when the time ran out.
 * Each finished ticket is reported once, in completion order. */
fw_status fw_srv_wait_any(fw_srv *s, int32_t timeout_ms, uint64_t *ticket);

fw_status fw_srv_get_info(fw_srv *s, fw_srv_info *info);

/* Stop the worker (requests still queued or resident are dropped) and free. */
void fw_srv_destroy(fw_srv *s);

/* ------------------------------------------------------------------------
 * Allocation-free energy evaluation.
 *
 * The paper has no counterpart to this call: it is a service entry point.  It
 * evaluates the objective E(U) = 1/2 <U, L U> (the Laplacian quadratic form)
 * + (1/eps) sum u (1 - u) (the penalty) + 1/2 sum_i omega_i ||u_hat_i - u_i||^2
 * (the fidelity term), the value fw_seg_objective gives for a handle, for a
 * graph and an iterate that are already in the caller's device memory,
 * without allocating device memory.
 * It is meant for callers that cannot allocate: a process whose device memory
 * is held by another allocator (cudaMalloc would fail), or a loop that must
 * not call cudaMalloc / cudaFree (they may synchronise the device).  Its
 * scratch is a static device array of FW_NOALLOC_MAX_N doubles plus 256 bytes
 * (8 MiB + 256 B per device, part of the library's module image).
 *
 * Arguments (all *_dev pointers are device memory on the current device, read
 * only, owned by the caller):
 *   n, K              1 <= n <= FW_NOALLOC_MAX_N, 2 <= K <= 32
 *   row_ptr_dev[n+1], col_dev[nnz], w_dev[nnz]
 *                     CSR of W with the conventions at the top of this file
 *                     (int32 indices, FP64 weights); nnz = row_ptr[n].
 *   U_dev             FP64, row-major n x K with row stride ldu >= K elements
 *   labels_dev        int32[n]: fidelity class in [0, K) or -1 (no fidelity);
 *                     NULL means no fidelity node
 *   eps, omega0       as in fw_seg_opts (eps may be +inf)
 *   laplacian         FW_LAPLACIAN_SYM (L_s) or FW_LAPLACIAN_COMB (D - W)
 *   cuda_stream       stream of the work (NULL: the legacy default stream);
 *                     the call synchronises it before returning
 *   E_host            receives E(U), FP64 sums combined exactly across blocks,
 *                     so the result is bitwise reproducible
 * Errors: FW_ERR_UNSUPPORTED if n > FW_NOALLOC_MAX_N (nothing is launched);
 * FW_ERR_INVALID_ARG for bad sizes, pointers, options or labels; FW_ERR_GRAPH
 * for a row_ptr extent or column outside [0, nnz) / [0, n) (never read);
 * FW_ERR_ISOLATED for a node of degree 0; FW_ERR_NUMERIC for a non-finite
 * energy; FW_ERR_CUDA.  Symmetry of W is not checked.
 * The first call on each device looks up the scratch array's address
 * (cudaGetSymbolAddress, which may load the module's device data) and caches
 * it with the identity of the current CUDA context; a call in a new context
 * of the device (after cudaDeviceReset, say) looks it up again.  Make the
 * first call on a device before any stream capture.  All calls on a device
 * share its one scratch array: calls that overlap in time on the same device
 * race and may return wrong values, so the caller serialises them.
 * ---------------------------------------------------------------------- */
#define FW_NOALLOC_MAX_N 1048576

fw_status fw_energy_noalloc(int64_t n, int32_t K, const int32_t *row_ptr_dev,
                            const int32_t *col_dev, const double *w_dev, int64_t nnz,
                            const double *U_dev, int64_t ldu, const int32_t *labels_dev,
                            double eps, double omega0, int32_t laplacian, void *cuda_stream,
                            double *E_host);

/* Message of the last error on the calling thread ("" if none). */
const char *fw_seg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FW_SEG_H */
