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
    int32_t reserved;
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

/* Fill *opts with defaults: eps 50, omega0 1000 (the paper's network values,
 * Sec. 5.2), gap_tol 0, FW_TOL_ABS, max_iters 500, FP32 weights, L_s, greedy
 * oracle, exact step, refresh_every 0, iters_per_launch 32, lanes auto. */
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
 * Alg. 3.  stats may be NULL.  Errors: FW_ERR_NUMERIC, FW_ERR_CUDA. */
fw_status fw_seg_solve(fw_seg *h, fw_seg_stats *stats);

/* Run at most `iters` iterations (fewer if the stop rule holds first) and
 * leave the updated iterate in place; used for lockstep checks. */
fw_status fw_seg_step(fw_seg *h, int32_t iters, fw_seg_stats *stats);

/* Segmentation: labels_host[i] = argmax_k u_ik (lowest index on ties). */
fw_status fw_seg_labels(fw_seg *h, int32_t *labels_host);

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

/* Recompute L U from scratch (drift control for the recurrence). */
fw_status fw_seg_refresh(fw_seg *h);

/* Restart from U_0 = U_hat on the device (no host copy): same state as right
 * after fw_seg_create.  Used to time repeated solves of one resident graph. */
fw_status fw_seg_reset(fw_seg *h);

/* Measurement: run `iters` iterations as separate launches with CUDA events
 * around each pass on the handle's stream; *ms_row_pass and *ms_csr_pass get
 * the mean device time of pass A (update, gradient, GLMO, gap) and pass B
 * (one-hot L S, line search) in milliseconds.  The iterate advances. */
fw_status fw_seg_profile(fw_seg *h, int32_t iters, double *ms_row_pass, double *ms_csr_pass);

/* Statistics of the handle's current state. */
fw_status fw_seg_get_stats(fw_seg *h, fw_seg_stats *stats);

void fw_seg_destroy(fw_seg *h);

/* Message of the last error on the calling thread ("" if none). */
const char *fw_seg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FW_SEG_H */
