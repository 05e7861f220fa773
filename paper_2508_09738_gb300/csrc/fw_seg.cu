// Single-problem solver: the fw_seg_* entry points of include/fw_seg.h.
//
// Device state of a handle (one GPU, resident for the handle's lifetime):
//   padded CSR of the off-diagonal operator (int32 row_ptr / col, WT weights),
//   U, L U, L S in class-major layout (T[K][npad]), choice (uint8) and fid (int8)
//   per row, per-tile FP64 partials and one ProbState.
// A solve launches a CUDA graph that holds `iters_per_launch` iterations
// (pass A + pass B each) and reads back the 128-byte state after each launch;
// nothing else crosses the host-device boundary during the iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "fw_device.cuh"
#include "fw_internal.h"

namespace fw {

// Validation and degrees of the input CSR (one thread per row):
//   columns strictly increasing and in range, no self loop, w finite and >= 0,
//   w_ij == w_ji (binary search in row j), d_i = sum_j w_ij > 0 (Sec. 1).
// err bits: 1 graph structure / weights, 2 asymmetric, 4 isolated node.
__global__ void k_validate(int64_t n, const int32_t* rp, const int32_t* col, const double* w,
                           double* deg, int* err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e0 = rp[i], e1 = rp[i + 1];
    double d = 0.0;
    int bad = 0;
    int prev = -1;
    for (int e = e0; e < e1; ++e) {
        const int j = col[e];
        const double x = w[e];
        if (j < 0 || j >= n || j == i || j <= prev || !(x >= 0.0) || isinf(x)) {
            bad |= 1;
            break;
        }
        prev = j;
        d += x;
        int lo = rp[j], hi = rp[j + 1] - 1, pos = -1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const int cm = col[mid];
            if (cm == i) { pos = mid; break; }
            if (cm < i) lo = mid + 1; else hi = mid - 1;
        }
        if (pos < 0 || w[pos] != x) bad |= 2;
    }
    if (!bad && !(d > 0.0)) bad |= 4;
    deg[i] = d;
    if (bad) atomicOr(err, bad);
}


static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

fw_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return FW_ERR_CUDA;
}

int kmax_for(int K) { return K <= 4 ? 4 : K <= 8 ? 8 : K <= 12 ? 12 : K <= 16 ? 16 : 32; }

Ops* make_ops(int weight_dtype, int K) {
    const int km = kmax_for(K);
    switch (weight_dtype) {
        case FW_WEIGHTS_F32: return make_ops_f32(km);
        case FW_WEIGHTS_BF16: return make_ops_bf16(km);
        case FW_WEIGHTS_F64: return make_ops_f64(km);
        default: return nullptr;
    }
}

int tile_rows_for(int64_t n) {
    const int64_t per = (n + kTilesTarget - 1) / kTilesTarget;
    return int(round_up(std::max<int64_t>(per, 1), kBlock));
}

int default_lanes(double avg_padded_degree) {
    int L = 1;
    while (L < 32 && avg_padded_degree > 12.0 * L) L *= 2;
    return L;
}

static fw_status invalid(const std::string& m) {
    set_error(m);
    return FW_ERR_INVALID_ARG;
}

static fw_status check_opts(const fw_seg_opts& o) {
    if (!(o.eps > 0.0)) return invalid("eps must be > 0 (or +inf)");
    if (!(o.omega0 >= 0.0) || std::isinf(o.omega0)) return invalid("omega0 must be finite and >= 0");
    if (!(o.gap_tol >= 0.0)) return invalid("gap_tol must be >= 0");
    if (o.max_iters < 0) return invalid("max_iters must be >= 0");
    if (o.tol_mode != FW_TOL_ABS && o.tol_mode != FW_TOL_REL) return invalid("bad tol_mode");
    if (o.weight_dtype < FW_WEIGHTS_F32 || o.weight_dtype > FW_WEIGHTS_F64)
        return invalid("bad weight_dtype");
    if (o.laplacian != FW_LAPLACIAN_SYM && o.laplacian != FW_LAPLACIAN_COMB)
        return invalid("bad laplacian");
    if (o.oracle != FW_ORACLE_GREEDY && o.oracle != FW_ORACLE_FULL) return invalid("bad oracle");
    if (o.step_rule != FW_STEP_EXACT && o.step_rule != FW_STEP_ARMIJO)
        return invalid("bad step_rule");
    if (o.refresh_every < 0) return invalid("refresh_every must be >= 0");
    if (o.iters_per_launch < 1 || o.iters_per_launch > 4096)
        return invalid("iters_per_launch must be in [1, 4096]");
    const int L = o.lanes_per_row;
    if (L != 0 && (L < 1 || L > 32 || (L & (L - 1)) != 0))
        return invalid("lanes_per_row must be 0 or a power of two <= 32");
    return FW_OK;
}

// Host validation of the CSR header and the labels; fills the padded row_ptr.
static fw_status check_host_graph(int64_t n, const int32_t* rp, const int32_t* labels, int32_t K,
                                  std::vector<int32_t>& rpp, int64_t& nnz, int64_t& nnz_pad) {
    if (rp[0] != 0) {
        set_error("row_ptr[0] must be 0");
        return FW_ERR_GRAPH;
    }
    rpp.assign(size_t(n) + 1, 0);
    int64_t acc = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t d = int64_t(rp[i + 1]) - rp[i];
        if (d < 0) {
            set_error("row_ptr must be non-decreasing");
            return FW_ERR_GRAPH;
        }
        acc += round_up(d, kPadW);
        if (acc >= (int64_t(1) << 31)) {
            set_error("padded nnz must stay below 2^31");
            return FW_ERR_UNSUPPORTED;
        }
        rpp[size_t(i) + 1] = int32_t(acc);
    }
    nnz = rp[n];
    nnz_pad = acc;
    for (int64_t i = 0; i < n; ++i)
        if (labels[i] < -1 || labels[i] >= K) {
            set_error("labels must be -1 or in [0, K)");
            return FW_ERR_INVALID_ARG;
        }
    return FW_OK;
}

}  // namespace fw

using namespace fw;

static_assert(sizeof(fw_seg_opts) == 72, "fw_seg_opts ABI");
static_assert(sizeof(fw_seg_stats) == 64, "fw_seg_stats ABI");

struct fw_seg {
    int device = 0;
    int64_t n = 0, nnz = 0, nnz_pad = 0;
    int32_t K = 0;
    fw_seg_opts opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::unique_ptr<Ops> ops;
    Bufs b;
    ProbState* h_state = nullptr;  // pinned mirror of *b.st
    cudaGraphExec_t graph = nullptr;
    int32_t* d_labels = nullptr;
    double* d_opart = nullptr;
    void* d_tmp = nullptr;      // T[K][npad] scratch: fresh L U, gradient
    uint8_t* d_ch = nullptr;    // choice scratch for fw_seg_get_grad
    int last_refresh = 0;
    int launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void*> dev_allocs;

    template <typename P>
    fw_status alloc(P** p, size_t bytes) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " +
                      cudaGetErrorString(e));
            return FW_ERR_NO_MEMORY;
        }
        dev_allocs.push_back(q);
        *p = reinterpret_cast<P*>(q);
        return FW_OK;
    }
    void release(void* p) {
        auto it = std::find(dev_allocs.begin(), dev_allocs.end(), p);
        if (it != dev_allocs.end()) {
            cudaFree(p);
            dev_allocs.erase(it);
        }
    }
    ~fw_seg() {
        if (stream) cudaStreamSynchronize(stream);
        if (graph) cudaGraphExecDestroy(graph);
        for (void* p : dev_allocs) cudaFree(p);
        if (h_state) cudaFreeHost(h_state);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

#define FW_TRY(x)                          \
    do {                                   \
        fw_status s_ = (x);                \
        if (s_ != FW_OK) return s_;        \
    } while (0)

static fw_status launch_check(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return FW_OK;
}

static fw_status read_state(fw_seg* h) {
    FW_CUDA(cudaMemcpyAsync(h->h_state, h->b.st, sizeof(ProbState), cudaMemcpyDeviceToHost,
                            h->stream));
    FW_CUDA(cudaStreamSynchronize(h->stream));
    return FW_OK;
}

static void fill_stats(fw_seg* h, fw_seg_stats* s, float ms) {
    if (!s) return;
    const ProbState& st = *h->h_state;
    s->iters = st.iter;
    s->status = st.done ? st.status : FW_PENDING;
    s->active_rows = st.active;
    s->launches = h->launches;
    s->gap = st.g;
    s->gap0 = st.g0;
    s->q = st.q;
    s->alpha = st.alpha;
    s->objective = st.E;
    s->ms = ms;
}

// Apply a pending update so that U / L U hold the current iterate.
static fw_status flush(fw_seg* h) {
    h->ops->flush(h->b, h->stream);
    ++h->launches;
    return launch_check("flush kernel");
}

static fw_status refresh_lu(fw_seg* h) {
    FW_TRY(flush(h));
    h->ops->spmm(h->b, h->b.U, h->b.LU, h->stream);
    ++h->launches;
    FW_TRY(launch_check("spmm kernel"));
    h->last_refresh = h->h_state->iter;
    return FW_OK;
}

// E(U) evaluated directly; LU scratch gets a fresh L U.
static fw_status direct_objective(fw_seg* h, double* E) {
    h->ops->spmm(h->b, h->b.U, h->d_tmp, h->stream);
    h->ops->objective(h->b, h->d_tmp, h->d_opart, h->stream);
    h->launches += 2;
    FW_TRY(launch_check("objective kernels"));
    const int64_t nb = (h->n + kBlock - 1) / kBlock;
    std::vector<double> part(size_t(nb), 0.0);
    FW_CUDA(cudaMemcpyAsync(part.data(), h->d_opart, sizeof(double) * nb,
                            cudaMemcpyDeviceToHost, h->stream));
    FW_CUDA(cudaStreamSynchronize(h->stream));
    double s = 0.0;
    for (double x : part) s += x;
    *E = s;
    return FW_OK;
}

// Reset the iteration state at the current U (after create / set_U).
static fw_status restart(fw_seg* h) {
    h->ops->spmm(h->b, h->b.U, h->b.LU, h->stream);
    ++h->launches;
    FW_TRY(launch_check("spmm kernel"));
    double E0 = 0.0;
    FW_TRY(direct_objective(h, &E0));
    ProbState st;
    std::memset(&st, 0, sizeof(st));
    st.status = FW_PENDING;
    st.E = E0;
    *h->h_state = st;
    FW_CUDA(cudaMemcpyAsync(h->b.st, h->h_state, sizeof(ProbState), cudaMemcpyHostToDevice,
                            h->stream));
    FW_CUDA(cudaStreamSynchronize(h->stream));
    h->last_refresh = 0;
    return FW_OK;
}

static fw_status build_graph(fw_seg* h) {
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    FW_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < h->opts.iters_per_launch; ++i) {
        h->ops->passA(h->b, h->stream);
        h->ops->passB(h->b, h->stream);
    }
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return FW_OK;
}

static fw_status status_of(const ProbState& st) {
    if (!st.done) return FW_NOT_CONVERGED;
    if (st.status == FW_ERR_NUMERIC) {
        set_error("non-finite FW gap or curvature");
        return FW_ERR_NUMERIC;
    }
    return fw_status(st.status);
}

extern "C" {

const char* fw_seg_last_error(void) { return g_last_error.c_str(); }

fw_status fw_seg_default_opts(fw_seg_opts* o) {
    if (!o) return invalid("opts is NULL");
    std::memset(o, 0, sizeof(*o));
    o->eps = 50.0;
    o->omega0 = 1000.0;
    o->gap_tol = 0.0;
    o->max_iters = 500;
    o->tol_mode = FW_TOL_ABS;
    o->weight_dtype = FW_WEIGHTS_F32;
    o->laplacian = FW_LAPLACIAN_SYM;
    o->oracle = FW_ORACLE_GREEDY;
    o->step_rule = FW_STEP_EXACT;
    o->refresh_every = 0;
    o->iters_per_launch = 32;
    o->lanes_per_row = 0;
    o->cuda_stream = nullptr;
    return FW_OK;
}

size_t fw_seg_footprint(int64_t n, int64_t nnz, int32_t K, int32_t weight_dtype) {
    const size_t te = weight_dtype == FW_WEIGHTS_F64 ? 8 : 4;
    const size_t we = weight_dtype == FW_WEIGHTS_F64 ? 8 : weight_dtype == FW_WEIGHTS_BF16 ? 2 : 4;
    const size_t npad = size_t(round_up(n, 32));
    const size_t nnzp = size_t(nnz) + size_t(kPadW) * size_t(n);  // upper bound
    size_t b = 0;
    b += 4 * (size_t(n) + 1) + nnzp * (4 + we);             // padded CSR
    b += 4 * te * npad * size_t(K);                           // U, LU, LS, scratch
    b += 3 * size_t(n) + 4 * size_t(n) + te * size_t(n);      // choice, fid, ch, labels, diag
    b += size_t(kTilesTarget + 1) * 8 * (kNumA + kNumB) + 8 * size_t(n / kBlock + 1);
    b += 4 * (size_t(n) + 1) + size_t(nnz) * 12 + 8 * size_t(n) + 4 * size_t(n);  // create temps
    return b + 4096;
}

fw_status fw_seg_create(fw_seg** out, int64_t n, const int32_t* row_ptr, const int32_t* col,
                        const double* w, int32_t K, const int32_t* labels,
                        const fw_seg_opts* opts_in) {
    try {
        if (!out) return invalid("out is NULL");
        *out = nullptr;
        fw_seg_opts o;
        if (opts_in) o = *opts_in; else fw_seg_default_opts(&o);
        FW_TRY(check_opts(o));
        if (n < 1 || n >= (int64_t(1) << 31) - 1) return invalid("n must be in [1, 2^31-1)");
        if (K < 2 || K > 32) {
            set_error("K must be in [2, 32]");
            return FW_ERR_UNSUPPORTED;
        }
        if (!row_ptr || !labels) return invalid("row_ptr and labels must not be NULL");
        std::vector<int32_t> rpp;
        int64_t nnz = 0, nnz_pad = 0;
        FW_TRY(check_host_graph(n, row_ptr, labels, K, rpp, nnz, nnz_pad));
        if (nnz > 0 && (!col || !w)) return invalid("col and w must not be NULL");

        std::unique_ptr<fw_seg> h(new fw_seg());
        FW_CUDA(cudaGetDevice(&h->device));
        h->n = n;
        h->K = K;
        h->nnz = nnz;
        h->nnz_pad = nnz_pad;
        h->opts = o;
        if (o.cuda_stream) {
            h->stream = static_cast<cudaStream_t>(o.cuda_stream);
        } else {
            FW_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
            h->own_stream = true;
        }
        h->ops.reset(make_ops(o.weight_dtype, K));
        if (!h->ops) return invalid("no kernels for this weight dtype / K");
        FW_CUDA(h->ops->configure());
        FW_CUDA(cudaMallocHost(&h->h_state, sizeof(ProbState)));
        FW_CUDA(cudaEventCreate(&h->ev0));
        FW_CUDA(cudaEventCreate(&h->ev1));

        const size_t te = h->ops->elem(), we = h->ops->welem();
        const int64_t npad = round_up(n, 32);
        ProbDesc& pd = h->b.pd;
        pd.row0 = 0;
        pd.uoff = 0;
        pd.n = int32_t(n);
        pd.npad = int32_t(npad);
        pd.K = K;
        pd.tile_rows = tile_rows_for(n);
        pd.ntiles = int32_t((n + pd.tile_rows - 1) / pd.tile_rows);
        pd.tile0 = 0;
        pd.inv_eps = std::isinf(o.eps) ? 0.0 : 1.0 / o.eps;
        pd.omega0 = o.omega0;
        pd.gap_tol = o.gap_tol;
        pd.tol_mode = o.tol_mode;
        pd.max_iters = o.max_iters;
        pd.oracle = o.oracle;
        pd.step_rule = o.step_rule;
        pd.lanes = o.lanes_per_row ? o.lanes_per_row
                                   : default_lanes(double(nnz_pad) / double(n));
        pd.comb = o.laplacian == FW_LAPLACIAN_COMB;

        Bufs& b = h->b;
        const cudaStream_t s = h->stream;
        FW_TRY(h->alloc(&b.rp, 4 * (size_t(n) + 1)));
        FW_TRY(h->alloc(&b.col, 4 * size_t(nnz_pad)));
        FW_TRY(h->alloc(&b.val, we * size_t(nnz_pad)));
        if (pd.comb) FW_TRY(h->alloc(&b.diag, te * size_t(n)));
        FW_TRY(h->alloc(&b.U, te * size_t(npad) * K));
        FW_TRY(h->alloc(&b.LU, te * size_t(npad) * K));
        FW_TRY(h->alloc(&b.LS, te * size_t(npad) * K));
        FW_TRY(h->alloc(&h->d_tmp, te * size_t(npad) * K));
        FW_TRY(h->alloc(&b.choice, size_t(n)));
        FW_TRY(h->alloc(&b.fid, size_t(n)));
        FW_TRY(h->alloc(&h->d_ch, size_t(n)));
        FW_TRY(h->alloc(&h->d_labels, 4 * size_t(n)));
        FW_TRY(h->alloc(&b.partA, 8 * size_t(pd.ntiles) * kNumA));
        FW_TRY(h->alloc(&b.partB, 8 * size_t(pd.ntiles) * kNumB));
        FW_TRY(h->alloc(&h->d_opart, 8 * size_t((n + kBlock - 1) / kBlock)));
        FW_TRY(h->alloc(&b.st, sizeof(ProbState)));
        FW_CUDA(cudaMemsetAsync(b.U, 0, te * size_t(npad) * K, s));
        FW_CUDA(cudaMemsetAsync(b.LS, 0, te * size_t(npad) * K, s));
        FW_CUDA(cudaMemsetAsync(b.st, 0, sizeof(ProbState), s));

        // raw input on the device (temporary)
        int32_t *d_rp = nullptr, *d_col = nullptr, *d_lab = nullptr;
        double *d_w = nullptr, *d_deg = nullptr;
        int* d_err = nullptr;
        FW_TRY(h->alloc(&d_rp, 4 * (size_t(n) + 1)));
        FW_TRY(h->alloc(&d_col, 4 * size_t(nnz)));
        FW_TRY(h->alloc(&d_w, 8 * size_t(nnz)));
        FW_TRY(h->alloc(&d_deg, 8 * size_t(n)));
        FW_TRY(h->alloc(&d_lab, 4 * size_t(n)));
        FW_TRY(h->alloc(&d_err, sizeof(int)));
        FW_CUDA(cudaMemcpyAsync(d_rp, row_ptr, 4 * (size_t(n) + 1), cudaMemcpyHostToDevice, s));
        if (nnz) {
            FW_CUDA(cudaMemcpyAsync(d_col, col, 4 * size_t(nnz), cudaMemcpyHostToDevice, s));
            FW_CUDA(cudaMemcpyAsync(d_w, w, 8 * size_t(nnz), cudaMemcpyHostToDevice, s));
        }
        FW_CUDA(cudaMemcpyAsync(d_lab, labels, 4 * size_t(n), cudaMemcpyHostToDevice, s));
        FW_CUDA(cudaMemcpyAsync(b.rp, rpp.data(), 4 * (size_t(n) + 1), cudaMemcpyHostToDevice, s));
        FW_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
        const unsigned g = unsigned((n + kBlock - 1) / kBlock);
        k_validate<<<g, kBlock, 0, s>>>(n, d_rp, d_col, d_w, d_deg, d_err);
        FW_TRY(launch_check("validate kernel"));
        int err = 0;
        FW_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        FW_CUDA(cudaStreamSynchronize(s));
        if (err & 3) {
            set_error(err & 1 ? "graph: column out of range / not increasing / self loop / bad weight"
                              : "graph: W is not symmetric");
            return FW_ERR_GRAPH;
        }
        if (err & 4) {
            set_error("graph: a node has degree 0");
            return FW_ERR_ISOLATED;
        }
        h->ops->build(n, 0, d_rp, d_col, d_w, d_deg, b.rp, b.col, b.val, b.diag, pd.comb, s);
        FW_TRY(launch_check("build kernel"));
        h->ops->init(b, d_lab, s);
        FW_TRY(launch_check("init kernel"));
        FW_CUDA(cudaStreamSynchronize(s));
        for (void* p : {(void*)d_rp, (void*)d_col, (void*)d_w, (void*)d_deg, (void*)d_lab,
                        (void*)d_err})
            h->release(p);
        FW_TRY(restart(h.get()));
        if (build_graph(h.get()) != FW_OK) {
            // streams that cannot be captured (the legacy default stream) run
            // the same kernels as direct launches
            cudaGetLastError();
            h->graph = nullptr;
        }
        *out = h.release();
        return FW_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

fw_status fw_seg_solve(fw_seg* h, fw_seg_stats* stats) {
    if (!h) return invalid("handle is NULL");
    h->launches = 0;
    FW_CUDA(cudaEventRecord(h->ev0, h->stream));
    FW_TRY(read_state(h));
    const int m = h->opts.iters_per_launch;
    while (!h->h_state->done) {
        const int R = h->opts.refresh_every;
        if (R > 0 && h->h_state->iter - h->last_refresh >= R) FW_TRY(refresh_lu(h));
        const int remaining = h->opts.max_iters - h->h_state->iter;
        if (remaining >= m && h->graph) {
            FW_CUDA(cudaGraphLaunch(h->graph, h->stream));
            h->launches += 2 * m;
        } else if (remaining >= m) {
            for (int i = 0; i < m; ++i) {
                h->ops->passA(h->b, h->stream);
                h->ops->passB(h->b, h->stream);
            }
            h->launches += 2 * m;
            FW_TRY(launch_check("iteration kernels"));
        } else {
            // tail: the last `remaining` iterations, then the final evaluation
            // (pass A at the iteration cap applies the last step and stops)
            for (int i = 0; i < remaining; ++i) {
                h->ops->passA(h->b, h->stream);
                h->ops->passB(h->b, h->stream);
            }
            h->ops->passA(h->b, h->stream);
            h->launches += 2 * remaining + 1;
            FW_TRY(launch_check("iteration kernels"));
        }
        FW_TRY(read_state(h));
    }
    FW_CUDA(cudaEventRecord(h->ev1, h->stream));
    FW_CUDA(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    fill_stats(h, stats, ms);
    return status_of(*h->h_state);
}

fw_status fw_seg_reset(fw_seg* h) {
    if (!h) return invalid("handle is NULL");
    h->ops->reinit(h->b, h->stream);
    ++h->launches;
    FW_TRY(launch_check("reinit kernel"));
    FW_CUDA(cudaMemsetAsync(h->b.st, 0, sizeof(ProbState), h->stream));
    return restart(h);
}

fw_status fw_seg_profile(fw_seg* h, int32_t iters, double* ms_a, double* ms_b) {
    if (!h || iters < 1) return invalid("bad arguments");
    cudaEvent_t ev[3];
    for (auto& e : ev) FW_CUDA(cudaEventCreate(&e));
    double ta = 0.0, tb = 0.0;
    int done = 0;
    fw_status rc = FW_OK;
    for (int i = 0; i < iters; ++i) {
        cudaEventRecord(ev[0], h->stream);
        h->ops->passA(h->b, h->stream);
        cudaEventRecord(ev[1], h->stream);
        h->ops->passB(h->b, h->stream);
        cudaEventRecord(ev[2], h->stream);
        cudaError_t e = cudaEventSynchronize(ev[2]);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "profile iteration");
            break;
        }
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&b, ev[1], ev[2]);
        ta += a;
        tb += b;
        ++done;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (rc != FW_OK) return rc;
    if (ms_a) *ms_a = ta / done;
    if (ms_b) *ms_b = tb / done;
    return flush(h);
}

fw_status fw_seg_step(fw_seg* h, int32_t iters, fw_seg_stats* stats) {
    if (!h) return invalid("handle is NULL");
    if (iters < 0) return invalid("iters must be >= 0");
    h->launches = 0;
    FW_CUDA(cudaEventRecord(h->ev0, h->stream));
    FW_TRY(read_state(h));
    for (int i = 0; i < iters && !h->h_state->done; ++i) {
        const int R = h->opts.refresh_every;
        if (R > 0 && h->h_state->iter - h->last_refresh >= R) FW_TRY(refresh_lu(h));
        h->ops->passA(h->b, h->stream);
        h->ops->passB(h->b, h->stream);
        h->launches += 2;
        FW_TRY(launch_check("iteration kernels"));
        FW_TRY(read_state(h));
    }
    FW_TRY(flush(h));
    FW_CUDA(cudaEventRecord(h->ev1, h->stream));
    FW_CUDA(cudaEventSynchronize(h->ev1));
    FW_TRY(read_state(h));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    fill_stats(h, stats, ms);
    return h->h_state->done ? status_of(*h->h_state) : FW_OK;
}

fw_status fw_seg_labels(fw_seg* h, int32_t* labels_host) {
    if (!h || !labels_host) return invalid("NULL argument");
    FW_TRY(flush(h));
    h->ops->labels(h->b, h->d_labels, h->stream);
    FW_TRY(launch_check("labels kernel"));
    FW_CUDA(cudaMemcpyAsync(labels_host, h->d_labels, 4 * size_t(h->n), cudaMemcpyDeviceToHost,
                            h->stream));
    FW_CUDA(cudaStreamSynchronize(h->stream));
    return FW_OK;
}

static fw_status copy_soa_to_host(fw_seg* h, const void* dev, double* out) {
    const size_t te = h->ops->elem();
    const size_t npad = size_t(h->b.pd.npad), K = size_t(h->K), n = size_t(h->n);
    std::vector<unsigned char> tmp(te * npad * K);
    FW_CUDA(cudaMemcpyAsync(tmp.data(), dev, tmp.size(), cudaMemcpyDeviceToHost, h->stream));
    FW_CUDA(cudaStreamSynchronize(h->stream));
    if (te == 4) {
        const float* t = reinterpret_cast<const float*>(tmp.data());
        for (size_t i = 0; i < n; ++i)
            for (size_t k = 0; k < K; ++k) out[i * K + k] = double(t[k * npad + i]);
    } else {
        const double* t = reinterpret_cast<const double*>(tmp.data());
        for (size_t i = 0; i < n; ++i)
            for (size_t k = 0; k < K; ++k) out[i * K + k] = t[k * npad + i];
    }
    return FW_OK;
}

fw_status fw_seg_get_U(fw_seg* h, double* U_host) {
    if (!h || !U_host) return invalid("NULL argument");
    try {
        FW_TRY(flush(h));
        return copy_soa_to_host(h, h->b.U, U_host);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

fw_status fw_seg_set_U(fw_seg* h, const double* U_host) {
    if (!h || !U_host) return invalid("NULL argument");
    try {
        const size_t te = h->ops->elem();
        const size_t npad = size_t(h->b.pd.npad), K = size_t(h->K), n = size_t(h->n);
        for (size_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (size_t k = 0; k < K; ++k) {
                const double x = U_host[i * K + k];
                if (!(x >= 0.0) || x > 1.0) return invalid("U entries must lie in [0, 1]");
                s += x;
            }
            if (std::fabs(s - 1.0) > 1e-5) return invalid("rows of U must sum to 1");
        }
        std::vector<unsigned char> tmp(te * npad * K, 0);
        if (te == 4) {
            float* t = reinterpret_cast<float*>(tmp.data());
            for (size_t i = 0; i < n; ++i)
                for (size_t k = 0; k < K; ++k) t[k * npad + i] = float(U_host[i * K + k]);
        } else {
            double* t = reinterpret_cast<double*>(tmp.data());
            for (size_t i = 0; i < n; ++i)
                for (size_t k = 0; k < K; ++k) t[k * npad + i] = U_host[i * K + k];
        }
        FW_CUDA(cudaStreamSynchronize(h->stream));
        FW_CUDA(cudaMemcpyAsync(h->b.U, tmp.data(), tmp.size(), cudaMemcpyHostToDevice, h->stream));
        FW_CUDA(cudaMemsetAsync(h->b.st, 0, sizeof(ProbState), h->stream));
        FW_CUDA(cudaStreamSynchronize(h->stream));
        return restart(h);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

fw_status fw_seg_get_grad(fw_seg* h, double* G_host, int32_t* choice_host, uint8_t* active_host) {
    if (!h) return invalid("handle is NULL");
    try {
        FW_TRY(flush(h));
        h->ops->grad(h->b, h->d_tmp, h->d_ch, h->stream);
        FW_TRY(launch_check("grad kernel"));
        if (G_host) FW_TRY(copy_soa_to_host(h, h->d_tmp, G_host));
        if (choice_host || active_host) {
            std::vector<uint8_t> ch(size_t(h->n));
            FW_CUDA(cudaMemcpyAsync(ch.data(), h->d_ch, size_t(h->n), cudaMemcpyDeviceToHost,
                                    h->stream));
            FW_CUDA(cudaStreamSynchronize(h->stream));
            for (int64_t i = 0; i < h->n; ++i) {
                if (choice_host) choice_host[i] = ch[size_t(i)] & 0x7f;
                if (active_host) active_host[i] = (ch[size_t(i)] & kActiveBit) ? 1 : 0;
            }
        }
        return FW_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

fw_status fw_seg_objective(fw_seg* h, double* E) {
    if (!h || !E) return invalid("NULL argument");
    try {
        FW_TRY(flush(h));
        return direct_objective(h, E);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

fw_status fw_seg_refresh(fw_seg* h) {
    if (!h) return invalid("handle is NULL");
    FW_TRY(refresh_lu(h));
    FW_CUDA(cudaStreamSynchronize(h->stream));
    return FW_OK;
}

fw_status fw_seg_get_stats(fw_seg* h, fw_seg_stats* stats) {
    if (!h || !stats) return invalid("NULL argument");
    FW_TRY(read_state(h));
    fill_stats(h, stats, 0.f);
    return FW_OK;
}

void fw_seg_destroy(fw_seg* h) { delete h; }

}  // extern "C"
