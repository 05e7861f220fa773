// Single-problem solver: the fw_seg_* entry points of include/fw_seg.h.
//
// Device state of a handle (one GPU, resident for the handle's lifetime, one
// allocation): padded CSR of the off-diagonal operator (int32 row_ptr / col,
// WT weights), U, L U, L S in class-major layout (T[K][npad]), choice (uint8)
// and fid (int8) per row, 4-bit classes for K <= 16, two banks of exact
// fixed-point totals, and one ProbState.  Both passes add their block totals
// into the iteration's bank; the stop test and the step follow from the bank
// (k_finish, or the next pass A inside a captured graph).
// A solve launches a CUDA graph that holds `iters_per_launch` iterations
// (pass A + pass B each, one k_finish at the end) and reads the state back
// after each launch; nothing else crosses the host-device boundary during the
// iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "fw_internal.h"

namespace fw {
const char* last_error_text();
}

using namespace fw;

static_assert(sizeof(fw_seg_opts) == 80, "fw_seg_opts ABI");
static_assert(sizeof(fw_seg_stats) == 64, "fw_seg_stats ABI");
static_assert(sizeof(fw_seg_forms) == 32, "fw_seg_forms ABI");

static fw_status invalid(const std::string& m) {
    set_error(m);
    return FW_ERR_INVALID_ARG;
}

#define FW_TRY(x)                          \
    do {                                   \
        fw_status s_ = (x);                \
        if (s_ != FW_OK) return s_;        \
    } while (0)

struct fw_seg {
    int device = 0;
    fw_seg_opts opts{};
    ProbLayout lay;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::unique_ptr<Ops> ops;
    ProbDesc pd{};
    ProbState* st = nullptr;        // device
    ProbState* h_state = nullptr;   // pinned mirror (start of one pinned block of three)
    ProbState* h_ring = nullptr;    // h_state + 1, [2]: state copies of queued graph launches
    cudaEvent_t ring_ev[2] = {nullptr, nullptr};
    char* mem = nullptr;            // the problem's arrays
    void* d_tmp = nullptr;          // T[K][npad]: fresh L U, gradient
    uint8_t* d_ch = nullptr;        // choice scratch of fw_seg_get_grad
    int32_t* d_labels = nullptr;
    double* d_opart = nullptr;
    cudaGraphExec_t graph = nullptr;
    int last_refresh = 0;
    int launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void*> dev_allocs;

    // device arrays: stream-ordered on the handle's stream, from the
    // library's pool (fast to re-create after a destroy)
    template <typename P>
    fw_status alloc(P** p, size_t bytes) {
        void* q = nullptr;
        const fw_status st = pool_alloc(&q, bytes, stream);
        if (st != FW_OK) return st;
        dev_allocs.push_back(q);
        *p = reinterpret_cast<P*>(q);
        return FW_OK;
    }
    ~fw_seg() {
        if (stream) cudaStreamSynchronize(stream);
        if (graph) cudaGraphExecDestroy(graph);
        for (void* p : dev_allocs) cudaFreeAsync(p, stream);   // back to the pool
        if (h_state) cudaFreeHost(h_state);   // h_ring lives in the same block
        for (cudaEvent_t e : ring_ev)
            if (e) cudaEventDestroy(e);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

static fw_status launch_check(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return FW_OK;
}

static fw_status read_state(fw_seg* h) {
    FW_CUDA(cudaMemcpyAsync(h->h_state, h->st, sizeof(ProbState), cudaMemcpyDeviceToHost,
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
    h->ops->flush(h->pd, h->st, h->stream);
    ++h->launches;
    return launch_check("flush kernel");
}

static fw_status refresh_lu(fw_seg* h) {
    FW_TRY(flush(h));
    h->ops->spmm(h->pd, h->pd.U, h->pd.LU, h->stream);
    ++h->launches;
    FW_TRY(launch_check("spmm kernel"));
    h->last_refresh = h->h_state->iter;
    return FW_OK;
}

// E(U) evaluated directly; d_tmp gets a fresh L U.
static fw_status direct_objective(fw_seg* h, double* E) {
    h->ops->spmm(h->pd, h->pd.U, h->d_tmp, h->stream);
    h->ops->objective(h->pd, h->d_tmp, h->d_opart, h->stream);
    h->launches += 2;
    FW_TRY(launch_check("objective kernels"));
    const int64_t nb = (h->lay.n + kBlock - 1) / kBlock;
    std::vector<double> part(size_t(nb), 0.0);
    FW_CUDA(cudaMemcpyAsync(part.data(), h->d_opart, sizeof(double) * nb,
                            cudaMemcpyDeviceToHost, h->stream));
    FW_CUDA(cudaStreamSynchronize(h->stream));
    double s = 0.0;
    for (double x : part) s += x;
    *E = s;
    return FW_OK;
}

// One GFW iteration: pass A, pass B, finish (3 launches).
static void iteration(fw_seg* h) {
    h->ops->passA(h->pd, h->st, h->stream, 0);
    h->ops->passB(h->pd, h->st, h->stream);
    h->ops->finish(h->pd, h->st, h->stream);
}

// Launches of one captured graph of m iterations: the step decision of each
// iteration but the last is taken inside the next pass A, so only the last
// iteration ends with k_finish.
static int graph_launches(int m) { return 2 * m + 1; }

static fw_status build_graph(fw_seg* h) {
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    FW_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < h->opts.iters_per_launch; ++i) {
        h->ops->passA(h->pd, h->st, h->stream, i > 0 ? 1 : 0);
        h->ops->passB(h->pd, h->st, h->stream);
    }
    h->ops->finish(h->pd, h->st, h->stream);
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

static fw_status copy_soa_to_host(fw_seg* h, const void* dev, double* out) {
    const size_t te = h->ops->elem();
    const size_t npad = size_t(h->lay.npad), K = size_t(h->lay.K), n = size_t(h->lay.n);
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

// ---------------------------------------------------------------- profile
// Everything a pass may change, copied aside so that timing runs of repeated
// passes leave the iterate as it was.
struct Snapshot {
    void *U = nullptr, *LU = nullptr, *LS = nullptr, *ch = nullptr, *c4 = nullptr;
    void *acc = nullptr, *st = nullptr;
};

static fw_status copy_problem_state(fw_seg* h, const Snapshot& s, bool save) {
    const size_t blk = h->ops->elem() * size_t(h->lay.npad) * size_t(h->lay.K);
    const size_t n = size_t(h->lay.n);
    struct Piece {
        void* dev;
        void* keep;
        size_t bytes;
    } pieces[] = {{h->pd.U, s.U, blk},
                  {h->pd.LU, s.LU, blk},
                  {h->pd.LS, s.LS, blk},
                  {h->pd.choice, s.ch, n},
                  {h->pd.cls4, s.c4, h->pd.cls4 ? (n + 1) / 2 : 0},
                  {h->pd.acc, s.acc, 8 * size_t(kAccTotal)},
                  {h->st, s.st, sizeof(ProbState)}};
    for (const Piece& p : pieces) {
        if (!p.bytes) continue;
        FW_CUDA(cudaMemcpyAsync(save ? p.keep : p.dev, save ? p.dev : p.keep, p.bytes,
                                cudaMemcpyDeviceToDevice, h->stream));
    }
    return FW_OK;
}

// Enqueue `body` once, as a captured graph when the stream can be captured
// (else directly), between two events recorded on the stream around it;
// *ms = the elapsed time.  The graph is uploaded before the first event so
// that the time is its execution only.
template <typename Body>
static fw_status time_enqueued(fw_seg* h, bool graph, Body body, cudaEvent_t e0, cudaEvent_t e1,
                               float* ms) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (graph) {
        FW_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        body();
        cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (e == cudaSuccess) e = cudaGraphUpload(ge, h->stream);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            if (ge) cudaGraphExecDestroy(ge);
            return cuda_fail(e, "profile graph");
        }
    }
    FW_CUDA(cudaEventRecord(e0, h->stream));
    if (graph) {
        const cudaError_t e = cudaGraphLaunch(ge, h->stream);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(ge);
            return cuda_fail(e, "cudaGraphLaunch");
        }
    } else {
        body();
    }
    FW_CUDA(cudaEventRecord(e1, h->stream));
    FW_CUDA(cudaEventSynchronize(e1));
    if (ge) cudaGraphExecDestroy(ge);
    FW_TRY(launch_check("profile kernels"));
    FW_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return FW_OK;
}

// Whether the handle's stream can be captured (the legacy default stream
// cannot); the capture error, if any, is cleared.
static bool stream_capturable(fw_seg* h) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const bool ok = cudaStreamEndCapture(h->stream, &g) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return ok;
}

extern "C" {

const char* fw_seg_last_error(void) { return last_error_text(); }

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
    o->class_table = FW_TABLE_AUTO;
    o->cuda_stream = nullptr;
    return FW_OK;
}

size_t fw_seg_footprint(int64_t n, int64_t nnz, int32_t K, int32_t weight_dtype) {
    const size_t te = weight_dtype == FW_WEIGHTS_F64 ? 8 : 4;
    const size_t we = weight_dtype == FW_WEIGHTS_F64 ? 8 : weight_dtype == FW_WEIGHTS_BF16 ? 2 : 4;
    ProbLayout lay;
    lay.n = n;
    lay.nnz = nnz;
    lay.nnz_pad = nnz + int64_t(kPadW - 1) * n;  // upper bound
    lay.npad = round_up(n, 32);
    lay.K = K;
    lay.tile_rows = tile_rows_for(n);
    lay.ntiles = int32_t((n + lay.tile_rows - 1) / lay.tile_rows);
    lay.cls4 = K <= 16;
    size_t b = problem_bytes(lay, te, we, true);
    b += te * size_t(lay.npad) * size_t(K) + 5 * size_t(n) + 8 * size_t(n / kBlock + 1);
    // stream-ordered temporaries of create
    b += 4 * (size_t(n) + 1) + 12 * size_t(nnz) + 12 * size_t(n) + 4096;
    return b;
}

fw_status fw_seg_create(fw_seg** out, int64_t n, const int32_t* row_ptr, const int32_t* col,
                        const double* w, int32_t K, const int32_t* labels,
                        const fw_seg_opts* opts_in) {
    try {
        if (!out) return invalid("out is NULL");
        *out = nullptr;
        fw_seg_opts o;
        if (opts_in) o = *opts_in;
        else fw_seg_default_opts(&o);
        FW_TRY(check_opts(o));
        const HostGraph g{n, row_ptr, col, w, K, labels};
        std::unique_ptr<fw_seg> h(new fw_seg());
        // Large inputs start their upload before the host's planning pass
        // over row_ptr and labels, which then runs while the copies are in
        // flight.  The O(1) checks (n, K, pointers, row_ptr ends) come first,
        // and so does the full planning pass whenever the padded entry count
        // could reach the 2^31 limit, so that a size the library rejects never
        // queues a copy.  On every error path the handle's destructor waits
        // for its stream, so the caller's arrays are not read after the call
        // returns.
        bool upload_first = n >= (int64_t(1) << 20);
        if (upload_first) {
            FW_TRY(check_graph_args(g));
            upload_first = int64_t(row_ptr[n]) + int64_t(kPadW - 1) * n < (int64_t(1) << 31);
        }
        if (!upload_first) FW_TRY(plan_problem(g, o, h->lay));
        FW_CUDA(cudaGetDevice(&h->device));
        h->opts = o;
        if (o.cuda_stream) {
            h->stream = static_cast<cudaStream_t>(o.cuda_stream);
        } else {
            FW_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
            h->own_stream = true;
        }
        Upload up(h->stream);
        FW_TRY(upload_inputs(g, up));
        if (upload_first) FW_TRY(plan_problem(g, o, h->lay));
        h->lay.cls4 = K <= 16;   // pass B gathers 4-bit classes (KMAX <= 16 forms)
        h->ops.reset(make_ops(o.weight_dtype, K));
        if (!h->ops) return invalid("no kernels for this weight dtype / K");
        FW_CUDA(h->ops->configure());
        FW_CUDA(cudaMallocHost(&h->h_state, 3 * sizeof(ProbState)));
        h->h_ring = h->h_state + 1;
        for (cudaEvent_t& e : h->ring_ev)
            FW_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        FW_CUDA(cudaEventCreate(&h->ev0));
        FW_CUDA(cudaEventCreate(&h->ev1));
        const size_t te = h->ops->elem(), we = h->ops->welem();
        const bool comb = o.laplacian == FW_LAPLACIAN_COMB;
        const ProbLayout& lay = h->lay;
        FW_TRY(h->alloc(&h->mem, problem_bytes(lay, te, we, comb)));
        place_problem(h->mem, lay, te, we, o, h->pd);
        FW_TRY(h->alloc(&h->st, sizeof(ProbState)));
        FW_TRY(h->alloc(&h->d_tmp, te * size_t(lay.npad) * size_t(lay.K)));
        FW_TRY(h->alloc(&h->d_ch, size_t(lay.n)));
        FW_TRY(h->alloc(&h->d_labels, 4 * size_t(lay.n)));
        FW_TRY(h->alloc(&h->d_opart, 8 * size_t((lay.n + kBlock - 1) / kBlock)));
        FW_TRY(assemble_uploaded(h->ops.get(), up, lay, h->pd, h->st, h->stream));
        FW_TRY(read_state(h.get()));
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
    const int R = h->opts.refresh_every;
    if (h->graph && R <= 0) {
        // Graph launches run one ahead of the host: while launch k+1 runs,
        // the state copied back after launch k is inspected, so the GPU does
        // not idle between launches.  A launch queued after the stop finds
        // `done` set and returns at once (it changes nothing).
        int queued = 0, head = 0;
        while (!h->h_state->done) {
            const int planned = h->h_state->iter + queued * m;   // if nothing stops
            if (queued < 2 && h->opts.max_iters - planned >= m) {
                const int slot = (head + queued) & 1;
                FW_CUDA(cudaGraphLaunch(h->graph, h->stream));
                FW_CUDA(cudaMemcpyAsync(h->h_ring + slot, h->st, sizeof(ProbState),
                                        cudaMemcpyDeviceToHost, h->stream));
                FW_CUDA(cudaEventRecord(h->ring_ev[slot], h->stream));
                h->launches += graph_launches(m);
                ++queued;
                continue;
            }
            if (queued == 0) break;   // fewer than m iterations left: the tail below
            FW_CUDA(cudaEventSynchronize(h->ring_ev[head]));
            *h->h_state = h->h_ring[head];
            head ^= 1;
            --queued;
        }
        if (queued) FW_TRY(read_state(h));   // the launch queued after the stop
    }
    while (!h->h_state->done) {
        if (R > 0 && h->h_state->iter - h->last_refresh >= R) FW_TRY(refresh_lu(h));
        const int remaining = h->opts.max_iters - h->h_state->iter;
        if (remaining >= m && h->graph) {
            FW_CUDA(cudaGraphLaunch(h->graph, h->stream));
            h->launches += graph_launches(m);
        } else {
            // direct launches with the decisions fused as in the graph; the
            // tail (< m iterations left) ends with one more pass pair whose
            // stop test, at the iteration cap, ends the solve
            const int it = remaining >= m ? m : remaining + 1;
            for (int i = 0; i < it; ++i) {
                h->ops->passA(h->pd, h->st, h->stream, i > 0 ? 1 : 0);
                h->ops->passB(h->pd, h->st, h->stream);
            }
            h->ops->finish(h->pd, h->st, h->stream);
            h->launches += 2 * it + 1;
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
    FW_TRY(restart_problem(h->ops.get(), h->pd, h->st, false, h->stream));
    h->launches += 4;
    h->last_refresh = 0;
    return FW_OK;
}

fw_status fw_seg_profile(fw_seg* h, int32_t iters, double* ms_a, double* ms_b, double* ms_f,
                         double* ms_iter, int32_t* in_graph) {
    if (!h || iters < 1 || iters > 4096) return invalid("bad arguments (iters in [1, 4096])");
    FW_TRY(read_state(h));
    if (h->h_state->done) return invalid("the solve has stopped: reset before profiling");
    const int m = iters;
    const bool graph = stream_capturable(h);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FW_CUDA(cudaEventCreate(&e0));
    FW_CUDA(cudaEventCreate(&e1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } guard{e0, e1};
    // 1. the solve's own form: m fused iterations and one finish
    float t_ab = 0.f, t_a = 0.f, t_b = 0.f, t_f = 0.f;
    FW_TRY(time_enqueued(h, graph, [&] {
        for (int i = 0; i < m; ++i) {
            h->ops->passA(h->pd, h->st, h->stream, i > 0 ? 1 : 0);
            h->ops->passB(h->pd, h->st, h->stream);
        }
        h->ops->finish(h->pd, h->st, h->stream);
    }, e0, e1, &t_ab));
    FW_TRY(read_state(h));
    if (h->h_state->done)
        return invalid("the stop rule held while profiling: reset and profile fewer iterations");
    // 2. one more iteration without its finish: its totals wait in bank cur,
    //    the state a fused pass A starts from
    h->ops->passA(h->pd, h->st, h->stream, 0);
    h->ops->passB(h->pd, h->st, h->stream);
    FW_TRY(launch_check("profile kernels"));
    Temps t(h->stream);
    Snapshot s;
    const size_t blk = h->ops->elem() * size_t(h->lay.npad) * size_t(h->lay.K);
    FW_TRY(t.get(&s.U, blk));
    FW_TRY(t.get(&s.LU, blk));
    FW_TRY(t.get(&s.LS, blk));
    FW_TRY(t.get(&s.ch, size_t(h->lay.n)));
    FW_TRY(t.get(&s.c4, size_t(h->lay.n) / 2 + 1));
    FW_TRY(t.get(&s.acc, 8 * size_t(kAccTotal)));
    FW_TRY(t.get(&s.st, sizeof(ProbState)));
    FW_TRY(copy_problem_state(h, s, true));
    // 3. m launches of pass B back to back (each recomputes the same L S)
    FW_TRY(time_enqueued(h, graph, [&] {
        for (int i = 0; i < m; ++i) h->ops->passB(h->pd, h->st, h->stream);
    }, e0, e1, &t_b));
    FW_TRY(copy_problem_state(h, s, false));
    // 4. m launches of the fused pass A back to back (each takes the same
    //    decision from bank cur and applies it once more)
    FW_TRY(time_enqueued(h, graph, [&] {
        for (int i = 0; i < m; ++i) h->ops->passA(h->pd, h->st, h->stream, 1);
    }, e0, e1, &t_a));
    FW_TRY(copy_problem_state(h, s, false));
    // 5. the finishing kernel of that iteration, which also leaves the
    //    handle in a consistent state (iters + 1 iterations done)
    FW_TRY(time_enqueued(h, false, [&] { h->ops->finish(h->pd, h->st, h->stream); }, e0, e1,
                         &t_f));
    if (ms_a) *ms_a = double(t_a) / m;
    if (ms_b) *ms_b = double(t_b) / m;
    if (ms_f) *ms_f = double(t_f);
    if (ms_iter) *ms_iter = double(t_ab) / m;
    if (in_graph) *in_graph = graph ? 1 : 0;
    h->launches += 2 * m + 1 + 2 + 2 * m + 1;
    FW_TRY(read_state(h));
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
        iteration(h);
        h->launches += 3;
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
    h->ops->labels(h->pd, h->d_labels, h->stream);
    FW_TRY(launch_check("labels kernel"));
    FW_CUDA(cudaMemcpyAsync(labels_host, h->d_labels, 4 * size_t(h->lay.n),
                            cudaMemcpyDeviceToHost, h->stream));
    FW_CUDA(cudaStreamSynchronize(h->stream));
    return FW_OK;
}

fw_status fw_seg_oneshot(fw_seg* h, int32_t* labels_host, double* ms) {
    if (!h) return invalid("handle is NULL");
    FW_CUDA(cudaEventRecord(h->ev0, h->stream));
    h->ops->oneshot(h->pd, h->d_labels, h->stream);
    FW_TRY(launch_check("one-shot kernel"));
    FW_CUDA(cudaEventRecord(h->ev1, h->stream));
    if (labels_host)
        FW_CUDA(cudaMemcpyAsync(labels_host, h->d_labels, 4 * size_t(h->lay.n),
                                cudaMemcpyDeviceToHost, h->stream));
    FW_CUDA(cudaStreamSynchronize(h->stream));
    if (ms) {
        float t = 0.f;
        FW_CUDA(cudaEventElapsedTime(&t, h->ev0, h->ev1));
        *ms = t;
    }
    return FW_OK;
}

fw_status fw_seg_get_U(fw_seg* h, double* U_host) {
    if (!h || !U_host) return invalid("NULL argument");
    try {
        FW_TRY(flush(h));
        return copy_soa_to_host(h, h->pd.U, U_host);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

fw_status fw_seg_set_U(fw_seg* h, const double* U_host) {
    if (!h || !U_host) return invalid("NULL argument");
    try {
        const size_t te = h->ops->elem();
        const size_t npad = size_t(h->lay.npad), K = size_t(h->lay.K), n = size_t(h->lay.n);
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
        FW_CUDA(cudaMemcpyAsync(h->pd.U, tmp.data(), tmp.size(), cudaMemcpyHostToDevice,
                                h->stream));
        FW_TRY(restart_problem(h->ops.get(), h->pd, h->st, true, h->stream));
        FW_CUDA(cudaStreamSynchronize(h->stream));
        h->last_refresh = 0;
        return read_state(h);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

fw_status fw_seg_get_grad(fw_seg* h, double* G_host, int32_t* choice_host, uint8_t* active_host) {
    if (!h) return invalid("handle is NULL");
    try {
        FW_TRY(flush(h));
        h->ops->grad(h->pd, h->st, h->d_tmp, h->d_ch, h->stream);
        FW_TRY(launch_check("grad kernel"));
        if (G_host) FW_TRY(copy_soa_to_host(h, h->d_tmp, G_host));
        if (choice_host || active_host) {
            std::vector<uint8_t> ch(size_t(h->lay.n));
            FW_CUDA(cudaMemcpyAsync(ch.data(), h->d_ch, size_t(h->lay.n), cudaMemcpyDeviceToHost,
                                    h->stream));
            FW_CUDA(cudaStreamSynchronize(h->stream));
            for (int64_t i = 0; i < h->lay.n; ++i) {
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

fw_status fw_seg_lmo_gap(fw_seg* h, double* gap) {
    if (!h || !gap) return invalid("NULL argument");
    try {
        FW_TRY(flush(h));
        h->ops->spmm(h->pd, h->pd.U, h->d_tmp, h->stream);
        h->ops->lmo_gap(h->pd, h->d_tmp, h->d_opart, h->stream);
        h->launches += 2;
        FW_TRY(launch_check("LMO gap kernels"));
        const int64_t nb = (h->lay.n + kBlock - 1) / kBlock;
        std::vector<double> part(size_t(nb), 0.0);
        FW_CUDA(cudaMemcpyAsync(part.data(), h->d_opart, sizeof(double) * nb,
                                cudaMemcpyDeviceToHost, h->stream));
        FW_CUDA(cudaStreamSynchronize(h->stream));
        double s = 0.0;
        for (double x : part) s += x;
        *gap = s;
        return FW_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

fw_status fw_seg_refresh(fw_seg* h) {
    if (!h) return invalid("handle is NULL");
    FW_TRY(read_state(h));
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

fw_status fw_seg_get_forms(fw_seg* h, fw_seg_forms* f) {
    if (!h || !f) return invalid("NULL argument");
    std::memset(f, 0, sizeof(*f));
    f->lanes_per_row = h->pd.lanes;
    f->index_width = h->pd.col16 ? 16 : 32;
    f->class_table = h->pd.tab_grid > 0 ? 1 : 0;
    f->table_blocks = h->pd.tab_grid;
    f->tiles = h->pd.ntiles;
    f->tile_rows = h->pd.tile_rows;
    f->kmax = h->ops ? h->ops->kmax() : 0;
    return FW_OK;
}

void fw_seg_destroy(fw_seg* h) { delete h; }

}  // extern "C"
