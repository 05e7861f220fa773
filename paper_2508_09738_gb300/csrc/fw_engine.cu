// Batch engine, batched solves (fw_batch_*) and the serving loop (fw_srv_*).
//
// The engine owns one device pool holding every resident problem at its own
// offsets (first-fit allocation, 256-byte aligned), a descriptor and a state
// per slot, the work list of the persistent kernel and its grid barrier.
// run() launches the persistent kernel over the tiles of every live problem.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fw_batch.cuh"
#include "fw_internal.h"

namespace fw {

BatchKern* make_batch_kern_f32(int kmax);
BatchKern* make_batch_kern_bf16(int kmax);
BatchKern* make_batch_kern_f64(int kmax);

BatchKern* make_batch_kern(int weight_dtype, int kmax) {
    switch (weight_dtype) {
        case FW_WEIGHTS_F32: return make_batch_kern_f32(kmax);
        case FW_WEIGHTS_BF16: return make_batch_kern_bf16(kmax);
        case FW_WEIGHTS_F64: return make_batch_kern_f64(kmax);
        default: return nullptr;
    }
}

static fw_status invalid(const std::string& m) {
    set_error(m);
    return FW_ERR_INVALID_ARG;
}

#define FW_TRY(x)                      \
    do {                               \
        fw_status s_ = (x);            \
        if (s_ != FW_OK) return s_;    \
    } while (0)

// First-fit allocator of byte ranges [0, cap), 256-byte granules.
class RangeAlloc {
public:
    void init(size_t cap) {
        free_.clear();
        cap_ = cap / 256 * 256;
        if (cap_) free_[0] = cap_;
        used_ = 0;
    }
    // offset, or SIZE_MAX when no free range is large enough
    size_t alloc(size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const {
        size_t m = 0;
        for (auto& kv : free_) m = std::max(m, kv.second);
        return m;
    }
    size_t used() const { return used_; }
    size_t cap() const { return cap_; }

private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0;
};

struct Slot {
    bool used = false;
    ProbLayout lay;
    ProbDesc pd{};
    fw_seg_opts opts{};
    size_t off = 0, bytes = 0;
};

class Engine {
public:
    int wd = 0, kmax = 4;
    size_t te = 4, we = 4;
    std::unique_ptr<Ops> ops;
    std::unique_ptr<BatchKern> bk;
    cudaStream_t stream = nullptr, side = nullptr;
    bool own_stream = false;
    char* pool = nullptr;
    RangeAlloc ra;
    std::vector<Slot> slots;
    ProbDesc* d_desc = nullptr;
    ProbState* d_state = nullptr;
    ProbState* h_state = nullptr;  // pinned mirror of every slot's state
    int2* d_work = nullptr;
    size_t work_cap = 0;
    std::vector<int2> h_work;
    int* d_live = nullptr;          // live problems (per-item schedule's finish)
    std::vector<int> h_live;
    bool two_stage = false;         // a live problem has multi-sub-tile tiles
    GridBar* d_bar = nullptr;
    GridBar* h_bar = nullptr;      // pinned
    int sms = 0, occ = 0, bps = 0, grid = 0, schedule = FW_SCHED_DYNAMIC;
    // use_graph: FW_GRAPH_OFF, FW_GRAPH_REQUIRED or FW_GRAPH_PREFERRED;
    // graph_captured: 1 when the last launch ran from a captured graph;
    // graph_error: the CUDA error of the last failed capture (0: none)
    int use_graph = FW_GRAPH_REQUIRED, graph_captured = 0, graph_error = 0, expect_extra = 0;
    int kmax_kern = 4;     // class bound of the persistent kernel (>= kmax)
    int lanes_all = 0;     // lanes per row of every problem (0: each problem's own)
    // serving: a lone live problem runs the single-problem kernels (slots then
    // carry the 4-bit class array those kernels gather)
    bool plain_path = false;
    std::map<int, std::unique_ptr<Ops>> plain;   // per class bound
    // Lone-problem epochs (serving): a captured graph of lone_iters fused
    // iterations of slot lone_slot, kept up to two launches ahead of the host;
    // after each launch the slot's state is copied into a pinned ring entry
    // whose event the host waits for, so the GPU does not idle between epochs.
    cudaGraphExec_t lone_graph = nullptr;
    int lone_slot = -1, lone_iters = 0;
    ProbState* h_ring = nullptr;                 // pinned [2]
    cudaEvent_t ring_ev[2] = {nullptr, nullptr};
    int ring_head = 0, ring_queued = 0;
    long long budget = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = -1;
    bool work_dirty = true;
    int32_t* d_labels = nullptr;
    size_t d_labels_cap = 0;

    ~Engine() {
        if (stream) cudaStreamSynchronize(stream);
        if (side) cudaStreamSynchronize(side);
        if (graph) cudaGraphExecDestroy(graph);
        if (lone_graph) cudaGraphExecDestroy(lone_graph);
        for (cudaEvent_t ev : ring_ev)
            if (ev) cudaEventDestroy(ev);
        if (h_ring) cudaFreeHost(h_ring);
        for (void* p : {(void*)pool, (void*)d_desc, (void*)d_state, (void*)d_work, (void*)d_bar,
                        (void*)d_labels, (void*)d_live})
            if (p) cudaFree(p);
        if (h_state) cudaFreeHost(h_state);
        if (h_bar) cudaFreeHost(h_bar);
        if (side) cudaStreamDestroy(side);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }

    fw_status dev_alloc(void** p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 256));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " +
                      cudaGetErrorString(e));
            return FW_ERR_NO_MEMORY;
        }
        return FW_OK;
    }

    fw_status init(int weight_dtype, int K_max, size_t pool_bytes, int max_slots, void* user_stream,
                   int spin_ms, int blocks_per_sm, int sched) {
        wd = weight_dtype;
        kmax = kmax_for(K_max);
        ops.reset(make_ops(wd, kmax));
        bk.reset(make_batch_kern(wd, kmax));
        if (!ops || !bk) return invalid("no kernels for this weight dtype / K");
        te = ops->elem();
        we = ops->welem();
        FW_CUDA(ops->configure());
        FW_CUDA(bk->configure());
        if (user_stream) {
            stream = static_cast<cudaStream_t>(user_stream);
        } else {
            FW_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
            own_stream = true;
        }
        FW_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        FW_TRY(dev_alloc((void**)&pool, pool_bytes));
        ra.init(pool_bytes);
        slots.assign(size_t(max_slots), Slot());
        FW_TRY(dev_alloc((void**)&d_desc, sizeof(ProbDesc) * size_t(max_slots)));
        FW_TRY(dev_alloc((void**)&d_state, sizeof(ProbState) * size_t(max_slots)));
        FW_TRY(dev_alloc((void**)&d_live, sizeof(int) * size_t(max_slots)));
        FW_CUDA(cudaMemset(d_state, 0, sizeof(ProbState) * size_t(max_slots)));
        FW_CUDA(cudaMallocHost(&h_state, sizeof(ProbState) * size_t(max_slots)));
        std::memset(h_state, 0, sizeof(ProbState) * size_t(max_slots));
        FW_TRY(dev_alloc((void**)&d_bar, sizeof(GridBar)));
        FW_CUDA(cudaMallocHost(&h_bar, sizeof(GridBar)));
        int dev = 0;
        FW_CUDA(cudaGetDevice(&dev));
        FW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int coop = 0;
        FW_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        if (!coop) {
            set_error("device does not support cooperative launches");
            return FW_ERR_UNSUPPORTED;
        }
        kmax_kern = kmax;
        FW_CUDA(bk->occupancy(&occ));
        if (occ < 1) {
            set_error("persistent kernel cannot be resident");
            return FW_ERR_UNSUPPORTED;
        }
        int clock_khz = 0;
        FW_CUDA(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev));
        if (clock_khz <= 0) clock_khz = 2100000;
        budget = (long long)std::max(spin_ms, 1) * (long long)clock_khz;
        set_grid(blocks_per_sm > 0 ? blocks_per_sm : occ,
                 (sched == FW_SCHED_STATIC || sched == FW_SCHED_ITEMS) ? sched : FW_SCHED_DYNAMIC);
        return FW_OK;
    }

    // Persistent kernel compiled for class bound km >= kmax (the same
    // arithmetic for every K <= kmax; only bin strides and guards differ).
    fw_status set_kernel_kmax(int km) {
        if (km == kmax_kern) return FW_OK;
        std::unique_ptr<BatchKern> k(make_batch_kern(wd, km));
        if (!k) return invalid("no persistent kernel for this class bound");
        FW_CUDA(k->configure());
        int o = 0;
        FW_CUDA(k->occupancy(&o));
        if (o < 1) {
            set_error("persistent kernel cannot be resident");
            return FW_ERR_UNSUPPORTED;
        }
        bk = std::move(k);
        kmax_kern = km;
        occ = o;
        set_grid(std::min(bps, occ), schedule);
        return FW_OK;
    }

    // Lanes per CSR row of every problem (0: each problem's planned count).
    fw_status set_lanes(int L) {
        lanes_all = L;
        for (int s = 0; s < nslots(); ++s) {
            Slot& sl = slots[size_t(s)];
            if (!sl.used) continue;
            sl.pd.lanes = L > 0 ? L : sl.lay.lanes;
            FW_CUDA(cudaMemcpyAsync(d_desc + s, &sl.pd, sizeof(ProbDesc), cudaMemcpyHostToDevice,
                                    stream));
        }
        FW_CUDA(cudaStreamSynchronize(stream));
        invalidate_graph();
        return FW_OK;
    }

    void set_grid(int b, int sched) {
        bps = std::max(1, std::min(b, occ));
        grid = bps * sms;
        schedule = sched;
        invalidate_graph();
    }
    void invalidate_graph() {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        graph_iters = -1;
    }

    int nslots() const { return int(slots.size()); }
    int free_slot() const {
        for (int i = 0; i < nslots(); ++i)
            if (!slots[i].used) return i;
        return -1;
    }
    size_t bytes_for(const ProbLayout& lay, const fw_seg_opts& o) const {
        return problem_bytes(lay, te, we, o.laplacian == FW_LAPLACIAN_COMB);
    }
    bool fits(size_t bytes) const { return ra.largest() >= (bytes + 255) / 256 * 256; }

    // Upload and assemble a planned problem into a free slot (side stream).
    fw_status add(const HostGraph& g, const fw_seg_opts& o, const ProbLayout& lay, int* out) {
        if (lay.K > kmax) {
            set_error("K above the engine's class bound");
            return FW_ERR_UNSUPPORTED;
        }
        const int s = free_slot();
        if (s < 0) {
            set_error("no free slot");
            return FW_ERR_NO_MEMORY;
        }
        const size_t bytes = bytes_for(lay, o);
        const size_t off = ra.alloc(bytes);
        if (off == SIZE_MAX) {
            set_error("problem does not fit the free device pool");
            return FW_ERR_NO_MEMORY;
        }
        Slot& sl = slots[size_t(s)];
        sl.lay = lay;
        sl.opts = o;
        sl.off = off;
        sl.bytes = bytes;
        place_problem(pool + off, lay, te, we, o, sl.pd);
        fw_status rc = assemble_problem(ops.get(), g, lay, sl.pd, d_state + s, side);
        if (rc == FW_OK) {
            cudaError_t e = cudaMemcpyAsync(d_desc + s, &sl.pd, sizeof(ProbDesc),
                                            cudaMemcpyHostToDevice, side);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h_state + s, d_state + s, sizeof(ProbState),
                                                      cudaMemcpyDeviceToHost, side);
            if (e == cudaSuccess) e = cudaStreamSynchronize(side);
            if (e != cudaSuccess) rc = cuda_fail(e, "slot upload");
        }
        if (rc != FW_OK) {
            cudaStreamSynchronize(side);
            ra.release(off, bytes);
            sl = Slot();
            return rc;
        }
        sl.used = true;
        work_dirty = true;
        *out = s;
        return FW_OK;
    }

    void remove(int s) {
        Slot& sl = slots[size_t(s)];
        if (!sl.used) return;
        if (s == lone_slot) {   // queued lone epochs still name this slot's memory
            drain_lone();
            if (lone_graph) cudaGraphExecDestroy(lone_graph);
            lone_graph = nullptr;
            lone_slot = -1;
        }
        ra.release(sl.off, sl.bytes);
        sl = Slot();
        work_dirty = true;
    }

    fw_status restart(int s, cudaStream_t st) {
        return restart_problem(ops.get(), slots[size_t(s)].pd, d_state + s, false, st);
    }

    // Problems of at least this many rows stay out of batched launches (the
    // server runs them alone); the batch API keeps every problem.
    int64_t shared_max_rows = INT64_MAX;

    // Work list of the live problems (used, not done, below shared_max_rows).
    int build_work() {
        std::vector<int2> w;
        std::vector<int> live;
        bool two = false;
        for (int s = 0; s < nslots(); ++s) {
            if (!slots[size_t(s)].used || h_state[s].done) continue;
            if (slots[size_t(s)].lay.n >= shared_max_rows) continue;
            live.push_back(s);
            two = two || slots[size_t(s)].lay.tile_rows > kBlock;
            for (int t = 0; t < slots[size_t(s)].lay.ntiles; ++t) w.push_back(make_int2(s, t));
        }
        if (w.size() != h_work.size() || live != h_live ||
            !std::equal(w.begin(), w.end(), h_work.begin(),
                        [](const int2& x, const int2& y) { return x.x == y.x && x.y == y.y; }))
            work_dirty = true;
        h_work.swap(w);
        h_live.swap(live);
        two_stage = two;
        return int(h_live.size());
    }

    fw_status ensure_work_cap(size_t n) {
        if (n <= work_cap) return FW_OK;
        if (d_work) cudaFree(d_work);
        d_work = nullptr;
        work_cap = std::max<size_t>(n, 2 * work_cap);
        return dev_alloc((void**)&d_work, sizeof(int2) * work_cap);
    }

    BatchArgs args(int nlive, int iters) const {
        BatchArgs a{};
        a.desc = d_desc;
        a.state = d_state;
        a.work = d_work;
        a.nwork = int32_t(h_work.size());
        a.nlive = nlive;
        a.iters = iters;
        a.dynamic = schedule == FW_SCHED_DYNAMIC;
        a.expect_extra = expect_extra;
        a.bar = d_bar;
        a.budget = budget;
        return a;
    }

    // Enqueue one persistent launch of `iters` iterations over the live
    // problems on `stream`; *nlive_out = live problems (0: nothing launched).
    fw_status launch(int iters, int* nlive_out) {
        FW_TRY(drain_lone());
        const int nlive = build_work();
        *nlive_out = nlive;
        if (nlive == 0) return FW_OK;
        if (work_dirty) {
            FW_TRY(ensure_work_cap(h_work.size()));
            FW_CUDA(cudaMemcpyAsync(d_work, h_work.data(), sizeof(int2) * h_work.size(),
                                    cudaMemcpyHostToDevice, stream));
            FW_CUDA(cudaMemcpyAsync(d_live, h_live.data(), sizeof(int) * h_live.size(),
                                    cudaMemcpyHostToDevice, stream));
            invalidate_graph();
            work_dirty = false;
        }
        const BatchArgs a = args(nlive, iters);
        const ItemArgs ia{d_desc, d_state, d_work, d_live};
        const bool items = schedule == FW_SCHED_ITEMS;
        // one launch's work: the barrier record cleared, then the persistent
        // kernel or the per-item launches
        auto enqueue = [&]() -> cudaError_t {
            cudaError_t e = cudaMemsetAsync(d_bar, 0, sizeof(GridBar), stream);
            if (e != cudaSuccess) return e;
            if (items)
                return bk->launch_items(ia, int(h_work.size()), nlive, iters, two_stage, stream);
            return bk->launch(a, grid, stream);
        };
        bool from_graph = false;
        if (use_graph != FW_GRAPH_OFF) {
            if (!graph || graph_iters != iters) {
                invalidate_graph();
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    const cudaError_t e2 = enqueue();
                    e = cudaStreamEndCapture(stream, &g);
                    if (e == cudaSuccess) e = e2;
                    if (e == cudaSuccess) e = cudaGraphInstantiate(&graph, g, 0);
                    if (g) cudaGraphDestroy(g);
                }
                cudaGetLastError();
                if (e != cudaSuccess) {
                    graph = nullptr;
                    graph_captured = 0;
                    graph_error = int(e);
                    if (use_graph == FW_GRAPH_REQUIRED)
                        return cuda_fail(e, "capturing the persistent launch in a CUDA graph "
                                            "(use_graph = FW_GRAPH_PREFERRED allows direct "
                                            "launches)");
                } else {
                    graph_iters = iters;
                    graph_error = 0;
                }
            }
            if (graph) {
                FW_CUDA(cudaGraphLaunch(graph, stream));
                from_graph = true;
            }
        }
        if (!from_graph) FW_CUDA(enqueue());
        graph_captured = from_graph ? 1 : 0;
        return FW_OK;
    }

    fw_status plain_ops(int K, Ops** out) {
        const int km = kmax_for(K);
        auto it = plain.find(km);
        if (it == plain.end()) {
            std::unique_ptr<Ops> o(make_ops(wd, K));
            if (!o) return invalid("no kernels for this weight dtype / K");
            FW_CUDA(o->configure());
            it = plain.emplace(km, std::move(o)).first;
        }
        *out = it->second.get();
        return FW_OK;
    }

    // The one live problem when there is exactly one (else -1).
    int lone_live() const {
        int live = -1, cnt = 0;
        for (int s = 0; s < nslots(); ++s)
            if (slots[size_t(s)].used && !h_state[s].done) {
                live = s;
                ++cnt;
            }
        return cnt == 1 ? live : -1;
    }

    // Wait for queued lone epochs; h_state then holds the device state.
    fw_status drain_lone() {
        if (ring_queued == 0) return FW_OK;
        ring_queued = 0;
        FW_CUDA(cudaStreamSynchronize(stream));
        FW_CUDA(cudaMemcpy(h_state, d_state, sizeof(ProbState) * slots.size(),
                           cudaMemcpyDeviceToHost));
        return FW_OK;
    }

    // Queue lone epochs of `iters` iterations of slot s until two are in
    // flight.  false: the stream cannot be captured (nothing queued).
    fw_status lone_queue(int s, int iters, bool* ok) {
        *ok = false;
        if (!h_ring) {
            FW_CUDA(cudaMallocHost(&h_ring, 2 * sizeof(ProbState)));
            for (cudaEvent_t& ev : ring_ev)
                FW_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        }
        if (!lone_graph || lone_slot != s || lone_iters != iters) {
            FW_TRY(drain_lone());
            if (lone_graph) cudaGraphExecDestroy(lone_graph);
            lone_graph = nullptr;
            lone_slot = -1;
            Ops* op = nullptr;
            FW_TRY(plain_ops(slots[size_t(s)].lay.K, &op));
            const ProbDesc& pd = slots[size_t(s)].pd;
            ProbState* st = d_state + s;
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (int i = 0; i < iters; ++i) {
                    op->passA(pd, st, stream, i > 0 ? 1 : 0);
                    op->passB(pd, st, stream);
                }
                op->finish(pd, st, stream);
                e = cudaStreamEndCapture(stream, &g);
                if (e == cudaSuccess) e = cudaGraphInstantiate(&lone_graph, g, 0);
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();
            if (e != cudaSuccess) {
                lone_graph = nullptr;
                return FW_OK;
            }
            lone_slot = s;
            lone_iters = iters;
        }
        while (ring_queued < 2) {
            const int k = (ring_head + ring_queued) & 1;
            FW_CUDA(cudaGraphLaunch(lone_graph, stream));
            FW_CUDA(cudaMemcpyAsync(h_ring + k, d_state + s, sizeof(ProbState),
                                    cudaMemcpyDeviceToHost, stream));
            FW_CUDA(cudaEventRecord(ring_ev[k], stream));
            ++ring_queued;
        }
        graph_captured = 1;
        *ok = true;
        return FW_OK;
    }

    // The state after the oldest queued lone epoch (the newer one keeps running).
    fw_status lone_collect() {
        FW_CUDA(cudaEventSynchronize(ring_ev[ring_head]));
        h_state[lone_slot] = h_ring[ring_head];
        ring_head ^= 1;
        --ring_queued;
        return FW_OK;
    }

    // One epoch of `iters` iterations.  With a single live problem (serving)
    // they run as the single-problem kernels of fw_seg_solve: pass A with the
    // previous decision fused in and pass B per iteration, one finish at the
    // end -- the same arithmetic as the persistent kernel, in its faster
    // compile-time forms, and without grid barriers.  The state either path
    // leaves (decision committed, totals cleared) is the one the other starts
    // from.  Otherwise the persistent launch over every live problem.
    fw_status launch_epoch(int iters, int* nlive_out) {
        if (plain_path) {
            int live = -1, cnt = 0;
            for (int s = 0; s < nslots(); ++s)
                if (slots[size_t(s)].used && !h_state[s].done) {
                    live = s;
                    ++cnt;
                }
            if (cnt == 1) {
                Ops* op = nullptr;
                FW_TRY(plain_ops(slots[size_t(live)].lay.K, &op));
                const ProbDesc& pd = slots[size_t(live)].pd;
                ProbState* st = d_state + live;
                FW_CUDA(cudaMemsetAsync(d_bar, 0, sizeof(GridBar), stream));
                for (int i = 0; i < iters; ++i) {
                    op->passA(pd, st, stream, i > 0 ? 1 : 0);
                    op->passB(pd, st, stream);
                }
                op->finish(pd, st, stream);
                FW_CUDA(cudaGetLastError());
                graph_captured = 0;
                *nlive_out = 1;
                return FW_OK;
            }
        }
        return launch(iters, nlive_out);
    }

    // Copy every slot's state and the barrier record back after a launch.
    fw_status collect() {
        FW_CUDA(cudaMemcpyAsync(h_state, d_state, sizeof(ProbState) * slots.size(),
                                cudaMemcpyDeviceToHost, stream));
        FW_CUDA(cudaMemcpyAsync(h_bar, d_bar, sizeof(GridBar), cudaMemcpyDeviceToHost, stream));
        FW_CUDA(cudaStreamSynchronize(stream));
        if (h_bar->error) {
            set_error("grid barrier wait ran out of its budget");
            return FW_ERR_TIMEOUT;
        }
        return FW_OK;
    }

    fw_status run(int iters) {
        int nlive = 0;
        FW_TRY(launch(iters, &nlive));
        if (nlive == 0) return FW_OK;
        return collect();
    }

    fw_status labels(int s, int32_t* out, cudaStream_t st) {
        const Slot& sl = slots[size_t(s)];
        if (size_t(sl.lay.n) > d_labels_cap) {
            if (d_labels) cudaFree(d_labels);
            d_labels = nullptr;
            d_labels_cap = size_t(sl.lay.n);
            FW_TRY(dev_alloc((void**)&d_labels, 4 * d_labels_cap));
        }
        ops->labels(sl.pd, d_labels, st);
        FW_CUDA(cudaGetLastError());
        FW_CUDA(cudaMemcpyAsync(out, d_labels, 4 * size_t(sl.lay.n), cudaMemcpyDeviceToHost, st));
        FW_CUDA(cudaStreamSynchronize(st));
        return FW_OK;
    }

    fw_status get_U(int s, double* out) {
        const Slot& sl = slots[size_t(s)];
        const size_t np = size_t(sl.lay.npad), K = size_t(sl.lay.K), n = size_t(sl.lay.n);
        std::vector<unsigned char> tmp(te * np * K);
        FW_CUDA(cudaMemcpyAsync(tmp.data(), sl.pd.U, tmp.size(), cudaMemcpyDeviceToHost, stream));
        FW_CUDA(cudaStreamSynchronize(stream));
        for (size_t i = 0; i < n; ++i)
            for (size_t k = 0; k < K; ++k)
                out[i * K + k] = te == 4 ? double(reinterpret_cast<float*>(tmp.data())[k * np + i])
                                         : reinterpret_cast<double*>(tmp.data())[k * np + i];
        return FW_OK;
    }
};

static void fill_stats_from(const ProbState& st, fw_seg_stats* s, int launches, double ms) {
    s->iters = st.iter;
    s->status = st.done ? st.status : FW_PENDING;
    s->active_rows = st.active;
    s->launches = launches;
    s->gap = st.g;
    s->gap0 = st.g0;
    s->q = st.q;
    s->alpha = st.alpha;
    s->objective = st.E;
    s->ms = ms;
}

}  // namespace fw

using namespace fw;

static_assert(sizeof(fw_graph) == 48, "fw_graph ABI");
static_assert(sizeof(fw_batch_opts) == 48, "fw_batch_opts ABI");
static_assert(sizeof(fw_batch_info) == 56, "fw_batch_info ABI");
static_assert(sizeof(fw_srv_opts) == 48, "fw_srv_opts ABI");
static_assert(sizeof(fw_srv_info) == 72, "fw_srv_info ABI");

// =================================================================== batch

struct fw_batch {
    Engine eng;
    int P = 0;
    fw_batch_opts bo{};
    int ipl = 0;            // iterations per launch in use (0: all in one)
    int max_iters = 0;
    int tuned = 0;
    double tune_ms = 0.0;
    int launches = 0;
};

static std::string tune_signature(const fw_batch* b) {
    int64_t rows = 0, nnz = 0, tiles = 0;
    for (const Slot& s : b->eng.slots) {
        rows += s.lay.n;
        nnz += s.lay.nnz_pad;
        tiles += s.lay.ntiles;
    }
    cudaDeviceProp p{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&p, dev);
    char buf[512];
    std::snprintf(buf, sizeof(buf), "v2|%s|wd%d|k%d|P%d|rows%lld|nnz%lld|tiles%lld|want%d%d%d%d",
                  p.name, b->eng.wd, b->eng.kmax, b->P, (long long)rows, (long long)nnz,
                  (long long)tiles, b->bo.blocks_per_sm, b->bo.schedule, b->bo.lanes_per_row,
                  b->bo.iters_per_launch);
    std::string s(buf);
    for (char& c : s)
        if (c == ' ') c = '_';
    return s;
}

static const char* tune_path(const fw_batch* b) {
    if (b->bo.tune_cache) return b->bo.tune_cache;
    return std::getenv("FW_TUNE_CACHE");
}

// A tuned configuration of the persistent launch.
struct TuneChoice {
    int bps = 0, sched = FW_SCHED_DYNAMIC, lanes = 0, kmax = 4, ipl = 0;
};

static bool tune_lookup(const fw_batch* b, const std::string& sig, TuneChoice* c) {
    const char* path = tune_path(b);
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024], key[600];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        TuneChoice t;
        if (std::sscanf(line, "%599s %d %d %d %d %d", key, &t.bps, &t.sched, &t.lanes, &t.kmax,
                        &t.ipl) == 6 &&
            sig == key) {
            *c = t;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

static void tune_store(const fw_batch* b, const std::string& sig, const TuneChoice& c) {
    const char* path = tune_path(b);
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d %d\n", sig.c_str(), c.bps, c.sched, c.lanes, c.kmax, c.ipl);
    std::fclose(f);
}

static fw_status batch_reset(fw_batch* b) {
    Engine& e = b->eng;
    for (int s = 0; s < e.nslots(); ++s)
        if (e.slots[size_t(s)].used) FW_TRY(e.restart(s, e.stream));
    FW_CUDA(cudaMemcpyAsync(e.h_state, e.d_state, sizeof(ProbState) * e.slots.size(),
                            cudaMemcpyDeviceToHost, e.stream));
    FW_CUDA(cudaStreamSynchronize(e.stream));
    e.work_dirty = true;
    return FW_OK;
}

static fw_status apply_choice(fw_batch* b, const TuneChoice& c) {
    Engine& e = b->eng;
    FW_TRY(e.set_kernel_kmax(c.kmax));
    e.set_grid(c.bps, c.sched);
    FW_TRY(e.set_lanes(c.lanes));
    b->ipl = c.ipl;
    return FW_OK;
}

// Device time of `iters` iterations of the whole batch from U_0 in launches
// of `per` iterations (0: one launch), best of two runs.
static fw_status time_batch(fw_batch* b, int iters, int per, cudaEvent_t ev0, cudaEvent_t ev1,
                            float* best) {
    Engine& e = b->eng;
    *best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
        FW_TRY(batch_reset(b));
        FW_CUDA(cudaEventRecord(ev0, e.stream));
        int left = iters;
        while (left > 0) {
            const int it = per > 0 ? std::min(per, left) : left;
            int nlive = 0;
            FW_TRY(e.launch(it, &nlive));
            if (nlive == 0) break;
            FW_TRY(e.collect());
            left -= it;
        }
        FW_CUDA(cudaEventRecord(ev1, e.stream));
        FW_CUDA(cudaEventSynchronize(ev1));
        float ms = 0.f;
        FW_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
        *best = std::min(*best, ms);
    }
    return FW_OK;
}

// Autotune the persistent launch (see fw_batch_default_opts): one dimension
// after the other, each candidate timed on a few iterations of the batch
// itself; the problems are reset to U_0 afterwards.
static fw_status batch_tune(fw_batch* b) {
    Engine& e = b->eng;
    const fw_batch_opts& o = b->bo;
    const std::string sig = tune_signature(b);
    TuneChoice c;
    if (tune_lookup(b, sig, &c)) {
        FW_TRY(apply_choice(b, c));
        b->tuned = 2;
        return batch_reset(b);
    }
    const auto t0 = std::chrono::steady_clock::now();
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    FW_CUDA(cudaEventCreate(&ev0));
    FW_CUDA(cudaEventCreate(&ev1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } guard{ev0, ev1};
    const int keep_graph = e.use_graph;
    e.use_graph = FW_GRAPH_OFF;   // candidates change the launch; graphs come after
    c.kmax = e.kmax;
    c.lanes = std::max(0, o.lanes_per_row);
    c.ipl = std::max(0, o.iters_per_launch);
    c.sched = (o.schedule == FW_SCHED_STATIC || o.schedule == FW_SCHED_ITEMS) ? o.schedule
                                                                               : FW_SCHED_DYNAMIC;
    c.bps = o.blocks_per_sm > 0 ? std::min(o.blocks_per_sm, e.occ) : e.occ;
    const int it = 4;
    float best = 1e30f, ms = 0.f;
    auto consider = [&](const TuneChoice& t, int iters, int per) -> fw_status {
        FW_TRY(apply_choice(b, t));
        FW_TRY(time_batch(b, iters, per, ev0, ev1, &ms));
        if (ms < best) {
            best = ms;
            c = t;
        }
        return FW_OK;
    };
    // schedule: per-item launches, or the persistent kernel (static or
    // dynamic) at each blocks-per-SM count
    {
        std::vector<int> scheds;
        if (o.schedule == FW_SCHED_AUTO)
            scheds = {FW_SCHED_ITEMS, FW_SCHED_STATIC, FW_SCHED_DYNAMIC};
        else scheds = {c.sched};
        std::vector<int> grids;
        if (o.blocks_per_sm > 0) grids = {c.bps};
        else
            for (int x = 1; x <= e.occ; ++x) grids.push_back(x);
        const TuneChoice base = c;
        for (int sc : scheds)
            for (int x : grids) {
                if (sc == FW_SCHED_ITEMS && x != grids.back()) continue;   // one candidate
                TuneChoice t = base;
                t.sched = sc;
                t.bps = x;
                FW_TRY(consider(t, it, 0));
            }
    }
    // lanes per row
    if (o.lanes_per_row < 0) {
        const TuneChoice base = c;
        best = 1e30f;
        for (int L : {0, 1, 2, 4, 8}) {
            TuneChoice t = base;
            t.lanes = L;
            FW_TRY(consider(t, it, 0));
        }
    }
    // class bound of the compiled kernel: the smallest that holds K, or the next
    {
        const TuneChoice base = c;
        best = 1e30f;
        FW_TRY(consider(base, it, 0));
        const int nxt = kmax_for(base.kmax + 1);
        if (nxt > base.kmax) {
            TuneChoice t = base;
            t.kmax = nxt;
            t.bps = std::min(t.bps, e.occ);   // re-clamped to the new kernel's occupancy
            FW_TRY(consider(t, it, 0));
        }
    }
    // iterations per launch: 32 iterations as one launch, or launches of 16
    if (o.iters_per_launch < 0) {
        const TuneChoice base = c;
        best = 1e30f;
        for (int per : {0, 64, 16}) {
            TuneChoice t = base;
            t.ipl = per;
            FW_TRY(consider(t, 32, per));
        }
    }
    e.use_graph = keep_graph;
    FW_TRY(apply_choice(b, c));
    c.bps = e.bps;   // as clamped
    FW_TRY(batch_reset(b));
    tune_store(b, sig, c);
    b->tuned = 1;
    b->tune_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return FW_OK;
}

extern "C" {

fw_status fw_batch_default_opts(fw_batch_opts* o) {
    if (!o) return invalid("opts is NULL");
    std::memset(o, 0, sizeof(*o));
    o->weight_dtype = FW_WEIGHTS_F32;
    o->blocks_per_sm = 0;
    o->schedule = FW_SCHED_AUTO;
    o->iters_per_launch = -1;
    o->use_graph = FW_GRAPH_REQUIRED;
    o->spin_budget_ms = 2000;
    o->lanes_per_row = -1;
    return FW_OK;
}

fw_status fw_batch_create(fw_batch** out, int32_t P, const fw_graph* graphs,
                          const fw_seg_opts* opts, const fw_batch_opts* bopts) {
    try {
        if (!out) return invalid("out is NULL");
        *out = nullptr;
        if (P < 1 || !graphs || !opts) return invalid("P >= 1 graphs and options are required");
        if (bopts) {
            const int L = bopts->lanes_per_row;
            if (L < -1 || L > 32 || (L > 0 && (L & (L - 1)) != 0))
                return invalid("lanes_per_row must be -1, 0 or a power of two <= 32");
            if (bopts->iters_per_launch < -1) return invalid("iters_per_launch must be >= -1");
            if (bopts->use_graph < FW_GRAPH_OFF || bopts->use_graph > FW_GRAPH_PREFERRED)
                return invalid("bad use_graph");
            if (bopts->schedule < FW_SCHED_AUTO || bopts->schedule > FW_SCHED_ITEMS)
                return invalid("bad schedule");
        }
        std::unique_ptr<fw_batch> b(new fw_batch());
        if (bopts) b->bo = *bopts;
        else fw_batch_default_opts(&b->bo);
        b->P = P;
        std::vector<ProbLayout> lays(static_cast<size_t>(P));
        int Kmax = 2;
        size_t total = 0;
        for (int p = 0; p < P; ++p) {
            fw_seg_opts o = opts[p];
            o.weight_dtype = b->bo.weight_dtype;
            FW_TRY(check_opts(o));
            const fw_graph& g = graphs[p];
            const HostGraph hg{g.n, g.row_ptr_host, g.col_host, g.w_host, g.K, g.labels_host};
            FW_TRY(plan_problem(hg, o, lays[size_t(p)]));
            lays[size_t(p)].cls4 = g.K <= 16;   // gathered by the per-item schedule's pass B
            Kmax = std::max(Kmax, g.K);
            b->max_iters = std::max(b->max_iters, o.max_iters);
            const size_t te = b->bo.weight_dtype == FW_WEIGHTS_F64 ? 8 : 4;
            const size_t we = b->bo.weight_dtype == FW_WEIGHTS_F64   ? 8
                              : b->bo.weight_dtype == FW_WEIGHTS_BF16 ? 2
                                                                      : 4;
            total += problem_bytes(lays[size_t(p)], te, we, o.laplacian == FW_LAPLACIAN_COMB) + 256;
        }
        Engine& e = b->eng;
        e.use_graph = b->bo.use_graph;
        e.expect_extra = b->bo.test_barrier_extra;
        FW_TRY(e.init(b->bo.weight_dtype, Kmax, total, P, b->bo.cuda_stream,
                      b->bo.spin_budget_ms > 0 ? b->bo.spin_budget_ms : 2000, b->bo.blocks_per_sm,
                      b->bo.schedule));
        for (int p = 0; p < P; ++p) {
            fw_seg_opts o = opts[p];
            o.weight_dtype = b->bo.weight_dtype;
            const fw_graph& g = graphs[p];
            const HostGraph hg{g.n, g.row_ptr_host, g.col_host, g.w_host, g.K, g.labels_host};
            int slot = -1;
            FW_TRY(e.add(hg, o, lays[size_t(p)], &slot));
        }
        b->ipl = std::max(0, b->bo.iters_per_launch);
        if (b->bo.blocks_per_sm <= 0 || b->bo.schedule == FW_SCHED_AUTO ||
            b->bo.lanes_per_row < 0 || b->bo.iters_per_launch < 0)
            FW_TRY(batch_tune(b.get()));
        else if (b->bo.lanes_per_row > 0)
            FW_TRY(e.set_lanes(b->bo.lanes_per_row));
        *out = b.release();
        return FW_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

fw_status fw_batch_solve(fw_batch* b, fw_seg_stats* stats) {
    if (!b) return invalid("batch is NULL");
    Engine& e = b->eng;
    const int per = b->ipl > 0 ? b->ipl : b->max_iters + 1;
    cudaEvent_t ev0, ev1;
    FW_CUDA(cudaEventCreate(&ev0));
    FW_CUDA(cudaEventCreate(&ev1));
    cudaEventRecord(ev0, e.stream);
    b->launches = 0;
    fw_status rc = FW_OK;
    for (int guard = 0; guard < 1 << 20; ++guard) {
        int nlive = 0;
        rc = e.launch(per, &nlive);
        if (rc != FW_OK || nlive == 0) break;
        ++b->launches;
        rc = e.collect();
        if (rc != FW_OK) break;
    }
    cudaEventRecord(ev1, e.stream);
    cudaEventSynchronize(ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (rc != FW_OK) return rc;
    fw_status worst = FW_OK;
    for (int p = 0; p < b->P; ++p) {
        const ProbState& st = e.h_state[p];
        if (stats) fill_stats_from(st, stats + p, b->launches, ms);
        if (st.status == FW_ERR_NUMERIC) worst = FW_ERR_NUMERIC;
        else if (st.status == FW_NOT_CONVERGED && worst == FW_OK) worst = FW_NOT_CONVERGED;
    }
    if (worst == FW_ERR_NUMERIC) set_error("non-finite FW gap or curvature in a problem");
    return worst;
}

fw_status fw_batch_reset(fw_batch* b) {
    if (!b) return invalid("batch is NULL");
    return batch_reset(b);
}

fw_status fw_batch_labels(fw_batch* b, int32_t p, int32_t* labels_host) {
    if (!b || p < 0 || p >= b->P || !labels_host) return invalid("bad arguments");
    return b->eng.labels(p, labels_host, b->eng.stream);
}

fw_status fw_batch_get_U(fw_batch* b, int32_t p, double* U_host) {
    if (!b || p < 0 || p >= b->P || !U_host) return invalid("bad arguments");
    try {
        return b->eng.get_U(p, U_host);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

fw_status fw_batch_get_info(fw_batch* b, fw_batch_info* info) {
    if (!b || !info) return invalid("bad arguments");
    info->grid = b->eng.grid;
    info->blocks_per_sm = b->eng.bps;
    info->schedule = b->eng.schedule;
    info->graph_captured = b->eng.graph_captured;
    info->tuned = b->tuned;
    info->kmax = b->eng.kmax_kern;
    info->lanes_per_row = b->eng.lanes_all;
    info->iters_per_launch = b->ipl;
    info->graph_error = b->eng.graph_error;
    info->reserved = 0;
    info->tune_ms = b->tune_ms;
    info->pool_bytes = b->eng.ra.cap();
    return FW_OK;
}

void fw_batch_destroy(fw_batch* b) { delete b; }

}  // extern "C"

// ================================================================= serving

namespace {

// A host array left uninitialised until filled (no zero-fill pass over
// pages that the copy writes anyway).
template <typename V>
struct HostBuf {
    std::unique_ptr<V[]> p;
    V* data() { return p.get(); }
};

struct Request {
    uint64_t ticket = 0;
    int64_t n = 0;
    int32_t K = 0;
    HostBuf<int32_t> rp, col, labels;
    HostBuf<double> w;
    fw_seg_opts opts{};
    ProbLayout lay;
    size_t bytes = 0;
};

struct Result {
    fw_status status = FW_PENDING;
    std::vector<int32_t> labels;
    fw_seg_stats stats{};
    bool done = false;
};

}  // namespace

// memcpy split over up to 8 host threads for large arrays (a 1024^2 image's
// request is about 110 MB; one thread copies it in about 9 ms on Grace).
// Parts whose thread cannot be started are copied by the calling thread.
static void copy_parallel(void* dst, const void* src, size_t bytes) {
    constexpr size_t kChunk = size_t(8) << 20;
    const size_t hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nt = std::min<size_t>({8, hw, bytes / kChunk});
    auto part = [&](size_t t) {
        const size_t a = bytes * t / nt, b = bytes * (t + 1) / nt;
        std::memcpy(static_cast<char*>(dst) + a, static_cast<const char*>(src) + a, b - a);
    };
    if (nt < 2) {
        if (bytes) std::memcpy(dst, src, bytes);
        return;
    }
    std::vector<std::thread> th;
    size_t t = 1;
    try {
        for (; t < nt; ++t) th.emplace_back(part, t);
    } catch (const std::system_error&) {
    }
    for (size_t u = t; u < nt; ++u) part(u);
    part(0);
    for (auto& x : th) x.join();
}

template <typename V>
static void assign_parallel(HostBuf<V>& v, const V* src, size_t n) {
    v.p.reset(new V[n > 0 ? n : 1]);
    copy_parallel(v.data(), src, n * sizeof(V));
}

// A resident request with at least this many rows (about 512 row tiles of 256,
// enough to fill a GB300 by itself) runs alone when it is the oldest.
constexpr int64_t kAloneRows = int64_t(1) << 17;

struct fw_srv {
    Engine eng;
    fw_srv_opts so{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::unique_ptr<Request>> queue;
    std::unordered_map<uint64_t, Result> results;
    std::deque<uint64_t> finished;   // tickets in completion order, for fw_srv_wait_any
    std::vector<uint64_t> slot_ticket;
    std::vector<int> slot_epochs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    fw_srv_info info{};

    void loop();
    void harvest();
};

void fw_srv::harvest() {
    Engine& e = eng;
    for (int s = 0; s < e.nslots(); ++s) {
        if (!e.slots[size_t(s)].used) continue;
        const ProbState& st = e.h_state[s];
        if (!st.done) continue;
        Result r;
        r.done = true;
        r.status = fw_status(st.status);
        r.labels.resize(size_t(e.slots[size_t(s)].lay.n));
        fw_status rc = e.labels(s, r.labels.data(), e.stream);
        if (rc != FW_OK) r.status = rc;
        fill_stats_from(st, &r.stats, slot_epochs[size_t(s)], 0.0);
        const uint64_t t = slot_ticket[size_t(s)];
        e.remove(s);
        std::lock_guard<std::mutex> lk(mu);
        info.completed++;
        if (r.status < 0) info.failed++;
        info.resident--;
        results[t] = std::move(r);
        finished.push_back(t);
    }
    cv_done.notify_all();
}

void fw_srv::loop() {
    cudaSetDevice(device);
    Engine& e = eng;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (info.resident == 0)
                cv_work.wait(lk, [&] { return stop || !queue.empty(); });
            if (stop) return;
        }
        // start the epoch over the resident requests (four times longer while
        // no request waits for admission: a problem that stops early in it
        // skips the rest at once, so a long epoch only delays admissions) ...
        bool waiting = false;
        {
            std::lock_guard<std::mutex> lk(mu);
            waiting = !queue.empty();
        }
        int nlive = 0;
        const int iters = so.iters_per_epoch * (waiting ? 1 : 4);
        // a lone resident, or the oldest resident when it is large enough to
        // fill the GPU by itself, runs alone on the single-problem kernels
        // (first in, first out); otherwise one batched epoch iterates the
        // small residents (the large ones wait for their turn as the oldest:
        // in a shared epoch every iteration would cost the small ones the
        // large one's time), and a single small one runs alone too
        int lone = e.lone_live();
        if (lone < 0) {
            uint64_t first = UINT64_MAX;
            int oldest = -1, small = -1, nsmall = 0;
            for (int q = 0; q < e.nslots(); ++q) {
                if (!e.slots[size_t(q)].used || e.h_state[q].done) continue;
                if (slot_ticket[size_t(q)] < first) {
                    first = slot_ticket[size_t(q)];
                    oldest = q;
                }
                if (e.slots[size_t(q)].lay.n < kAloneRows) {
                    small = q;
                    ++nsmall;
                }
            }
            if (oldest >= 0 && e.slots[size_t(oldest)].lay.n >= kAloneRows) lone = oldest;
            else if (nsmall == 1) lone = small;
        }
        bool piped = false;
        fw_status rc = lone >= 0 ? e.lone_queue(lone, iters, &piped) : FW_OK;
        if (rc == FW_OK && piped) nlive = 1;
        else if (rc == FW_OK) rc = e.launch_epoch(iters, &nlive);
        // ... and admit queued requests (FIFO) while it runs: upload and
        // assembly go to the side stream, the pool range is taken in order
        for (;;) {
            std::unique_ptr<Request> rq;
            {
                std::lock_guard<std::mutex> lk(mu);
                if (queue.empty() || e.free_slot() < 0 || !e.fits(queue.front()->bytes)) break;
                rq = std::move(queue.front());
                queue.pop_front();
                info.queued = int32_t(queue.size());
            }
            const HostGraph hg{rq->n, rq->rp.data(), rq->col.data(), rq->w.data(), rq->K,
                               rq->labels.data()};
            int slot = -1;
            const fw_status ra = e.add(hg, rq->opts, rq->lay, &slot);
            std::lock_guard<std::mutex> lk(mu);
            if (ra != FW_OK) {
                Result r;
                r.done = true;
                r.status = ra;
                results[rq->ticket] = std::move(r);
                finished.push_back(rq->ticket);
                info.failed++;
                info.completed++;
                cv_done.notify_all();
            } else {
                slot_ticket[size_t(slot)] = rq->ticket;
                slot_epochs[size_t(slot)] = 0;
                info.admitted++;
                info.resident++;
            }
        }
        if (rc == FW_OK && nlive > 0) {
            rc = piped ? e.lone_collect() : e.collect();
            std::lock_guard<std::mutex> lk(mu);
            info.epochs++;
            for (int s = 0; s < e.nslots(); ++s)
                if (e.slots[size_t(s)].used) slot_epochs[size_t(s)]++;
        }
        if (rc != FW_OK) {
            // a failed epoch fails every resident request
            std::lock_guard<std::mutex> lk(mu);
            for (int s = 0; s < e.nslots(); ++s) {
                if (!e.slots[size_t(s)].used) continue;
                Result r;
                r.done = true;
                r.status = rc;
                results[slot_ticket[size_t(s)]] = std::move(r);
                finished.push_back(slot_ticket[size_t(s)]);
                e.remove(s);
                info.failed++;
                info.completed++;
                info.resident--;
            }
            cv_done.notify_all();
            continue;
        }
        harvest();
    }
}

extern "C" {

fw_status fw_srv_default_opts(fw_srv_opts* o) {
    if (!o) return invalid("opts is NULL");
    std::memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = size_t(8) << 30;
    o->max_slots = 64;
    o->max_K = 8;
    o->weight_dtype = FW_WEIGHTS_F32;
    o->iters_per_epoch = 16;
    o->blocks_per_sm = 0;
    o->schedule = FW_SCHED_ITEMS;
    o->spin_budget_ms = 2000;
    return FW_OK;
}

fw_status fw_srv_create(fw_srv** out, const fw_srv_opts* opts) {
    try {
        if (!out) return invalid("out is NULL");
        *out = nullptr;
        std::unique_ptr<fw_srv> s(new fw_srv());
        if (opts) s->so = *opts;
        else fw_srv_default_opts(&s->so);
        const fw_srv_opts& o = s->so;
        if (o.max_slots < 1 || o.max_K < 2 || o.max_K > 32 || o.iters_per_epoch < 1 ||
            o.hbm_budget_bytes < 4096 || o.schedule < FW_SCHED_AUTO || o.schedule > FW_SCHED_ITEMS)
            return invalid("bad serving options");
        FW_CUDA(cudaGetDevice(&s->device));
        s->eng.use_graph = FW_GRAPH_PREFERRED;
        s->eng.plain_path = true;
        s->eng.shared_max_rows = kAloneRows;   // large requests run alone, in arrival order
        FW_TRY(s->eng.init(o.weight_dtype, o.max_K, o.hbm_budget_bytes, o.max_slots, o.cuda_stream,
                           o.spin_budget_ms > 0 ? o.spin_budget_ms : 2000, o.blocks_per_sm,
                           (o.schedule == FW_SCHED_STATIC || o.schedule == FW_SCHED_DYNAMIC)
                               ? o.schedule
                               : FW_SCHED_ITEMS));
        s->slot_ticket.assign(size_t(o.max_slots), 0);
        s->slot_epochs.assign(size_t(o.max_slots), 0);
        s->info.pool_bytes = s->eng.ra.cap();
        fw_srv* raw = s.get();
        s->worker = std::thread([raw] { raw->loop(); });
        *out = s.release();
        return FW_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    } catch (const std::system_error&) {
        set_error("could not start the serving thread");
        return FW_ERR_INVALID_ARG;
    }
}

fw_status fw_srv_submit(fw_srv* s, const fw_graph* g, const fw_seg_opts* opts, uint64_t* ticket) {
    if (!s || !g || !ticket) return invalid("bad arguments");
    try {
        fw_seg_opts o;
        if (opts) o = *opts;
        else fw_seg_default_opts(&o);
        o.weight_dtype = s->so.weight_dtype;
        FW_TRY(check_opts(o));
        if (g->K > s->so.max_K) {
            set_error("K above the server's max_K");
            std::lock_guard<std::mutex> lk(s->mu);
            s->info.rejected++;
            return FW_ERR_UNSUPPORTED;
        }
        std::unique_ptr<Request> rq(new Request());
        const HostGraph hg{g->n, g->row_ptr_host, g->col_host, g->w_host, g->K, g->labels_host};
        FW_TRY(plan_problem(hg, o, rq->lay));
        rq->lay.cls4 = g->K <= 16;   // for the single-problem kernels of a lone request
        rq->bytes = s->eng.bytes_for(rq->lay, o);
        if (rq->bytes + 256 > s->eng.ra.cap()) {
            set_error("request can never fit the server's device pool");
            std::lock_guard<std::mutex> lk(s->mu);
            s->info.rejected++;
            return FW_ERR_NO_MEMORY;
        }
        rq->n = g->n;
        rq->K = g->K;
        rq->opts = o;
        const int64_t nnz = g->row_ptr_host[g->n];
        assign_parallel(rq->rp, g->row_ptr_host, size_t(g->n) + 1);
        assign_parallel(rq->col, g->col_host, size_t(nnz));
        assign_parallel(rq->w, g->w_host, size_t(nnz));
        assign_parallel(rq->labels, g->labels_host, size_t(g->n));
        std::lock_guard<std::mutex> lk(s->mu);
        rq->ticket = s->next_ticket++;
        *ticket = rq->ticket;
        s->results[rq->ticket] = Result();
        s->queue.push_back(std::move(rq));
        s->info.submitted++;
        s->info.queued = int32_t(s->queue.size());
        s->cv_work.notify_one();
        return FW_PENDING;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FW_ERR_NO_MEMORY;
    }
}

static fw_status take_result(fw_srv* s, uint64_t ticket, int32_t* labels, fw_seg_stats* stats,
                             std::unique_lock<std::mutex>& lk, bool* found) {
    (void)lk;
    auto it = s->results.find(ticket);
    *found = it != s->results.end();
    if (!*found) return invalid("unknown ticket");
    if (!it->second.done) return FW_PENDING;
    Result r = std::move(it->second);
    s->results.erase(it);
    if (labels && !r.labels.empty()) std::memcpy(labels, r.labels.data(), 4 * r.labels.size());
    if (stats) *stats = r.stats;
    if (r.status < 0) set_error("request failed");
    return r.status;
}

fw_status fw_srv_poll(fw_srv* s, uint64_t ticket, int32_t* labels_host, fw_seg_stats* stats) {
    if (!s) return invalid("server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    bool found = false;
    return take_result(s, ticket, labels_host, stats, lk, &found);
}

fw_status fw_srv_wait(fw_srv* s, uint64_t ticket, int32_t timeout_ms, int32_t* labels_host,
                      fw_seg_stats* stats) {
    if (!s) return invalid("server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        auto it = s->results.find(ticket);
        return it == s->results.end() || it->second.done;
    };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    bool found = false;
    return take_result(s, ticket, labels_host, stats, lk, &found);
}

fw_status fw_srv_wait_any(fw_srv* s, int32_t timeout_ms, uint64_t* ticket) {
    if (!s || !ticket) return invalid("bad arguments");
    std::unique_lock<std::mutex> lk(s->mu);
    // tickets already taken by poll / wait are skipped
    auto ready = [&] {
        while (!s->finished.empty() && !s->results.count(s->finished.front()))
            s->finished.pop_front();
        return !s->finished.empty();
    };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    if (!ready()) return FW_PENDING;
    *ticket = s->finished.front();
    s->finished.pop_front();
    return FW_OK;
}

fw_status fw_srv_get_info(fw_srv* s, fw_srv_info* info) {
    if (!s || !info) return invalid("bad arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    *info = s->info;
    info->pool_used = s->eng.ra.used();
    info->pool_bytes = s->eng.ra.cap();
    return FW_OK;
}

void fw_srv_destroy(fw_srv* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
}

}  // extern "C"
