// Persistent batched kernel: many independent problems iterate together in
// one cooperative launch.  Each launch runs `iters` GFW iterations; one
// iteration is phase A (row tiles of every live problem), a grid barrier,
// phase B (same tiles), a grid barrier.  A block takes (problem, tile) work
// items in a static grid stride or from an atomic counter (dynamic schedule).
// Per-problem reductions go through the same tile partials and last-block
// rule as the single-problem kernels, so a problem's arithmetic does not
// depend on the batch it runs in.
#pragma once
#include "fw_kernels.cuh"

namespace fw {

struct GridBar {
    uint32_t count;   // arrivals at the current barrier
    uint32_t gen;     // barrier generation
    uint32_t ndone;   // problems that stopped during this launch
    int32_t error;    // 1: a barrier wait ran out of its clock budget
    int32_t exit;     // 1: every live problem stopped (set by the last arrival)
    uint32_t ctr[2];  // dynamic-schedule work counters (phase A, phase B)
    uint32_t pad_;
};

struct BatchArgs {
    const ProbDesc* desc;   // [P]
    ProbState* state;       // [P]
    const int2* work;       // [nwork] (problem, tile), tiles of live problems
    int32_t nwork;
    int32_t nlive;          // problems not done when the launch starts
    int32_t iters;          // iterations in this launch
    int32_t dynamic;        // 1: atomic work counter, 0: static grid stride
    int32_t expect_extra;   // test hook: barrier waits for this many extra blocks
    int32_t pad_;
    GridBar* bar;
    long long budget;       // clock cycles one barrier wait may take
};

__device__ __forceinline__ uint32_t ld_vol(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

// Grid-wide barrier with a bounded wait.  Returns 0 to continue, 1 when the
// last arrival saw every live problem done, -1 when the wait ran out (the
// error flag is then set and the caller returns).
__device__ __forceinline__ int grid_sync(GridBar* bar, long long budget, int nlive, int extra) {
    __shared__ int s_r;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t g = ld_vol(&bar->gen);
        __threadfence();
        const uint32_t arrived = atomicAdd(&bar->count, 1u) + 1u;
        int r = 0;
        if (arrived == gridDim.x + uint32_t(extra)) {
            atomicExch(&bar->count, 0u);
            atomicExch(&bar->exit, ld_vol(&bar->ndone) >= uint32_t(nlive) ? 1 : 0);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (ld_vol(&bar->gen) == g) {
                if (clock64() - t0 > budget) {
                    atomicExch(&bar->error, 1);
                    r = -1;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (r == 0) r = *reinterpret_cast<const volatile int32_t*>(&bar->exit);
        s_r = r;
    }
    __syncthreads();
    return s_r;
}

// Held to 48 registers for the FP32 iterate so that 5 blocks per SM stay
// resident; pass A stages one 256-row sub-tile at a time (a batch item is
// usually a single sub-tile, so a second buffer would only cost residency).
template <typename T, typename WT, int KMAX>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 5 : 2) k_persistent(BatchArgs a) {
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm_lane = reinterpret_cast<T*>(smraw);
    T* sm_row = sm_lane + kBlock * (KMAX | 1);
    T* stage = reinterpret_cast<T*>(smraw);        // phases A and B use the buffer in turn
    // two item slots: warp 1 fetches the next (problem, tile) item, its
    // descriptor and its scalars while the block works on the current one
    __shared__ ProbDesc s_pd[2];
    __shared__ int s_w[2], s_skip[2], s_upd[2];
    __shared__ T s_alpha[2];
    __shared__ __align__(8) uint64_t bars[2];
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
    }
    __syncthreads();
    uint32_t mb_phases = 0;   // parities of the two bulk-copy mbarriers
    for (int it = 0; it < a.iters; ++it) {
        for (int phase = 0; phase < 2; ++phase) {
            // one thread fills slot `sl` with the item after `w` in this block's order
            auto fetch = [&](int sl, int w) {
                const int ww = a.dynamic ? int(atomicAdd(&a.bar->ctr[phase], 1u)) : w;
                s_w[sl] = ww;
                if (ww < a.nwork) {
                    const int2 wk = a.work[ww];
                    s_pd[sl] = a.desc[wk.x];
                    const ProbState* st = a.state + wk.x;
                    s_skip[sl] = ld_cg(&st->done);
                    s_upd[sl] = ld_cg(&st->has_update);
                    s_alpha[sl] = alpha_of<T>(st);
                }
            };
            int w = blockIdx.x;
            int c = 0;
            if (threadIdx.x == 32) fetch(0, w);
            __syncthreads();
            for (;;) {
                const int ww = s_w[c];
                if (ww >= a.nwork) break;
                if (threadIdx.x == 32) fetch(c ^ 1, w + int(gridDim.x));
                if (!s_skip[c]) {
                    const int2 wk = a.work[ww];
                    ProbState* st = a.state + wk.x;
                    if (phase == 0)
                        tile_A<T, KMAX>(s_pd[c], st, wk.y, s_upd[c] != 0, s_alpha[c],
                                        FuseCtl{false, nullptr, nullptr}, s_pd[c].acc, stage, 1,
                                        bars, mb_phases);
                    else
                        tile_B<T, WT, KMAX, false, true>(s_pd[c], st, wk.y, sm_lane, sm_row,
                                                         sm_row + kBlock * (KMAX | 1),
                                                         s_pd[c].acc, &a.bar->ndone);
                }
                __syncthreads();   // the prefetched slot is complete, the current one free
                c ^= 1;
                w += gridDim.x;
            }
            const int r = grid_sync(a.bar, a.budget, a.nlive, a.expect_extra);
            if (r < 0) return;
            // the counter of this phase is idle until after the next barrier
            if (a.dynamic && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&a.bar->ctr[phase], 0u);
            if (phase == 1 && r == 1) return;
        }
    }
}

// ---------------------------------------------------- per-item schedule
// The alternative to the persistent kernel: per iteration one launch of the
// single-problem pass A over every (problem, tile) item of the live
// problems, one launch of pass B, and after the last iteration one warp per
// live problem to finish, all captured in a CUDA graph; the kernel
// boundaries are the grid-wide barriers.  Each block copies its item's
// descriptor into shared memory and runs the single-problem per-tile code,
// so every problem's arithmetic is that of solving it alone (with the same
// lanes per row), and tens of thousands of item blocks keep the SMs busy.
struct ItemArgs {
    const ProbDesc* desc;   // [slots]
    ProbState* state;       // [slots]
    const int2* work;       // [nwork] (problem, tile) of the live problems
    const int* live;        // [nlive] live problems
};

// Warp 0 copies the item's descriptor (8-byte words) into shared memory.
__device__ __forceinline__ int2 item_desc(const ItemArgs& a, ProbDesc* s_pd) {
    static_assert(sizeof(ProbDesc) % 8 == 0 && sizeof(ProbDesc) / 8 <= 32, "descriptor words");
    const int2 wk = a.work[blockIdx.x];
    if (threadIdx.x < sizeof(ProbDesc) / 8)
        reinterpret_cast<unsigned long long*>(s_pd)[threadIdx.x] =
            reinterpret_cast<const unsigned long long*>(a.desc + wk.x)[threadIdx.x];
    __syncthreads();
    return wk;
}

template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock, passA_min_blocks<T, KMAX>()) k_itemA(ItemArgs a, int fin) {
    __shared__ __align__(16) ProbDesc s_pd;
    const int2 wk = item_desc(a, &s_pd);
    extern __shared__ __align__(128) unsigned char smraw[];
    passA_step<T, KMAX, false>(s_pd, a.state + wk.x, fin, reinterpret_cast<T*>(smraw), wk.y);
}

// Item pass B blocks per SM the registers are held to: 6 (40 registers) for
// an FP32 iterate with at most 12 classes, which measured 6% faster than
// 4 blocks at 64 registers on the 256-problem batch (8 blocks spilled and
// lost); wider class bounds keep their registers.
template <typename T, int KMAX>
constexpr int itemB_min_blocks() {
    return (sizeof(T) == 4 && KMAX <= 12) ? 6 : 1;
}

template <typename T, typename WT, int KMAX>
__global__ void __launch_bounds__(kBlock, itemB_min_blocks<T, KMAX>()) k_itemB(ItemArgs a) {
    __shared__ __align__(16) ProbDesc s_pd;
    const int2 wk = item_desc(a, &s_pd);
    ProbState* st = a.state + wk.x;
    bool done;
    unsigned long long* accb = passB_bank(s_pd, st, done, wk.y);
    if (done) return;
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm_lane = reinterpret_cast<T*>(smraw);
    T* sm_row = sm_lane + kBlock * (KMAX | 1);
    tile_B<T, WT, KMAX, true, false>(s_pd, st, wk.y, sm_lane, sm_row,
                                     sm_row + kBlock * (KMAX | 1), accb, nullptr);
}

// One warp per live problem: the step decision of the last iteration.
static __global__ void k_itemFinish(ItemArgs a) {
    const int p = a.live[blockIdx.x];
    ProbState* st = a.state + p;
    if (ld_cg(&st->done)) return;
    const ProbDesc& pd = a.desc[p];
    warp_finish(pd, st, pd.acc + ld_cg(&st->cur) * kAccBank);
}

// Launcher of the persistent kernel (and of the per-item schedule) for one
// (T, WT, KMAX).
class BatchKern {
public:
    virtual ~BatchKern() {}
    virtual size_t smem() const = 0;
    virtual cudaError_t configure() = 0;
    virtual cudaError_t occupancy(int* blocks_per_sm) = 0;
    virtual cudaError_t launch(const BatchArgs& a, int grid, cudaStream_t s) = 0;
    // `iters` iterations of the per-item schedule; two_stage: some live
    // problem has tiles of more than one 256-row sub-tile
    virtual cudaError_t launch_items(const ItemArgs& a, int nwork, int nlive, int iters,
                                     bool two_stage, cudaStream_t s) = 0;
};

template <typename T, typename WT, int KMAX>
class BatchKernImpl final : public BatchKern {
public:
    size_t smem() const override {
        const size_t b = 2 * size_t(kBlock) * (KMAX | 1) * sizeof(T) +
                         passB_prefetch_bytes<T, KMAX>();
        const size_t a = 3 * size_t(kBlock) * KMAX * sizeof(T);   // one staging buffer
        const size_t r = size_t(kBlock) * kNumR * sizeof(double);
        const size_t m = a > b ? a : b;
        return m > r ? m : r;
    }
    static size_t smem_itemA(bool two_stage) {
        return (two_stage ? max_stages<T, KMAX>() : 1) * 3 * size_t(kBlock) * KMAX * sizeof(T);
    }
    static size_t smem_itemB() {
        return 2 * size_t(kBlock) * (KMAX | 1) * sizeof(T);
    }
    cudaError_t configure() override {
        cudaError_t e = cudaFuncSetAttribute(k_persistent<T, WT, KMAX>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem()));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_itemA<T, KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem_itemA(true)));
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_itemB<T, WT, KMAX>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(smem_itemB()));
    }
    cudaError_t launch_items(const ItemArgs& a, int nwork, int nlive, int iters, bool two_stage,
                             cudaStream_t s) override {
        for (int i = 0; i < iters; ++i) {
            k_itemA<T, KMAX><<<nwork, kBlock, smem_itemA(two_stage), s>>>(a, i > 0 ? 1 : 0);
            k_itemB<T, WT, KMAX><<<nwork, kBlock, smem_itemB(), s>>>(a);
        }
        k_itemFinish<<<nlive, 32, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaError_t occupancy(int* bps) override {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_persistent<T, WT, KMAX>, kBlock,
                                                             smem());
    }
    // Cooperative launch (all blocks co-resident, which the grid barrier
    // needs) through the extensible launch API, which stream capture records
    // as a cooperative kernel node.
    cudaError_t launch(const BatchArgs& a, int grid, cudaStream_t s) override {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(grid));
        cfg.blockDim = dim3(kBlock);
        cfg.dynamicSmemBytes = smem();
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_persistent<T, WT, KMAX>, a);
    }
};

template <typename T, typename WT>
BatchKern* make_batch_kern_t(int kmax) {
    switch (kmax) {
        case 4: return new BatchKernImpl<T, WT, 4>();
        case 8: return new BatchKernImpl<T, WT, 8>();
        case 10: return new BatchKernImpl<T, WT, 10>();
        case 12: return new BatchKernImpl<T, WT, 12>();
        case 16: return new BatchKernImpl<T, WT, 16>();
        case 32: return new BatchKernImpl<T, WT, 32>();
        default: return nullptr;
    }
}

BatchKern* make_batch_kern(int weight_dtype, int kmax);

}  // namespace fw
