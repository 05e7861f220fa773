// Problem set-up shared by the single-problem handle and the batch engine:
// option and CSR checks, device layout, upload, validation, Laplacian
// assembly (Sec. 1), U_0 = U_hat (Sec. 5.1), L U_0 and the initial state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <mutex>
#include <system_error>
#include <thread>
#include <vector>

#include "fw_device.cuh"
#include "fw_internal.h"

namespace fw {

// ------------------------------------------------------------- kernels
// Validation and degrees of the input CSR (one thread per row):
//   columns strictly increasing and in range, no self loop, w finite and >= 0,
//   w_ij == w_ji (binary search in row j), d_i = sum_j w_ij > 0 (Sec. 1).
// err bits: 1 graph structure / weights, 2 asymmetric, 4 isolated node,
// 8 (not an error) some |j - i| >= 2^15, so 16-bit column offsets cannot hold it.
__global__ void k_validate(int64_t n, const int32_t* rp, const int32_t* col, const double* w,
                           double* deg, int* err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e0 = rp[i], e1 = rp[i + 1];
    double d = 0.0;
    int bad = 0, far = 0;
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
        far |= (j - int(i) > 32767) | (int(i) - j > 32767);
        int lo = rp[j], hi = rp[j + 1] - 1, pos = -1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const int cm = col[mid];
            if (cm == i) {
                pos = mid;
                break;
            }
            if (cm < i) lo = mid + 1;
            else hi = mid - 1;
        }
        if (pos < 0 || w[pos] != x) bad |= 2;
    }
    if (!bad && !(d > 0.0)) bad |= 4;
    deg[i] = d;
    if (bad | far) atomicOr(err, bad | (far ? 8 : 0));
}

__global__ void __launch_bounds__(kBlock) k_state_init(ProbState* st, const double* part, int nb) {
    __shared__ double red[kBlock];
    double S[1];
    sum_partials<1>(part, nb, S, red);   // nb may exceed kBlock: loops
    if (threadIdx.x == 0) {
        ProbState z = {};
        z.status = 2;  // FW_PENDING
        z.E = S[0];
        z.in[0].E = S[0];   // cur = 0: the first decision reads in[0]
        *st = z;
    }
}

// Padded row offsets (every row rounded up to kPadW entries), an exclusive
// scan over the rows in three steps: per 1024-row block, over the block
// totals (one block), then the block offsets added back.  Integer, so exact.
constexpr int kScanRows = 4 * kBlock;

__global__ void __launch_bounds__(kBlock)
k_pad_scan_local(int64_t n, const int32_t* __restrict__ rp, int32_t* __restrict__ out,
                 int32_t* __restrict__ bsum) {
    __shared__ int32_t wsum[kBlock / 32];
    const int64_t base = blockIdx.x * int64_t(kScanRows) + threadIdx.x * 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t v[4];
    int32_t s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = base + q;
        const int32_t d = i < n ? rp[i + 1] - rp[i] : 0;
        v[q] = (d + (kPadW - 1)) & ~(kPadW - 1);
        s += v[q];
    }
    int32_t x = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int w = 0; w < kBlock / 32; ++w) {
            const int32_t t = wsum[w];
            wsum[w] = run;
            run += t;
        }
        bsum[blockIdx.x] = run;
    }
    __syncthreads();
    int32_t excl = x - s + wsum[warp];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = base + q;
        if (i < n) out[i] = excl;
        excl += v[q];
    }
}

// Exclusive scan of the nb block totals in place (one block); total -> out[n].
__global__ void __launch_bounds__(kBlock)
k_pad_scan_blocks(int64_t n, int nb, int32_t* __restrict__ bsum, int32_t* __restrict__ out) {
    __shared__ int32_t wsum[kBlock / 32];
    __shared__ int32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += kBlock) {
        const int b = b0 + threadIdx.x;
        const int32_t s = b < nb ? bsum[b] : 0;
        int32_t x = s;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t run = 0;
            for (int w = 0; w < kBlock / 32; ++w) {
                const int32_t t = wsum[w];
                wsum[w] = run;
                run += t;
            }
        }
        __syncthreads();
        const int32_t c = carry;
        if (b < nb) bsum[b] = c + x - s + wsum[warp];
        __syncthreads();
        if (threadIdx.x == kBlock - 1) carry = c + x + wsum[warp];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_pad_scan_add(int64_t n, const int32_t* __restrict__ bsum, int32_t* out) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i < n) out[i] += bsum[i / kScanRows];
}

// d_i <- 1 / sqrt(d_i) in place (FP64), so that k_build forms
// W_hat_ij = w_ij d_i^{-1/2} d_j^{-1/2} with two products per entry.
__global__ void k_inv_sqrt(int64_t n, double* deg) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) deg[i] = 1.0 / sqrt(deg[i]);
}

__global__ void k_fid(int64_t n, const int32_t* labels, int8_t* fid) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) fid[i] = int8_t(labels[i]);
}

// ------------------------------------------------------------- errors
static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_text() { return g_last_error.c_str(); }

fw_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return FW_ERR_CUDA;
}

static fw_status invalid(const std::string& m) {
    set_error(m);
    return FW_ERR_INVALID_ARG;
}

// ------------------------------------------------------------- choices
int kmax_for(int K) {
    return K <= 4 ? 4 : K <= 8 ? 8 : K <= 10 ? 10 : K <= 12 ? 12 : K <= 16 ? 16 : 32;
}

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
    const int64_t sub = (n + kBlock - 1) / kBlock;               // 256-row sub-tiles
    const int64_t per = (sub + kTilesTarget - 1) / kTilesTarget;  // sub-tiles per tile
    return int(std::max<int64_t>(per, 1) * kBlock);
}


// Lanes per CSR row in pass B from the mean padded row length.  Measured on a
// GB300 (whole solves of stochastic block models with K = 4, 10, 16 and mean
// degree 12 to 30): one lane wins up to about 20 padded entries (by up to 15%
// at 13); from 20 to 32 entries two lanes stay within 2.2% of the best, while
// one lane falls up to 20% behind at 32; four lanes pay off only for longer
// rows.  The persistent kernels use the same count (so batched and single
// solves agree bit for bit); on batches of k-NN graphs with 13 to 18 padded
// entries one and two lanes measured the same there, four lanes 8% slower.
int default_lanes(double avg_padded_degree) {
    int L = 1;
    while (L < 32 && avg_padded_degree > 20.0 * L) L *= 2;
    return L;
}

fw_status check_opts(const fw_seg_opts& o) {
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
    if (o.index_width != 0 && o.index_width != 32) return invalid("index_width must be 0 or 32");
    if (o.class_table < FW_TABLE_AUTO || o.class_table > FW_TABLE_ON)
        return invalid("class_table must be FW_TABLE_AUTO, FW_TABLE_OFF or FW_TABLE_ON");
    const int L = o.lanes_per_row;
    if (L != 0 && (L < 1 || L > 32 || (L & (L - 1)) != 0))
        return invalid("lanes_per_row must be 0 or a power of two <= 32");
    return FW_OK;
}

fw_status plan_problem(const HostGraph& g, const fw_seg_opts& o, ProbLayout& lay) {
    if (g.n < 1 || g.n >= (int64_t(1) << 31) - 1) return invalid("n must be in [1, 2^31-1)");
    if (g.K < 2 || g.K > 32) {
        set_error("K must be in [2, 32]");
        return FW_ERR_UNSUPPORTED;
    }
    if (!g.rp || !g.labels) return invalid("row_ptr and labels must not be NULL");
    if (g.rp[0] != 0) {
        set_error("row_ptr[0] must be 0");
        return FW_ERR_GRAPH;
    }
    const int64_t n = g.n;
    // branch-free passes over row_ptr and labels (the padded row offsets
    // themselves are formed on the device): a negative row length sets the
    // sign bit of `neg`.  Large inputs are split over a few host threads.
    struct Part {
        int64_t acc = 0, neg = 0;
        int bad = 0;
    };
    auto scan_part = [&g](int64_t i0, int64_t i1, Part& p) {
        const int32_t* __restrict__ rp = g.rp;
        const int32_t* __restrict__ lab = g.labels;
        int64_t acc = 0, neg = 0;
        int bad = 0;
        for (int64_t i = i0; i < i1; ++i) {
            const int64_t d = int64_t(rp[i + 1]) - int64_t(rp[i]);
            neg |= d;
            acc += (d + (kPadW - 1)) & ~int64_t(kPadW - 1);
            bad |= int(lab[i] < -1) | int(lab[i] >= g.K);
        }
        p.acc = acc;
        p.neg = neg;
        p.bad = bad;
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = n >= (int64_t(1) << 20) ? int(std::min(8u, hw)) : 1;
    std::vector<Part> parts(static_cast<size_t>(nt));
    bool threaded = false;
    if (nt > 1) {
        std::vector<std::thread> th;
        try {
            for (int t = 0; t < nt; ++t)
                th.emplace_back(scan_part, n * t / nt, n * (t + 1) / nt,
                                std::ref(parts[size_t(t)]));
            threaded = true;
        } catch (const std::system_error&) {
            threaded = false;   // no threads available: one pass below
        }
        for (auto& x : th) x.join();
    }
    if (!threaded) {
        parts.assign(1, Part());
        scan_part(0, n, parts[0]);
    }
    int64_t acc = 0, neg = 0;
    int bad = 0;
    for (const Part& p : parts) {
        acc += p.acc;
        neg |= p.neg;
        bad |= p.bad;
    }
    if (neg < 0) {
        set_error("row_ptr must be non-decreasing");
        return FW_ERR_GRAPH;
    }
    if (acc >= (int64_t(1) << 31)) {
        set_error("padded nnz must stay below 2^31");
        return FW_ERR_UNSUPPORTED;
    }
    if (bad) return invalid("labels must be -1 or in [0, K)");
    lay.n = n;
    lay.nnz = g.rp[n];
    lay.nnz_pad = acc;
    if (lay.nnz > 0 && (!g.col || !g.w)) return invalid("col and w must not be NULL");
    lay.npad = round_up(n, 32);
    lay.K = g.K;
    lay.tile_rows = tile_rows_for(n);
    lay.ntiles = int32_t((n + lay.tile_rows - 1) / lay.tile_rows);
    lay.lanes = o.lanes_per_row ? o.lanes_per_row : default_lanes(double(acc) / double(n));
    lay.allow16 = o.index_width != 32;
    lay.tab_mode = o.class_table;
    return FW_OK;
}

static size_t a256(size_t x) { return (x + 255) / 256 * 256; }

size_t problem_bytes(const ProbLayout& lay, size_t te, size_t we, bool comb) {
    const size_t n = size_t(lay.n), np = size_t(lay.npad), K = size_t(lay.K);
    size_t b = a256(4 * (n + 1)) + a256(4 * size_t(lay.nnz_pad)) + a256(we * size_t(lay.nnz_pad));
    if (comb) b += a256(te * n);
    b += 3 * a256(te * np * K) + a256(n) + a256(n);
    if (lay.cls4) b += a256((n + 1) / 2);
    b += a256(8 * size_t(kAccTotal));
    return b;
}

void place_problem(char* base, const ProbLayout& lay, size_t te, size_t we, const fw_seg_opts& o,
                   ProbDesc& pd) {
    const size_t n = size_t(lay.n), np = size_t(lay.npad), K = size_t(lay.K);
    const bool comb = o.laplacian == FW_LAPLACIAN_COMB;
    char* p = base;
    auto take = [&](size_t bytes) {
        char* q = p;
        p += a256(bytes);
        return q;
    };
    std::memset(&pd, 0, sizeof(pd));
    pd.rp = reinterpret_cast<const int32_t*>(take(4 * (n + 1)));
    pd.col = reinterpret_cast<const int32_t*>(take(4 * size_t(lay.nnz_pad)));
    pd.val = take(we * size_t(lay.nnz_pad));
    pd.diag = comb ? take(te * n) : nullptr;
    pd.U = take(te * np * K);
    pd.LU = take(te * np * K);
    pd.LS = take(te * np * K);
    pd.choice = reinterpret_cast<uint8_t*>(take(n));
    pd.cls4 = lay.cls4 ? reinterpret_cast<uint8_t*>(take((n + 1) / 2)) : nullptr;
    pd.fid = reinterpret_cast<const int8_t*>(take(n));
    pd.acc = reinterpret_cast<unsigned long long*>(take(8 * size_t(kAccTotal)));
    pd.n = int32_t(lay.n);
    pd.npad = int32_t(lay.npad);
    pd.K = lay.K;
    pd.tile_rows = lay.tile_rows;
    pd.ntiles = lay.ntiles;
    pd.lanes = lay.lanes;
    pd.comb = comb;
    pd.oracle = o.oracle;
    pd.step_rule = o.step_rule;
    pd.tol_mode = o.tol_mode;
    pd.max_iters = o.max_iters;
    pd.inv_eps = std::isinf(o.eps) ? 0.0 : 1.0 / o.eps;
    pd.omega0 = o.omega0;
    pd.gap_tol = o.gap_tol;
    pd.c2 = 2.0 * pd.inv_eps;
    pd.c2f = float(pd.c2);
    pd.omf = float(pd.omega0);
}

#define FW_TRYS(x)                      \
    do {                                \
        fw_status s_ = (x);             \
        if (s_ != FW_OK) return s_;     \
    } while (0)

// ------------------------------------------------------------- memory
// Handle arrays and create-time temporaries come from one stream-ordered
// memory pool per device.  Unlike the device's default pool, which gives
// freed memory back at every synchronisation, it keeps up to kPoolKeepBytes
// of freed memory mapped, so repeated create / destroy cycles (a request
// stream, the end-to-end loop) map no new memory.
constexpr uint64_t kPoolKeepBytes = 4ull << 30;
constexpr int kPoolMaxDevices = 64;

static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[kPoolMaxDevices] = {};

static cudaError_t device_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kPoolMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = kPoolKeepBytes;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pools[dev] = p;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

fw_status pool_alloc(void** out, size_t bytes, cudaStream_t s) {
    *out = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(out, std::max<size_t>(bytes, 16), pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        set_error(std::string("device allocation of ") + std::to_string(bytes) +
                  " bytes failed: " + cudaGetErrorString(e));
        return FW_ERR_NO_MEMORY;
    }
    return FW_OK;
}


static fw_status launched(const char* what) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FW_OK : cuda_fail(e, what);
}

fw_status restart_problem(Ops* ops, const ProbDesc& pd, ProbState* st, bool from_current,
                          cudaStream_t s) {
    Temps t(s);
    const int nb = int((pd.n + kBlock - 1) / kBlock);
    double* opart = nullptr;
    FW_TRYS(t.get(&opart, 8 * size_t(nb)));
    FW_CUDA(cudaMemsetAsync(pd.acc, 0, 8 * size_t(kAccTotal), s));
    if (from_current) {
        ops->spmm(pd, pd.U, pd.LU, s);
    } else {
        ops->reinit(pd, s);
        ops->spmm_hat(pd, pd.LU, s);
    }
    ops->objective(pd, pd.LU, opart, s);
    k_state_init<<<1, kBlock, 0, s>>>(st, opart, nb);
    return launched("restart kernels");
}

fw_status check_graph_args(const HostGraph& g) {
    if (g.n < 1 || g.n >= (int64_t(1) << 31) - 1) return invalid("n must be in [1, 2^31-1)");
    if (g.K < 2 || g.K > 32) {
        set_error("K must be in [2, 32]");
        return FW_ERR_UNSUPPORTED;
    }
    if (!g.rp || !g.labels) return invalid("row_ptr and labels must not be NULL");
    if (g.rp[0] != 0) {
        set_error("row_ptr[0] must be 0");
        return FW_ERR_GRAPH;
    }
    if (g.rp[g.n] < 0) {
        set_error("row_ptr[n] must be >= 0");
        return FW_ERR_GRAPH;
    }
    if (g.rp[g.n] > 0 && (!g.col || !g.w)) return invalid("col and w must not be NULL");
    return FW_OK;
}

fw_status upload_inputs(const HostGraph& g, Upload& up) {
    const cudaStream_t s = up.t.s;
    const int64_t n = g.n, nnz = g.rp[g.n];
    up.n = n;
    up.nnz = nnz;
    FW_TRYS(up.t.get(&up.rp, 4 * (size_t(n) + 1)));
    FW_TRYS(up.t.get(&up.col, 4 * size_t(nnz)));
    FW_TRYS(up.t.get(&up.w, 8 * size_t(nnz)));
    FW_TRYS(up.t.get(&up.lab, 4 * size_t(n)));
    FW_CUDA(cudaMemcpyAsync(up.rp, g.rp, 4 * (size_t(n) + 1), cudaMemcpyHostToDevice, s));
    if (nnz) {
        FW_CUDA(cudaMemcpyAsync(up.col, g.col, 4 * size_t(nnz), cudaMemcpyHostToDevice, s));
        FW_CUDA(cudaMemcpyAsync(up.w, g.w, 8 * size_t(nnz), cudaMemcpyHostToDevice, s));
    }
    FW_CUDA(cudaMemcpyAsync(up.lab, g.labels, 4 * size_t(n), cudaMemcpyHostToDevice, s));
    return FW_OK;
}

// Pass B with the class table in shared memory (k_passB_tab): where the
// table and the bins fit one block's shared memory, the tiles are single
// 256-row sub-tiles and the lane count has a compiled form.  AUTO takes it for
// graphs whose columns are not banded (their class gathers miss L1; banded
// ones hit it) and that have at least one tile per SM; ON wherever it fits.
static fw_status choose_tab(Ops* ops, const ProbLayout& lay, ProbDesc& pd) {
    pd.tab_grid = 0;
    if (lay.tab_mode == FW_TABLE_OFF || !pd.cls4 || lay.tile_rows != kBlock) return FW_OK;
    if (lay.lanes != 1 && lay.lanes != 2 && lay.lanes != 4) return FW_OK;
    const size_t need = ops->tab_smem(lay.lanes, lay.n);
    if (need == 0 || need > size_t(kTabSmemMax)) return FW_OK;
    int dev = 0, sms = 0, optin = 0;
    FW_CUDA(cudaGetDevice(&dev));
    FW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FW_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (need + 2048 > size_t(optin)) return FW_OK;
    if (lay.tab_mode == FW_TABLE_AUTO && (pd.col16 || lay.ntiles < sms)) return FW_OK;
    const int grid = std::max(std::min(sms, lay.ntiles),
                              (lay.ntiles + kTabMaxTiles - 1) / kTabMaxTiles);
    pd.tab_grid = grid;
    return FW_OK;
}

fw_status assemble_problem(Ops* ops, const HostGraph& g, const ProbLayout& lay, ProbDesc& pd,
                           ProbState* st, cudaStream_t s) {
    Upload up(s);
    FW_TRYS(check_graph_args(g));
    FW_TRYS(upload_inputs(g, up));
    return assemble_uploaded(ops, up, lay, pd, st, s);
}

fw_status assemble_uploaded(Ops* ops, Upload& up, const ProbLayout& lay, ProbDesc& pd,
                            ProbState* st, cudaStream_t s) {
    Temps& t = up.t;
    const int64_t n = lay.n;
    const size_t te = ops->elem();
    const int32_t* d_rp = up.rp;
    const int32_t* d_col = up.col;
    const double* d_w = up.w;
    const int32_t* d_lab = up.lab;
    double* d_deg = nullptr;
    int* d_err = nullptr;
    FW_TRYS(t.get(&d_deg, 8 * size_t(n)));
    FW_TRYS(t.get(&d_err, sizeof(int)));
    {   // padded row offsets into pd.rp
        const int nb = int((n + kScanRows - 1) / kScanRows);
        int32_t* d_bsum = nullptr;
        FW_TRYS(t.get(&d_bsum, 4 * size_t(nb)));
        int32_t* prp = const_cast<int32_t*>(pd.rp);
        k_pad_scan_local<<<nb, kBlock, 0, s>>>(n, d_rp, prp, d_bsum);
        k_pad_scan_blocks<<<1, kBlock, 0, s>>>(n, nb, d_bsum, prp);
        k_pad_scan_add<<<unsigned((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, d_bsum, prp);
        FW_TRYS(launched("row offset scan"));
    }
    const size_t blk = te * size_t(lay.npad) * size_t(lay.K);
    FW_CUDA(cudaMemsetAsync(pd.U, 0, blk, s));
    FW_CUDA(cudaMemsetAsync(pd.LS, 0, blk, s));
    FW_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    const unsigned gr = unsigned((n + kBlock - 1) / kBlock);
    k_validate<<<gr, kBlock, 0, s>>>(n, d_rp, d_col, d_w, d_deg, d_err);
    FW_TRYS(launched("validate kernel"));
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
    // banded graphs (pixel grids, meshes) keep 16-bit column offsets: the
    // same entries in half the column bytes of every sparse pass
    pd.col16 = (lay.allow16 && !(err & 8)) ? 1 : 0;
    FW_TRYS(choose_tab(ops, lay, pd));
    if (!pd.comb) k_inv_sqrt<<<gr, kBlock, 0, s>>>(n, d_deg);
    ops->build(n, d_rp, d_col, d_w, d_deg, pd.rp, const_cast<int32_t*>(pd.col),
               const_cast<void*>(pd.val), const_cast<void*>(pd.diag), pd.comb, pd.col16, s);
    k_fid<<<gr, kBlock, 0, s>>>(n, d_lab, const_cast<int8_t*>(pd.fid));
    FW_TRYS(launched("build kernels"));
    return restart_problem(ops, pd, st, false, s);
}

}  // namespace fw
