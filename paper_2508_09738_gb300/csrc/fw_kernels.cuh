// __global__ kernels of the single-problem path and of graph assembly.
#pragma once
#include "fw_device.cuh"

namespace fw {

// ---------------------------------------------------------------- hot loop
// Step pass A of one tile (k_passA, k_passA_exact).  With `fin` the block first
// takes the previous iteration's step decision itself (no k_finish between
// the passes; see ProbState); otherwise it applies the step k_finish stored.
// `tile`: the problem's row tile this block works on (its block index in the
// single-problem launch, its work item's tile in a batched item launch).
template <typename T, int KMAX, bool EXACT>
__device__ __forceinline__ void passA_step(const ProbDesc& pd, ProbState* st, int fin, T* stage,
                                           int tile) {
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ double s_alpha;
    __shared__ int s_stop, s_done, s_cur;
    // Block 0 of this launch may commit a stop (done = 1) while other blocks
    // start: one thread reads the flag (and the parity) and the whole block
    // follows it, so no block splits between leaving and waiting on the bulk
    // copies; that thread issues the copies as soon as it knows.
    if (threadIdx.x == 0) {
        const int d = ld_cg(&st->done);
        const int c0 = ld_cg(&st->cur);
        s_done = d;
        s_cur = c0;
        if (!d) {
            mbar_init(&bars[0], 1);
            mbar_init(&bars[1], 1);
            if (fin) {   // the first copies go out at once (a step is always pending)
                const int r0 = tile * pd.tile_rows;
                stage_issue<T, KMAX>(pd, r0, min(kBlock, pd.n - r0), true, stage, &bars[0]);
            } else if (tile == 0) {
                st->cur_b = c0;
            }
        }
    }
    __syncthreads();
    if (s_done) return;
    const int c = s_cur;
    if (fin && threadIdx.x < 32) {
        // warp 0 takes the previous iteration's decision while the copies are
        // in flight; block 0 commits it
        double a;
        const int stop = warp_decide(pd.acc + c * kAccBank, st, c, step_cfg(pd), tile == 0, &a);
        if (threadIdx.x == 0) {
            s_stop = stop;
            s_alpha = a;
            if (tile == 0) st->cur_b = c ^ 1;
        }
    }
    const bool upd = fin ? true : ld_cg(&st->has_update) != 0;
    const T alpha = fin ? T(0) : alpha_of<T>(st);
    __syncthreads();
    uint32_t phases = 0;
    const int nst = (pd.tile_rows > kBlock && max_stages<T, KMAX>() == 2) ? 2 : 1;
    const int bank = fin ? (c ^ 1) : c;
    tile_A<T, KMAX, EXACT>(pd, st, tile, upd, alpha, FuseCtl{fin != 0, &s_stop, &s_alpha},
                           pd.acc + bank * kAccBank, stage, nst, bars, phases);
}

// Pass B entry: this iteration's bank (set by pass A); block 0 makes it the
// pending bank and clears the other one, which the next pass A will fill.
__device__ __forceinline__ unsigned long long* passB_bank(const ProbDesc& pd, ProbState* st,
                                                          bool& done, int tile) {
    const int b = ld_cg(&st->cur_b);
    done = ld_cg(&st->done) != 0;
    if (tile == 0 && threadIdx.x == 0) {
        st->cur = b;
        unsigned long long* z = pd.acc + (b ^ 1) * kAccBank;
#pragma unroll
        for (int w = 0; w < kAccWords; ++w) z[w] = 0ull;
    }
    return pd.acc + b * kAccBank;
}

// Blocks of pass A that one SM holds by shared memory (one stage buffer; at
// most 8, or 5 for an FP64 iterate, whose rows need more registers): the
// register budget is set to match, so that the fused step decision does not
// lower the occupancy.
template <typename T, int KMAX>
constexpr int passA_min_blocks() {
    constexpr int cap = sizeof(T) == 8 ? 5 : 8;
    constexpr int b = (227 * 1024) / (3 * kBlock * KMAX * int(sizeof(T)) + 1024);
    return b < 1 ? 1 : (b > cap ? cap : b);
}

// Pass A: one block per row tile.
//   MODE_STEP applies the pending step and evaluates (passA_step);
//   MODE_FLUSH applies a pending step only; MODE_GRAD writes G' and the choice.
template <typename T, int KMAX, int MODE>
__global__ void __launch_bounds__(kBlock, MODE == MODE_STEP ? passA_min_blocks<T, KMAX>() : 1)
    k_passA(ProbDesc pd, ProbState* st, T* Gout, uint8_t* chout, int fin) {
    if constexpr (MODE == MODE_STEP) {
        extern __shared__ __align__(128) unsigned char smraw[];
        passA_step<T, KMAX, false>(pd, st, fin, reinterpret_cast<T*>(smraw), blockIdx.x);
    } else {
        if (MODE != MODE_GRAD && ld_cg(&st->done)) return;
        const bool upd = ld_cg(&st->has_update) != 0;
        const T alpha = alpha_of<T>(st);
        const int r0 = blockIdx.x * pd.tile_rows;
        const int r1 = min(pd.n, r0 + pd.tile_rows);
        AccA<T> acc{T(0), T(0), T(0), T(0), T(0)};
        passA_rows<T, KMAX, MODE>(pd, r0, r1, upd, alpha, acc, Gout, chout);
        if (MODE == MODE_FLUSH) {
            if (last_to_arrive(&st->cntF, pd.ntiles) && threadIdx.x == 0) {
                st->has_update = 0;
                st->cntF = 0;
            }
        }
    }
}

// Pass A (step) for exactly KMAX classes with an FP32 iterate: the class loop
// is fully known at compile time, which removes the per-class guards.  Used
// for four classes, where it is held to 32 registers (8 blocks per SM).
template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock, passA_min_blocks<T, KMAX>())
    k_passA_exact(ProbDesc pd, ProbState* st, int fin) {
    extern __shared__ __align__(128) unsigned char smraw[];
    passA_step<T, KMAX, true>(pd, st, fin, reinterpret_cast<T*>(smraw), blockIdx.x);
}

// Pass B: one block per row tile; each adds its tile total to the exact
// accumulators (no block waits for another).
template <typename T, typename WT, int KMAX>
__global__ void __launch_bounds__(kBlock) k_passB(ProbDesc pd, ProbState* st) {
    bool done;
    unsigned long long* accb = passB_bank(pd, st, done, blockIdx.x);
    if (done) return;
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm_lane = reinterpret_cast<T*>(smraw);
    T* sm_row = sm_lane + kBlock * (KMAX | 1);
    tile_B<T, WT, KMAX, true, false>(pd, st, blockIdx.x, sm_lane, sm_row,
                                     sm_row + kBlock * (KMAX | 1), accb, nullptr);
}

// Pass B with LC lanes per row known at compile time (1 for low-degree graphs
// such as images, 2 or 4 for denser ones); EXACT for exactly KMAX classes.
// Same sums, in the same order, as k_passB.
template <typename T, typename WT, int KMAX, int LC, bool EXACT>
__device__ __forceinline__ void passB_lc_body(const ProbDesc& pd, ProbState* st) {
    bool done;
    unsigned long long* accb = passB_bank(pd, st, done, blockIdx.x);
    if (done) return;
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm_lane = reinterpret_cast<T*>(smraw);
    T* sm_row = sm_lane + kBlock * (KMAX | 1);
    tile_B<T, WT, KMAX, true, false, LC, EXACT>(pd, st, blockIdx.x, sm_lane, sm_row,
                                                sm_row + kBlock * (KMAX | 1), accb, nullptr);
}

template <typename T, typename WT, int KMAX, int LC, bool EXACT>
__global__ void __launch_bounds__(kBlock) k_passB_lc(ProbDesc pd, ProbState* st) {
    passB_lc_body<T, WT, KMAX, LC, EXACT>(pd, st);
}

// The 2- and 4-lane forms for 5 to 12 classes of FP32 need 44-48 registers,
// i.e. 5 blocks per SM, and a problem with more tiles than 5 x 152 then runs
// a second wave (sbm200k: 782 tiles).  Held to 40 registers (6 blocks per SM,
// a few spilled words) they measured 7% faster there.
template <typename T, typename WT, int KMAX, int LC, bool EXACT>
__global__ void __launch_bounds__(kBlock, 6) k_passB_lc6(ProbDesc pd, ProbState* st) {
    passB_lc_body<T, WT, KMAX, LC, EXACT>(pd, st);
}

// Pass B with the class table in shared memory (see passB_unit): one block
// of kTabThreads threads per SM over a contiguous run of at most
// kTabMaxTiles 256-row tiles.  The table arrives by bulk copies while the
// block starts; a copy that does not arrive within the bounded wait raises
// the problem's error flag and the block adds nothing.
template <typename T, typename WT, int KMAX, int LC, bool EXACT>
__global__ void __launch_bounds__(kTabThreads, 1) k_passB_tab(ProbDesc pd, ProbState* st) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ T s_part[kTabMaxTiles * (kBlock / 32)];
    const int G = gridDim.x;
    const int t0 = int(int64_t(blockIdx.x) * pd.ntiles / G);
    const int t1 = int(int64_t(blockIdx.x + 1) * pd.ntiles / G);
    bool done;
    unsigned long long* accb = passB_bank(pd, st, done, t0);   // block 0 holds tile 0
    if (done) return;
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm_lane = reinterpret_cast<T*>(smraw);
    T* sm_row = sm_lane + kTabThreads * (KMAX | 1);   // unused with one lane per row
    uint8_t* tab = smraw + tab_bins_bytes<T, KMAX>(LC);
    if (threadIdx.x == 0) {
        const uint32_t tb = tab_bytes(pd.n);
        mbar_init(&bar, 1);
        fence_proxy_async();
        mbar_expect_tx(&bar, tb);
        for (uint32_t o = 0; o < tb; o += 32768u)
            bulk_g2s(tab + o, pd.cls4 + o, min(32768u, tb - o), &bar);
    }
    {
        // while the table arrives, pull the block's CSR slice (row offsets,
        // columns, weights) into L2, so the warps' dependent loads below wait
        // on L2 rather than DRAM
        const int rb = t0 * kBlock, re = min(pd.n, t1 * kBlock);
        const int e0 = __ldg(pd.rp + rb), e1 = __ldg(pd.rp + re);
        const int cw = pd.col16 ? 2 : 4;
        prefetch_l2_range(reinterpret_cast<const char*>(pd.col) + int64_t(e0) * cw,
                          int64_t(e1 - e0) * cw);
        prefetch_l2_range(static_cast<const WT*>(pd.val) + e0, int64_t(e1 - e0) * sizeof(WT));
        prefetch_l2_range(pd.rp + rb, int64_t(re - rb + 1) * 4);
    }
    __syncthreads();   // the barrier is initialised before any thread waits on it
    const bool got = mbar_wait(&bar, 0);
    if (__syncthreads_or(!got)) {
        if (!got) mbar_wait(&bar, 0);   // bounded: let copies still in flight land
        __syncthreads();
        if (threadIdx.x == 0) atomicExch(&st->err, 1);
        return;
    }
    // warp w takes units w, w + 32, ...; unit u is warp (u % 8) of tile t0 + u / 8
    const int nunits = (t1 - t0) * (kBlock / 32);
    for (int u = threadIdx.x >> 5; u < nunits; u += kTabThreads / 32) {
        const int tile = t0 + u / (kBlock / 32);
        const int row0 = tile * kBlock + (u % (kBlock / 32)) * 32;
        const int r_end = min(pd.n, tile * kBlock + kBlock);
        T x = passB_unit<T, WT, KMAX, LC, EXACT>(pd, row0, r_end, sm_lane, sm_row, tab);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x = add_(x, __shfl_xor_sync(0xffffffffu, x, off));
        if ((threadIdx.x & 31) == 0) s_part[u] = x;
    }
    __syncthreads();
    // each tile's total: its 8 warp sums in warp order (block_accumulate's order)
    if (threadIdx.x < t1 - t0) {
        T sum = T(0);
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) sum = add_(sum, s_part[threadIdx.x * (kBlock / 32) + w]);
        fx_add(acc_slot(accb, (t0 + int(threadIdx.x)) % kAccCopies, kNumA), accb + kAccFlag,
               double(sum));
    }
}

// One thread after pass B: read the iteration's totals (complete after the
// kernel boundary, in bank cur), run the stop test and the step.  Inside a
// captured graph only the last iteration ends with it; the others leave the
// decision to the next pass A.  (Doing it in the last block of pass B instead
// costs every block a fence and an arrival, which measured slower.)
static __global__ void k_finish(ProbDesc pd, ProbState* st) {   // one warp
    if (ld_cg(&st->done)) return;
    warp_finish(pd, st, pd.acc + ld_cg(&st->cur) * kAccBank);
}

// One-Shot Frank-Wolfe (Alg. 4): labels of U_1 = GLMO(grad E(U_hat)) in one
// CSR pass; the iterate arrays are not touched.  There is no reduction, so
// each block takes one 256-row sub-tile (fine-grained, no tail wave).
template <typename T, typename WT, int KMAX>
__global__ void __launch_bounds__(kBlock) k_osfw(ProbDesc pd, int32_t* labels) {
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm_lane = reinterpret_cast<T*>(smraw);
    T* sm_row = sm_lane + kBlock * (KMAX | 1);
    const int r0 = blockIdx.x * kBlock;
    const int r1 = min(pd.n, r0 + kBlock);
    osfw_rows<T, WT, KMAX>(pd, labels, r0, r1, sm_lane, sm_row);
}

// OUT = L X (initial L U_0, refresh, direct objective).
template <typename T, typename WT, int KMAX>
__global__ void __launch_bounds__(kBlock) k_spmm(ProbDesc pd, const T* X, T* OUT) {
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm_lane = reinterpret_cast<T*>(smraw);
    T* sm_row = sm_lane + kBlock * (KMAX | 1);
    const int r0 = blockIdx.x * pd.tile_rows;
    const int r1 = min(pd.n, r0 + pd.tile_rows);
    spmm_rows<T, WT, KMAX>(pd, X, OUT, r0, r1, sm_lane, sm_row);
}

// L U_0 for U_0 = U_hat (the state reinit writes): the off-diagonal product
// from the fidelity bytes (an unlabelled neighbour adds w/K to every class, a
// labelled one w to its class), bitwise the dense SpMM of U_hat and without
// its K gathers per entry.
template <typename T, typename WT, int KMAX>
__global__ void __launch_bounds__(kBlock) k_spmm_hat(ProbDesc pd, T* OUT) {
    extern __shared__ __align__(128) unsigned char smraw[];
    T* sm_lane = reinterpret_cast<T*>(smraw);
    T* sm_row = sm_lane + kBlock * (KMAX | 1);
    const int r0 = blockIdx.x * pd.tile_rows;
    const int r1 = min(pd.n, r0 + pd.tile_rows);
    spmm_rows<T, WT, KMAX, kSrcUhat>(pd, static_cast<const T*>(pd.U), OUT, r0, r1, sm_lane,
                                     sm_row);
}

// ------------------------------------------------------------ read-outs
// labels[i] = argmax_k u_ik, lowest index on ties.
template <typename T>
__global__ void k_labels(ProbDesc pd, int32_t* out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= pd.n) return;
    const T* Ub = static_cast<const T*>(pd.U);
    T best = Ub[r];
    int b = 0;
    for (int k = 1; k < pd.K; ++k) {
        const T x = Ub[(int64_t)k * pd.npad + r];
        if (x > best) {
            best = x;
            b = k;
        }
    }
    out[r] = b;
}

// Per-block FP64 partials of E(U) with a freshly computed LUf = L U
// (eq. gradgl_vv2): 1/2 <U, L U> + 1/eps sum u(1-u) + 1/2 sum w_i ||u_hat_i - u_i||^2.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_objective(ProbDesc pd, const T* LUf, double* part) {
    // per row in the iterate type (FP64 per element was the bulk of this
    // kernel on GB300), across rows in FP64
    const int r = blockIdx.x * kBlock + threadIdx.x;
    double e = 0.0;
    if (r < pd.n) {
        const T* Ub = static_cast<const T*>(pd.U);
        const int f = pd.fid[r];
        T quad = T(0), pen = T(0), fidt = T(0);
        for (int k = 0; k < pd.K; ++k) {
            const T u = Ub[(int64_t)k * pd.npad + r];
            quad = fma_(u, LUf[(int64_t)k * pd.npad + r], quad);
            pen = fma_(u, sub_(T(1), u), pen);
            if (f >= 0) {
                const T d = sub_(k == f ? T(1) : T(0), u);
                fidt = fma_(d, d, fidt);
            }
        }
        e = 0.5 * double(quad) + pd.inv_eps * double(pen) + 0.5 * pd.omega0 * double(fidt);
    }
    const double v[1] = {e};
    block_partials<double, 1>(v, part + blockIdx.x);
}

// Classic (full-LMO) FW gap at U (Alg. 2), the stationarity measure over
// Sigma: per row sum_k u_ik (G'_ik - min_j G'_ij) with G' from a freshly
// computed LUf = L U (the constant 1/eps term cancels); FP64 block partials.
template <typename T, int KMAX>
__global__ void __launch_bounds__(kBlock) k_lmo_gap(ProbDesc pd, const T* LUf, double* part) {
    const int r = blockIdx.x * kBlock + threadIdx.x;
    double e = 0.0;
    if (r < pd.n) {
        const T* Ub = static_cast<const T*>(pd.U);
        const int f = pd.fid[r];
        const T c2 = c2_of<T>(pd);
        const T om = om_of<T>(pd);
        T u[KMAX], g[KMAX];
        T mn = inf_<T>();
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < pd.K) {
                u[k] = Ub[(int64_t)k * pd.npad + r];
                T gk = fma_(-c2, u[k], LUf[(int64_t)k * pd.npad + r]);
                if (f >= 0) gk = fma_(om, sub_(u[k], k == f ? T(1) : T(0)), gk);
                g[k] = gk;
                mn = gk < mn ? gk : mn;
            }
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < pd.K) acc = fma_(u[k], sub_(g[k], mn), acc);
        e = double(acc);
    }
    const double v[1] = {e};
    block_partials<double, 1>(v, part + blockIdx.x);
}

// Fresh iteration state: E_0 = fixed-order sum of the objective partials,
// everything else zero, status FW_PENDING (one block).
__global__ void __launch_bounds__(kBlock) k_state_init(ProbState* st, const double* part, int nb);

// ------------------------------------------------------------- assembly
// Padded CSR of the off-diagonal operator: sym: W^_ij = w_ij / sqrt(d_i d_j)
// rounded to WT (bf16 via float, both nearest-even); comb: w_ij.  Padding
// entries point at the row itself with weight 0.  diag (comb only) = d_i.
template <typename WT, typename T>
__global__ void k_build(int64_t n, const int32_t* rp, const int32_t* col, const double* w,
                        const double* deg, const int32_t* rpp, int32_t* colp, WT* valp, T* diag,
                        int comb, int col16) {
    // deg holds d_i for L = D - W and d_i^{-1/2} for L_s (k_inv_sqrt): the
    // normalised weight is then two FP64 products per entry, since FP64
    // square roots and divisions per entry dominated this kernel on GB300
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e0 = rp[i], e1 = rp[i + 1];
    int p = rpp[i];
    const int pend = rpp[i + 1];
    const double di = deg[i];
    int16_t* colp16 = reinterpret_cast<int16_t*>(colp);
    for (int e = e0; e < e1; ++e, ++p) {
        const int j = col[e];
        const double x = comb ? w[e] : (w[e] * di) * deg[j];
        if (col16) colp16[p] = int16_t(j - int(i));   // |j - i| < 2^15 (checked)
        else colp[p] = j;
        if constexpr (sizeof(WT) == 2)
            valp[p] = __float2bfloat16_rn(__double2float_rn(x));
        else if constexpr (sizeof(WT) == 4)
            valp[p] = __double2float_rn(x);
        else
            valp[p] = x;
    }
    for (; p < pend; ++p) {
        if (col16) colp16[p] = 0;
        else colp[p] = int32_t(i);
        valp[p] = WT(0.0f);
    }
    if (comb) diag[i] = T(di);
}

// U_0 = U_hat (Sec. 5.1): e_c on fidelity rows, 1/K elsewhere; choice reset.
template <typename T>
__global__ void k_reinit(ProbDesc pd) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;   // blockDim.x = kBlock
    int cls = 0;
    if (r < pd.n) {
        const int c = pd.fid[r];
        const T unif = T(1) / T(pd.K);
        T* Ub = static_cast<T*>(pd.U);
        for (int k = 0; k < pd.K; ++k)
            Ub[(int64_t)k * pd.npad + r] = c >= 0 ? (k == c ? T(1) : T(0)) : unif;
        cls = c >= 0 ? c : 0;
        pd.choice[r] = uint8_t(cls);
    }
    if (pd.cls4) {
        const int hi = __shfl_down_sync(0xffffffffu, cls, 1);
        if ((r & 1) == 0 && r < pd.n) pd.cls4[r >> 1] = uint8_t(cls | (hi << 4));
    }
}

}  // namespace fw
