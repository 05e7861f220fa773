// Device code of the Greedy Frank-Wolfe (GFW) hot path, shared by the plain
// per-pass kernels and the persistent batched kernel.
//
// One GFW iteration (Alg. 3) is two passes over a problem's rows:
//   pass A (row pass):  apply the pending update of the previous step
//                       U <- (1-a) U + a S,  LU <- (1-a) LU + a LS   (Sec. 4, Alg. 3 step 6)
//                       then G' = LU - (2/eps) U + D_w (U - U_hat)    (eq. gradgl_vv2g without 1/eps)
//                       the greedy LMO choice (eq. eq:LMOpr) and the per-row pieces of
//                       the FW gap g = -<G, D> and of ||D||^2, sum w_i ||D_i||^2, <D, LU>.
//   pass B (CSR pass):  LS = L S for the one-hot S: (L S)_ik = [s_i = k] - sum_{j: s_j = k} W^_ij,
//                       and the per-row <D_i, LS_i>.
// Both passes add block totals into exact fixed-point accumulators; from the
// totals one warp (warp_decide) forms q = <D, L D> + sum w_i||D_i||^2 -
// (2/eps)||D||^2 (Hessian of App. C), runs the stop test and takes the exact
// step a = min(1, g/q) (1 if q <= 0), either in k_finish or at the start of
// the next pass A.
// L U is never recomputed inside the loop: it follows the recurrence above, and a
// separate SpMM (spmm_rows) builds it at the start and on refresh.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "fw_types.h"

namespace fw {

// --------------------------------------------------------------- rounding
// Explicitly rounded operations: every instantiation and every kernel that
// evaluates the same formula produces the same bits (no contraction choices).
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T> __device__ __forceinline__ T inf_();
template <> __device__ __forceinline__ float inf_<float>() { return CUDART_INF_F; }
template <> __device__ __forceinline__ double inf_<double>() { return CUDART_INF; }

// ------------------------------------------------------------ weight loads
// Four consecutive entries of a padded CSR row (start is a multiple of 4).
__device__ __forceinline__ int4 ld_stream(const int4* p);
__device__ __forceinline__ float4 ld_stream(const float4* p);
__device__ __forceinline__ uint2 ld_stream(const uint2* p);
__device__ __forceinline__ double2 ld_stream(const double2* p);

__device__ __forceinline__ void ld_w4(const float* p, float (&v)[4]) {
    const float4 t = ld_stream(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld_w4(const __nv_bfloat16* p, float (&v)[4]) {
    // bf16 is the upper half of an fp32 pattern: widening is a shift (exact)
    const uint2 t = ld_stream(reinterpret_cast<const uint2*>(p));
    v[0] = __uint_as_float(t.x << 16);
    v[1] = __uint_as_float(t.x & 0xffff0000u);
    v[2] = __uint_as_float(t.y << 16);
    v[3] = __uint_as_float(t.y & 0xffff0000u);
}
__device__ __forceinline__ void ld_w4(const double* p, double (&v)[4]) {
    const double2 a = ld_stream(reinterpret_cast<const double2*>(p));
    const double2 b = ld_stream(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Plain (coherent) loads for data written inside a persistent launch.
template <typename T> __device__ __forceinline__ T ld_cg(const T* p) { return __ldcg(p); }

// Streaming loads that do not allocate in L1 (CSR columns and weights), so
// that the gathered class bytes keep their L1 lines.
__device__ __forceinline__ int4 ld_stream(const int4* p) {
    int4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_stream(const float4* p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ uint2 ld_stream(const uint2* p) {
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];"
                 : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ double2 ld_stream(const double2* p) {
    double2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];"
                 : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}

// Per-iteration constants in the iterate type (precomputed on the host, so
// the kernels do no FP64 work per thread in the FP32 path).
template <typename T> __device__ __forceinline__ T c2_of(const ProbDesc& pd);
template <> __device__ __forceinline__ float c2_of<float>(const ProbDesc& pd) { return pd.c2f; }
template <> __device__ __forceinline__ double c2_of<double>(const ProbDesc& pd) { return pd.c2; }
template <typename T> __device__ __forceinline__ T om_of(const ProbDesc& pd);
template <> __device__ __forceinline__ float om_of<float>(const ProbDesc& pd) { return pd.omf; }
template <> __device__ __forceinline__ double om_of<double>(const ProbDesc& pd) { return pd.omega0; }
template <typename T> __device__ __forceinline__ T alpha_of(const ProbState* st);
template <> __device__ __forceinline__ float alpha_of<float>(const ProbState* st) {
    return __ldcg(&st->alpha_f);
}
template <> __device__ __forceinline__ double alpha_of<double>(const ProbState* st) {
    return __ldcg(&st->alpha);
}

// ------------------------------------------------ bulk async copies (TMA)
// 1-D cp.async.bulk global -> shared completing on an mbarrier.  Addresses
// and sizes must be multiples of 16 bytes; callers guarantee it.
constexpr unsigned long long kMbarWaitNs = 2000000000ull;   // bound of one mbarrier wait: 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or about `ns` nanoseconds pass, instead of re-issuing polls.
__device__ __forceinline__ bool mbar_test_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity, bounded in time by kMbarWaitNs;
// false when the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_test_sleep(bar, parity, 20000u)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 <= kMbarWaitNs)
        if (mbar_test_sleep(bar, parity, 20000u)) return true;
    return mbar_test(bar, parity);
}

// 16-byte asynchronous global -> shared copies (L2 only, so data written by
// other blocks before a grid barrier is seen), completed per thread.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}
// L2 prefetch of the 128-byte lines of [p, p + bytes) by the block's threads.
// The caller's array starts on a 128-byte boundary, so every line touched lies
// in it.
__device__ __forceinline__ void prefetch_l2_range(const void* p, int64_t bytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uintptr_t end = a + uintptr_t(bytes);
    for (uintptr_t q = (a & ~uintptr_t(127)) + uintptr_t(threadIdx.x) * 128u; q < end;
         q += uintptr_t(blockDim.x) * 128u)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
}
__device__ __forceinline__ int ld_shared_u8(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(addr));
    return int(v);
}

// ------------------------------------------------------- block reductions
// GB300 executes FP64 at a small fraction of the FP32 rate, so FP64 is used
// only where sums span many tiles: rows of one 256-row tile are summed in the
// iterate type T (warp butterfly, then the 8 warps in a fixed order) and the
// tile total is widened to double once per quantity.

// Sum NQ per-thread values over the block; thread q < NQ writes out[q].
// Must be reached by every thread of the block.
template <typename T, int NQ>
__device__ __forceinline__ void block_partials(const T (&v)[NQ], double* __restrict__ out) {
    __shared__ T red[kBlock / 32][NQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        T x = v[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x = add_(x, __shfl_xor_sync(0xffffffffu, x, off));
        if (lane == 0) red[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        T s = T(0);
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) s = add_(s, red[w][threadIdx.x]);
        out[threadIdx.x] = double(s);
    }
    __syncthreads();
}

// True in exactly one block: the last of `total` arrivals on *cnt.  The
// partials the arriving blocks wrote before are visible to it afterwards.
__device__ __forceinline__ bool last_to_arrive(uint32_t* cnt, uint32_t total) {
    __shared__ uint32_t s_prev;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_prev = atomicAdd(cnt, 1u);
    }
    __syncthreads();
    const bool last = (s_prev == total - 1);
    if (last) __threadfence();
    return last;
}

// ------------------------------------------ exact order-free accumulation
// A finite double v with |v| < 2^52 is added to a 128-bit two's-complement
// fixed-point number with 64 fraction bits (slot[0] = lo, slot[1] = hi):
// v = hi + frac with hi = floor(v), frac in [0, 1) exactly, and frac * 2^64
// truncated to an integer (parts below 2^-64 are dropped).  The carry of the
// low-word add is exact, so the total is the exact sum of the added values
// whatever the order of the atomic operations.  A problem has at most
// kTilesTarget (< 2^11) tiles, so a total of values below 2^52 cannot
// overflow the signed high word.  Non-finite or larger values raise *flag.
__device__ __forceinline__ void fx_add(unsigned long long* slot, unsigned long long* flag,
                                       double v) {
    static_assert(kTilesTarget < 2048, "fixed-point totals assume < 2^11 tiles");
    if (!isfinite(v) || fabs(v) >= 0x1p52) {
        atomicOr(flag, 1ull);
        return;
    }
    const double fl = floor(v);
    const unsigned long long lo = __double2ull_rz(ldexp(v - fl, 64));
    const unsigned long long hi = static_cast<unsigned long long>(__double2ll_rz(fl));
    const unsigned long long old = atomicAdd(&slot[0], lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    atomicAdd(&slot[1], hi + carry);
}

__device__ __forceinline__ unsigned long long* acc_slot(unsigned long long* acc, int copy, int q) {
    return acc + (copy * kNumR + q) * kAccLine;
}

// Exact total of quantity q over the accumulator copies (128-bit sum), as a
// double.
__device__ __forceinline__ double fx_total(const unsigned long long* acc, int q) {
    unsigned long long lo = 0ull, hi = 0ull;
#pragma unroll
    for (int c = 0; c < kAccCopies; ++c) {
        const unsigned long long* sl = acc + (c * kNumR + q) * kAccLine;
        const unsigned long long l = __ldcg(sl), h = __ldcg(sl + 1);
        const unsigned long long lo2 = lo + l;
        hi += h + (lo2 < lo ? 1ull : 0ull);
        lo = lo2;
    }
    return double(static_cast<long long>(hi)) + ldexp(double(lo), -64);
}

// Sum NQ per-thread values over the block (FP32 warp butterfly, then the
// warps in a fixed order) and add the block total of quantity q0+q to copy
// `copy` of the fixed-point accumulators.
template <typename T, int NQ>
__device__ __forceinline__ void block_accumulate(const T (&v)[NQ], unsigned long long* acc, int q0,
                                                 int copy) {
    __shared__ T red[kBlock / 32][NQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        T x = v[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x = add_(x, __shfl_xor_sync(0xffffffffu, x, off));
        if (lane == 0) red[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        T s = T(0);
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) s = add_(s, red[w][threadIdx.x]);
        fx_add(acc_slot(acc, copy, q0 + threadIdx.x), acc + kAccFlag, double(s));
    }
    __syncthreads();
}

// Fixed-order FP64 sum of `count` records of NQ doubles: thread t loads
// records t, t+kBlock, ... (four records ahead, so up to 4*kBlock records take
// one round trip) and adds them in that order; warp 0 then adds the threads'
// sums (lane l: threads l, l+32, ..., in order) and a butterfly finishes.
// `scratch` is kBlock*NQ doubles of shared memory.  Every thread of the block
// must call it; out[] is valid in all threads.
template <int NQ>
__device__ __forceinline__ void sum_partials(const double* __restrict__ part, int count,
                                             double (&out)[NQ], double* scratch) {
    constexpr int kAhead = 4;
    double s[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) s[q] = 0.0;
    for (int t0 = threadIdx.x; t0 < count; t0 += kAhead * kBlock) {
        double v[kAhead][NQ];
#pragma unroll
        for (int a = 0; a < kAhead; ++a) {
            const int t = t0 + a * kBlock;
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                v[a][q] = t < count ? __ldcg(part + (size_t)t * NQ + q) : 0.0;
        }
#pragma unroll
        for (int a = 0; a < kAhead; ++a)
#pragma unroll
            for (int q = 0; q < NQ; ++q) s[q] = add_(s[q], v[a][q]);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) scratch[threadIdx.x * NQ + q] = s[q];
    __syncthreads();
    if (threadIdx.x < 32) {
        double w[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) w[q] = 0.0;
#pragma unroll
        for (int i = 0; i < kBlock / 32; ++i)
#pragma unroll
            for (int q = 0; q < NQ; ++q) w[q] = add_(w[q], scratch[(threadIdx.x + 32 * i) * NQ + q]);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                w[q] = add_(w[q], __shfl_xor_sync(0xffffffffu, w[q], off));
        }
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) scratch[q] = w[q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) out[q] = scratch[q];
    __syncthreads();
}

// ------------------------------------------------------------- per-row math
// Gradient without its constant 1/eps term, the (G)LMO choice and the per-row
// terms of the FW gap, ||D_i||^2 and <D_i, LU_i>.
//   binary row  <=> every stored entry is exactly 0 or 1;  supp = {k : u_k > 0}
//   greedy:  active = !binary, s = lowest argmin of G' over supp (eq. eq:LMOpr)
//   full:    active = every row, s = lowest argmin of G' over all classes (Alg. 2)
//   inactive rows keep s = position of their 1.
// moved = the row has D_i != 0 (greedy: active; full: unless u_i is already e_s).
template <typename T, int KMAX>
__device__ __forceinline__ void row_eval(int K, const T (&u)[KMAX], const T (&lu)[KMAX], int fidc,
                                         T c2, T om, bool greedy, T (&G)[KMAX], int& s,
                                         bool& moved, T& gap, T& nD, T& tLU) {
    bool binary = true;
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
        if (k < K) binary = binary && (u[k] == T(0) || u[k] == T(1));
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < K) {
            T gk = fma_(-c2, u[k], lu[k]);
            if (fidc >= 0) gk = fma_(om, sub_(u[k], k == fidc ? T(1) : T(0)), gk);
            G[k] = gk;
        }
    }
    const bool active = greedy ? !binary : true;
    s = -1;
    T gs = T(0);
    if (active) {
        T best = inf_<T>();
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < K && (!greedy || u[k] > T(0)) && G[k] < best) {
                best = G[k];
                s = k;
            }
        gs = best;
        if (s < 0) {  // no finite candidate: keep the first admissible class, gap becomes NaN
#pragma unroll
            for (int k = KMAX - 1; k >= 0; --k)
                if (k < K && (!greedy || u[k] > T(0))) s = k;
            if (s < 0) s = 0;
            gs = CUDART_NAN_F;
        }
    } else {
#pragma unroll
        for (int k = KMAX - 1; k >= 0; --k)
            if (k < K && u[k] == T(1)) s = k;
        if (s < 0) s = 0;
    }
    bool at_vertex = binary;
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
        if (k == s) at_vertex = at_vertex && (u[k] == T(1));
    moved = active && !at_vertex;
    gap = T(0);
    nD = T(0);
    tLU = T(0);
    if (moved) {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k < K) {
                const T d = sub_(k == s ? T(1) : T(0), u[k]);
                gap = fma_(u[k], sub_(G[k], gs), gap);
                nD = fma_(d, d, nD);
                tLU = fma_(d, lu[k], tLU);
            }
        }
    }
}

enum PassAMode { MODE_STEP = 0, MODE_FLUSH = 1, MODE_GRAD = 2 };

template <typename T>
struct AccA {
    T g, nD, nW, tLU, act;
};

// Pass A over rows [r_begin, r_end) of one problem, one thread per row.
//  MODE_STEP:  apply the pending update (if upd), evaluate, store U, LU, choice.
//  MODE_FLUSH: apply the pending update only.
//  MODE_GRAD:  evaluate only; G' goes to Gout (SoA), choice to chout.
template <typename T, int KMAX, int MODE>
__device__ __forceinline__ void passA_rows(const ProbDesc& pd, int r_begin, int r_end, bool upd,
                                           T alpha, AccA<T>& acc, T* __restrict__ Gout,
                                           uint8_t* __restrict__ chout) {
    static_assert(MODE != MODE_STEP, "the step pass is passA_staged (it keeps cls4 current)");
    const int K = pd.K;
    const int64_t np = pd.npad;
    T* __restrict__ Ub = static_cast<T*>(pd.U);
    T* __restrict__ LUb = static_cast<T*>(pd.LU);
    const T* __restrict__ LSb = static_cast<const T*>(pd.LS);
    uint8_t* __restrict__ choice = pd.choice;
    const T c2 = c2_of<T>(pd);
    const T om = om_of<T>(pd);
    const T oma = sub_(T(1), alpha);
    const bool greedy = pd.oracle == 0;
    for (int r = r_begin + threadIdx.x; r < r_end; r += kBlock) {
        T u[KMAX], lu[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < K) {
                u[k] = ld_cg(Ub + k * np + r);
                lu[k] = ld_cg(LUb + k * np + r);
            }
        if (MODE != MODE_GRAD && upd) {
            const uint8_t sv = ld_cg(choice + r);
            const int sp = sv & 0x7f;
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) {
                    lu[k] = fma_(alpha, ld_cg(LSb + k * np + r), mul_(oma, lu[k]));
                    LUb[k * np + r] = lu[k];
                }
            if (sv & kActiveBit) {
#pragma unroll
                for (int k = 0; k < KMAX; ++k)
                    if (k < K) {
                        u[k] = (k == sp) ? fma_(oma, u[k], alpha) : mul_(oma, u[k]);
                        Ub[k * np + r] = u[k];
                    }
            }
        }
        if (MODE == MODE_FLUSH) continue;
        const int f = __ldg(pd.fid + r);
        T G[KMAX];
        int s;
        bool moved;
        T gap, nD, tLU;
        row_eval<T, KMAX>(K, u, lu, f, c2, om, greedy, G, s, moved, gap, nD, tLU);
        const uint8_t cv = uint8_t(s) | (moved ? kActiveBit : uint8_t(0));
        if (MODE == MODE_GRAD) {
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) Gout[k * np + r] = G[k];
            chout[r] = cv;
        } else {
            choice[r] = cv;
        }
        acc.g = add_(acc.g, gap);
        acc.nD = add_(acc.nD, nD);
        if (f >= 0) acc.nW = fma_(om, nD, acc.nW);
        acc.tLU = add_(acc.tLU, tLU);
        acc.act = add_(acc.act, moved ? T(1) : T(0));
    }
}

// ------------------------------------------------------------ scalar steps
// The problem's constants of the stop test and step rule.
struct StepCfg {
    double inv_eps, gap_tol;
    int tol_mode, max_iters, step_rule;
};

__device__ __forceinline__ StepCfg step_cfg(const ProbDesc& pd) {
    return StepCfg{pd.inv_eps, pd.gap_tol, pd.tol_mode, pd.max_iters, pd.step_rule};
}

static_assert(kAccCopies == 1, "warp_decide reads one accumulator copy");

// The step decision of one iteration, taken by one warp (all 32 lanes call
// it) from the iteration's totals S = (g, ||D||^2, sum w||D||^2, <D,LU>, |I|,
// <D,LS>) in accumulator bank `accb` and the inputs in[c]: the stop test of
// Alg. 3 step 4, then the curvature q = <D, H D> and the step (exact line
// search, eq. 10, or Armijo halving).
//
// Lane l loads word l of the bank; lanes 16..19 load in[c] and the error
// flag, so everything arrives in one round trip, and lane 2q turns quantity
// q into a double.  Spread this way the decision needs few registers per
// thread, which matters where it is fused into pass A.  With `commit` the
// warp writes the result into the state (each statistic from its lane, the
// rest from lane 0), in[c ^ 1] included; q and alpha keep their last values
// once done.  k_finish, pass A (fused) and the persistent kernel's last block
// all run this code, so their decisions agree bit for bit.
// Returns `done` in every lane; *alpha = the step.
__device__ __forceinline__ int warp_decide(const unsigned long long* accb, ProbState* st, int c,
                                           const StepCfg& cfg, bool commit, double* alpha) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned long long* inw = reinterpret_cast<const unsigned long long*>(&st->in[c]);
    unsigned long long w = 0ull;
    if (lane < kAccWords) w = __ldcg(accb + lane);
    else if (lane >= 16 && lane < 19) w = __ldcg(inw + (lane - 16));
    else if (lane == 19) w = static_cast<unsigned long long>(static_cast<unsigned>(__ldcg(&st->err)));
    // Q64.64 (lo word in lane 2q, hi in 2q+1) -> double
    const unsigned long long hw = __shfl_down_sync(full, w, 1);
    double Sq = double(static_cast<long long>(hw)) + ldexp(double(w), -64);
    if (__shfl_sync(full, w, kAccFlag) != 0ull && lane == 0) Sq = CUDART_NAN;
    const bool bad = (lane == 0 || lane == 2 || lane == 4 || lane == 6 || lane == 10) && !isfinite(Sq);
    const bool nonfinite = __any_sync(full, bad);
    const double g = __shfl_sync(full, Sq, 0);
    const int active = int(__shfl_sync(full, Sq, 8));
    const double qL = __shfl_sync(full, Sq, 10) - __shfl_sync(full, Sq, 6);   // <D, L D>
    const double q =
        qL + __shfl_sync(full, Sq, 4) - 2.0 * cfg.inv_eps * __shfl_sync(full, Sq, 2);  // <D, H D>
    const double E = __longlong_as_double(static_cast<long long>(__shfl_sync(full, w, 16)));
    const double g0in = __longlong_as_double(static_cast<long long>(__shfl_sync(full, w, 17)));
    const unsigned long long ig = __shfl_sync(full, w, 18);
    const int iter = int(static_cast<unsigned>(ig));
    const int g0_set = int(static_cast<unsigned>(ig >> 32));
    const int err = int(__shfl_sync(full, w, 19));
    const double g0 = g0_set ? g0in : g;
    int status = 2;  // FW_PENDING
    int done = 0;
    if (err) {
        status = -7;  // FW_ERR_TIMEOUT
        done = 1;
    } else if (nonfinite) {
        status = -6;  // FW_ERR_NUMERIC
        done = 1;
    } else if (active == 0 || g <= 0.0) {
        status = 0;
        done = 1;
    } else if (g <= (cfg.tol_mode ? cfg.gap_tol * g0 : cfg.gap_tol)) {
        status = 0;
        done = 1;
    } else if (iter >= cfg.max_iters) {
        status = 1;  // FW_NOT_CONVERGED
        done = 1;
    } else if (!isfinite(q)) {
        status = -6;
        done = 1;
    }
    double a = 1.0;
    if (!done && q > 0.0) {
        const double r = g / q;   // one division serves both rules
        if (cfg.step_rule == 0) {
            a = fmin(1.0, r);
        } else {
            // Armijo: largest 0.5^j with E(U) - E(U + a D) = a g - a^2 q / 2 >= 1e-6 a g,
            // i.e. a <= 2 (1 - 1e-6) g / q
            const double amax = 2.0 * (1.0 - 1e-6) * r;
            for (int j = 0; j < 1100 && a > amax; ++j) a *= 0.5;
        }
    }
    if (commit) {
        if (lane == 0) st->g = Sq;
        if (lane == 2) st->nD = Sq;
        if (lane == 4) st->nW = Sq;
        if (lane == 6) st->tLU = Sq;
        if (lane == 8) st->active = int(Sq);
        if (lane == 10) st->pLS = Sq;
        if (lane == 0) {
            st->g0 = g0;
            st->g0_set = 1;
            st->status = status;
            st->done = done;
            StepIn nx;
            nx.E = E;
            nx.g0 = g0;
            nx.iter = iter;
            nx.g0_set = 1;
            if (!done) {
                st->q = q;
                st->alpha = a;
                st->alpha_f = float(a);
                nx.E = E - a * g + 0.5 * a * a * q;
                nx.iter = iter + 1;
            }
            st->has_update = done ? 0 : 1;
            st->E = nx.E;
            st->iter = nx.iter;
            st->in[c ^ 1] = nx;
        }
    }
    *alpha = a;
    return done;
}

// k_finish and the persistent kernel's last block: one warp decides on bank
// `accb` (the totals of the iteration that just ended), clears it, commits,
// and advances the parity.  Returns done.
__device__ __forceinline__ int warp_finish(const ProbDesc& pd, ProbState* st,
                                           unsigned long long* accb) {
    const int c = __ldcg(&st->cur);
    double a;
    const int done = warp_decide(accb, st, c, step_cfg(pd), true, &a);
    if ((threadIdx.x & 31) < kAccWords) accb[threadIdx.x & 31] = 0ull;   // after its own load
    if ((threadIdx.x & 31) == 0) st->cur = c ^ 1;
    return done;
}

// Staged pass A over rows [r_begin, r_end) in 256-row sub-tiles.  For each
// sub-tile one thread issues bulk copies of its class columns of U, LU (and LS
// when a step is pending) into a stage buffer (T[3][KMAX][256]) completing on
// that buffer's mbarrier; with two stages the copies of sub-tile j+1 are in
// flight while sub-tile j is computed.  Each thread updates and evaluates its
// row from shared memory in two sweeps (argmin, then the gap terms), with the
// operation sequence of passA_rows / row_eval, so results are bitwise the
// same.  Returns false when a copy wait ran out of its bound (the copies are
// then waited for once more).
// Stages of the pass-A staging buffer that fit next to the rest (2 unless one
// stage is larger than 100 KB, e.g. FP64 with K > 16).
template <typename T, int KMAX>
__host__ __device__ constexpr int max_stages() {
    return 2 * 3 * kBlock * KMAX * int(sizeof(T)) <= 200 * 1024 ? 2 : 1;
}

template <typename T, int KMAX>
__device__ __forceinline__ void stage_issue(const ProbDesc& pd, int base, int rows, bool upd,
                                            T* stage, uint64_t* bar) {
    constexpr int kVec = 16 / int(sizeof(T));
    const int K = pd.K;
    const int64_t np = pd.npad;
    // whole 16-byte units; the extra elements lie inside the npad-long columns
    const uint32_t seg = uint32_t((rows + kVec - 1) / kVec * kVec) * uint32_t(sizeof(T));
    fence_proxy_async();
    mbar_expect_tx(bar, seg * uint32_t(K) * (upd ? 3u : 2u));
    const T* Ub = static_cast<const T*>(pd.U);
    const T* LUb = static_cast<const T*>(pd.LU);
    const T* LSb = static_cast<const T*>(pd.LS);
    for (int k = 0; k < K; ++k) {
        bulk_g2s(stage + k * kBlock, Ub + k * np + base, seg, bar);
        bulk_g2s(stage + (KMAX + k) * kBlock, LUb + k * np + base, seg, bar);
        if (upd) bulk_g2s(stage + (2 * KMAX + k) * kBlock, LSb + k * np + base, seg, bar);
    }
}

// Pass A with the previous iteration's step decision fused in (ProbState):
// when `fin`, the block decides on accumulator bank `cur` and in[cur] while
// its first copies are in flight, and block 0 (`commit`) writes the result.
struct FuseCtl {
    bool fin;
    const int* stop;        // shared memory: the decision stops the solve
    const double* alpha;    // shared memory: the decided step
};

// Outcomes of passA_staged.
enum { kPassOk = 0, kPassTimeout = 1, kPassStopped = 2 };

// EXACT: the problem has exactly KMAX classes, so every per-class guard of
// the unrolled loops is known at compile time.  With fc.fin, `upd` must be
// true and `alpha` is replaced by the decided step; if the decision stops the
// solve, the block waits for its copies and returns kPassStopped without
// touching the iterate.
template <typename T, int KMAX, bool EXACT = false>
__device__ __forceinline__ int passA_staged(const ProbDesc& pd, int r_begin, int r_end, bool upd,
                                            T alpha, const FuseCtl& fc, AccA<T>& acc, T* stage,
                                            int nstages, uint64_t* bars, uint32_t& phases) {
    const int K = EXACT ? KMAX : pd.K;
    const int64_t np = pd.npad;
    T* __restrict__ Ub = static_cast<T*>(pd.U);
    T* __restrict__ LUb = static_cast<T*>(pd.LU);
    const T c2 = c2_of<T>(pd);
    const T om = om_of<T>(pd);
    T oma = sub_(T(1), alpha);
    const bool greedy = pd.oracle == 0;
    const int stage_elems = 3 * KMAX * kBlock;
    int rc = kPassOk;
    // with fc.fin the caller has issued the first sub-tile's copies and taken
    // the decision (s_stop, s_alpha) before calling
    if (!fc.fin && threadIdx.x == 0 && r_begin < r_end)
        stage_issue<T, KMAX>(pd, r_begin, min(kBlock, r_end - r_begin), upd, stage, &bars[0]);
    int j = 0;
    for (int base = r_begin; base < r_end; base += kBlock, ++j) {
        const int buf = nstages > 1 ? (j & 1) : 0;
        // one buffer: this sub-tile's copy is issued once the previous one has
        // been consumed (the __syncthreads at the end of the last iteration)
        if (nstages == 1 && j > 0 && threadIdx.x == 0)
            stage_issue<T, KMAX>(pd, base, min(kBlock, r_end - base), upd, stage, &bars[0]);
        const int rows = min(kBlock, r_end - base);
        T* sU = stage + buf * stage_elems;
        T* sL = sU + KMAX * kBlock;
        T* sS = sU + 2 * KMAX * kBlock;
        const int t = threadIdx.x;
        const int r = base + t;
        // per-row bytes are loaded before the wait so their latency overlaps the copies
        const uint8_t sv = (t < rows && upd) ? ld_cg(pd.choice + r) : uint8_t(0);
        const int f = t < rows ? int(__ldg(pd.fid + r)) : -1;
        int my_cls = 0;
        if (nstages > 1 && threadIdx.x == 0 && base + kBlock < r_end) {
            const int nb = base + kBlock;   // prefetch the next sub-tile into the other buffer
            stage_issue<T, KMAX>(pd, nb, min(kBlock, r_end - nb), upd,
                                 stage + (buf ^ 1) * stage_elems, &bars[buf ^ 1]);
        }
        const uint32_t par = (phases >> buf) & 1u;
        const bool got = mbar_wait(&bars[buf], par);
        if (__syncthreads_or(!got)) {
            // a copy did not arrive in time: wait (bounded) for the copies still
            // in flight into this block's buffers, then leave the tile; the
            // caller raises the problem's error flag
            rc = kPassTimeout;
            if (got || mbar_wait(&bars[buf], par)) phases ^= 1u << buf;
            if (nstages > 1 && base + kBlock < r_end &&
                mbar_wait(&bars[buf ^ 1], (phases >> (buf ^ 1)) & 1u))
                phases ^= 1u << (buf ^ 1);
            __syncthreads();
            break;
        }
        phases ^= 1u << buf;
        if (fc.fin && j == 0) {
            if (*fc.stop) {   // stopped: nothing is applied; let the prefetch land
                if (nstages > 1 && base + kBlock < r_end &&
                    mbar_wait(&bars[buf ^ 1], (phases >> (buf ^ 1)) & 1u))
                    phases ^= 1u << (buf ^ 1);
                return kPassStopped;
            }
            alpha = T(*fc.alpha);
            oma = sub_(T(1), alpha);
        }
        if (t < rows) {
            const int sp = sv & 0x7f;
            const bool mv = (sv & kActiveBit) != 0;
            bool binary = true;
            T best = inf_<T>();
            int s = -1, first_adm = -1, first_one = -1;
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                if (k < K) {
                    T u = sU[k * kBlock + t];
                    T lu = sL[k * kBlock + t];
                    if (upd) {
                        lu = fma_(alpha, sS[k * kBlock + t], mul_(oma, lu));
                        LUb[k * np + r] = lu;
                        sL[k * kBlock + t] = lu;
                        if (mv) {
                            u = (k == sp) ? fma_(oma, u, alpha) : mul_(oma, u);
                            Ub[k * np + r] = u;
                            sU[k * kBlock + t] = u;
                        }
                    }
                    binary = binary && (u == T(0) || u == T(1));
                    if (first_one < 0 && u == T(1)) first_one = k;
                    T gk = fma_(-c2, u, lu);
                    if (f >= 0) gk = fma_(om, sub_(u, k == f ? T(1) : T(0)), gk);
                    const bool adm = !greedy || u > T(0);
                    if (adm && first_adm < 0) first_adm = k;
                    if (adm && gk < best) {
                        best = gk;
                        s = k;
                    }
                }
            }
            const bool active = greedy ? !binary : true;
            T gs = best;
            if (active) {
                if (s < 0) {   // no finite candidate: the gap becomes NaN
                    s = first_adm < 0 ? 0 : first_adm;
                    gs = CUDART_NAN_F;
                }
            } else {
                s = first_one < 0 ? 0 : first_one;
            }
            const bool at_vertex = binary && sU[s * kBlock + t] == T(1);
            const bool moved = active && !at_vertex;
            T gap = T(0), nD = T(0), tLU = T(0);
            if (moved) {
#pragma unroll
                for (int k = 0; k < KMAX; ++k) {
                    if (k < K) {
                        const T u = sU[k * kBlock + t];
                        const T lu = sL[k * kBlock + t];
                        T gk = fma_(-c2, u, lu);
                        if (f >= 0) gk = fma_(om, sub_(u, k == f ? T(1) : T(0)), gk);
                        const T d = sub_(k == s ? T(1) : T(0), u);
                        gap = fma_(u, sub_(gk, gs), gap);
                        nD = fma_(d, d, nD);
                        tLU = fma_(d, lu, tLU);
                    }
                }
            }
            acc.g = add_(acc.g, gap);
            acc.nD = add_(acc.nD, nD);
            if (f >= 0) acc.nW = fma_(om, nD, acc.nW);
            acc.tLU = add_(acc.tLU, tLU);
            acc.act = add_(acc.act, moved ? T(1) : T(0));
            pd.choice[r] = uint8_t(s) | (moved ? kActiveBit : uint8_t(0));
            my_cls = s;
        }
        if (pd.cls4) {   // rows 2m, 2m+1 are adjacent lanes (base is a multiple of 256)
            const int hi = __shfl_down_sync(0xffffffffu, my_cls, 1);
            if ((t & 1) == 0 && t < rows) pd.cls4[r >> 1] = uint8_t(my_cls | (hi << 4));
        }
        __syncthreads();
    }
    return rc;
}

// Stage 1 of the sparse passes: for each row of a 256-row sub-tile, `L` lanes
// walk the padded CSR row in 4-entry chunks and accumulate into per-lane bins
// in shared memory (`sm_lane`, class-major: class k of thread slot t at
// k * S + t, S the block's thread count, so the 32 lanes of a warp always hit
// 32 different banks whatever classes they update); the lanes of a row then
// add their slots in lane order into `sm_row` (class k of row slot r at
// k * S + r).  Warp w handles
// exactly rows 32w .. 32w+31 of the sub-tile (32/L rows at a time), so the
// row sums never leave the warp: __syncwarp orders them, and the caller needs
// no block barrier before thread t reads sm_row[t].
//   ONEHOT: bin[s_j] += w_ij            (pass B: row i of W^ S)
//   else:   bin[k]  += w_ij * X[k][j]   (SpMM: row i of W^ X)
// A lane keeps two chunks (8 entries) in flight: their column, weight and
// gather loads are issued before the bins are updated, in entry order.
// RO: gathers may use the read-only path (the gathered array is not written
// during the launch); otherwise plain loads, ordered by the caller's fences.
template <bool RO, typename V>
__device__ __forceinline__ V ld_gather(const V* p) {
    if constexpr (RO) return __ldg(p);
    else return *p;
}

// Value of U_hat (Sec. 2, the start point U_0 of Sec. 5.1) at class k of a row
// with fidelity class f: e_f for a fidelity row, 1/K everywhere otherwise --
// the same expression k_reinit stores, so products with it are bitwise those
// of the stored U_0.
template <typename T>
__device__ __forceinline__ T uhat_val(int f, int k, T unif) {
    return f >= 0 ? (k == f ? T(1) : T(0)) : unif;
}

// Gather sources of csr_bins: the one-hot S of the choice bytes (pass B), a
// dense class-major X (SpMM), or U_hat formed from the fidelity bytes (OSFW).
enum { kSrcOneHot = 0, kSrcDense = 1, kSrcUhat = 2 };

// LC: lanes per row known at compile time (0: the runtime pd.lanes).  With one
// lane each thread's bins are its own row's sums, so the lane-sum stage is
// skipped and the caller reads sm_lane (a sum over one lane is the value
// itself, so nothing changes).  EXACT: the problem has exactly KMAX classes.
// TAB (one-hot only): the 4-bit class pairs are read from a copy of pd.cls4
// in shared memory (`tab`) instead of being gathered from global memory.
template <typename T, typename WT, int KMAX, int SRC, bool RO, int LC = 0, bool EXACT = false,
          bool TAB = false, int S = kBlock>
__device__ __forceinline__ void csr_bins(const ProbDesc& pd, const T* __restrict__ X, int base,
                                         int r_end, T* __restrict__ sm_lane,
                                         T* __restrict__ sm_row,
                                         const uint8_t* __restrict__ tab = nullptr) {
    constexpr bool ONEHOT = SRC == kSrcOneHot;
    const int K = EXACT ? KMAX : pd.K;
    const int L = LC ? LC : pd.lanes;
    const int64_t np = pd.npad;
    const int32_t* __restrict__ rp = pd.rp;
    const int32_t* __restrict__ col = pd.col;
    const int16_t* __restrict__ col16 = reinterpret_cast<const int16_t*>(pd.col);
    const bool c16 = pd.col16 != 0;   // uniform over the launch's problem
    const WT* __restrict__ val = static_cast<const WT*>(pd.val);
    const uint8_t* __restrict__ choice = pd.choice;
    const int tid = threadIdx.x;
    const int lane = tid & (L - 1);
    const int grp = tid / L;                    // lane group: its lanes are adjacent threads
    const int wrow = (tid & ~31) + (tid & 31) / L;
    T* my = sm_lane + tid;   // my[k * S]: this thread's bin of class k
    for (int j = 0; j < L; ++j) {
        const int rl = wrow + (32 / L) * j;     // a row of this warp's 32
        const int r = base + rl;
        T acc[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) acc[k] = T(0);
        if (ONEHOT) {
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) my[k * S] = T(0);
        }
        if (r < r_end) {
            const int e0 = __ldg(rp + r);
            const int e1 = __ldg(rp + r + 1);
            for (int e = e0 + 4 * lane; e < e1; e += 8 * L) {
                const int e2 = e + 4 * L;
                const bool two = e2 < e1;
                int cc[8];
                T v[8];
                if (c16) {
                    // four 16-bit offsets j - r in 8 bytes, sign-extended
                    const uint2 c = ld_stream(reinterpret_cast<const uint2*>(col16 + e));
                    cc[0] = r + (int(c.x << 16) >> 16); cc[1] = r + (int(c.x) >> 16);
                    cc[2] = r + (int(c.y << 16) >> 16); cc[3] = r + (int(c.y) >> 16);
                    if (two) {
                        const uint2 d = ld_stream(reinterpret_cast<const uint2*>(col16 + e2));
                        cc[4] = r + (int(d.x << 16) >> 16); cc[5] = r + (int(d.x) >> 16);
                        cc[6] = r + (int(d.y << 16) >> 16); cc[7] = r + (int(d.y) >> 16);
                    } else {
                        cc[4] = cc[5] = cc[6] = cc[7] = r;
                    }
                } else {
                    const int4 c = ld_stream(reinterpret_cast<const int4*>(col + e));
                    cc[0] = c.x; cc[1] = c.y; cc[2] = c.z; cc[3] = c.w;
                    if (two) {
                        const int4 d = ld_stream(reinterpret_cast<const int4*>(col + e2));
                        cc[4] = d.x; cc[5] = d.y; cc[6] = d.z; cc[7] = d.w;
                    } else {
                        cc[4] = cc[5] = cc[6] = cc[7] = r;
                    }
                }
                if constexpr (sizeof(WT) == 2) {
                    float vf[4];
                    ld_w4(val + e, vf);
#pragma unroll
                    for (int t = 0; t < 4; ++t) v[t] = vf[t];
                    if (two) {
                        ld_w4(val + e2, vf);
#pragma unroll
                        for (int t = 0; t < 4; ++t) v[4 + t] = vf[t];
                    }
                } else {
                    T w4[4];
                    ld_w4(val + e, w4);
#pragma unroll
                    for (int t = 0; t < 4; ++t) v[t] = w4[t];
                    if (two) {
                        ld_w4(val + e2, w4);
#pragma unroll
                        for (int t = 0; t < 4; ++t) v[4 + t] = w4[t];
                    }
                }
                const int nt = two ? 8 : 4;
                if (ONEHOT) {
                    int sj[8];
                    if constexpr (TAB) {
                        static_assert(KMAX <= 16, "the class table holds 4-bit classes");
                        const uint32_t tb = smem_u32(tab);
#pragma unroll
                        for (int t = 0; t < 8; ++t)
                            sj[t] = (ld_shared_u8(tb + uint32_t(cc[t] >> 1)) >> ((cc[t] & 1) << 2)) & 15;
                    } else if constexpr (KMAX <= 16 && RO) {
                        // 4-bit classes: half the gathered footprint, so more of it
                        // stays in L1.  Only the two-kernel path (RO) keeps them;
                        // the persistent kernel gathers the class bytes.
                        // the nibble selectors of the 8 gathers share one register
                        uint32_t odd = 0;
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            sj[t] = ld_gather<RO>(pd.cls4 + (cc[t] >> 1));
                            odd |= uint32_t(cc[t] & 1) << (2 + 4 * t);
                        }
#pragma unroll
                        for (int t = 0; t < 8; ++t) sj[t] = (sj[t] >> ((odd >> 4 * t) & 4)) & 15;
                    } else {
#pragma unroll
                        for (int t = 0; t < 8; ++t) sj[t] = ld_gather<RO>(choice + cc[t]) & 0x7f;
                    }
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        if (t < nt) my[sj[t] * S] = add_(my[sj[t] * S], v[t]);
                } else if constexpr (SRC == kSrcDense) {
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        if (t < nt) {
#pragma unroll
                            for (int k = 0; k < KMAX; ++k)
                                if (k < K)
                                    acc[k] = fma_(v[t], ld_gather<RO>(X + k * np + cc[t]), acc[k]);
                        }
                    }
                } else {
                    // the SpMM of U_hat, entry by entry: an unlabelled neighbour
                    // adds v/K to every class (one fma each), a labelled one
                    // adds v to its class only -- fma(v, 1, a) = a + v and
                    // fma(v, 0, a) = a exactly, so the sums are bitwise those
                    // of fma(v, U_hat[j][k], a) over every class
                    const T unif = T(1) / T(K);
                    int fj[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) fj[t] = __ldg(pd.fid + cc[t]);
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        if (t < nt) {
                            if (fj[t] < 0) {
#pragma unroll
                                for (int k = 0; k < KMAX; ++k)
                                    if (k < K) acc[k] = fma_(v[t], unif, acc[k]);
                            } else {
#pragma unroll
                                for (int k = 0; k < KMAX; ++k)
                                    if (k == fj[t]) acc[k] = add_(acc[k], v[t]);
                            }
                        }
                    }
                }
            }
        }
        if (!ONEHOT) {
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) my[k * S] = acc[k];
        }
        if constexpr (LC != 1) {
            __syncwarp();
            for (int k = lane; k < K; k += L) {
                T s = T(0);
                for (int l2 = 0; l2 < L; ++l2) s = add_(s, sm_lane[k * S + grp * L + l2]);
                sm_row[k * S + rl] = s;
            }
            __syncwarp();
        }
    }
}

// Shared memory pass B needs beyond its bins (sm_lane, sm_row): the rows' U
// values and choice bytes, prefetched while the CSR rows are walked.
template <typename T, int KMAX>
__host__ __device__ constexpr size_t passB_prefetch_bytes() {
    return size_t(kBlock) * KMAX * sizeof(T) + kBlock;
}
// Forms that prefetch: one lane per row with at most 8 classes (pixel grids
// and other low-degree graphs, whose U streams from HBM; the extra shared
// memory leaves their occupancy unchanged), and the persistent kernel (!RO).
// The 2- and 4-lane forms for more classes keep their bins-only footprint,
// which their one-wave occupancy and L1 class gathers need.
template <int KMAX, bool RO, int LC>
__host__ __device__ constexpr bool passB_prefetches() {
    return (LC == 1 && KMAX <= 8) || !RO;
}

// Pass B output of row r from its row sums rs[k * S], k < K (bins of the
// one-hot product): LS_r = [k = s_r] d_r - rs[k], and, when the row moved
// (active bit of its choice byte sv), <D_r, LS_r> with D_r = e_{s_r} - U_r
// added to accq.  With PF the row's U values are read from shared memory
// (uPF[k * kBlock]), else from global memory.
template <typename T, int KMAX, bool EXACT, bool PF, int S = kBlock>
__device__ __forceinline__ void passB_row_out(const ProbDesc& pd, int r, uint8_t sv,
                                              const T* rs, const T* uPF, T& accq) {
    const int K = EXACT ? KMAX : pd.K;
    const int64_t np = pd.npad;
    const T* __restrict__ Ub = static_cast<const T*>(pd.U);
    T* __restrict__ LSb = static_cast<T*>(pd.LS);
    const T* __restrict__ diag = static_cast<const T*>(pd.diag);
    const int si = sv & 0x7f;
    const bool act = (sv & kActiveBit) != 0;
    const T dg = pd.comb ? diag[r] : T(1);
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
        if (k < K) {
            const T b = rs[k * S];
            LSb[k * np + r] = (k == si) ? sub_(dg, b) : -b;
        }
    if (act) {
        // all K loads first (one round trip), then <D_i, LS_i>; LS_i is
        // re-formed from the row sums rather than kept in registers
        T u[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < K) u[k] = PF ? uPF[k * kBlock] : ld_cg(Ub + k * np + r);
        T qi = T(0);
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < K) {
                const T b = rs[k * S];
                const T ls = (k == si) ? sub_(dg, b) : -b;
                qi = fma_(sub_(k == si ? T(1) : T(0), u[k]), ls, qi);
            }
        accq = add_(accq, qi);
    }
}

// Pass B over rows [r_begin, r_end): LS = L S (one-hot S) and sum_i <D_i, LS_i>.
// sm_pf: passB_prefetch_bytes() of shared memory, 16-byte aligned.  Each warp
// copies its 32 rows' U values (class-major, 128 bytes per class) and choice
// bytes into it with asynchronous 16-byte copies before it walks their CSR
// rows, so those loads do not add a memory latency after the walk.
template <typename T, typename WT, int KMAX, bool RO, int LC = 0, bool EXACT = false>
__device__ __forceinline__ void passB_rows(const ProbDesc& pd, int r_begin, int r_end, T& accq,
                                           T* sm_lane, T* sm_row_in, T* sm_pf) {
    constexpr int kV = 16 / int(sizeof(T));   // values per 16-byte copy
    constexpr int kC = 32 / kV;               // copies per class for a warp's 32 rows
    const int K = EXACT ? KMAX : pd.K;
    T* const sm_row = LC == 1 ? sm_lane : sm_row_in;   // one lane: its bins are the row sums
    const T* __restrict__ Ub = static_cast<const T*>(pd.U);
    const int64_t np = pd.npad;
    constexpr bool PF = passB_prefetches<KMAX, RO, LC>();
    T* const sU = sm_pf;
    uint8_t* const sC = reinterpret_cast<uint8_t*>(sm_pf + KMAX * kBlock);
    const int lane = threadIdx.x & 31, w0 = threadIdx.x & ~31;
    for (int base = r_begin; base < r_end; base += kBlock) {
        const int bw = base + w0;   // the warp's first row; U and choice are padded to 32 rows
        if (PF && bw < r_end) {
            for (int c = lane; c < K * kC; c += 32) {
                const int k = c / kC, q = c - k * kC;
                cp_async16(sU + k * kBlock + w0 + q * kV, Ub + k * np + bw + q * kV);
            }
            if (lane < 2) cp_async16(sC + w0 + 16 * lane, pd.choice + bw + 16 * lane);
        }
        if (PF) cp_async_commit();
        csr_bins<T, WT, KMAX, kSrcOneHot, RO, LC, EXACT>(pd, nullptr, base, r_end, sm_lane, sm_row);
        if (PF) {
            cp_async_wait_all();
            __syncwarp();   // the warp's copies (and its sm_row sums) are visible to all its lanes
        }
        const int r = base + threadIdx.x;
        if (r < r_end)
            passB_row_out<T, KMAX, EXACT, PF>(pd, r, PF ? sC[threadIdx.x] : ld_cg(pd.choice + r),
                                              sm_row + threadIdx.x,
                                              PF ? sU + threadIdx.x : nullptr, accq);
        __syncwarp();   // the warp's bins are reused by the next sub-tile
    }
}

// ------------------------------------- pass B with a shared class table
// For graphs whose columns scatter over the whole problem (random-graph
// models, k-NN graphs), pass B's 4-bit class gathers miss L1 about half the
// time and their wavefronts fill the L1 data path.  When the problem's class
// array fits in shared memory next to the bins, one 1024-thread block per SM
// copies it once and its 32 warps walk the block's row tiles 32 rows at a
// time, reading classes from shared memory.  Tile totals are formed exactly
// as passB_rows + block_accumulate form them, so results are bitwise those
// of the direct kernels.
constexpr int kTabThreads = 1024;
constexpr int kTabMaxTiles = 16;   // tiles of one block (the grid is sized for it)
constexpr int kTabSmemMax = 230400;   // dynamic shared memory of one block (227 KB less the static)

// Shared memory of the bins of kTabThreads threads (the row sums as well
// unless one lane per row) and of the class table.
template <typename T, int KMAX>
__host__ __device__ constexpr size_t tab_bins_bytes(int lanes) {
    return size_t(lanes == 1 ? 1 : 2) * kTabThreads * (KMAX | 1) * sizeof(T);
}
__host__ __device__ inline uint32_t tab_bytes(int n) {
    return uint32_t((int64_t(n + 1) / 2 + 15) / 16 * 16);
}

// One 32-row unit of pass B by the calling warp: rows row0 .. row0 + 31 of a
// 256-row tile whose rows end at r_end.  Lane l takes row row0 + l, the row
// that lane l of the same warp position takes in passB_rows, and the row
// arithmetic is the same, so the returned value (the lane's <D_i, LS_i>, or 0)
// is the one passB_rows accumulates.  sm_lane / sm_row: bins of the whole
// block (kTabThreads slots); tab: the class table in shared memory.
template <typename T, typename WT, int KMAX, int LC, bool EXACT>
__device__ __forceinline__ T passB_unit(const ProbDesc& pd, int row0, int r_end, T* sm_lane,
                                        T* sm_row_in, const uint8_t* tab) {
    T* const sm_row = LC == 1 ? sm_lane : sm_row_in;
    const int w0 = threadIdx.x & ~31;
    // csr_bins places the warp's rows at base + (its thread slots)
    csr_bins<T, WT, KMAX, kSrcOneHot, true, LC, EXACT, true, kTabThreads>(
        pd, nullptr, row0 - w0, r_end, sm_lane, sm_row, tab);
    T accq = T(0);
    const int r = row0 + (threadIdx.x & 31);
    if (r < r_end)
        passB_row_out<T, KMAX, EXACT, false, kTabThreads>(pd, r, ld_cg(pd.choice + r),
                                                          sm_row + threadIdx.x, nullptr, accq);
    __syncwarp();   // the warp's bins are reused by its next unit
    return accq;
}

// OUT = L X for rows [r_begin, r_end) (SoA in and out; OUT may not alias X).
template <typename T, typename WT, int KMAX, int SRC = kSrcDense>
__device__ __forceinline__ void spmm_rows(const ProbDesc& pd, const T* __restrict__ X,
                                          T* __restrict__ OUT, int r_begin, int r_end, T* sm_lane,
                                          T* sm_row) {
    const int K = pd.K;
    const int64_t np = pd.npad;
    const T* __restrict__ diag = static_cast<const T*>(pd.diag);
    for (int base = r_begin; base < r_end; base += kBlock) {
        // X == U_hat (the stored U_0): its off-diagonal product comes from the
        // fidelity bytes, bitwise the dense product (see csr_bins)
        csr_bins<T, WT, KMAX, SRC, true>(pd, SRC == kSrcDense ? X : nullptr, base, r_end, sm_lane,
                                         sm_row);
        const int r = base + threadIdx.x;
        if (r < r_end) {
            const T dg = pd.comb ? diag[r] : T(1);
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K)
                    OUT[k * np + r] = sub_(mul_(dg, ld_cg(X + k * np + r)),
                                           sm_row[k * kBlock + threadIdx.x]);
        }
        __syncwarp();
    }
}

// One-Shot Frank-Wolfe (Alg. 4) for rows [r_begin, r_end): U_1 = GLMO(grad
// E(U_0)) at U_0 = U_hat, so label_i = s_i.  L U_hat is formed in the CSR pass
// from the fidelity bytes (the SpMM of the stored U_0, same operation order),
// and G', the binary/support tests and the argmin are those of pass A at U_0,
// so s_i is bitwise the choice the iteration makes at U_0.
template <typename T, typename WT, int KMAX>
__device__ __forceinline__ void osfw_rows(const ProbDesc& pd, int32_t* __restrict__ labels,
                                          int r_begin, int r_end, T* sm_lane, T* sm_row) {
    const int K = pd.K;
    const T* __restrict__ diag = static_cast<const T*>(pd.diag);
    const T c2 = c2_of<T>(pd);
    const T om = om_of<T>(pd);
    const T unif = T(1) / T(K);
    const bool greedy = pd.oracle == 0;
    for (int base = r_begin; base < r_end; base += kBlock) {
        csr_bins<T, WT, KMAX, kSrcUhat, true>(pd, nullptr, base, r_end, sm_lane, sm_row);
        const int r = base + threadIdx.x;
        if (r < r_end) {
            const int f = __ldg(pd.fid + r);
            const T dg = pd.comb ? diag[r] : T(1);
            bool binary = true;
            T best = inf_<T>();
            int s = -1, first_adm = -1, first_one = -1;
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) {
                    const T u = uhat_val<T>(f, k, unif);
                    const T lu = sub_(mul_(dg, u), sm_row[k * kBlock + threadIdx.x]);
                    binary = binary && (u == T(0) || u == T(1));
                    if (first_one < 0 && u == T(1)) first_one = k;
                    T gk = fma_(-c2, u, lu);
                    if (f >= 0) gk = fma_(om, sub_(u, k == f ? T(1) : T(0)), gk);
                    const bool adm = !greedy || u > T(0);
                    if (adm && first_adm < 0) first_adm = k;
                    if (adm && gk < best) {
                        best = gk;
                        s = k;
                    }
                }
            const bool active = greedy ? !binary : true;
            if (active) {
                if (s < 0) s = first_adm < 0 ? 0 : first_adm;
            } else {
                s = first_one < 0 ? 0 : first_one;
            }
            labels[r] = s;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------- row tiles
// One row tile of pass A with its block reduction; the last tile of the
// problem to finish runs the stop test.  `ndone` (nullable) counts problems
// that stop in this pass.  Every thread of the block must call it.
template <typename T, int KMAX, bool EXACT = false>
__device__ __forceinline__ void tile_A(const ProbDesc& pd, ProbState* st, int tile, bool upd,
                                       T alpha, const FuseCtl& fc, unsigned long long* accb,
                                       T* stage, int nstages, uint64_t* bars, uint32_t& phases) {
    const int r0 = tile * pd.tile_rows;
    const int r1 = min(pd.n, r0 + pd.tile_rows);
    AccA<T> acc{T(0), T(0), T(0), T(0), T(0)};
    const int rc =
        passA_staged<T, KMAX, EXACT>(pd, r0, r1, upd, alpha, fc, acc, stage, nstages, bars, phases);
    if (rc == kPassStopped) return;
    if (rc == kPassTimeout && threadIdx.x == 0) atomicExch(&st->err, 1);
    const T v[kNumA] = {acc.g, acc.nD, acc.nW, acc.tLU, acc.act};
    block_accumulate<T, kNumA>(v, accb, 0, tile % kAccCopies);
}

// One row tile of pass B, accumulating into bank `accb`.  With LAST, the last
// tile of the problem to finish takes the step decision on that bank
// (persistent kernel); otherwise k_finish or the next pass A does.  `ndone`
// (nullable) counts problems that stop.
template <typename T, typename WT, int KMAX, bool RO, bool LAST, int LC = 0,
          bool EXACT = false>
__device__ __forceinline__ void tile_B(const ProbDesc& pd, ProbState* st, int tile, T* sm_lane,
                                       T* sm_row, T* sm_pf, unsigned long long* accb,
                                       uint32_t* ndone) {
    const int r0 = tile * pd.tile_rows;
    const int r1 = min(pd.n, r0 + pd.tile_rows);
    T accq = T(0);
    passB_rows<T, WT, KMAX, RO, LC, EXACT>(pd, r0, r1, accq, sm_lane, sm_row, sm_pf);
    const T v[kNumB] = {accq};
    block_accumulate<T, kNumB>(v, accb, kNumA, tile % kAccCopies);
    if (LAST && last_to_arrive(&st->cnt, pd.ntiles) && threadIdx.x < 32) {
        const int done = warp_finish(pd, st, accb);
        if (threadIdx.x == 0) {
            st->cnt = 0;
            if (ndone && done) atomicAdd(ndone, 1u);
        }
    }
}

}  // namespace fw
