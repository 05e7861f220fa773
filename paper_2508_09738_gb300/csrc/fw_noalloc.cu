// fw_energy_noalloc: the objective E(U) -- the Laplacian quadratic form
// 1/2 <U, L U>, plus the penalty (1/eps) sum u (1 - u), plus the fidelity
// term 1/2 sum_i omega_i ||u_hat_i - u_i||^2 -- of a graph and an iterate
// that live in the caller's device memory, with no device allocation by the
// call.  The paper has no counterpart to this entry point: it is a service
// of the library.
//
// This is the allocation-free variant of the handle's objective evaluation
// (k_objective, which takes its fresh L U product and its partial sums from
// memory owned by a handle).  Here the only scratch is the file-scope array
// g_noalloc_scratch below: FW_NOALLOC_MAX_N degrees (FP64) plus 256 bytes of
// accumulator words.  Callers that cannot allocate are the reason it exists:
//  * a process whose device memory is already held by another allocator
//    (a serving framework's caching allocator that reserved the free HBM),
//    where cudaMalloc would fail even though the evaluation needs little;
//  * a latency-bound loop that must not call cudaMalloc / cudaFree, which
//    may synchronise the device.
// Nothing here calls cudaMalloc, cudaMallocAsync, cudaFree or any library
// routine that allocates device memory.
//
// Set-up: the first call on each device, with that device current, looks the
// scratch array up with cudaGetSymbolAddress (which may load the module's
// device data) and caches the address together with the identity of the
// current CUDA context.  A later call in another context of that device (for
// instance after cudaDeviceReset) looks the address up again.  Make the first
// call on a device before any stream capture.
//
// Calls share the one scratch array of their device: two calls that overlap
// in time on the same device (from two host threads, or on two streams
// without an ordering between them) race on it and may return wrong values.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "fw_device.cuh"
#include "fw_internal.h"

namespace fw {
namespace {

constexpr int64_t kNaMaxN = FW_NOALLOC_MAX_N;
constexpr int kNaErrWord = kAccWords;           // graph / label error bits
constexpr int kNaAccWords = 32;                 // 256 bytes of accumulator words
static_assert(kNaErrWord < kNaAccWords, "accumulators exceed the scratch words");
constexpr size_t kNaScratchBytes = size_t(kNaAccWords) * 8 + size_t(kNaMaxN) * 8;
constexpr int kNaMaxBlocks = 1024;              // < 2^11 block totals (fx_add range)
constexpr int kNaMaxDevices = 64;

// error bits of the graph / label word
constexpr unsigned long long kNaBadRowPtr = 1, kNaBadCol = 2, kNaIsolated = 4, kNaBadLabel = 8;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

// d_i = sum_j w_ij in CSR order (FP64).  Rows with an out-of-range extent or
// column, or with no positive degree, raise an error bit; nothing outside
// [0, nnz) or [0, n) is read.
__global__ void __launch_bounds__(kBlock)
k_na_degrees(int64_t n, int64_t nnz, const int32_t* __restrict__ rp,
             const int32_t* __restrict__ col, const double* __restrict__ w,
             double* __restrict__ deg, unsigned long long* acc) {
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    for (int64_t i = blockIdx.x * int64_t(kBlock) + threadIdx.x; i < n; i += stride) {
        const int64_t e0 = rp[i], e1 = rp[i + 1];
        double d = 0.0;
        if (e0 < 0 || e1 > nnz || e1 < e0) {
            atomicOr(&acc[kNaErrWord], kNaBadRowPtr);
        } else {
            for (int64_t e = e0; e < e1; ++e) {
                const int32_t j = col[e];
                if (j < 0 || j >= n) {
                    atomicOr(&acc[kNaErrWord], kNaBadCol);
                    continue;
                }
                d += w[e];
            }
            if (!(d > 0.0)) atomicOr(&acc[kNaErrWord], kNaIsolated);
        }
        deg[i] = d;
    }
}

// Per row i (FP64): 1/2 sum_k u_ik (L u)_ik + 1/eps sum_k u_ik (1 - u_ik)
// + 1/2 omega_i sum_k (uhat_ik - u_ik)^2, with (L u)_ik = u_ik - sum_j
// w_ij u_jk / sqrt(d_i d_j) (L_s) or d_i u_ik - sum_j w_ij u_jk (L = D - W).
// Threads add their rows in order; the block adds its threads in a fixed
// order and adds its total into the exact fixed-point accumulator, so the
// result does not depend on the order in which blocks finish.
__global__ void __launch_bounds__(kBlock)
k_na_energy(int64_t n, int64_t nnz, int K, const int32_t* __restrict__ rp,
            const int32_t* __restrict__ col, const double* __restrict__ w,
            const double* __restrict__ deg, const double* __restrict__ U, int64_t ldu,
            const int32_t* __restrict__ labels, double inv_eps, double omega0, int comb,
            unsigned long long* acc) {
    const int64_t stride = int64_t(gridDim.x) * kBlock;
    double e_thr = 0.0;
    for (int64_t i = blockIdx.x * int64_t(kBlock) + threadIdx.x; i < n; i += stride) {
        const int64_t e0 = rp[i], e1 = rp[i + 1];
        const double di = deg[i];
        if (e0 < 0 || e1 > nnz || e1 < e0 || !(di > 0.0)) continue;  // flagged by k_na_degrees
        int f = labels ? labels[i] : -1;
        if (f < -1 || f >= K) {
            atomicOr(&acc[kNaErrWord], kNaBadLabel);
            f = -1;
        }
        const double* ui = U + i * ldu;
        double quad = 0.0, pen = 0.0, fidt = 0.0;
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int64_t e = e0; e < e1; ++e) {
                const int32_t j = col[e];
                if (j < 0 || j >= n) continue;
                const double wij = comb ? w[e] : w[e] / sqrt(di * deg[j]);
                s += wij * U[j * ldu + k];
            }
            const double u = ui[k];
            const double lu = (comb ? di : 1.0) * u - s;
            quad += u * lu;
            pen += u * (1.0 - u);
            if (f >= 0) {
                const double dlt = (k == f ? 1.0 : 0.0) - u;
                fidt += dlt * dlt;
            }
        }
        e_thr += 0.5 * quad + inv_eps * pen + (f >= 0 ? 0.5 * omega0 * fidt : 0.0);
    }
    const double v[1] = {e_thr};
    block_accumulate<double, 1>(v, acc, 0, int(blockIdx.x % kAccCopies));
}

std::mutex g_na_mu;
struct NaCache {
    unsigned long long ctx = 0;   // unique id of the context the address belongs to
    void* ptr = nullptr;
};
NaCache g_na_cache[kNaMaxDevices];

// Unique id of the current CUDA context (the driver's cuCtxGetCurrent and
// cuCtxGetId, reached through the runtime's entry-point query, so the library
// needs no link against the driver library).  0 when it cannot be read: the
// caller then looks the address up on every call.
unsigned long long current_ctx_id() {
    typedef CUresult (*get_current_fn)(CUcontext*);
    typedef CUresult (*get_id_fn)(CUcontext, unsigned long long*);
    static get_current_fn get_current = nullptr;
    static get_id_fn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<get_current_fn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<get_id_fn>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
    if (get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of this device's scratch array, looked up once per device
// and context.
fw_status na_scratch(void** out) {
    int dev = 0;
    FW_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("fw_energy_noalloc: device ordinal out of the supported range");
        return FW_ERR_UNSUPPORTED;
    }
    // before the process's first CUDA work no context is current yet (id 0):
    // the lookup below then creates it, and the next call caches its id
    const unsigned long long ctx = current_ctx_id();
    std::lock_guard<std::mutex> lock(g_na_mu);
    NaCache& c = g_na_cache[dev];
    if (!c.ptr || ctx == 0 || c.ctx != ctx) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        c.ptr = p;
        c.ctx = ctx;
    }
    *out = c.ptr;
    return FW_OK;
}

fw_status na_invalid(const char* m) {
    set_error(m);
    return FW_ERR_INVALID_ARG;
}

}  // namespace
}  // namespace fw

using namespace fw;

extern "C" fw_status fw_energy_noalloc(int64_t n, int32_t K, const int32_t* row_ptr_dev,
                                       const int32_t* col_dev, const double* w_dev, int64_t nnz,
                                       const double* U_dev, int64_t ldu,
                                       const int32_t* labels_dev, double eps, double omega0,
                                       int32_t laplacian, void* cuda_stream, double* E_host) {
    if (!E_host) return na_invalid("fw_energy_noalloc: E_host is NULL");
    if (n < 1) return na_invalid("fw_energy_noalloc: n must be >= 1");
    if (n > kNaMaxN) {
        set_error("fw_energy_noalloc: n = " + std::to_string(n) +
                  " exceeds the static scratch limit FW_NOALLOC_MAX_N = " +
                  std::to_string(kNaMaxN) + " rows");
        return FW_ERR_UNSUPPORTED;
    }
    if (K < 2 || K > 32) return na_invalid("fw_energy_noalloc: K must be in [2, 32]");
    if (nnz < 0 || nnz >= (int64_t(1) << 31))
        return na_invalid("fw_energy_noalloc: nnz must be in [0, 2^31)");
    if (!row_ptr_dev || !U_dev || (nnz > 0 && (!col_dev || !w_dev)))
        return na_invalid("fw_energy_noalloc: NULL device pointer");
    if (ldu < K) return na_invalid("fw_energy_noalloc: ldu must be >= K");
    if (!(eps > 0.0)) return na_invalid("fw_energy_noalloc: eps must be > 0 (or +inf)");
    if (!(omega0 >= 0.0) || std::isinf(omega0))
        return na_invalid("fw_energy_noalloc: omega0 must be finite and >= 0");
    if (laplacian != FW_LAPLACIAN_SYM && laplacian != FW_LAPLACIAN_COMB)
        return na_invalid("fw_energy_noalloc: bad laplacian");

    void* base = nullptr;
    const fw_status ss = na_scratch(&base);
    if (ss != FW_OK) return ss;
    unsigned long long* acc = static_cast<unsigned long long*>(base);
    double* deg = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kNaAccWords * 8);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // the accumulators and error words must start at zero; the degrees are
    // written in full before they are read
    FW_CUDA(cudaMemsetAsync(acc, 0, kNaAccWords * 8, s));
    const int64_t want = (n + kBlock - 1) / kBlock;
    const int blocks = int(want < kNaMaxBlocks ? want : kNaMaxBlocks);
    k_na_degrees<<<blocks, kBlock, 0, s>>>(n, nnz, row_ptr_dev, col_dev, w_dev, deg, acc);
    FW_CUDA(cudaGetLastError());
    k_na_energy<<<blocks, kBlock, 0, s>>>(n, nnz, K, row_ptr_dev, col_dev, w_dev, deg, U_dev,
                                          ldu, labels_dev, std::isinf(eps) ? 0.0 : 1.0 / eps,
                                          omega0, laplacian == FW_LAPLACIAN_COMB ? 1 : 0, acc);
    FW_CUDA(cudaGetLastError());
    unsigned long long h[kNaAccWords];
    FW_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    FW_CUDA(cudaStreamSynchronize(s));

    const unsigned long long err = h[kNaErrWord];
    if (err & (kNaBadRowPtr | kNaBadCol)) {
        set_error("fw_energy_noalloc: row_ptr extent or column index out of range");
        return FW_ERR_GRAPH;
    }
    if (err & kNaIsolated) {
        set_error("fw_energy_noalloc: a node has degree 0");
        return FW_ERR_ISOLATED;
    }
    if (err & kNaBadLabel) return na_invalid("fw_energy_noalloc: label outside [-1, K)");
    if (h[kAccFlag]) {
        set_error("fw_energy_noalloc: non-finite or out-of-range partial energy");
        return FW_ERR_NUMERIC;
    }
    // exact 128-bit total of the accumulator copies of quantity 0
    unsigned long long lo = 0ull, hi = 0ull;
    for (int c = 0; c < kAccCopies; ++c) {
        const unsigned long long l = h[c * kNumR * kAccLine], hw = h[c * kNumR * kAccLine + 1];
        const unsigned long long lo2 = lo + l;
        hi += hw + (lo2 < lo ? 1ull : 0ull);
        lo = lo2;
    }
    *E_host = double(static_cast<long long>(hi)) + std::ldexp(double(lo), -64);
    return FW_OK;
}
