// Host-side internals shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/fw_seg.h"
#include "fw_types.h"

namespace fw {

// Thread-local error text behind fw_seg_last_error().
void set_error(const std::string& msg);
fw_status cuda_fail(cudaError_t e, const char* what);

#define FW_CUDA(call)                                         \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return fw::cuda_fail(e_, #call); \
    } while (0)

// Kernel launchers for one (iterate type, weight type, class bound) choice.
// Every launcher takes the problem's descriptor (device pointers inside).
class Ops {
public:
    virtual ~Ops() {}
    virtual size_t elem() const = 0;    // sizeof(T)
    virtual size_t welem() const = 0;   // sizeof(WT)
    virtual int kmax() const = 0;
    // fin: take the previous iteration's step decision inside this pass (the
    // previous iteration then has no k_finish); 0: apply the stored step
    virtual void passA(const ProbDesc& pd, ProbState* st, cudaStream_t s, int fin) = 0;
    virtual void passB(const ProbDesc& pd, ProbState* st, cudaStream_t s) = 0;
    // one thread: read the exact totals, stop test, step
    virtual void finish(const ProbDesc& pd, ProbState* st, cudaStream_t s) = 0;
    virtual void flush(const ProbDesc& pd, ProbState* st, cudaStream_t s) = 0;
    virtual void grad(const ProbDesc& pd, ProbState* st, void* Gout, uint8_t* chout,
                      cudaStream_t s) = 0;
    virtual void spmm(const ProbDesc& pd, const void* X, void* out, cudaStream_t s) = 0;
    // out = L U_hat, valid while U holds U_hat (right after reinit)
    virtual void spmm_hat(const ProbDesc& pd, void* out, cudaStream_t s) = 0;
    // classic FW gap partials per row block (fresh LUf)
    virtual void lmo_gap(const ProbDesc& pd, const void* LUf, double* part, cudaStream_t s) = 0;
    // One-Shot Frank-Wolfe labels (Alg. 4) in one CSR pass
    virtual void oneshot(const ProbDesc& pd, int32_t* labels, cudaStream_t s) = 0;
    virtual void build(int64_t n, const int32_t* rp, const int32_t* col, const double* w,
                       const double* deg, const int32_t* rpp, int32_t* colp, void* valp,
                       void* diag, int comb, int col16, cudaStream_t s) = 0;
    virtual void reinit(const ProbDesc& pd, cudaStream_t s) = 0;
    virtual void labels(const ProbDesc& pd, int32_t* out, cudaStream_t s) = 0;
    virtual void objective(const ProbDesc& pd, const void* LUf, double* part, cudaStream_t s) = 0;
    virtual cudaError_t configure() = 0;   // dynamic shared-memory limits
    // Dynamic shared memory of k_passB_tab for this many lanes per row and
    // rows; 0 when the instantiation has no such form (FP64 iterate, K > 16).
    virtual size_t tab_smem(int lanes, int64_t n) const = 0;
};

// Non-template kernels (defined in fw_seg.cu).
__global__ void k_validate(int64_t n, const int32_t* rp, const int32_t* col, const double* w,
                           double* deg, int* err);
__global__ void k_state_init(ProbState* st, const double* part, int nb);
__global__ void k_fid(int64_t n, const int32_t* labels, int8_t* fid);

// Factories, one per translation unit.  kmax in {4, 8, 10, 12, 16, 32}.
Ops* make_ops_f32(int kmax);
Ops* make_ops_bf16(int kmax);
Ops* make_ops_f64(int kmax);
Ops* make_ops(int weight_dtype, int K);
int kmax_for(int K);

// A graph on the host, as passed to the C ABI.
struct HostGraph {
    int64_t n;
    const int32_t* rp;
    const int32_t* col;
    const double* w;
    int32_t K;
    const int32_t* labels;
};

// Host-side layout of one problem: sizes, tiles and the padded row_ptr.
struct ProbLayout {
    int64_t n = 0, nnz = 0, nnz_pad = 0, npad = 0;
    int32_t K = 0, tile_rows = 0, ntiles = 0, lanes = 1;
    // keep the 4-bit class array (ProbDesc::cls4): set by the two-kernel
    // single-problem path for K <= 16; the persistent kernels do not use it
    bool cls4 = false;
    // store columns as 16-bit offsets when the graph allows (fw_seg_opts::index_width)
    bool allow16 = true;
    // pass B with the class table in shared memory (fw_seg_opts::class_table)
    int32_t tab_mode = FW_TABLE_AUTO;
};

// Host checks (options, row_ptr, labels) and the padded layout.
fw_status check_opts(const fw_seg_opts& o);
fw_status plan_problem(const HostGraph& g, const fw_seg_opts& o, ProbLayout& lay);
// Device bytes of one problem's persistent arrays (256-byte aligned pieces).
size_t problem_bytes(const ProbLayout& lay, size_t te, size_t we, bool comb);
// Carve the problem's arrays out of [base, base + problem_bytes) and fill pd.
void place_problem(char* base, const ProbLayout& lay, size_t te, size_t we, const fw_seg_opts& o,
                   ProbDesc& pd);
// Stream-ordered device allocation from the library's per-device pool (freed
// with cudaFreeAsync on a stream ordered after every use).  FW_ERR_NO_MEMORY
// with the message set on failure.
fw_status pool_alloc(void** out, size_t bytes, cudaStream_t s);

// Stream-ordered temporaries, released (stream-ordered) when the object dies.
struct Temps {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Temps(cudaStream_t st) : s(st) {}
    ~Temps() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    template <typename P>
    fw_status get(P** out, size_t bytes) {
        void* q = nullptr;
        const fw_status st = pool_alloc(&q, bytes, s);
        if (st != FW_OK) return st;
        ptrs.push_back(q);
        *out = reinterpret_cast<P*>(q);
        return FW_OK;
    }
};

// Device copies of a caller's input arrays (row_ptr, col, w, labels).
struct Upload {
    Temps t;
    int64_t n = 0, nnz = 0;
    int32_t *rp = nullptr, *col = nullptr, *lab = nullptr;
    double* w = nullptr;
    explicit Upload(cudaStream_t s) : t(s) {}
};
// The O(1) checks the upload relies on: n, K, pointers, row_ptr[0] and nnz.
fw_status check_graph_args(const HostGraph& g);
// Enqueue the copies of g's arrays on up's stream (asynchronous from pinned
// host memory; the caller's arrays must stay valid until the stream passes).
fw_status upload_inputs(const HostGraph& g, Upload& up);
// Upload, validate and build the problem into pd's arrays; U_0, L U_0 and the
// fresh state *st.  Temporaries are stream-ordered (pool_alloc).  Waits
// for the validation result on `s`.
fw_status assemble_problem(Ops* ops, const HostGraph& g, const ProbLayout& lay, ProbDesc& pd,
                           ProbState* st, cudaStream_t s);
// The same from inputs already uploaded (or in flight) on stream s.
// Sets pd.col16 from the validated graph.
fw_status assemble_uploaded(Ops* ops, Upload& up, const ProbLayout& lay, ProbDesc& pd,
                            ProbState* st, cudaStream_t s);
// Restart pd at U_0 (or at its current U when from_current) with a fresh state.
fw_status restart_problem(Ops* ops, const ProbDesc& pd, ProbState* st, bool from_current,
                          cudaStream_t s);

// Geometry helpers.
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
int tile_rows_for(int64_t n);
int default_lanes(double avg_padded_degree);

}  // namespace fw
