// Host-side internals shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

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

// Device buffers and geometry of one problem (or of a concatenated batch).
struct Bufs {
    ProbDesc pd{};
    ProbState* st = nullptr;
    int32_t* rp = nullptr;     // padded row_ptr, global rows (+1)
    int32_t* col = nullptr;    // padded columns, global row indices
    void* val = nullptr;       // padded weights (WT)
    void* diag = nullptr;      // T[n], combinatorial Laplacian only
    void* U = nullptr;         // T, SoA
    void* LU = nullptr;
    void* LS = nullptr;
    uint8_t* choice = nullptr; // class chosen by the last evaluation | active bit
    int8_t* fid = nullptr;     // fidelity class or -1
    double* partA = nullptr;   // [ntiles][kNumA]
    double* partB = nullptr;   // [ntiles][kNumB]
};

// Kernel launchers for one (iterate type, weight type, class bound) choice.
class Ops {
public:
    virtual ~Ops() {}
    virtual size_t elem() const = 0;    // sizeof(T)
    virtual size_t welem() const = 0;   // sizeof(WT)
    virtual int kmax() const = 0;
    virtual void passA(const Bufs& b, cudaStream_t s) = 0;
    virtual void passB(const Bufs& b, cudaStream_t s) = 0;
    virtual void flush(const Bufs& b, cudaStream_t s) = 0;
    virtual void grad(const Bufs& b, void* Gout, uint8_t* chout, cudaStream_t s) = 0;
    virtual void spmm(const Bufs& b, const void* in, void* out, cudaStream_t s) = 0;
    virtual void build(int64_t n, int64_t row0, const int32_t* rp, const int32_t* col,
                       const double* w, const double* deg, const int32_t* rpp, int32_t* colp,
                       void* valp, void* diag, int comb, cudaStream_t s) = 0;
    virtual void init(const Bufs& b, const int32_t* labels, cudaStream_t s) = 0;
    virtual void reinit(const Bufs& b, cudaStream_t s) = 0;
    virtual void labels(const Bufs& b, int32_t* out, cudaStream_t s) = 0;
    virtual void objective(const Bufs& b, const void* LUf, double* part, cudaStream_t s) = 0;
    virtual cudaError_t configure() = 0;   // dynamic shared-memory limits
};

// Factories, one per translation unit.  kmax in {4, 8, 12, 16, 32}.
Ops* make_ops_f32(int kmax);
Ops* make_ops_bf16(int kmax);
Ops* make_ops_f64(int kmax);
Ops* make_ops(int weight_dtype, int K);
int kmax_for(int K);

// Geometry helpers.
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
int tile_rows_for(int64_t n);
int default_lanes(double avg_padded_degree);

}  // namespace fw
