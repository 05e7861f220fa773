// Ops implementation for one (T, WT, KMAX) instantiation.
#pragma once
#include "fw_internal.h"
#include "fw_kernels.cuh"

namespace fw {

template <typename T, typename WT, int KMAX>
class OpsImpl final : public Ops {
public:
    size_t elem() const override { return sizeof(T); }
    size_t welem() const override { return sizeof(WT); }
    int kmax() const override { return KMAX; }
    static size_t smem() { return 2 * size_t(kBlock) * (KMAX | 1) * sizeof(T); }

    cudaError_t configure() override {
        cudaError_t e = cudaFuncSetAttribute(k_passB<T, WT, KMAX>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_spmm<T, WT, KMAX>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
    }
    void passA(const Bufs& b, cudaStream_t s) override {
        k_passA<T, KMAX, MODE_STEP><<<b.pd.ntiles, kBlock, 0, s>>>(
            b.pd, b.st, (T*)b.U, (T*)b.LU, (const T*)b.LS, b.choice, b.fid, b.partA, nullptr,
            nullptr);
    }
    void flush(const Bufs& b, cudaStream_t s) override {
        k_passA<T, KMAX, MODE_FLUSH><<<b.pd.ntiles, kBlock, 0, s>>>(
            b.pd, b.st, (T*)b.U, (T*)b.LU, (const T*)b.LS, b.choice, b.fid, b.partA, nullptr,
            nullptr);
    }
    void grad(const Bufs& b, void* Gout, uint8_t* chout, cudaStream_t s) override {
        k_passA<T, KMAX, MODE_GRAD><<<b.pd.ntiles, kBlock, 0, s>>>(
            b.pd, b.st, (T*)b.U, (T*)b.LU, (const T*)b.LS, b.choice, b.fid, b.partA, (T*)Gout,
            chout);
    }
    void passB(const Bufs& b, cudaStream_t s) override {
        k_passB<T, WT, KMAX><<<b.pd.ntiles, kBlock, smem(), s>>>(
            b.pd, b.st, b.rp, b.col, (const WT*)b.val, (const T*)b.diag, b.choice, (const T*)b.U,
            (T*)b.LS, b.partB);
    }
    void spmm(const Bufs& b, const void* in, void* out, cudaStream_t s) override {
        k_spmm<T, WT, KMAX><<<b.pd.ntiles, kBlock, smem(), s>>>(
            b.pd, b.rp, b.col, (const WT*)b.val, (const T*)b.diag, (const T*)in, (T*)out);
    }
    void build(int64_t n, int64_t row0, const int32_t* rp, const int32_t* col, const double* w,
               const double* deg, const int32_t* rpp, int32_t* colp, void* valp, void* diag,
               int comb, cudaStream_t s) override {
        const unsigned g = unsigned((n + kBlock - 1) / kBlock);
        k_build<WT, T><<<g, kBlock, 0, s>>>(n, row0, rp, col, w, deg, rpp, colp, (WT*)valp,
                                             (T*)diag, comb);
    }
    void init(const Bufs& b, const int32_t* labels, cudaStream_t s) override {
        const unsigned g = unsigned((b.pd.n + kBlock - 1) / kBlock);
        k_init<T><<<g, kBlock, 0, s>>>(b.pd, labels, (T*)b.U, b.fid, b.choice);
    }
    void reinit(const Bufs& b, cudaStream_t s) override {
        const unsigned g = unsigned((b.pd.n + kBlock - 1) / kBlock);
        k_reinit<T><<<g, kBlock, 0, s>>>(b.pd, (T*)b.U, b.fid, b.choice);
    }
    void labels(const Bufs& b, int32_t* out, cudaStream_t s) override {
        const unsigned g = unsigned((b.pd.n + kBlock - 1) / kBlock);
        k_labels<T><<<g, kBlock, 0, s>>>(b.pd, (const T*)b.U, out);
    }
    void objective(const Bufs& b, const void* LUf, double* part, cudaStream_t s) override {
        const unsigned g = unsigned((b.pd.n + kBlock - 1) / kBlock);
        k_objective<T><<<g, kBlock, 0, s>>>(b.pd, (const T*)b.U, (const T*)LUf, b.fid, part);
    }
};

template <typename T, typename WT>
Ops* make_ops_t(int kmax) {
    switch (kmax) {
        case 4: return new OpsImpl<T, WT, 4>();
        case 8: return new OpsImpl<T, WT, 8>();
        case 12: return new OpsImpl<T, WT, 12>();
        case 16: return new OpsImpl<T, WT, 16>();
        case 32: return new OpsImpl<T, WT, 32>();
        default: return nullptr;
    }
}

}  // namespace fw
