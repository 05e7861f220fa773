// Ops implementation for one (T, WT, KMAX) instantiation.
#pragma once
#include "fw_internal.h"
#include "fw_kernels.cuh"

namespace fw {

template <typename T, typename WT, int KMAX>
class OpsImpl final : public Ops {
public:
    // exactly KMAX classes, FP32 iterate: the compile-time class-count forms
    // (pass A only for four classes: with more, the fully unrolled row keeps
    // its classes in registers and spills at the occupancy it needs)
    static constexpr bool kExactA = sizeof(T) == 4 && KMAX == 4;
    static constexpr bool kExactB = sizeof(T) == 4 && KMAX <= 12;
    // 2 / 4 lanes per row, 5..12 classes, FP32 iterate: the 40-register pass B
    static constexpr bool kBound6 = sizeof(T) == 4 && KMAX >= 8 && KMAX <= 12;
    // pass B with the class table in shared memory: FP32 iterate, 4-bit classes
    static constexpr bool kTab = sizeof(T) == 4 && KMAX <= 16;
    size_t elem() const override { return sizeof(T); }
    size_t welem() const override { return sizeof(WT); }
    int kmax() const override { return KMAX; }
    // pass B / SpMM bins
    static size_t smem() { return 2 * size_t(kBlock) * (KMAX | 1) * sizeof(T); }
    // pass B: bins plus, in the forms that prefetch, the rows' U values and
    // choice bytes
    static size_t smemB() { return smem() + passB_prefetch_bytes<T, KMAX>(); }
    template <int LC>
    static size_t smemB_lc() {
        return passB_prefetches<KMAX, true, LC>() ? smemB() : smem();
    }
    static size_t smemA() { return max_stages<T, KMAX>() * 3 * size_t(kBlock) * KMAX * sizeof(T); }
    static size_t smemA(const ProbDesc& pd) {
        return (pd.tile_rows > kBlock ? max_stages<T, KMAX>() : 1) * 3 * size_t(kBlock) * KMAX *
               sizeof(T);
    }
    static unsigned rows_grid(const ProbDesc& pd) { return unsigned((pd.n + kBlock - 1) / kBlock); }

    cudaError_t configure() override {
        cudaError_t e = cudaFuncSetAttribute(k_passA<T, KMAX, MODE_STEP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smemA()));
        if (e != cudaSuccess) return e;
        if constexpr (kExactA) {
            e = cudaFuncSetAttribute(k_passA_exact<T, KMAX>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(smemA()));
            if (e != cudaSuccess) return e;
        }
        e = cudaFuncSetAttribute(k_passB<T, WT, KMAX>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(smemB()));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_osfw<T, WT, KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem()));
        if (e != cudaSuccess) return e;
        for (auto f : {k_passB_lc<T, WT, KMAX, 1, false>, k_passB_lc<T, WT, KMAX, 2, false>,
                       k_passB_lc<T, WT, KMAX, 4, false>, k_passB_lc6<T, WT, KMAX, 2, false>,
                       k_passB_lc6<T, WT, KMAX, 4, false>}) {
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smemB()));
            if (e != cudaSuccess) return e;
        }
        if constexpr (kExactB) {
            for (auto f : {k_passB_lc<T, WT, KMAX, 1, true>, k_passB_lc<T, WT, KMAX, 2, true>,
                           k_passB_lc<T, WT, KMAX, 4, true>, k_passB_lc6<T, WT, KMAX, 2, true>,
                           k_passB_lc6<T, WT, KMAX, 4, true>}) {
                e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smemB()));
                if (e != cudaSuccess) return e;
            }
        }
        if constexpr (kTab) {
            for (auto f : {k_passB_tab<T, WT, KMAX, 1, false>, k_passB_tab<T, WT, KMAX, 2, false>,
                           k_passB_tab<T, WT, KMAX, 4, false>, k_passB_tab<T, WT, KMAX, 1, true>,
                           k_passB_tab<T, WT, KMAX, 2, true>, k_passB_tab<T, WT, KMAX, 4, true>}) {
                e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kTabSmemMax);
                if (e != cudaSuccess) return e;
            }
        }
        e = cudaFuncSetAttribute(k_spmm_hat<T, WT, KMAX>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_spmm<T, WT, KMAX>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
    }
    void passA(const ProbDesc& pd, ProbState* st, cudaStream_t s, int fin) override {
        if constexpr (kExactA) {
            if (pd.K == KMAX) {
                k_passA_exact<T, KMAX><<<pd.ntiles, kBlock, smemA(pd), s>>>(pd, st, fin);
                return;
            }
        }
        k_passA<T, KMAX, MODE_STEP><<<pd.ntiles, kBlock, smemA(pd), s>>>(pd, st, nullptr, nullptr,
                                                                         fin);
    }
    void flush(const ProbDesc& pd, ProbState* st, cudaStream_t s) override {
        k_passA<T, KMAX, MODE_FLUSH><<<pd.ntiles, kBlock, 0, s>>>(pd, st, nullptr, nullptr, 0);
    }
    void grad(const ProbDesc& pd, ProbState* st, void* Gout, uint8_t* chout,
              cudaStream_t s) override {
        k_passA<T, KMAX, MODE_GRAD><<<pd.ntiles, kBlock, 0, s>>>(pd, st, (T*)Gout, chout, 0);
    }
    template <bool EXACT>
    void passB_lanes(const ProbDesc& pd, ProbState* st, cudaStream_t s) {
        const unsigned g = unsigned(pd.ntiles);
        if (pd.lanes == 1)
            k_passB_lc<T, WT, KMAX, 1, EXACT><<<g, kBlock, smemB_lc<1>(), s>>>(pd, st);
        else if (pd.lanes == 2 && kBound6)
            k_passB_lc6<T, WT, KMAX, 2, EXACT><<<g, kBlock, smemB_lc<2>(), s>>>(pd, st);
        else if (pd.lanes == 4 && kBound6)
            k_passB_lc6<T, WT, KMAX, 4, EXACT><<<g, kBlock, smemB_lc<4>(), s>>>(pd, st);
        else if (pd.lanes == 2)
            k_passB_lc<T, WT, KMAX, 2, EXACT><<<g, kBlock, smemB_lc<2>(), s>>>(pd, st);
        else
            k_passB_lc<T, WT, KMAX, 4, EXACT><<<g, kBlock, smemB_lc<4>(), s>>>(pd, st);
    }
    size_t tab_smem(int lanes, int64_t n) const override {
        if constexpr (kTab) return tab_bins_bytes<T, KMAX>(lanes) + tab_bytes(int(n));
        return 0;
    }
    template <bool EXACT>
    void passB_tab(const ProbDesc& pd, ProbState* st, cudaStream_t s) {
        const unsigned g = unsigned(pd.tab_grid);
        const size_t sm = tab_smem(pd.lanes, pd.n);
        if (pd.lanes == 1)
            k_passB_tab<T, WT, KMAX, 1, EXACT><<<g, kTabThreads, sm, s>>>(pd, st);
        else if (pd.lanes == 2)
            k_passB_tab<T, WT, KMAX, 2, EXACT><<<g, kTabThreads, sm, s>>>(pd, st);
        else
            k_passB_tab<T, WT, KMAX, 4, EXACT><<<g, kTabThreads, sm, s>>>(pd, st);
    }
    void passB(const ProbDesc& pd, ProbState* st, cudaStream_t s) override {
        if constexpr (kTab) {
            if (pd.tab_grid > 0) {   // choose_tab checked lanes, tiles and the fit
                if (pd.K == KMAX) passB_tab<true>(pd, st, s);
                else passB_tab<false>(pd, st, s);
                return;
            }
        }
        if (pd.lanes != 1 && pd.lanes != 2 && pd.lanes != 4) {
            k_passB<T, WT, KMAX><<<unsigned(pd.ntiles), kBlock, smemB_lc<0>(), s>>>(pd, st);
            return;
        }
        if constexpr (kExactB) {
            if (pd.K == KMAX) {
                passB_lanes<true>(pd, st, s);
                return;
            }
        }
        passB_lanes<false>(pd, st, s);
    }
    void finish(const ProbDesc& pd, ProbState* st, cudaStream_t s) override {
        k_finish<<<1, 32, 0, s>>>(pd, st);
    }
    void oneshot(const ProbDesc& pd, int32_t* labels, cudaStream_t s) override {
        k_osfw<T, WT, KMAX><<<rows_grid(pd), kBlock, smem(), s>>>(pd, labels);
    }
    void spmm_hat(const ProbDesc& pd, void* out, cudaStream_t s) override {
        k_spmm_hat<T, WT, KMAX><<<pd.ntiles, kBlock, smem(), s>>>(pd, (T*)out);
    }
    void spmm(const ProbDesc& pd, const void* X, void* out, cudaStream_t s) override {
        k_spmm<T, WT, KMAX><<<pd.ntiles, kBlock, smem(), s>>>(pd, (const T*)X, (T*)out);
    }
    void build(int64_t n, const int32_t* rp, const int32_t* col, const double* w,
               const double* deg, const int32_t* rpp, int32_t* colp, void* valp, void* diag,
               int comb, int col16, cudaStream_t s) override {
        const unsigned g = unsigned((n + kBlock - 1) / kBlock);
        k_build<WT, T><<<g, kBlock, 0, s>>>(n, rp, col, w, deg, rpp, colp, (WT*)valp, (T*)diag,
                                             comb, col16);
    }
    void reinit(const ProbDesc& pd, cudaStream_t s) override {
        k_reinit<T><<<rows_grid(pd), kBlock, 0, s>>>(pd);
    }
    void labels(const ProbDesc& pd, int32_t* out, cudaStream_t s) override {
        k_labels<T><<<rows_grid(pd), kBlock, 0, s>>>(pd, out);
    }
    void lmo_gap(const ProbDesc& pd, const void* LUf, double* part, cudaStream_t s) override {
        k_lmo_gap<T, KMAX><<<rows_grid(pd), kBlock, 0, s>>>(pd, (const T*)LUf, part);
    }
    void objective(const ProbDesc& pd, const void* LUf, double* part, cudaStream_t s) override {
        k_objective<T><<<rows_grid(pd), kBlock, 0, s>>>(pd, (const T*)LUf, part);
    }
};

template <typename T, typename WT>
Ops* make_ops_t(int kmax) {
    switch (kmax) {
        case 4: return new OpsImpl<T, WT, 4>();
        case 8: return new OpsImpl<T, WT, 8>();
        case 10: return new OpsImpl<T, WT, 10>();
        case 12: return new OpsImpl<T, WT, 12>();
        case 16: return new OpsImpl<T, WT, 16>();
        case 32: return new OpsImpl<T, WT, 32>();
        default: return nullptr;
    }
}

}  // namespace fw
