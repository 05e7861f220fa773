// __global__ kernels of the single-problem path and of graph assembly.
#pragma once
#include "fw_device.cuh"

namespace fw {

// ---------------------------------------------------------------- hot loop
// Pass A: one block per row tile; the last block runs the stop test.
template <typename T, int KMAX, int MODE>
__global__ void __launch_bounds__(kBlock)
    k_passA(ProbDesc pd, ProbState* st, T* U, T* LU, const T* LS, uint8_t* choice,
            const int8_t* fid, double* partA, T* Gout, uint8_t* chout) {
    if (MODE != MODE_GRAD && ld_cg(&st->done)) return;
    const bool upd = ld_cg(&st->has_update) != 0;
    const T alpha = T(ld_cg(&st->alpha));
    const int tile = blockIdx.x;
    const int r0 = tile * pd.tile_rows;
    const int r1 = min(pd.n, r0 + pd.tile_rows);
    AccA<T> acc{T(0), T(0), T(0), T(0), T(0)};
    passA_rows<T, KMAX, MODE>(pd, U, LU, LS, choice, fid, r0, r1, upd, alpha, acc, Gout, chout);
    if (MODE == MODE_GRAD) return;
    if (MODE == MODE_FLUSH) {
        if (last_to_arrive(&st->cntF, pd.ntiles) && threadIdx.x == 0) {
            st->has_update = 0;
            st->cntF = 0;
        }
        return;
    }
    const T v[kNumA] = {acc.g, acc.nD, acc.nW, acc.tLU, acc.act};
    block_partials<T, kNumA>(v, partA + (size_t)(pd.tile0 + tile) * kNumA);
    if (last_to_arrive(&st->cntA, pd.ntiles)) {
        double S[kNumA];
        sum_partials<kNumA>(partA + (size_t)pd.tile0 * kNumA, pd.ntiles, S);
        if (threadIdx.x == 0) finish_A(pd, st, S);
    }
}

// Pass B: one block per row tile; the last block forms q and the step.
template <typename T, typename WT, int KMAX>
__global__ void __launch_bounds__(kBlock)
    k_passB(ProbDesc pd, ProbState* st, const int32_t* row_ptr, const int32_t* col, const WT* val,
            const T* diag, const uint8_t* choice, const T* U, T* LS, double* partB) {
    if (ld_cg(&st->done)) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm_lane = reinterpret_cast<T*>(smraw);
    T* sm_row = sm_lane + kBlock * (KMAX | 1);
    const int tile = blockIdx.x;
    const int r0 = tile * pd.tile_rows;
    const int r1 = min(pd.n, r0 + pd.tile_rows);
    T accq = T(0);
    passB_rows<T, WT, KMAX>(pd, row_ptr, col, val, diag, choice, U, LS, r0, r1, accq, sm_lane,
                            sm_row);
    const T v[kNumB] = {accq};
    block_partials<T, kNumB>(v, partB + (size_t)(pd.tile0 + tile) * kNumB);
    if (last_to_arrive(&st->cntB, pd.ntiles)) {
        double S[kNumB];
        sum_partials<kNumB>(partB + (size_t)pd.tile0 * kNumB, pd.ntiles, S);
        if (threadIdx.x == 0) finish_B(pd, st, S);
    }
}

// OUT = L U (initial L U_0, refresh, direct objective).
template <typename T, typename WT, int KMAX>
__global__ void __launch_bounds__(kBlock)
    k_spmm(ProbDesc pd, const int32_t* row_ptr, const int32_t* col, const WT* val, const T* diag,
           const T* U, T* OUT) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm_lane = reinterpret_cast<T*>(smraw);
    T* sm_row = sm_lane + kBlock * (KMAX | 1);
    const int r0 = blockIdx.x * pd.tile_rows;
    const int r1 = min(pd.n, r0 + pd.tile_rows);
    spmm_rows<T, WT, KMAX>(pd, row_ptr, col, val, diag, U, OUT, r0, r1, sm_lane, sm_row);
}

// ------------------------------------------------------------ read-outs
// labels[i] = argmax_k u_ik, lowest index on ties.
template <typename T>
__global__ void k_labels(ProbDesc pd, const T* U, int32_t* out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= pd.n) return;
    const T* Ub = U + pd.uoff;
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
__global__ void __launch_bounds__(kBlock)
    k_objective(ProbDesc pd, const T* U, const T* LUf, const int8_t* fid, double* part) {
    const int r = blockIdx.x * kBlock + threadIdx.x;
    double e = 0.0;
    if (r < pd.n) {
        const T* Ub = U + pd.uoff;
        const T* Lb = LUf + pd.uoff;
        const int f = fid[pd.row0 + r];
        double quad = 0.0, pen = 0.0, fidt = 0.0;
        for (int k = 0; k < pd.K; ++k) {
            const double u = double(Ub[(int64_t)k * pd.npad + r]);
            quad += u * double(Lb[(int64_t)k * pd.npad + r]);
            pen += u * (1.0 - u);
            if (f >= 0) {
                const double d = (k == f ? 1.0 : 0.0) - u;
                fidt += d * d;
            }
        }
        e = 0.5 * quad + pd.inv_eps * pen + 0.5 * pd.omega0 * fidt;
    }
    const double v[1] = {e};
    block_partials<double, 1>(v, part + blockIdx.x);
}

// ------------------------------------------------------------- assembly
// Padded CSR of the off-diagonal operator: sym: W^_ij = w_ij / sqrt(d_i d_j)
// rounded to WT (bf16 via float, both nearest-even); comb: w_ij.  Padding
// entries point at the row itself with weight 0.  diag (comb only) = d_i.
template <typename WT, typename T>
__global__ void k_build(int64_t n, int64_t row0, const int32_t* rp, const int32_t* col,
                        const double* w, const double* deg, const int32_t* rpp, int32_t* colp,
                        WT* valp, T* diag, int comb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e0 = rp[i], e1 = rp[i + 1];
    int p = rpp[i];
    const int pend = rpp[i + 1];
    const double di = deg[i];
    for (int e = e0; e < e1; ++e, ++p) {
        const int j = col[e];
        const double x = comb ? w[e] : w[e] / sqrt(di * deg[j]);
        colp[p] = int32_t(j + row0);
        if constexpr (sizeof(WT) == 2)
            valp[p] = __float2bfloat16_rn(__double2float_rn(x));
        else if constexpr (sizeof(WT) == 4)
            valp[p] = __double2float_rn(x);
        else
            valp[p] = x;
    }
    for (; p < pend; ++p) {
        colp[p] = int32_t(i + row0);
        valp[p] = WT(0.0f);
    }
    if (comb) diag[row0 + i] = T(di);
}

// U_0 = U_hat (Sec. 5.1): e_c on fidelity rows, 1/K elsewhere; fid and choice.
template <typename T>
__global__ void k_init(ProbDesc pd, const int32_t* labels, T* U, int8_t* fid, uint8_t* choice) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= pd.n) return;
    const int c = labels[r];
    const T unif = T(1) / T(pd.K);
    T* Ub = U + pd.uoff;
    for (int k = 0; k < pd.K; ++k) Ub[(int64_t)k * pd.npad + r] = c >= 0 ? (k == c ? T(1) : T(0)) : unif;
    fid[pd.row0 + r] = int8_t(c);
    choice[pd.row0 + r] = uint8_t(c >= 0 ? c : 0);
}

// Restart: U_0 = U_hat from the stored fidelity classes.
template <typename T>
__global__ void k_reinit(ProbDesc pd, T* U, const int8_t* fid, uint8_t* choice) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= pd.n) return;
    const int c = fid[pd.row0 + r];
    const T unif = T(1) / T(pd.K);
    T* Ub = U + pd.uoff;
    for (int k = 0; k < pd.K; ++k) Ub[(int64_t)k * pd.npad + r] = c >= 0 ? (k == c ? T(1) : T(0)) : unif;
    choice[pd.row0 + r] = uint8_t(c >= 0 ? c : 0);
}

}  // namespace fw
