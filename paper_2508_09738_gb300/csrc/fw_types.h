// Internal POD types shared by host and device code of the GFW library.
#pragma once
#include <stdint.h>

namespace fw {

constexpr int kBlock = 256;         // threads per block of every row / CSR kernel
constexpr int kPadW = 4;            // CSR rows padded to a multiple of 4 entries (int4 loads)
constexpr int kTilesTarget = 608;   // a problem is cut into at most this many row tiles
constexpr int kNumA = 5;            // row-pass partials: g, ||D||^2, sum w||D||^2, <D,LU>, |I|
constexpr int kNumB = 1;            // CSR-pass partial: <D, L S>
constexpr uint8_t kActiveBit = 0x80;  // bit 7 of the choice byte: row moved by the oracle

// Static description of one problem inside a (possibly concatenated) batch.
// Iterate arrays are stored class-major ("SoA"): column k of problem p lives at
// U[uoff + k*npad : uoff + k*npad + n], so a warp reading one class of 32
// consecutive rows issues one coalesced 128-byte access.
struct ProbDesc {
    int64_t row0;       // first global row (index into choice / fid / row_ptr)
    int64_t uoff;       // element offset of this problem's U / LU / LS block
    int32_t n;          // rows
    int32_t npad;       // class stride of the SoA block (multiple of 32)
    int32_t K;          // classes
    int32_t tile_rows;  // rows per tile (multiple of kBlock)
    int32_t ntiles;     // tiles of this problem
    int32_t tile0;      // first tile's slot in the global partial arrays
    double inv_eps;     // 1/eps (0 when eps = +inf)
    double omega0;      // fidelity weight
    double gap_tol;
    int32_t tol_mode;   // 0 abs, 1 relative to g_0
    int32_t max_iters;
    int32_t oracle;     // 0 greedy (Alg. 3), 1 full LMO (Alg. 2)
    int32_t step_rule;  // 0 exact, 1 Armijo
    int32_t lanes;      // lanes per CSR row (1..32, power of two)
    int32_t comb;       // 1: L = D - W (diag array used), 0: L_s (unit diagonal)
};

// Mutable per-problem state, in device memory.  Written only by the last
// block to finish a pass of the problem, read by all blocks of the next pass.
struct ProbState {
    double g, g0, nD, nW, tLU, pLS, q, alpha, E;
    int32_t iter;        // updates applied
    int32_t status;      // fw_status once done, FW_PENDING (2) while running
    int32_t active;      // |I_k|
    int32_t has_update;  // 1: alpha / choice / LS of the last step not yet applied
    int32_t done;        // 1: stop rule met, later passes skip this problem
    int32_t g0_set;
    uint32_t cntA, cntB, cntF;  // arrival counters of the last-block reductions
    uint32_t pad_;
};

}  // namespace fw
