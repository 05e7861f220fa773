// Internal POD types shared by host and device code of the GFW library.
#pragma once
#include <stdint.h>

namespace fw {

constexpr int kBlock = 256;         // threads per block of every row / CSR kernel
constexpr int kPadW = 4;            // CSR rows padded to a multiple of 4 entries (int4 loads)
constexpr int kTilesTarget = 1216;  // a problem has at most this many row tiles (8 per SM)
constexpr int kNumA = 5;            // row-pass partials: g, ||D||^2, sum w||D||^2, <D,LU>, |I|
constexpr int kNumB = 1;            // CSR-pass partial: <D, L S>
constexpr int kNumR = kNumA + kNumB;  // accumulated quantities (pass A 0..4, pass B 5)
constexpr uint8_t kActiveBit = 0x80;  // bit 7 of the choice byte: row moved by the oracle
// Exact tile-total accumulators: kAccCopies copies of the kNumR Q64.64
// quantities (lo, hi words, kAccLine words apart), then a non-finite flag.
// Tile t adds into copy t % kAccCopies.  (Spreading the copies over separate
// 128-byte lines measured no faster than one compact copy, so one is used.)
constexpr int kAccCopies = 1;
constexpr int kAccLine = 2;                               // 8-byte words per slot
constexpr int kAccFlag = kAccCopies * kNumR * kAccLine;   // index of the flag word
constexpr int kAccWords = kAccFlag + kAccLine;
// Two such banks, 128 bytes apart: iteration t accumulates into one while the
// totals of iteration t-1 are still read from the other (the step decision of
// t-1 is taken inside pass A of t; see ProbState::cur).
constexpr int kAccBank = 16;
constexpr int kAccTotal = 2 * kAccBank;
static_assert(kAccWords <= kAccBank, "accumulator bank overflows its 128 bytes");

// One problem on the device.  Every array is the problem's own (row-local
// indexing, column indices local to the problem); in a batch they are slices
// of one contiguous pool.  Iterate arrays are class-major ("SoA"): class k of
// row i lives at U[k*npad + i], so a warp reading one class of 32 consecutive
// rows issues one coalesced 128-byte access.
struct ProbDesc {
    const int32_t* rp;   // padded row_ptr [n+1] (entries start on multiples of 4)
    const int32_t* col;  // padded columns [nnz_pad] (padding: the row itself); with col16
                         // the same entries as int16 offsets j - i (padding: 0)
    const void* val;     // padded weights WT[nnz_pad] (padding: 0)
    const void* diag;    // T[n], combinatorial Laplacian only (else unused)
    void* U;             // T[K][npad]
    void* LU;            // T[K][npad], L U by recurrence
    void* LS;            // T[K][npad], L S of the last step
    uint8_t* choice;     // [n] class chosen by the last evaluation | kActiveBit
    uint8_t* cls4;       // [(n+1)/2] the same classes as 4-bit pairs (row 2m low nibble,
                         // 2m+1 high) for K <= 16, gathered by pass B; NULL for K > 16
    const int8_t* fid;   // [n] fidelity class or -1
    unsigned long long* acc;  // [kAccTotal]: two banks of kAccWords Q64.64 totals (see
                              // kAccCopies) and a non-finite flag; exact and order-free
    int32_t n;           // rows
    int32_t npad;        // class stride of the SoA block (multiple of 32)
    int32_t K;           // classes
    int32_t tile_rows;   // rows per tile (kBlock)
    int32_t ntiles;      // tiles of this problem
    int32_t lanes;       // lanes per CSR row (1..32, power of two)
    int32_t comb;        // 1: L = D - W (diag used), 0: L_s (unit diagonal)
    int32_t oracle;      // 0 greedy (Alg. 3), 1 full LMO (Alg. 2)
    int32_t step_rule;   // 0 exact, 1 Armijo
    int32_t tol_mode;    // 0 abs, 1 relative to g_0
    int32_t max_iters;
    int32_t col16;       // 1: col holds 16-bit offsets (every |j - i| < 2^15)
    int32_t tab_grid;    // > 0: pass B runs k_passB_tab on this many blocks (class table
                         // in shared memory); 0: the direct pass-B kernels
    int32_t pad_;
    double inv_eps;      // 1/eps (0 when eps = +inf)
    double omega0;       // fidelity weight
    double gap_tol;
    double c2;           // 2/eps rounded to the iterate type by the kernels
    float c2f;           // 2/eps as float (FP32 iterate)
    float omf;           // omega0 as float
};

// The inputs of a step decision besides the iteration's totals: the running
// objective, g_0 for the relative stop rule, and the updates applied so far.
struct StepIn {
    double E, g0;
    int32_t iter, g0_set;
};

// Mutable per-problem state, in device memory.  The first block (iterate
// fields) or the single finishing thread writes it; the next pass reads it.
//
// Step decisions.  Iteration t's totals complete when its pass B ends; the
// stop test and the step length that follow from them are needed by pass A of
// t+1.  Either a one-thread k_finish takes the decision between the passes,
// or (inside a captured graph) every block of pass A of t+1 takes the same
// decision from the same totals and inputs, and only its first block writes
// the result here.  So that no block reads a field another block of the same
// pass writes, the inputs are kept twice (in[cur] is read, in[cur ^ 1]
// written) and the totals alternate between the two accumulator banks:
//   pass A (decision fused): reads bank cur and in[cur], accumulates into
//                            bank cur ^ 1, block 0 writes in[cur ^ 1] and
//                            cur_b = cur ^ 1;
//   pass A (plain):          accumulates into bank cur, block 0 writes
//                            cur_b = cur;
//   pass B:                  accumulates into bank cur_b; block 0 sets
//                            cur = cur_b and clears bank cur_b ^ 1;
//   k_finish:                reads and clears bank cur, reads in[cur], writes
//                            in[cur ^ 1], cur ^= 1.
// The persistent batch kernel always accumulates into bank 0 and decides in
// its last block; it uses in[] / cur the same way.
struct ProbState {
    double g, g0, nD, nW, tLU, pLS, q, alpha, E;
    float alpha_f;       // alpha rounded to float, for the FP32 update
    int32_t err;         // set by any block whose bulk-copy wait ran out
    int32_t iter;        // updates applied
    int32_t status;      // fw_status once done, FW_PENDING (2) while running
    int32_t active;      // |I_k|
    int32_t has_update;  // 1: alpha / choice / LS of the last step not yet applied
    int32_t done;        // 1: stop rule met, later passes skip this problem
    int32_t g0_set;
    uint32_t cnt;        // pass-B tiles arrived (the last one finishes the iteration)
    uint32_t cntF;       // flush tiles arrived
    int32_t cur;         // parity: step inputs in[cur]; bank of the pending totals
    int32_t cur_b;       // accumulator bank of the running iteration's pass B
    StepIn in[2];
};

}  // namespace fw
