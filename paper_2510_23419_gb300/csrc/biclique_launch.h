// biclique_launch.h -- host/device interface of the complete-bipartite
// (K_{n,n}) p-bit kernels (arXiv 2510.23419, Sec. 3).
#pragma once

#include "pb_common.h"

namespace pb {

// Spin encodings in global memory, one per coupling type, so that the spin
// matrix is directly the B operand of the tensor-core field:
//   PM1: FP8 e4m3, +1 = 0x38, -1 = 0xB8      (1 byte)
//   F32: BF16,     +1 = 0x3F80, -1 = 0xBF80  (2 bytes)
constexpr uint8_t kE4m3Plus = 0x38, kE4m3Minus = 0xB8;
constexpr uint16_t kBf16Plus = 0x3F80, kBf16Minus = 0xBF80;

struct BqDevice {
    int32_t n, jtype, has_h, hmax;
    const float* Jf;        // [n][n] couplings as float (PM1: +-1.0)
    const float* Jft;       // [n][n] transpose
    const int8_t* h8;       // PM1 [2n] or null
    const float* hf;        // F32 [2n] (zeros when no field)
    const void* Jraw;       // [n][n] int8 or float, for the exact energy
    const void* hraw;       // [2n] int8 or float, or null
    // tensor-core operands, [n][ldj] row-major (row stride ldj elements, a multiple of 16)
    int32_t ldj;
    const uint8_t* Jq;      // e4m3 J (PM1)
    const uint8_t* Jqt;     // e4m3 J^T
    const uint16_t* Jhi;    // bf16 high part of J (F32): hi = bf16(J)
    const uint16_t* Jlo;    // bf16 residual: lo = bf16(J - hi)
    const uint16_t* Jthi;
    const uint16_t* Jtlo;
};

struct BqJob {
    BqDevice inst;
    uint32_t key0, key1;
    int32_t S, step, nF, fmin;
    const uint32_t* table;  // PM1: the threshold windows of all levels, concatenated (see TabWindow)
    const float* betaf;     // F32 [levels]
    int32_t R, Rpad;        // replicas, padded to the replica tile
    int32_t ld;             // leading dimension of a spin row (>= n, padded for the tensor form)
    void* spins[2];         // [Rpad][ld] the state a launch reads and writes: side A (colour 0), side B (colour 1)
    void* buf[2][2];        // [side][parity] live states: sweep s writes parity s & 1 (the initial state: 1), so
                            // state s - 1 is intact during sweep s
    void* best[2];          // [Rpad][ld] best states
    int32_t nblk;           // partial rows per side: row blocks of the field kernels (tensor form: 32-row quarters)
    void* part;             // [2][nblk][Rpad] energy partials (int32 PM1 / float F32): [0] -h.a, [1] -b.F_B
    int32_t* E_best_i;
    float* E_best_f;
    int32_t* best_sweep;
    int32_t* hit_sweep;
    int32_t has_target, target_i;  // has_target: 0 none, 1 record the target sweep, 2 also stop there (see pbit.h)
    float target_f;
    int32_t* stop;          // has_target == 2: [0] replicas that reached the target, [1] the sweep after which all
                            // had (-1 while running); the sweep counters jump to S then
    double* epart;          // [ceil(n/64)][R] row-tile parts of the exact readout energy
    const int32_t* win;     // PM1 [levels][3]: threshold window (lo, width, off) of each beta level
    int32_t tabmode;        // tensor form: where the decisions read the windows (widest level decides)
    int32_t tile_split;     // tensor form: 1 = a sparse last round of tiles is split into 128-replica tiles
    int32_t pdl;            // tensor form: the sweep loop's launches are programmatic dependents of the one
                            // before (set for runs whose half-sweep fills every cluster)
    uint64_t wait_ns;       // tensor form: limit of every device-side wait (ns of the global timer)
    int32_t stall_loads;    // tensor form, failure-path tests only: the load warp issues no loads
};

constexpr uint64_t kBqWaitNs = 1000000000ull;   // 1 s: far above any tile's MMA chain or epilogue
constexpr uint64_t kBqTestWaitNs = 2000000ull;  // 2 ms: the limit under PB_FLAG_TEST_EXPIRE_WAITS

constexpr int kBqResReps = 32;      // resident form: replicas per CTA
constexpr int kBqResMaxNpm1 = 256;  // resident form: largest n (+-1 couplings, int8 J in shared memory)
constexpr int kBqResMaxNf32 = 128;  // resident form: largest n (real couplings, FP32 J in shared memory)

constexpr int kBqTileRows = 64;   // CUDA-core field kernel: rows (spins of the updated side) per block
constexpr int kBqTileReps = 64;   // replicas per block

cudaError_t bq_launch_init(const BqJob& job, cudaStream_t st);
// Resident form: the whole anneal of every 32-replica block in one CTA (grid
// Rpad / 32); tab_cap = the widest threshold window of the run (+-1).
size_t bq_res_smem_bytes(int jtype, int n, int tab_cap);
cudaError_t bq_res_set_smem(int jtype, size_t bytes);
cudaError_t bq_launch_res(const BqJob& job, int tab_cap, size_t smem, cudaStream_t st);
// Field + decision of one side (side 0 = A uses J, side 1 = B uses J^T).
// decide = 0: no update, only the energy partials of the current state.
// fields_out != null: write F[r][side*n + i] (row stride 2n) and change nothing.
// The sweep index is s, or, when sp is not null, the device value *sp (read at
// kernel start; a decision launch whose sweep is >= S does nothing).
cudaError_t bq_launch_cc_half(const BqJob& job, int side, int s, const int32_t* sp, int decide, float* fields_out,
                              cudaStream_t st);
// End of sweep s (or of sweep *sp_read): energies, running best, snapshots; with
// sp_write, stores the next sweep index there.
// The best state of a replica whose last improvement was sweep s - 1 is copied
// from the parity-(s-1) buffers when sweep s does not improve it (before sweep
// s + 1 overwrites them), so a run of improving sweeps costs one copy.
cudaError_t bq_launch_sweep_end(const BqJob& job, int s, int init, const int32_t* sp_read, int32_t* sp_write,
                                cudaStream_t st);
// After the last sweep (S): copy the replicas whose best is state S - 1.
cudaError_t bq_launch_best_flush(const BqJob& job, cudaStream_t st);
cudaError_t bq_launch_readout(const BqJob& job, int which /*0 final, 1 best*/, int8_t* out_pm, double* out_E,
                              cudaStream_t st);
cudaError_t bq_launch_encode(const BqJob& job, const int8_t* d_states, cudaStream_t st);

}  // namespace pb
