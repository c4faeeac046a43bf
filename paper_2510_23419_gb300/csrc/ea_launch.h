// ea_launch.h -- host/device interface of the EA (periodic L^3 cube) kernels.
#pragma once

#include "pb_common.h"

namespace pb {

// One anneal job as the kernels see it (plain form: one tile with WT = R/4
// rounded up; resident form: tiles of 4*WT replicas).  State buffers use the
// tile layout: word ((tile*2 + c)*half + k)*WT + w holds replicas
// tile*4*WT + 4w + (0..3) of the site of colour c and class rank k.
struct EaJob {
    EaDevice inst;
    uint32_t key0, key1;      // Philox key = seed
    int32_t S;                // sweeps
    int32_t step;             // sweeps per beta level (1 for explicit schedules)
    int32_t nF;               // PM1: threshold table width (F_max - F_min + 1)
    int32_t fmin;             // PM1: F_min
    const uint32_t* table;    // PM1: [levels][nF] thresholds
    const float* betaf;       // F32: [levels] beta as float
    int32_t R;                // replicas requested
    int32_t WT;               // words (4 replicas each) per site in one tile
    int32_t n_tiles;
    int32_t has_target;       // 0: none; 1: record the first sweep at the target; 2: also freeze the
                              // running best there and stop once every replica has reached it
    int32_t target_i;         // PM1 target energy (integer)
    float target_f;           // F32 target energy
    uint32_t* best_words;     // tile layout
    uint32_t* final_words;    // tile layout (plain form: the live state)
    int32_t* E_best_i;        // PM1 running-best energy  [n_tiles*4*WT]
    float* E_best_f;          // F32 running-best energy
    int32_t* best_sweep;      // [n_tiles*4*WT]
    int32_t* hit_sweep;       // [n_tiles*4*WT]
    int32_t* n_hit;           // plain form, has_target == 2: replicas that reached the target (device counter)
    int32_t s0;               // first sweep (resident form: > 0 only for a resumed run)
    int32_t resume;           // resident form: the initial state is final_words, the running best
                              // (best_words, E_best_*, best_sweep) is given
};

// Tile code of the resident kernels (chosen on the host, so the kernel
// branches on one word of the work item).
enum EaTilePath : int32_t {
    kEaPathFieldsGeneric = 0,  // +-1 couplings with integer fields: generic tile
    kEaPathFast32 = 1,         // compile-time tile L = 32, WT = 1
    kEaPathFast16 = 2,         // L = 16, WT = 4
    kEaPathFast8 = 3,          // L = 8, WT = 16
    kEaPathGeneric = 4,        // any other even L <= 32
    kEaPathGen12 = 6,          // generic tile with compile-time L = 12, WT = 4 (+-1 kernel; FP32: generic)
    kEaPathFast24 = 7,         // compile-time tile L = 24, WT = 1 (576 of the CTA's threads hold sites)
};

struct EaWork {
    int32_t job;
    int32_t tile;
    int32_t path;  // EaTilePath of the job
};

inline int32_t ea_tile_path(const EaJob& j)
{
    if (j.inst.jtype == PB_J_PM1_I8 && j.inst.has_h) return kEaPathFieldsGeneric;
    if (j.inst.L == 32 && j.WT == 1) return kEaPathFast32;
    if (j.inst.L == 16 && j.WT == 4) return kEaPathFast16;
    if (j.inst.L == 8 && j.WT == 16) return kEaPathFast8;
    if (j.inst.L == 24 && j.WT == 1) return kEaPathFast24;
    if (j.inst.L == 12 && j.WT == 4) return kEaPathGen12;
    return kEaPathGeneric;
}

// Persistent resident kernels: one for +-1 couplings and two for FP32, which
// differ in their compile-time tiles -- the L = 32 tile, or the L = 24 tile,
// beside L = 16, L = 8 and the runtime-shaped generic tile.  With both the
// L = 32 and the L = 24 tile in one kernel, the register allocation they share
// slowed the L = 32 tile by 8%.  A batch takes the L = 24 kernel when its FP32
// tiles include L = 24 ones and no L = 32 ones; otherwise L = 24 FP32 tiles
// run the generic tile of the first kernel.
enum EaKernel : int32_t { kEaKernelPm1 = 0, kEaKernelF32 = 1, kEaKernelF32L24 = 2, kEaKernels = 3 };

// Shared memory of one resident tile, in bytes.
__host__ __device__ inline size_t ea_resident_smem(int L, int WT, int jtype, int has_h, int nF)
{
    const size_t N = (size_t)L * L * L;
    size_t b = N * (size_t)WT * 4;                       // spins [2][half][WT]
    if (jtype == PB_J_PM1_I8) {
        b += (N + 15) / 16 * 16;                         // bond-sign bytes [2][half]
        if (has_h) b += (N + 15) / 16 * 16;              // h bytes
    }
    const int tabw = (jtype == PB_J_PM1_I8) ? (has_h ? nF : 64) : 0;
    b += (size_t)2 * ((tabw + 3) / 4 * 4) * 4;           // double-buffered threshold row
    b += (size_t)(1024 / 32) * 4 * WT * 4;               // per-warp energy partials
    if (jtype == PB_J_PM1_I8 && has_h) b += (size_t)(1024 / 32) * 4 * WT * 4;  // per-warp h.m partials
    b += (size_t)4 * WT;                                 // improved flags
    // compile-time-shaped tiles keep their bond bytes as [2][L/8][threads] words
    const bool fast =
        !has_h && ((L == 32 && WT == 1) || (L == 16 && WT == 4) || (L == 8 && WT == 16) || (L == 24 && WT == 1));
    if (fast && jtype == PB_J_PM1_I8) {
        const size_t f = N * (size_t)WT * 4 + (size_t)(1024 / 32) * 4 * WT * 4 + 128 + (size_t)2 * (L / 8) * 1024 * 4;
        if (f > b) b = f;
    }
    return (b + 127) / 128 * 128;
}

constexpr int kResidentThreads = 1024;
constexpr int kResidentWarpsH = kResidentThreads / 32;
constexpr int kResidentMaxWT = 32;
constexpr size_t kResidentSmemLimit = 227 * 1024;

// Largest power-of-two WT <= min(32, cap) such that the column-words of a
// class fit half the CTA (h2*L*WT <= kResidentThreads/2: two threads, one per
// z parity, per column) and the tile fits shared memory; 0 if none.
int ea_resident_pick_wt(int L, int jtype, int has_h, int nF, int cap_words);

// Opt the persistent kernel `kernel` (EaKernel) into `smem` bytes of dynamic
// shared memory (outside any capture).
cudaError_t ea_resident_set_smem(int kernel, size_t smem);
// Persistent kernel `kernel` (EaKernel) over n_work items of its coupling
// type.  after_previous: programmatic dependent launch on the kernel launched
// just before it on `st` (its CTAs start as that kernel's CTAs leave; the
// caller orders any later consumer after both).
cudaError_t ea_launch_resident(int kernel, const EaJob* d_jobs, const EaWork* d_work, int n_work, int* d_counter,
                               size_t smem, int grid, bool after_previous, cudaStream_t st);
// Random-word ceiling: `blocks` CTAs of kResidentThreads threads, each thread drawing the
// decision words of 32 sites (one L = 32 column, both colours) per sweep; sink holds
// blocks * kResidentThreads words.  Updates counted: blocks * kResidentThreads * 32 * 4 per sweep.
cudaError_t ea_launch_philox_ceiling(uint64_t seed, int sweeps, int blocks, uint32_t* sink, cudaStream_t st);
cudaError_t ea_launch_plain_init(const EaJob& job, cudaStream_t st);
cudaError_t ea_launch_plain_sweep(const EaJob& job, int s, cudaStream_t st);
cudaError_t ea_launch_plain_energy(const EaJob& job, int s, bool init, cudaStream_t st);
// Tile layout -> [R][N] int8 +-1, and energies recomputed from those states
// (int64 for PM1, FP64 for F32).
cudaError_t ea_launch_readout(const EaJob& job, const uint32_t* words, int8_t* out_pm, double* out_E,
                              cudaStream_t st);
cudaError_t ea_launch_fields(const EaDevice& inst, const int8_t* d_states, int R, float* d_out, cudaStream_t st);

}  // namespace pb
