// csr_launch.h -- host/device interface of the p-bit update on general sparse
// instances (arXiv 2510.23419: the general graph of Eq. 1, update groups of
// Sec. 1.2.2 from a proper colouring with k >= 2 colours).
#pragma once

#include "pb_common.h"

namespace pb {

// Device copy of a general instance.  Spins carry labels: the classes are
// listed one after the other, each in ascending original index, and a spin's
// label is its position in that list, so class c is the label range
// cls_off[c] .. cls_off[c+1]-1 and label - cls_off[c] is the class rank (the
// Philox counter word 0).  Each undirected edge (u, v, J) is stored from both
// ends in compressed rows over the labels (+-1 rows: the J = +1 half-edges
// first, each part in edge order); fields and colours are per label.  States
// cross the interface in the original order (orig / pos translate).
struct CsrDevice {
    int32_t N, jtype, n_colours, maxdeg, has_h, hmax;
    const int32_t* rowptr;   // [N + 1] rows by label
    const int32_t* rowneg;   // PM1: [N] first half-edge of row i with J = -1 (J = +1 ones come first)
    const int32_t* col;      // [2E] neighbour of each half-edge
    const int8_t* J8;        // [2E] +-1 couplings (PM1)
    const float* Jf;         // [2E] real couplings (F32)
    const int8_t* h8;        // [N] or null (PM1)
    const float* hf;         // [N] or null (F32)
    const int32_t* cls_off;  // [n_colours + 1] first label of each class
    const int32_t* orig;     // [N] original index of label p
    const int32_t* pos;      // [N] label of original vertex i
    const int32_t* colour;   // [N] colour of label p
    // +-1 instances of degree <= kCsrEllSlots (else null): row p as kCsrEllSlots
    // labels (the J = +1 neighbours first), unused slots naming label N, whose
    // spin words are kept zero; ell_nd[p] = (J = +1 count) | degree << 8
    const int4* ell;         // [N][kCsrEllSlots / 4]
    const uint16_t* ell_nd;  // [N]
};

// Spin words: 4 replicas per uint32, one byte each, byte = 0 <=> m = +1,
// 1 <=> m = -1; state [N][Rw], Rw = ceil(R / 4), replica r in byte r % 4 of word r / 4.
struct CsrJob {
    CsrDevice g;
    uint32_t key0, key1;
    int32_t S, step, nF, fmin;
    int32_t s0;              // first sweep (0, or the sweep a resumed run continues from)
    const uint32_t* table;   // PM1: threshold windows of all levels, concatenated
    const int32_t* win;      // PM1: [levels][3] (lo, width, off)
    const float* betaf;      // F32: [levels]
    int32_t R, Rw;
    uint32_t* spins;         // [N][Rw] (+ one zero row, label N, for the padded rows)
    uint32_t* best;          // [N][Rw]
    int32_t nchunk;          // vertex chunks of the energy partials
    double* part;            // [nchunk][4 Rw] energy partials (PM1: 2E as exact integers)
    int32_t ndchunk;         // class chunks of the sweep's energy changes, over all classes
    const int32_t* dchunk_off;  // [n_colours + 1] first class chunk of each class
    double* dpart;           // F32: [ndchunk][4 Rw] energy change of each class chunk in the last sweep
    unsigned long long* dacc;  // PM1: [4 Rw] energy change of the sweep so far (int64 two's complement)
    double* E_best;          // [4 Rw]
    int32_t* best_sweep;     // [4 Rw]
    int32_t* hit_sweep;      // [4 Rw]
    uint8_t* improved;       // [4 Rw] + 1 "any" flag at [4 Rw]
    int32_t has_target;        // 0 none, 1 record the target sweep, 2 also stop there (see pbit.h)
    int32_t* stop;             // has_target == 2: [0] replicas that reached the target, [1] the sweep after
                               // which all had (-1 while running); later launches return at once
    double target;
    double* E_cur;             // [4 Rw] energy after the last sweep
    // parallel tempering (null temp: annealing with the schedule)
    uint8_t* temp;             // [4 Rw] temperature index of every slot (= replica)
    int32_t* slot_of;          // [M][C] slot holding temperature t of chain r
    int32_t M, C;              // temperatures, chains; slot g = k C + r starts at temperature k
    const float* xdb;          // [M-1] (beta_{t+1} - beta_t) log2 e, rounded to FP32 (real couplings)
    const uint32_t* xtab;      // +-1: exchange thresholds floor(exp(dbeta_t * (-d)) 2^32), d = 1, 2, ...
    const int32_t* xwin;       // +-1: [M-1][2] (length, offset) of pair t's thresholds in xtab
    unsigned long long* n_accept;  // [M-1] accepted exchanges per pair
};

constexpr int kCsrChunk = 64;  // vertices per energy chunk
constexpr int kCsrLanesQ = 32;  // class kernel: replica words per block
constexpr int kCsrLanesV = 8;   // class kernel: vertex lanes per block
constexpr int kCsrEllSlots = 8;  // padded rows for +-1 instances of degree <= 8
constexpr int kCsrMaxVpt = 16;  // class kernel: most class spins one thread takes in a launch

cudaError_t csr_launch_init(const CsrJob& job, cudaStream_t st);
// Blocks (class chunks) of one class launch for a class of ncls spins: whole
// waves of resident blocks (SMs x blocks per SM of the kernel variant), at most
// kCsrMaxVpt spins per thread; a function of the device and the shapes only, so
// a run's energy partials are summed in the same order whatever runs beside it.
// -1 on a CUDA error.
int csr_class_blocks(int jtype, bool temp, int Rw, int ncls, int maxdeg, int hmax);
// Update of colour class c in sweep s (Eq. 2, Eq. 3) and its energy changes
// (nchunks = csr_class_blocks(...) of the class).
cudaError_t csr_launch_class(const CsrJob& job, int c, int nchunks, int s, cudaStream_t st);
// Energy partials of the state `m` ([N][Rw] words); exact FP64 per term when exact != 0.
cudaError_t csr_launch_energy(const CsrJob& job, const uint32_t* m, int exact, cudaStream_t st);
// Parallel tempering: exchange of temperatures between adjacent pairs of every
// chain after sweep s (pairs t = s mod 2, t + 2, ...).
cudaError_t csr_launch_exchange(const CsrJob& job, int s, cudaStream_t st);
// Running best after sweep s (init 1: the initial state, whose energy comes from
// csr_launch_energy, becomes the best; init 2: a resumed run's state, whose
// energy is set and whose given best is kept; init 0: later sweeps add the class
// launches' energy changes to the previous energy) and the improved flags.  The
// next sweep's class launches copy the flagged replicas' state into the best
// state as they read it; csr_launch_snapshot does so after the last sweep.
cudaError_t csr_launch_sweep_end(const CsrJob& job, int s, int init, cudaStream_t st);
cudaError_t csr_launch_snapshot(const CsrJob& job, cudaStream_t st);
// States [R][N] int8 +-1 and energies (from the partials of the same state) of `m`.
cudaError_t csr_launch_readout(const CsrJob& job, const uint32_t* m, int8_t* out_pm, double* out_E, cudaStream_t st);
// Fields F[r][i] = sum_j J_ij m_j + h_i of given +-1 states [R][N] (written as [R][N] float).
cudaError_t csr_launch_fields(const CsrJob& job, const int8_t* states, float* out, cudaStream_t st);

}  // namespace pb
