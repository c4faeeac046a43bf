// biclique_tc.h -- host interface of the tcgen05 biclique field kernel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "biclique_launch.h"

namespace pb {

// TMA descriptors of one run: a[0], a[1] = J (e4m3, or bf16 hi and lo),
// a[2], a[3] = J^T; b[2 side + parity] = the live spin buffers.
struct BqTcMaps {
    CUtensorMap a[4];
    CUtensorMap b[4];
};

constexpr int kBqTcRows = 128;   // rows of a tile (tensor-memory lanes)
constexpr int kBqTcReps = 256;   // replicas of a tile (accumulator columns)
constexpr int kBqTcWindowMax = 256;  // widest threshold window kept as 32 conflict-free copies

size_t bq_tc_smem_bytes(int kind);
cudaError_t bq_tc_set_smem();
cudaError_t bq_tc_make_map(CUtensorMap* map, const void* base, int elem_bytes, uint64_t cols, uint64_t rows,
                           uint64_t ld_bytes, int box_rows);
// The sweep index is s, or the device value *sp when sp is not null (see
// bq_launch_cc_half); the threshold windows are read from job.win, from where
// job.tabmode says (0 global, 1 shared, 2 shared with 32 copies).
// bsel: index in maps.b of the other side's spins (the B operand); job.spins
// must name the matching buffers.
cudaError_t bq_launch_tc_half(const BqTcMaps& maps, int bsel, const BqJob& job, int side, int s, const int32_t* sp,
                              int decide, float* fields_out, int* err, cudaStream_t st);
// CTA pairs a half-sweep launch of an n x n biclique with Rpad replicas occupies
// (kind 0 e4m3, 1 split BF16; split: the last round's tiles halved).
int bq_tc_clusters(int n, int Rpad, int kind, bool split);
// Whether a half-sweep launch of an n x n biclique with Rpad replicas has at
// least one 256-replica tile for every CTA pair that fits on the device.
bool bq_tc_fills_device(int n, int Rpad, int kind);

}  // namespace pb
