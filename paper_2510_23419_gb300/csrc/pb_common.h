// pb_common.h -- internal definitions shared by the host runtime and the
// sm_103a kernels of the p-bit annealer (arXiv 2510.23419).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pbit.h"

#define PB_HD __host__ __device__ __forceinline__

namespace pb {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Each round multiplies
// counter words 0 and 2 by the published constants (32x32 -> 64 bits), xors
// the high halves into words 1 and 3 together with the round key, and swaps;
// the key advances by the published Weyl increments between rounds.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u;
constexpr uint32_t kPhiloxWeylB = 0xBB67AE85u;

struct U4 {
    uint32_t x, y, z, w;
};

PB_HD void mulhilo32(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

PB_HD U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        uint32_t hA, lA, hB, lB;
        mulhilo32(kPhiloxMulA, c0, hA, lA);
        mulhilo32(kPhiloxMulB, c2, hB, lB);
        const uint32_t n0 = hB ^ c1 ^ k0;
        const uint32_t n2 = hA ^ c3 ^ k1;
        c0 = n0;
        c1 = lB;
        c2 = n2;
        c3 = lA;
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }
    return U4{c0, c1, c2, c3};
}

// Threshold window of one beta level (+-1 couplings): the row T[F - F_min]
// restricted to indices [lo, lo + width), stored at table + off; indices
// outside the window take the value at its nearer edge.
struct TabWindow {
    int32_t off, lo, width;
};

// Stream tags (counter word 3, bits 24..31).
constexpr uint32_t kTagDecision = 0u;
constexpr uint32_t kTagInit = 1u;
constexpr uint32_t kTagInstance = 2u;

// ---------------------------------------------------------------------------
// Internal status plumbing (host only).
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
pb_status fail(pb_status st, const std::string& msg);
pb_status cuda_fail(cudaError_t e, const char* what);

#define PB_CUDA_TRY(call)                                    \
    do {                                                     \
        cudaError_t pb_e_ = (call);                          \
        if (pb_e_ != cudaSuccess) return ::pb::cuda_fail(pb_e_, #call); \
    } while (0)

// Bond order of an EA site inside the kernels: +x, -x, +y, -y, +z, -z.
constexpr int kEaDegree = 6;

// Device copy of one EA instance in the kernels' layouts.  Sites of colour c
// are stored by their class rank k = i >> 1 (a bijection for even L).
struct EaDevice {
    int32_t L, N, half;     // N = L^3, half = N/2
    int32_t jtype;          // pb_jtype
    int32_t has_h;          // PM1: an int8 field is present
    int32_t hmax;           // PM1: max |h|
    const uint8_t* jbits;   // PM1 [2][half]: bit (2+b) set <=> bond b negative (pre-shifted by 2)
    const int8_t* h8;       // PM1 [2][half] or null
    const float* j6;        // F32 [2][half][8]: 6 bond values, h (0 without a field), 1 pad per site
    const float* hf;        // F32 [2][half] (zeros when no field)
    const void* J3;         // original layout [3][N] (int8 or float) for the energy recompute
    const void* hraw;       // original layout [N] (int8 or float) or null
};

}  // namespace pb
