// ea_kernels.cuh -- device-side pieces of the EA (3D Edwards-Anderson,
// periodic L^3 cube) p-bit update, shared by the plain and resident forms.
//
// Spin words: 4 replicas per uint32, one byte each, byte value 0 <=> m = +1,
// 1 <=> m = -1.  Sites of colour c are addressed by their class rank
// k = i >> 1; a class array is [half][WT] words (w fastest).
//
// Field of a +-1 site (Eq. 3): bit b of the 6-bit "pattern" of a replica is
// (neighbour-b spin bit) XOR (bond-b sign bit); it is set exactly when the
// term J_b m_b is negative, so F = 6 - 2 popcount(pattern) (+ h).  The
// pattern of 4 replicas is built at once, shifted to bits 2..7 of each byte,
// so a byte is directly the byte offset of the threshold in a 64-entry
// table of uint32 (Eq. 2 decision).
#pragma once

#include "pb_common.h"

namespace pb {

// Pattern word of 4 replicas: bits (2+b) of every byte <- neighbour b's spin
// byte (0/1), then xor with the site's bond-sign byte broadcast to 4 bytes.
__device__ __forceinline__ uint32_t ea_pattern(uint32_t n0, uint32_t n1, uint32_t n2, uint32_t n3, uint32_t n4,
                                               uint32_t n5, uint32_t jb)
{
    uint32_t p = (n0 << 2) | (n1 << 3) | (n2 << 4) | (n3 << 5) | (n4 << 6) | (n5 << 7);
    return p ^ (jb * 0x01010101u);
}

// Per-byte count of set bits among bits 2..7 (6-bit fields), SWAR.
__device__ __forceinline__ uint32_t ea_popc6_bytes(uint32_t y)
{
    uint32_t v = y >> 2;                       // bits 0..5 of each byte (bits 0,1 of y are zero)
    v = v - ((v >> 1) & 0x15151515u);          // 2-bit counts in pairs (0,1), (2,3), (4,5)
    v = (v & 0x33333333u) + ((v >> 2) & 0x33333333u);
    v = (v + (v >> 4)) & 0x0F0F0F0Fu;
    return v;
}

// Decision of one replica: new spin bit (1 <=> m = -1) is 1 unless r < T.
__device__ __forceinline__ uint32_t decide_bit(uint32_t r, uint32_t T) { return r >= T ? 1u : 0u; }

// 2^x on the special-function unit, results below 2^-126 flushed to zero.
// In the decision below a flushed e cannot change the outcome: u >= 2^-24,
// so u + u e rounds to u < 1 for every e < 2^-126.
__device__ __forceinline__ float ex2_ftz(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// FP32 decision of the F32 path (Eq. 2): m = +1 with probability
// P = 1/2 + tanh(beta F)/2 = 1 / (1 + e^{-2 beta F}).  The word r gives
// u = ((r >> 9) + 1/2) 2^-23, the comparison u < P is evaluated as
// u (1 + e^{-2 beta F}) < 1, so it needs one exp2 and no reciprocal or
// float->int conversion.  It is computed on 2u (exact), whose product
// 2u (1 + e) is >= 2 exactly when u (1 + e) >= 1: the outcome is then bit 30
// of the (positive) result, with no compare.  cexp = -2 beta log2(e).
__device__ __forceinline__ float uniform2_f32(uint32_t r)
{
    return __uint_as_float(0x40000000u | (r >> 9)) - __uint_as_float(0x3FFFFFFFu);  // 2u, exactly
}
// Bits of 2u (1 + e^{-2 beta F}); bit 30 set <=> m = -1.
__device__ __forceinline__ uint32_t decide_f32_bits(uint32_t r, float F, float cexp)
{
    const float u2 = uniform2_f32(r);
    const float e = ex2_ftz(cexp * F);
    return __float_as_uint(fmaf(u2, e, u2));
}
// The new spin bit (1 <=> m = -1).
__device__ __forceinline__ uint32_t decide_f32(uint32_t r, float F, float cexp)
{
    return decide_f32_bits(r, F, cexp) >> 30;
}
// Four decisions as one F32 spin word (byte b = 0x3F for m = +1, 0xBF for
// m = -1, see below): the top bytes of the four results gathered, their bit 6
// (bit 30 of the result) moved to bit 7.
__device__ __forceinline__ uint32_t decide_f32_word(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, float F0,
                                                    float F1, float F2, float F3, float cexp)
{
    const uint32_t v0 = decide_f32_bits(r0, F0, cexp), v1 = decide_f32_bits(r1, F1, cexp);
    const uint32_t v2 = decide_f32_bits(r2, F2, cexp), v3 = decide_f32_bits(r3, F3, cexp);
    const uint32_t g = (__byte_perm(v0, v1, 0x7373u) & 0x0000FFFFu) | (__byte_perm(v2, v3, 0x7373u) & 0xFFFF0000u);
    return 0x3F3F3F3Fu | ((g << 1) & 0x80808080u);
}

// Merge the replicas of one spin word that `flags` selects (byte b = 1: replica b)
// into a global snapshot word: the whole word when all four are selected.
// Otherwise, with BYTES, a byte store per selected replica: the destination is
// never read, so the snapshot does not wait on global memory (the
// read-modify-write did, with every warp of the tile snapshotting after the same
// barrier).  Tiles with one replica word per column (WT = 1) take it: all lanes
// of a warp then hold the same four replicas and take the same branch.  With
// several words per column neighbouring lanes hold different replicas, their
// byte stores diverge, and the read-modify-write measured faster.
template <bool BYTES>
__device__ __forceinline__ void snapshot_word(uint32_t* dst, uint32_t v, uint32_t flags)
{
    if (flags == 0x01010101u) {
        *dst = v;
    } else if constexpr (BYTES) {
        unsigned char* d = reinterpret_cast<unsigned char*>(dst);
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if ((flags >> (8 * b)) & 1u) d[b] = (unsigned char)(v >> (8 * b));
    } else {
        const uint32_t mask = flags * 0xFFu;
        *dst = (*dst & ~mask) | (v & mask);
    }
}

__device__ __forceinline__ float f32_cexp(float beta) { return -2.0f * beta * 1.4426950408889634f; }

// F32 spin words: byte b is the top byte of the float +-1.0 of replica b
// (0x3F <=> m = +1, 0xBF <=> m = -1), so one byte permute yields the spin as
// a float.  (+-1 instances use bytes 0 / 1, see above.)
__device__ __forceinline__ float f32_sign(uint32_t n, int b)
{
    return __uint_as_float(__byte_perm(n, 0x3F800000u, 0x0654u | ((uint32_t)b << 12)));
}
// spin word from four "minus" bits (1 <=> m = -1)
__device__ __forceinline__ uint32_t f32_word(uint32_t s0, uint32_t s1, uint32_t s2, uint32_t s3)
{
    return 0x3F3F3F3Fu | (s0 << 7) | (s1 << 15) | (s2 << 23) | (s3 << 31);
}
__device__ __forceinline__ uint32_t f32_minus(uint32_t n, int b) { return (n >> (8 * b + 7)) & 1u; }

// FP32 local field of replica b (byte b of the neighbour words), Eq. 3, in the
// fixed order h + (+x) + (-x) + (+y) + (-y) + (+z) + (-z); each term is one
// fused multiply-add by the exact +-1.0, i.e. the rounded sum F + (+-J).
__device__ __forceinline__ float ea_field_f32(const float (&jv)[6], float h, const uint32_t (&n)[6], int b)
{
    float F = h;
#pragma unroll
    for (int k = 0; k < 6; ++k) F = fmaf(jv[k], f32_sign(n[k], b), F);
    return F;
}

// Neighbour rank offsets (in sites, inside the other colour's class array) of
// the sites of one column: fixed x = 2q + px and y, z running.
struct EaColumn {
    int dxp, dxm, dyp, dym;  // +x, -x, +y, -y offsets relative to the site's own rank
};

__device__ __forceinline__ EaColumn ea_column(int L, int h2, int q, int y, int px)
{
    EaColumn o;
    o.dxp = px ? ((q + 1 == h2) ? -(h2 - 1) : 1) : 0;
    o.dxm = px ? 0 : ((q == 0) ? (h2 - 1) : -1);
    o.dyp = (y + 1 == L) ? -(L - 1) * h2 : h2;
    o.dym = (y == 0) ? (L - 1) * h2 : -h2;
    return o;
}

}  // namespace pb
