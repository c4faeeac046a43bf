// ea_fast.cuh -- compile-time-shaped resident tile of the EA p-bit update
// (arXiv 2510.23419: Eqs. 2-3, update groups of Sec. 1.2.2, classical
// annealing of Sec. 1.3.1) for cubes whose colour-class columns exactly fill
// half the CTA: thread (cw, zp) owns the column (q, y, w) for z = zp mod 2 of
// both colours, i.e. the sites x = 2q + parity, fixed y, every other z, for 4
// replicas.
//
// Shapes whose columns fill fewer than half the CTA (L = 24: 288 column-words,
// 576 of the 1024 threads) leave the remaining warps without sites: they take
// part in the barriers and add zero energy partials.
//
// Same arithmetic, random words and outputs as the generic tile; what changes
// is only the instruction budget:
//  * x and y neighbours (and their periodic wrap) are per-thread bases, the
//    two z-wrapping sites are peeled out of the z loop;
//  * the Philox round keys live in registers, and the first round's products
//    of counter words 1..3 (sweep, replica quad, colour) are hoisted;
//  * the thread's bond-sign bytes live in registers (one PRMT broadcasts a
//    site's byte to the 4 replica lanes);
//  * the threshold row sits at a fixed shared address.
#pragma once

#include <type_traits>

#include "ea_kernels.cuh"
#include "ea_launch.h"

namespace pb {

struct RoundKeys {
    uint32_t k0[10], k1[10];
};

__device__ __forceinline__ RoundKeys round_keys(uint32_t key0, uint32_t key1)
{
    RoundKeys k;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = key0 + (uint32_t)r * kPhiloxWeylA;
        k.k1[r] = key1 + (uint32_t)r * kPhiloxWeylB;
    }
    return k;
}

// First-round terms that do not depend on counter word 0.
struct PhiloxPre {
    uint32_t n0, n1, x3;
};

__device__ __forceinline__ PhiloxPre philox_pre(uint32_t c1, uint32_t c2, uint32_t c3, const RoundKeys& k)
{
    uint32_t hB, lB;
    mulhilo32(kPhiloxMulB, c2, hB, lB);
    return PhiloxPre{hB ^ c1 ^ k.k0[0], lB, c3 ^ k.k1[0]};
}

// Philox4x32-10 of counter (c0, c1, c2, c3), with (c1, c2, c3) folded into `p`.
__device__ __forceinline__ U4 philox_c0(uint32_t c0, const PhiloxPre& p, const RoundKeys& k)
{
    uint32_t hA, lA;
    mulhilo32(kPhiloxMulA, c0, hA, lA);
    uint32_t x0 = p.n0, x1 = p.n1, x2 = hA ^ p.x3, x3 = lA;
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        uint32_t hA2, lA2, hB2, lB2;
        mulhilo32(kPhiloxMulA, x0, hA2, lA2);
        mulhilo32(kPhiloxMulB, x2, hB2, lB2);
        const uint32_t y0 = hB2 ^ x1 ^ k.k0[r];
        const uint32_t y2 = hA2 ^ x3 ^ k.k1[r];
        x0 = y0;
        x1 = lB2;
        x2 = y2;
        x3 = lA2;
    }
    return U4{x0, x1, x2, x3};
}

constexpr int kResidentWarps = kResidentThreads / 32;

template <int L, int WT, int JT>
struct EaFastTile {
    static constexpr int T = kResidentThreads;
    static constexpr int h2 = L / 2;
    static constexpr int CWN = h2 * L * WT;  // column-words: two threads (z parities) per column
    static constexpr int TB = 2 * CWN;       // threads with sites; the others only join the barriers
    static constexpr bool kAllBusy = TB == kResidentThreads;
    static constexpr int half = h2 * L * L;
    static constexpr int N = 2 * half;
    static_assert(TB <= T && TB % 32 == 0 && L % 8 == 0, "fast tile: whole warps of column-word pairs");
    static constexpr int SZ = L * h2 * WT;  // words between z planes of a class array
    static constexpr int CLS = half * WT;   // words of one class array
    static constexpr int NREP = 4 * WT;
    static constexpr int NW = kResidentWarps;
    static constexpr bool PM1 = JT == PB_J_PM1_I8;

    const EaJob& job;
    int tile, t, lane, warp, w, q, y, zp, base0, oyp, oym;
    bool busy;  // the thread owns a column-word (always, when the columns fill the CTA)
    uint32_t tq;
    uint32_t* sp;
    int32_t* spart_i;
    float* spart_f;
    uint8_t* sflag;
    uint32_t* s_tab;
    RoundKeys rk;
    const uint32_t* sjb4;  // bond-sign bytes of the thread's sites: word [(c*L/8 + zz/4)*T + t] byte zz%4, z = zp + 2 zz

    __device__ __forceinline__ EaFastTile(const EaJob& j, int tile_, unsigned char* smem, uint32_t* tab)
        : job(j), tile(tile_), s_tab(tab)
    {
        t = threadIdx.x;
        lane = t & 31;
        warp = t >> 5;
        busy = kAllBusy || t < TB;
        const int cw = t % CWN;
        zp = t / CWN;
        w = cw % WT;
        q = (cw / WT) % h2;
        y = cw / (WT * h2);
        sp = reinterpret_cast<uint32_t*>(smem);
        spart_i = reinterpret_cast<int32_t*>(sp + N * WT);
        spart_f = reinterpret_cast<float*>(spart_i);
        sflag = reinterpret_cast<uint8_t*>(spart_i + NW * NREP);
        rk = round_keys(job.key0, job.key1);
        tq = (uint32_t)(tile * WT + w);
        base0 = (q + h2 * y) * WT + w;
        oyp = ((y + 1 == L) ? -(L - 1) * h2 : h2) * WT;
        oym = ((y == 0) ? (L - 1) * h2 : -h2) * WT;
        uint32_t* jw = reinterpret_cast<uint32_t*>(sflag + 128);
        sjb4 = jw;
        if (PM1 && (kAllBusy || busy)) {
#pragma unroll 1
            for (int c = 0; c < 2; ++c)
#pragma unroll 1
                for (int z4 = 0; z4 < L / 8; ++z4) {
                    uint32_t v = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int z = zp + 2 * (4 * z4 + b);
                        v |= (uint32_t)job.inst.jbits[c * half + q + h2 * (y + L * z)] << (8 * b);
                    }
                    jw[(c * (L / 8) + z4) * T + t] = v;
                }
        }
    }

    __device__ __forceinline__ void init_state()
    {
        if constexpr (!kAllBusy)
            if (!busy) return;
        if (job.resume) {  // resumed run: the given state, in the tile layout of final_words
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const uint32_t* src = job.final_words + ((size_t)tile * 2 + c) * CLS + base0;
                for (int z = zp; z < L; z += 2) sp[c * CLS + base0 + z * SZ] = src[z * SZ];
            }
            return;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll 4
            for (int z = zp; z < L; z += 2) {
                const int k = q + h2 * (y + L * z);
                const U4 r = philox10((uint32_t)k, 0u, tq, (kTagInit << 24) | (uint32_t)c, job.key0, job.key1);
                sp[c * CLS + base0 + z * SZ] =
                    PM1 ? ((r.x >> 31) | ((r.y >> 31) << 8) | ((r.z >> 31) << 16) | ((r.w >> 31) << 24))
                        : f32_word(r.x >> 31, r.y >> 31, r.z >> 31, r.w >> 31);
            }
    }

    __device__ __forceinline__ void load_table(int s)
    {
        if (PM1 && t < 64) {
            const uint32_t* row = job.table + (size_t)(s / job.step) * job.nF;
            s_tab[t] = row[6 - 2 * __popc((unsigned)t) - job.fmin];
        }
    }

    // One colour class: update (DECIDE) or only accumulate the energy terms of
    // the current state.  PM1: unsatisfied bonds of class-1 sites in byte lanes;
    // F32: -m F over class 1 and -h m over class 0.
    template <int C, bool DECIDE>
    __device__ __forceinline__ void half_sweep(int s, uint32_t& uacc, float (&ef)[4])
    {
        if constexpr (!kAllBusy)
            if (!busy) return;
        const uint32_t* o = sp + (1 - C) * CLS;
        uint32_t* own = sp + C * CLS;
        const int zp = this->zp;
        const PhiloxPre pre = philox_pre((uint32_t)s, tq, (kTagDecision << 24) | (uint32_t)C, rk);
        float cexp = 0.0f;
        if constexpr (!PM1) cexp = f32_cexp(job.betaf[s / job.step]);
        {
            const int px = (C + y + zp) & 1;
            const int oxp = (px ? ((q + 1 == h2) ? -(h2 - 1) : 1) : 0) * WT;
            const int oxm = (px ? 0 : ((q == 0) ? (h2 - 1) : -1)) * WT;
            const uint32_t* bxp = o + base0 + oxp;
            const uint32_t* bxm = o + base0 + oxm;
            const uint32_t* byp = o + base0 + oyp;
            const uint32_t* bym = o + base0 + oym;
            const uint32_t* bz = o + base0;
            // the wrapping sites (z = 0 for the even pass, z = L-1 for the odd pass) are
            // peeled; the others take their z neighbours at z +- 1.  Two +-1 sites per
            // iteration let their Philox chains overlap (no spills at 64 registers); the
            // FP32 sites hold their couplings too and would spill, so they go one at a time.
            if (zp == 0) site<C, DECIDE>(0, 1, L - 1, bxp, bxm, byp, bym, bz, own, pre, cexp, uacc, ef);
            if constexpr (PM1) {
#pragma unroll 2
                for (int z = 2 - zp; z < L - 1 - zp; z += 2)
                    site<C, DECIDE>(z, z + 1, z - 1, bxp, bxm, byp, bym, bz, own, pre, cexp, uacc, ef);
            } else {
#pragma unroll 1
                for (int z = 2 - zp; z < L - 1 - zp; z += 2)
                    site<C, DECIDE>(z, z + 1, z - 1, bxp, bxm, byp, bym, bz, own, pre, cexp, uacc, ef);
            }
            if (zp == 1) site<C, DECIDE>(L - 1, 0, L - 2, bxp, bxm, byp, bym, bz, own, pre, cexp, uacc, ef);
        }
    }

    template <int C, bool DECIDE>
    __device__ __forceinline__ void site(int z, int zup, int zdn, const uint32_t* bxp, const uint32_t* bxm,
                                         const uint32_t* byp, const uint32_t* bym, const uint32_t* bz, uint32_t* own,
                                         const PhiloxPre& pre, float cexp, uint32_t& uacc, float (&ef)[4])
    {
        const int k = q + h2 * (y + L * z);
        const uint32_t n0 = bxp[z * SZ], n1 = bxm[z * SZ], n2 = byp[z * SZ], n3 = bym[z * SZ];
        const uint32_t n4 = bz[zup * SZ], n5 = bz[zdn * SZ];
        uint32_t snew;
        if constexpr (PM1) {
            const int zz = z >> 1;
            const uint32_t jb = __byte_perm(jword<C>(zz >> 2), 0u, (uint32_t)(zz & 3) * 0x1111u);
            const uint32_t X = ((n0 << 2) | (n1 << 3) | (n2 << 4) | (n3 << 5) | (n4 << 6) | (n5 << 7)) ^ jb;
            if constexpr (DECIDE) {
                const U4 r = philox_c0((uint32_t)k, pre, rk);
                const unsigned char* tb = reinterpret_cast<const unsigned char*>(s_tab);
                const uint32_t T0 = *reinterpret_cast<const uint32_t*>(tb + (X & 0xFFu));
                const uint32_t T1 = *reinterpret_cast<const uint32_t*>(tb + __byte_perm(X, 0u, 0x4441u));
                const uint32_t T2 = *reinterpret_cast<const uint32_t*>(tb + __byte_perm(X, 0u, 0x4442u));
                const uint32_t T3 = *reinterpret_cast<const uint32_t*>(tb + (X >> 24));
                snew = decide_bit(r.x, T0) + decide_bit(r.y, T1) * 0x100u + decide_bit(r.z, T2) * 0x10000u +
                       decide_bit(r.w, T3) * 0x1000000u;
                own[base0 + z * SZ] = snew;
            } else {
                snew = own[base0 + z * SZ];
            }
            if (C == 1) uacc += ea_popc6_bytes(X ^ (snew * 0xFCu));
        } else {
            const size_t site_i = (size_t)C * half + k;
            const float4 ja = __ldg(reinterpret_cast<const float4*>(job.inst.j6) + 2 * site_i);
            const float4 jb = __ldg(reinterpret_cast<const float4*>(job.inst.j6) + 2 * site_i + 1);
            const float jv[6] = {ja.x, ja.y, ja.z, ja.w, jb.x, jb.y};
            const float hv = jb.z;  // the site's field rides in the coupling vector
            const uint32_t nb[6] = {n0, n1, n2, n3, n4, n5};
            float F[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) F[b] = ea_field_f32(jv, hv, nb, b);
            if constexpr (DECIDE) {
                const U4 r = philox_c0((uint32_t)k, pre, rk);
                snew = decide_f32_word(r.x, r.y, r.z, r.w, F[0], F[1], F[2], F[3], cexp);
                own[base0 + z * SZ] = snew;
            } else {
                snew = own[base0 + z * SZ];
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float m = f32_sign(snew, b);  // -m F (class 1), -h m (class 0)
                if (C == 1)
                    ef[b] = fmaf(-m, F[b], ef[b]);
                else if (job.inst.has_h)
                    ef[b] = fmaf(-m, hv, ef[b]);
            }
        }
    }

    // bond-sign bytes of 4 consecutive z of the thread's colour-C column
    template <int C>
    __device__ __forceinline__ uint32_t jword(int z4) const
    {
        return sjb4[(C * (L / 8) + z4) * T + t];
    }

    __device__ __forceinline__ void partials(uint32_t uacc, const float (&ef)[4])
    {
        if constexpr (PM1) {
            uint32_t a = uacc & 0x00FF00FFu, b = (uacc >> 8) & 0x00FF00FFu;
#pragma unroll
            for (int o2 = WT; o2 < 32; o2 <<= 1) {
                a += __shfl_xor_sync(0xFFFFFFFFu, a, o2);
                b += __shfl_xor_sync(0xFFFFFFFFu, b, o2);
            }
            if (lane < WT) {
                int32_t* p = spart_i + warp * NREP + 4 * lane;
                p[0] = (int32_t)(a & 0xFFFFu);
                p[1] = (int32_t)(b & 0xFFFFu);
                p[2] = (int32_t)(a >> 16);
                p[3] = (int32_t)(b >> 16);
            }
        } else {
            float v0 = ef[0], v1 = ef[1], v2 = ef[2], v3 = ef[3];
#pragma unroll
            for (int o2 = WT; o2 < 32; o2 <<= 1) {
                v0 += __shfl_xor_sync(0xFFFFFFFFu, v0, o2);
                v1 += __shfl_xor_sync(0xFFFFFFFFu, v1, o2);
                v2 += __shfl_xor_sync(0xFFFFFFFFu, v2, o2);
                v3 += __shfl_xor_sync(0xFFFFFFFFu, v3, o2);
            }
            if (lane < WT) {
                float* p = spart_f + warp * NREP + 4 * lane;
                p[0] = v0;
                p[1] = v1;
                p[2] = v2;
                p[3] = v3;
            }
        }
    }

    __device__ __forceinline__ void energy_of(int r, int32_t& Ei, float& Ef) const
    {
        if constexpr (PM1) {
            int32_t U = 0;
#pragma unroll
            for (int v = 0; v < NW; ++v) U += spart_i[v * NREP + r];
            Ei = -(3 * N - 2 * U);
        } else {
            float E = 0.0f;
#pragma unroll
            for (int v = 0; v < NW; ++v) E += spart_f[v * NREP + r];
            Ef = E;
        }
    }

    // the thread's words of both colours into a global state buffer, the replicas
    // that `flags` selects (byte b = 1: replica 4w + b; 0x01010101: all four)
    __device__ __forceinline__ void store_words(uint32_t* gdst, uint32_t flags) const
    {
        if (flags == 0u || (!kAllBusy && !busy)) return;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            uint32_t* dst = gdst + ((size_t)tile * 2 + c) * CLS + base0;
            const uint32_t* src = sp + c * CLS + base0;
#pragma unroll 4
            for (int z = zp; z < L; z += 2) snapshot_word<WT == 1>(dst + z * SZ, src[z * SZ], flags);
        }
    }

    __device__ __forceinline__ void run()
    {
        init_state();
        load_table(job.s0 < job.S ? job.s0 : 0);
        __syncthreads();
        {
            uint32_t uacc = 0;
            float ef[4] = {0.f, 0.f, 0.f, 0.f};
            half_sweep<0, false>(0, uacc, ef);
            half_sweep<1, false>(0, uacc, ef);
            partials(uacc, ef);
        }
        __syncthreads();
        int32_t bestEi = 0, hit = -1, bsweep = -1;
        float bestEf = 0.0f;
        if (t < NREP) energy_of(t, bestEi, bestEf);
        if (job.resume) {  // the running best carried over
            if (t < NREP) {
                const int r = tile * NREP + t;
                if constexpr (PM1)
                    bestEi = job.E_best_i[r];
                else
                    bestEf = job.E_best_f[r];
                bsweep = job.best_sweep[r];
            }
        } else {
            store_words(job.best_words, 0x01010101u);
        }

        const bool stop_mode = job.has_target == 2;
        for (int s = job.s0; s < job.S; ++s) {
            uint32_t uacc = 0;
            float ef[4] = {0.f, 0.f, 0.f, 0.f};
            half_sweep<0, true>(s, uacc, ef);
            __syncthreads();
            half_sweep<1, true>(s, uacc, ef);
            partials(uacc, ef);
            __syncthreads();
            if (t < NREP) {
                int32_t Ei = 0;
                float Ef = 0.0f;
                energy_of(t, Ei, Ef);
                const bool live = job.has_target != 2 || hit < 0;  // stop mode: the best is frozen at the target
                bool imp;
                if constexpr (PM1) {
                    imp = live && Ei < bestEi;
                    if (imp) bestEi = Ei;
                    if (job.has_target && hit < 0 && Ei <= job.target_i) hit = s;
                } else {
                    imp = live && Ef < bestEf;
                    if (imp) bestEf = Ef;
                    if (job.has_target && hit < 0 && Ef <= job.target_f) hit = s;
                }
                if (imp) bsweep = s;
                sflag[t] = imp ? 1 : 0;
            }
            if (s + 1 < job.S) load_table(s + 1);  // row s was last read before the barrier above
            __syncthreads();
            const uint32_t f = reinterpret_cast<const uint32_t*>(sflag)[w];
            store_words(job.best_words, f);
            // stop mode: the tile ends once all its replicas (padding included) have reached the target
            if (stop_mode && __syncthreads_and(t >= NREP || hit >= 0 || tile * NREP + t >= job.R)) break;
        }

        store_words(job.final_words, 0x01010101u);
        if (t < NREP) {
            const int r = tile * NREP + t;
            if constexpr (PM1)
                job.E_best_i[r] = bestEi;
            else
                job.E_best_f[r] = bestEf;
            job.best_sweep[r] = bsweep;
            job.hit_sweep[r] = hit;
        }
        __syncthreads();
    }
};

template <int L, int WT, int JT>
__device__ __forceinline__ void ea_tile_fast(const EaJob& job, int tile, unsigned char* smem)
{
    __shared__ __align__(16) uint32_t s_tab[64];
    EaFastTile<L, WT, JT> tl(job, tile, smem, s_tab);
    tl.run();
}

// Fast-tile shapes: (L, WT) with (L/2) L WT == kResidentThreads / 2, and L = 24,
// WT = 1 (its 288 column-words fill 576 of the threads).
__host__ __device__ constexpr bool ea_fast_shape(int L, int WT)
{
    return (L == 32 && WT == 1) || (L == 16 && WT == 4) || (L == 8 && WT == 16) || (L == 24 && WT == 1);
}

}  // namespace pb
