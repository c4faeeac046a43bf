// ea.cu -- sm_103a kernels of the graph-coloured p-bit update on the periodic
// 3D Edwards-Anderson cube (arXiv 2510.23419, Sec. 2; update groups Sec. 1.2.2;
// p-bit Eqs. 2-3; classical annealing Sec. 1.3.1).
//
// Two forms compute identical trajectories (same random words, same fields,
// same thresholds):
//  * resident: one persistent kernel per coupling type; a CTA takes a tile (one job, 4*WT
//    replicas), keeps that tile's whole lattice in shared memory for all
//    sweeps, and only touches global memory for best-state snapshots and the
//    final state.  The shared-neighbour reuse of Sec. 1.2.2 is total: every
//    neighbour word is read from shared memory.
//  * plain: spins in global memory, one launch per colour class and sweep,
//    plus one energy/best launch per sweep.
#include "ea_fast.cuh"
#include "ea_kernels.cuh"
#include <mutex>

#include "ea_launch.h"

namespace pb {

namespace {

// ---------------------------------------------------------------------------
// Resident form
// ---------------------------------------------------------------------------
struct TileCtx {
    int L, WT, h2, half, N, CW, P;
    int t, lane, warp;
    bool active;
    int w, q, y, zfirst, zstep;  // thread's column (q, y, w) and its z values zfirst, zfirst+zstep, ...
    uint32_t tq;                 // Philox counter word 2 = replica quad index
};

template <int LT, int WTT>
__device__ __forceinline__ TileCtx tile_ctx(const EaJob& job, int tile)
{
    TileCtx g;
    g.L = LT ? LT : job.inst.L;
    g.WT = WTT ? WTT : job.WT;
    g.h2 = g.L >> 1;
    g.half = g.h2 * g.L * g.L;
    g.N = 2 * g.half;
    g.CW = g.h2 * g.L * g.WT;
    g.P = (2 * g.CW <= kResidentThreads) ? 2 : 1;
    g.t = threadIdx.x;
    g.lane = g.t & 31;
    g.warp = g.t >> 5;
    const int cw = (g.P == 2) ? (g.t % g.CW) : g.t;
    g.active = g.t < g.P * g.CW;
    g.w = g.t % g.WT;  // == cw % WT since CW and blockDim are multiples of WT
    g.q = (cw / g.WT) % g.h2;
    g.y = cw / (g.WT * g.h2);
    if (g.P == 2) {
        g.zfirst = g.t / g.CW;
        g.zstep = 2;
    } else {
        g.zfirst = 0;
        g.zstep = 1;
    }
    g.tq = (uint32_t)(tile * g.WT + g.w);
    return g;
}

// Sum 4 per-thread values over the lanes that hold the same w, then store the
// warp's sums in part[warp][4w + b].
template <typename T>
__device__ __forceinline__ void warp_partials(const TileCtx& g, T v0, T v1, T v2, T v3, T* part)
{
    for (int o = g.WT; o < 32; o <<= 1) {
        v0 += __shfl_xor_sync(0xFFFFFFFFu, v0, o);
        v1 += __shfl_xor_sync(0xFFFFFFFFu, v1, o);
        v2 += __shfl_xor_sync(0xFFFFFFFFu, v2, o);
        v3 += __shfl_xor_sync(0xFFFFFFFFu, v3, o);
    }
    if (g.lane < g.WT) {
        T* p = part + g.warp * 4 * g.WT + 4 * g.lane;
        p[0] = v0; p[1] = v1; p[2] = v2; p[3] = v3;
    }
}

// Byte-lane counts (<= 255 each) -> four int32 partials.
__device__ __forceinline__ void warp_partials_bytes(const TileCtx& g, uint32_t acc, int32_t* part)
{
    uint32_t a = acc & 0x00FF00FFu;         // replicas 0 and 2 in 16-bit lanes
    uint32_t b = (acc >> 8) & 0x00FF00FFu;  // replicas 1 and 3
    for (int o = g.WT; o < 32; o <<= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
    }
    if (g.lane < g.WT) {
        int32_t* p = part + g.warp * 4 * g.WT + 4 * g.lane;
        p[0] = (int32_t)(a & 0xFFFFu);
        p[1] = (int32_t)(b & 0xFFFFu);
        p[2] = (int32_t)(a >> 16);
        p[3] = (int32_t)(b >> 16);
    }
}

// Merge the thread's words of both colours into a global state buffer for the
// replicas that `flags` selects (byte b = 1: replica 4w + b of each word;
// 0x01010101: all), with the same word partition as the half-sweeps.
template <int LT, int WTT>
__device__ __forceinline__ void tile_store_words(const TileCtx& g, const uint32_t* sp, uint32_t* gdst, int tile,
                                                 uint32_t flags)
{
    if (!g.active || flags == 0u) return;
    const int L = LT ? LT : g.L;
    const int WT = WTT ? WTT : g.WT;
    const int h2 = L >> 1;
    const int half = h2 * L * L;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
        const uint32_t* src = sp + (size_t)c * half * WT;
        uint32_t* dst = gdst + ((size_t)tile * 2 + c) * half * WT;
        for (int z = g.zfirst; z < L; z += g.zstep) {
            const int kw = (g.q + h2 * (g.y + L * z)) * WT + g.w;
            if (WT == 1)
                snapshot_word<true>(dst + kw, src[kw], flags);
            else
                snapshot_word<false>(dst + kw, src[kw], flags);
        }
    }
}

template <int LT, int WTT, int JT, bool HH>
__device__ void ea_tile(const EaJob& job, int tile, unsigned char* smem)
{
    const TileCtx g = tile_ctx<LT, WTT>(job, tile);
    const int L = LT ? LT : g.L;
    const int WT = WTT ? WTT : g.WT;
    const int h2 = L >> 1;
    const int half = h2 * L * L;
    const int N = 2 * half;
    const int nrep = 4 * WT;

    // ---- shared memory carve-up (must match ea_resident_smem) ----
    unsigned char* p = smem;
    uint32_t* sp = reinterpret_cast<uint32_t*>(p);
    p += (size_t)N * WT * 4;
    uint8_t* sjb = nullptr;
    int8_t* sh8 = nullptr;
    if (JT == PB_J_PM1_I8) {
        sjb = p;
        p += (N + 15) / 16 * 16;
        if (HH) {
            sh8 = reinterpret_cast<int8_t*>(p);
            p += (N + 15) / 16 * 16;
        }
    }
    const int tabw = (JT == PB_J_PM1_I8) ? (HH ? job.nF : 64) : 0;
    const int tabw4 = (tabw + 3) / 4 * 4;
    uint32_t* stab = reinterpret_cast<uint32_t*>(p);
    p += (size_t)2 * tabw4 * 4;
    int32_t* spart_i = reinterpret_cast<int32_t*>(p);
    float* spart_f = reinterpret_cast<float*>(p);
    p += (size_t)kResidentWarps * nrep * 4;
    int32_t* spart_h = reinterpret_cast<int32_t*>(p);
    if (JT == PB_J_PM1_I8 && HH) p += (size_t)kResidentWarps * nrep * 4;
    uint8_t* sflag = p;

    const uint32_t key0 = job.key0, key1 = job.key1;
    const int t = g.t;

    // ---- instance data and initial state (tag 1) ----
    if (JT == PB_J_PM1_I8) {
        for (int i = t; i < N; i += kResidentThreads) sjb[i] = job.inst.jbits[i];
        if (HH)
            for (int i = t; i < N; i += kResidentThreads) sh8[i] = job.inst.h8[i];
    }
    for (int j = t; j < N * WT; j += kResidentThreads) {
        if (job.resume) {  // resumed run: the given state, in the tile layout of final_words
            sp[j] = job.final_words[(size_t)tile * N * WT + j];
            continue;
        }
        const int w2 = j % WT;
        const int ck = j / WT;
        const int c = ck >= half ? 1 : 0;
        const int k = ck - c * half;
        const U4 r = philox10((uint32_t)k, 0u, (uint32_t)(tile * WT + w2), (kTagInit << 24) | (uint32_t)c, key0, key1);
        sp[j] = (JT == PB_J_PM1_I8) ? ((r.x >> 31) | ((r.y >> 31) << 8) | ((r.z >> 31) << 16) | ((r.w >> 31) << 24))
                                    : f32_word(r.x >> 31, r.y >> 31, r.z >> 31, r.w >> 31);
    }

    auto build_table = [&](int s, int buf) {
        if (JT != PB_J_PM1_I8) return;
        const int level = s / job.step;
        const uint32_t* row = job.table + (size_t)level * job.nF;
        if (!HH) {
            if (t < 64) {
                const int F = 6 - 2 * __popc((unsigned)t);
                stab[buf * tabw4 + t] = row[F - job.fmin];
            }
        } else {
            for (int f = t; f < job.nF; f += kResidentThreads) stab[buf * tabw4 + f] = row[f];
        }
    };

    // One colour class: update (decide = true) or only accumulate the energy
    // terms (decide = false, for the initial state).  Returns the thread's
    // per-replica accumulators: PM1 -> unsatisfied-bond counts in byte lanes
    // (class 1 only) and h.m sums; F32 -> -m F (class 1) and -h m (class 0).
    auto half_sweep = [&](int c, int s, bool decide, uint32_t& uacc, int32_t (&hm)[4], float (&ef)[4]) {
        if (!g.active) return;
        const uint32_t* o = sp + (size_t)(1 - c) * half * WT;
        uint32_t* own = sp + (size_t)c * half * WT;
        const uint32_t c3 = (kTagDecision << 24) | (uint32_t)c;
        const int buf = s & 1;
        const uint32_t* tab = stab + buf * tabw4;
        float cexp = 0.0f;
        if (JT == PB_J_F32) cexp = f32_cexp(job.betaf[s / job.step]);
        for (int zp = 0; zp < (g.zstep == 1 ? 2 : 1); ++zp) {
            const int z0 = (g.zstep == 1) ? zp : g.zfirst;
            const int px = (c + g.y + z0) & 1;
            const EaColumn col = ea_column(L, h2, g.q, g.y, px);
            const int oxp = col.dxp * WT, oxm = col.dxm * WT, oyp = col.dyp * WT, oym = col.dym * WT;
            const int sz = L * h2 * WT;
#pragma unroll 2
            for (int z = z0; z < L; z += 2) {
                const int k = g.q + h2 * (g.y + L * z);
                const int kw = k * WT + g.w;
                const int ozp = (z + 1 == L) ? -(L - 1) * sz : sz;
                const int ozm = (z == 0) ? (L - 1) * sz : -sz;
                const uint32_t n0 = o[kw + oxp], n1 = o[kw + oxm], n2 = o[kw + oyp];
                const uint32_t n3 = o[kw + oym], n4 = o[kw + ozp], n5 = o[kw + ozm];
                if (JT == PB_J_PM1_I8) {
                    const uint32_t X = ea_pattern(n0, n1, n2, n3, n4, n5, sjb[c * half + k]);
                    uint32_t snew;
                    if (decide) {
                        const U4 r = philox10((uint32_t)k, (uint32_t)s, g.tq, c3, key0, key1);
                        if (!HH) {
                            const unsigned char* tb = reinterpret_cast<const unsigned char*>(tab);
                            const uint32_t T0 = *reinterpret_cast<const uint32_t*>(tb + (X & 0xFFu));
                            const uint32_t T1 = *reinterpret_cast<const uint32_t*>(tb + ((X >> 8) & 0xFFu));
                            const uint32_t T2 = *reinterpret_cast<const uint32_t*>(tb + ((X >> 16) & 0xFFu));
                            const uint32_t T3 = *reinterpret_cast<const uint32_t*>(tb + (X >> 24));
                            snew = decide_bit(r.x, T0) | (decide_bit(r.y, T1) << 8) | (decide_bit(r.z, T2) << 16) |
                                   (decide_bit(r.w, T3) << 24);
                        } else {
                            const int hi = sh8[c * half + k];
                            const int base = 6 + hi - job.fmin;  // index of F = 6 - 2n + h
                            const uint32_t T0 = tab[base - 2 * __popc(X & 0xFCu)];
                            const uint32_t T1 = tab[base - 2 * __popc((X >> 8) & 0xFCu)];
                            const uint32_t T2 = tab[base - 2 * __popc((X >> 16) & 0xFCu)];
                            const uint32_t T3 = tab[base - 2 * __popc((X >> 24) & 0xFCu)];
                            snew = decide_bit(r.x, T0) | (decide_bit(r.y, T1) << 8) | (decide_bit(r.z, T2) << 16) |
                                   (decide_bit(r.w, T3) << 24);
                        }
                        own[kw] = snew;
                    } else {
                        snew = own[kw];
                    }
                    if (c == 1) uacc += ea_popc6_bytes(X ^ (snew * 0xFCu));
                    if (HH) {
                        const int hi = sh8[c * half + k];
                        hm[0] += (snew & 0x1u) ? -hi : hi;
                        hm[1] += (snew & 0x100u) ? -hi : hi;
                        hm[2] += (snew & 0x10000u) ? -hi : hi;
                        hm[3] += (snew & 0x1000000u) ? -hi : hi;
                    }
                } else {
                    const size_t site = (size_t)c * half + k;
                    const float4 ja = __ldg(reinterpret_cast<const float4*>(job.inst.j6) + 2 * site);
                    const float4 jb = __ldg(reinterpret_cast<const float4*>(job.inst.j6) + 2 * site + 1);
                    const float jv[6] = {ja.x, ja.y, ja.z, ja.w, jb.x, jb.y};
                    const float hv = jb.z;  // the site's field rides in the coupling vector
                    const uint32_t nb[6] = {n0, n1, n2, n3, n4, n5};
                    uint32_t snew = 0;
                    float F[4];
#pragma unroll
                    for (int b = 0; b < 4; ++b) F[b] = ea_field_f32(jv, hv, nb, b);
                    if (decide) {
                        const U4 r = philox10((uint32_t)k, (uint32_t)s, g.tq, c3, key0, key1);
                        snew = decide_f32_word(r.x, r.y, r.z, r.w, F[0], F[1], F[2], F[3], cexp);
                        own[kw] = snew;
                    } else {
                        snew = own[kw];
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const bool dn = f32_minus(snew, b);  // m = -1
                        if (c == 1)
                            ef[b] += dn ? F[b] : -F[b];           // -m F
                        else if (job.inst.has_h)
                            ef[b] += dn ? hv : -hv;               // -h m
                    }
                }
            }
        }
    };

    // Collect the per-replica energy of the state now in shared memory.
    auto energy_partials = [&](uint32_t uacc, const int32_t (&hm)[4], const float (&ef)[4]) {
        if (JT == PB_J_PM1_I8) {
            warp_partials_bytes(g, uacc, spart_i);
            if (HH) warp_partials<int32_t>(g, hm[0], hm[1], hm[2], hm[3], spart_h);
        } else {
            warp_partials<float>(g, ef[0], ef[1], ef[2], ef[3], spart_f);
        }
    };
    // Thread r < nrep: energy of replica r from the warp partials (fixed order).
    auto energy_of = [&](int r, int32_t& Ei, float& Ef) {
        if (JT == PB_J_PM1_I8) {
            int32_t U = 0, H = 0;
            for (int v = 0; v < kResidentWarps; ++v) {
                U += spart_i[v * nrep + r];
                if (HH) H += spart_h[v * nrep + r];
            }
            // E = -(#satisfied - #unsatisfied) - sum h m = -(3N - 2U) - sum h m
            Ei = -(3 * N - 2 * U) - H;
        } else {
            float E = 0.0f;
            for (int v = 0; v < kResidentWarps; ++v) E += spart_f[v * nrep + r];
            Ef = E;
        }
    };

    // ---- initial energy; the initial state is the first best state (unless resumed) ----
    const int s_first = job.s0 < job.S ? job.s0 : 0;
    build_table(s_first, s_first & 1);
    __syncthreads();
    {
        uint32_t uacc = 0;
        int32_t hm[4] = {0, 0, 0, 0};
        float ef[4] = {0.f, 0.f, 0.f, 0.f};
        half_sweep(0, 0, false, uacc, hm, ef);
        half_sweep(1, 0, false, uacc, hm, ef);
        energy_partials(uacc, hm, ef);
    }
    __syncthreads();
    int32_t bestEi = 0, hit = -1, bsweep = -1;
    float bestEf = 0.0f;
    if (t < nrep) energy_of(t, bestEi, bestEf);
    if (job.resume) {  // the running best carried over
        if (t < nrep) {
            const int r = tile * nrep + t;
            if (JT == PB_J_PM1_I8)
                bestEi = job.E_best_i[r];
            else
                bestEf = job.E_best_f[r];
            bsweep = job.best_sweep[r];
        }
    } else {
        tile_store_words<LT, WTT>(g, sp, job.best_words, tile, 0x01010101u);
    }

    // ---- sweeps ----
    const bool stop_mode = job.has_target == 2;
    for (int s = job.s0; s < job.S; ++s) {
        uint32_t uacc = 0;
        int32_t hm[4] = {0, 0, 0, 0};
        float ef[4] = {0.f, 0.f, 0.f, 0.f};
        half_sweep(0, s, true, uacc, hm, ef);
        __syncthreads();
        half_sweep(1, s, true, uacc, hm, ef);
        energy_partials(uacc, hm, ef);
        if (s + 1 < job.S) build_table(s + 1, (s + 1) & 1);
        __syncthreads();
        if (t < nrep) {
            int32_t Ei = 0;
            float Ef = 0.0f;
            energy_of(t, Ei, Ef);
            const bool live = job.has_target != 2 || hit < 0;  // stop mode: the best is frozen at the target
            bool imp;
            if (JT == PB_J_PM1_I8) {
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
        __syncthreads();
        const uint32_t f = reinterpret_cast<const uint32_t*>(sflag)[g.w];
        tile_store_words<LT, WTT>(g, sp, job.best_words, tile, f);
        // stop mode: the tile ends once all its replicas (padding included) have reached the target
        if (stop_mode && __syncthreads_and(t >= nrep || hit >= 0 || tile * nrep + t >= job.R)) break;
    }

    // ---- results ----
    tile_store_words<LT, WTT>(g, sp, job.final_words, tile, 0x01010101u);
    if (t < nrep) {
        const int r = tile * nrep + t;
        if (JT == PB_J_PM1_I8)
            job.E_best_i[r] = bestEi;
        else
            job.E_best_f[r] = bestEf;
        job.best_sweep[r] = bsweep;
        job.hit_sweep[r] = hit;
    }
    __syncthreads();
}

// One persistent kernel per coupling type in a batch (for FP32, one of two
// variants, EaKernel): a kernel holding both types' tiles gets one register
// allocation for all of them, and the FP32 tiles' pressure then costs the +-1
// tiles spill traffic.  The tile code comes with the work
// item (a branch on the job's own fields also led the compiler to spill).
// Every CTA lets a programmatically dependent launch (the other type's kernel
// of the same batch) start at once, so that kernel's CTAs take the SMs this
// one leaves as its list runs out.
template <int K>
__global__ void __launch_bounds__(kResidentThreads, 1)
    ea_resident_kernel(const EaJob* __restrict__ jobs, const EaWork* __restrict__ work, int n_work, int* counter)
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_work) break;
        const EaWork wk = work[item];
        const EaJob& job = jobs[wk.job];
        if constexpr (K == kEaKernelPm1) {
            if (wk.path == kEaPathFieldsGeneric)
                ea_tile<0, 0, PB_J_PM1_I8, true>(job, wk.tile, smem);
            else if (wk.path == kEaPathFast32)
                ea_tile_fast<32, 1, PB_J_PM1_I8>(job, wk.tile, smem);
            else if (wk.path == kEaPathFast16)
                ea_tile_fast<16, 4, PB_J_PM1_I8>(job, wk.tile, smem);
            else if (wk.path == kEaPathFast8)
                ea_tile_fast<8, 16, PB_J_PM1_I8>(job, wk.tile, smem);
            else if (wk.path == kEaPathFast24)
                ea_tile_fast<24, 1, PB_J_PM1_I8>(job, wk.tile, smem);
            else if (wk.path == kEaPathGen12)
                ea_tile<12, 4, PB_J_PM1_I8, false>(job, wk.tile, smem);
            else
                ea_tile<0, 0, PB_J_PM1_I8, false>(job, wk.tile, smem);
        } else {
            // the compile-time L = 12 shape in either FP32 kernel makes it spill: its tiles
            // run the generic tile, as do L = 24 tiles in the first kernel
            if (K == kEaKernelF32 && wk.path == kEaPathFast32)
                ea_tile_fast<32, 1, PB_J_F32>(job, wk.tile, smem);
            else if (K == kEaKernelF32L24 && wk.path == kEaPathFast24)
                ea_tile_fast<24, 1, PB_J_F32>(job, wk.tile, smem);
            else if (wk.path == kEaPathFast16)
                ea_tile_fast<16, 4, PB_J_F32>(job, wk.tile, smem);
            else if (wk.path == kEaPathFast8)
                ea_tile_fast<8, 16, PB_J_F32>(job, wk.tile, smem);
            else
                ea_tile<0, 0, PB_J_F32, false>(job, wk.tile, smem);
        }
    }
}

// ---------------------------------------------------------------------------
// Random-word ceiling of the EA update: the decision words of an L = 32 tile
// (same counters, round keys and first-round hoisting as the fast tile: one
// Philox4x32-10 call per site and 4 replicas, i.e. one word per update) and
// nothing else -- no field, no threshold, no state.  Each thread takes the
// sites of one column of both colours, two sites per iteration as the +-1
// tile does; the words are folded into one xor per thread so none is dead.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kResidentThreads, 1)
    ea_philox_ceiling_kernel(uint32_t key0, uint32_t key1, int sweeps, uint32_t* __restrict__ sink)
{
    constexpr int L = 32, h2 = L / 2;
    const RoundKeys rk = round_keys(key0, key1);
    const int t = threadIdx.x;
    const int cw = t % (kResidentThreads / 2), zp = t / (kResidentThreads / 2);
    const int q = cw % h2, y = cw / h2;
    const uint32_t tq = blockIdx.x;
    uint32_t acc = 0;
    for (int s = 0; s < sweeps; ++s) {
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            const PhiloxPre pre = philox_pre((uint32_t)s, tq, (kTagDecision << 24) | (uint32_t)c, rk);
#pragma unroll 2
            for (int z = zp; z < L; z += 2) {
                const U4 r = philox_c0((uint32_t)(q + h2 * (y + L * z)), pre, rk);
                acc ^= r.x ^ r.y ^ r.z ^ r.w;
            }
        }
    }
    sink[(size_t)blockIdx.x * kResidentThreads + t] = acc;
}

// ---------------------------------------------------------------------------
// Plain form (global memory state, one tile with WT = Rw)
// ---------------------------------------------------------------------------
struct SiteGeom {
    int x, y, z, q, row;
};

__device__ __forceinline__ SiteGeom site_of_rank(int L, int c, int k)
{
    SiteGeom s;
    const int h2 = L >> 1;
    s.row = k / h2;
    s.q = k - s.row * h2;
    s.y = s.row % L;
    s.z = s.row / L;
    s.x = 2 * s.q + ((c + s.y + s.z) & 1);
    return s;
}

// Class ranks of the 6 neighbours (+x, -x, +y, -y, +z, -z) of a site.
__device__ __forceinline__ void neighbour_ranks(int L, const SiteGeom& s, int (&kn)[6])
{
    const int h2 = L >> 1;
    const int xp = (s.x + 1 == L) ? 0 : s.x + 1, xm = (s.x == 0) ? L - 1 : s.x - 1;
    const int yp = (s.y + 1 == L) ? 0 : s.y + 1, ym = (s.y == 0) ? L - 1 : s.y - 1;
    const int zp = (s.z + 1 == L) ? 0 : s.z + 1, zm = (s.z == 0) ? L - 1 : s.z - 1;
    kn[0] = (xp >> 1) + h2 * (s.y + L * s.z);
    kn[1] = (xm >> 1) + h2 * (s.y + L * s.z);
    kn[2] = s.q + h2 * (yp + L * s.z);
    kn[3] = s.q + h2 * (ym + L * s.z);
    kn[4] = s.q + h2 * (s.y + L * zp);
    kn[5] = s.q + h2 * (s.y + L * zm);
}

// Plain form in stop mode: every replica has reached the target, the launches
// of the remaining sweeps return at once.
__device__ __forceinline__ bool ea_plain_stopped(const EaJob& job)
{
    return job.has_target == 2 && *reinterpret_cast<const volatile int32_t*>(job.n_hit) >= job.R;
}

template <int JT, bool HH>
__global__ void __launch_bounds__(256) ea_plain_half_kernel(EaJob job, int c, int s)
{
    if (ea_plain_stopped(job)) return;
    __shared__ uint32_t stab[256];
    const int L = job.inst.L;
    const int half = job.inst.half;
    const int WT = job.WT;
    if (JT == PB_J_PM1_I8) {
        const uint32_t* row = job.table + (size_t)(s / job.step) * job.nF;
        if (!HH) {
            if (threadIdx.x < 64) stab[threadIdx.x] = row[6 - 2 * __popc(threadIdx.x) - job.fmin];
        } else {
            for (int f = threadIdx.x; f < job.nF; f += blockDim.x) stab[f] = row[f];
        }
        __syncthreads();
    }
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (long long)half * WT) return;
    const int k = (int)(j / WT);
    const int w = (int)(j - (long long)k * WT);
    const SiteGeom sg = site_of_rank(L, c, k);
    int kn[6];
    neighbour_ranks(L, sg, kn);
    const uint32_t* o = job.final_words + (size_t)(1 - c) * half * WT;
    uint32_t nb[6];
#pragma unroll
    for (int b = 0; b < 6; ++b) nb[b] = o[(size_t)kn[b] * WT + w];
    const U4 r = philox10((uint32_t)k, (uint32_t)s, (uint32_t)w, (kTagDecision << 24) | (uint32_t)c, job.key0, job.key1);
    uint32_t snew;
    if (JT == PB_J_PM1_I8) {
        const uint32_t X = ea_pattern(nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], job.inst.jbits[c * half + k]);
        if (!HH) {
            const unsigned char* tb = reinterpret_cast<const unsigned char*>(stab);
            snew = decide_bit(r.x, *reinterpret_cast<const uint32_t*>(tb + (X & 0xFFu))) |
                   (decide_bit(r.y, *reinterpret_cast<const uint32_t*>(tb + ((X >> 8) & 0xFFu))) << 8) |
                   (decide_bit(r.z, *reinterpret_cast<const uint32_t*>(tb + ((X >> 16) & 0xFFu))) << 16) |
                   (decide_bit(r.w, *reinterpret_cast<const uint32_t*>(tb + (X >> 24))) << 24);
        } else {
            const int base = 6 + job.inst.h8[c * half + k] - job.fmin;
            snew = decide_bit(r.x, stab[base - 2 * __popc(X & 0xFCu)]) |
                   (decide_bit(r.y, stab[base - 2 * __popc((X >> 8) & 0xFCu)]) << 8) |
                   (decide_bit(r.z, stab[base - 2 * __popc((X >> 16) & 0xFCu)]) << 16) |
                   (decide_bit(r.w, stab[base - 2 * __popc((X >> 24) & 0xFCu)]) << 24);
        }
    } else {
        const size_t site = (size_t)c * half + k;
        const float4 ja = __ldg(reinterpret_cast<const float4*>(job.inst.j6) + 2 * site);
        const float4 jb = __ldg(reinterpret_cast<const float4*>(job.inst.j6) + 2 * site + 1);
        const float jv[6] = {ja.x, ja.y, ja.z, ja.w, jb.x, jb.y};
        const float hv = __ldg(job.inst.hf + site);
        const float cexp = f32_cexp(job.betaf[s / job.step]);
        snew = decide_f32_word(r.x, r.y, r.z, r.w, ea_field_f32(jv, hv, nb, 0), ea_field_f32(jv, hv, nb, 1),
                               ea_field_f32(jv, hv, nb, 2), ea_field_f32(jv, hv, nb, 3), cexp);
    }
    job.final_words[(size_t)c * half * WT + j] = snew;
}

__global__ void __launch_bounds__(256) ea_plain_init_kernel(EaJob job)
{
    const int half = job.inst.half;
    const int WT = job.WT;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 2LL * half * WT) return;
    const int w = (int)(j % WT);
    const long long ck = j / WT;
    const int c = ck >= half ? 1 : 0;
    const int k = (int)(ck - (long long)c * half);
    const U4 r = philox10((uint32_t)k, 0u, (uint32_t)w, (kTagInit << 24) | (uint32_t)c, job.key0, job.key1);
    job.final_words[j] = (job.inst.jtype == PB_J_PM1_I8)
                             ? ((r.x >> 31) | ((r.y >> 31) << 8) | ((r.z >> 31) << 16) | ((r.w >> 31) << 24))
                             : f32_word(r.x >> 31, r.y >> 31, r.z >> 31, r.w >> 31);
}

// One block per word column w (4 replicas): energy of the current state, best
// update, best snapshot.  init: the current state is the initial state.
template <int JT, bool HH>
__global__ void __launch_bounds__(256) ea_plain_energy_kernel(EaJob job, int s, int init)
{
    if (!init && ea_plain_stopped(job)) return;
    __shared__ int32_t red_i[8][256 / 32];
    __shared__ float red_f[4][256 / 32];
    __shared__ uint32_t s_mask;
    const int L = job.inst.L;
    const int half = job.inst.half;
    const int N = job.inst.N;
    const int WT = job.WT;
    const int w = blockIdx.x;
    const int t = threadIdx.x;
    uint32_t lo = 0, hi = 0;
    int32_t hm[4] = {0, 0, 0, 0};
    float ef[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c = 0; c < 2; ++c) {
        const uint32_t* own = job.final_words + (size_t)c * half * WT;
        const uint32_t* o = job.final_words + (size_t)(1 - c) * half * WT;
        for (int k = t; k < half; k += blockDim.x) {
            const uint32_t sv = own[(size_t)k * WT + w];
            if (JT == PB_J_PM1_I8) {
                if (c == 1) {
                    const SiteGeom sg = site_of_rank(L, c, k);
                    int kn[6];
                    neighbour_ranks(L, sg, kn);
                    uint32_t nb[6];
#pragma unroll
                    for (int b = 0; b < 6; ++b) nb[b] = o[(size_t)kn[b] * WT + w];
                    const uint32_t X = ea_pattern(nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], job.inst.jbits[c * half + k]);
                    const uint32_t u = ea_popc6_bytes(X ^ (sv * 0xFCu));
                    lo += u & 0x00FF00FFu;
                    hi += (u >> 8) & 0x00FF00FFu;
                }
                if (HH) {
                    const int hv = job.inst.h8[c * half + k];
#pragma unroll
                    for (int b = 0; b < 4; ++b) hm[b] += ((sv >> (8 * b)) & 1u) ? -hv : hv;
                }
            } else {
                const size_t site = (size_t)c * half + k;
                const float hv = job.inst.hf[site];
                if (c == 1) {
                    const SiteGeom sg = site_of_rank(L, c, k);
                    int kn[6];
                    neighbour_ranks(L, sg, kn);
                    uint32_t nb[6];
#pragma unroll
                    for (int b = 0; b < 6; ++b) nb[b] = o[(size_t)kn[b] * WT + w];
                    const float4 ja = reinterpret_cast<const float4*>(job.inst.j6)[2 * site];
                    const float4 jb = reinterpret_cast<const float4*>(job.inst.j6)[2 * site + 1];
                    const float jv[6] = {ja.x, ja.y, ja.z, ja.w, jb.x, jb.y};
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const float F = ea_field_f32(jv, hv, nb, b);
                        ef[b] += f32_minus(sv, b) ? F : -F;
                    }
                } else if (job.inst.has_h) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) ef[b] += f32_minus(sv, b) ? hv : -hv;
                }
            }
        }
    }
    // deterministic block reduction
    const int lane = t & 31, warp = t >> 5;
    int32_t v[8] = {(int32_t)(lo & 0xFFFFu), (int32_t)(hi & 0xFFFFu), (int32_t)(lo >> 16), (int32_t)(hi >> 16),
                    hm[0], hm[1], hm[2], hm[3]};
#pragma unroll
    for (int a = 0; a < 8; ++a)
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_xor_sync(0xFFFFFFFFu, v[a], o);
#pragma unroll
    for (int a = 0; a < 4; ++a)
        for (int o = 16; o > 0; o >>= 1) ef[a] += __shfl_xor_sync(0xFFFFFFFFu, ef[a], o);
    if (lane == 0) {
        for (int a = 0; a < 8; ++a) red_i[a][warp] = v[a];
        for (int a = 0; a < 4; ++a) red_f[a][warp] = ef[a];
    }
    __syncthreads();
    if (t < 4) {
        const int r = 4 * w + t;
        bool imp;
        if (JT == PB_J_PM1_I8) {
            int32_t U = 0, H = 0;
            for (int q = 0; q < 8; ++q) {
                U += red_i[t][q];
                H += red_i[4 + t][q];
            }
            const int32_t E = -(3 * N - 2 * U) - H;
            imp = init || ((job.has_target != 2 || job.hit_sweep[r] < 0) && E < job.E_best_i[r]);
            if (imp) job.E_best_i[r] = E;
            if (!init && job.has_target && job.hit_sweep[r] < 0 && E <= job.target_i) {
                job.hit_sweep[r] = s;
                if (job.has_target == 2 && r < job.R) atomicAdd(job.n_hit, 1);
            }
        } else {
            float E = 0.0f;
            for (int q = 0; q < 8; ++q) E += red_f[t][q];
            imp = init || ((job.has_target != 2 || job.hit_sweep[r] < 0) && E < job.E_best_f[r]);
            if (imp) job.E_best_f[r] = E;
            if (!init && job.has_target && job.hit_sweep[r] < 0 && E <= job.target_f) {
                job.hit_sweep[r] = s;
                if (job.has_target == 2 && r < job.R) atomicAdd(job.n_hit, 1);
            }
        }
        if (init) job.hit_sweep[r] = -1;
        if (imp) job.best_sweep[r] = init ? -1 : s;
        const uint32_t m = imp ? (0xFFu << (8 * t)) : 0u;
        if (t == 0) s_mask = 0u;
        __syncwarp(0xFu);
        atomicOr(&s_mask, m);
    }
    __syncthreads();
    const uint32_t mask = s_mask;
    if (mask == 0u) return;
    for (int j = t; j < N; j += blockDim.x) {
        const size_t idx = (size_t)j * WT + w;
        const uint32_t v2 = job.final_words[idx];
        if (mask == 0xFFFFFFFFu)
            job.best_words[idx] = v2;
        else
            job.best_words[idx] = (job.best_words[idx] & ~mask) | (v2 & mask);
    }
}

// ---------------------------------------------------------------------------
// Readout and exact energies
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ea_readout_kernel(EaJob job, const uint32_t* __restrict__ words,
                                                         int8_t* __restrict__ out)
{
    const int L = job.inst.L;
    const int N = job.inst.N, half = job.inst.half, WT = job.WT;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (long long)job.R * N) return;
    const int r = (int)(j / N);
    const int i = (int)(j - (long long)r * N);
    const int x = i % L, y = (i / L) % L, z = i / (L * L);
    const int c = (x + y + z) & 1;
    const int k = i >> 1;
    const int tile = r / (4 * WT);
    const int w = (r / 4) % WT;
    const int b = r & 3;
    const uint32_t v = words[(((size_t)tile * 2 + c) * half + k) * WT + w];
    const uint32_t minus = (job.inst.jtype == PB_J_PM1_I8) ? ((v >> (8 * b)) & 1u) : f32_minus(v, b);
    out[j] = minus ? (int8_t)-1 : (int8_t)1;
}

// E = -sum_{d,i} J[d][i] m_i m_{i+d} - sum_i h_i m_i, one block per replica;
// int64 for PM1, FP64 for F32 (the only FP64 on the device).
template <int JT>
__global__ void __launch_bounds__(256) ea_energy_kernel(EaJob job, const int8_t* __restrict__ m, double* __restrict__ E)
{
    __shared__ long long red_i[8];
    __shared__ double red_f[8];
    const int L = job.inst.L, N = job.inst.N;
    const int r = blockIdx.x;
    const int8_t* mr = m + (size_t)r * N;
    long long ai = 0;
    double af = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int x = i % L, y = (i / L) % L, z = i / (L * L);
        const int nbr[3] = {((x + 1) % L) + L * (y + L * z), x + L * (((y + 1) % L) + L * z),
                            x + L * (y + L * ((z + 1) % L))};
        const int mi = mr[i];
        if (JT == PB_J_PM1_I8) {
            const int8_t* J = static_cast<const int8_t*>(job.inst.J3);
            for (int d = 0; d < 3; ++d) ai -= (long long)J[(size_t)d * N + i] * mi * mr[nbr[d]];
            if (job.inst.hraw) ai -= (long long)static_cast<const int8_t*>(job.inst.hraw)[i] * mi;
        } else {
            const float* J = static_cast<const float*>(job.inst.J3);
            for (int d = 0; d < 3; ++d) af -= (double)J[(size_t)d * N + i] * (double)(mi * mr[nbr[d]]);
            if (job.inst.hraw) af -= (double)static_cast<const float*>(job.inst.hraw)[i] * (double)mi;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ai += __shfl_xor_sync(0xFFFFFFFFu, ai, o);
        af += __shfl_xor_sync(0xFFFFFFFFu, af, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red_i[threadIdx.x >> 5] = ai;
        red_f[threadIdx.x >> 5] = af;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long si = 0;
        double sf = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            si += red_i[q];
            sf += red_f[q];
        }
        E[r] = (JT == PB_J_PM1_I8) ? (double)si : sf;
    }
}

// Fields of given states with the anneal kernels' arithmetic.
__global__ void __launch_bounds__(256) ea_fields_kernel(EaDevice inst, const int8_t* __restrict__ m, int R,
                                                        float* __restrict__ out)
{
    const int L = inst.L, N = inst.N, half = inst.half;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (long long)R * N) return;
    const int r = (int)(j / N);
    const int i = (int)(j - (long long)r * N);
    const int x = i % L, y = (i / L) % L, z = i / (L * L);
    const int c = (x + y + z) & 1;
    const int k = i >> 1;
    const int8_t* mr = m + (size_t)r * N;
    const SiteGeom sg = site_of_rank(L, c, k);
    int kn[6];
    neighbour_ranks(L, sg, kn);
    // class rank -> site index of the other colour: i' = 2k' + parity
    uint32_t nb[6];
#pragma unroll
    for (int b = 0; b < 6; ++b) {
        const int kk = kn[b];
        const int row = kk / (L >> 1), qq = kk - row * (L >> 1);
        const int yy = row % L, zz = row / L;
        const int xx = 2 * qq + ((1 - c + yy + zz) & 1);
        const bool minus = mr[xx + L * (yy + L * zz)] < 0;
        nb[b] = (inst.jtype == PB_J_PM1_I8) ? (minus ? 1u : 0u) : (minus ? 0xBFu : 0x3Fu);
    }
    if (inst.jtype == PB_J_PM1_I8) {
        const uint32_t X = ea_pattern(nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], inst.jbits[c * half + k]);
        const int h = inst.h8 ? inst.h8[c * half + k] : 0;
        out[j] = (float)(6 - 2 * __popc(X & 0xFCu) + h);
    } else {
        const size_t site = (size_t)c * half + k;
        const float4 ja = reinterpret_cast<const float4*>(inst.j6)[2 * site];
        const float4 jb = reinterpret_cast<const float4*>(inst.j6)[2 * site + 1];
        const float jv[6] = {ja.x, ja.y, ja.z, ja.w, jb.x, jb.y};
        out[j] = ea_field_f32(jv, inst.hf[site], nb, 0);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
int ea_resident_pick_wt(int L, int jtype, int has_h, int nF, int cap_words)
{
    const int h2 = L / 2;
    int best = 0;
    for (int wt = 1; wt <= kResidentMaxWT; wt *= 2) {
        if ((long long)h2 * L * wt > kResidentThreads / 2) break;
        if (ea_resident_smem(L, wt, jtype, has_h, nF) > kResidentSmemLimit) break;
        best = wt;
        if (wt >= cap_words) break;
    }
    return best;
}

// The limit is a property of the kernel, shared by every run of the process
// on a device: it only grows, so preparing a run never lowers the limit that
// another prepared run will launch with.
template <int K>
static cudaError_t ea_resident_attr(size_t smem)
{
    return cudaFuncSetAttribute(ea_resident_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t ea_resident_set_smem(int kernel, size_t smem)
{
    static std::mutex mu;
    static size_t current[kEaKernels][64] = {};
    if (kernel < 0 || kernel >= kEaKernels) return cudaErrorInvalidValue;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t* cur = (dev >= 0 && dev < 64) ? &current[kernel][dev] : nullptr;
    if (cur && smem <= *cur) return cudaSuccess;
    const cudaError_t e = kernel == kEaKernelPm1   ? ea_resident_attr<kEaKernelPm1>(smem)
                          : kernel == kEaKernelF32 ? ea_resident_attr<kEaKernelF32>(smem)
                                                   : ea_resident_attr<kEaKernelF32L24>(smem);
    if (e == cudaSuccess && cur) *cur = smem;
    return e;
}

cudaError_t ea_launch_resident(int kernel, const EaJob* d_jobs, const EaWork* d_work, int n_work, int* d_counter,
                               size_t smem, int grid, bool after_previous, cudaStream_t st)
{
    if (kernel < 0 || kernel >= kEaKernels) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kResidentThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (after_previous) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    if (kernel == kEaKernelPm1)
        return cudaLaunchKernelEx(&cfg, ea_resident_kernel<kEaKernelPm1>, d_jobs, d_work, n_work, d_counter);
    if (kernel == kEaKernelF32)
        return cudaLaunchKernelEx(&cfg, ea_resident_kernel<kEaKernelF32>, d_jobs, d_work, n_work, d_counter);
    return cudaLaunchKernelEx(&cfg, ea_resident_kernel<kEaKernelF32L24>, d_jobs, d_work, n_work, d_counter);
}

cudaError_t ea_launch_philox_ceiling(uint64_t seed, int sweeps, int blocks, uint32_t* sink, cudaStream_t st)
{
    ea_philox_ceiling_kernel<<<blocks, kResidentThreads, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32), sweeps, sink);
    return cudaGetLastError();
}

static unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

cudaError_t ea_launch_plain_init(const EaJob& job, cudaStream_t st)
{
    const long long n = 2LL * job.inst.half * job.WT;
    ea_plain_init_kernel<<<blocks_for(n, 256), 256, 0, st>>>(job);
    return cudaGetLastError();
}

cudaError_t ea_launch_plain_sweep(const EaJob& job, int s, cudaStream_t st)
{
    const long long n = (long long)job.inst.half * job.WT;
    const unsigned nb = blocks_for(n, 256);
    for (int c = 0; c < 2; ++c) {
        if (job.inst.jtype == PB_J_PM1_I8) {
            if (job.inst.has_h)
                ea_plain_half_kernel<PB_J_PM1_I8, true><<<nb, 256, 0, st>>>(job, c, s);
            else
                ea_plain_half_kernel<PB_J_PM1_I8, false><<<nb, 256, 0, st>>>(job, c, s);
        } else {
            ea_plain_half_kernel<PB_J_F32, false><<<nb, 256, 0, st>>>(job, c, s);
        }
    }
    return cudaGetLastError();
}

cudaError_t ea_launch_plain_energy(const EaJob& job, int s, bool init, cudaStream_t st)
{
    if (job.inst.jtype == PB_J_PM1_I8) {
        if (job.inst.has_h)
            ea_plain_energy_kernel<PB_J_PM1_I8, true><<<job.WT, 256, 0, st>>>(job, s, init ? 1 : 0);
        else
            ea_plain_energy_kernel<PB_J_PM1_I8, false><<<job.WT, 256, 0, st>>>(job, s, init ? 1 : 0);
    } else {
        ea_plain_energy_kernel<PB_J_F32, false><<<job.WT, 256, 0, st>>>(job, s, init ? 1 : 0);
    }
    return cudaGetLastError();
}

cudaError_t ea_launch_readout(const EaJob& job, const uint32_t* words, int8_t* out_pm, double* out_E, cudaStream_t st)
{
    const long long n = (long long)job.R * job.inst.N;
    ea_readout_kernel<<<blocks_for(n, 256), 256, 0, st>>>(job, words, out_pm);
    if (job.inst.jtype == PB_J_PM1_I8)
        ea_energy_kernel<PB_J_PM1_I8><<<job.R, 256, 0, st>>>(job, out_pm, out_E);
    else
        ea_energy_kernel<PB_J_F32><<<job.R, 256, 0, st>>>(job, out_pm, out_E);
    return cudaGetLastError();
}

cudaError_t ea_launch_fields(const EaDevice& inst, const int8_t* d_states, int R, float* d_out, cudaStream_t st)
{
    const long long n = (long long)R * inst.N;
    ea_fields_kernel<<<blocks_for(n, 256), 256, 0, st>>>(inst, d_states, R, d_out);
    return cudaGetLastError();
}

}  // namespace pb
