// csr.cu -- p-bit update on general sparse instances (arXiv 2510.23419: the
// Ising graph of Eq. 1 with an arbitrary edge set; the update groups of
// Sec. 1.2.2 are the classes of a proper colouring, k >= 2 of them, updated in
// turn).  One launch per colour class and sweep (the plain form).
//
// Spins carry class-contiguous labels (a class is a label range).  A thread
// keeps one spin word (4 replicas) and walks its block's share of the class:
// for each spin i, F_r = sum_j J_ij m_j(r) + h_i (Eq. 3) over i's row, then the
// p-bit decision (Eq. 2) with the Philox word of (class rank of i, s, word,
// colour).  Spins of one class have no edge between them, so the class is
// updated in place.
#include <algorithm>

#include "csr_launch.h"
#include "ea_kernels.cuh"

namespace pb {

namespace {

__device__ __forceinline__ uint32_t byte_of(uint32_t w, int b) { return (w >> (8 * b)) & 0xFFu; }

// Per-byte counts of the replicas' -1 spins over the neighbours x in [a, e),
// added to d with sign sgn: packed byte counters, emptied every 255 neighbours
// so no byte overflows.
__device__ __forceinline__ void count_minus(const CsrJob& job, const uint32_t* m, int a, int e, int q, int sgn,
                                            int (&d)[4])
{
    for (int seg = a; seg < e; seg += 255) {
        const int end = min(e, seg + 255);
        uint32_t acc = 0;
#pragma unroll 4
        for (int x = seg; x < end; ++x) acc += m[(size_t)job.g.col[x] * job.Rw + q];
#pragma unroll
        for (int b = 0; b < 4; ++b) d[b] += sgn * (int)byte_of(acc, b);
    }
}

// sum_j J_ij (1 - 2 bit_j) for 4 replicas of a +-1 row.  A row lists its
// J = +1 neighbours first and its J = -1 neighbours from rowneg[i] on, so the
// walk reads no coupling: G = sum_j J_ij - 2 (minus spins among the J = +1
// neighbours - minus spins among the J = -1 neighbours).
__device__ __forceinline__ void pm1_row(const CsrJob& job, const uint32_t* m, int i, int q, int (&G)[4])
{
    const int a0 = job.g.rowptr[i], an = job.g.rowneg[i], a1 = job.g.rowptr[i + 1];
    int d[4] = {0, 0, 0, 0};
    count_minus(job, m, a0, an, q, 1, d);
    count_minus(job, m, an, a1, q, -1, d);
    const int sumJ = (an - a0) - (a1 - an);
#pragma unroll
    for (int b = 0; b < 4; ++b) G[b] = sumJ - 2 * d[b];
}

// pm1_row of a padded row: all kCsrEllSlots neighbour words are fetched at once
// (unused slots read the zero row), then added to the J = +1 or J = -1 counter.
// The words go through the read-only data path: a class launch never writes
// another class's rows, and the zero row is never written.
__device__ __forceinline__ void pm1_row_ell(const CsrJob& job, const uint32_t* m, int p, int q, int (&G)[4])
{
    const int4 s0 = __ldg(job.g.ell + 2 * p), s1 = __ldg(job.g.ell + 2 * p + 1);
    const int nd = __ldg(job.g.ell_nd + p);
    const int np = nd & 0xFF, deg = nd >> 8;
    const int nb[kCsrEllSlots] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
    uint32_t w[kCsrEllSlots];
#pragma unroll
    for (int u = 0; u < kCsrEllSlots; ++u) w[u] = __ldg(m + (size_t)nb[u] * job.Rw + q);
    uint32_t accp = 0, accn = 0;  // at most 8 per byte: no overflow
#pragma unroll
    for (int u = 0; u < kCsrEllSlots; ++u) {
        if (u < np) accp += w[u];
        else accn += w[u];
    }
    const int sumJ = 2 * np - deg;
#pragma unroll
    for (int b = 0; b < 4; ++b) G[b] = sumJ - 2 * ((int)byte_of(accp, b) - (int)byte_of(accn, b));
}

template <typename T>
__device__ __forceinline__ void f32_row(const CsrJob& job, const uint32_t* m, int i, int q, T (&G)[4])
{
    const int a0 = job.g.rowptr[i], a1 = job.g.rowptr[i + 1];
#pragma unroll
    for (int b = 0; b < 4; ++b) G[b] = T(0);
    for (int a = a0; a < a1; ++a) {
        const uint32_t w = m[(size_t)job.g.col[a] * job.Rw + q];
        const T J = (T)job.g.Jf[a];
#pragma unroll
        for (int b = 0; b < 4; ++b) G[b] += byte_of(w, b) ? -J : J;
    }
}

__global__ void __launch_bounds__(256) csr_init_kernel(CsrJob job)
{
    const long long total = (long long)job.g.N * job.Rw;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(idx / job.Rw), q = (int)(idx - (long long)p * job.Rw);
        const int i = p;  // label
        const int c = job.g.colour[p];
        const uint32_t k = (uint32_t)(p - job.g.cls_off[c]);
        const U4 r = philox10(k, 0u, (uint32_t)q, (kTagInit << 24) | (uint32_t)c, job.key0, job.key1);
        const uint32_t ws[4] = {r.x, r.y, r.z, r.w};
        uint32_t w = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) w |= (ws[b] >= 0x80000000u ? 1u : 0u) << (8 * b);
        job.spins[(size_t)i * job.Rw + q] = w;
    }
}

// Block (kCsrLanesQ replica words) x (kCsrLanesV vertex lanes); block x takes
// the x-th of gridDim.x even, contiguous shares of the class's spins (the
// class chunk) and its vertex lanes walk that share with stride kCsrLanesV.  A
// thread keeps its replica word, adding the energy change of every flip,
// -2 m_new F (Eq. 3 fields); the block sums its lanes in a fixed order, then
// adds the +-1 sums (exact integers, so in any order) to the sweep's per-replica
// accumulator with 64-bit atomics, or stores the FP32 sums as the class chunk's
// partial.  Before a spin is overwritten, its value (the state at the end of the
// previous sweep: a class is not touched by the other classes' launches) is
// merged into the best state for the replicas whose energy improved then.
// ELL: +-1 rows padded to kCsrEllSlots labels (degree <= kCsrEllSlots).
// TEMP: tempering (each replica slot has its own temperature); otherwise one
// level for the launch, whose +-1 threshold window the block stages in shared
// memory (windows wider than kCsrWinSmem stay in global memory).
constexpr int kCsrWinSmem = 256;

template <int JT, bool TEMP, bool ELL>
__global__ void __launch_bounds__(kCsrLanesQ* kCsrLanesV) csr_class_kernel(CsrJob job, int c, int s)
{
    constexpr bool PM1 = JT == PB_J_PM1_I8;
    if (job.has_target == 2 && job.stop[1] >= 0) return;  // stop mode: every replica has reached the target
    __shared__ int32_t red_i[kCsrLanesV][kCsrLanesQ][4];
    __shared__ float red_f[kCsrLanesV][kCsrLanesQ][4];
    __shared__ uint32_t s_win[kCsrWinSmem];
    const int off = job.g.cls_off[c], ncls = job.g.cls_off[c + 1] - off;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int q = blockIdx.y * kCsrLanesQ + tx;
    TabWindow win{0, 0, 1};
    float cexp = 0.0f;
    const uint32_t* wtab = nullptr;  // the window's entries (shared or global)
    if constexpr (!TEMP) {
        const int lev = s / job.step;
        if constexpr (PM1) {
            win = TabWindow{job.win[3 * lev + 2], job.win[3 * lev], job.win[3 * lev + 1]};
            if (win.width <= kCsrWinSmem) {
                for (int e = ty * kCsrLanesQ + tx; e < win.width; e += kCsrLanesQ * kCsrLanesV)
                    s_win[e] = job.table[win.off + e];
                __syncthreads();
                wtab = s_win;
            } else {
                wtab = job.table + win.off;
            }
        } else {
            cexp = f32_cexp(job.betaf[lev]);
        }
    }
    int32_t di[4] = {0, 0, 0, 0};  // |changes| <= kCsrMaxVpt * 2 (maxdeg + hmax) < 2^31 (checked at setup)
    float df[4] = {0.f, 0.f, 0.f, 0.f};
    if (q < job.Rw) {
        const uint32_t fl = *reinterpret_cast<const uint32_t*>(job.improved + 4 * q);  // 4 flag bytes
        const uint32_t fmask = fl * 0xFFu;                                             // 0x01 -> 0xFF per byte
        const int t0 = (int)((long long)ncls * blockIdx.x / gridDim.x);
        const int t1 = (int)((long long)ncls * (blockIdx.x + 1) / gridDim.x);
        for (int t = t0 + ty; t < t1; t += kCsrLanesV) {
            const int i = off + t;  // label
            const U4 r = philox10((uint32_t)t, (uint32_t)s, (uint32_t)q, (kTagDecision << 24) | (uint32_t)c, job.key0,
                                  job.key1);
            const uint32_t ws[4] = {r.x, r.y, r.z, r.w};
            const uint32_t wold = job.spins[(size_t)i * job.Rw + q];
            if (fmask) {
                uint32_t* bp = job.best + (size_t)i * job.Rw + q;
                *bp = (wold & fmask) | (*bp & ~fmask);
            }
            uint32_t w = 0;
            if constexpr (PM1) {
                int G[4];
                if constexpr (ELL)
                    pm1_row_ell(job, job.spins, i, q, G);
                else
                    pm1_row(job, job.spins, i, q, G);
                const int h = job.g.h8 ? job.g.h8[i] : 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int F = G[b] + h;
                    uint32_t T;
                    if constexpr (TEMP) {
                        const int l = job.temp[4 * q + b];
                        const TabWindow wb{job.win[3 * l + 2], job.win[3 * l], job.win[3 * l + 1]};
                        T = job.table[wb.off + min(max(F - job.fmin, wb.lo), wb.lo + wb.width - 1) - wb.lo];
                    } else {
                        T = wtab[min(max(F - job.fmin - win.lo, 0), win.width - 1)];
                    }
                    const uint32_t nb = decide_bit(ws[b], T);
                    w |= nb << (8 * b);
                    if (nb != byte_of(wold, b)) di[b] += nb ? 2 * F : -2 * F;  // -2 m_new F
                }
            } else {
                float G[4];
                f32_row(job, job.spins, i, q, G);
                const float h = job.g.hf ? job.g.hf[i] : 0.0f;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float cb = TEMP ? f32_cexp(job.betaf[job.temp[4 * q + b]]) : cexp;
                    const float F = G[b] + h;
                    const uint32_t nb = decide_f32(ws[b], F, cb);
                    w |= nb << (8 * b);
                    if (nb != byte_of(wold, b)) df[b] += nb ? 2.0f * F : -2.0f * F;
                }
            }
            job.spins[(size_t)i * job.Rw + q] = w;
        }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        if constexpr (PM1)
            red_i[ty][tx][b] = di[b];
        else
            red_f[ty][tx][b] = df[b];
    }
    __syncthreads();
    if (ty == 0 && q < job.Rw) {
        if constexpr (PM1) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                long long t = 0;
                for (int v = 0; v < kCsrLanesV; ++v) t += red_i[v][tx][b];
                if (t) atomicAdd(job.dacc + 4 * q + b, (unsigned long long)t);
            }
        } else {
            double* out = job.dpart + (size_t)(job.dchunk_off[c] + blockIdx.x) * 4 * job.Rw + 4 * q;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                double t = 0.0;
                for (int v = 0; v < kCsrLanesV; ++v) t += (double)red_f[v][tx][b];
                out[b] = t;
            }
        }
    }
}

// 2E partials per chunk of kCsrChunk vertices: -(sum_i m_i G_i) - 2 sum_i h_i m_i,
// with G_i = sum_j J_ij m_j (every edge seen from both ends).  +-1: exact
// integers; real couplings: FP32 rows (running energy) or FP64 rows (EXACT).
template <int JT, bool EXACT>
__global__ void __launch_bounds__(128) csr_energy_kernel(CsrJob job, const uint32_t* __restrict__ m)
{
    const int q = blockIdx.y * blockDim.x + threadIdx.x;
    if (q >= job.Rw) return;
    const int i0 = blockIdx.x * kCsrChunk, i1 = min(job.g.N, i0 + kCsrChunk);
    double e[4] = {0.0, 0.0, 0.0, 0.0};
    long long ei[4] = {0, 0, 0, 0};
    for (int i = i0; i < i1; ++i) {
        const uint32_t mw = m[(size_t)i * job.Rw + q];
        if (JT == PB_J_PM1_I8) {
            int G[4];
            pm1_row(job, m, i, q, G);
            const int h = job.g.h8 ? job.g.h8[i] : 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int mi = byte_of(mw, b) ? -1 : 1;
                ei[b] -= (long long)mi * (G[b] + 2 * h);
            }
        } else if (EXACT) {
            double G[4];
            f32_row(job, m, i, q, G);
            const double h = job.g.hf ? (double)job.g.hf[i] : 0.0;
#pragma unroll
            for (int b = 0; b < 4; ++b) e[b] -= (byte_of(mw, b) ? -1.0 : 1.0) * (G[b] + 2.0 * h);
        } else {
            float G[4];
            f32_row(job, m, i, q, G);
            const float h = job.g.hf ? job.g.hf[i] : 0.0f;
#pragma unroll
            for (int b = 0; b < 4; ++b) e[b] -= (double)((byte_of(mw, b) ? -1.0f : 1.0f) * (G[b] + 2.0f * h));
        }
    }
    double* out = job.part + (size_t)blockIdx.x * 4 * job.Rw + 4 * q;
#pragma unroll
    for (int b = 0; b < 4; ++b) out[b] = JT == PB_J_PM1_I8 ? (double)ei[b] : e[b];
}

__device__ __forceinline__ double csr_energy_of(const CsrJob& job, int r)
{
    double t = 0.0;
    for (int ch = 0; ch < job.nchunk; ++ch) t += job.part[(size_t)ch * 4 * job.Rw + r];
    return 0.5 * t;
}

// 32 replicas per block.  +-1: the sweep's change is the accumulator, which is
// reset for the next sweep; FP32: kSweepEndWarps warps, warp w sums the
// class-chunk changes w, w + kSweepEndWarps, ... of its lane's replica, then
// the warp sums are added in order.
constexpr int kSweepEndWarps = 32;

__global__ void __launch_bounds__(kSweepEndWarps * 32) csr_sweep_end_kernel(CsrJob job, int s, int init)
{
    __shared__ double acc[kSweepEndWarps][32];
    // stop mode: nothing changes after the sweep at which every replica had reached the target
    if (!init && job.has_target == 2 && job.stop[1] >= 0) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int r = blockIdx.x * 32 + lane;
    const bool live = r < 4 * job.Rw;
    if (!init && !job.dacc) {
        double t = 0.0;
        if (live)
            for (int ch = wp; ch < job.ndchunk; ch += kSweepEndWarps) t += job.dpart[(size_t)ch * 4 * job.Rw + r];
        acc[wp][lane] = t;
    }
    __syncthreads();
    if (wp != 0 || !live) return;
    double E;
    if (init) {
        E = csr_energy_of(job, r);
    } else {
        double dE = 0.0;
        if (job.dacc) {
            dE = (double)(long long)job.dacc[r];
            job.dacc[r] = 0ull;
        } else {
            for (int w = 0; w < kSweepEndWarps; ++w) dE += acc[w][lane];
        }
        E = job.E_cur[r] + dE;  // energy changes of the sweep's classes
    }
    job.E_cur[r] = E;
    bool imp;
    if (init == 1) {
        imp = true;
        job.E_best[r] = E;
        job.best_sweep[r] = -1;
        job.hit_sweep[r] = -1;
    } else if (init == 2) {
        imp = false;  // resumed: the given best stays
        job.hit_sweep[r] = -1;
    } else {
        imp = (job.has_target != 2 || job.hit_sweep[r] < 0) && E < job.E_best[r];  // stop mode: frozen at the target
        if (imp) {
            job.E_best[r] = E;
            job.best_sweep[r] = s;
        }
        if (job.has_target && job.hit_sweep[r] < 0 && E <= job.target) {
            job.hit_sweep[r] = s;
            if (job.has_target == 2 && r < job.R && atomicAdd(job.stop, 1) + 1 == job.R) job.stop[1] = s;
        }
    }
    job.improved[r] = imp ? 1 : 0;
}

// best <- spins for the replicas flagged as improved (byte masks per word).
// A thread owns one replica word q and walks the vertices with a stride; it
// reads its 4 flag bytes once and leaves at once when none is set, which late
// in an anneal is nearly every word.
__global__ void __launch_bounds__(256) csr_snapshot_kernel(CsrJob job)
{
    const int q = blockIdx.x * 32 + (threadIdx.x & 31);
    if (q >= job.Rw) return;
    const uint32_t f = *reinterpret_cast<const uint32_t*>(job.improved + 4 * q);  // 4 flag bytes
    if (!f) return;
    const uint32_t mask = f * 0xFFu;  // 0x01 -> 0xFF per byte
    const int N = job.g.N;
    for (int i = blockIdx.y * 8 + (threadIdx.x >> 5); i < N; i += gridDim.y * 8) {
        const size_t idx = (size_t)i * job.Rw + q;
        job.best[idx] = (job.spins[idx] & mask) | (job.best[idx] & ~mask);
    }
}

// Replica exchange after sweep s (tempering): one thread per chain, pairs of
// the sweep's parity in increasing order; accepted with probability
// min(1, exp((beta_{t+1} - beta_t)(E_b - E_a))) by the word of counter
// (t, s, r >> 2, 3 << 24), index r & 3.  +-1: the host's FP64 threshold table
// (bit-exact with the oracle); real couplings: an FP32 rule like the p-bit
// decision's -- the exponent in FP32 (energies rounded to FP32, the pair's
// beta step times log2 e from the host), one exp2, and the uniform
// u = ((w >> 9) + 1/2) 2^-23 -- so no FP64 arithmetic runs on the device here.
__global__ void __launch_bounds__(128) csr_exchange_kernel(CsrJob job, int s)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= job.C) return;
    for (int t = s & 1; t + 1 < job.M; t += 2) {
        const int a = job.slot_of[t * job.C + r], b = job.slot_of[(t + 1) * job.C + r];
        const U4 rw = philox10((uint32_t)t, (uint32_t)s, (uint32_t)(r >> 2), 3u << 24, job.key0, job.key1);
        const uint32_t ws[4] = {rw.x, rw.y, rw.z, rw.w};
        const uint32_t w = ws[r & 3];
        bool accept;
        if (job.g.jtype == PB_J_PM1_I8) {
            // integer energies (held exactly): the host's FP64 table of floor(exp(dbeta (-d)) 2^32), d = 1, 2, ...
            const long long d = __double2ll_rn(job.E_cur[a]) - __double2ll_rn(job.E_cur[b]);
            if (d <= 0) {
                accept = true;
            } else {
                const int len = job.xwin[2 * t], off = job.xwin[2 * t + 1];
                accept = d <= len && w < job.xtab[off + (int)(d - 1)];
            }
        } else {
            const float y = job.xdb[t] * ((float)job.E_cur[b] - (float)job.E_cur[a]);  // x log2 e
            const float u = __uint_as_float(0x3F800000u | (w >> 9)) - 0.99999994f;
            accept = y >= 0.0f || u < ex2_ftz(y);
        }
        if (accept) {
            job.temp[a] = (uint8_t)(t + 1);
            job.temp[b] = (uint8_t)t;
            job.slot_of[t * job.C + r] = b;
            job.slot_of[(t + 1) * job.C + r] = a;
            atomicAdd(job.n_accept + t, 1ull);
        }
    }
}

__global__ void __launch_bounds__(256) csr_states_kernel(CsrJob job, const uint32_t* __restrict__ m, int8_t* out)
{
    const long long total = (long long)job.R * job.g.N;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / job.g.N), i = (int)(idx - (long long)r * job.g.N);  // original order
        const int p = job.g.pos[i];
        out[idx] = byte_of(m[(size_t)p * job.Rw + (r >> 2)], r & 3) ? (int8_t)-1 : (int8_t)1;
    }
}

__global__ void __launch_bounds__(256) csr_energy_out_kernel(CsrJob job, double* out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < job.R) out[r] = csr_energy_of(job, r);
}

__global__ void __launch_bounds__(256) csr_fields_kernel(CsrJob job, const int8_t* __restrict__ st, float* out)
{
    const long long total = (long long)job.R * job.g.N;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / job.g.N), i = (int)(idx - (long long)r * job.g.N);  // original order
        const int p = job.g.pos[i];
        const int8_t* mr = st + (size_t)r * job.g.N;
        float F = job.g.jtype == PB_J_PM1_I8 ? (job.g.h8 ? (float)job.g.h8[p] : 0.0f) : (job.g.hf ? job.g.hf[p] : 0.0f);
        for (int a = job.g.rowptr[p]; a < job.g.rowptr[p + 1]; ++a) {
            const float J = job.g.jtype == PB_J_PM1_I8 ? (float)job.g.J8[a] : job.g.Jf[a];
            F = fmaf(J, (float)mr[job.g.orig[job.g.col[a]]], F);
        }
        out[idx] = F;
    }
}

unsigned grid_for(long long total) { return (unsigned)std::max(1LL, std::min<long long>((total + 255) / 256, 152LL * 16)); }

}  // namespace

cudaError_t csr_launch_init(const CsrJob& job, cudaStream_t st)
{
    csr_init_kernel<<<grid_for((long long)job.g.N * job.Rw), 256, 0, st>>>(job);
    return cudaGetLastError();
}

int csr_class_blocks(int jtype, bool temp, int Rw, int ncls, int maxdeg, int hmax)
{
    if (ncls <= 0) return 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    const int threads = kCsrLanesQ * kCsrLanesV;
    cudaError_t e;
    const bool ell = jtype == PB_J_PM1_I8 && maxdeg <= kCsrEllSlots;
    if (jtype == PB_J_PM1_I8 && ell)
        e = temp ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_class_kernel<PB_J_PM1_I8, true, true>, threads, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_class_kernel<PB_J_PM1_I8, false, true>, threads, 0);
    else if (jtype == PB_J_PM1_I8)
        e = temp ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_class_kernel<PB_J_PM1_I8, true, false>, threads, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_class_kernel<PB_J_PM1_I8, false, false>, threads, 0);
    else
        e = temp ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_class_kernel<PB_J_F32, true, false>, threads, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_class_kernel<PB_J_F32, false, false>, threads, 0);
    if (e != cudaSuccess || per_sm < 1) return -1;
    // spins per thread: at most kCsrMaxVpt, and few enough that the int32 energy
    // changes cannot overflow
    const long long per_spin = 2LL * ((long long)maxdeg + hmax) + 1;
    const long long vpt = std::max(1LL, std::min<long long>(kCsrMaxVpt, 0x7FFFFFFFLL / per_spin));
    const long long gy = (Rw + kCsrLanesQ - 1) / kCsrLanesQ;
    const long long wave = std::max(1LL, (long long)per_sm * sms / gy);  // class blocks per full wave
    const long long lanes = ((long long)ncls + kCsrLanesV - 1) / kCsrLanesV;
    const long long need = (lanes + vpt - 1) / vpt;  // fewest blocks within the per-thread cap
    const long long waves = (need + wave - 1) / wave;
    return (int)std::min(lanes, waves * wave);
}

cudaError_t csr_launch_class(const CsrJob& job, int c, int nchunks, int s, cudaStream_t st)
{
    if (nchunks < 1) return cudaSuccess;
    const dim3 grid((unsigned)nchunks, (unsigned)((job.Rw + kCsrLanesQ - 1) / kCsrLanesQ));
    const dim3 block(kCsrLanesQ, kCsrLanesV);
    const bool pm1 = job.g.jtype == PB_J_PM1_I8, temp = job.temp != nullptr;
    const bool ell = job.g.ell != nullptr;
    if (pm1 && ell)
        temp ? csr_class_kernel<PB_J_PM1_I8, true, true><<<grid, block, 0, st>>>(job, c, s)
             : csr_class_kernel<PB_J_PM1_I8, false, true><<<grid, block, 0, st>>>(job, c, s);
    else if (pm1)
        temp ? csr_class_kernel<PB_J_PM1_I8, true, false><<<grid, block, 0, st>>>(job, c, s)
             : csr_class_kernel<PB_J_PM1_I8, false, false><<<grid, block, 0, st>>>(job, c, s);
    else if (!temp)
        csr_class_kernel<PB_J_F32, false, false><<<grid, block, 0, st>>>(job, c, s);
    else
        csr_class_kernel<PB_J_F32, true, false><<<grid, block, 0, st>>>(job, c, s);
    return cudaGetLastError();
}

cudaError_t csr_launch_energy(const CsrJob& job, const uint32_t* m, int exact, cudaStream_t st)
{
    const dim3 grid((unsigned)job.nchunk, (unsigned)((job.Rw + 127) / 128));
    if (job.g.jtype == PB_J_PM1_I8)
        csr_energy_kernel<PB_J_PM1_I8, true><<<grid, 128, 0, st>>>(job, m);
    else if (exact)
        csr_energy_kernel<PB_J_F32, true><<<grid, 128, 0, st>>>(job, m);
    else
        csr_energy_kernel<PB_J_F32, false><<<grid, 128, 0, st>>>(job, m);
    return cudaGetLastError();
}

cudaError_t csr_launch_sweep_end(const CsrJob& job, int s, int init, cudaStream_t st)
{
    csr_sweep_end_kernel<<<(4 * job.Rw + 31) / 32, kSweepEndWarps * 32, 0, st>>>(job, s, init);
    return cudaGetLastError();
}

cudaError_t csr_launch_snapshot(const CsrJob& job, cudaStream_t st)
{
    const int gx = (job.Rw + 31) / 32;
    const int gy = std::max(1, std::min((job.g.N + 7) / 8, 152 * 8 / gx));
    csr_snapshot_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(job);
    return cudaGetLastError();
}

cudaError_t csr_launch_exchange(const CsrJob& job, int s, cudaStream_t st)
{
    csr_exchange_kernel<<<(job.C + 127) / 128, 128, 0, st>>>(job, s);
    return cudaGetLastError();
}

cudaError_t csr_launch_readout(const CsrJob& job, const uint32_t* m, int8_t* out_pm, double* out_E, cudaStream_t st)
{
    csr_states_kernel<<<grid_for((long long)job.R * job.g.N), 256, 0, st>>>(job, m, out_pm);
    cudaError_t e = csr_launch_energy(job, m, 1, st);
    if (e != cudaSuccess) return e;
    csr_energy_out_kernel<<<(job.R + 255) / 256, 256, 0, st>>>(job, out_E);
    return cudaGetLastError();
}

cudaError_t csr_launch_fields(const CsrJob& job, const int8_t* states, float* out, cudaStream_t st)
{
    csr_fields_kernel<<<grid_for((long long)job.R * job.g.N), 256, 0, st>>>(job, states, out);
    return cudaGetLastError();
}

}  // namespace pb
