// biclique_res.cu -- resident form of the biclique p-bit anneal for small
// instances (arXiv 2510.23419, Sec. 3; update groups of Sec. 1.2.2: the two
// sides of K_{n,n}).  One CTA anneals one block of 32 replicas from the initial
// state to the last sweep without leaving the SM: J and J^T and the spins of
// both sides live in shared memory, the two half-sweeps are separated by CTA
// barriers, and the energy, running best and best-state copies happen in the
// same launch.  Small instances are latency-bound in the per-half-sweep
// launches of the other forms; here a sweep costs no launch at all.
//
//  +-1 couplings (n <= 256): J as packed int8 words, fields by __dp4a (exact
//      integers), decisions against the FP64 threshold window of the level.
//  real couplings (n <= 128): J in FP32, fields by FFMA, the FP32 rule.
//
// Random words, thresholds and the energy convention are those of the other
// forms, so the trajectories are the same as theirs (bit-exact for +-1).
#include <cuda_runtime.h>

#include <mutex>

#include "biclique_launch.h"
#include "ea_kernels.cuh"

namespace pb {

namespace {

constexpr int kRB = kBqResReps;             // replicas per CTA
constexpr int kThreads = 1024;
constexpr int kQuads = kRB / 4;             // replica quads per row
constexpr int kGroups = kThreads / kQuads;  // threads per replica quad

struct ResLayout {
    size_t J, sp, red, tab, total;
};

__host__ __device__ inline ResLayout res_layout(int jtype, int n, int tab_cap)
{
    ResLayout L{};
    const size_t n4 = (size_t)(n + 3) / 4;
    if (jtype == PB_J_PM1_I8) {
        L.J = 2 * n4 * n * 4;     // Jw [n4][n], JTw [n4][n] words
        L.sp = 2 * n4 * kRB * 4;  // sa, sb [n4][kRB] words
    } else {
        L.J = 2 * (size_t)n * n * 4;  // Jt [n][n], Jr [n][n] floats
        L.sp = 2 * (size_t)n * kRB * 4;
    }
    L.red = (size_t)kGroups * kRB * 8;  // per-thread-group energies (int64 or double)
    L.tab = (size_t)tab_cap * 4;
    // every segment starts on a 16-byte boundary (vector loads of spin words)
    L.J = (L.J + 15) & ~(size_t)15;
    L.sp = (L.sp + 15) & ~(size_t)15;
    L.red = (L.red + 15) & ~(size_t)15;
    L.tab = (L.tab + 15) & ~(size_t)15;
    L.total = L.J + L.sp + L.red + L.tab;
    return L;
}

__device__ __forceinline__ uint8_t enc_byte(bool minus) { return minus ? kE4m3Minus : kE4m3Plus; }
__device__ __forceinline__ uint16_t enc_half(bool minus) { return minus ? kBf16Minus : kBf16Plus; }

template <int JT>
__global__ void __launch_bounds__(kThreads, 1) bq_res_kernel(BqJob job, int tab_cap)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int n = job.inst.n, n4 = (n + 3) / 4;
    const int t = threadIdx.x;
    const int rb = blockIdx.x * kRB;  // first global replica of the block
    const ResLayout Lo = res_layout(JT, n, tab_cap);
    unsigned char* pJ = sm;
    unsigned char* pS = sm + Lo.J;
    unsigned char* pR = pS + Lo.sp;
    uint32_t* stab = reinterpret_cast<uint32_t*>(pR + Lo.red);
    constexpr bool PM1 = JT == PB_J_PM1_I8;

    // ---- J (and J^T) into shared memory
    if (PM1) {
        uint32_t* Jw = reinterpret_cast<uint32_t*>(pJ);  // Jw[j4 n + i] = J[i][4 j4 .. 4 j4 + 3]
        uint32_t* JTw = Jw + (size_t)n4 * n;              // JTw[i4 n + j] = J[4 i4 .. 4 i4 + 3][j]
        const int8_t* J = static_cast<const int8_t*>(job.inst.Jraw);
        for (int idx = t; idx < n4 * n; idx += kThreads) {
            const int w4 = idx / n, x = idx - w4 * n;
            uint32_t a = 0, b = 0;
            for (int k = 0; k < 4; ++k) {
                const int y = 4 * w4 + k;
                if (y < n) {
                    a |= (uint32_t)(uint8_t)J[(size_t)x * n + y] << (8 * k);
                    b |= (uint32_t)(uint8_t)J[(size_t)y * n + x] << (8 * k);
                }
            }
            Jw[idx] = a;
            JTw[idx] = b;
        }
    } else {
        float* Jt = reinterpret_cast<float*>(pJ);  // Jt[j n + i] = J[i][j]
        float* Jr = Jt + (size_t)n * n;             // Jr[i n + j] = J[i][j]
        for (int idx = t; idx < n * n; idx += kThreads) {
            Jt[idx] = job.inst.Jft[idx];
            Jr[idx] = job.inst.Jf[idx];
        }
    }

    // ---- initial state (tag 1); 0 in the padding bytes of +-1 words
    if (PM1) {
        uint32_t* sw = reinterpret_cast<uint32_t*>(pS);  // [side][n4][kRB]
        for (int idx = t; idx < 2 * n4 * kRB; idx += kThreads) sw[idx] = 0;
    }
    __syncthreads();
    for (int idx = t; idx < 2 * n * kQuads; idx += kThreads) {
        const int side = idx / (n * kQuads), rem = idx - side * n * kQuads;
        const int i = rem / kQuads, q4 = rem - i * kQuads;
        const U4 w = philox10((uint32_t)i, 0u, (uint32_t)((rb + 4 * q4) >> 2), (kTagInit << 24) | (uint32_t)side,
                              job.key0, job.key1);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        for (int k = 0; k < 4; ++k) {
            const bool minus = ws[k] >= 0x80000000u;
            const int r = 4 * q4 + k;
            if (PM1)
                pS[(((size_t)side * n4 + (i >> 2)) * kRB + r) * 4 + (i & 3)] = minus ? 0xFFu : 0x01u;
            else
                reinterpret_cast<float*>(pS)[((size_t)side * n + i) * kRB + r] = minus ? -1.0f : 1.0f;
        }
    }
    __syncthreads();

    // A thread owns replica quad rq (replicas r0 .. r0 + 3 of the block) and rows
    // g, g + kGroups, ... of a side; it accumulates its energy terms in ei / ef.
    const int rq = t % kQuads, g = t / kQuads;
    const int r0 = 4 * rq;
    long long ei[4];
    double ef[4];
    // Field (and, with decide, the p-bit decision) of one side for this thread's rows.
    auto half = [&](int side, int s, bool decide, TabWindow win, float cexp) {
        const int8_t* hs8 = job.inst.h8 ? job.inst.h8 + side * n : nullptr;
        const float* hsf = job.inst.hf + side * n;
        for (int i = g; i < n; i += kGroups) {
            float Ff[4];
            int Fi[4];
            if (PM1) {
                const uint32_t* Jm = reinterpret_cast<const uint32_t*>(pJ) + (side == 0 ? 0 : (size_t)n4 * n);
                const uint32_t* so = reinterpret_cast<const uint32_t*>(pS) + (size_t)(1 - side) * n4 * kRB;
                int acc[4] = {0, 0, 0, 0};
                for (int w4 = 0; w4 < n4; ++w4) {
                    const int jw = (int)Jm[(size_t)w4 * n + i];
                    const uint4 bw = *reinterpret_cast<const uint4*>(so + (size_t)w4 * kRB + r0);
                    acc[0] = __dp4a(jw, (int)bw.x, acc[0]);
                    acc[1] = __dp4a(jw, (int)bw.y, acc[1]);
                    acc[2] = __dp4a(jw, (int)bw.z, acc[2]);
                    acc[3] = __dp4a(jw, (int)bw.w, acc[3]);
                }
                const int h = hs8 ? hs8[i] : 0;
                for (int k = 0; k < 4; ++k) Fi[k] = acc[k] + h;
            } else {
                const float* Jm = reinterpret_cast<const float*>(pJ) + (side == 0 ? 0 : (size_t)n * n);
                const float* so = reinterpret_cast<const float*>(pS) + (size_t)(1 - side) * n * kRB;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                for (int j = 0; j < n; ++j) {
                    const float Jv = Jm[(size_t)j * n + i];  // side 0: J[i][j]; side 1: J[j][i] (i is the B index)
                    const float4 bv = *reinterpret_cast<const float4*>(so + (size_t)j * kRB + r0);
                    acc[0] = fmaf(Jv, bv.x, acc[0]);
                    acc[1] = fmaf(Jv, bv.y, acc[1]);
                    acc[2] = fmaf(Jv, bv.z, acc[2]);
                    acc[3] = fmaf(Jv, bv.w, acc[3]);
                }
                for (int k = 0; k < 4; ++k) Ff[k] = acc[k] + hsf[i];
            }
            bool mn[4];
            if (decide) {
                const U4 w = philox10((uint32_t)i, (uint32_t)s, (uint32_t)((rb + r0) >> 2),
                                      (kTagDecision << 24) | (uint32_t)side, job.key0, job.key1);
                const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
                for (int k = 0; k < 4; ++k) {
                    if (PM1) {
                        const int f = min(max(Fi[k] - job.fmin, win.lo), win.lo + win.width - 1) - win.lo;
                        mn[k] = ws[k] >= stab[f];
                        pS[(((size_t)side * n4 + (i >> 2)) * kRB + r0 + k) * 4 + (i & 3)] = mn[k] ? 0xFFu : 0x01u;
                    } else {
                        mn[k] = decide_f32(ws[k], Ff[k], cexp) != 0u;
                        reinterpret_cast<float*>(pS)[((size_t)side * n + i) * kRB + r0 + k] = mn[k] ? -1.0f : 1.0f;
                    }
                }
            } else {
                for (int k = 0; k < 4; ++k)
                    mn[k] = PM1 ? pS[(((size_t)side * n4 + (i >> 2)) * kRB + r0 + k) * 4 + (i & 3)] == 0xFFu
                                : reinterpret_cast<const float*>(pS)[((size_t)side * n + i) * kRB + r0 + k] < 0.0f;
            }
            // energy: side 1 contributes -b F_B (F_B includes h_B), side 0 only -h_A a
            for (int k = 0; k < 4; ++k) {
                if (PM1) {
                    const long long x = side == 1 ? Fi[k] : (hs8 ? hs8[i] : 0);
                    ei[k] += mn[k] ? x : -x;
                } else {
                    const double x = side == 1 ? (double)Ff[k] : (double)hsf[i];
                    ef[k] += mn[k] ? x : -x;
                }
            }
        }
    };
    // Per-replica energy from the thread groups' terms, summed in a fixed order.
    auto reduce_energy = [&](double* Eout) {
        for (int k = 0; k < 4; ++k) {
            if (PM1) reinterpret_cast<long long*>(pR)[(size_t)g * kRB + r0 + k] = ei[k];
            else reinterpret_cast<double*>(pR)[(size_t)g * kRB + r0 + k] = ef[k];
        }
        __syncthreads();
        if (t < kRB) {
            if (PM1) {
                long long e = 0;
                for (int q = 0; q < kGroups; ++q) e += reinterpret_cast<const long long*>(pR)[(size_t)q * kRB + t];
                *Eout = (double)e;
            } else {
                double e = 0.0;
                for (int q = 0; q < kGroups; ++q) e += reinterpret_cast<const double*>(pR)[(size_t)q * kRB + t];
                *Eout = e;
            }
        }
    };
    // Copy the replicas flagged in s_flag (a bit per replica) to the best buffers.
    __shared__ uint32_t s_flag;
    auto copy_best = [&]() {
        const uint32_t f = s_flag;
        if (!f) return;
        for (int idx = t; idx < 2 * n * kRB; idx += kThreads) {
            const int side = idx / (n * kRB), rem = idx - side * n * kRB;
            const int r = rem / n, i = rem - r * n;
            if (!((f >> r) & 1u)) continue;
            const size_t off = (size_t)(rb + r) * job.ld + i;
            if (PM1) {
                const bool minus = pS[(((size_t)side * n4 + (i >> 2)) * kRB + r) * 4 + (i & 3)] == 0xFFu;
                static_cast<uint8_t*>(job.best[side])[off] = enc_byte(minus);
            } else {
                const bool minus = reinterpret_cast<const float*>(pS)[((size_t)side * n + i) * kRB + r] < 0.0f;
                static_cast<uint16_t*>(job.best[side])[off] = enc_half(minus);
            }
        }
    };

    // ---- energy of the initial state: the first best (sweep -1)
    double E = 0.0, Ebest = 0.0;
    int bsweep = -1, hit = -1;
    for (int k = 0; k < 4; ++k) {
        ei[k] = 0;
        ef[k] = 0.0;
    }
    const TabWindow none{0, 0, 1};
    half(0, 0, false, none, 0.0f);
    half(1, 0, false, none, 0.0f);
    reduce_energy(&E);
    if (t == 0) s_flag = 0xFFFFFFFFu;
    if (t < kRB) Ebest = E;
    __syncthreads();
    copy_best();

    for (int s = 0; s < job.S; ++s) {
        const int lev = s / job.step;
        TabWindow win = none;
        float cexp = 0.0f;
        __syncthreads();  // the previous sweep's copies are done before the spins change
        if (PM1) {
            win = TabWindow{job.win[3 * lev + 2], job.win[3 * lev], job.win[3 * lev + 1]};
            for (int f = t; f < win.width; f += kThreads) stab[f] = job.table[win.off + f];
        } else {
            cexp = f32_cexp(job.betaf[lev]);
        }
        for (int k = 0; k < 4; ++k) {
            ei[k] = 0;
            ef[k] = 0.0;
        }
        if (t == 0) s_flag = 0;
        __syncthreads();
        half(0, s, true, win, cexp);
        __syncthreads();
        half(1, s, true, win, cexp);
        reduce_energy(&E);  // its barrier ends side B
        if (t < kRB) {
            if ((job.has_target != 2 || hit < 0) && E < Ebest) {  // stop mode: the best is frozen at the target
                Ebest = E;
                bsweep = s;
                atomicOr(&s_flag, 1u << t);
            }
            if (job.has_target && hit < 0 && E <= (PM1 ? (double)job.target_i : (double)job.target_f)) hit = s;
        }
        __syncthreads();
        copy_best();
        // stop mode: the block ends once its replicas (padding included) have reached the target; its
        // final state still goes to the buffers of the last sweep's parity, where the readout looks
        if (job.has_target == 2 && __syncthreads_and(t >= kRB || hit >= 0 || rb + t >= job.R)) break;
    }
    // ---- outputs: final state (in the buffers of the last sweep's parity), best energies and sweeps
    __syncthreads();
    const int last = (job.S - 1) & 1;
    for (int idx = t; idx < 2 * n * kRB; idx += kThreads) {
        const int side = idx / (n * kRB), rem = idx - side * n * kRB;
        const int r = rem / n, i = rem - r * n;
        const size_t off = (size_t)(rb + r) * job.ld + i;
        if (PM1) {
            const bool minus = pS[(((size_t)side * n4 + (i >> 2)) * kRB + r) * 4 + (i & 3)] == 0xFFu;
            static_cast<uint8_t*>(job.buf[side][last])[off] = enc_byte(minus);
        } else {
            const bool minus = reinterpret_cast<const float*>(pS)[((size_t)side * n + i) * kRB + r] < 0.0f;
            static_cast<uint16_t*>(job.buf[side][last])[off] = enc_half(minus);
        }
    }
    if (t < kRB) {
        if (PM1) job.E_best_i[rb + t] = (int32_t)Ebest;
        else job.E_best_f[rb + t] = (float)Ebest;
        job.best_sweep[rb + t] = bsweep;
        job.hit_sweep[rb + t] = hit;
    }
}

}  // namespace

size_t bq_res_smem_bytes(int jtype, int n, int tab_cap) { return res_layout(jtype, n, tab_cap).total; }

// The limit belongs to the kernel and is shared by every run of the process:
// it only grows, so preparing a smaller run never breaks a larger prepared one.
cudaError_t bq_res_set_smem(int jtype, size_t bytes)
{
    static std::mutex mu;
    static size_t current[64][2] = {};
    const int k = jtype == PB_J_PM1_I8 ? 0 : 1;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    size_t* cur = (dev >= 0 && dev < 64) ? &current[dev][k] : nullptr;
    if (cur && bytes <= *cur) return cudaSuccess;
    const cudaError_t e =
        k == 0 ? cudaFuncSetAttribute(bq_res_kernel<PB_J_PM1_I8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
               : cudaFuncSetAttribute(bq_res_kernel<PB_J_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && cur) *cur = bytes;
    return e;
}

cudaError_t bq_launch_res(const BqJob& job, int tab_cap, size_t smem, cudaStream_t st)
{
    const unsigned grid = (unsigned)(job.Rpad / kRB);
    if (job.inst.jtype == PB_J_PM1_I8)
        bq_res_kernel<PB_J_PM1_I8><<<grid, kThreads, smem, st>>>(job, tab_cap);
    else
        bq_res_kernel<PB_J_F32><<<grid, kThreads, smem, st>>>(job, tab_cap);
    return cudaGetLastError();
}

}  // namespace pb
