// biclique.cu -- CUDA-core kernels of the p-bit update on complete bipartite
// graphs K_{n,n} (arXiv 2510.23419, Sec. 3; update groups Sec. 1.2.2: the
// two sides are the two colour classes, every neighbour is shared by the
// whole class, so the field of a side is one dense product J M over replicas).
//
// The field F_A[r][i] = sum_j J[i][j] b[r][j] + h_i (Eq. 3) is an FP32 FMA
// tile product; the epilogue applies the p-bit decision (Eq. 2) with the
// Philox word of (i, s, r >> 2, side) and writes the new spins.  Fields of
// +-1 instances are exact integers in FP32 (|F| <= n + |h| < 2^24).
#include "biclique_launch.h"
#include "ea_kernels.cuh"

namespace pb {

namespace {

template <int SB>
struct SpinCode;
template <>
struct SpinCode<1> {
    using T = uint8_t;
    __device__ static float to_f(T v) { return __uint_as_float(0x3F800000u | ((uint32_t)(v & 0x80u) << 24)); }
    __device__ static T enc(bool minus) { return minus ? kE4m3Minus : kE4m3Plus; }
    __device__ static bool minus(T v) { return (v & 0x80u) != 0; }
};
template <>
struct SpinCode<2> {
    using T = uint16_t;
    __device__ static float to_f(T v) { return __uint_as_float((uint32_t)v << 16); }
    __device__ static T enc(bool minus) { return minus ? kBf16Minus : kBf16Plus; }
    __device__ static bool minus(T v) { return (v & 0x8000u) != 0; }
};


__global__ void __launch_bounds__(256) bq_init_kernel(BqJob job)
{
    const int n = job.inst.n;
    const long long tot = 2LL * job.Rpad * n;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= tot) return;
    const int side = (int)(j / ((long long)job.Rpad * n));
    const long long rem = j - (long long)side * job.Rpad * n;
    const int r = (int)(rem / n);
    const int i = (int)(rem - (long long)r * n);
    const U4 w = philox10((uint32_t)i, 0u, (uint32_t)(r >> 2), (kTagInit << 24) | (uint32_t)side, job.key0, job.key1);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    const bool minus = ws[r & 3] >= 0x80000000u;
    const size_t off = (size_t)r * job.ld + i;
    if (job.inst.jtype == PB_J_PM1_I8)
        static_cast<uint8_t*>(job.spins[side])[off] = minus ? kE4m3Minus : kE4m3Plus;
    else
        static_cast<uint16_t*>(job.spins[side])[off] = minus ? kBf16Minus : kBf16Plus;
}

// +-1 states (int8, [R][2n]) -> encoded spins of both sides.
__global__ void __launch_bounds__(256) bq_encode_kernel(BqJob job, const int8_t* __restrict__ m)
{
    const int n = job.inst.n;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (long long)job.R * 2 * n) return;
    const int r = (int)(j / (2 * n));
    const int c = (int)(j - (long long)r * 2 * n);
    const int side = c >= n ? 1 : 0;
    const int i = c - side * n;
    const bool minus = m[j] < 0;
    const size_t off = (size_t)r * job.ld + i;
    if (job.inst.jtype == PB_J_PM1_I8)
        static_cast<uint8_t*>(job.spins[side])[off] = minus ? kE4m3Minus : kE4m3Plus;
    else
        static_cast<uint16_t*>(job.spins[side])[off] = minus ? kBf16Minus : kBf16Plus;
}

constexpr int BM = kBqTileRows, BN = kBqTileReps, BK = 32;

template <int SB>
__global__ void __launch_bounds__(256) bq_cc_half_kernel(BqJob job, int side, int s, int decide, float* fields_out)
{
    using SC = SpinCode<SB>;
    using ST = typename SC::T;
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];
    __shared__ float red[16][BN + 1];
    __shared__ float redh[16][BN + 1];

    const int n = job.inst.n;
    const float* __restrict__ Jm = side == 0 ? job.inst.Jf : job.inst.Jft;
    const ST* __restrict__ other = static_cast<const ST*>(job.spins[1 - side]);
    ST* __restrict__ own = static_cast<ST*>(job.spins[side]);
    const int i0 = blockIdx.x * BM;
    const int r0 = blockIdx.y * BN;
    const int t = threadIdx.x;
    const int ty = t >> 4, tx = t & 15;

    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;

    const int lrow = t >> 2;          // 0..63
    const int lcol = (t & 3) * 8;     // 0, 8, 16, 24
    for (int j0 = 0; j0 < n; j0 += BK) {
        {
            const int i = i0 + lrow;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = j0 + lcol + q;
                As[lcol + q][lrow] = (i < n && j < n) ? __ldg(Jm + (size_t)i * n + j) : 0.0f;
            }
            const int r = r0 + lrow;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = j0 + lcol + q;
                Bs[lcol + q][lrow] = (j < n) ? SC::to_f(other[(size_t)r * job.ld + j]) : 0.0f;
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
        }
        __syncthreads();
    }

    // ---- epilogue: decisions (Eq. 2), energy partials ----
    const bool pm1 = job.inst.jtype == PB_J_PM1_I8;
    const uint32_t* trow = nullptr;
    float cexp = 0.0f;
    if (pm1)
        trow = job.table + (size_t)(s / job.step) * job.nF;
    else
        cexp = f32_cexp(job.betaf[s / job.step]);
    float e_field[4] = {0.f, 0.f, 0.f, 0.f};  // -m F  (side B)
    float e_h[4] = {0.f, 0.f, 0.f, 0.f};      // -h m  (side A)
    const int rq = r0 + tx * 4;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int i = i0 + ty * 4 + x;
        if (i >= n) continue;
        const float hv = pm1 ? (job.inst.h8 ? (float)job.inst.h8[side * n + i] : 0.0f) : job.inst.hf[side * n + i];
        float F[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) F[b] = acc[x][b] + hv;
        if (fields_out) {
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (rq + b < job.R) fields_out[(size_t)(rq + b) * 2 * n + side * n + i] = F[b];
            continue;
        }
        bool mn[4];
        if (decide) {
            const U4 w = philox10((uint32_t)i, (uint32_t)s, (uint32_t)(rq >> 2), (kTagDecision << 24) | (uint32_t)side,
                                  job.key0, job.key1);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                mn[b] = pm1 ? (ws[b] >= trow[(int)F[b] - job.fmin]) : (decide_f32(ws[b], F[b], cexp) != 0u);
                own[(size_t)(rq + b) * job.ld + i] = SC::enc(mn[b]);
            }
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) mn[b] = SC::minus(own[(size_t)(rq + b) * job.ld + i]);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (side == 1) e_field[b] += mn[b] ? F[b] : -F[b];
            e_h[b] += mn[b] ? hv : -hv;
        }
    }
    if (fields_out) return;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        red[ty][tx * 4 + b] = e_field[b];
        redh[ty][tx * 4 + b] = e_h[b];
    }
    __syncthreads();
    if (t < BN) {
        float ef = 0.0f, eh = 0.0f;
        for (int q = 0; q < 16; ++q) {
            ef += red[q][t];
            eh += redh[q][t];
        }
        // side A: -h.a ; side B: -b.F_B (F_B includes h_B) -> partial rows [0] and [1]
        const size_t off = ((size_t)side * job.nblk + blockIdx.x) * job.Rpad + r0 + t;
        const float v = side == 0 ? eh : ef;
        if (pm1)
            static_cast<int32_t*>(job.part)[off] = (int32_t)v;
        else
            static_cast<float*>(job.part)[off] = v;
    }
}

// One block per replica: energy of the state after the sweep, running best,
// snapshot of improved replicas.
__global__ void __launch_bounds__(128) bq_sweep_end_kernel(BqJob job, int s, int init)
{
    __shared__ int s_imp;
    const int r = blockIdx.x;
    const bool pm1 = job.inst.jtype == PB_J_PM1_I8;
    if (threadIdx.x == 0) {
        bool imp;
        if (pm1) {
            const int32_t* p = static_cast<const int32_t*>(job.part);
            int32_t E = 0;
            for (int side = 0; side < 2; ++side)
                for (int b = 0; b < job.nblk; ++b) E += p[((size_t)side * job.nblk + b) * job.Rpad + r];
            imp = init || E < job.E_best_i[r];
            if (imp) job.E_best_i[r] = E;
            if (!init && job.has_target && job.hit_sweep[r] < 0 && E <= job.target_i) job.hit_sweep[r] = s;
        } else {
            const float* p = static_cast<const float*>(job.part);
            float E = 0.0f;
            for (int side = 0; side < 2; ++side)
                for (int b = 0; b < job.nblk; ++b) E += p[((size_t)side * job.nblk + b) * job.Rpad + r];
            imp = init || E < job.E_best_f[r];
            if (imp) job.E_best_f[r] = E;
            if (!init && job.has_target && job.hit_sweep[r] < 0 && E <= job.target_f) job.hit_sweep[r] = s;
        }
        if (init) job.hit_sweep[r] = -1;
        if (imp) job.best_sweep[r] = init ? -1 : s;
        s_imp = imp ? 1 : 0;
    }
    __syncthreads();
    if (!s_imp) return;
    const int bytes = job.ld * (pm1 ? 1 : 2);
    for (int side = 0; side < 2; ++side) {
        const uint8_t* src = static_cast<const uint8_t*>(job.spins[side]) + (size_t)r * bytes;
        uint8_t* dst = static_cast<uint8_t*>(job.best[side]) + (size_t)r * bytes;
        for (int q = threadIdx.x * 4; q < bytes; q += blockDim.x * 4)
            *reinterpret_cast<uint32_t*>(dst + q) = *reinterpret_cast<const uint32_t*>(src + q);
    }
}

__global__ void __launch_bounds__(256) bq_readout_kernel(BqJob job, int which, int8_t* __restrict__ out)
{
    const int n = job.inst.n;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (long long)job.R * 2 * n) return;
    const int r = (int)(j / (2 * n));
    const int c = (int)(j - (long long)r * 2 * n);
    const int side = c >= n ? 1 : 0;
    const int i = c - side * n;
    void* const* src = which ? job.best : job.spins;
    bool minus;
    if (job.inst.jtype == PB_J_PM1_I8)
        minus = static_cast<const uint8_t*>(src[side])[(size_t)r * job.ld + i] & 0x80u;
    else
        minus = static_cast<const uint16_t*>(src[side])[(size_t)r * job.ld + i] & 0x8000u;
    out[j] = minus ? (int8_t)-1 : (int8_t)1;
}

// E = -sum_ij J_ij a_i b_j - sum h m, one block per replica: int64 (PM1) or FP64 (F32).
template <int JT>
__global__ void __launch_bounds__(256) bq_energy_kernel(BqJob job, const int8_t* __restrict__ m, double* __restrict__ E)
{
    __shared__ long long red_i[8];
    __shared__ double red_f[8];
    const int n = job.inst.n;
    const int r = blockIdx.x;
    const int8_t* a = m + (size_t)r * 2 * n;
    const int8_t* b = a + n;
    long long ai = 0;
    double af = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (JT == PB_J_PM1_I8) {
            const int8_t* Jr = static_cast<const int8_t*>(job.inst.Jraw) + (size_t)i * n;
            int u = 0;  // |u| <= n: exact in int32
            for (int j = 0; j < n; ++j) u += Jr[j] * b[j];
            ai -= (long long)u * a[i];
        } else {
            const float* Jr = static_cast<const float*>(job.inst.Jraw) + (size_t)i * n;
            double u = 0.0;
            for (int j = 0; j < n; ++j) u += (double)Jr[j] * (double)b[j];
            af -= u * (double)a[i];
        }
    }
    if (job.inst.hraw) {
        for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) {
            if (JT == PB_J_PM1_I8)
                ai -= (long long)static_cast<const int8_t*>(job.inst.hraw)[c] * a[c];
            else
                af -= (double)static_cast<const float*>(job.inst.hraw)[c] * (double)a[c];
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

unsigned nblocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t bq_launch_init(const BqJob& job, cudaStream_t st)
{
    const long long tot = 2LL * job.Rpad * job.inst.n;
    bq_init_kernel<<<nblocks(tot, 256), 256, 0, st>>>(job);
    return cudaGetLastError();
}

cudaError_t bq_launch_encode(const BqJob& job, const int8_t* d_states, cudaStream_t st)
{
    bq_encode_kernel<<<nblocks((long long)job.R * 2 * job.inst.n, 256), 256, 0, st>>>(job, d_states);
    return cudaGetLastError();
}

cudaError_t bq_launch_cc_half(const BqJob& job, int side, int s, int decide, float* fields_out, cudaStream_t st)
{
    dim3 grid((unsigned)((job.inst.n + BM - 1) / BM), (unsigned)(job.Rpad / BN));
    if (job.inst.jtype == PB_J_PM1_I8)
        bq_cc_half_kernel<1><<<grid, 256, 0, st>>>(job, side, s, decide, fields_out);
    else
        bq_cc_half_kernel<2><<<grid, 256, 0, st>>>(job, side, s, decide, fields_out);
    return cudaGetLastError();
}

cudaError_t bq_launch_sweep_end(const BqJob& job, int s, int init, cudaStream_t st)
{
    bq_sweep_end_kernel<<<job.Rpad, 128, 0, st>>>(job, s, init);
    return cudaGetLastError();
}

cudaError_t bq_launch_readout(const BqJob& job, int which, int8_t* out_pm, double* out_E, cudaStream_t st)
{
    bq_readout_kernel<<<nblocks((long long)job.R * 2 * job.inst.n, 256), 256, 0, st>>>(job, which, out_pm);
    if (job.inst.jtype == PB_J_PM1_I8)
        bq_energy_kernel<PB_J_PM1_I8><<<job.R, 256, 0, st>>>(job, out_pm, out_E);
    else
        bq_energy_kernel<PB_J_F32><<<job.R, 256, 0, st>>>(job, out_pm, out_E);
    return cudaGetLastError();
}

}  // namespace pb
