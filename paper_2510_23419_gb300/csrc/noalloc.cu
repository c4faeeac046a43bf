// noalloc.cu -- an EA +-1 anneal entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool or
// arena it does not own (a serving framework that pre-plans all device
// memory), code running while another component holds the allocator, or
// real-time loops where an allocation (and the device synchronisation it may
// cause) is not allowed.  For them, pb_anneal_ea_noalloc runs the same
// resident kernel as pb_anneal, but every scratch buffer it needs lives in one
// file-scope device array of fixed size, and inputs and outputs are device
// buffers the caller already owns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "ea_launch.h"
#include "pb_common.h"

namespace pb {
int sm_count();
pb_status schedule_levels(const pb_schedule* sc, std::vector<double>& betas, int& step);
uint32_t threshold_u32(double beta, double F);
}  // namespace pb

namespace {

using namespace pb;

constexpr size_t kScratchBytes = 16u << 20;  // 16 MiB, held on every device that loads the library

// The scratch of pb_anneal_ea_noalloc.  In host code this name is only a
// host-side stand-in; its device address comes from cudaGetSymbolAddress.
// The library is built without relocatable device code and CUDA may load
// modules lazily, so a device may reserve this array only when this file's
// module is first used there -- normally inside the first call on that device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
pb_status scratch_address(unsigned char** out)
{
    int dev = 0;
    PB_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(PB_EUNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return PB_OK;
}

// +-1 couplings [3][N] -> per-site bond-sign bytes in the kernels' layout
// (bond order +x, -x, +y, -y, +z, -z; bit 2+b set when bond b is negative).
__global__ void __launch_bounds__(256) noalloc_jbits_kernel(const int8_t* __restrict__ J, int L, uint8_t* __restrict__ jb,
                                                            int* __restrict__ bad)
{
    const int N = L * L * L, half = N / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int x = i % L, y = (i / L) % L, z = i / (L * L);
    const int xm = (x + L - 1) % L, ym = (y + L - 1) % L, zm = (z + L - 1) % L;
    const int bonds[6] = {i, xm + L * (y + L * z), N + i, N + x + L * (ym + L * z), 2 * N + i, 2 * N + x + L * (y + L * zm)};
    uint8_t bits = 0;
    for (int b = 0; b < 6; ++b) {
        const int v = J[bonds[b]];
        if (v != 1 && v != -1) atomicOr(bad, 1);
        if (v < 0) bits |= (uint8_t)(1u << (2 + b));
    }
    jb[((x + y + z) & 1) * half + (i >> 1)] = bits;
}

// Couplings other than +-1 were seen (flag set by noalloc_jbits_kernel): mark every
// replica's outputs so the caller can tell, without this call reading anything back.
__global__ void __launch_bounds__(256) noalloc_mark_bad_kernel(const int* __restrict__ bad, int R, double* best_E,
                                                               double* final_E, int32_t* best_sweep)
{
    if (*bad == 0) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    best_E[r] = __longlong_as_double(0x7FF8000000000000LL);
    final_E[r] = __longlong_as_double(0x7FF8000000000000LL);
    best_sweep[r] = PB_NOALLOC_BAD_COUPLINGS;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" pb_status pb_anneal_ea_noalloc(int32_t L, const int8_t* J_dev, const pb_schedule* sched, int32_t replicas,
                                          uint64_t seed, double* best_E_dev, int32_t* best_sweep_dev,
                                          int8_t* best_states_dev, double* final_E_dev, int8_t* final_states_dev,
                                          void* stream)
{
    if (!J_dev || !sched || !best_E_dev || !best_sweep_dev || !best_states_dev || !final_E_dev || !final_states_dev)
        return fail(PB_EINVAL, "null argument");
    if (L < 2 || L > 32) return fail(PB_EINVAL, "pb_anneal_ea_noalloc: L must be in [2, 32]");
    if (L % 2) return fail(PB_ECOLOUR, "the checkerboard colouring of a periodic cube needs an even L");
    if (replicas < 1) return fail(PB_EINVAL, "replicas must be >= 1");
    std::vector<double> betas;
    int step = 1;
    pb_status ps = schedule_levels(sched, betas, step);
    if (ps != PB_OK) return ps;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const int N = L * L * L;
    const int nF = 13, fmin = -6;
    const int Rw = (replicas + 3) / 4;
    int WT = ea_resident_pick_wt(L, PB_J_PM1_I8, 0, nF, Rw);
    if (WT == 0) return fail(PB_EUNSUPPORTED, "lattice too large for the resident form");
    const int sms = sm_count();
    while (WT > 1 && (Rw + WT - 1) / WT < sms) WT /= 2;
    const int n_tiles = (Rw + WT - 1) / WT;
    const int Rpad = n_tiles * 4 * WT;
    const int nlev = std::max<int>(1, (int)betas.size());

    // scratch layout
    size_t off = 0;
    const size_t o_job = off;      off = align256(off + sizeof(EaJob));
    const size_t o_work = off;     off = align256(off + (size_t)n_tiles * sizeof(EaWork));
    const size_t o_ctr = off;      off = align256(off + 16);
    const size_t o_jb = off;       off = align256(off + (size_t)N);
    const size_t o_tab = off;      off = align256(off + (size_t)nlev * nF * 4);
    const size_t o_best = off;     off = align256(off + (size_t)Rpad * N);
    const size_t o_final = off;    off = align256(off + (size_t)Rpad * N);
    const size_t o_E = off;        off = align256(off + (size_t)Rpad * 4);
    const size_t o_bs = off;       off = align256(off + (size_t)Rpad * 4);
    const size_t o_hit = off;      off = align256(off + (size_t)Rpad * 4);
    if (off > kScratchBytes)
        return fail(PB_EINVAL, "pb_anneal_ea_noalloc: request needs " + std::to_string(off) +
                                   " bytes of scratch; the fixed maximum is " + std::to_string(kScratchBytes) +
                                   " bytes (fewer replicas, a smaller L or fewer sweeps fit)");

    unsigned char* S = nullptr;
    ps = scratch_address(&S);
    if (ps != PB_OK) return ps;

    // threshold table (Eq. 2), FP64 on the host
    std::vector<uint32_t> tab((size_t)nlev * nF, 0x80000000u);
    for (size_t l = 0; l < betas.size(); ++l)
        for (int f = 0; f < nF; ++f) tab[l * nF + f] = threshold_u32(betas[l], (double)(f + fmin));

    EaJob j{};
    j.inst.L = L;
    j.inst.N = N;
    j.inst.half = N / 2;
    j.inst.jtype = PB_J_PM1_I8;
    j.inst.jbits = S + o_jb;
    j.inst.J3 = J_dev;
    j.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
    j.key1 = (uint32_t)(seed >> 32);
    j.S = sched->n_sweeps;
    j.step = step;
    j.nF = nF;
    j.fmin = fmin;
    j.table = reinterpret_cast<const uint32_t*>(S + o_tab);
    j.R = replicas;
    j.WT = WT;
    j.n_tiles = n_tiles;
    j.best_words = reinterpret_cast<uint32_t*>(S + o_best);
    j.final_words = reinterpret_cast<uint32_t*>(S + o_final);
    j.E_best_i = reinterpret_cast<int32_t*>(S + o_E);
    j.best_sweep = reinterpret_cast<int32_t*>(S + o_bs);
    j.hit_sweep = reinterpret_cast<int32_t*>(S + o_hit);
    std::vector<EaWork> work(n_tiles);
    for (int t = 0; t < n_tiles; ++t) work[t] = EaWork{0, t, ea_tile_path(j)};

    // Every call reuses the same array: reset what must start at zero (the tile
    // counter and the bad-coupling flag); everything else is overwritten before it is read.
    int* bad = reinterpret_cast<int*>(S + o_ctr + 8);
    PB_CUDA_TRY(cudaMemsetAsync(S + o_ctr, 0, 16, st));
    PB_CUDA_TRY(cudaMemcpyAsync(S + o_job, &j, sizeof(EaJob), cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(S + o_work, work.data(), work.size() * sizeof(EaWork), cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(S + o_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, st));
    noalloc_jbits_kernel<<<(N + 255) / 256, 256, 0, st>>>(J_dev, L, S + o_jb, bad);
    PB_CUDA_TRY(cudaGetLastError());

    const size_t smem = ea_resident_smem(L, WT, PB_J_PM1_I8, 0, nF);
    PB_CUDA_TRY(ea_resident_set_smem(kEaKernelPm1, smem));
    PB_CUDA_TRY(ea_launch_resident(kEaKernelPm1, reinterpret_cast<const EaJob*>(S + o_job),
                                   reinterpret_cast<const EaWork*>(S + o_work), n_tiles, reinterpret_cast<int*>(S + o_ctr),
                                   smem, std::min(n_tiles, sms), false, st));
    PB_CUDA_TRY(ea_launch_readout(j, j.final_words, final_states_dev, final_E_dev, st));
    PB_CUDA_TRY(ea_launch_readout(j, j.best_words, best_states_dev, best_E_dev, st));
    PB_CUDA_TRY(cudaMemcpyAsync(best_sweep_dev, j.best_sweep, (size_t)replicas * 4, cudaMemcpyDeviceToDevice, st));
    // the coupling check is reported in the outputs, so the call never waits for the GPU
    noalloc_mark_bad_kernel<<<(replicas + 255) / 256, 256, 0, st>>>(bad, replicas, best_E_dev, final_E_dev,
                                                                     best_sweep_dev);
    PB_CUDA_TRY(cudaGetLastError());
    return PB_OK;
}
