// biclique_tc.cu -- tcgen05 tensor-core field of the biclique p-bit update
// (arXiv 2510.23419, Sec. 3; update groups Sec. 1.2.2: each side is one colour
// class, so the fields of a whole side are one dense product J M over
// replicas).  A pair of CTAs computes a 256-row x 256-replica tile of
//     F[i][r] = sum_j J[i][j] m[r][j] + h_i                      (Eq. 3)
// with the FP32 accumulator in tensor memory, then applies the p-bit decision
// (Eq. 2) to it and writes the new spins of the side (and the energy
// partials of the sweep).  The kernel is persistent: clusters of two CTAs
// loop over the tiles, with two accumulators in tensor memory so that the
// epilogue of one tile overlaps the MMAs of the next.
//
//  +-1 couplings: A = J in FP8 e4m3, B = spins in e4m3 (+-1 exact),
//                 tcgen05.mma kind::f8f6f4, exact integer sums in FP32.
//  real couplings: J = hi + lo with hi = bf16(J), lo = bf16(J - hi); spins
//                 bf16 +-1; two kind::f16 MMAs per K step into one accumulator.
//
// Two CTAs (a cluster) form a pair that computes a 256-row x 256-replica tile
// with tcgen05.mma.cta_group::2 (M = 256): each CTA stages its own 128 rows of
// J and half of the spin tile, and keeps its 128 rows of the accumulator.
// Warp roles per CTA: warp 0 issues TMA loads (128-byte swizzle, K-major) into
// a STAGES-deep ring, warp 1 allocates tensor memory (and, in the even CTA,
// issues the MMAs), warps 2..17 run the epilogue (warp w reads tensor-memory
// lanes 32 (w % 4) .. +31, i.e. 32 rows, and a quarter of the 256 columns).
// Every mbarrier wait is bounded; on timeout the CTA records an error and
// still releases its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "biclique_launch.h"
#include "biclique_tc.h"
#include "ea_kernels.cuh"

namespace pb {

namespace {

constexpr int TBM = kBqTcRows;   // rows per tile (tensor-memory lanes)
constexpr int TBN = kBqTcReps;   // replicas per tile (accumulator columns)
constexpr int KBYTES = 128;     // K bytes per stage (one 128-byte swizzle row)
constexpr int kEpiWarps = 16;   // epilogue warps: four per tensor-memory lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kEpiCols = TBN / (kEpiWarps / 4);  // accumulator columns per epilogue warp

template <int KIND>
struct TcCfg;
// Per-CTA stage: this CTA's 128 rows of J (one or two operands) and its half
// (128 replicas) of the spin tile, 128 bytes of K each.
template <>
struct TcCfg<0> {  // e4m3
    static_assert(kBqTcWindowMax * 32 * 4 <= 33 * 1024, "replicated threshold window must fit the table region");
    static constexpr int STAGES = 5;
    static constexpr int TAB_BYTES = 33 * 1024;  // threshold row of up to 8448 entries (n + |h| <= 4223)
    static constexpr int A_BYTES = TBM * KBYTES;
    static constexpr int B_BYTES = (TBN / 2) * KBYTES;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int KELEM = 128;  // elements per stage
    static constexpr int KSTEP_BYTES = 32;  // one MMA consumes K = 32 e4m3
};
template <>
struct TcCfg<1> {  // bf16 hi + lo
    static constexpr int STAGES = 4;
    static constexpr int TAB_BYTES = 0;
    static constexpr int A_BYTES = TBM * KBYTES;
    static constexpr int B_BYTES = (TBN / 2) * KBYTES;
    static constexpr int STAGE_BYTES = 2 * A_BYTES + B_BYTES;
    static constexpr int KELEM = 64;
    static constexpr int KSTEP_BYTES = 32;  // one MMA consumes K = 16 bf16
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase with the given parity; returns false once
// `limit_ns` of the global timer have passed without it (the caller records
// an error word and stops waiting, so the kernel still ends).  Each try_wait
// may suspend the warp for up to 100 us (less under a shorter limit) until the
// phase completes, so a waiting warp issues almost nothing: the epilogue warps
// that wait for an accumulator share their schedulers with the load and MMA
// threads.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns)
{
    const uint32_t a = smem_u32(bar);
    const uint32_t hint = (uint32_t)(limit_ns < 100000u ? limit_ns / 4 : 100000u);
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity), "r"(hint)
            : "memory");
        if (ok) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// TMA load into this CTA's shared memory that signals the barrier at shared::cluster
// address `bar`, which may live in the peer CTA of the pair.
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}

// shared::cluster address of `p` (same offset) in the CTA of rank `rank`.
__device__ __forceinline__ uint32_t map_rank(const void* p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

// Philox4x32-10 of the counter (c0, c1, c2, c3) for a thread whose c0, c1, c3
// are fixed over a tile and c2 varies: the first round's c0 product and the
// key/counter words it is combined with are computed once per tile.
struct PhiloxFixed {
    uint32_t n0x;  // c1 ^ k0
    uint32_t n2;   // hi(MulA * c0) ^ c3 ^ k1
    uint32_t x3;   // lo(MulA * c0)
};

__device__ __forceinline__ PhiloxFixed philox_fixed(uint32_t c0, uint32_t c1, uint32_t c3, uint32_t k0, uint32_t k1)
{
    uint32_t hA, lA;
    mulhilo32(kPhiloxMulA, c0, hA, lA);
    return PhiloxFixed{c1 ^ k0, hA ^ c3 ^ k1, lA};
}

__device__ __forceinline__ U4 philox_c2(uint32_t c2, const PhiloxFixed& f, uint32_t k0, uint32_t k1)
{
    uint32_t hB, lB;
    mulhilo32(kPhiloxMulB, c2, hB, lB);
    uint32_t x0 = hB ^ f.n0x, x1 = lB, x2 = f.n2, x3 = f.x3;
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
        uint32_t hA2, lA2, hB2, lB2;
        mulhilo32(kPhiloxMulA, x0, hA2, lA2);
        mulhilo32(kPhiloxMulB, x2, hB2, lB2);
        const uint32_t y0 = hB2 ^ x1 ^ k0;
        const uint32_t y2 = hA2 ^ x3 ^ k1;
        x0 = y0;
        x1 = lB2;
        x2 = y2;
        x3 = lA2;
    }
    return U4{x0, x1, x2, x3};
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);            // start address
    d |= (uint64_t)(16u >> 4) << 16;                    // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;                  // stride byte offset
    d |= (uint64_t)1 << 46;                             // descriptor version
    d |= (uint64_t)2 << 61;                             // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format, both K-major, N, M.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t ab_format, int M, int N)
{
    return (1u << 4)                      // D format: F32
           | (ab_format << 7)              // A format
           | (ab_format << 10)             // B format
           | ((uint32_t)(N >> 3) << 17)    // N / 8
           | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// One M=256 MMA over the CTA pair: A rows 0..127 and B columns 0..127 from the
// issuing (even) CTA, A rows 128..255 and B columns 128..255 from its peer, at
// the same shared-memory offsets; each CTA's tensor memory holds its 128 rows.
template <int KIND>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    if (KIND == 0) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    }
}

// Arrive on the barrier at this shared offset in both CTAs of the pair once the MMAs complete.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "h"((uint16_t)0x3)
                 : "memory");
}

// 32 columns of this warp's 32 tensor-memory lanes.  The load and its wait are
// one asm statement, so the registers are defined only once the data has
// arrived (no use of them can be scheduled between the two).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// Sum over the 32 lanes of a warp, per column: lane l holds e[0..31] (columns)
// and ends with the sum of column l in e[0] (31 shuffles).
__device__ __forceinline__ float warp_transpose_sum(float (&e)[32], int lane)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int j = 0; j < o; ++j) {
            const float send = up ? e[j] : e[j + o];
            const float keep = up ? e[j + o] : e[j];
            e[j] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, o);
        }
    }
    return e[0];
}

// Cluster-tile vt of a launch: row pair p, first replica rb and replica count.
// The tiles of a side are (row pair, 256-replica block) pairs, T of them; when
// the last round of the persistent loop would keep at most half the clusters
// busy (L = T mod clusters tiles, 2L <= clusters, including the case of a
// single round), those L tiles are split into 2L tiles of 128 replicas (an
// N = 128 MMA chain each), so that the last round takes about half as long.
// Each half still loads its full J rows, so the split trades SM-time for
// latency: a lone run gains, a crowded batch loses; the run's tile_split flag
// (the autotuner's choice per shape, on by default) decides.
struct TcTile {
    int p, rb, ncols;
};

__host__ __device__ __forceinline__ void tc_tile_split(int T, int nclus, bool allow, int& nfull, int& nvirt)
{
    const int L = T % nclus;
    const bool split = allow && L > 0 && 2 * L <= nclus;
    nfull = split ? T - L : T;
    nvirt = split ? T + L : T;
}

__device__ __forceinline__ TcTile tc_tile(int vt, int nrp, int nfull)
{
    if (vt < nfull) return TcTile{vt % nrp, (vt / nrp) * TBN, TBN};
    const int h = vt - nfull, t = nfull + (h >> 1);
    return TcTile{t % nrp, (t / nrp) * TBN + (h & 1) * (TBN / 2), TBN / 2};
}

// Persistent kernel over CTA pairs (clusters of two).  Cluster c processes// Persistent kernel over CTA pairs (clusters of two).  Cluster c processes
// the cluster-tiles ct = c, c + nclusters, ...; cluster-tile ct is (row pair
// p = ct % nrp, replica block b = ct / nrp), a 256-row x 256-replica tile
// computed by one M=256, N=256 MMA chain over the pair: the CTA of rank k
// loads row tile 2p + k of J and replicas 128k..128k+127 of the block's spins
// into its own ring, both signalling the even CTA's "full" barrier; the even
// CTA issues the MMAs and its commits release the stage in both CTAs.  The
// FP32 accumulator is double-buffered in tensor memory (2 x 256 columns), so
// the epilogue of one tile (each CTA its 128 rows) overlaps the MMAs of the
// next; a buffer is reused once the epilogue warps of both CTAs released it.
//
// TABMODE (+-1 couplings) says where the decisions read the threshold window
// of the sweep's beta level (the row T[F - F_min] restricted to the indices
// [lo, lo + width) outside which T is saturated; a field outside the window is
// clamped to its edge, which holds the saturated value, so every decision
// compares against the same table value):
//   0  global memory (window too wide for shared memory);
//   1  the window, copied into shared memory once per launch;
//   2  the window copied 32 times (width <= 256) so that lane l reads copy l:
//      a conflict-free shared-memory load.
template <int KIND, int TABMODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    bq_tc_half_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
                      const __grid_constant__ CUtensorMap tmB, BqJob job, int side, int s_arg, const int32_t* sp,
                      int decide, float* fields_out, int* err)
{
    // Launched as a programmatic dependent of the sweep loop's previous kernel: wait
    // for it (its spins, partials and sweep counter) before reading anything it
    // writes, and let the next launch start its CTAs as this one's leave.  Without
    // such a dependency both instructions do nothing.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int s = sp ? *sp : s_arg;
    if (decide && s >= job.S) return;  // uniform over the grid: before any barrier or allocation
    TabWindow win{0, 0, 1};
    if (KIND == 0 && decide) {
        const int l = s / job.step;
        win = TabWindow{job.win[3 * l + 2], job.win[3 * l], job.win[3 * l + 1]};
    }
    using Cfg = TcCfg<KIND>;
    constexpr int S = Cfg::STAGES;
    constexpr int NA = KIND == 1 ? 2 : 1;  // J operands per stage
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint32_t* stab = reinterpret_cast<uint32_t*>(smem + S * Cfg::STAGE_BYTES);
    __shared__ __align__(8) uint64_t full_bar[S];
    __shared__ __align__(8) uint64_t empty_bar[S];
    __shared__ __align__(8) uint64_t accf_bar[2];
    __shared__ __align__(8) uint64_t acce_bar[2];
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = job.inst.n;
    const int nkb = (n + Cfg::KELEM - 1) / Cfg::KELEM;
    const int nrp = (((n + TBM - 1) / TBM) + 1) / 2;
    const int clus = blockIdx.x >> 1, nclus = gridDim.x >> 1;
    int nfull, nct;  // whole tiles, and all tiles of the launch (whole + halves of the last round)
    tc_tile_split(nrp * (job.Rpad / TBN), nclus, job.tile_split != 0, nfull, nct);
    const uint32_t crank = cluster_rank();

    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full_bar[q], 1);   // even CTA: its producer's arrive + both CTAs' bytes
            mbar_init(&empty_bar[q], 1);  // the pair's MMA commit
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&accf_bar[q], 1);
            mbar_init(&acce_bar[q], 2 * kEpiWarps);  // even CTA: epilogue warps of both CTAs
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * TBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    cluster_sync();  // both CTAs' barriers exist before any remote signal reaches them
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        // (stall_loads: failure-path tests, no loads, so the consumers' waits run out)
        if (lane == 0 && !job.stall_loads) {
            // stage index and phase advance incrementally; the even CTA's "full"
            // barriers are consecutive words, so their cluster addresses are too
            int st = 0;
            uint32_t ph = 0;
            const uint32_t fb0 = map_rank(&full_bar[0], 0);
            bool ok = true;
            for (int ct = clus; ct < nct && ok; ct += nclus) {
                // (a 128-replica tile still loads a 128-row box per CTA; its MMA reads the first 64)
                const TcTile tl = tc_tile(ct, nrp, nfull);
                const int i0 = (2 * tl.p + (int)crank) * TBM;
                const int r0 = tl.rb + (int)crank * (tl.ncols / 2);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&empty_bar[st], ph ^ 1u, job.wait_ns)) {
                        atomicOr(err, 1);
                        ok = false;
                        break;
                    }
                    unsigned char* sa = smem + st * Cfg::STAGE_BYTES;
                    const uint32_t fb = fb0 + (uint32_t)st * (uint32_t)sizeof(uint64_t);
                    if (crank == 0) mbar_expect_tx(&full_bar[st], (uint32_t)(2 * Cfg::STAGE_BYTES));
                    const int kc = kb * Cfg::KELEM;
                    tma_load_2d_pair(sa, &tmA, fb, kc, i0);
                    if (KIND == 1) tma_load_2d_pair(sa + Cfg::A_BYTES, &tmA2, fb, kc, i0);
                    tma_load_2d_pair(sa + NA * Cfg::A_BYTES, &tmB, fb, kc, r0);
                    if (++st == S) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (even CTA only) ----------------
        if (lane == 0 && crank == 0) {
            constexpr uint32_t idesc_full = instr_desc(KIND == 0 ? 0u : 1u, 2 * TBM, TBN);
            constexpr uint32_t idesc_half = instr_desc(KIND == 0 ? 0u : 1u, 2 * TBM, TBN / 2);
            // descriptor of the ring's first byte; a stage or K offset only adds to
            // the start-address field (shared addresses stay below 2^18, so the
            // 14-bit field of addr >> 4 never carries)
            const uint64_t desc0 = smem_desc(smem_u32(smem));
            int st = 0;
            uint32_t ph = 0, j = 0;
            bool ok = true;
            for (int ct = clus; ct < nct && ok; ct += nclus, ++j) {
                const uint32_t idesc = ct < nfull ? idesc_full : idesc_half;
                const uint32_t buf = j & 1u, aph = (j >> 1) & 1u;
                if (!mbar_wait(&acce_bar[buf], aph ^ 1u, job.wait_ns)) {
                    atomicOr(err, 8);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + buf * TBN;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&full_bar[st], ph, job.wait_ns)) {
                        atomicOr(err, 2);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t da = desc0 + (uint64_t)((st * Cfg::STAGE_BYTES) >> 4);
                    const uint64_t db = da + (uint64_t)((NA * Cfg::A_BYTES) >> 4);
#pragma unroll
                    for (int k = 0; k < KBYTES / Cfg::KSTEP_BYTES; ++k) {
                        const uint64_t bd = db + (uint64_t)((k * Cfg::KSTEP_BYTES) >> 4);
                        mma_issue<KIND>(d, da + (uint64_t)((k * Cfg::KSTEP_BYTES) >> 4), bd, idesc, (kb | k) ? 1u : 0u);
                        if (KIND == 1)
                            mma_issue<KIND>(d, da + (uint64_t)((Cfg::A_BYTES + k * Cfg::KSTEP_BYTES) >> 4), bd, idesc,
                                            1u);
                    }
                    mma_commit_pair(&empty_bar[st]);
                    if (++st == S) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) mma_commit_pair(&accf_bar[buf]);
            }
        }
    } else {
        // ---------------- epilogue: 16 warps, four per tensor-memory lane quarter ----------------
        const int quarter = warp & 3;
        const int slot = (warp - 2) >> 2;  // which quarter of the columns
        const int row = quarter * 32 + lane;
        const int et = threadIdx.x - 64;
        constexpr int ET = 32 * kEpiWarps;
        const bool pm1 = KIND == 0;
        const uint32_t acce_r0 = map_rank(&acce_bar[0], 0), acce_r1 = map_rank(&acce_bar[1], 0);
        float cexp = 0.0f;
        const uint32_t* trow = pm1 ? job.table + win.off : nullptr;
        const int wlo = win.lo, ww = win.width;
        if (TABMODE == 2) {
            for (int f = et; f < ww; f += ET) {
                const uint32_t v = __ldg(trow + f);
#pragma unroll 8
                for (int c = 0; c < 32; ++c) stab[f * 32 + ((c + f) & 31)] = v;
            }
        }
        if (TABMODE == 1) {
            for (int f0 = et; f0 < ww; f0 += ET * 4) {
                uint32_t v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int f = f0 + u * ET;
                    v[u] = f < ww ? __ldg(trow + f) : 0u;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int f = f0 + u * ET;
                    if (f < ww) stab[f] = v[u];
                }
            }
        }
        if (!pm1) cexp = f32_cexp(job.betaf[s / job.step]);
        // Energy partials of this side: side 1 contributes -b.F_B (F_B includes h_B),
        // side 0 only -h_A.a, which is zero without a field (its partials stay zero).
        const bool energy = !fields_out && (side == 1 || job.inst.has_h);
        asm volatile("bar.sync 1, %0;" ::"r"(ET) : "memory");
        uint32_t j = 0;
        bool ok = true;
        for (int ct = clus; ct < nct; ct += nclus, ++j) {
            const uint32_t buf = j & 1u, aph = (j >> 1) & 1u;
            const TcTile tl = tc_tile(ct, nrp, nfull);
            const bool half_tile = tl.ncols != TBN;  // 128 replicas: one 32-column chunk per epilogue warp
            const int rt = 2 * tl.p + (int)crank;
            const int i = rt * TBM + row;
            const int r0 = tl.rb;
            if (ok && !mbar_wait(&accf_bar[buf], aph, job.wait_ns)) {
                atomicOr(err, 4);
                ok = false;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const bool live = ok && i < n;
            const float hv = (i < n) ? (pm1 ? (job.inst.h8 ? (float)job.inst.h8[side * n + i] : 0.0f)
                                            : job.inst.hf[side * n + i])
                                     : 0.0f;
            // +-1 couplings: the accumulator is an exact integer below 2^22 in
            // magnitude, so v + (h + 1.5 * 2^23) is exact and its bit pattern is
            // 0x4B400000 + F: the integer field without a float-to-int conversion.
            const float hmag = hv + 12582912.0f;
            const int hi_ = (int)hv;
            const uint32_t taddr = tmem + buf * TBN + ((uint32_t)(quarter * 32) << 16);
            const PhiloxFixed pf = philox_fixed((uint32_t)i, (uint32_t)s, (kTagDecision << 24) | (uint32_t)side, job.key0,
                                                job.key1);
            for (int cc = 0; cc < kEpiCols / 32; ++cc) {
                const int c = half_tile ? slot : slot * (kEpiCols / 32) + cc;
                const bool last = cc == kEpiCols / 32 - 1;
                if ((half_tile && cc > 0) || r0 + c * 32 >= job.R) {
                    // 32 replicas of the tile's padding: nothing to decide, store or sum (their
                    // columns of the product depend only on their own spins, which stay as set);
                    // a 128-replica tile has only one chunk per warp
                    if (last) {
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive_cluster(buf ? acce_r1 : acce_r0);
                    }
                    continue;
                }
                float v[32];
                tmem_ld32(taddr + (uint32_t)(c * 32), v);
                if (last) {
                    // this warp has read its part of the accumulator: release the buffer
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive_cluster(buf ? acce_r1 : acce_r0);
                }
                float e[32];  // energy terms: FP32 (real couplings)
                int ei[32];   // energy terms: exact integers (+-1 couplings)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int rq = r0 + c * 32 + 4 * q;
                    float F[4];
                    int Fi[4];  // +-1 couplings: F as an integer
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        if (pm1) {
                            Fi[b] = __float_as_int(v[4 * q + b] + hmag) - 0x4B400000;
                            F[b] = (float)Fi[b];
                        } else {
                            F[b] = v[4 * q + b] + hv;
                        }
                    }
                    bool mn[4] = {false, false, false, false};
                    if (live) {
                        if (fields_out) {
#pragma unroll
                            for (int b = 0; b < 4; ++b)
                                if (rq + b < job.R) fields_out[(size_t)(rq + b) * 2 * n + side * n + i] = F[b];
                        } else if (decide) {
                            const U4 w = philox_c2((uint32_t)(rq >> 2), pf, job.key0, job.key1);
                            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                            for (int b = 0; b < 4; ++b) {
                                if (pm1) {
                                    const int f = min(max(Fi[b] - job.fmin - wlo, 0), ww - 1);
                                    uint32_t T;
                                    if (TABMODE == 2)
                                        T = stab[f * 32 + lane];
                                    else if (TABMODE == 1)
                                        T = stab[f];
                                    else
                                        T = __ldg(trow + f);
                                    mn[b] = ws[b] >= T;
                                } else {
                                    mn[b] = decide_f32(ws[b], F[b], cexp) != 0u;
                                }
                                const size_t off = (size_t)(rq + b) * job.ld + i;
                                if (pm1)
                                    static_cast<uint8_t*>(job.spins[side])[off] = mn[b] ? kE4m3Minus : kE4m3Plus;
                                else
                                    static_cast<uint16_t*>(job.spins[side])[off] = mn[b] ? kBf16Minus : kBf16Plus;
                            }
                        } else {
#pragma unroll
                            for (int b = 0; b < 4; ++b) {
                                const size_t off = (size_t)(rq + b) * job.ld + i;
                                mn[b] = pm1 ? (static_cast<const uint8_t*>(job.spins[side])[off] & 0x80u) != 0
                                            : (static_cast<const uint16_t*>(job.spins[side])[off] & 0x8000u) != 0;
                            }
                        }
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        // side 1: -m F (F includes h);  side 0: -h m
                        if (pm1) {
                            const int xi = (side == 1) ? Fi[b] : hi_;
                            ei[4 * q + b] = live ? (mn[b] ? xi : -xi) : 0;
                        } else {
                            const float x = (side == 1) ? F[b] : hv;
                            e[4 * q + b] = live ? (mn[b] ? x : -x) : 0.0f;
                        }
                    }
                }
                if (energy) {
                    // one partial row per 32-row quarter of the tile: no CTA barrier
                    const size_t off = ((size_t)side * job.nblk + 4 * rt + quarter) * job.Rpad + r0 + c * 32 + lane;
                    if (pm1) {
                        // column sums over the warp's 32 rows, one integer reduction per column
                        int mine = 0;
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            const int t = __reduce_add_sync(0xFFFFFFFFu, ei[k]);
                            if (lane == k) mine = t;
                        }
                        static_cast<int32_t*>(job.part)[off] = mine;
                    } else {
                        static_cast<float*>(job.part)[off] = warp_transpose_sum(e, lane);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    cluster_sync();  // no CTA leaves while its peer may still signal its barriers
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TBN));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder()
{
    // looked up once (a function-local static is initialised once, also when
    // several threads prepare runs at the same time)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        return nullptr;
    }();
    return fn;
}

}  // namespace

size_t bq_tc_smem_bytes(int kind);

namespace {

// How many two-CTA clusters of the kernel can be resident at once on this
// device (a GPC with an odd number of free SMs leaves one SM unused); cached
// per device and kind.
int tc_active_clusters(int kind)
{
    static int cache[64][2] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && cache[dev][kind] > 0) return cache[dev][kind];
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int n = 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * std::max(1, sms / 2));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = bq_tc_smem_bytes(kind);
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = 2;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    const cudaError_t e = kind == 0 ? cudaOccupancyMaxActiveClusters(&n, bq_tc_half_kernel<0, 2>, &cfg)
                                    : cudaOccupancyMaxActiveClusters(&n, bq_tc_half_kernel<1, 0>, &cfg);
    if (e != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        n = std::max(1, sms / 2);
    }
    if (dev >= 0 && dev < 64) cache[dev][kind] = n;
    return n;
}

}  // namespace

size_t bq_tc_smem_bytes(int kind)
{
    const size_t st = kind == 0 ? (size_t)TcCfg<0>::STAGES * TcCfg<0>::STAGE_BYTES + TcCfg<0>::TAB_BYTES
                                : (size_t)TcCfg<1>::STAGES * TcCfg<1>::STAGE_BYTES + TcCfg<1>::TAB_BYTES;
    return st + 1024;  // + alignment slack
}

// 2D row-major [rows][cols] matrix of elem_bytes elements (row stride ld_bytes),
// loaded as boxes of [box_rows][128 bytes] with the 128-byte swizzle.
cudaError_t bq_tc_make_map(CUtensorMap* map, const void* base, int elem_bytes, uint64_t cols, uint64_t rows,
                           uint64_t ld_bytes, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encoder();
    if (!enc) return cudaErrorNotSupported;
    const CUtensorMapDataType dt = elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t bq_tc_set_smem()
{
    cudaError_t e = cudaFuncSetAttribute(bq_tc_half_kernel<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bq_tc_smem_bytes(0));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(bq_tc_half_kernel<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bq_tc_smem_bytes(0));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(bq_tc_half_kernel<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bq_tc_smem_bytes(0));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(bq_tc_half_kernel<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bq_tc_smem_bytes(1));
    if (e != cudaSuccess) return e;
    tc_active_clusters(0);  // occupancy queries outside any stream capture
    tc_active_clusters(1);
    return cudaSuccess;
}

cudaError_t bq_launch_tc_half(const BqTcMaps& maps, int bsel, const BqJob& job, int side, int s, const int32_t* sp,
                              int decide, float* fields_out, int* err, cudaStream_t st)
{
    const int kind = job.inst.jtype == PB_J_PM1_I8 ? 0 : 1;
    const size_t smem = bq_tc_smem_bytes(kind);
    const int nrp = (((job.inst.n + TBM - 1) / TBM) + 1) / 2;
    const int active = tc_active_clusters(kind);
    int nfull = 0, nvirt = 0;  // the kernel makes the same split from the grid it gets
    tc_tile_split(nrp * (job.Rpad / TBN), active, job.tile_split != 0, nfull, nvirt);
    const int nclus = std::max(1, std::min(nvirt, active));
    dim3 grid((unsigned)(2 * nclus));  // persistent clusters of two CTAs
    const CUtensorMap& A = side == 0 ? maps.a[0] : maps.a[2];
    const CUtensorMap& A2 = side == 0 ? maps.a[1] : maps.a[3];
    const CUtensorMap& B = maps.b[bsel];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (job.pdl && sp) {  // inside the sweep loop: a programmatic dependent of the launch before it
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    if (kind == 0 && job.tabmode == 2)
        return cudaLaunchKernelEx(&cfg, bq_tc_half_kernel<0, 2>, A, A2, B, job, side, s, sp, decide, fields_out, err);
    if (kind == 0 && job.tabmode == 1)
        return cudaLaunchKernelEx(&cfg, bq_tc_half_kernel<0, 1>, A, A2, B, job, side, s, sp, decide, fields_out, err);
    if (kind == 0)
        return cudaLaunchKernelEx(&cfg, bq_tc_half_kernel<0, 0>, A, A2, B, job, side, s, sp, decide, fields_out, err);
    return cudaLaunchKernelEx(&cfg, bq_tc_half_kernel<1, 0>, A, A2, B, job, side, s, sp, decide, fields_out, err);
}

bool bq_tc_fills_device(int n, int Rpad, int kind)
{
    const int nrp = (((n + TBM - 1) / TBM) + 1) / 2;
    return nrp * (Rpad / TBN) >= tc_active_clusters(kind);
}

int bq_tc_clusters(int n, int Rpad, int kind, bool split)
{
    const int nrp = (((n + TBM - 1) / TBM) + 1) / 2;
    const int active = tc_active_clusters(kind);
    int nfull = 0, nvirt = 0;
    tc_tile_split(nrp * (Rpad / TBN), active, split, nfull, nvirt);
    return std::max(1, std::min(nvirt, active));
}

}  // namespace pb
