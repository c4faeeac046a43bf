// host_api.cpp -- C-ABI entry points and host runtime of the p-bit annealer
// (arXiv 2510.23419): instance store, seeded generators, colouring
// validation, annealing schedules, FP64 threshold tables, run management.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "pb_handles.h"

namespace pb {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

pb_status fail(pb_status st, const std::string& msg)
{
    g_last_error = msg;
    return st;
}

pb_status cuda_fail(cudaError_t e, const char* what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? PB_ENOMEM : PB_EDEVICE;
}

// ---------------------------------------------------------------------------
// Seeded couplings (tag-2 Philox stream).
// ---------------------------------------------------------------------------
static constexpr double kTwoPi = 6.283185307179586476925286766559;
static constexpr double kTwo32 = 4294967296.0;

static void gen_couplings(int dist, uint64_t seed, int64_t count, void* out)
{
    const uint32_t c3 = kTagInstance << 24;
    if (dist == PB_DIST_PM1) {
        int8_t* J = static_cast<int8_t*>(out);
        for (int64_t e4 = 0; e4 < count; e4 += 4) {
            const U4 r = philox10((uint32_t)(e4 >> 2), 0u, 0u, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
            const uint32_t w[4] = {r.x, r.y, r.z, r.w};
            for (int b = 0; b < 4 && e4 + b < count; ++b) J[e4 + b] = (w[b] < 0x80000000u) ? 1 : -1;
        }
    } else if (dist == PB_DIST_GAUSS) {
        float* J = static_cast<float*>(out);
        for (int64_t e = 0; e < count; ++e) {
            const U4 r = philox10((uint32_t)e, 1u, 0u, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
            const double u0 = ((double)r.x + 0.5) / kTwo32;
            const double u1 = ((double)r.y + 0.5) / kTwo32;
            J[e] = (float)(std::sqrt(-2.0 * std::log(u0)) * std::cos(kTwoPi * u1));
        }
    } else {
        float* J = static_cast<float*>(out);
        for (int64_t e4 = 0; e4 < count; e4 += 4) {
            const U4 r = philox10((uint32_t)(e4 >> 2), 2u, 0u, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
            const uint32_t w[4] = {r.x, r.y, r.z, r.w};
            for (int b = 0; b < 4 && e4 + b < count; ++b) J[e4 + b] = (float)(2.0 * (((double)w[b] + 0.5) / kTwo32) - 1.0);
        }
    }
}

// ---------------------------------------------------------------------------
// Schedules and thresholds.
// ---------------------------------------------------------------------------
pb_status schedule_levels(const pb_schedule* sc, std::vector<double>& betas, int& step)
{
    if (!sc) return fail(PB_EINVAL, "schedule is null");
    if (sc->n_sweeps < 0) return fail(PB_EINVAL, "n_sweeps < 0");
    const int S = sc->n_sweeps;
    if (sc->kind == PB_SCHED_EXPLICIT) {
        if (S > 0 && !sc->betas) return fail(PB_EINVAL, "explicit schedule without betas");
        betas.assign(sc->betas, sc->betas + S);
        step = 1;
    } else if (sc->kind == PB_SCHED_LINEAR || sc->kind == PB_SCHED_GEOMETRIC) {
        if (sc->step_duration < 1) return fail(PB_EINVAL, "step_duration < 1");
        step = sc->step_duration;
        const int Lv = (S + step - 1) / step;
        betas.resize(Lv);
        if (sc->kind == PB_SCHED_GEOMETRIC && Lv > 1 && !(sc->beta0 > 0.0 && sc->beta1 > 0.0))
            return fail(PB_EINVAL, "geometric schedule needs beta0, beta1 > 0");
        for (int l = 0; l < Lv; ++l) {
            const double frac = (Lv > 1) ? (double)l / (double)(Lv - 1) : 0.0;
            betas[l] = (sc->kind == PB_SCHED_LINEAR) ? sc->beta0 + (sc->beta1 - sc->beta0) * frac
                                                     : sc->beta0 * std::pow(sc->beta1 / sc->beta0, frac);
        }
    } else {
        return fail(PB_EINVAL, "unknown schedule kind");
    }
    for (double b : betas)
        if (!std::isfinite(b) || b < 0.0) return fail(PB_EINVAL, "betas must be finite and >= 0");
    return PB_OK;
}

// Threshold of Eq. 2: floor((0.5 + 0.5 tanh(beta F)) 2^32), saturated to 2^32 - 1 (FP64).
uint32_t threshold_u32(double beta, double F)
{
    const double P = 0.5 + 0.5 * std::tanh(beta * F);
    double T = std::floor(P * kTwo32);
    if (T > 4294967295.0) T = 4294967295.0;
    if (T < 0.0) T = 0.0;
    return (uint32_t)T;
}

// f(begin, end) over [0, n), split into contiguous ranges across host threads;
// one range (no thread) below 2 x `grain` items.
template <typename F>
static void parallel_ranges(int n, int grain, F&& f)
{
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nt = std::min(hw, std::max(1, n / std::max(1, grain)));
    if (nt <= 1) {
        f(0, n);
        return;
    }
    std::vector<std::thread> ts;
    ts.reserve((size_t)nt);
    for (int k = 0; k < nt; ++k) {
        const int b = (int)((long long)n * k / nt), e = (int)((long long)n * (k + 1) / nt);
        ts.emplace_back([&f, b, e] { f(b, e); });
    }
    for (std::thread& t : ts) t.join();
}

// Threshold rows (Eq. 2, FP64 on the host), one per beta level, stored as the
// window of the row outside which T is saturated: T is nondecreasing in F, so
// every entry below the window is 0 and every entry above it 2^32 - 1, and the
// window keeps one saturated entry on each side; a lookup clamps the index into
// the window.  The window edges are found by bisection, so a level costs
// O(width + log nF) evaluations instead of nF.  win gets (lo, width, off) per level.
void threshold_windows(const std::vector<double>& betas, int nF, int fmin, std::vector<uint32_t>& tab,
                       std::vector<int32_t>& win)
{
    const int nlev = std::max<int>(1, (int)betas.size());
    win.assign((size_t)nlev * 3, 0);
    // levels are independent: ranges of them on host threads, each into its own
    // segment, then the segments in level order (the same table as one pass)
    std::vector<std::vector<uint32_t>> seg((size_t)nlev);
    parallel_ranges(nlev, 512, [&](int l0, int l1) {
        for (int l = l0; l < l1; ++l) {
            const double beta = betas.empty() ? 0.0 : betas[(size_t)l];
            auto T = [&](int f) { return threshold_u32(beta, (double)(f + fmin)); };
            int a = 0, b = nF;  // first index with T > 0
            while (a < b) {
                const int m = (a + b) / 2;
                if (T(m) > 0u) b = m; else a = m + 1;
            }
            const int lo = std::max(0, a - 1);
            a = 0;
            b = nF;  // first index with T = 2^32 - 1
            while (a < b) {
                const int m = (a + b) / 2;
                if (T(m) == 0xFFFFFFFFu) b = m; else a = m + 1;
            }
            const int hi = std::max(lo, std::min(nF - 1, a));
            win[3 * (size_t)l] = lo;
            win[3 * (size_t)l + 1] = hi - lo + 1;
            std::vector<uint32_t>& v = seg[(size_t)l];
            v.resize((size_t)(hi - lo + 1));
            for (int f = lo; f <= hi; ++f) v[(size_t)(f - lo)] = T(f);
        }
    });
    size_t total = 0;
    for (int l = 0; l < nlev; ++l) {
        win[3 * (size_t)l + 2] = (int32_t)total;
        total += seg[(size_t)l].size();
    }
    tab.resize(total);
    for (int l = 0; l < nlev; ++l)
        std::copy(seg[(size_t)l].begin(), seg[(size_t)l].end(), tab.begin() + win[3 * (size_t)l + 2]);
}

}  // namespace pb

namespace pb {

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// EA instance -> kernel layouts.
static pb_status ea_build(pb_instance* I, const pb_instance_desc* d, cudaStream_t st)
{
    const int L = d->L;
    if (L < 2 || L > 64) return fail(PB_EINVAL, "EA side L must be in [2, 64]");
    if (L % 2) return fail(PB_ECOLOUR, "the checkerboard colouring of a periodic cube needs an even L");
    const int64_t N = (int64_t)L * L * L;
    const int64_t half = N / 2;
    I->L = L;
    I->N = N;
    I->maxdeg = 6;
    auto idx = [L](int x, int y, int z) { return (int64_t)x + (int64_t)L * (y + (int64_t)L * z); };
    // canonical colouring check
    if (d->colour) {
        bool canonical = true;
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    const int64_t i = idx(x, y, z);
                    const int ci = d->colour[i];
                    const int64_t nb[3] = {idx((x + 1) % L, y, z), idx(x, (y + 1) % L, z), idx(x, y, (z + 1) % L)};
                    for (int b = 0; b < 3; ++b)
                        if (d->colour[nb[b]] == ci)
                            return fail(PB_ECOLOUR, "colouring has an edge inside a colour class (site " +
                                                        std::to_string(i) + ")");
                    if (ci != ((x + y + z) & 1)) canonical = false;
                }
        if (!canonical) return fail(PB_EUNSUPPORTED, "only the canonical checkerboard colouring (colour 0 at the origin) is implemented");
    }
    // bond values by (class c, rank k, bond b in +x,-x,+y,-y,+z,-z)
    std::vector<uint8_t> jb;
    std::vector<int8_t> h8;
    std::vector<float> j6, hf;
    const bool pm1 = d->jtype == PB_J_PM1_I8;
    if (pm1) {
        const int8_t* J = static_cast<const int8_t*>(d->J);
        for (int64_t e = 0; e < 3 * N; ++e)
            if (J[e] != 1 && J[e] != -1) return fail(PB_EINVAL, "PM1 couplings must be +1 or -1 (bond " + std::to_string(e) + ")");
        jb.assign((size_t)N, 0);
        if (d->h) {
            const int8_t* h = static_cast<const int8_t*>(d->h);
            int hm = 0;
            for (int64_t i = 0; i < N; ++i) hm = std::max(hm, std::abs((int)h[i]));
            if (hm > 64) return fail(PB_EINVAL, "PM1 fields must satisfy |h| <= 64");
            I->has_h = 1;
            I->hmax = hm;
            h8.assign((size_t)N, 0);
        }
    } else {
        j6.assign((size_t)N * 8, 0.0f);
        hf.assign((size_t)N, 0.0f);
        I->has_h = d->h ? 1 : 0;
    }
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                const int64_t i = idx(x, y, z);
                const int c = (x + y + z) & 1;
                const int64_t slot = c * half + (i >> 1);
                const int64_t bonds[6] = {0 * N + i, 0 * N + idx((x + L - 1) % L, y, z),
                                          1 * N + i, 1 * N + idx(x, (y + L - 1) % L, z),
                                          2 * N + i, 2 * N + idx(x, y, (z + L - 1) % L)};
                if (pm1) {
                    const int8_t* J = static_cast<const int8_t*>(d->J);
                    uint8_t bits = 0;
                    for (int b = 0; b < 6; ++b)
                        if (J[bonds[b]] < 0) bits |= (uint8_t)(1u << (2 + b));
                    jb[slot] = bits;
                    if (d->h) h8[slot] = static_cast<const int8_t*>(d->h)[i];
                } else {
                    const float* J = static_cast<const float*>(d->J);
                    for (int b = 0; b < 6; ++b) {
                        if (!std::isfinite(J[bonds[b]])) return fail(PB_EINVAL, "F32 couplings must be finite");
                        j6[slot * 8 + b] = J[bonds[b]];
                    }
                    if (d->h) {
                        hf[slot] = static_cast<const float*>(d->h)[i];
                        j6[slot * 8 + 6] = hf[slot];  // the field also rides in the site's second vector
                    }
                }
            }
    const size_t esz = pm1 ? 1 : 4;
    PB_ALLOC(I->J3, 3 * N * esz);
    PB_CUDA_TRY(cudaMemcpyAsync(I->J3.p, d->J, 3 * N * esz, cudaMemcpyHostToDevice, st));
    if (d->h) {
        PB_ALLOC(I->hraw, N * esz);
        PB_CUDA_TRY(cudaMemcpyAsync(I->hraw.p, d->h, N * esz, cudaMemcpyHostToDevice, st));
    }
    if (pm1) {
        PB_ALLOC(I->jbits, N);
        PB_CUDA_TRY(cudaMemcpyAsync(I->jbits.p, jb.data(), N, cudaMemcpyHostToDevice, st));
        if (d->h) {
            PB_ALLOC(I->h8, N);
            PB_CUDA_TRY(cudaMemcpyAsync(I->h8.p, h8.data(), N, cudaMemcpyHostToDevice, st));
        }
    } else {
        PB_ALLOC(I->j6, N * 8 * 4);
        PB_CUDA_TRY(cudaMemcpyAsync(I->j6.p, j6.data(), N * 32, cudaMemcpyHostToDevice, st));
        PB_ALLOC(I->hf, N * 4);
        PB_CUDA_TRY(cudaMemcpyAsync(I->hf.p, hf.data(), N * 4, cudaMemcpyHostToDevice, st));
    }
    // pageable sources: make sure the copies are done before the host vectors go
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    EaDevice& e = I->ea;
    e.L = L;
    e.N = (int32_t)N;
    e.half = (int32_t)half;
    e.jtype = d->jtype;
    e.has_h = I->has_h;
    e.hmax = I->hmax;
    e.jbits = I->jbits.as<uint8_t>();
    e.h8 = I->h8.as<int8_t>();
    e.j6 = I->j6.as<float>();
    e.hf = I->hf.as<float>();
    e.J3 = I->J3.p;
    e.hraw = I->hraw.p;
    return PB_OK;
}

// ---------------------------------------------------------------------------
// EA runs
// ---------------------------------------------------------------------------
pb_status ea_prepare_run(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                                const pb_anneal_opts* opts, int form, int WT, cudaStream_t st)
{
    std::vector<double> betas;
    int step = 1;
    pb_status ps = schedule_levels(sc, betas, step);
    if (ps != PB_OK) return ps;
    run->inst = I;
    run->form = form;
    run->R = R;
    run->S = sc->n_sweeps;
    run->N = I->N;
    run->stream = st;
    EaJob& j = run->job;
    j = EaJob{};
    j.inst = I->ea;
    j.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
    j.key1 = (uint32_t)(seed >> 32);
    j.S = sc->n_sweeps;
    j.step = step;
    j.R = R;
    const int Rw = (R + 3) / 4;
    if (form == PB_FORM_PLAIN) {
        j.WT = Rw;
        j.n_tiles = 1;
    } else {
        j.WT = WT;
        j.n_tiles = (Rw + WT - 1) / WT;
    }
    const int Rpad = j.n_tiles * 4 * j.WT;
    const size_t words = (size_t)j.n_tiles * I->N * j.WT;
    const int nlev = std::max<int>(1, (int)betas.size());
    if (I->jtype == PB_J_PM1_I8) {
        const int fmax = 6 + I->hmax;
        j.fmin = -fmax;
        j.nF = 2 * fmax + 1;
        std::vector<uint32_t> tab((size_t)nlev * j.nF, 0x80000000u);
        parallel_ranges((int)betas.size(), 2048, [&](int l0, int l1) {
            for (int l = l0; l < l1; ++l)
                for (int f = 0; f < j.nF; ++f)
                    tab[(size_t)l * j.nF + f] = threshold_u32(betas[(size_t)l], (double)(f + j.fmin));
        });
        PB_ALLOC(run->table, tab.size() * 4);
        PB_CUDA_TRY(cudaMemcpyAsync(run->table.p, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaStreamSynchronize(st));
        j.table = run->table.as<uint32_t>();
        PB_ALLOC(run->E_best_i, (size_t)Rpad * 4);
        j.E_best_i = run->E_best_i.as<int32_t>();
    } else {
        std::vector<float> bf(nlev, 0.0f);
        for (size_t l = 0; l < betas.size(); ++l) bf[l] = (float)betas[l];
        PB_ALLOC(run->betaf, bf.size() * 4);
        PB_CUDA_TRY(cudaMemcpyAsync(run->betaf.p, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaStreamSynchronize(st));
        j.betaf = run->betaf.as<float>();
        PB_ALLOC(run->E_best_f, (size_t)Rpad * 4);
        j.E_best_f = run->E_best_f.as<float>();
    }
    j.has_target = 0;
    if (opts && !std::isnan(opts->target_energy)) {
        j.has_target = (opts->flags & PB_FLAG_STOP_AT_TARGET) ? 2 : 1;
        const double tg = opts->target_energy;
        j.target_i = (int32_t)std::max(-2.0e9, std::min(2.0e9, std::floor(tg)));
        j.target_f = (float)tg;
    }
    PB_ALLOC(run->best_words, words * 4);
    PB_ALLOC(run->final_words, words * 4);
    PB_ALLOC(run->best_sweep, (size_t)Rpad * 4);
    PB_ALLOC(run->hit_sweep, (size_t)Rpad * 4);
    j.best_words = run->best_words.as<uint32_t>();
    j.final_words = run->final_words.as<uint32_t>();
    j.best_sweep = run->best_sweep.as<int32_t>();
    j.hit_sweep = run->hit_sweep.as<int32_t>();
    j.n_hit = nullptr;
    if (j.has_target == 2 && form == PB_FORM_PLAIN) {
        PB_ALLOC(run->n_hit, 16);
        PB_CUDA_TRY(cudaMemsetAsync(run->n_hit.p, 0, 16, st));
        j.n_hit = run->n_hit.as<int32_t>();
    }
    PB_ALLOC(run->best_pm, (size_t)R * I->N);
    PB_ALLOC(run->final_pm, (size_t)R * I->N);
    PB_ALLOC(run->E_out, (size_t)2 * R * 8);
    PB_CUDA_TRY(cudaEventCreate(&run->ev_start));
    PB_CUDA_TRY(cudaEventCreate(&run->ev_stop));
    return PB_OK;
}

static pb_status ea_enqueue_readout(pb_run* run, cudaStream_t st)
{
    PB_CUDA_TRY(ea_launch_readout(run->job, run->job.final_words, run->final_pm.as<int8_t>(), run->E_out.as<double>(), st));
    PB_CUDA_TRY(ea_launch_readout(run->job, run->job.best_words, run->best_pm.as<int8_t>(), run->E_out.as<double>() + run->R, st));
    return PB_OK;
}

pb_status ea_enqueue_plain(pb_run* run, cudaStream_t st)
{
    const EaJob& j = run->job;
    PB_CUDA_TRY(cudaEventCreate(&run->ev_k0));
    PB_CUDA_TRY(cudaEventCreate(&run->ev_k1));
    PB_CUDA_TRY(cudaEventRecord(run->ev_start, st));
    PB_CUDA_TRY(cudaEventRecord(run->ev_k0, st));
    PB_CUDA_TRY(ea_launch_plain_init(j, st));
    PB_CUDA_TRY(ea_launch_plain_energy(j, -1, true, st));
    for (int s = 0; s < j.S; ++s) {
        PB_CUDA_TRY(ea_launch_plain_sweep(j, s, st));
        PB_CUDA_TRY(ea_launch_plain_energy(j, s, false, st));
    }
    PB_CUDA_TRY(cudaEventRecord(run->ev_k1, st));
    pb_status ps = ea_enqueue_readout(run, st);
    if (ps != PB_OK) return ps;
    PB_CUDA_TRY(cudaEventRecord(run->ev_stop, st));
    return PB_OK;
}

struct TileCost {
    int job, tile;
    double cost;
};

// One persistent kernel per coupling type present, tiles ordered longest
// first inside each; the kernels run as a chain of programmatic dependent
// launches (the group holding the longest tile first), so the second one's
// CTAs take the SMs the first one leaves.  Set-up (device arrays of jobs and
// work items) and launch are separate so that a batch can prepare all of its
// jobs before any of them starts.
pb_status ea_batch_setup(std::vector<pb_run*>& runs, cudaStream_t st, std::shared_ptr<BatchShared>& out)
{
    auto shared = std::make_shared<BatchShared>();
    PB_CUDA_TRY(cudaEventCreate(&shared->ev_k0));
    PB_CUDA_TRY(cudaEventCreate(&shared->ev_k1));
    std::vector<EaJob> jobs;
    std::vector<TileCost> tiles[2];
    EaGroup grp[2];
    // FP32 kernel: the one with the L = 24 tile if the batch has L = 24 FP32 tiles and no L = 32 ones
    bool f32_l24 = false, f32_l32 = false;
    for (const pb_run* r : runs) {
        if (r->job.inst.jtype != PB_J_F32) continue;
        f32_l24 |= ea_tile_path(r->job) == kEaPathFast24;
        f32_l32 |= ea_tile_path(r->job) == kEaPathFast32;
    }
    grp[0].kernel = kEaKernelPm1;
    grp[1].kernel = f32_l24 && !f32_l32 ? kEaKernelF32L24 : kEaKernelF32;
    for (size_t q = 0; q < runs.size(); ++q) {
        const EaJob& j = runs[q]->job;
        jobs.push_back(j);
        const int t = j.inst.jtype == PB_J_F32 ? 1 : 0;
        grp[t].smem = std::max(grp[t].smem, ea_resident_smem(j.inst.L, j.WT, j.inst.jtype, j.inst.has_h, j.nF));
        const double per = (double)j.inst.N * 4.0 * j.WT * std::max(1, j.S) * (t ? 1.8 : 1.0);
        for (int k = 0; k < j.n_tiles; ++k) tiles[t].push_back({(int)q, k, per});
        grp[t].cost += per * j.n_tiles;
        grp[t].longest = std::max(grp[t].longest, per);
    }
    std::vector<int> order;
    for (int t = 0; t < 2; ++t)
        if (!tiles[t].empty()) order.push_back(t);
    if (order.size() == 2 && grp[1].longest > grp[0].longest) std::swap(order[0], order[1]);
    std::vector<EaWork> work;
    const int sms = sm_count();
    for (int t : order) {
        std::stable_sort(tiles[t].begin(), tiles[t].end(),
                         [](const TileCost& a, const TileCost& b) { return a.cost > b.cost; });
        grp[t].offset = (int)work.size();
        grp[t].n = (int)tiles[t].size();
        grp[t].grid = std::max(1, std::min(grp[t].n, sms));
        for (const TileCost& c : tiles[t]) work.push_back(EaWork{c.job, c.tile, ea_tile_path(jobs[(size_t)c.job])});
        shared->groups.push_back(grp[t]);
        cudaEvent_t e = nullptr;
        PB_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        shared->ev_group.push_back(e);
    }
    PB_ALLOC(shared->jobs, jobs.size() * sizeof(EaJob));
    PB_ALLOC(shared->work, work.size() * sizeof(EaWork));
    PB_ALLOC(shared->counter, 16);
    PB_CUDA_TRY(cudaMemcpyAsync(shared->jobs.p, jobs.data(), jobs.size() * sizeof(EaJob), cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(shared->work.p, work.data(), work.size() * sizeof(EaWork), cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    shared->n_work = (int)work.size();
    for (const EaGroup& g : shared->groups) PB_CUDA_TRY(ea_resident_set_smem(g.kernel, g.smem));
    out = shared;
    return PB_OK;
}

void ea_batch_limit_sms(BatchShared& shared, int sms)
{
    double total = 0.0;
    for (const EaGroup& g : shared.groups) total += g.cost;
    const int ng = (int)shared.groups.size();
    int left = std::max(ng, sms);
    for (int k = 0; k < ng; ++k) {
        EaGroup& g = shared.groups[(size_t)k];
        const int later = ng - k - 1;  // at least one SM for each later group
        const int share = later == 0 ? left
                                     : std::max(1, std::min(left - later, (int)std::lround(sms * g.cost /
                                                                                             std::max(total, 1e-30))));
        g.grid = std::max(1, std::min(g.grid, share));
        left -= g.grid;
    }
}

pb_status ea_batch_launch(std::vector<pb_run*>& runs, const std::shared_ptr<BatchShared>& shared, cudaStream_t st)
{
    // The launch sequence (counter reset, persistent kernels, readouts) is
    // captured into a CUDA graph when the stream allows capture.  Inside the
    // capture the kernels after the first are programmatic dependents of the
    // one before, and the readouts wait for every kernel; without a capture
    // the kernels simply run one after the other.
    const bool capture = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    cudaGraph_t graph = nullptr;
    for (pb_run* r : runs) PB_CUDA_TRY(cudaEventRecord(r->ev_start, st));  // every run spans the shared launch
    if (capture) PB_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    auto body = [&]() -> pb_status {
        PB_CUDA_TRY(cudaMemsetAsync(shared->counter.p, 0, 16, st));
        // inside a capture an event becomes a graph node only when recorded as external
        const unsigned evf = capture ? cudaEventRecordExternal : cudaEventRecordDefault;
        PB_CUDA_TRY(cudaEventRecordWithFlags(shared->ev_k0, st, evf));
        for (size_t k = 0; k < shared->groups.size(); ++k) {
            const EaGroup& g = shared->groups[k];
            PB_CUDA_TRY(ea_launch_resident(g.kernel, shared->jobs.as<EaJob>(), shared->work.as<EaWork>() + g.offset, g.n,
                                           shared->counter.as<int>() + k, g.smem, g.grid, capture && k > 0, st));
            if (capture) PB_CUDA_TRY(cudaEventRecord(shared->ev_group[k], st));
        }
        if (capture)
            for (size_t k = 0; k + 1 < shared->groups.size(); ++k)
                PB_CUDA_TRY(cudaStreamWaitEvent(st, shared->ev_group[k], 0));
        PB_CUDA_TRY(cudaEventRecordWithFlags(shared->ev_k1, st, evf));
        for (pb_run* r : runs) {
            pb_status ps = ea_enqueue_readout(r, st);
            if (ps != PB_OK) return ps;
        }
        return PB_OK;
    };
    pb_status ps = body();
    if (capture) {
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (ps != PB_OK) {
            if (graph) cudaGraphDestroy(graph);
            return ps;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&shared->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        PB_CUDA_TRY(cudaGraphLaunch(shared->exec, st));
    } else if (ps != PB_OK) {
        return ps;
    }
    for (pb_run* r : runs) PB_CUDA_TRY(cudaEventRecord(r->ev_stop, st));
    for (pb_run* r : runs) r->batch = shared;
    return PB_OK;
}

static pb_status ea_enqueue_resident(std::vector<pb_run*>& runs, cudaStream_t st)
{
    std::shared_ptr<BatchShared> shared;
    pb_status ps = ea_batch_setup(runs, st, shared);
    if (ps != PB_OK) return ps;
    return ea_batch_launch(runs, shared, st);
}

int ea_choose_wt(const pb_instance* I, int R, int nF)
{
    return ea_resident_pick_wt(I->L, I->jtype, I->has_h, nF, (R + 3) / 4);
}

pb_status wait_run(pb_run* run, int32_t timeout_ms)
{
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(run->ev_stop);
        if (e == cudaSuccess) {
            if (run->dev_err) {
                int code = 0;
                PB_CUDA_TRY(cudaMemcpy(&code, run->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
                if (code) return fail(PB_ETIMEOUT, "a device-side wait of the run timed out (code " + std::to_string(code) + ")");
            }
            return PB_OK;
        }
        if (e != cudaErrorNotReady) return cuda_fail(e, "run failed");
        if (timeout_ms >= 0) {
            const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
            if (el.count() >= timeout_ms) return fail(PB_ETIMEOUT, "run not finished within the timeout");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace pb

using namespace pb;

extern "C" {

const char* pb_version(void) { return "pbit-gb300 0.1 (sm_103a)"; }

const char* pb_status_string(pb_status s)
{
    switch (s) {
        case PB_OK: return "PB_OK";
        case PB_EINVAL: return "PB_EINVAL";
        case PB_ECOLOUR: return "PB_ECOLOUR";
        case PB_ENOMEM: return "PB_ENOMEM";
        case PB_EDEVICE: return "PB_EDEVICE";
        case PB_ETIMEOUT: return "PB_ETIMEOUT";
        case PB_EBUSY: return "PB_EBUSY";
        case PB_EUNSUPPORTED: return "PB_EUNSUPPORTED";
    }
    return "unknown status";
}

const char* pb_last_error(void) { return g_last_error.c_str(); }

pb_status pb_generate_ea(int32_t L, int32_t dist, uint64_t seed, void* J_out, int64_t out_bytes)
{
    if (L < 1 || L > 1024) return fail(PB_EINVAL, "L out of range");
    if (dist < 0 || dist > 2) return fail(PB_EINVAL, "unknown coupling law");
    if (!J_out) return fail(PB_EINVAL, "J_out is null");
    const int64_t count = 3LL * L * L * L;
    if (out_bytes < count * (dist == PB_DIST_PM1 ? 1 : 4)) return fail(PB_EINVAL, "J_out too small");
    gen_couplings(dist, seed, count, J_out);
    return PB_OK;
}

pb_status pb_generate_biclique(int32_t n, int32_t dist, uint64_t seed, void* J_out, int64_t out_bytes)
{
    if (n < 1 || n > 65536) return fail(PB_EINVAL, "n out of range");
    if (dist < 0 || dist > 2) return fail(PB_EINVAL, "unknown coupling law");
    if (!J_out) return fail(PB_EINVAL, "J_out is null");
    const int64_t count = (int64_t)n * n;
    if (out_bytes < count * (dist == PB_DIST_PM1 ? 1 : 4)) return fail(PB_EINVAL, "J_out too small");
    gen_couplings(dist, seed, count, J_out);
    return PB_OK;
}

pb_status pb_create_instance(const pb_instance_desc* d, void* stream, pb_instance** out)
{
    pb::TraceRange trace_("pb_create_instance");
    if (!d || !out) return fail(PB_EINVAL, "null argument");
    *out = nullptr;
    if (!d->J) return fail(PB_EINVAL, "J is null");
    if (d->jtype != PB_J_PM1_I8 && d->jtype != PB_J_F32) return fail(PB_EINVAL, "unknown jtype");
    std::unique_ptr<pb_instance> I(new (std::nothrow) pb_instance());
    if (!I) return fail(PB_ENOMEM, "host allocation failed");
    I->topo = d->topo;
    I->jtype = d->jtype;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pb_status ps;
    if (d->topo == PB_TOPO_EA3D)
        ps = ea_build(I.get(), d, st);
    else if (d->topo == PB_TOPO_BICLIQUE)
        ps = bq_build(I.get(), d, st);
    else
        return fail(PB_EINVAL, "unknown topology");
    if (ps != PB_OK) return ps;
    *out = I.release();
    return PB_OK;
}

void pb_instance_destroy(pb_instance* inst) { delete inst; }

int64_t pb_instance_spins(const pb_instance* inst) { return inst ? inst->N : -1; }

pb_status pb_anneal_ex(pb_instance* I, const pb_schedule* sc, int32_t R, uint64_t seed, const pb_anneal_opts* opts,
                       void* stream, pb_run** out)
{
    pb::TraceRange trace_("pb_anneal");
    if (!I || !sc || !out) return fail(PB_EINVAL, "null argument");
    *out = nullptr;
    if (R < 1) return fail(PB_EINVAL, "replicas must be >= 1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int form = opts ? opts->form : PB_FORM_AUTO;
    std::unique_ptr<pb_run> run(new (std::nothrow) pb_run());
    if (!run) return fail(PB_ENOMEM, "host allocation failed");
    if (I->topo == PB_TOPO_EA3D) {
        int f = 0, WT = 0;
        choose_form(I, R, form, f, WT);
        if (f == PB_FORM_RESIDENT) {
            if (WT == 0) return fail(PB_EUNSUPPORTED, "lattice too large for the resident form");
            // enough tiles for the SMs: split replica blocks of a lone job
            const int sms = sm_count();
            while (WT > 1 && ((R + 3) / 4 + WT - 1) / WT < sms) WT /= 2;
        }
        if (f != PB_FORM_PLAIN && f != PB_FORM_RESIDENT) return fail(PB_EUNSUPPORTED, "form not available for EA instances");
        pb_status ps = ea_prepare_run(run.get(), I, sc, R, seed, opts, f, WT, st);
        if (ps != PB_OK) return ps;
        if (f == PB_FORM_PLAIN) {
            ps = ea_enqueue_plain(run.get(), st);
        } else {
            std::vector<pb_run*> v{run.get()};
            ps = ea_enqueue_resident(v, st);
        }
        if (ps != PB_OK) return ps;
    } else if (I->topo == PB_TOPO_CSR) {
        pb_status ps = csr_setup(run.get(), I, sc, R, seed, opts, st);
        if (ps == PB_OK) ps = csr_launch(run.get(), st);
        if (ps != PB_OK) return ps;
    } else {
        int f = 0, wt = 0;
        choose_form(I, R, form, f, wt);
        pb_anneal_opts o = opts ? *opts : pb_anneal_opts{PB_FORM_AUTO, 0, NAN};
        o.form = f;
        pb_status ps = bq_anneal(run.get(), I, sc, R, seed, &o, st, wt);
        if (ps != PB_OK) return ps;
    }
    *out = run.release();
    return PB_OK;
}

pb_status pb_anneal(pb_instance* inst, const pb_schedule* sched, int32_t replicas, uint64_t seed, void* stream,
                    pb_run** out)
{
    return pb_anneal_ex(inst, sched, replicas, seed, nullptr, stream, out);
}

// EA part of pb_anneal_resume: the resident form, with the given state and
// running best written into the run's tile-layout buffers before the launch.
static pb_status ea_anneal_resume(pb_instance* I, const pb_schedule* sc, int32_t R, uint64_t seed, int32_t s0,
                                  const int8_t* state, const int8_t* best_state, const double* best_E,
                                  const int32_t* best_sweep, cudaStream_t st, pb_run** out)
{
    int f = 0, WT = 0;
    choose_form(I, R, PB_FORM_RESIDENT, f, WT);
    if (f != PB_FORM_RESIDENT || WT == 0) return fail(PB_EUNSUPPORTED, "lattice too large for the resident form");
    const int sms = sm_count();
    while (WT > 1 && ((R + 3) / 4 + WT - 1) / WT < sms) WT /= 2;
    std::unique_ptr<pb_run> run(new (std::nothrow) pb_run());
    if (!run) return fail(PB_ENOMEM, "host allocation failed");
    pb_status ps = ea_prepare_run(run.get(), I, sc, R, seed, nullptr, PB_FORM_RESIDENT, WT, st);
    if (ps != PB_OK) return ps;
    EaJob& j = run->job;
    const bool pm1 = I->jtype == PB_J_PM1_I8;
    const int64_t N = I->N, half = N / 2, L = I->L, Rpad = (int64_t)j.n_tiles * 4 * j.WT;
    // [R][N] +-1 -> tile layout: word ((tile * 2 + c) * half + k) * WT + w, byte b of replica
    // r = (tile * WT + w) * 4 + b; +-1: bit 8b set <=> m = -1; FP32: byte 0x3F / 0xBF; padding replicas +1
    const uint32_t fill = pm1 ? 0u : 0x3F3F3F3Fu;
    std::vector<uint32_t> w((size_t)(Rpad / 4 * N), fill), wb((size_t)(Rpad / 4 * N), fill);
    for (int64_t r = 0; r < R; ++r) {
        const int64_t tile = r / (4 * j.WT), ww = (r / 4) % j.WT, b = r & 3;
        const uint32_t bit = pm1 ? (1u << (8 * b)) : (0x80u << (8 * b));
        for (int64_t i = 0; i < N; ++i) {
            const int8_t m = state[r * N + i], mb = best_state[r * N + i];
            if ((m != 1 && m != -1) || (mb != 1 && mb != -1)) return fail(PB_EINVAL, "states must hold +1 or -1");
            const int64_t x = i % L, y = (i / L) % L, z = i / (L * L);
            const int64_t c = (x + y + z) & 1, k = i >> 1;
            const size_t idx = (size_t)(((tile * 2 + c) * half + k) * j.WT + ww);
            if (m < 0) w[idx] |= bit;
            if (mb < 0) wb[idx] |= bit;
        }
    }
    std::vector<int32_t> bs((size_t)Rpad, -1), ei((size_t)Rpad, INT32_MAX);
    std::vector<float> ef((size_t)Rpad, 3.0e38f);  // padding replicas: any state improves on it
    for (int64_t r = 0; r < R; ++r) {
        bs[(size_t)r] = best_sweep[r];
        if (pm1) {
            if (best_E[r] != std::floor(best_E[r]) || std::fabs(best_E[r]) > 2.0e9)
                return fail(PB_EINVAL, "best energies of +-1 instances are integers");
            ei[(size_t)r] = (int32_t)best_E[r];
        } else {
            ef[(size_t)r] = (float)best_E[r];
        }
    }
    PB_CUDA_TRY(cudaMemcpyAsync(j.final_words, w.data(), w.size() * 4, cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(j.best_words, wb.data(), wb.size() * 4, cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(j.best_sweep, bs.data(), bs.size() * 4, cudaMemcpyHostToDevice, st));
    if (pm1)
        PB_CUDA_TRY(cudaMemcpyAsync(j.E_best_i, ei.data(), ei.size() * 4, cudaMemcpyHostToDevice, st));
    else
        PB_CUDA_TRY(cudaMemcpyAsync(j.E_best_f, ef.data(), ef.size() * 4, cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaStreamSynchronize(st));  // staging arrays go out of scope; the anneal stays asynchronous
    j.s0 = s0;
    j.resume = 1;
    std::vector<pb_run*> v{run.get()};
    ps = ea_enqueue_resident(v, st);
    if (ps != PB_OK) return ps;
    *out = run.release();
    return PB_OK;
}

pb_status pb_anneal_resume(pb_instance* I, const pb_schedule* sched, int32_t replicas, uint64_t seed,
                           int32_t first_sweep, const int8_t* state, const int8_t* best_state, const double* best_E,
                           const int32_t* best_sweep, void* stream, pb_run** out)
{
    pb::TraceRange trace_("pb_anneal_resume");
    if (!I || !sched || !state || !best_state || !best_E || !best_sweep || !out) return fail(PB_EINVAL, "null argument");
    *out = nullptr;
    if (replicas < 1) return fail(PB_EINVAL, "replicas must be >= 1");
    if (first_sweep < 0 || first_sweep > sched->n_sweeps) return fail(PB_EINVAL, "first_sweep must be in [0, n_sweeps]");
    for (int64_t r = 0; r < replicas; ++r)
        if (best_sweep[r] < -1 || best_sweep[r] >= first_sweep)
            return fail(PB_EINVAL, "best_sweep must be in [-1, first_sweep)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (I->topo == PB_TOPO_CSR)
        return csr_anneal_resume(I, sched, replicas, seed, first_sweep, state, best_state, best_E, best_sweep, st, out);
    if (I->topo == PB_TOPO_EA3D)
        return ea_anneal_resume(I, sched, replicas, seed, first_sweep, state, best_state, best_E, best_sweep, st, out);
    return fail(PB_EUNSUPPORTED,
                "resume runs on EA cubes (resident form) and general sparse instances (a biclique via its edge list)");
}

pb_status pb_wait(pb_run* run, int32_t timeout_ms)
{
    if (!run) return fail(PB_EINVAL, "null run");
    return wait_run(run, timeout_ms);
}

pb_status pb_query(pb_run* run)
{
    if (!run) return fail(PB_EINVAL, "null run");
    cudaError_t e = cudaEventQuery(run->ev_stop);
    if (e == cudaSuccess) return PB_OK;
    if (e == cudaErrorNotReady) return PB_EBUSY;
    return cuda_fail(e, "run failed");
}

pb_status pb_energy(pb_run* run, double* final_E, double* best_E, int32_t* best_sweep)
{
    pb::TraceRange trace_("pb_energy");
    if (!run) return fail(PB_EINVAL, "null run");
    pb_status ps = wait_run(run, -1);
    if (ps != PB_OK) return ps;
    const size_t R = (size_t)run->R;
    if (final_E) PB_CUDA_TRY(cudaMemcpy(final_E, run->E_out.p, R * 8, cudaMemcpyDeviceToHost));
    if (best_E) PB_CUDA_TRY(cudaMemcpy(best_E, run->E_out.as<double>() + R, R * 8, cudaMemcpyDeviceToHost));
    if (best_sweep) PB_CUDA_TRY(cudaMemcpy(best_sweep, run->best_sweep.p, R * 4, cudaMemcpyDeviceToHost));
    return PB_OK;
}

static pb_status copy_states(pb_run* run, const DevBuf& src, int8_t* out, int64_t out_bytes)
{
    if (!run || !out) return fail(PB_EINVAL, "null argument");
    const int64_t need = (int64_t)run->R * run->N;
    if (out_bytes < need) return fail(PB_EINVAL, "output buffer too small");
    pb_status ps = wait_run(run, -1);
    if (ps != PB_OK) return ps;
    PB_CUDA_TRY(cudaMemcpy(out, src.p, (size_t)need, cudaMemcpyDeviceToHost));
    return PB_OK;
}

pb_status pb_best_states(pb_run* run, int8_t* out, int64_t out_bytes)
{
    pb::TraceRange trace_("pb_best_states");
    if (!run) return fail(PB_EINVAL, "null run");
    return copy_states(run, run->best_pm, out, out_bytes);
}

pb_status pb_final_states(pb_run* run, int8_t* out, int64_t out_bytes)
{
    pb::TraceRange trace_("pb_final_states");
    if (!run) return fail(PB_EINVAL, "null run");
    return copy_states(run, run->final_pm, out, out_bytes);
}

pb_status pb_target_sweeps(pb_run* run, int32_t* first_sweep)
{
    if (!run || !first_sweep) return fail(PB_EINVAL, "null argument");
    pb_status ps = wait_run(run, -1);
    if (ps != PB_OK) return ps;
    PB_CUDA_TRY(cudaMemcpy(first_sweep, run->hit_sweep.p, (size_t)run->R * 4, cudaMemcpyDeviceToHost));
    return PB_OK;
}

pb_status pb_run_device_ms(pb_run* run, float* ms)
{
    if (!run || !ms) return fail(PB_EINVAL, "null argument");
    pb_status ps = wait_run(run, -1);
    if (ps != PB_OK) return ps;
    PB_CUDA_TRY(cudaEventElapsedTime(ms, run->ev_start, run->ev_stop));
    return PB_OK;
}

pb_status pb_philox_ceiling(int32_t sweeps, int32_t blocks, void* stream, float* ms, double* updates)
{
    pb::TraceRange trace_("pb_philox_ceiling");
    if (!ms || !updates || sweeps < 1) return fail(PB_EINVAL, "pb_philox_ceiling: null output or sweeps < 1");
    if (blocks <= 0) blocks = sm_count();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (sink) cudaFree(sink);
    };
    cudaError_t e = cudaMalloc(&sink, (size_t)blocks * kResidentThreads * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = ea_launch_philox_ceiling(0x5EEDu, 2, blocks, sink, st);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = ea_launch_philox_ceiling(0x5EEDu, sweeps, blocks, sink, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "pb_philox_ceiling");
    *updates = (double)blocks * kResidentThreads * 32.0 * 4.0 * sweeps;
    return PB_OK;
}

pb_status pb_run_kernel_ms(pb_run* run, float* ms)
{
    if (!run || !ms) return fail(PB_EINVAL, "null argument");
    pb_status ps = wait_run(run, -1);
    if (ps != PB_OK) return ps;
    if (run->batch && run->batch->ev_k0)
        PB_CUDA_TRY(cudaEventElapsedTime(ms, run->batch->ev_k0, run->batch->ev_k1));
    else if (run->ev_k0)
        PB_CUDA_TRY(cudaEventElapsedTime(ms, run->ev_k0, run->ev_k1));
    else
        PB_CUDA_TRY(cudaEventElapsedTime(ms, run->ev_start, run->ev_stop));
    return PB_OK;
}

void pb_run_destroy(pb_run* run)
{
    if (!run) return;
    if (run->ev_stop) cudaEventSynchronize(run->ev_stop);
    delete run;
}

pb_status pb_fields(pb_instance* I, const int8_t* states, int32_t R, float* fields_out, int64_t out_bytes, void* stream)
{
    return pb_fields_ex(I, states, R, PB_FORM_AUTO, fields_out, out_bytes, stream);
}

pb_status pb_fields_ex(pb_instance* I, const int8_t* states, int32_t R, int32_t form, float* fields_out,
                       int64_t out_bytes, void* stream)
{
    if (!I || !states || !fields_out) return fail(PB_EINVAL, "null argument");
    if (R < 1) return fail(PB_EINVAL, "R must be >= 1");
    const int64_t n = (int64_t)R * I->N;
    if (out_bytes < n * 4) return fail(PB_EINVAL, "fields_out too small");
    for (int64_t j = 0; j < n; ++j)
        if (states[j] != 1 && states[j] != -1) return fail(PB_EINVAL, "states must be +1 or -1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf dm, df;
    PB_ALLOC(dm, (size_t)n);
    PB_ALLOC(df, (size_t)n * 4);
    PB_CUDA_TRY(cudaMemcpyAsync(dm.p, states, (size_t)n, cudaMemcpyHostToDevice, st));
    if (I->topo == PB_TOPO_EA3D) {
        PB_CUDA_TRY(ea_launch_fields(I->ea, dm.as<int8_t>(), R, df.as<float>(), st));
    } else if (I->topo == PB_TOPO_CSR) {
        pb_status ps = csr_fields(I, dm.as<int8_t>(), R, df.as<float>(), st);
        if (ps != PB_OK) return ps;
    } else {
        pb_status ps = bq_fields(I, dm.as<int8_t>(), R, form, df.as<float>(), st);
        if (ps != PB_OK) return ps;
    }
    PB_CUDA_TRY(cudaMemcpyAsync(fields_out, df.p, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    return PB_OK;
}

}  // extern "C"
