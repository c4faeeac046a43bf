// biclique_host.cpp -- host runtime of the complete-bipartite (K_{n,n}) p-bit
// annealer (arXiv 2510.23419, Sec. 3): instance layouts, runs, launch order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "pb_handles.h"

namespace pb {

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

pb_status bq_build(pb_instance* I, const pb_instance_desc* d, cudaStream_t st)
{
    const int n = d->n;
    if (n < 1 || n > 16384) return fail(PB_EINVAL, "biclique side n must be in [1, 16384]");
    I->n = n;
    I->N = 2LL * n;
    I->maxdeg = n;
    const bool pm1 = d->jtype == PB_J_PM1_I8;
    if (d->colour) {
        bool canonical = true;
        for (int i = 0; i < 2 * n; ++i)
            if (d->colour[i] != (i >= n ? 1 : 0)) canonical = false;
        if (!canonical) {
            // a proper colouring of K_{n,n} (n >= 1) puts each side in one class
            for (int i = 1; i < n; ++i)
                if (d->colour[i] != d->colour[0]) return fail(PB_ECOLOUR, "left side split over colour classes");
            for (int j = n + 1; j < 2 * n; ++j)
                if (d->colour[j] != d->colour[n]) return fail(PB_ECOLOUR, "right side split over colour classes");
            if (d->colour[0] == d->colour[n]) return fail(PB_ECOLOUR, "colouring has an edge inside a colour class");
            return fail(PB_EUNSUPPORTED, "only the canonical side colouring (left = colour 0) is implemented");
        }
    }
    const size_t nn = (size_t)n * n;
    std::vector<float> Jf(nn), Jft(nn);
    if (pm1) {
        const int8_t* J = static_cast<const int8_t*>(d->J);
        for (size_t e = 0; e < nn; ++e)
            if (J[e] != 1 && J[e] != -1) return fail(PB_EINVAL, "PM1 couplings must be +1 or -1");
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                Jf[(size_t)i * n + j] = (float)J[(size_t)i * n + j];
                Jft[(size_t)j * n + i] = (float)J[(size_t)i * n + j];
            }
    } else {
        const float* J = static_cast<const float*>(d->J);
        for (size_t e = 0; e < nn; ++e)
            if (!std::isfinite(J[e])) return fail(PB_EINVAL, "F32 couplings must be finite");
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                Jf[(size_t)i * n + j] = J[(size_t)i * n + j];
                Jft[(size_t)j * n + i] = J[(size_t)i * n + j];
            }
    }
    std::vector<float> hf(2 * (size_t)n, 0.0f);
    if (d->h) {
        if (pm1) {
            const int8_t* h = static_cast<const int8_t*>(d->h);
            int hm = 0;
            for (int i = 0; i < 2 * n; ++i) hm = std::max(hm, std::abs((int)h[i]));
            if (hm > 64) return fail(PB_EINVAL, "PM1 fields must satisfy |h| <= 64");
            I->hmax = hm;
        } else {
            const float* h = static_cast<const float*>(d->h);
            for (int i = 0; i < 2 * n; ++i) hf[i] = h[i];
        }
        I->has_h = 1;
    }
    DevBuf* B = I->bq_bufs;  // 0 Jf, 1 Jft, 2 h8, 3 hf, 4 Jraw, 5 hraw
    const size_t esz = pm1 ? 1 : 4;
    PB_ALLOC(B[0], nn * 4);
    PB_ALLOC(B[1], nn * 4);
    PB_ALLOC(B[3], 2 * (size_t)n * 4);
    PB_ALLOC(B[4], nn * esz);
    PB_CUDA_TRY(cudaMemcpyAsync(B[0].p, Jf.data(), nn * 4, cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(B[1].p, Jft.data(), nn * 4, cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(B[3].p, hf.data(), 2 * (size_t)n * 4, cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(B[4].p, d->J, nn * esz, cudaMemcpyHostToDevice, st));
    if (d->h) {
        PB_ALLOC(B[5], 2 * (size_t)n * esz);
        PB_CUDA_TRY(cudaMemcpyAsync(B[5].p, d->h, 2 * (size_t)n * esz, cudaMemcpyHostToDevice, st));
        if (pm1) {
            PB_ALLOC(B[2], 2 * (size_t)n);
            PB_CUDA_TRY(cudaMemcpyAsync(B[2].p, d->h, 2 * (size_t)n, cudaMemcpyHostToDevice, st));
        }
    }
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    BqDevice& q = I->bq;
    q = BqDevice{};
    q.n = n;
    q.jtype = d->jtype;
    q.has_h = I->has_h;
    q.hmax = I->hmax;
    q.Jf = B[0].as<float>();
    q.Jft = B[1].as<float>();
    q.h8 = B[2].as<int8_t>();
    q.hf = B[3].as<float>();
    q.Jraw = B[4].p;
    q.hraw = B[5].p;
    return PB_OK;
}

static pb_status bq_prepare(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                            const pb_anneal_opts* opts, cudaStream_t st)
{
    std::vector<double> betas;
    int step = 1;
    pb_status ps = schedule_levels(sc, betas, step);
    if (ps != PB_OK) return ps;
    const int n = I->n;
    const bool pm1 = I->jtype == PB_J_PM1_I8;
    run->inst = I;
    run->R = R;
    run->S = sc->n_sweeps;
    run->N = I->N;
    run->stream = st;
    BqJob& j = run->bjob;
    j = BqJob{};
    j.inst = I->bq;
    j.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
    j.key1 = (uint32_t)(seed >> 32);
    j.S = sc->n_sweeps;
    j.step = step;
    j.R = R;
    j.Rpad = round_up(R, kBqTileReps);
    j.ld = round_up(n, 16);
    j.nblk = (n + kBqTileRows - 1) / kBqTileRows;
    const int nlev = std::max<int>(1, (int)betas.size());
    if (pm1) {
        const int fmax = n + I->hmax;
        j.fmin = -fmax;
        j.nF = 2 * fmax + 1;
        std::vector<uint32_t> tab((size_t)nlev * j.nF, 0x80000000u);
        for (size_t l = 0; l < betas.size(); ++l)
            for (int f = 0; f < j.nF; ++f) tab[l * j.nF + f] = threshold_u32(betas[l], (double)(f + j.fmin));
        PB_ALLOC(run->table, tab.size() * 4);
        PB_CUDA_TRY(cudaMemcpyAsync(run->table.p, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaStreamSynchronize(st));
        j.table = run->table.as<uint32_t>();
        PB_ALLOC(run->E_best_i, (size_t)j.Rpad * 4);
        j.E_best_i = run->E_best_i.as<int32_t>();
    } else {
        std::vector<float> bf(nlev, 0.0f);
        for (size_t l = 0; l < betas.size(); ++l) bf[l] = (float)betas[l];
        PB_ALLOC(run->betaf, bf.size() * 4);
        PB_CUDA_TRY(cudaMemcpyAsync(run->betaf.p, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaStreamSynchronize(st));
        j.betaf = run->betaf.as<float>();
        PB_ALLOC(run->E_best_f, (size_t)j.Rpad * 4);
        j.E_best_f = run->E_best_f.as<float>();
    }
    if (opts && !std::isnan(opts->target_energy)) {
        j.has_target = 1;
        j.target_i = (int32_t)std::max(-2.0e9, std::min(2.0e9, std::floor(opts->target_energy)));
        j.target_f = (float)opts->target_energy;
    }
    const size_t side_bytes = (size_t)j.Rpad * j.ld * (pm1 ? 1 : 2);
    for (int s = 0; s < 2; ++s) {
        PB_ALLOC(run->extra[s], side_bytes);
        PB_ALLOC(run->extra[2 + s], side_bytes);
        PB_CUDA_TRY(cudaMemsetAsync(run->extra[s].p, 0, side_bytes, st));
        PB_CUDA_TRY(cudaMemsetAsync(run->extra[2 + s].p, 0, side_bytes, st));
        j.spins[s] = run->extra[s].p;
        j.best[s] = run->extra[2 + s].p;
    }
    PB_ALLOC(run->extra[4], (size_t)2 * j.nblk * j.Rpad * 4);
    PB_CUDA_TRY(cudaMemsetAsync(run->extra[4].p, 0, (size_t)2 * j.nblk * j.Rpad * 4, st));
    j.part = run->extra[4].p;
    PB_ALLOC(run->best_sweep, (size_t)j.Rpad * 4);
    PB_ALLOC(run->hit_sweep, (size_t)j.Rpad * 4);
    j.best_sweep = run->best_sweep.as<int32_t>();
    j.hit_sweep = run->hit_sweep.as<int32_t>();
    PB_ALLOC(run->best_pm, (size_t)R * I->N);
    PB_ALLOC(run->final_pm, (size_t)R * I->N);
    PB_ALLOC(run->E_out, (size_t)2 * R * 8);
    PB_CUDA_TRY(cudaEventCreate(&run->ev_start));
    PB_CUDA_TRY(cudaEventCreate(&run->ev_stop));
    return PB_OK;
}

static pb_status bq_enqueue_body(pb_run* run, cudaStream_t st)
{
    const BqJob& j = run->bjob;
    PB_CUDA_TRY(bq_launch_init(j, st));
    // energy of the initial state: side B fields of the initial A, no decisions
    PB_CUDA_TRY(bq_launch_cc_half(j, 0, 0, 0, nullptr, st));
    PB_CUDA_TRY(bq_launch_cc_half(j, 1, 0, 0, nullptr, st));
    PB_CUDA_TRY(bq_launch_sweep_end(j, -1, 1, st));
    for (int s = 0; s < j.S; ++s) {
        PB_CUDA_TRY(bq_launch_cc_half(j, 0, s, 1, nullptr, st));
        PB_CUDA_TRY(bq_launch_cc_half(j, 1, s, 1, nullptr, st));
        PB_CUDA_TRY(bq_launch_sweep_end(j, s, 0, st));
    }
    PB_CUDA_TRY(bq_launch_readout(j, 0, run->final_pm.as<int8_t>(), run->E_out.as<double>(), st));
    PB_CUDA_TRY(bq_launch_readout(j, 1, run->best_pm.as<int8_t>(), run->E_out.as<double>() + run->R, st));
    return PB_OK;
}

pb_status bq_anneal(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                    const pb_anneal_opts* opts, cudaStream_t st)
{
    const int form = opts ? opts->form : PB_FORM_AUTO;
    if (form != PB_FORM_AUTO && form != PB_FORM_CUDACORE)
        return fail(PB_EUNSUPPORTED, "form not available for biclique instances");
    pb_status ps = bq_prepare(run, I, sc, R, seed, opts, st);
    if (ps != PB_OK) return ps;
    run->form = PB_FORM_CUDACORE;
    PB_CUDA_TRY(cudaEventRecord(run->ev_start, st));
    const bool capture = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    if (capture) {
        auto shared = std::make_shared<BatchShared>();
        cudaGraph_t graph = nullptr;
        PB_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        ps = bq_enqueue_body(run, st);
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
        run->batch = shared;
    } else {
        ps = bq_enqueue_body(run, st);
        if (ps != PB_OK) return ps;
    }
    PB_CUDA_TRY(cudaEventRecord(run->ev_stop, st));
    return PB_OK;
}

pb_status bq_fields(pb_instance* I, const int8_t* d_states, int R, float* d_out, cudaStream_t st)
{
    pb_run run;
    pb_schedule sc{};
    sc.kind = PB_SCHED_LINEAR;
    sc.n_sweeps = 1;
    sc.step_duration = 1;
    sc.beta0 = sc.beta1 = 0.0;
    pb_status ps = bq_prepare(&run, I, &sc, R, 0, nullptr, st);
    if (ps != PB_OK) return ps;
    PB_CUDA_TRY(bq_launch_encode(run.bjob, d_states, st));
    PB_CUDA_TRY(bq_launch_cc_half(run.bjob, 0, 0, 0, d_out, st));
    PB_CUDA_TRY(bq_launch_cc_half(run.bjob, 1, 0, 0, d_out, st));
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    return PB_OK;
}

}  // namespace pb
