// biclique_host.cpp -- host runtime of the complete-bipartite (K_{n,n}) p-bit
// annealer (arXiv 2510.23419, Sec. 3): instance layouts, runs, launch order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pb_handles.h"

namespace pb {

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

// float -> bf16 with round to nearest even (finite inputs), and back
static uint16_t bf16_rne(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static float bf16_to_f(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

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
    // tensor-core operands: e4m3 (+-1) or bf16 hi/lo (F32), row stride ldj (a multiple of 16 elements)
    const int ldj = round_up(n, 16);
    const size_t tn = (size_t)n * ldj;
    if (pm1) {
        std::vector<uint8_t> q8(tn, 0), q8t(tn, 0);
        const int8_t* J = static_cast<const int8_t*>(d->J);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const uint8_t v = J[(size_t)i * n + j] > 0 ? kE4m3Plus : kE4m3Minus;
                q8[(size_t)i * ldj + j] = v;
                q8t[(size_t)j * ldj + i] = v;
            }
        PB_ALLOC(B[6], tn);
        PB_ALLOC(B[7], tn);
        PB_CUDA_TRY(cudaMemcpyAsync(B[6].p, q8.data(), tn, cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaMemcpyAsync(B[7].p, q8t.data(), tn, cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        std::vector<uint16_t> hi(tn, 0), lo(tn, 0), hit(tn, 0), lot(tn, 0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const float v = Jf[(size_t)i * n + j];
                const uint16_t h = bf16_rne(v);
                const uint16_t l = bf16_rne(v - bf16_to_f(h));
                hi[(size_t)i * ldj + j] = h;
                lo[(size_t)i * ldj + j] = l;
                hit[(size_t)j * ldj + i] = h;
                lot[(size_t)j * ldj + i] = l;
            }
        for (int b = 0; b < 4; ++b) PB_ALLOC(B[6 + b], tn * 2);
        PB_CUDA_TRY(cudaMemcpyAsync(B[6].p, hi.data(), tn * 2, cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaMemcpyAsync(B[7].p, lo.data(), tn * 2, cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaMemcpyAsync(B[8].p, hit.data(), tn * 2, cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaMemcpyAsync(B[9].p, lot.data(), tn * 2, cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaStreamSynchronize(st));
    }
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    BqDevice& q = I->bq;
    q = BqDevice{};
    q.ldj = ldj;
    if (pm1) {
        q.Jq = B[6].as<uint8_t>();
        q.Jqt = B[7].as<uint8_t>();
    } else {
        q.Jhi = B[6].as<uint16_t>();
        q.Jlo = B[7].as<uint16_t>();
        q.Jthi = B[8].as<uint16_t>();
        q.Jtlo = B[9].as<uint16_t>();
    }
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

bool bq_resident_fits(const pb_instance* I)
{
    const int nmax = I->jtype == PB_J_PM1_I8 ? kBqResMaxNpm1 : kBqResMaxNf32;
    if (I->topo != PB_TOPO_BICLIQUE || I->n > nmax) return false;
    // the widest threshold window is at most the whole row (2 (n + |h|) + 1 entries)
    const int tab = I->jtype == PB_J_PM1_I8 ? 2 * (I->n + I->hmax) + 1 : 0;
    return bq_res_smem_bytes(I->jtype, I->n, tab) <= 227 * 1024;
}

static pb_status bq_prepare(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                            const pb_anneal_opts* opts, int form, int tile_split, cudaStream_t st)
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
    j.wait_ns = kBqWaitNs;
    if (opts && (opts->flags & PB_FLAG_TEST_EXPIRE_WAITS)) {
        j.stall_loads = 1;  // failure-path test: the tensor form's waits for operands run out
        j.wait_ns = kBqTestWaitNs;
    }
    j.inst = I->bq;
    j.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
    j.key1 = (uint32_t)(seed >> 32);
    j.S = sc->n_sweeps;
    j.step = step;
    j.R = R;
    j.tile_split = tile_split;
    const bool tensor = form == PB_FORM_TENSOR;
    const bool resident = form == PB_FORM_RESIDENT;
    run->form = form;
    j.Rpad = round_up(R, tensor ? kBqTcReps : (resident ? kBqResReps : kBqTileReps));
    j.ld = round_up(n, 16);
    j.nblk = (n + (tensor ? kBqTcRows : kBqTileRows) - 1) / (tensor ? kBqTcRows : kBqTileRows);
    if (tensor) j.nblk = 4 * ((j.nblk + 1) & ~1);  // row tiles in pairs, one partial row per 32-row quarter
    const int nlev = std::max<int>(1, (int)betas.size());
    if (pm1) {
        const int fmax = n + I->hmax;
        j.fmin = -fmax;
        j.nF = 2 * fmax + 1;
        std::vector<uint32_t> tab;
        threshold_windows(betas, j.nF, j.fmin, tab, run->bq_win);
        int wmax = 0;
        for (int l = 0; l < nlev; ++l) wmax = std::max(wmax, run->bq_win[3 * l + 1]);
        j.tabmode = wmax <= kBqTcWindowMax ? 2 : (wmax * 4 <= 33 * 1024 ? 1 : 0);
        run->res_tab = wmax;
        PB_ALLOC(run->extra[7], run->bq_win.size() * 4);
        PB_CUDA_TRY(cudaMemcpyAsync(run->extra[7].p, run->bq_win.data(), run->bq_win.size() * 4, cudaMemcpyHostToDevice, st));
        j.win = run->extra[7].as<int32_t>();
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
    j.stop = nullptr;
    if (opts && !std::isnan(opts->target_energy)) {
        j.has_target = (opts->flags & PB_FLAG_STOP_AT_TARGET) ? 2 : 1;
        j.target_i = (int32_t)std::max(-2.0e9, std::min(2.0e9, std::floor(opts->target_energy)));
        j.target_f = (float)opts->target_energy;
    }
    if (j.has_target == 2) {
        const int32_t init_stop[2] = {0, -1};
        PB_ALLOC(run->n_hit, sizeof(init_stop));
        PB_CUDA_TRY(cudaMemcpyAsync(run->n_hit.p, init_stop, sizeof(init_stop), cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaStreamSynchronize(st));
        j.stop = run->n_hit.as<int32_t>();
    }
    const size_t side_bytes = (size_t)j.Rpad * j.ld * (pm1 ? 1 : 2);
    for (int s = 0; s < 2; ++s) {
        PB_ALLOC(run->extra[s], side_bytes);
        PB_ALLOC(run->bq_alt[s], side_bytes);
        PB_ALLOC(run->extra[2 + s], side_bytes);
        PB_CUDA_TRY(cudaMemsetAsync(run->extra[s].p, 0, side_bytes, st));
        PB_CUDA_TRY(cudaMemsetAsync(run->bq_alt[s].p, 0, side_bytes, st));
        PB_CUDA_TRY(cudaMemsetAsync(run->extra[2 + s].p, 0, side_bytes, st));
        j.buf[s][0] = run->extra[s].p;
        j.buf[s][1] = run->bq_alt[s].p;
        j.spins[s] = j.buf[s][0];
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
    PB_ALLOC(run->extra[5], 16);
    PB_CUDA_TRY(cudaMemsetAsync(run->extra[5].p, 0, 16, st));
    run->dev_err = run->extra[5].as<int>();  // [0] device error word, [2], [3] sweep counters
    PB_ALLOC(run->extra[6], (size_t)((n + 63) / 64) * R * 8);
    j.epart = run->extra[6].as<double>();
    if (tensor) {
        const int esz = pm1 ? 1 : 2;
        const BqDevice& q = I->bq;
        const void* a[4] = {pm1 ? (const void*)q.Jq : (const void*)q.Jhi, pm1 ? (const void*)q.Jq : (const void*)q.Jlo,
                            pm1 ? (const void*)q.Jqt : (const void*)q.Jthi, pm1 ? (const void*)q.Jqt : (const void*)q.Jtlo};
        for (int k = 0; k < 4; ++k)
            PB_CUDA_TRY(bq_tc_make_map(&run->maps.a[k], a[k], esz, (uint64_t)n, (uint64_t)n, (uint64_t)q.ldj * esz,
                                       kBqTcRows));
        for (int sd = 0; sd < 2; ++sd)
            for (int par = 0; par < 2; ++par)
                PB_CUDA_TRY(bq_tc_make_map(&run->maps.b[2 * sd + par], j.buf[sd][par], esz, (uint64_t)n,
                                           (uint64_t)j.Rpad, (uint64_t)j.ld * esz,
                                           kBqTcReps / 2));  // half a tile per cluster CTA
        PB_CUDA_TRY(bq_tc_set_smem());
        // Runs whose half-sweeps fill every cluster chain their sweep loop's launches
        // by programmatic dependent launch (the next launch's CTAs take the SMs as the
        // previous one's leave).  Smaller runs, typical of batches and the request
        // server, keep whole-kernel ordering: there, CTAs waiting for their
        // predecessor would hold SMs other jobs could use.
        j.pdl = bq_tc_fills_device(n, j.Rpad, pm1 ? 0 : 1) ? 1 : 0;
    }
    if (resident) {
        run->res_smem = bq_res_smem_bytes(I->jtype, n, pm1 ? run->res_tab : 0);
        PB_CUDA_TRY(bq_res_set_smem(I->jtype, run->res_smem));
    }
    PB_CUDA_TRY(cudaEventCreate(&run->ev_start));
    PB_CUDA_TRY(cudaEventCreate(&run->ev_stop));
    PB_CUDA_TRY(cudaEventCreate(&run->ev_k0));
    PB_CUDA_TRY(cudaEventCreate(&run->ev_k1));
    return PB_OK;
}

// The job as one launch sees it: its own side's state in the buffer of parity
// `own`, the other side's in the buffer of parity `other`.
static BqJob bq_view(const BqJob& j, int side, int own, int other)
{
    BqJob v = j;
    v.spins[side] = j.buf[side][own];
    v.spins[1 - side] = j.buf[1 - side][other];
    return v;
}

static cudaError_t bq_half(pb_run* run, int side, int own, int other, int s, const int32_t* sp, int decide,
                           float* fields_out, cudaStream_t st)
{
    const BqJob v = bq_view(run->bjob, side, own, other);
    if (run->form == PB_FORM_TENSOR)
        return bq_launch_tc_half(run->maps, 2 * (1 - side) + other, v, side, s, sp, decide, fields_out, run->dev_err,
                                 st);
    return bq_launch_cc_half(v, side, s, sp, decide, fields_out, st);
}

// Sweeps per captured chunk for an anneal of S sweeps: even (the two sweep
// counters alternate within a chunk), at most 32.  The chunk is launched
// ceil(S / c) times; the launches of the last chunk past sweep S still cost
// nearly a sweep each (their kernels start and return at once), and each
// further chunk launch costs about a quarter of that (measured on n = 512 and
// 1024 bicliques: ~21 us per idle sweep, ~5 us per chunk boundary), so the
// chunk minimises 4 x idle sweeps + chunks.
static int bq_chunk_sweeps(int S)
{
    int best = 32;
    long long best_cost = -1;
    for (int c = 32; c >= 2; c -= 2) {
        const long long n = (S + c - 1) / c;
        const long long cost = 4 * (n * c - S) + n;
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = c;
        }
    }
    return best;
}

// One chunk of sweeps.  Sweep k of the chunk reads its index from counter
// k % 2 and its sweep end stores the next index into the other counter, so no
// launch reads a counter that a concurrent block writes.  Sweeps past S do
// nothing, so the same chunk serves every part of the anneal.
static pb_status bq_enqueue_chunk(pb_run* run, int nsweeps, cudaStream_t st)
{
    const BqJob& j = run->bjob;
    int32_t* ctr = run->dev_err + 2;
    for (int k = 0; k < nsweeps; ++k) {
        const int32_t* rd = ctr + (k & 1);
        int32_t* wr = ctr + ((k + 1) & 1);
        const int p = k & 1;  // parity of the sweep (chunks start at even sweeps)
        // side A reads side B of the previous sweep; side B reads side A of this sweep
        PB_CUDA_TRY(bq_half(run, 0, p, 1 - p, 0, rd, 1, nullptr, st));
        PB_CUDA_TRY(bq_half(run, 1, p, p, 0, rd, 1, nullptr, st));
        PB_CUDA_TRY(bq_launch_sweep_end(j, 0, 0, rd, wr, st));
    }
    return PB_OK;
}

pb_status bq_setup(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                   const pb_anneal_opts* opts, cudaStream_t st, int tile_split)
{
    int form = opts ? opts->form : PB_FORM_AUTO;
    if (form == PB_FORM_AUTO) form = PB_FORM_TENSOR;
    if (form != PB_FORM_TENSOR && form != PB_FORM_CUDACORE && form != PB_FORM_RESIDENT)
        return fail(PB_EUNSUPPORTED, "form not available for biclique instances");
    if (form == PB_FORM_RESIDENT && !bq_resident_fits(I))
        return fail(PB_EUNSUPPORTED, "biclique too large for the resident form (n <= 256 for +-1, n <= 128 for F32)");
    return bq_prepare(run, I, sc, R, seed, opts, form, tile_split, st);
}

// The anneal on `st`: initial state and its energy, the sweeps as repeated
// launches of one captured chunk graph (bq_chunk_sweeps(S) sweeps; plain launches
// when the stream cannot be captured), then the readout.  The sweep index lives
// in device memory, so the chunk is the same for every part of the anneal and
// the host work does not grow with the number of sweeps.
// Resident form: the whole anneal in one launch, then the readout.
static pb_status bq_launch_resident(pb_run* run, cudaStream_t st)
{
    const BqJob& j = run->bjob;
    PB_CUDA_TRY(cudaEventRecord(run->ev_start, st));
    PB_CUDA_TRY(cudaEventRecord(run->ev_k0, st));
    PB_CUDA_TRY(bq_launch_res(j, j.inst.jtype == PB_J_PM1_I8 ? run->res_tab : 0, run->res_smem, st));
    PB_CUDA_TRY(cudaEventRecord(run->ev_k1, st));
    const int last = (j.S - 1) & 1;
    PB_CUDA_TRY(bq_launch_readout(bq_view(j, 0, last, last), 0, run->final_pm.as<int8_t>(), run->E_out.as<double>(), st));
    PB_CUDA_TRY(bq_launch_readout(j, 1, run->best_pm.as<int8_t>(), run->E_out.as<double>() + run->R, st));
    PB_CUDA_TRY(cudaEventRecord(run->ev_stop, st));
    return PB_OK;
}

pb_status bq_launch(pb_run* run, cudaStream_t st)
{
    if (run->form == PB_FORM_RESIDENT) return bq_launch_resident(run, st);
    const BqJob& j = run->bjob;
    PB_CUDA_TRY(cudaEventRecord(run->ev_start, st));
    PB_CUDA_TRY(cudaMemsetAsync(run->dev_err + 2, 0, 2 * sizeof(int32_t), st));
    // the initial state is "sweep -1": parity 1
    const BqJob init_view = bq_view(j, 0, 1, 1);
    PB_CUDA_TRY(bq_launch_init(init_view, st));
    // energy of the initial state: side B fields of the initial A, no decisions
    PB_CUDA_TRY(bq_half(run, 0, 1, 1, 0, nullptr, 0, nullptr, st));
    PB_CUDA_TRY(bq_half(run, 1, 1, 1, 0, nullptr, 0, nullptr, st));
    PB_CUDA_TRY(bq_launch_sweep_end(j, -1, 1, nullptr, nullptr, st));
    PB_CUDA_TRY(cudaEventRecord(run->ev_k0, st));
    if (j.S > 0) {
        const int chunk = bq_chunk_sweeps(j.S);
        const int nchunks = (j.S + chunk - 1) / chunk;
        const bool capture = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
        if (capture) {
            // one captured chunk, launched ceil(S / chunk) times; launches past the last sweep (or, in stop
            // mode, past the sweep at which every replica had reached the target) return at once.  A graph
            // while node that ends the loop on the device was measured slower: served stream p50 13 -> 17 ms,
            // mixed batch 2.66 -> 3.19 s.
            auto shared = std::make_shared<BatchShared>();
            cudaGraph_t graph = nullptr;
            PB_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            pb_status ps = bq_enqueue_chunk(run, chunk, st);
            cudaError_t e = cudaStreamEndCapture(st, &graph);
            if (ps != PB_OK) {
                if (graph) cudaGraphDestroy(graph);
                return ps;
            }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&shared->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            for (int c = 0; c < nchunks; ++c) PB_CUDA_TRY(cudaGraphLaunch(shared->exec, st));
            run->batch = shared;
        } else {
            for (int c = 0; c < nchunks; ++c) {
                pb_status ps = bq_enqueue_chunk(run, chunk, st);
                if (ps != PB_OK) return ps;
            }
        }
    }
    PB_CUDA_TRY(bq_launch_best_flush(j, st));
    PB_CUDA_TRY(cudaEventRecord(run->ev_k1, st));
    const int last = (j.S - 1) & 1;  // parity of the final state (S = 0: the initial state)
    PB_CUDA_TRY(bq_launch_readout(bq_view(j, 0, last, last), 0, run->final_pm.as<int8_t>(), run->E_out.as<double>(), st));
    PB_CUDA_TRY(bq_launch_readout(j, 1, run->best_pm.as<int8_t>(), run->E_out.as<double>() + run->R, st));
    PB_CUDA_TRY(cudaEventRecord(run->ev_stop, st));
    return PB_OK;
}

pb_status bq_anneal(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                    const pb_anneal_opts* opts, cudaStream_t st, int tile_split)
{
    pb_status ps = bq_setup(run, I, sc, R, seed, opts, st, tile_split);
    if (ps != PB_OK) return ps;
    return bq_launch(run, st);
}

pb_status bq_fields(pb_instance* I, const int8_t* d_states, int R, int form, float* d_out, cudaStream_t st)
{
    if (form == PB_FORM_AUTO) form = PB_FORM_TENSOR;
    if (form != PB_FORM_TENSOR && form != PB_FORM_CUDACORE)
        return fail(PB_EUNSUPPORTED, "form not available for biclique instances");
    pb_run run;
    pb_schedule sc{};
    sc.kind = PB_SCHED_LINEAR;
    sc.n_sweeps = 1;
    sc.step_duration = 1;
    sc.beta0 = sc.beta1 = 0.0;
    pb_status ps = bq_prepare(&run, I, &sc, R, 0, nullptr, form, 1, st);
    if (ps != PB_OK) return ps;
    PB_CUDA_TRY(bq_launch_encode(run.bjob, d_states, st));
    PB_CUDA_TRY(bq_half(&run, 0, 0, 0, 0, nullptr, 0, d_out, st));
    PB_CUDA_TRY(bq_half(&run, 1, 0, 0, 0, nullptr, 0, d_out, st));
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    int code = 0;
    PB_CUDA_TRY(cudaMemcpy(&code, run.dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (code) return fail(PB_ETIMEOUT, "a device-side wait timed out (code " + std::to_string(code) + ")");
    return PB_OK;
}

}  // namespace pb
