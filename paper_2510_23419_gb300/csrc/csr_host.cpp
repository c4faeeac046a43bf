// csr_host.cpp -- general sparse instances (arXiv 2510.23419, Eq. 1 on an
// arbitrary edge set; update groups of Sec. 1.2.2 from a proper colouring):
// instance build, greedy colouring, runs of the plain per-class form.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "pb_handles.h"

namespace pb {

namespace {

// Greedy colouring, vertices by decreasing degree (ties by index): each takes
// the smallest colour that none of its coloured neighbours has.  Returns the
// number of colours.
int greedy_colouring(int32_t N, int64_t E, const int32_t* eu, const int32_t* ev, int32_t* colour)
{
    std::vector<int64_t> off((size_t)N + 1, 0);
    for (int64_t e = 0; e < E; ++e) {
        off[(size_t)eu[e] + 1]++;
        off[(size_t)ev[e] + 1]++;
    }
    for (int32_t i = 0; i < N; ++i) off[(size_t)i + 1] += off[i];
    std::vector<int32_t> adj((size_t)(2 * E));
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    for (int64_t e = 0; e < E; ++e) {
        adj[(size_t)fill[eu[e]]++] = ev[e];
        adj[(size_t)fill[ev[e]]++] = eu[e];
    }
    std::vector<int32_t> order((size_t)N);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    std::fill(colour, colour + N, -1);
    std::vector<int64_t> seen;  // seen[c] == i: colour c is taken by a neighbour of i
    int k = 0;
    for (int32_t i : order) {
        for (int64_t a = off[i]; a < off[i + 1]; ++a) {
            const int32_t c = colour[adj[(size_t)a]];
            if (c >= 0) {
                if ((size_t)c >= seen.size()) seen.resize((size_t)c + 1, -1);
                seen[(size_t)c] = i;
            }
        }
        int c = 0;
        while ((size_t)c < seen.size() && seen[(size_t)c] == i) ++c;
        colour[i] = c;
        k = std::max(k, c + 1);
    }
    return k;
}

}  // namespace

pb_status csr_build(pb_instance* I, int32_t N, int64_t E, const int32_t* eu, const int32_t* ev, int jtype,
                    const void* J, const void* h, const int32_t* colour_in, cudaStream_t st)
{
    if (N < 1 || E < 0) return fail(PB_EINVAL, "graph needs N >= 1 and n_edges >= 0");
    if (E > 0 && (!eu || !ev || !J)) return fail(PB_EINVAL, "edge arrays are null");
    if (2 * E > 2000000000LL) return fail(PB_EINVAL, "too many edges");
    const bool pm1 = jtype == PB_J_PM1_I8;
    for (int64_t e = 0; e < E; ++e) {
        if (eu[e] < 0 || eu[e] >= N || ev[e] < 0 || ev[e] >= N) return fail(PB_EINVAL, "edge end out of range");
        if (eu[e] == ev[e]) return fail(PB_EINVAL, "self-loop edge");
        if (pm1) {
            const int v = static_cast<const int8_t*>(J)[e];
            if (v != 1 && v != -1) return fail(PB_EINVAL, "PM1 couplings must be +1 or -1");
        }
    }
    // colouring: given (validated) or greedy
    std::vector<int32_t> colour((size_t)N);
    int k = 0;
    if (colour_in) {
        for (int32_t i = 0; i < N; ++i) {
            if (colour_in[i] < 0 || colour_in[i] > 254) return fail(PB_ECOLOUR, "colour out of range [0, 254]");
            colour[i] = colour_in[i];
            k = std::max(k, colour[i] + 1);
        }
        for (int64_t e = 0; e < E; ++e)
            if (colour[eu[e]] == colour[ev[e]]) return fail(PB_ECOLOUR, "an edge joins two spins of the same colour");
    } else {
        k = greedy_colouring(N, E, eu, ev, colour.data());
        if (k > 255) return fail(PB_ECOLOUR, "greedy colouring needs more than 255 colours");
    }
    // classes in ascending index; a spin's label is its position in the class
    // list, so class c holds the labels cls_off[c] .. cls_off[c+1]-1
    std::vector<int32_t> cls_off((size_t)k + 1, 0);
    for (int32_t i = 0; i < N; ++i) cls_off[(size_t)colour[i] + 1]++;
    for (int c = 0; c < k; ++c) cls_off[(size_t)c + 1] += cls_off[c];
    std::vector<int32_t> orig((size_t)N), pos((size_t)N), cf(cls_off.begin(), cls_off.end() - 1);
    for (int32_t i = 0; i < N; ++i) {
        const int32_t p = cf[colour[i]]++;
        orig[(size_t)p] = i;
        pos[(size_t)i] = p;
    }
    // compressed rows over the labels, half-edges in edge order
    std::vector<int32_t> rowptr((size_t)N + 1, 0);
    for (int64_t e = 0; e < E; ++e) {
        rowptr[(size_t)pos[eu[e]] + 1]++;
        rowptr[(size_t)pos[ev[e]] + 1]++;
    }
    for (int32_t p = 0; p < N; ++p) rowptr[(size_t)p + 1] += rowptr[p];
    std::vector<int32_t> col((size_t)(2 * E));
    std::vector<int8_t> J8(pm1 ? (size_t)(2 * E) : 0);
    std::vector<float> Jf(pm1 ? 0 : (size_t)(2 * E));
    std::vector<int32_t> fill(rowptr.begin(), rowptr.end() - 1);
    for (int64_t e = 0; e < E; ++e) {
        const int32_t ends[2][2] = {{pos[eu[e]], pos[ev[e]]}, {pos[ev[e]], pos[eu[e]]}};
        for (auto& uv : ends) {
            const int32_t a = fill[uv[0]]++;
            col[(size_t)a] = uv[1];
            if (pm1) J8[(size_t)a] = static_cast<const int8_t*>(J)[e];
            else Jf[(size_t)a] = static_cast<const float*>(J)[e];
        }
    }
    // +-1 rows: J = +1 half-edges first (stable), so the field walk needs no coupling
    std::vector<int32_t> rowneg(pm1 ? (size_t)N : 0);
    if (pm1) {
        std::vector<int32_t> tc;
        for (int32_t p = 0; p < N; ++p) {
            const int32_t a0 = rowptr[p], a1 = rowptr[(size_t)p + 1];
            tc.clear();
            int32_t w = a0;
            for (int32_t a = a0; a < a1; ++a) {
                if (J8[(size_t)a] > 0) col[(size_t)w++] = col[(size_t)a];
                else tc.push_back(col[(size_t)a]);
            }
            rowneg[(size_t)p] = w;
            for (int32_t v : tc) col[(size_t)w++] = v;
            for (int32_t a = a0; a < a1; ++a) J8[(size_t)a] = a < rowneg[(size_t)p] ? 1 : -1;
        }
    }
    int maxdeg = 0;
    for (int32_t p = 0; p < N; ++p) maxdeg = std::max(maxdeg, rowptr[(size_t)p + 1] - rowptr[p]);
    // +-1, degree <= kCsrEllSlots: padded rows (unused slots name the zero row N)
    const bool ell = pm1 && maxdeg <= kCsrEllSlots;
    std::vector<int32_t> ellv(ell ? (size_t)N * kCsrEllSlots : 0, N);
    std::vector<uint16_t> ellnd(ell ? (size_t)N : 0);
    for (int32_t p = 0; ell && p < N; ++p) {
        const int32_t a0 = rowptr[p], a1 = rowptr[(size_t)p + 1];
        for (int32_t a = a0; a < a1; ++a) ellv[(size_t)p * kCsrEllSlots + (a - a0)] = col[(size_t)a];
        ellnd[(size_t)p] = (uint16_t)((rowneg[(size_t)p] - a0) | ((a1 - a0) << 8));
    }
    // per-label colour and field
    std::vector<int32_t> colour_l((size_t)N);
    for (int32_t p = 0; p < N; ++p) colour_l[(size_t)p] = colour[orig[(size_t)p]];
    std::vector<int8_t> h8l(h && pm1 ? (size_t)N : 0);
    std::vector<float> hfl(h && !pm1 ? (size_t)N : 0);
    for (int32_t p = 0; h && p < N; ++p) {
        if (pm1) h8l[(size_t)p] = static_cast<const int8_t*>(h)[orig[(size_t)p]];
        else hfl[(size_t)p] = static_cast<const float*>(h)[orig[(size_t)p]];
    }
    int hmax = 0;
    if (h && pm1) {
        for (int32_t i = 0; i < N; ++i) hmax = std::max(hmax, std::abs((int)static_cast<const int8_t*>(h)[i]));
        if (hmax > 64) return fail(PB_EINVAL, "PM1 fields must satisfy |h| <= 64");
    }

    I->topo = PB_TOPO_CSR;
    I->jtype = jtype;
    I->N = N;
    I->n = N;
    I->has_h = h ? 1 : 0;
    I->hmax = hmax;
    I->maxdeg = maxdeg;
    I->n_colours = k;
    I->csr_cls_off = cls_off;
    I->csr_orig = orig;
    DevBuf* B = I->csr_bufs;  // 0 rowptr, 1 col, 2 J, 3 h, 4 cls_off, 5 orig, 6 colour, 7 rowneg, 8 pos
    auto up = [&](DevBuf& b, const void* src, size_t bytes) -> pb_status {
        PB_ALLOC(b, bytes);
        if (bytes) PB_CUDA_TRY(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st));
        return PB_OK;
    };
    pb_status ps;
    if ((ps = up(B[0], rowptr.data(), rowptr.size() * 4)) != PB_OK) return ps;
    if ((ps = up(B[1], col.data(), col.size() * 4)) != PB_OK) return ps;
    if ((ps = pm1 ? up(B[2], J8.data(), J8.size()) : up(B[2], Jf.data(), Jf.size() * 4)) != PB_OK) return ps;
    if (h && (ps = pm1 ? up(B[3], h8l.data(), h8l.size()) : up(B[3], hfl.data(), hfl.size() * 4)) != PB_OK) return ps;
    if ((ps = up(B[4], cls_off.data(), cls_off.size() * 4)) != PB_OK) return ps;
    if ((ps = up(B[5], orig.data(), orig.size() * 4)) != PB_OK) return ps;
    if ((ps = up(B[6], colour_l.data(), colour_l.size() * 4)) != PB_OK) return ps;
    if (pm1 && (ps = up(B[7], rowneg.data(), rowneg.size() * 4)) != PB_OK) return ps;
    if ((ps = up(B[8], pos.data(), pos.size() * 4)) != PB_OK) return ps;
    if (ell && (ps = up(B[9], ellv.data(), ellv.size() * 4)) != PB_OK) return ps;
    if (ell && (ps = up(B[10], ellnd.data(), ellnd.size() * 2)) != PB_OK) return ps;
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    CsrDevice& g = I->csr;
    g = CsrDevice{};
    g.N = N;
    g.jtype = jtype;
    g.n_colours = k;
    g.maxdeg = maxdeg;
    g.has_h = I->has_h;
    g.hmax = hmax;
    g.rowptr = B[0].as<int32_t>();
    g.col = B[1].as<int32_t>();
    g.rowneg = pm1 ? B[7].as<int32_t>() : nullptr;
    g.J8 = pm1 ? B[2].as<int8_t>() : nullptr;
    g.Jf = pm1 ? nullptr : B[2].as<float>();
    g.h8 = (h && pm1) ? B[3].as<int8_t>() : nullptr;
    g.hf = (h && !pm1) ? B[3].as<float>() : nullptr;
    g.cls_off = B[4].as<int32_t>();
    g.orig = B[5].as<int32_t>();
    g.pos = B[8].as<int32_t>();
    g.colour = B[6].as<int32_t>();
    g.ell = ell ? B[9].as<int4>() : nullptr;
    g.ell_nd = ell ? B[10].as<uint16_t>() : nullptr;
    return PB_OK;
}

// Buffers and tables of a run of R replicas over the levels `betas` (schedule
// levels for annealing, the temperature ladder for tempering).
static pb_status csr_prepare(pb_run* run, pb_instance* I, const std::vector<double>& betas, int step, int S, int R,
                             uint64_t seed, const pb_anneal_opts* opts, cudaStream_t st, bool temp = false)
{
    run->inst = I;
    run->form = PB_FORM_PLAIN;
    run->R = R;
    run->S = S;
    run->N = I->N;
    run->stream = st;
    CsrJob& j = run->cjob;
    j = CsrJob{};
    j.g = I->csr;
    j.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
    j.key1 = (uint32_t)(seed >> 32);
    j.S = S;
    j.step = step;
    j.R = R;
    j.Rw = (R + 3) / 4;
    const int nlev = std::max<int>(1, (int)betas.size());
    if (I->jtype == PB_J_PM1_I8) {
        const int fmax = I->maxdeg + I->hmax;
        j.fmin = -fmax;
        j.nF = 2 * fmax + 1;
        std::vector<uint32_t> tab;
        threshold_windows(betas, j.nF, j.fmin, tab, run->bq_win);
        PB_ALLOC(run->table, tab.size() * 4);
        PB_CUDA_TRY(cudaMemcpyAsync(run->table.p, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, st));
        PB_ALLOC(run->extra[7], run->bq_win.size() * 4);
        PB_CUDA_TRY(cudaMemcpyAsync(run->extra[7].p, run->bq_win.data(), run->bq_win.size() * 4,
                                    cudaMemcpyHostToDevice, st));
        j.table = run->table.as<uint32_t>();
        j.win = run->extra[7].as<int32_t>();
    } else {
        std::vector<float> bf((size_t)nlev, 0.0f);
        for (size_t l = 0; l < betas.size(); ++l) bf[l] = (float)betas[l];
        PB_ALLOC(run->betaf, bf.size() * 4);
        PB_CUDA_TRY(cudaMemcpyAsync(run->betaf.p, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice, st));
        j.betaf = run->betaf.as<float>();
    }
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    j.stop = nullptr;
    if (opts && !std::isnan(opts->target_energy)) {
        j.has_target = (opts->flags & PB_FLAG_STOP_AT_TARGET) ? 2 : 1;
        j.target = opts->target_energy;
    }
    if (j.has_target == 2) {
        const int32_t init_stop[2] = {0, -1};
        PB_ALLOC(run->n_hit, sizeof(init_stop));
        PB_CUDA_TRY(cudaMemcpyAsync(run->n_hit.p, init_stop, sizeof(init_stop), cudaMemcpyHostToDevice, st));
        PB_CUDA_TRY(cudaStreamSynchronize(st));
        j.stop = run->n_hit.as<int32_t>();
    }
    const size_t words = (size_t)I->N * j.Rw;
    j.nchunk = (int)((I->N + kCsrChunk - 1) / kCsrChunk);
    PB_ALLOC(run->final_words, words * 4 + (size_t)j.Rw * 4);  // + the zero row of the padded rows
    PB_CUDA_TRY(cudaMemsetAsync(run->final_words.as<uint32_t>() + words, 0, (size_t)j.Rw * 4, st));
    PB_ALLOC(run->best_words, words * 4);
    PB_ALLOC(run->extra[0], (size_t)j.nchunk * 4 * j.Rw * 8);
    PB_ALLOC(run->extra[1], (size_t)4 * j.Rw * 8);
    PB_ALLOC(run->best_sweep, (size_t)4 * j.Rw * 4);
    PB_ALLOC(run->hit_sweep, (size_t)4 * j.Rw * 4);
    PB_ALLOC(run->extra[2], (size_t)4 * j.Rw + 16);
    PB_ALLOC(run->extra[3], (size_t)4 * j.Rw * 8);
    j.E_cur = run->extra[3].as<double>();
    // class chunks of the energy changes
    const int k = I->n_colours;
    run->csr_nchunk.assign((size_t)k, 0);
    std::vector<int32_t> doff((size_t)k + 1, 0);
    for (int c = 0; c < k; ++c) {
        const int ncls = I->csr_cls_off[(size_t)c + 1] - I->csr_cls_off[(size_t)c];
        const int nb = csr_class_blocks(I->jtype, temp, j.Rw, ncls, I->maxdeg, I->hmax);
        if (nb < 0) return fail(PB_EDEVICE, "occupancy query of the class kernel failed");
        run->csr_nchunk[(size_t)c] = nb;
        doff[(size_t)c + 1] = doff[(size_t)c] + run->csr_nchunk[(size_t)c];
    }
    j.ndchunk = doff[(size_t)k];
    PB_ALLOC(run->extra[4], doff.size() * 4);
    PB_CUDA_TRY(cudaMemcpyAsync(run->extra[4].p, doff.data(), doff.size() * 4, cudaMemcpyHostToDevice, st));
    // +-1: one int64 accumulator per replica; FP32: a partial per class chunk
    const bool pm1 = I->jtype == PB_J_PM1_I8;
    const size_t dbytes = (pm1 ? (size_t)1 : (size_t)std::max(1, j.ndchunk)) * 4 * j.Rw * 8;
    PB_ALLOC(run->extra[5], dbytes);
    PB_CUDA_TRY(cudaMemsetAsync(run->extra[5].p, 0, dbytes, st));
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    j.dchunk_off = run->extra[4].as<int32_t>();
    j.dpart = pm1 ? nullptr : run->extra[5].as<double>();
    j.dacc = pm1 ? run->extra[5].as<unsigned long long>() : nullptr;
    j.spins = run->final_words.as<uint32_t>();
    j.best = run->best_words.as<uint32_t>();
    j.part = run->extra[0].as<double>();
    j.E_best = run->extra[1].as<double>();
    j.best_sweep = run->best_sweep.as<int32_t>();
    j.hit_sweep = run->hit_sweep.as<int32_t>();
    j.improved = run->extra[2].as<uint8_t>();
    PB_ALLOC(run->best_pm, (size_t)R * I->N);
    PB_ALLOC(run->final_pm, (size_t)R * I->N);
    PB_ALLOC(run->E_out, (size_t)2 * R * 8);
    PB_CUDA_TRY(cudaEventCreate(&run->ev_start));
    PB_CUDA_TRY(cudaEventCreate(&run->ev_stop));
    PB_CUDA_TRY(cudaEventCreate(&run->ev_k0));
    PB_CUDA_TRY(cudaEventCreate(&run->ev_k1));
    return PB_OK;
}

pb_status csr_setup(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                    const pb_anneal_opts* opts, cudaStream_t st)
{
    const int form = opts ? opts->form : PB_FORM_AUTO;
    if (form != PB_FORM_AUTO && form != PB_FORM_PLAIN)
        return fail(PB_EUNSUPPORTED, "general sparse instances run in the plain form");
    std::vector<double> betas;
    int step = 1;
    pb_status ps = schedule_levels(sc, betas, step);
    if (ps != PB_OK) return ps;
    return csr_prepare(run, I, betas, step, sc->n_sweeps, R, seed, opts, st);
}

// Parallel tempering: M temperatures x C chains = M C slots; slot g = k C + r
// starts at temperature k.  +-1 exchange thresholds floor(exp(dbeta (-d)) 2^32)
// for d = 1, 2, ... until they reach 0, in FP64 on the host (the expression the
// oracle evaluates).
static pb_status csr_setup_pt(pb_run* run, pb_instance* I, const double* ladder, int M, int S, int C, uint64_t seed,
                              cudaStream_t st)
{
    std::vector<double> lad(ladder, ladder + M);
    pb_status ps = csr_prepare(run, I, lad, 1, S, M * C, seed, nullptr, st, true);
    if (ps != PB_OK) return ps;
    CsrJob& j = run->cjob;
    j.M = M;
    j.C = C;
    std::vector<uint8_t> temp((size_t)4 * j.Rw, 0);
    std::vector<int32_t> slot_of((size_t)M * C);
    for (int g = 0; g < M * C; ++g) {
        temp[(size_t)g] = (uint8_t)(g / C);
        slot_of[(size_t)g] = g;
    }
    DevBuf* P = run->pt;  // 0 temp, 1 slot_of, 2 xdb, 3 xtab, 4 xwin, 5 n_accept
    PB_ALLOC(P[0], temp.size());
    PB_CUDA_TRY(cudaMemcpyAsync(P[0].p, temp.data(), temp.size(), cudaMemcpyHostToDevice, st));
    PB_ALLOC(P[1], slot_of.size() * 4);
    PB_CUDA_TRY(cudaMemcpyAsync(P[1].p, slot_of.data(), slot_of.size() * 4, cudaMemcpyHostToDevice, st));
    // real couplings: the exponent's beta step per pair, times log2 e, in FP32 for the device rule
    std::vector<float> xdb((size_t)std::max(1, M - 1), 0.0f);
    for (int t = 0; t + 1 < M; ++t) xdb[(size_t)t] = (float)((ladder[t + 1] - ladder[t]) * 1.4426950408889634);
    PB_ALLOC(P[2], xdb.size() * 4);
    PB_CUDA_TRY(cudaMemcpyAsync(P[2].p, xdb.data(), xdb.size() * 4, cudaMemcpyHostToDevice, st));
    std::vector<uint32_t> xtab;
    std::vector<int32_t> xwin((size_t)2 * std::max(1, M - 1), 0);
    if (I->jtype == PB_J_PM1_I8) {
        for (int t = 0; t + 1 < M; ++t) {
            const double db = ladder[t + 1] - ladder[t];
            xwin[(size_t)2 * t + 1] = (int32_t)xtab.size();
            for (long long d = 1;; ++d) {
                const double A = std::floor(std::exp(db * (double)(-d)) * 4294967296.0);
                if (A <= 0.0) break;
                if (d > (1LL << 22))
                    return fail(PB_EINVAL, "temperature spacing too small for the exchange table (> 2^22 entries)");
                xtab.push_back((uint32_t)A);
                xwin[(size_t)2 * t] = (int32_t)d;
            }
        }
    }
    PB_ALLOC(P[3], std::max<size_t>(1, xtab.size()) * 4);
    if (!xtab.empty()) PB_CUDA_TRY(cudaMemcpyAsync(P[3].p, xtab.data(), xtab.size() * 4, cudaMemcpyHostToDevice, st));
    PB_ALLOC(P[4], xwin.size() * 4);
    PB_CUDA_TRY(cudaMemcpyAsync(P[4].p, xwin.data(), xwin.size() * 4, cudaMemcpyHostToDevice, st));
    PB_ALLOC(P[5], (size_t)std::max(1, M - 1) * 8);
    PB_CUDA_TRY(cudaMemsetAsync(P[5].p, 0, (size_t)std::max(1, M - 1) * 8, st));
    PB_CUDA_TRY(cudaStreamSynchronize(st));
    j.temp = P[0].as<uint8_t>();
    j.slot_of = P[1].as<int32_t>();
    j.xdb = P[2].as<float>();
    j.xtab = P[3].as<uint32_t>();
    j.xwin = P[4].as<int32_t>();
    j.n_accept = P[5].as<unsigned long long>();
    return PB_OK;
}

// Plain form: one launch per colour class and sweep, then the energy of the
// sweep and the running best (Sec. 1.2.2, Eq. 2, Eq. 3).
pb_status csr_launch(pb_run* run, cudaStream_t st)
{
    const CsrJob& j = run->cjob;
    PB_CUDA_TRY(cudaEventRecord(run->ev_start, st));
    if (!run->resumed) PB_CUDA_TRY(csr_launch_init(j, st));
    PB_CUDA_TRY(csr_launch_energy(j, j.spins, 0, st));
    PB_CUDA_TRY(csr_launch_sweep_end(j, j.s0 - 1, run->resumed ? 2 : 1, st));
    PB_CUDA_TRY(cudaEventRecord(run->ev_k0, st));
    for (int s = j.s0; s < j.S; ++s) {
        for (int c = 0; c < j.g.n_colours; ++c)
            PB_CUDA_TRY(csr_launch_class(j, c, run->csr_nchunk[(size_t)c], s, st));
        PB_CUDA_TRY(csr_launch_sweep_end(j, s, 0, st));
        if (j.temp) PB_CUDA_TRY(csr_launch_exchange(j, s, st));
    }
    PB_CUDA_TRY(csr_launch_snapshot(j, st));  // the last sweep's improvements
    PB_CUDA_TRY(cudaEventRecord(run->ev_k1, st));
    PB_CUDA_TRY(csr_launch_readout(j, j.spins, run->final_pm.as<int8_t>(), run->E_out.as<double>(), st));
    PB_CUDA_TRY(csr_launch_readout(j, j.best, run->best_pm.as<int8_t>(), run->E_out.as<double>() + run->R, st));
    PB_CUDA_TRY(cudaEventRecord(run->ev_stop, st));
    return PB_OK;
}

pb_status csr_fields(pb_instance* I, const int8_t* d_states, int R, float* d_out, cudaStream_t st)
{
    CsrJob j{};
    j.g = I->csr;
    j.R = R;
    j.Rw = (R + 3) / 4;
    PB_CUDA_TRY(csr_launch_fields(j, d_states, d_out, st));
    return PB_OK;
}

}  // namespace pb

using namespace pb;

extern "C" {

int32_t pb_greedy_colouring(int32_t N, int64_t n_edges, const int32_t* eu, const int32_t* ev, int32_t* colour_out)
{
    if (N < 1 || n_edges < 0 || !colour_out || (n_edges > 0 && (!eu || !ev))) return -1;
    for (int64_t e = 0; e < n_edges; ++e)
        if (eu[e] < 0 || eu[e] >= N || ev[e] < 0 || ev[e] >= N || eu[e] == ev[e]) return -1;
    return greedy_colouring(N, n_edges, eu, ev, colour_out);
}

pb_status pb_create_graph_instance(const pb_graph_desc* d, void* stream, pb_instance** out)
{
    pb::TraceRange trace_("pb_create_graph_instance");
    if (!d || !out) return fail(PB_EINVAL, "null argument");
    *out = nullptr;
    if (d->jtype != PB_J_PM1_I8 && d->jtype != PB_J_F32) return fail(PB_EINVAL, "unknown jtype");
    std::unique_ptr<pb_instance> I(new (std::nothrow) pb_instance());
    if (!I) return fail(PB_ENOMEM, "host allocation failed");
    pb_status ps = csr_build(I.get(), d->N, d->n_edges, d->eu, d->ev, d->jtype, d->J, d->h, d->colour,
                             static_cast<cudaStream_t>(stream));
    if (ps != PB_OK) return ps;
    *out = I.release();
    return PB_OK;
}

}  // extern "C"

namespace pb {

// General-graph part of pb_anneal_resume (arguments checked by the caller).
pb_status csr_anneal_resume(pb_instance* I, const pb_schedule* sched, int32_t replicas, uint64_t seed,
                            int32_t first_sweep, const int8_t* state, const int8_t* best_state, const double* best_E,
                            const int32_t* best_sweep, cudaStream_t st, pb_run** out)
{
    const int64_t N = I->N, R = replicas;
    std::unique_ptr<pb_run> run(new (std::nothrow) pb_run());
    if (!run) return fail(PB_ENOMEM, "host allocation failed");
    pb_status ps = csr_setup(run.get(), I, sched, replicas, seed, nullptr, st);
    if (ps != PB_OK) return ps;
    CsrJob& j = run->cjob;
    j.s0 = first_sweep;
    run->resumed = true;
    // [R][N] +-1 (original order) -> [N][Rw] words by label (byte b of word q: replica
    // 4q + b, 1 <=> m = -1; padding replicas +1)
    const int64_t Rw = j.Rw;
    std::vector<uint32_t> w((size_t)(N * Rw)), wb((size_t)(N * Rw));
    for (int64_t p = 0; p < N; ++p) {
        const int64_t i = I->csr_orig[(size_t)p];
        for (int64_t r = 0; r < R; ++r) {
            const int8_t m = state[r * N + i], mb = best_state[r * N + i];
            if ((m != 1 && m != -1) || (mb != 1 && mb != -1)) return fail(PB_EINVAL, "states must hold +1 or -1");
            const uint32_t sh = 8u * (uint32_t)(r & 3);
            w[(size_t)(p * Rw + (r >> 2))] |= (m < 0 ? 1u : 0u) << sh;
            wb[(size_t)(p * Rw + (r >> 2))] |= (mb < 0 ? 1u : 0u) << sh;
        }
    }
    std::vector<double> eb((size_t)(4 * Rw), 1e300);  // padding replicas: any state improves on it
    std::vector<int32_t> bs((size_t)(4 * Rw), -1);
    for (int64_t r = 0; r < R; ++r) {
        eb[(size_t)r] = best_E[r];
        bs[(size_t)r] = best_sweep[r];
    }
    PB_CUDA_TRY(cudaMemcpyAsync(j.spins, w.data(), w.size() * 4, cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(j.best, wb.data(), wb.size() * 4, cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(j.E_best, eb.data(), eb.size() * 8, cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaMemcpyAsync(j.best_sweep, bs.data(), bs.size() * 4, cudaMemcpyHostToDevice, st));
    PB_CUDA_TRY(cudaStreamSynchronize(st));  // the host staging arrays go out of scope; the anneal stays asynchronous
    ps = csr_launch(run.get(), st);
    if (ps != PB_OK) return ps;
    *out = run.release();
    return PB_OK;
}

}  // namespace pb

extern "C" {

pb_status pb_anneal_pt(pb_instance* I, const double* ladder, int32_t M, int32_t n_sweeps, int32_t chains,
                       uint64_t seed, void* stream, pb_run** out)
{
    pb::TraceRange trace_("pb_anneal_pt");
    if (!I || !ladder || !out) return fail(PB_EINVAL, "null argument");
    *out = nullptr;
    if (I->topo != PB_TOPO_CSR)
        return fail(PB_EUNSUPPORTED, "parallel tempering runs on general sparse instances (pb_create_graph_instance)");
    if (M < 1 || M > 255 || chains < 1 || n_sweeps < 0) return fail(PB_EINVAL, "need 1 <= M <= 255, chains >= 1");
    for (int t = 0; t + 1 < M; ++t)
        if (!(ladder[t] < ladder[t + 1])) return fail(PB_EINVAL, "the ladder must increase");
    if ((int64_t)M * chains > (1LL << 30)) return fail(PB_EINVAL, "too many slots");
    std::unique_ptr<pb_run> run(new (std::nothrow) pb_run());
    if (!run) return fail(PB_ENOMEM, "host allocation failed");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pb_status ps = csr_setup_pt(run.get(), I, ladder, M, n_sweeps, chains, seed, st);
    if (ps == PB_OK) ps = csr_launch(run.get(), st);
    if (ps != PB_OK) return ps;
    *out = run.release();
    return PB_OK;
}

pb_status pb_pt_state(pb_run* run, int32_t* slot_temp, int64_t* n_accept)
{
    if (!run) return fail(PB_EINVAL, "null argument");
    if (!run->cjob.temp) return fail(PB_EINVAL, "not a parallel-tempering run");
    pb_status ps = wait_run(run, -1);
    if (ps != PB_OK) return ps;
    const CsrJob& j = run->cjob;
    if (slot_temp) {
        std::vector<uint8_t> t((size_t)j.M * j.C);
        PB_CUDA_TRY(cudaMemcpy(t.data(), j.temp, t.size(), cudaMemcpyDeviceToHost));
        for (size_t g = 0; g < t.size(); ++g) slot_temp[g] = t[g];
    }
    if (n_accept && j.M > 1)
        PB_CUDA_TRY(cudaMemcpy(n_accept, j.n_accept, (size_t)(j.M - 1) * 8, cudaMemcpyDeviceToHost));
    return PB_OK;
}

int32_t pb_instance_colours(const pb_instance* inst)
{
    if (!inst) return -1;
    if (inst->topo == PB_TOPO_CSR) return inst->n_colours;
    return 2;
}

}  // extern "C"
