// batch.cpp -- batched anneals of mixed topology and the autotuner
// (arXiv 2510.23419: many independent annealing runs, Sec. 1.2.2 update
// groups, the instance families of Sec. 2 and Sec. 3).
//
// A batch prepares every job first (allocations, threshold tables, copies on
// the caller's stream, one synchronisation), then launches:
//   * all EA jobs that fit the resident form share ONE graph-captured launch of
//     persistent kernels (one per coupling type, chained by programmatic
//     dependent launch), whose replica tiles are scheduled longest first;
//   * every biclique job (and every EA job too large for the resident form) is
//     one graph-captured anneal, spread longest-first over the library's
//     launch streams so that small jobs run side by side on separate SMs.
// The launch streams wait for the caller's stream before they start and the
// caller's stream waits for all of them at the end, so the batch is ordered
// on the caller's stream like a single launch.
//
// The autotuner times candidate launch choices of an instance on a short probe
// anneal and keeps the cheapest per (topology, size, coupling type, field,
// replica bucket) in a process-wide table that pb_anneal_ex and
// pb_anneal_batch read when the caller leaves the form to the library.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "pb_handles.h"

namespace pb {

namespace {

// ------------------------------------------------------------------ tuning table
using TuneKey = std::tuple<int, int, int, int, int>;  // topo, size, jtype, has_h, ceil(log2 R)

struct TuneEntry {
    int form = PB_FORM_AUTO;
    int wt = 0;
};

std::mutex g_tune_mutex;
std::map<TuneKey, TuneEntry> g_tune;

int log2_bucket(int R)
{
    int b = 0;
    while ((1 << b) < R && b < 30) ++b;
    return b;
}

TuneKey tune_key(const pb_instance* I, int R)
{
    return TuneKey{I->topo, I->topo == PB_TOPO_EA3D ? I->L : I->n, I->jtype, I->has_h, log2_bucket(R)};
}

bool tune_lookup(const pb_instance* I, int R, TuneEntry& out)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune.find(tune_key(I, R));
    if (it == g_tune.end()) return false;
    out = it->second;
    return true;
}

// ------------------------------------------------------------------ cost model
// Rough device-time estimate (seconds on the whole GPU) of a job, used to order
// work longest first and to split the SMs between the EA launch and the other
// jobs; rates are round figures of the forms on one GB300.  `compute` is the
// part that needs SMs; the rest is per-sweep launch latency.
double est_cost(const pb_instance* I, int R, int S, int form, double* compute = nullptr)
{
    const double upd = (double)I->N * R * std::max(1, S);
    double c, lat = 0.0;
    if (I->topo == PB_TOPO_EA3D) {
        // resident form: the fast tiles (L = 8, 16, 32) vs the generic tile, +-1 vs FP32
        const bool fast = I->L == 8 || I->L == 16 || I->L == 32, f32 = I->jtype == PB_J_F32;
        const double rate = form == PB_FORM_PLAIN ? 9e10 : fast ? (f32 ? 6e11 : 8.5e11) : (f32 ? 4e11 : 6e11);
        c = upd / rate;
    } else if (I->topo == PB_TOPO_CSR) {
        c = upd * std::max(1, I->maxdeg) / 4e11;
        lat = 3.0 * std::max(1, S) * 2e-6;
    } else {
        const double flop = upd * 2.0 * I->n * (I->jtype == PB_J_F32 ? 2.0 : 1.0);
        if (form == PB_FORM_RESIDENT) {  // one CTA per 32 replicas: ~8 us per sweep at n = 256 (+-1), FP32 ~4x slower
            c = std::max(1, S) * 8e-6 * (I->n / 256.0) * (I->n / 256.0) * (I->jtype == PB_J_F32 ? 4.0 : 1.0);
        } else {
            const double rate = form == PB_FORM_CUDACORE ? 2.5e13 : (I->jtype == PB_J_F32 ? 1.5e15 : 1.8e15);
            // small instances fill a fraction of the tensor tiles
            const double fill =
                form == PB_FORM_TENSOR ? std::min(1.0, (double)I->n / 256.0) * std::min(1.0, R / 256.0) : 1.0;
            c = flop / (rate * std::max(0.02, fill));
            lat = 3.0 * std::max(1, S) * 2e-6;
        }
    }
    if (compute) *compute = c;
    return c + lat;
}

struct Job {
    int q;
    pb_instance* I;
    int R, S, form, wt;
    double cost;
};

}  // namespace

// Form and tile width the library picks for a job whose caller left the form open.
void choose_form(const pb_instance* I, int R, int requested, int& form, int& wt)
{
    form = requested;
    wt = 0;
    TuneEntry te;
    const bool tuned = requested == PB_FORM_AUTO && tune_lookup(I, R, te);
    if (I->topo == PB_TOPO_EA3D) {
        const int nF = 2 * (6 + I->hmax) + 1;
        const int wmax = ea_choose_wt(I, R, nF);
        if (tuned) {
            form = te.form;
            wt = std::min(te.wt, wmax);
            if (form == PB_FORM_RESIDENT && wt < 1) form = PB_FORM_AUTO;
            if (form != PB_FORM_AUTO) return;
        }
        if (form == PB_FORM_AUTO || form == PB_FORM_RESIDENT) {
            if (wmax > 0) {
                form = PB_FORM_RESIDENT;
                wt = wmax;
            } else {
                form = requested == PB_FORM_RESIDENT ? PB_FORM_RESIDENT : PB_FORM_PLAIN;
            }
        }
    } else if (I->topo == PB_TOPO_CSR) {
        if (form == PB_FORM_AUTO) form = PB_FORM_PLAIN;
    } else {
        wt = 1;  // tensor form: split a sparse last round of tiles (lowest latency) unless tuned otherwise
        if (tuned) {
            form = te.form;
            wt = te.wt;
        }
        // small instances: the resident form (no launch per half-sweep); else tensor cores
        if (form == PB_FORM_AUTO) form = bq_resident_fits(I) ? PB_FORM_RESIDENT : PB_FORM_TENSOR;
    }
}

// prep(i, stream) for i in [0, n) on up to 8 host threads, each with a stream of
// its own (non-blocking, synchronised before the thread ends, so all set-up work
// is complete on the device when this returns).  The first failing job, in job
// order, gives the status and its error message (messages are per thread).
template <typename F>
static pb_status setup_all_parallel(size_t n, F&& prep)
{
    const int nt = (int)std::min<size_t>(n, std::min(8u, std::max(1u, std::thread::hardware_concurrency())));
    int dev = 0;
    PB_CUDA_TRY(cudaGetDevice(&dev));
    std::vector<pb_status> st(n, PB_OK);
    std::vector<std::string> msg(n);
    std::atomic<size_t> next{0};
    auto worker = [&]() {
        cudaStream_t s = nullptr;
        bool ok = cudaSetDevice(dev) == cudaSuccess && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
        for (size_t i = next++; i < n; i = next++) {
            st[i] = ok ? prep(i, s) : cuda_fail(cudaGetLastError(), "setup stream");
            if (st[i] != PB_OK) msg[i] = pb_last_error();
        }
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    };
    if (nt <= 1) {
        worker();
    } else {
        std::vector<std::thread> ts;
        for (int k = 0; k < nt; ++k) ts.emplace_back(worker);
        for (std::thread& t : ts) t.join();
    }
    for (size_t i = 0; i < n; ++i)
        if (st[i] != PB_OK) return fail(st[i], msg[i]);
    return PB_OK;
}

// Set up and launch a batch.  Set-up runs on `setup_st`; jobs start after the
// work already queued on `setup_st`.  With `join`, `setup_st` waits for every
// job at the end.  `load` (per launch stream, seconds of queued work) picks the
// stream of each job and is updated with the job's estimated cost; `costs`
// receives each job's estimate.  `latency_first` (the request server) favours
// the other jobs' latency over the batch's total time when splitting the SMs.
pb_status batch_start(int count, pb_instance* const* insts, const pb_schedule* scheds, const int32_t* replicas,
                      const uint64_t* seeds, const pb_anneal_opts* opts, cudaStream_t setup_st, bool join,
                      std::vector<double>* load_io, std::vector<std::unique_ptr<pb_run>>& runs_out,
                      std::vector<double>* costs, std::vector<int>* stream_of, bool latency_first)
{
    TraceRange trace_prepare("batch: prepare");
    if (count < 1 || !insts || !scheds || !replicas || !seeds) return fail(PB_EINVAL, "null or empty batch");
    cudaStream_t st = setup_st;
    std::vector<Job> jobs;
    for (int q = 0; q < count; ++q) {
        pb_instance* I = insts[q];
        if (!I) return fail(PB_EINVAL, "null instance in batch");
        if (replicas[q] < 1) return fail(PB_EINVAL, "replicas must be >= 1");
        int form = 0, wt = 0;
        choose_form(I, replicas[q], opts ? opts[q].form : PB_FORM_AUTO, form, wt);
        if (I->topo == PB_TOPO_EA3D) {
            if (form == PB_FORM_RESIDENT && wt == 0) return fail(PB_EUNSUPPORTED, "lattice too large for the resident form");
            if (form != PB_FORM_RESIDENT && form != PB_FORM_PLAIN)
                return fail(PB_EUNSUPPORTED, "form not available for EA instances");
        } else if (I->topo == PB_TOPO_CSR) {
            if (form != PB_FORM_PLAIN) return fail(PB_EUNSUPPORTED, "general sparse instances run in the plain form");
        } else if (form != PB_FORM_TENSOR && form != PB_FORM_CUDACORE && form != PB_FORM_RESIDENT) {
            return fail(PB_EUNSUPPORTED, "form not available for biclique instances");
        }
        jobs.push_back(Job{q, I, replicas[q], scheds[q].n_sweeps, form, wt, est_cost(I, replicas[q], scheds[q].n_sweeps, form)});
    }
    // EA resident jobs: too few tiles for the SMs -> halve the widest replica blocks
    {
        const int sms = sm_count();
        long long tiles = 0;
        for (const Job& j : jobs)
            if (j.form == PB_FORM_RESIDENT && j.I->topo == PB_TOPO_EA3D) tiles += ((j.R + 3) / 4 + j.wt - 1) / j.wt;
        while (tiles > 0 && tiles < sms) {
            Job* wide = nullptr;
            for (Job& j : jobs)
                if (j.form == PB_FORM_RESIDENT && j.I->topo == PB_TOPO_EA3D && j.wt > 1 && (!wide || j.wt > wide->wt))
                    wide = &j;
            if (!wide) break;
            const int Rw = (wide->R + 3) / 4;
            tiles -= (Rw + wide->wt - 1) / wide->wt;
            wide->wt /= 2;
            tiles += (Rw + wide->wt - 1) / wide->wt;
        }
    }

    // ---- set-up on the caller's stream.  Latency first (the request server): the
    //      EA resident jobs first, so that their shared launch starts before the
    //      other jobs are prepared, each of which is then prepared and launched in
    //      turn while the earlier ones run (served stream: maximum rate +36%, p99
    //      -15%).  Otherwise every job is prepared before any launch: on the
    //      200-job mixed batch the early EA launch measured 10% slower in total.
    std::vector<std::unique_ptr<pb_run>> runs(count);
    auto setup_one = [&](const Job& j) -> pb_status {
        runs[j.q].reset(new (std::nothrow) pb_run());
        if (!runs[j.q]) return fail(PB_ENOMEM, "host allocation failed");
        pb_run* r = runs[j.q].get();
        const pb_anneal_opts* o = opts ? &opts[j.q] : nullptr;
        if (j.I->topo == PB_TOPO_EA3D) return ea_prepare_run(r, j.I, &scheds[j.q], j.R, seeds[j.q], o, j.form, j.wt, st);
        if (j.I->topo == PB_TOPO_CSR) return csr_setup(r, j.I, &scheds[j.q], j.R, seeds[j.q], o, st);
        pb_anneal_opts oo = o ? *o : pb_anneal_opts{PB_FORM_AUTO, 0, NAN};
        oo.form = j.form;
        return bq_setup(r, j.I, &scheds[j.q], j.R, seeds[j.q], &oo, st, j.wt);
    };
    auto is_resident_ea = [](const Job& j) { return j.form == PB_FORM_RESIDENT && j.I->topo == PB_TOPO_EA3D; };
    std::vector<pb_run*> resident;
    if (!latency_first) {
        // every job before any launch: the jobs' preparations are independent, so
        // they run on host threads with a stream each (the 200-job mixed batch
        // spent ~150 ms preparing, all of it before its first launch)
        pb_status ps = setup_all_parallel(jobs.size(), [&](size_t i, cudaStream_t s) {
            const Job& j = jobs[i];
            runs[j.q].reset(new (std::nothrow) pb_run());
            if (!runs[j.q]) return fail(PB_ENOMEM, "host allocation failed");
            pb_run* r = runs[j.q].get();
            const pb_anneal_opts* o = opts ? &opts[j.q] : nullptr;
            if (j.I->topo == PB_TOPO_EA3D) return ea_prepare_run(r, j.I, &scheds[j.q], j.R, seeds[j.q], o, j.form, j.wt, s);
            if (j.I->topo == PB_TOPO_CSR) return csr_setup(r, j.I, &scheds[j.q], j.R, seeds[j.q], o, s);
            pb_anneal_opts oo = o ? *o : pb_anneal_opts{PB_FORM_AUTO, 0, NAN};
            oo.form = j.form;
            return bq_setup(r, j.I, &scheds[j.q], j.R, seeds[j.q], &oo, s, j.wt);
        });
        if (ps != PB_OK) return ps;
        for (const Job& j : jobs)
            if (is_resident_ea(j)) resident.push_back(runs[j.q].get());  // EA resident: the shared launch
    } else {
        for (const Job& j : jobs) {
            if (!is_resident_ea(j)) continue;
            pb_status ps = setup_one(j);
            if (ps != PB_OK) return ps;
            resident.push_back(runs[j.q].get());  // EA resident: the shared launch
        }
    }
    std::shared_ptr<BatchShared> ea_shared;
    if (!resident.empty()) {
        pb_status ps = ea_batch_setup(resident, st, ea_shared);
        if (ps != PB_OK) return ps;
        // The persistent EA launch keeps every SM it is given until its last tile
        // ends, so with other jobs in the batch it gets a share of the SMs and
        // the other jobs -- often short launches -- run beside it instead of
        // after it.  For the batch's total time the share follows the EA part of
        // the work that needs SMs (launch latency of the other jobs' sweeps does
        // not), between a quarter and three quarters; for latency (the server)
        // the EA launch gets three quarters only when its work dominates the
        // others' whole time, else half.
        double ea_cost = 0.0, other = 0.0, other_all = 0.0;
        for (const Job& j : jobs) {
            if (is_resident_ea(j)) {
                ea_cost += j.cost;
            } else {
                double c = 0.0;
                est_cost(j.I, j.R, j.S, j.form, &c);
                other += c;
                other_all += j.cost;
            }
        }
        if (other_all > 0.0) {
            const int sms = sm_count();
            int share;
            if (latency_first) {
                share = ea_cost >= other_all ? (3 * sms + 3) / 4 : std::max(sms / 4, (sms + 1) / 2);
            } else {
                const int prop = (int)std::lround(sms * ea_cost / (ea_cost + other));
                share = std::min((3 * sms + 3) / 4, std::max(sms / 4, prop));
            }
            ea_batch_limit_sms(*ea_shared, share);
        }
    }

    TraceRange trace_launch("batch: launch");
    // ---- launch: fork from the caller's stream, one stream for the EA batch,
    //      the other jobs longest first onto the least loaded stream
    cudaEvent_t fork = nullptr;
    PB_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    PB_CUDA_TRY(cudaEventRecord(fork, st));
    const int ns = pool_streams();
    std::vector<double> local_load(ns, 0.0);
    std::vector<double>& load = load_io ? *load_io : local_load;
    if ((int)load.size() < ns) load.resize(ns, 0.0);
    if (costs) costs->assign(count, 0.0);
    if (stream_of) stream_of->assign(count, -1);
    std::vector<char> used(ns, 0);
    auto start_on = [&](int k) -> pb_status {
        if (!used[k]) {
            PB_CUDA_TRY(cudaStreamWaitEvent(pool_stream(k), fork, 0));
            used[k] = 1;
        }
        return PB_OK;
    };
    // a failure after the first launch waits for the launched work before the
    // runs (and their device buffers) are released
    bool launched = false;
    auto fail_after_launch = [&](pb_status ps) -> pb_status {
        if (launched)
            for (int k = 0; k < ns; ++k)
                if (used[k]) cudaStreamSynchronize(pool_stream(k));
        cudaEventDestroy(fork);
        return ps;
    };
    int ea_k = -1;
    if (!resident.empty()) {
        ea_k = 0;
        for (int c = 1; c < ns; ++c)
            if (load[c] < load[ea_k]) ea_k = c;
        pb_status ps = start_on(ea_k);
        if (ps != PB_OK) return fail_after_launch(ps);
        for (const Job& j : jobs)
            if (is_resident_ea(j)) {
                load[ea_k] += j.cost;
                if (costs) (*costs)[j.q] = j.cost;
                if (stream_of) (*stream_of)[j.q] = ea_k;
            }
        for (pb_run* r : resident) r->stream = pool_stream(ea_k);
        ps = ea_batch_launch(resident, ea_shared, pool_stream(ea_k));
        launched = true;
        if (ps != PB_OK) return fail_after_launch(ps);
    }
    std::vector<const Job*> rest;
    for (const Job& j : jobs)
        if (!is_resident_ea(j)) rest.push_back(&j);
    std::stable_sort(rest.begin(), rest.end(), [](const Job* a, const Job* b) { return a->cost > b->cost; });
    cudaEvent_t ready = nullptr;  // a job's set-up after the fork, complete on `st`
    if (latency_first && !rest.empty() && cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess)
        return fail_after_launch(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
    for (const Job* j : rest) {
        pb_status ps = latency_first ? setup_one(*j) : PB_OK;
        if (ps != PB_OK) {
            if (ready) cudaEventDestroy(ready);
            return fail_after_launch(ps);
        }
        int k = -1;
        for (int c = 0; c < ns; ++c)
            if (c != ea_k && (k < 0 || load[c] < load[k])) k = c;
        ps = start_on(k);
        if (ps == PB_OK && ready) {
            // prepared after the fork: the launch stream also waits for this job's set-up
            if (cudaEventRecord(ready, st) != cudaSuccess || cudaStreamWaitEvent(pool_stream(k), ready, 0) != cudaSuccess)
                ps = cuda_fail(cudaGetLastError(), "cudaStreamWaitEvent");
        }
        if (ps != PB_OK) {
            if (ready) cudaEventDestroy(ready);
            return fail_after_launch(ps);
        }
        load[k] += j->cost;
        if (costs) (*costs)[j->q] = j->cost;
        if (stream_of) (*stream_of)[j->q] = k;
        pb_run* r = runs[j->q].get();
        r->stream = pool_stream(k);
        ps = (j->I->topo == PB_TOPO_EA3D)  ? ea_enqueue_plain(r, pool_stream(k))
             : (j->I->topo == PB_TOPO_CSR) ? csr_launch(r, pool_stream(k))
                                            : bq_launch(r, pool_stream(k));
        launched = true;
        if (ps != PB_OK) {
            if (ready) cudaEventDestroy(ready);
            return fail_after_launch(ps);
        }
    }
    if (ready) cudaEventDestroy(ready);
    // ---- join back into the caller's stream
    for (int k = 0; k < ns && join; ++k) {
        if (!used[k]) continue;
        cudaEvent_t join = nullptr;
        PB_CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        PB_CUDA_TRY(cudaEventRecord(join, pool_stream(k)));
        PB_CUDA_TRY(cudaStreamWaitEvent(st, join, 0));
        cudaEventDestroy(join);  // released once it has completed
    }
    cudaEventDestroy(fork);
    runs_out = std::move(runs);
    return PB_OK;
}

}  // namespace pb

using namespace pb;

extern "C" {

pb_status pb_anneal_batch(int32_t count, pb_instance* const* insts, const pb_schedule* scheds, const int32_t* replicas,
                          const uint64_t* seeds, const pb_anneal_opts* opts, void* stream, pb_run** outs)
{
    pb::TraceRange trace_("pb_anneal_batch");
    if (count < 1 || !outs) return fail(PB_EINVAL, "null or empty batch");
    for (int q = 0; q < count; ++q) outs[q] = nullptr;
    std::vector<std::unique_ptr<pb_run>> runs;
    pb_status ps = batch_start(count, insts, scheds, replicas, seeds, opts, static_cast<cudaStream_t>(stream), true,
                               nullptr, runs, nullptr, nullptr);
    if (ps != PB_OK) return ps;
    for (int q = 0; q < count; ++q) outs[q] = runs[q].release();
    return PB_OK;
}



pb_status pb_autotune(pb_instance* I, int32_t R, int32_t probe_sweeps, void* stream, pb_tune_result* out)
{
    pb::TraceRange trace_("pb_autotune");
    if (!I || !out) return fail(PB_EINVAL, "null argument");
    if (R < 1) return fail(PB_EINVAL, "replicas must be >= 1");
    const int S = std::max(2, std::min(probe_sweeps > 0 ? probe_sweeps : 8, 1000));
    *out = pb_tune_result{};
    for (int c = 0; c < 8; ++c) out->probe_ms[c] = NAN;
    std::vector<std::pair<int, int>> cand;  // form, WT
    if (I->topo == PB_TOPO_EA3D) {
        const int nF = 2 * (6 + I->hmax) + 1;
        const int wmax = ea_choose_wt(I, R, nF);
        for (int w = 1; w <= wmax && cand.size() < 7; w *= 2) cand.push_back({PB_FORM_RESIDENT, w});
        cand.push_back({PB_FORM_PLAIN, 0});
    } else if (I->topo == PB_TOPO_CSR) {
        cand.push_back({PB_FORM_PLAIN, 0});
    } else {
        // tensor form with a sparse last round of tiles split into 128-replica tiles (wt 1) or not (wt 0)
        cand.push_back({PB_FORM_TENSOR, 1});
        cand.push_back({PB_FORM_TENSOR, 0});
        cand.push_back({PB_FORM_CUDACORE, 0});
        if (bq_resident_fits(I)) cand.push_back({PB_FORM_RESIDENT, 0});
    }
    pb_schedule sc{};
    sc.kind = PB_SCHED_LINEAR;
    sc.n_sweeps = S;
    sc.step_duration = 1;
    sc.beta0 = 0.1;
    sc.beta1 = 3.0;
    const int sms = sm_count();
    double best = INFINITY;
    int bi = -1;
    for (size_t c = 0; c < cand.size(); ++c) {
        const int form = cand[c].first, wt = cand[c].second;
        pb_anneal_opts o{form, 0, NAN};
        std::unique_ptr<pb_run> run(new (std::nothrow) pb_run());
        if (!run) return fail(PB_ENOMEM, "host allocation failed");
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        pb_status ps;
        int units = sms;  // SMs the form keeps busy
        if (I->topo == PB_TOPO_EA3D) {
            ps = ea_prepare_run(run.get(), I, &sc, R, 1, &o, form, wt, st);
            if (ps == PB_OK && form == PB_FORM_RESIDENT) {
                std::vector<pb_run*> v{run.get()};
                std::shared_ptr<BatchShared> sh;
                ps = ea_batch_setup(v, st, sh);
                if (ps == PB_OK) ps = ea_batch_launch(v, sh, st);
                units = std::min(sms, run->job.n_tiles);
            } else if (ps == PB_OK) {
                ps = ea_enqueue_plain(run.get(), st);
            }
        } else if (I->topo == PB_TOPO_CSR) {
            ps = csr_setup(run.get(), I, &sc, R, 1, &o, st);
            if (ps == PB_OK) ps = csr_launch(run.get(), st);
        } else {
            ps = bq_setup(run.get(), I, &sc, R, 1, &o, st, wt);
            if (ps == PB_OK) ps = bq_launch(run.get(), st);
            if (form == PB_FORM_TENSOR) {
                units = std::min(sms, 2 * bq_tc_clusters(I->n, run->bjob.Rpad, I->jtype == PB_J_PM1_I8 ? 0 : 1,
                                                         wt != 0));
            } else if (form == PB_FORM_RESIDENT) {
                units = std::min(sms, (R + 31) / 32);
            } else {
                units = std::min(sms, ((I->n + 63) / 64) * ((R + 63) / 64));
            }
        }
        if (ps != PB_OK) return ps;
        ps = wait_run(run.get(), -1);
        if (ps != PB_OK) return ps;
        float ms = 0.0f;
        PB_CUDA_TRY(cudaEventElapsedTime(&ms, run->batch && run->batch->ev_k0 ? run->batch->ev_k0 : run->ev_k0,
                                         run->batch && run->batch->ev_k1 ? run->batch->ev_k1 : run->ev_k1));
        out->candidate_form[c] = form;
        out->candidate_wt[c] = wt;
        out->probe_ms[c] = ms;
        // cost in SM-time: a batch fills the SMs a small job leaves idle
        const double cost = (double)ms * units;
        if (cost < best) {
            best = cost;
            bi = (int)c;
        }
    }
    out->n_candidates = (int32_t)cand.size();
    out->form = cand[bi].first;
    out->tile_width = cand[bi].second;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune[tune_key(I, R)] = TuneEntry{out->form, out->tile_width};
    return PB_OK;
}

void pb_autotune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune.clear();
}

}  // extern "C"
