// server.cpp -- request server with continuous batching for p-bit anneals
// (arXiv 2510.23419: independent annealing runs of the paper's instance
// families, Sec. 2 and Sec. 3, served as requests).
//
// One loop thread owns the device side.  Each pass it
//   1. admits queued requests in arrival order while the device footprint of
//      the admitted work stays within the budget and fewer than max_inflight
//      runs are on the device (a request that does not fit waits; later ones
//      wait behind it, so no request starves);
//   2. starts everything it admitted as one batch (EA jobs share a persistent
//      launch, bicliques are graph-captured anneals) on the library's launch
//      streams, choosing the streams with the least outstanding work, while
//      earlier rounds are still running: arrivals overlap with work in flight;
//   3. polls the completion events of the runs in flight, releases their
//      footprint and wakes the callers waiting for them.
// Latency is measured on the host from submit to the loop seeing the run's
// completion event.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "pb_handles.h"

namespace pb {

int64_t footprint_bytes(const pb_instance* I, const pb_schedule* sc, int R, const pb_anneal_opts* opts)
{
    if (!I || !sc || R < 1) return -1;
    std::vector<double> betas;
    int step = 1;
    if (schedule_levels(sc, betas, step) != PB_OK) return -1;
    const int64_t nlev = std::max<int64_t>(1, (int64_t)betas.size());
    int form = 0, wt = 0;
    choose_form(I, R, opts ? opts->form : PB_FORM_AUTO, form, wt);
    const int64_t N = I->N;
    const int64_t out = 2 * (int64_t)R * N + 2 * (int64_t)R * 8;  // readout states and energies
    if (I->topo == PB_TOPO_EA3D) {
        const int64_t Rw = (R + 3) / 4;
        const int64_t WT = form == PB_FORM_RESIDENT && wt > 0 ? wt : Rw;
        const int64_t tiles = (Rw + WT - 1) / WT;
        const int64_t Rpad = tiles * 4 * WT;
        const int64_t nF = 2 * (6 + I->hmax) + 1;
        return 2 * tiles * N * WT * 4 + 3 * Rpad * 4 + nlev * nF * 4 + out + 4096;
    }
    if (I->topo == PB_TOPO_CSR) {
        const int64_t Rw = (R + 3) / 4;
        const int64_t nF = 2 * (I->maxdeg + I->hmax) + 1;
        return 2 * N * Rw * 4 + (N + kCsrChunk - 1) / kCsrChunk * 4 * Rw * 8 + 4 * Rw * 20 + nlev * nF * 4 + out + 4096;
    }
    const int64_t n = I->n;
    const bool tensor = form == PB_FORM_TENSOR;
    const int64_t tile = tensor ? kBqTcReps : (form == PB_FORM_RESIDENT ? kBqResReps : kBqTileReps);
    const int64_t Rpad = (R + tile - 1) / tile * tile;
    const int64_t ld = (n + 15) / 16 * 16;
    const int64_t esz = I->jtype == PB_J_PM1_I8 ? 1 : 2;
    int64_t nblk = (n + (tensor ? kBqTcRows : kBqTileRows) - 1) / (tensor ? kBqTcRows : kBqTileRows);
    if (tensor) nblk = 4 * ((nblk + 1) & ~1LL);
    const int64_t nF = 2 * (n + I->hmax) + 1;
    return 4 * Rpad * ld * esz + 2 * nblk * Rpad * 4 + nlev * (I->jtype == PB_J_PM1_I8 ? nF : 1) * 4 + 3 * Rpad * 4 +
           (n + 63) / 64 * R * 8 + out + 4096;
}

}  // namespace pb

using namespace pb;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    pb_instance* inst = nullptr;
    pb_schedule sched{};
    std::vector<double> betas;  // copy of an explicit schedule
    int32_t R = 0;
    uint64_t seed = 0;
    pb_anneal_opts opts{PB_FORM_AUTO, 0, NAN};
    int64_t bytes = 0;
    Clock::time_point t_submit;
};

struct Flight {
    int64_t ticket;
    std::unique_ptr<pb_run> run;
    int64_t bytes;
    int stream;
    double cost;
    Clock::time_point t_submit;
};

struct Done {
    std::unique_ptr<pb_run> run;
    pb_status status = PB_OK;
    std::string error;
    double latency_ms = 0.0;
};

}  // namespace

struct pb_server {
    pb_server_opts opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work;  // loop: new requests or stop
    std::condition_variable cv_done;  // callers: a ticket finished
    std::deque<Request> queue;
    std::vector<Flight> flight;
    std::map<int64_t, Done> done;
    std::vector<double> latencies;
    std::vector<double> load;  // outstanding estimated work per launch stream
    int64_t next_ticket = 1;
    int64_t inflight_bytes = 0, peak_bytes = 0;
    int64_t submitted = 0, admitted = 0, completed = 0, failed = 0, rounds = 0;
    bool stop = false;
    cudaStream_t setup = nullptr;
    std::thread loop;

    void run_loop();
};

void pb_server::run_loop()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // ---- 1. admission
        std::vector<Request> round;
        if (!queue.empty() && opts.gather_us > 0 && flight.empty()) {
            // let a burst of arrivals gather into one round
            cv_work.wait_for(lk, std::chrono::microseconds(opts.gather_us));
        }
        int64_t bytes = inflight_bytes;
        size_t nin = flight.size();
        while (!queue.empty()) {
            const Request& q = queue.front();
            if (nin >= (size_t)opts.max_inflight || bytes + q.bytes > opts.max_device_bytes) break;
            bytes += q.bytes;
            ++nin;
            round.push_back(std::move(queue.front()));
            queue.pop_front();
        }
        // ---- 2. start the round (outside the lock: set-up synchronises the set-up stream)
        if (!round.empty()) {
            const int m = (int)round.size();
            std::vector<pb_instance*> insts(m);
            std::vector<pb_schedule> scheds(m);
            std::vector<int32_t> reps(m);
            std::vector<uint64_t> seeds(m);
            std::vector<pb_anneal_opts> os(m);
            for (int k = 0; k < m; ++k) {
                insts[k] = round[k].inst;
                scheds[k] = round[k].sched;
                if (!round[k].betas.empty()) scheds[k].betas = round[k].betas.data();
                reps[k] = round[k].R;
                seeds[k] = round[k].seed;
                os[k] = round[k].opts;
            }
            std::vector<double> load_copy = load;
            lk.unlock();
            std::vector<std::unique_ptr<pb_run>> runs;
            std::vector<double> costs;
            std::vector<int> streams;
            pb_status ps;
            {
                TraceRange trace_("server: admission round");
                ps = batch_start(m, insts.data(), scheds.data(), reps.data(), seeds.data(), os.data(), setup, false,
                                 &load_copy, runs, &costs, &streams, /*latency_first=*/true);
            }
            const std::string err = ps == PB_OK ? std::string() : std::string(pb_last_error());
            lk.lock();
            ++rounds;
            if (ps == PB_OK) {
                load = load_copy;
                for (int k = 0; k < m; ++k) {
                    inflight_bytes += round[k].bytes;
                    flight.push_back(Flight{round[k].ticket, std::move(runs[k]), round[k].bytes, streams[k], costs[k],
                                            round[k].t_submit});
                }
                admitted += m;
                peak_bytes = std::max(peak_bytes, inflight_bytes);
            } else {
                // a round that failed to start fails each of its requests
                for (int k = 0; k < m; ++k) {
                    Done d;
                    d.status = ps;
                    d.error = err;
                    done[round[k].ticket] = std::move(d);
                    ++failed;
                }
                cv_done.notify_all();
            }
        }
        // ---- 3. completions
        bool any = false;
        for (size_t k = 0; k < flight.size();) {
            const cudaError_t e = cudaEventQuery(flight[k].run->ev_stop);
            if (e == cudaErrorNotReady) {
                ++k;
                continue;
            }
            Flight f = std::move(flight[k]);
            flight.erase(flight.begin() + (long)k);
            Done d;
            d.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - f.t_submit).count();
            if (e == cudaSuccess) {
                d.status = PB_OK;
                if (f.run->dev_err) {
                    int code = 0;
                    if (cudaMemcpy(&code, f.run->dev_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && code) {
                        d.status = PB_ETIMEOUT;
                        d.error = "a device-side wait of the run timed out";
                    }
                }
            } else {
                d.status = PB_EDEVICE;
                d.error = std::string("run failed: ") + cudaGetErrorString(e);
            }
            if (d.status == PB_OK) {
                ++completed;
                latencies.push_back(d.latency_ms);
            } else {
                ++failed;
            }
            d.run = std::move(f.run);
            done[f.ticket] = std::move(d);
            inflight_bytes -= f.bytes;
            if (f.stream >= 0 && f.stream < (int)load.size()) load[f.stream] = std::max(0.0, load[f.stream] - f.cost);
            any = true;
        }
        if (any) cv_done.notify_all();
        if (stop && queue.empty() && flight.empty()) break;
        if (round.empty() && !any) {
            // nothing started or finished: sleep until a request arrives or a poll is due
            cv_work.wait_for(lk, std::chrono::microseconds(flight.empty() ? 2000 : 50));
        }
    }
}

extern "C" {

int64_t pb_run_footprint(const pb_instance* inst, const pb_schedule* sched, int32_t replicas, const pb_anneal_opts* opts)
{
    return footprint_bytes(inst, sched, replicas, opts);
}

pb_status pb_server_create(const pb_server_opts* opts, pb_server** out)
{
    if (!out) return fail(PB_EINVAL, "null argument");
    *out = nullptr;
    std::unique_ptr<pb_server> sv(new (std::nothrow) pb_server());
    if (!sv) return fail(PB_ENOMEM, "host allocation failed");
    if (opts) sv->opts = *opts;
    PB_CUDA_TRY(cudaGetDevice(&sv->device));
    if (sv->opts.max_device_bytes <= 0) {
        size_t fr = 0, tot = 0;
        PB_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        sv->opts.max_device_bytes = (int64_t)(0.8 * (double)fr);
    }
    if (sv->opts.max_inflight <= 0) sv->opts.max_inflight = 1024;
    if (sv->opts.gather_us < 0) sv->opts.gather_us = 0;
    sv->load.assign(pool_streams(), 0.0);
    PB_CUDA_TRY(cudaStreamCreateWithFlags(&sv->setup, cudaStreamNonBlocking));
    pb_server* raw = sv.get();
    try {
        sv->loop = std::thread([raw]() { raw->run_loop(); });
    } catch (...) {
        cudaStreamDestroy(sv->setup);
        return fail(PB_ENOMEM, "could not start the server thread");
    }
    *out = sv.release();
    return PB_OK;
}

pb_status pb_server_submit(pb_server* sv, pb_instance* inst, const pb_schedule* sched, int32_t replicas, uint64_t seed,
                           const pb_anneal_opts* opts, int64_t* ticket)
{
    if (!sv || !inst || !sched || !ticket) return fail(PB_EINVAL, "null argument");
    if (replicas < 1) return fail(PB_EINVAL, "replicas must be >= 1");
    Request r;
    r.inst = inst;
    r.sched = *sched;
    if (sched->kind == PB_SCHED_EXPLICIT && sched->n_sweeps > 0) {
        if (!sched->betas) return fail(PB_EINVAL, "explicit schedule without betas");
        r.betas.assign(sched->betas, sched->betas + sched->n_sweeps);
    }
    r.R = replicas;
    r.seed = seed;
    if (opts) r.opts = *opts;
    r.bytes = footprint_bytes(inst, sched, replicas, opts);
    if (r.bytes < 0) return fail(PB_EINVAL, "invalid request");
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->stop) return fail(PB_EBUSY, "server is stopping");
    if (r.bytes > sv->opts.max_device_bytes) return fail(PB_EINVAL, "request larger than the server's device budget");
    r.ticket = sv->next_ticket++;
    r.t_submit = Clock::now();
    *ticket = r.ticket;
    sv->queue.push_back(std::move(r));
    ++sv->submitted;
    sv->cv_work.notify_one();
    return PB_OK;
}

pb_status pb_server_wait(pb_server* sv, int64_t ticket, int32_t timeout_ms, pb_run** run, double* latency_ms)
{
    if (!sv || !run) return fail(PB_EINVAL, "null argument");
    *run = nullptr;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (ticket < 1 || ticket >= sv->next_ticket) return fail(PB_EINVAL, "unknown ticket");
    auto ready = [&]() { return sv->done.count(ticket) > 0; };
    if (timeout_ms < 0) {
        sv->cv_done.wait(lk, ready);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        return fail(PB_ETIMEOUT, "ticket not finished within the timeout");
    }
    Done d = std::move(sv->done[ticket]);
    sv->done.erase(ticket);
    if (latency_ms) *latency_ms = d.latency_ms;
    if (d.status != PB_OK) return fail(d.status, d.error);
    *run = d.run.release();
    return PB_OK;
}

pb_status pb_server_stats_get(pb_server* sv, pb_server_stats* out)
{
    if (!sv || !out) return fail(PB_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    pb_server_stats s{};
    s.submitted = sv->submitted;
    s.admitted = sv->admitted;
    s.completed = sv->completed;
    s.failed = sv->failed;
    s.queued = (int64_t)sv->queue.size();
    s.inflight = (int64_t)sv->flight.size();
    s.inflight_bytes = sv->inflight_bytes;
    s.peak_inflight_bytes = sv->peak_bytes;
    s.rounds = sv->rounds;
    if (!sv->latencies.empty()) {
        std::vector<double> v = sv->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            // nearest rank
            const size_t k = (size_t)std::ceil(p * (double)v.size());
            return v[std::min(v.size() - 1, k == 0 ? 0 : k - 1)];
        };
        s.p50_ms = pct(0.50);
        s.p99_ms = pct(0.99);
        double sum = 0.0;
        for (double x : v) sum += x;
        s.mean_ms = sum / (double)v.size();
        s.max_ms = v.back();
    }
    *out = s;
    return PB_OK;
}

void pb_server_destroy(pb_server* sv)
{
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        sv->cv_work.notify_all();
    }
    if (sv->loop.joinable()) sv->loop.join();
    for (auto& kv : sv->done)
        if (kv.second.run) pb_run_destroy(kv.second.run.release());
    if (sv->setup) cudaStreamDestroy(sv->setup);
    delete sv;
}

}  // extern "C"
