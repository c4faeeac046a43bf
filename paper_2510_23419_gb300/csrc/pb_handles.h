// pb_handles.h -- internal definitions of the opaque handles of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "biclique_launch.h"
#include "biclique_tc.h"
#include "csr_launch.h"
#include "ea_launch.h"
#include "pb_common.h"

#include <nvtx3/nvToolsExt.h>

namespace pb {

// A named NVTX range over a host-side phase of a call (instance build, run
// preparation, launch, readout, server admission round); NVTX-aware profilers
// show it on the timeline, without one it costs a few nanoseconds.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};


// ---------------------------------------------------------------------------
// Device memory of the handles comes from a library-owned stream-ordered pool
// (per device), allocated and freed on an internal non-blocking stream: a free
// never synchronises the device, so releasing a finished run does not wait for
// work that other runs still have in flight.  Buffers are released only when
// no launch that uses them is pending (pb_run_destroy waits for its run).
// ---------------------------------------------------------------------------
cudaError_t pool_alloc(void** p, size_t n);
void pool_free(void* p);

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf()
    {
        if (p) pool_free(p);
    }
    cudaError_t alloc(size_t n)
    {
        if (p) pool_free(p);
        p = nullptr;
        bytes = n;
        return pool_alloc(&p, n ? n : 16);
    }
    template <typename T>
    T* as() const
    {
        return static_cast<T*>(p);
    }
};

// Launch streams of batches and of the request server: a per-device set of
// non-blocking streams owned by the library.
cudaStream_t pool_stream(int k);
int pool_streams();

#define PB_ALLOC(buf, n)                                                  \
    do {                                                                  \
        cudaError_t pb_e_ = (buf).alloc(n);                               \
        if (pb_e_ != cudaSuccess) return ::pb::cuda_fail(pb_e_, "cudaMalloc"); \
    } while (0)

}  // namespace pb

struct pb_instance {
    int topo = 0, jtype = 0, L = 0, n = 0;
    int64_t N = 0;
    int has_h = 0, hmax = 0, maxdeg = 0;
    // EA
    pb::DevBuf jbits, h8, j6, hf, J3, hraw;
    pb::EaDevice ea{};
    // biclique
    pb::BqDevice bq{};
    pb::DevBuf bq_bufs[12];
    // general sparse instance
    int n_colours = 0;
    std::vector<int32_t> csr_cls_off;  // host copy of the class offsets
    std::vector<int32_t> csr_orig;     // host copy of the original index of each label
    pb::CsrDevice csr{};
    pb::DevBuf csr_bufs[12];
};

namespace pb {
// Tiles of one coupling type in a shared EA launch: work[offset, offset + n),
// the group's own counter word, one persistent kernel (EaKernel) of `grid` CTAs.
struct EaGroup {
    int kernel = 0, offset = 0, n = 0, grid = 0;
    size_t smem = 0;
    double cost = 0.0, longest = 0.0;  // estimated SM-time of all tiles / of the longest tile
};

struct BatchShared {
    DevBuf jobs, work, counter;
    int n_work = 0;
    std::vector<EaGroup> groups;  // launch order: the group holding the longest tile first
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;  // around the shared persistent launches
    std::vector<cudaEvent_t> ev_group;             // after each group's launch (joins inside the capture)
    ~BatchShared()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (ev_k0) cudaEventDestroy(ev_k0);
        if (ev_k1) cudaEventDestroy(ev_k1);
        for (cudaEvent_t e : ev_group)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace pb

struct pb_run {
    pb_instance* inst = nullptr;
    int form = 0;
    bool resumed = false;  // general graphs: state and best were given (pb_anneal_resume)
    int R = 0, S = 0;
    int64_t N = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;  // around the annealing kernels
    // EA
    pb::EaJob job{};
    // general sparse instance
    pb::CsrJob cjob{};
    // biclique
    pb::BqJob bjob{};
    pb::BqTcMaps maps{};
    int* dev_err = nullptr;  // device error word of bounded waits (null if the form has none)
    pb::DevBuf table, betaf, best_words, final_words, E_best_i, E_best_f, best_sweep, hit_sweep;
    pb::DevBuf n_hit;      // stop-at-target counters (replicas that reached the target; biclique: + sweep word)
    pb::DevBuf best_pm, final_pm, E_out;  // readout: [R][N] x2, [2R] doubles
    pb::DevBuf extra[8];
    pb::DevBuf pt[6];      // parallel tempering buffers of a general-graph run
    pb::DevBuf bq_alt[2];  // biclique: the parity-1 live spin buffers of sides A and B
    std::vector<int32_t> csr_nchunk;  // general graph: class chunks of each colour class
    int res_tab = 0;                  // biclique resident form: widest threshold window
    size_t res_smem = 0;              // biclique resident form: dynamic shared memory per CTA
    std::vector<int32_t> bq_win;  // biclique +-1: per beta level, (first index, width, offset) of its threshold window
    std::shared_ptr<pb::BatchShared> batch;
    ~pb_run()
    {
        if (ev_start) cudaEventDestroy(ev_start);
        if (ev_stop) cudaEventDestroy(ev_stop);
        if (ev_k0) cudaEventDestroy(ev_k0);
        if (ev_k1) cudaEventDestroy(ev_k1);
    }
};


namespace pb {
int sm_count();
pb_status schedule_levels(const pb_schedule* sc, std::vector<double>& betas, int& step);
uint32_t threshold_u32(double beta, double F);
pb_status bq_build(pb_instance* I, const pb_instance_desc* d, cudaStream_t st);
void threshold_windows(const std::vector<double>& betas, int nF, int fmin, std::vector<uint32_t>& tab,
                       std::vector<int32_t>& win);
// tile_split: tensor form, halve the tiles of a sparse last round (BqJob::tile_split)
pb_status bq_anneal(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                    const pb_anneal_opts* opts, cudaStream_t st, int tile_split = 1);
pb_status bq_fields(pb_instance* I, const int8_t* d_states, int R, int form, float* d_out, cudaStream_t st);
// Split forms of the anneal: set-up (allocations, tables, copies; may synchronise
// `st`) and launch (graph capture and launch on `st`, no synchronisation).
pb_status ea_prepare_run(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                         const pb_anneal_opts* opts, int form, int WT, cudaStream_t st);
pb_status ea_enqueue_plain(pb_run* run, cudaStream_t st);
pb_status ea_batch_setup(std::vector<pb_run*>& runs, cudaStream_t st, std::shared_ptr<BatchShared>& out);
pb_status ea_batch_launch(std::vector<pb_run*>& runs, const std::shared_ptr<BatchShared>& shared, cudaStream_t st);
// Keep the EA kernels of a shared launch within `sms` SMs in total (split over
// the coupling-type groups in proportion to their work).
void ea_batch_limit_sms(BatchShared& shared, int sms);
// The topology parts of pb_anneal_resume (arguments checked by the caller).
pb_status csr_anneal_resume(pb_instance* I, const pb_schedule* sched, int32_t replicas, uint64_t seed,
                            int32_t first_sweep, const int8_t* state, const int8_t* best_state, const double* best_E,
                            const int32_t* best_sweep, cudaStream_t st, pb_run** out);
int ea_choose_wt(const pb_instance* I, int R, int nF);
pb_status bq_setup(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                   const pb_anneal_opts* opts, cudaStream_t st, int tile_split = 1);
pb_status bq_launch(pb_run* run, cudaStream_t st);
bool bq_resident_fits(const pb_instance* I);
pb_status csr_build(pb_instance* I, int32_t N, int64_t n_edges, const int32_t* eu, const int32_t* ev, int jtype,
                    const void* J, const void* h, const int32_t* colour, cudaStream_t st);
pb_status csr_setup(pb_run* run, pb_instance* I, const pb_schedule* sc, int R, uint64_t seed,
                    const pb_anneal_opts* opts, cudaStream_t st);
pb_status csr_launch(pb_run* run, cudaStream_t st);
pb_status csr_fields(pb_instance* I, const int8_t* d_states, int R, float* d_out, cudaStream_t st);
pb_status wait_run(pb_run* run, int32_t timeout_ms);
// Form (and EA tile width) for a job: the caller's choice, else the autotuner's
// table entry for the job's shape, else the built-in rule.
// wt: EA resident tile width; biclique tensor form: 1 = split a sparse last round of tiles, 0 = whole tiles.
void choose_form(const pb_instance* I, int R, int requested, int& form, int& wt);
pb_status batch_start(int count, pb_instance* const* insts, const pb_schedule* scheds, const int32_t* replicas,
                      const uint64_t* seeds, const pb_anneal_opts* opts, cudaStream_t setup_st, bool join,
                      std::vector<double>* load_io, std::vector<std::unique_ptr<pb_run>>& runs_out,
                      std::vector<double>* costs, std::vector<int>* stream_of, bool latency_first = false);
}  // namespace pb
