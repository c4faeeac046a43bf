/*
 * pbit.h -- C ABI of the GB300 (sm_103a) graph-coloured parallel p-bit annealer.
 *
 * Method: "Probabilistic Computing Optimization of Complex Spin-Glass
 * Topologies" (arXiv 2510.23419).  For every colour class (update group,
 * Sec. 1.2.2) in turn, every p-bit i of the class takes the local field
 * F_i = sum_j J_ij m_j + h_i (Eq. 3) and sets m_i = +1 with probability
 * 1/2 + tanh(beta F_i)/2 (Eq. 2, bipolar form), under a beta schedule
 * (classical annealing, Sec. 1.3.1), for many independent replicas.
 *
 * Conventions that hold for every call:
 *  - Energy (Eq. 1 with the sign that Eqs. 2-3 sample):
 *      E(m) = - sum_{edges (i,j)} J_ij m_i m_j - sum_i h_i m_i.
 *    A coupling J > 0 favours aligned spins.  (The paper writes
 *    H = +sum J s s; its J is the negative of the J here.)
 *  - Decision rule: one uint32 word r per update;
 *      T = min(floor((0.5 + 0.5*tanh(beta*F)) * 2^32), 2^32 - 1) in FP64,
 *      m = +1 iff r < T.
 *    For +-1 couplings with integer fields T comes from a table built in FP64
 *    on the host, so results are bit-exact and reproducible.  For FP32
 *    couplings the kernels evaluate T in FP32 (see the per-call notes).
 *  - Random words: Philox4x32-10 (Salmon et al., SC'11), key = (seed lo,
 *    seed hi), counter = (k, s, r >> 2, (tag << 24) | c), word r & 3, where k
 *    is the rank of spin i inside its colour class c, s the sweep, r the
 *    replica; tag 0 = decisions, 1 = initial state (s = 0), 2 = instance
 *    generation.
 *  - Initial state: m_i = +1 iff the tag-1 word < 2^31.
 *  - One sweep updates colour 0, then colour 1.  After every sweep the energy
 *    is evaluated; the best (running lowest, Fig. 1A) state starts as the
 *    initial state with best sweep -1 and is replaced when E < best strictly.
 *  - Host arrays are read during the call and not kept.  Device memory is
 *    owned by the handles.  Output buffers are caller-owned host memory with
 *    an explicit size; a size that is too small gives PB_EINVAL.
 *  - Streams cross as void* (a cudaStream_t; NULL = the legacy default stream).
 *  - No C++ exception crosses this interface.  Every failing call returns a
 *    status and leaves a message for pb_last_error() (thread-local).
 *  - Lattice site index: i = x + L*(y + L*z); EA colour = (x + y + z) & 1
 *    (needs an even L).  Biclique: left spins 0..n-1 (colour 0), right spins
 *    n..2n-1 (colour 1).
 */
#ifndef PBIT_H
#define PBIT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pb_status {
    PB_OK = 0,
    PB_EINVAL = 1,        /* bad argument: null pointer, size, type or value out of range */
    PB_ECOLOUR = 2,       /* colouring has an edge inside a class, or the checkerboard needs an even L */
    PB_ENOMEM = 3,        /* host or device allocation failed */
    PB_EDEVICE = 4,       /* a CUDA call failed; pb_last_error() has the CUDA message */
    PB_ETIMEOUT = 5,      /* a wait ran out of time */
    PB_EBUSY = 6,         /* pb_query: the run has not finished */
    PB_EUNSUPPORTED = 7   /* valid request outside what this library implements */
} pb_status;

typedef enum pb_topology { PB_TOPO_EA3D = 0, PB_TOPO_BICLIQUE = 1, PB_TOPO_CSR = 2 } pb_topology;

/* Coupling storage of an instance.
 * PB_J_PM1_I8: int8 couplings in {-1, +1}; h (if any) int8, |h| <= 64.  Fields are
 *              integers and decisions use the FP64-built threshold table (bit-exact).
 * PB_J_F32:    float couplings and float h; fields in FP32 (EA) or tensor-core
 *              split-BF16 with FP32 accumulation (biclique). */
typedef enum pb_jtype { PB_J_PM1_I8 = 0, PB_J_F32 = 1 } pb_jtype;

/* Coupling laws of the seeded generators (Sec. 2 random cubes, Sec. 3 random
 * bicliques with couplings from [-1, 1]). */
typedef enum pb_dist { PB_DIST_PM1 = 0, PB_DIST_GAUSS = 1, PB_DIST_UNIF = 2 } pb_dist;

typedef struct pb_instance_desc {
    int32_t topo;          /* pb_topology */
    int32_t L;             /* EA: side of the periodic cube (even, 2..64); N = L^3 */
    int32_t n;             /* biclique: spins per side (1..16384); N = 2n */
    int32_t jtype;         /* pb_jtype */
    const void* J;         /* host.  EA: [3][N], bond (d, i) joins site i to its +x (d=0), +y (1), +z (2)
                              neighbour.  Biclique: [n][n] row-major, J[i][j] joins left i to right j.
                              int8 for PB_J_PM1_I8, float for PB_J_F32 */
    const void* h;         /* host [N], int8 (PM1) or float (F32); NULL = no field */
    const int32_t* colour; /* host [N]; NULL = canonical colouring.  A given colouring is
                              checked: an internal edge gives PB_ECOLOUR; a proper colouring
                              other than the canonical one gives PB_EUNSUPPORTED */
} pb_instance_desc;

typedef enum pb_sched_kind { PB_SCHED_LINEAR = 0, PB_SCHED_GEOMETRIC = 1, PB_SCHED_EXPLICIT = 2 } pb_sched_kind;

/* Classical annealing schedule (Sec. 1.3.1; Algorithm 1's linear beta step).
 * Level l = floor(s / d) of Lv = ceil(S / d) levels, end points included:
 *   linear    beta0 + (beta1 - beta0) * l / (Lv - 1)
 *   geometric beta0 * (beta1 / beta0)^(l / (Lv - 1))      (beta0, beta1 > 0)
 *   explicit  betas[s], one per sweep (host array of n_sweeps values)
 * A single level uses beta0.  All betas must be finite and >= 0. */
typedef struct pb_schedule {
    int32_t kind;          /* pb_sched_kind */
    int32_t n_sweeps;      /* S >= 0 */
    int32_t step_duration; /* d >= 1 */
    int32_t reserved;      /* 0 */
    double beta0;
    double beta1;
    const double* betas;   /* explicit only */
} pb_schedule;

/* How a run executes. */
typedef enum pb_form {
    PB_FORM_AUTO = 0,      /* the autotuner's choice for the shape if it has one; else: EA resident where it fits,
                              else plain; biclique resident where it fits, else tensor */
    PB_FORM_PLAIN = 1,     /* EA: spins in global memory, one launch per colour class and sweep */
    PB_FORM_RESIDENT = 2,  /* EA: persistent kernels, each replica block's lattice kept in shared memory;
                              biclique (n <= 256 for +-1, n <= 128 for F32): one CTA per 32 replicas runs the
                              whole anneal with J, J^T and both sides' spins in shared memory */
    PB_FORM_CUDACORE = 3,  /* biclique: CUDA-core field (FP32 FMA; exact integers for +-1) */
    PB_FORM_TENSOR = 4     /* biclique: tcgen05 tensor-core field (e4m3 for +-1, split BF16 for F32) */
} pb_form;

/* pb_anneal_opts.flags.  PB_FLAG_TEST_EXPIRE_WAITS is a test hook for the
 * failure path of the device-side waits (no counterpart in the paper): with it
 * the tensor form's load warp issues no loads, so the MMA issuer's and the
 * epilogue's waits for operands and accumulators run out after 2 ms (instead
 * of the normal 1 s limit); the kernels record an error word, skip their
 * writes, release their tensor memory and end, and pb_wait / pb_energy report
 * PB_ETIMEOUT.  The CUDA context stays usable.  Other forms have no device
 * waits and ignore the flag. */
#define PB_FLAG_TEST_EXPIRE_WAITS 0x40000000

/* pb_anneal_opts.flags: stop at the target (the quality criterion of Sec. 1.3.1 /
 * Fig. 1: a run is done once it reaches a given fraction of the ground-state
 * energy).  With a finite target_energy, each replica's running best stops
 * changing at the first sweep whose energy is <= target (its best energy, state
 * and sweep are then those of that sweep, the recorded target sweep), and the
 * run ends early once every replica has reached the target; otherwise after all
 * sweeps (forms that launch per sweep still issue their remaining launches, which
 * return at once).  The best results of a replica depend only on its own trajectory, so
 * they are the same in every form, alone or in a batch.  The final state and
 * energy are those of the sweep at which the replica's block of the run stopped,
 * which depends on the form. */
#define PB_FLAG_STOP_AT_TARGET 0x1

typedef struct pb_anneal_opts {
    int32_t form;          /* pb_form */
    int32_t flags;         /* 0, PB_FLAG_STOP_AT_TARGET, or PB_FLAG_TEST_EXPIRE_WAITS (failure-path tests only) */
    double target_energy;  /* record, per replica, the first sweep whose energy is <= target;
                              NaN disables the record */
} pb_anneal_opts;

typedef struct pb_instance pb_instance;  /* opaque: device copy of one instance */
typedef struct pb_run pb_run;            /* opaque: one anneal of R replicas of one instance */

/* Library version string and the text of a status. */
const char* pb_version(void);
const char* pb_status_string(pb_status status);
/* Message of the last failing call on this thread ("" if none). */
const char* pb_last_error(void);

/* Seeded instance generators (tag-2 Philox stream; Sec. 2 and Sec. 3).
 * Coupling e (EA: e = d*N + i; biclique: e = i*n + j) is
 *   PM1:   +1 iff word(e >> 2, 0, 0, 2 << 24)[e & 3] < 2^31, else -1   (int8 output)
 *   GAUSS: Box-Muller on words 0, 1 of (e, 1, 0, 2 << 24), u = (w + 0.5) / 2^32,
 *          z = sqrt(-2 ln u0) cos(2 pi u1) in FP64, rounded to float   (float output)
 *   UNIF:  2u - 1 with u = (word(e >> 2, 2, 0, 2 << 24)[e & 3] + 0.5) / 2^32, rounded to float
 * J_out is caller-owned host memory of out_bytes bytes (EA: 3 L^3 elements,
 * biclique: n^2 elements).  Errors: PB_EINVAL on a bad size or law. */
pb_status pb_generate_ea(int32_t L, int32_t dist, uint64_t seed, void* J_out, int64_t out_bytes);
pb_status pb_generate_biclique(int32_t n, int32_t dist, uint64_t seed, void* J_out, int64_t out_bytes);

/* Copy an instance to the device (Eq. 1 problem statement; the colouring of
 * Sec. 1.2.2 is validated).  Host arrays are copied before the call returns;
 * the work is ordered on `stream`.  Errors: PB_EINVAL (shape, type, +-1 check,
 * |h| range), PB_ECOLOUR (odd L, improper colouring), PB_EUNSUPPORTED, PB_ENOMEM,
 * PB_EDEVICE. */
pb_status pb_create_instance(const pb_instance_desc* desc, void* stream, pb_instance** out);
void pb_instance_destroy(pb_instance* inst);
/* Number of spins N of an instance (EA L^3, biclique 2n), or -1. */
int64_t pb_instance_spins(const pb_instance* inst);

/* General sparse instance (Eq. 1 on an arbitrary edge set): N spins, each
 * undirected edge (eu[e], ev[e]) listed once with coupling J[e] (int8 +-1 or
 * float; repeated pairs are separate edges), fields h ([N] or NULL).  The
 * update groups (Sec. 1.2.2) are the classes of `colour` ([N], values 0..254,
 * no edge inside a class: else PB_ECOLOUR) or, when colour is NULL, of the
 * greedy colouring below; classes are updated in increasing colour order and a
 * spin's Philox counter word 0 is its rank in its class (ascending index).
 * Runs use the plain form (one launch per class and sweep).  Errors: PB_EINVAL
 * (edge out of range, self-loop, PM1 value not +-1, |h| > 64), PB_ECOLOUR. */
typedef struct pb_graph_desc {
    int32_t N;
    int32_t jtype;         /* pb_jtype */
    int64_t n_edges;
    const int32_t* eu;     /* [n_edges] */
    const int32_t* ev;     /* [n_edges] */
    const void* J;         /* [n_edges] int8 or float */
    const void* h;         /* [N] int8 or float, NULL = 0 */
    const int32_t* colour; /* [N] or NULL = greedy colouring */
} pb_graph_desc;
pb_status pb_create_graph_instance(const pb_graph_desc* desc, void* stream, pb_instance** out);
/* Greedy colouring (host only, no device use): vertices by decreasing degree,
 * ties by index, each takes the smallest colour unused by its coloured
 * neighbours.  Writes colour_out[N]; returns the number of colours, or -1 on
 * invalid arguments (edge out of range, self-loop). */
int32_t pb_greedy_colouring(int32_t N, int64_t n_edges, const int32_t* eu, const int32_t* ev, int32_t* colour_out);
/* Number of colour classes of an instance (2 for EA and biclique), or -1. */
int32_t pb_instance_colours(const pb_instance* inst);

/* Resume an anneal of an EA cube or a general sparse instance (checkpoint / resume; no
 * counterpart in the paper, which runs each anneal start to end).  `sched` is
 * the FULL schedule; sweeps first_sweep .. n_sweeps-1 run, from `state`, the
 * replicas' spins after sweeps 0 .. first_sweep-1, with the running best
 * (`best_state`, `best_E`, `best_sweep`, the sweep of the best or -1 for the
 * initial state) carried over.  Arrays are caller-owned host memory, copied
 * before the call returns: state and best_state [replicas][N] int8 +1/-1,
 * best_E [replicas] (the energies pb_energy reported), best_sweep [replicas].
 * The decisions use the absolute sweep index in their Philox counters (Sec.
 * 1.2.2 update groups, Eq. 2), so for +-1 couplings a run of n_sweeps equals,
 * bit for bit, a run of the first first_sweep sweeps (an explicit schedule of
 * those betas) resumed here with that run's final state and best (real
 * couplings: the carried best energy is the FP64 recomputation, where an
 * uninterrupted run compares with its running FP32 energies, so a near-tie can
 * resolve differently).  The target-energy record restarts at first_sweep.
 * The anneal runs asynchronously on `stream` like pb_anneal.  PB_EINVAL:
 * first_sweep outside [0, n_sweeps], a best_sweep outside [-1, first_sweep),
 * a state value other than +-1, a non-integer best energy of a +-1 instance;
 * PB_EUNSUPPORTED: a biclique instance (resume it through its edge list with
 * pb_create_graph_instance) or an EA cube too large for the resident form,
 * which EA resumes use. */
pb_status pb_anneal_resume(pb_instance* inst, const pb_schedule* sched, int32_t replicas, uint64_t seed,
                           int32_t first_sweep, const int8_t* state, const int8_t* best_state, const double* best_E,
                           const int32_t* best_sweep, void* stream, pb_run** out);

/* Parallel tempering (replica exchange, Hukushima & Nemoto 1996; Sec. 6.1 names
 * it as a PC solving method) on a general sparse instance: M inverse
 * temperatures ladder[0] < ... < ladder[M-1] and `chains` independent chains
 * give M * chains slots; slot g = k * chains + r starts at temperature k with
 * its own random stream (replica index g).  Every sweep each slot updates all
 * colour classes at its temperature's beta; then, in every chain, the slots
 * holding temperatures t and t + 1 (t = sweep mod 2, t + 2, ...) exchange
 * temperatures with probability min(1, exp((beta_{t+1} - beta_t)(E_b - E_a))),
 * decided by the Philox word of counter (t, sweep, r >> 2, 3 << 24), index
 * r & 3, against floor(exp(.) 2^32) (FP64 table for +-1 instances: bit-exact).
 * The run's replicas are the slots: pb_energy / pb_best_states etc. return
 * M * chains entries; pb_pt_state gives each slot's final temperature and the
 * accepted exchanges per pair.  Errors: PB_EUNSUPPORTED (not a graph instance),
 * PB_EINVAL (ladder not increasing, M > 255, spacing below ~5e-6 for +-1). */
pb_status pb_anneal_pt(pb_instance* inst, const double* ladder, int32_t M, int32_t n_sweeps, int32_t chains,
                       uint64_t seed, void* stream, pb_run** out);
pb_status pb_pt_state(pb_run* run, int32_t* slot_temp, int64_t* n_accept);

/* Start an anneal of `replicas` independent replicas (Sec. 1.3.1) on `stream`.
 * Asynchronous: returns once the work is queued.  `opts` may be NULL (AUTO form,
 * no target).  The instance must outlive the run.  Errors: PB_EINVAL (schedule,
 * replicas < 1), PB_EUNSUPPORTED (form not available for the instance),
 * PB_ENOMEM, PB_EDEVICE. */
pb_status pb_anneal(pb_instance* inst, const pb_schedule* sched, int32_t replicas, uint64_t seed,
                    void* stream, pb_run** out);
pb_status pb_anneal_ex(pb_instance* inst, const pb_schedule* sched, int32_t replicas, uint64_t seed,
                       const pb_anneal_opts* opts, void* stream, pb_run** out);

/* Start `count` independent anneals of any topology as one batch, ordered on
 * `stream` like a single launch (the batch starts after the work queued on
 * `stream`, and `stream` waits for all of it).  All EA jobs that fit the
 * resident form share ONE graph-captured launch of persistent kernels (one per
 * coupling type, the second a programmatic dependent of the first) whose
 * replica blocks are scheduled longest first over all SMs; every biclique job, and EA
 * jobs too large for the resident form, run as one graph-captured anneal each,
 * spread longest first over the library's launch streams so that small jobs
 * run side by side.  Forms left at PB_FORM_AUTO come from the autotuner's
 * table (pb_autotune) when it has an entry for the job's shape.  Arrays have
 * `count` entries; `opts` may be NULL; outs[k] receives the run of job k.
 * Results are identical to running each job alone.  Errors as pb_anneal; on
 * error no run is returned. */
pb_status pb_anneal_batch(int32_t count, pb_instance* const* insts, const pb_schedule* scheds,
                          const int32_t* replicas, const uint64_t* seeds, const pb_anneal_opts* opts,
                          void* stream, pb_run** outs);

/* Sparsified biclique (host only; Sec. 5.3 outlook, construction of this
 * library): vertex v of K_{n,n} (left i = v, right j = v - n) becomes a path of
 * copies joined by ferromagnetic copy edges of strength copy_strength (for
 * PB_J_PM1_I8 as that many unit edges); biclique edge (i, j) of parity
 * (i + j) mod 2 joins a copy of i and a copy of j of that slot, each copy
 * carrying at most per_copy (1..4) edges, so no copy has more than
 * per_copy + 2 <= 6 neighbours.  colour[] is a proper 2-colouring (left copy:
 * slot, right copy: 1 - slot) and copy_of[] maps each copy to v.  J is the
 * biclique's [n][n] row-major coupling matrix.  With null output arrays only
 * *N_out is set and the number of edges returned (size query); otherwise fills
 * eu, ev, J_out (int8 or float), colour, copy_of and returns the number of
 * edges, or -1 on invalid arguments or too small capacities.  When all copies
 * of every vertex agree with a biclique state m, the copy graph's energy is
 * E(m) - copy_strength * (N_out - 2n). */
int64_t pb_sparsify_biclique(int32_t n, int32_t jtype, const void* J, int32_t per_copy, int32_t copy_strength,
                             int32_t* N_out, int32_t* eu, int32_t* ev, void* J_out, int32_t* colour,
                             int32_t* copy_of, int64_t edge_capacity, int32_t vertex_capacity);
/* Projection of copy-graph states [R][N_sparse] onto the original vertices
 * [R][n_orig]: the majority of each vertex's copies (a tie takes copy 0).
 * Host only; returns 0, or -1 on invalid arguments. */
int32_t pb_sparse_project(int32_t N_sparse, const int32_t* copy_of, int32_t n_orig, int32_t R, const int8_t* states,
                          int8_t* out);

/* Benchmarking protocol (Sec. 4.1.3, Algorithm 1): the smallest iteration
 * budget i in i_start, i_start + i_step, ... (<= i_max) at which `trials`
 * independent anneals, each of i iterations (one iteration = one colour-class
 * step, so ceil(i / k) sweeps for k classes) with beta linear from beta_i to
 * beta_f, have at most round(trials (1 - p_succ)) fails, a fail being a best
 * energy above theta = p * ground (ground < 0).  The trials of budget i are the
 * replicas of one anneal seeded seed + i; `budgets_per_launch` budgets (0 = 8)
 * run as one pb_anneal_batch.  Returns the same i as the paper's sequential loop
 * with early exit for the same trial outcomes; i_min = -1 if none passes.
 * Synchronous. */
typedef struct pb_imin_opts {
    double ground;
    double p;
    double p_succ;
    int32_t i_start, i_step, i_max;  /* i_max = 0: i_start + 1000 i_step */
    int32_t trials;
    double beta_i, beta_f;
    int32_t budgets_per_launch;
    int32_t form;                    /* pb_form of the anneals */
    uint64_t seed;
} pb_imin_opts;
typedef struct pb_imin_result {
    int32_t i_min;          /* -1: no budget passed */
    int32_t fails;          /* fails at i_min */
    int32_t budgets_tried;  /* budgets whose verdict was read, in order */
    int32_t launches;       /* batched launches */
} pb_imin_result;
pb_status pb_find_imin(pb_instance* inst, const pb_imin_opts* opts, void* stream, pb_imin_result* out);

/* Autotuner.  Times each candidate launch choice for `inst` with `replicas`
 * replicas on a short probe anneal of `probe_sweeps` sweeps (linear beta
 * 0.1 -> 3.0) on `stream`: EA resident form with every valid tile width (replica
 * words per tile) and the plain form; biclique tensor form with whole tiles and
 * with a sparse last round split into half-width tiles, the CUDA-core form and,
 * where it fits, the resident form.  The
 * cost of a candidate is its sweep-loop time times the SMs it keeps busy (a
 * batch fills the SMs that a small job leaves idle); the cheapest is returned
 * and stored in a process-wide table keyed by (topology, L or n, coupling type,
 * field present, ceil(log2 replicas)), which PB_FORM_AUTO jobs of pb_anneal_ex
 * and pb_anneal_batch then use.  Synchronous. */
typedef struct pb_tune_result {
    int32_t form;              /* chosen pb_form */
    int32_t tile_width;        /* EA resident: replica words (4 replicas each) per tile; biclique tensor
                                  form: 1 = a sparse last round of 256-replica tiles is split into
                                  128-replica tiles (shorter latency, more SM-time), 0 = whole tiles;
                                  else 0 */
    int32_t n_candidates;
    int32_t candidate_form[8];
    int32_t candidate_wt[8];
    float probe_ms[8];         /* sweep-loop time of each candidate */
} pb_tune_result;
pb_status pb_autotune(pb_instance* inst, int32_t replicas, int32_t probe_sweeps, void* stream, pb_tune_result* out);
/* Forget every autotuner entry. */
void pb_autotune_clear(void);

/* Device bytes that a run of `inst` with these arguments holds (state, best
 * states, tables, readout buffers), as used by the request server's admission.
 * Returns -1 on invalid arguments. */
int64_t pb_run_footprint(const pb_instance* inst, const pb_schedule* sched, int32_t replicas, const pb_anneal_opts* opts);

/* Request server with continuous batching.  A loop thread admits submitted
 * anneals in arrival order while their device footprint fits the budget and
 * fewer than max_inflight are on the device; every admission round is one
 * batch (pb_anneal_batch semantics, no join), started on the library's launch
 * streams while earlier rounds are still running, so arrivals overlap with work
 * in flight.  Run state stays on the device until the caller takes the run.
 * Results are the same as the same anneal run alone. */
typedef struct pb_server pb_server;
typedef struct pb_server_opts {
    int64_t max_device_bytes;  /* admission budget; 0 = 80% of the device memory free at creation */
    int32_t max_inflight;      /* 0 = 1024 */
    int32_t gather_us;         /* a round waits this long for more arrivals after the first (0 = none) */
} pb_server_opts;
typedef struct pb_server_stats {
    int64_t submitted, admitted, completed, failed, queued, inflight;
    int64_t inflight_bytes, peak_inflight_bytes, rounds;
    double p50_ms, p99_ms, mean_ms, max_ms;  /* latency from submit to result ready, completed jobs */
} pb_server_stats;
pb_status pb_server_create(const pb_server_opts* opts, pb_server** out);
/* Queue an anneal; the instance (and an explicit schedule's betas) must stay
 * valid until the ticket is waited for.  PB_EINVAL if the job alone exceeds the
 * budget. */
pb_status pb_server_submit(pb_server* sv, pb_instance* inst, const pb_schedule* sched, int32_t replicas,
                           uint64_t seed, const pb_anneal_opts* opts, int64_t* ticket);
/* Wait for a ticket: PB_OK and the finished run (owned by the caller, destroy
 * with pb_run_destroy) and its latency in ms; PB_ETIMEOUT after timeout_ms
 * (< 0 = no limit); the run's own error if it failed.  A ticket is waited for once. */
pb_status pb_server_wait(pb_server* sv, int64_t ticket, int32_t timeout_ms, pb_run** run, double* latency_ms);
pb_status pb_server_stats_get(pb_server* sv, pb_server_stats* out);
/* Stop admitting, wait for the work on the device, destroy unclaimed runs. */
void pb_server_destroy(pb_server* sv);

/* Wait for a run (host side): PB_OK when finished, PB_ETIMEOUT after timeout_ms
 * (< 0 = no limit), PB_EDEVICE if a kernel of the run failed. */
pb_status pb_wait(pb_run* run, int32_t timeout_ms);
/* PB_OK if finished, PB_EBUSY if not, PB_EDEVICE on a device error. */
pb_status pb_query(pb_run* run);

/* Results (each waits for the run).  Energies are recomputed from the returned
 * states on the device: exactly in int64 for PM1 instances, in FP64 for F32
 * instances.  Arrays have `replicas` entries; any pointer may be NULL.
 * best_sweep is -1 when the initial state was never beaten. */
pb_status pb_energy(pb_run* run, double* final_E, double* best_E, int32_t* best_sweep);
/* Best / final states, [replicas][N] int8 in {-1, +1}, out_bytes >= replicas * N. */
pb_status pb_best_states(pb_run* run, int8_t* out, int64_t out_bytes);
pb_status pb_final_states(pb_run* run, int8_t* out, int64_t out_bytes);
/* First sweep whose energy reached opts->target_energy, per replica (-1 = never,
 * or no target was set).  For F32 instances the comparison uses the kernel's
 * FP32 running energy. */
pb_status pb_target_sweeps(pb_run* run, int32_t* first_sweep);
/* Device time of the run's kernels in milliseconds (CUDA events around the launches). */
pb_status pb_run_device_ms(pb_run* run, float* ms);
/* Device time of the run's annealing kernels alone (without set-up and readout), from
 * CUDA events recorded on the run's stream around them; for a batch, the persistent
 * launch shared by all jobs. */
pb_status pb_run_kernel_ms(pb_run* run, float* ms);
void pb_run_destroy(pb_run* run);

/* Measurement helper (no counterpart in the paper; it bounds the decision step of
 * Eq. 2): the random-word ceiling of the EA update.  Runs a kernel that draws exactly
 * the decision words an L = 32 resident tile draws (Philox4x32-10, the same counter
 * layout, one 32-bit word per p-bit update) and does nothing else, on `blocks` CTAs of
 * 1024 threads (0 = one per SM) for `sweeps` sweeps; blocks until done.  Outputs: ms,
 * the kernel's duration (CUDA events on `stream`), and updates, the number of p-bit
 * updates whose words it drew (blocks * 1024 * 128 * sweeps).  Errors: PB_EINVAL
 * (null output, sweeps < 1), PB_EDEVICE. */
pb_status pb_philox_ceiling(int32_t sweeps, int32_t blocks, void* stream, float* ms, double* updates);

/* Local fields F_i = sum_j J_ij m_j + h_i (Eq. 3) of given states, computed on the
 * device with the same arithmetic the anneal kernels use for this instance
 * (integer for PM1; FP32 for EA F32).  states: host [R][N] int8 in {-1, +1};
 * fields_out: host [R][N] float, out_bytes >= 4 R N.  Synchronous. */
pb_status pb_fields(pb_instance* inst, const int8_t* states, int32_t R, float* fields_out, int64_t out_bytes,
                    void* stream);
/* pb_fields with the arithmetic of a given form (pb_form; AUTO = the form pb_anneal picks).
 * Biclique: PB_FORM_TENSOR (tensor-core e4m3, or split-BF16 products with FP32 accumulation)
 * or PB_FORM_CUDACORE (FP32 FMA).  Errors as pb_fields, PB_EUNSUPPORTED for a form the
 * instance has no kernel for. */
pb_status pb_fields_ex(pb_instance* inst, const int8_t* states, int32_t R, int32_t form, float* fields_out,
                       int64_t out_bytes, void* stream);

/* EA +-1 anneal that allocates no memory (no counterpart in the paper: it is a
 * deployment convenience).  For callers that cannot call cudaMalloc -- code that
 * runs inside a device-memory arena or pool it does not own, or in a loop where an
 * allocation and the synchronisation it can cause are not allowed.  It runs the
 * same resident kernel as pb_anneal (results are identical to pb_anneal with the
 * same arguments) but keeps every scratch buffer in one file-scope device array
 * of 16 MiB, which each GPU holds until the process exits once the library's
 * module holding it is loaded there.  CUDA may load modules lazily, so the first
 * call on a device may be the one that loads the module and reserves the 16 MiB;
 * callers that must not allocate later make one small warm-up call on each device
 * first (outside their arena or real-time loop).  The first call on a device also
 * looks up the array's device address (cudaGetSymbolAddress).
 * Inputs and outputs are caller-owned DEVICE buffers:
 *   J_dev            [3][L^3] int8 +-1 couplings (same layout as pb_instance_desc.J), h = 0
 *   best_E_dev, final_E_dev     [replicas] double (exact int energies)
 *   best_sweep_dev   [replicas] int32
 *   best_states_dev, final_states_dev  [replicas][L^3] int8 +-1
 * The schedule is read from host memory during the call.  L must be even
 * (else PB_ECOLOUR) and in [2, 32] (else PB_EINVAL).  A request whose scratch
 * (about 2 * replicas * L^3 bytes plus the threshold table of 52 bytes per beta
 * level) exceeds 16 MiB is rejected with PB_EINVAL.  The call does not wait for
 * earlier work on `stream`: it stages its small host-side descriptors and table
 * (cudaMemcpyAsync from pageable host memory, which returns once the bytes are
 * staged), queues the work and returns; results are ready when the stream
 * reaches that point.  The couplings are checked on the GPU, so a J_dev
 * holding a value other than +-1 is reported in the outputs, not by the return
 * code: every best_sweep_dev entry is PB_NOALLOC_BAD_COUPLINGS and every energy
 * is NaN (the states are then meaningless).
 * Every call uses the same array and leaves its contents behind: calls whose
 * work overlaps on the GPU (different streams, or threads without ordering)
 * race and corrupt each other -- order them on one stream. */
#define PB_NOALLOC_BAD_COUPLINGS (-2)
pb_status pb_anneal_ea_noalloc(int32_t L, const int8_t* J_dev, const pb_schedule* sched, int32_t replicas,
                               uint64_t seed, double* best_E_dev, int32_t* best_sweep_dev, int8_t* best_states_dev,
                               double* final_E_dev, int8_t* final_states_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PBIT_H */
