// imin.cpp -- the benchmarking protocol of arXiv 2510.23419 (Sec. 4.1.3,
// Algorithm 1): the smallest iteration budget i at which classical annealing
// with a linear beta schedule passes a tolerance test.
//
// At budget i, t independent trials anneal the instance for i iterations (an
// iteration is one update-group step, so a sweep of k colour classes is k
// iterations; the schedule runs linear from beta_i to beta_f over the sweeps);
// a trial fails when the lowest energy it found is above theta = p G (G < 0,
// the ground truth); the budget passes when at most m_max = round(t (1 -
// p_succ)) trials fail (round half up).  The budgets i_start, i_start + i_step, ... are tried
// in order and the first that passes is returned.
//
// GB300 form: the t trials of a budget are t replicas of one anneal, and
// `budgets_per_launch` consecutive budgets are evaluated together as one
// batch; the first passing budget of the batch is the answer.  The paper's
// loop stops counting a budget's fails once m > m_max, which changes only its
// running time, not its verdict, so both forms return the same i for the same
// trial outcomes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "pb_handles.h"

using namespace pb;

extern "C" {

pb_status pb_find_imin(pb_instance* inst, const pb_imin_opts* o, void* stream, pb_imin_result* out)
{
    pb::TraceRange trace_("pb_find_imin");
    if (!inst || !o || !out) return fail(PB_EINVAL, "null argument");
    if (o->trials < 1) return fail(PB_EINVAL, "trials must be >= 1");
    if (o->i_start < 1 || o->i_step < 1) return fail(PB_EINVAL, "i_start and i_step must be >= 1");
    if (!(o->ground < 0.0)) return fail(PB_EINVAL, "the ground truth G must be negative");
    if (o->p_succ < 0.0 || o->p_succ > 1.0) return fail(PB_EINVAL, "p_succ must be in [0, 1]");
    *out = pb_imin_result{-1, 0, 0, 0};
    const int k = pb_instance_colours(inst);
    const double theta = o->p * o->ground;
    const int m_max = (int)std::floor(o->trials * (1.0 - o->p_succ) + 0.5);  // round half up
    const int per = o->budgets_per_launch > 0 ? o->budgets_per_launch : 8;
    const int i_max = o->i_max > 0 ? o->i_max : o->i_start + 1000 * o->i_step;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<double> best((size_t)o->trials);
    for (int i0 = o->i_start; i0 <= i_max; i0 += per * o->i_step) {
        std::vector<int> budgets;
        for (int b = 0; b < per && i0 + b * o->i_step <= i_max; ++b) budgets.push_back(i0 + b * o->i_step);
        const int m = (int)budgets.size();
        std::vector<pb_instance*> insts((size_t)m, inst);
        std::vector<pb_schedule> sc((size_t)m);
        std::vector<int32_t> reps((size_t)m, o->trials);
        std::vector<uint64_t> seeds((size_t)m);
        std::vector<pb_anneal_opts> opts((size_t)m, pb_anneal_opts{o->form, 0, NAN});
        for (int b = 0; b < m; ++b) {
            sc[(size_t)b] = pb_schedule{};
            sc[(size_t)b].kind = PB_SCHED_LINEAR;
            sc[(size_t)b].n_sweeps = (budgets[(size_t)b] + k - 1) / k;  // iterations -> sweeps
            sc[(size_t)b].step_duration = 1;
            sc[(size_t)b].beta0 = o->beta_i;
            sc[(size_t)b].beta1 = o->beta_f;
            seeds[(size_t)b] = o->seed + (uint64_t)budgets[(size_t)b];  // trials of budget i: seed + i
        }
        std::vector<pb_run*> runs((size_t)m, nullptr);
        pb_status ps = pb_anneal_batch(m, insts.data(), sc.data(), reps.data(), seeds.data(), opts.data(), st, runs.data());
        if (ps != PB_OK) return ps;
        ++out->launches;
        int found = -1, found_fails = 0;
        for (int b = 0; b < m; ++b) {
            if (found < 0) {
                ps = pb_energy(runs[(size_t)b], nullptr, best.data(), nullptr);
                if (ps != PB_OK) {
                    for (pb_run* r : runs) pb_run_destroy(r);
                    return ps;
                }
                int fails = 0;
                for (double v : best) fails += v > theta ? 1 : 0;
                ++out->budgets_tried;
                if (fails <= m_max) {
                    found = budgets[(size_t)b];
                    found_fails = fails;
                }
            }
        }
        for (pb_run* r : runs) pb_run_destroy(r);
        if (found >= 0) {
            out->i_min = found;
            out->fails = found_fails;
            return PB_OK;
        }
    }
    return PB_OK;  // no budget up to i_max passed: i_min = -1
}

}  // extern "C"
