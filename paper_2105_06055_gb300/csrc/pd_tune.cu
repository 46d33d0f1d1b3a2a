// Autotuner for the FFT passes: picks, per plan, the rows per block of the
// row passes and their pipeline depth (one or two shared-memory stages), the
// tile width of the column passes (x2 and last axis) and the FFT stage
// schedule (radix-4/2 remainder stage first or last) by timing the plan's own
// force evaluation (pd_plan_autotune) or a chunk of its static solver's CG
// iterations (pd_plan_autotune_solve) on its workspace with CUDA events.
//
// The search covers (for the solver on FP32 cubes up to 128^3) whether the CG
// iteration's forward half runs as a plane pass, then rows x stages jointly, the inverse passes'
// stages, the schedule, the last-axis width and the x2 width one at a time; each candidate is timed as
// the median of nine force evaluations after three untimed ones. Candidates
// are limited to the shapes the passes accept (powers of two; at least one
// warp per row block; shared memory within the pass's own limit, which the
// configuration functions enforce by shrinking the candidate). The
// transforms compute the same values for every candidate (only the order of
// block partial sums in the solvers' inner products changes).
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "pd_force_impl.cuh"

using namespace pd;

struct pd_batch;
void pd_batch_invalidate(pd_batch *B);
extern "C" pd_plan *pd_batch_plan(pd_batch *B, int i);
extern "C" int pd_batch_size(const pd_batch *B);

namespace pd {
pd_status time_cg_chunk(pd_plan *p, cudaEvent_t e0, cudaEvent_t e1, float *ms_out);
template <typename T>
pd_status force_nl(pd_plan *p, const T *u, T *L, cudaStream_t st);
}

namespace {

void drop_graphs(pd_plan *p)
{
    for (int k = 0; k < 2; ++k)
        if (p->cg_graph[k]) {
            cudaGraphExecDestroy(p->cg_graph[k]);
            p->cg_graph[k] = nullptr;
        }
}

template <typename T>
pd_status time_force(pd_plan *p, cudaEvent_t e0, cudaEvent_t e1, float *ms_out)
{
    cudaStream_t st = p->own_stream;
    const T *u = (const T *)p->cg_e;
    T *L = (T *)p->cg_q;
    auto eval = [&]() { return p->nonlinear ? force_nl<T>(p, u, L, st) : force_plain<T>(p, u, nullptr, L, nullptr, st); };
    for (int k = 0; k < 3; ++k) PD_TRY(eval());
    std::vector<float> t;
    for (int k = 0; k < 9; ++k) {
        PD_CUDA_TRY(cudaEventRecord(e0, st));
        PD_TRY(eval());
        PD_CUDA_TRY(cudaEventRecord(e1, st));
        PD_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        PD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    *ms_out = t[4];
    return PD_OK;
}

// what the search times: 0 a force evaluation, 1 a chunk of static-solver
// CG iterations (its graph is recaptured for every candidate)
pd_status time_cfg(pd_plan *p, int target, cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    if (target == 1) {
        drop_graphs(p);
        return time_cg_chunk(p, e0, e1, ms);
    }
    return p->prob.fp64 ? time_force<double>(p, e0, e1, ms) : time_force<float>(p, e0, e1, ms);
}

pd_status tune_plan(pd_plan *p, cudaStream_t caller, int target = 0)
{
    PD_CUDA_TRY(cudaEventRecord(p->ev_join[0], caller));
    PD_CUDA_TRY(cudaStreamWaitEvent(p->own_stream, p->ev_join[0], 0));
    const size_t bytes = (size_t)p->dim * p->N * (p->prob.fp64 ? 8 : 4);
    PD_CUDA_TRY(cudaMemsetAsync(p->cg_e, 0, bytes, p->own_stream));
    const int prof = p->prof_on;
    p->prof_on = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PD_CUDA_TRY(cudaEventCreate(&e0));
    PD_CUDA_TRY(cudaEventCreate(&e1));
    pd_status s = PD_OK;
    auto best_of = [&](int *knob, const std::vector<int> &cands) {
        if (s != PD_OK || cands.size() < 2) return;
        int best = *knob;
        float tbest = 1e30f;
        for (int c : cands) {
            *knob = c;
            float ms = 0.f;
            s = time_cfg(p, target, e0, e1, &ms);
            if (s != PD_OK) return;
            if (ms < tbest) {
                tbest = ms;
                best = c;
            }
        }
        *knob = best;
    };
    // static solve on an FP32 cube with plane passes: whether the forward half
    // of the CG iteration runs as a plane pass, first, as the row knobs below
    // only act on the halves that stay row passes. The inverse plane pass is
    // not a candidate: a lone chunk timed it faster, whole solves slower (128^3:
    // 115.3 against 105.9 ms per solve).
    if (target == 1 && p->dim == 3 && !p->prob.fp64 && !p->state_based && p->n1 == p->n2 &&
        (p->n1 == 32 || p->n1 == 64 || p->n1 == 128))
        best_of(&p->plane_passes, {1, 0});
    // rows per tile and pipeline depth jointly (they interact through shared
    // memory), then the schedule and the column widths one at a time
    const int H = p->h;
    const int nt = H >> kLgV;
    {
        float tbest = 1e30f;
        int rbest = p->tune_rows, sbest = p->tune_stages;
        for (int r = std::max(1, 32 / nt); r * nt <= 256 && s == PD_OK; r *= 2) {
            if (p->nrows % r) continue;
            for (int ns : {2, 1}) {
                p->tune_rows = r;
                p->tune_stages = ns;
                float ms = 0.f;
                s = time_cfg(p, target, e0, e1, &ms);
                if (s != PD_OK) break;
                if (ms < tbest) {
                    tbest = ms;
                    rbest = r;
                    sbest = ns;
                }
            }
        }
        p->tune_rows = rbest;
        p->tune_stages = sbest;
    }
    best_of(&p->tune_stages_inv, {1, 2});
    // schedule: only lengths that are not powers of 8 have a remainder stage
    const bool rem = (ilog2(H) % kLgV) || (ilog2(p->n2) % kLgV) || (p->dim == 3 && (ilog2(p->n3) % kLgV));
    if (rem) best_of(&p->tune_sched, {0, 1});
    best_of(&p->tune_w[1], {32, 16, 8, 4});
    if (p->dim == 3) best_of(&p->tune_w[0], {32, 16, 8, 4});
    p->prof_on = prof;
    drop_graphs(p);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != PD_OK) return s;
    PD_CUDA_TRY(cudaEventRecord(p->ev_join[1], p->own_stream));
    PD_CUDA_TRY(cudaStreamWaitEvent(caller, p->ev_join[1], 0));
    return PD_OK;
}

}  // namespace

extern "C" pd_status pd_plan_autotune(pd_plan *p, void *stream)
{
    if (!p) {
        set_error("pd_plan_autotune: null plan");
        return PD_ERR_ARG;
    }
    return tune_plan(p, (cudaStream_t)stream);
}

extern "C" pd_status pd_plan_autotune_solve(pd_plan *p, void *stream)
{
    if (!p) {
        set_error("pd_plan_autotune_solve: null plan");
        return PD_ERR_ARG;
    }
    if (p->nonlinear) {
        set_error("pd_plan_autotune_solve: the nonlinear bond model is available through pd_force only");
        return PD_ERR_ARG;
    }

    return tune_plan(p, (cudaStream_t)stream, 1);
}

extern "C" pd_status pd_plan_tuning(const pd_plan *p, int *out6)
{
    if (!p || !out6) {
        set_error("pd_plan_tuning: null argument");
        return PD_ERR_ARG;
    }
    out6[0] = p->tune_rows;
    out6[1] = p->tune_w[0];
    out6[2] = p->tune_w[1];
    out6[3] = p->tune_sched;
    out6[4] = p->tune_stages;
    out6[5] = p->tune_stages_inv;
    return PD_OK;
}

extern "C" pd_status pd_batch_autotune(pd_batch *B, void *stream)
{
    if (!B) {
        set_error("pd_batch_autotune: null batch");
        return PD_ERR_ARG;
    }
    // one search per distinct grid / precision / operator; the others copy it
    std::map<std::tuple<int, int, int, int, int, int>, pd_plan *> done;
    for (int i = 0; i < pd_batch_size(B); ++i) {
        pd_plan *p = pd_batch_plan(B, i);
        const auto key = std::make_tuple(p->dim, p->n1, p->n2, p->n3, p->prob.fp64, p->state_based);
        auto it = done.find(key);
        if (it == done.end()) {
            PD_TRY(tune_plan(p, (cudaStream_t)stream));
            done[key] = p;
        } else {
            p->tune_rows = it->second->tune_rows;
            p->tune_w[0] = it->second->tune_w[0];
            p->tune_w[1] = it->second->tune_w[1];
            p->tune_sched = it->second->tune_sched;
            p->tune_stages = it->second->tune_stages;
            p->tune_stages_inv = it->second->tune_stages_inv;
            drop_graphs(p);
        }
    }
    pd_batch_invalidate(B);
    return PD_OK;
}

extern "C" pd_status pd_plan_set_plane_passes(pd_plan *p, int on)
{
    if (!p || on < 0 || on > 3) {
        set_error("pd_plan_set_plane_passes: null plan or mask not in 0..3");
        return PD_ERR_ARG;
    }
    p->plane_passes = on;
    drop_graphs(p);
    return PD_OK;
}

extern "C" pd_status pd_plan_set_tuning(pd_plan *p, const int *in6)
{
    if (!p || !in6) {
        set_error("pd_plan_set_tuning: null argument");
        return PD_ERR_ARG;
    }
    const int r = in6[0], wx = in6[1], wl = in6[2], sc = in6[3], ns = in6[4], ni = in6[5];
    auto pow2_or_zero = [](int v) { return v == 0 || (v > 0 && (v & (v - 1)) == 0); };
    // a column tile is at least 2 complex values wide: its first column, and so the
    // x coordinate of every tensor copy, is then a multiple of 16 bytes
    if (!pow2_or_zero(r) || r > 256 || !pow2_or_zero(wx) || wx == 1 || wx > 32 || !pow2_or_zero(wl) || wl == 1 ||
        wl > 32 || (sc != 0 && sc != 1) || ns < 0 || ns > 2 || ni < 0 || ni > 2) {
        set_error("pd_plan_set_tuning: rows and widths must be 0 or powers of two (rows <= 256, widths 2..32), "
                  "schedule 0 or 1, stages 0, 1 or 2");
        return PD_ERR_ARG;
    }
    p->tune_rows = r;
    p->tune_w[0] = wx;
    p->tune_w[1] = wl;
    p->tune_sched = sc;
    p->tune_stages = ns;
    p->tune_stages_inv = ni;
    drop_graphs(p);
    return PD_OK;
}
