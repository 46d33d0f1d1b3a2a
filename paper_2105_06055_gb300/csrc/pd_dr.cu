// Static FCBM-EC problems (Eq. 85-89) by adaptive dynamic relaxation, for one
// plan or for a batch of independent specimens, each specimen driven to
// convergence by device-side control flow inside one CUDA graph launch.
//
// The paper solves its static problems by CG (§4.3); dynamic relaxation is
// not in it. The method here is adaptive dynamic relaxation (ADR; Underwood
// 1983, in the peridynamic form of Kilic and Madenci, Theor. Appl. Fract.
// Mech. 53 (2010) 194-204): the correction equation A e = r
// (A e = -chi_O L(chi_O e), see pd_solve.cu) is read as the damped motion
//   rho_f e'' + c rho_f e' = F(e) = r - A e
// with a fictitious uniform density rho_f and unit pseudo time step,
// integrated by the damped central difference
//   v^{n+1/2} = ((2 - c^n) v^{n-1/2} + 2 F^n / rho_f) / (2 + c^n)
//   e^{n+1}  = e^n + v^{n+1/2}
// from e^0 = 0, v^{1/2} = F^0 / (2 rho_f) (the general step with v = 0 and
// c = 2 is exactly that start-up step). The damping tracks the lowest mode,
// c^n = 2 sqrt(omega^2), through the Rayleigh quotient of the current iterate
//   omega^2 = e^n.(A e^n) / (rho_f e^n.e^n),   A e^n = r - F^n,
// and c^n = 0 when the quotient is not positive. ADR as published estimates
// A e^n from a diagonal local stiffness, -(F^n_i - F^{n-1}_i) / v^{n-1/2}_i;
// here A e^n is known exactly (it is r - F^n, no extra work), and the
// diagonal estimate was seen to turn negative for whole stretches of steps
// and leave the iteration undamped. Stability of the central difference
// needs lambda_max(A) <= 4 rho_f; the chi cut and the restriction to Omega
// only remove bonds, so lambda_max(A) is at most the largest eigenvalue of
// the periodic symbol K^(0) - K^(k), and rho_f is 1.05/4 of it.
//
// The pseudo force is carried recursively, F^{n+1} = F^n - A v^{n+1/2}
// (e^{n+1} - e^n = v^{n+1/2}), so each step applies the operator to the
// velocity, which shrinks with F, and not to e: an FP32 evaluation of A e
// has an error of about eps32 lambda_max ||e||, which stalls the relaxation
// at eps32 kappa(A) relative to r, while the error of A v stays relative to
// F. The drift of the recursion is removed by the FP64 refinement.
//
// Precision and stopping follow pd_solve_static: the relaxation runs on the
// plan's FFT convolutions (FP32 on an FP32 plan) inside an iterative
// refinement whose residual R(u) = chi_O (b + L(u)) is recomputed with the
// FP64 operator; each relaxation cycle reduces ||F|| by 1e-3 (never below
// half the target) and the solve stops when ||R(u)|| <= rtol ||chi_O b|| (the
// initial ||R|| when chi_O b = 0).
//
// Device-side control: per specimen the graph holds
//   [bc, FP64 residual, check -> W] WHILE(W) { K relaxation steps,
//   check -> I, IF(I) { u += e, FP64 residual, check -> W, restart } }
// where the check kernels set the conditional handles with
// cudaGraphSetConditional. Every WHILE pass adds K steps and the step
// counter is capped by max_iter, after which the refinement check ends the
// loop, so the graph always terminates. Specimens are independent branches
// of the graph and run concurrently.
//
// One relaxation step (bond model) is the force pipeline with the update
// fused into its first and last passes:
//   rows  : v, e update (needs c^{n-1}); x1 transform of chi v
//   cols / last / cols : x2 transform, M^ multiply with x3, inverse (3D)
//   rows  : inverse x1, F += chi_O L(v), block partials of e.Ae, e.e
//           and ||F||^2
//   finish: c^n, ||F^n||^2
// The state-based operator (dilatation round between the halves) runs the
// update as separate vector kernels around the plain force.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "pd_force_impl.cuh"
#include "pd_solver_common.cuh"

namespace pd {
namespace {

constexpr int kDrChunk = 16;            // relaxation steps per WHILE pass
constexpr int kDrMaxCycles = 64;        // refinement cycles
constexpr int kDrPart = kMaxPart / 3;   // block partial triples
constexpr double kDrMaxSteps = 16777216.0;

// DR scalars in the plan's reduction buffer, after the CG scalars
enum {
    R_BN2 = 16, R_BN, R_TARGET, R_RN, R_ITOL2, R_C, R_FF, R_RHOINV, R_STEPS, R_MAXSTEPS, R_CYCLES,
    R_STATUS, R_GO, R_REL, R_BEST, R_SINCE, R_CSTEPS, R_RNPREV, R_SLOW, R_COUNT
};
// R_STATUS values
enum { DR_RUN = 0, DR_CONVERGED = 1, DR_MAXSTEPS = 2, DR_NONFINITE = 3, DR_TIMEOUT = 4, DR_CYCLES = 5,
       DR_STALLED = 6 };

__global__ void k_dr_start(double *red, double rho_inv, double max_steps)
{
    double *s = red + kRedScal;
    for (int i = R_BN2; i < R_COUNT; ++i) s[i] = 0.0;
    s[R_RHOINV] = rho_inv;
    s[R_MAXSTEPS] = max_steps;
}

// Refinement check after an FP64 residual: converged / out of budget /
// stalled / go on. Sets the WHILE handle; on "go on" arms the restart of the
// relaxation.
__global__ void k_dr_ir_check(double *red, const int *dev_status, cudaGraphConditionalHandle hw, int first,
                              double rtol)
{
    double *s = red + kRedScal;
    const double rn = sqrt(s[R_RN]);
    if (first) {
        // the residual is relative to ||chi_O b||; a problem driven by the
        // prescribed w alone (b = 0 on Omega) takes the initial residual instead
        const double rn0 = (rn > 0.0 && isfinite(rn)) ? rn : 1.0;
        s[R_BN] = s[R_BN2] > 0.0 ? sqrt(s[R_BN2]) : rn0;
        s[R_TARGET] = rtol * s[R_BN];
        s[R_RNPREV] = HUGE_VAL;
    }
    if (isfinite(rn)) s[R_REL] = rn / s[R_BN];
    // a cycle that did not halve the residual counts as slow; two in a row stall
    s[R_SLOW] = (rn > 0.5 * s[R_RNPREV]) ? s[R_SLOW] + 1.0 : 0.0;
    s[R_RNPREV] = rn;
    int st = (int)s[R_STATUS];
    if (st == DR_RUN) {
        if (*dev_status)
            st = DR_TIMEOUT;
        else if (!isfinite(rn))
            st = DR_NONFINITE;
        else if (rn <= s[R_TARGET])
            st = DR_CONVERGED;
        else if (s[R_STEPS] >= s[R_MAXSTEPS])
            st = DR_MAXSTEPS;
        else if (s[R_CYCLES] >= kDrMaxCycles)
            st = DR_CYCLES;
        else if (s[R_SLOW] >= 2.0)
            st = DR_STALLED;
    }
    s[R_STATUS] = st;
    const int go = st == DR_RUN;
    s[R_GO] = go;
    if (go) {
        s[R_CYCLES] += 1.0;
        const double itol = fmax(1e-3 * rn, 0.5 * s[R_TARGET]);
        s[R_ITOL2] = itol * itol;
        s[R_C] = 2.0;  // with v = 0: the start-up step v = F / (2 rho_f)
        s[R_BEST] = HUGE_VAL;
        s[R_SINCE] = 0.0;
        s[R_CSTEPS] = 0.0;
    }
    cudaGraphSetConditional(hw, go ? 1u : 0u);
}

// After K steps: is the relaxation cycle over? It is when ||F|| reaches the
// cycle's tolerance, when the step budget is spent, on a failure, or when
// ||F|| has stopped improving: no new minimum (by 2%) over the last half of
// the cycle and at least 1024 steps (the FP32 operator resolves F = r - A e
// only to about eps32 kappa(A) relative to r, below which the relaxation
// stalls; the refinement then starts the next cycle from the FP64 residual).
// Sets the IF handle of the refinement block. Backstop: should the step
// counter ever pass the budget by two passes without the refinement block
// having ended the loop, this kernel ends it itself.
__global__ void k_dr_check(double *red, const int *dev_status, cudaGraphConditionalHandle hif,
                           cudaGraphConditionalHandle hw, int K)
{
    double *s = red + kRedScal;
    s[R_STEPS] += K;
    s[R_CSTEPS] += K;
    const double ff = s[R_FF], c = s[R_C];
    if (ff < 0.9604 * s[R_BEST]) {  // 0.98^2: ||F|| down by 2%
        s[R_BEST] = ff;
        s[R_SINCE] = 0.0;
    } else {
        s[R_SINCE] += K;
    }
    const bool stalled = s[R_SINCE] >= 1024.0 && s[R_SINCE] >= 0.5 * s[R_CSTEPS];
    int done = ff <= s[R_ITOL2] || s[R_STEPS] >= s[R_MAXSTEPS] || stalled;
    if (!isfinite(ff) || !isfinite(c)) {
        if (s[R_STATUS] == DR_RUN) s[R_STATUS] = DR_NONFINITE;
        done = 1;
    }
    if (*dev_status) {
        if (s[R_STATUS] == DR_RUN) s[R_STATUS] = DR_TIMEOUT;
        done = 1;
    }
    if (s[R_STEPS] >= s[R_MAXSTEPS] + 2 * K) {
        if (s[R_STATUS] == DR_RUN) s[R_STATUS] = DR_MAXSTEPS;
        s[R_GO] = 0.0;
        cudaGraphSetConditional(hw, 0u);
        done = 0;
    }
    cudaGraphSetConditional(hif, done ? 1u : 0u);
}

// Restart of a relaxation cycle: r = (T) r64, F^0 = r, e = 0, v = 0.
template <typename T>
__global__ void k_dr_reset(const double *r64, T *rhs, T *e, T *v, T *F, int64_t n, const double *red)
{
    if (red[kRedScal + R_GO] == 0.0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T x = (T)r64[i];
        rhs[i] = x;
        F[i] = x;
        e[i] = T(0);
        v[i] = T(0);
    }
}

// u += e on Omega, unless the solve has already stopped with a failure
template <typename T>
__global__ void k_dr_ir_update(double *u, const T *e, const uint8_t *co, int64_t n, const double *red)
{
    if (red[kRedScal + R_STATUS] != DR_RUN) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (co[i]) u[i] += (double)e[i];
}

// Block partial triples (e.Ae, e.e, ||F||^2) -> c^n, ||F^n||^2 (one block of kFinishThreads)
__global__ void __launch_bounds__(kFinishThreads) k_dr_finish(double *red, int nparts)
{
    double a = 0.0, b = 0.0, f = 0.0, z = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        a += red[kRedPart + 3 * i];
        b += red[kRedPart + 3 * i + 1];
        f += red[kRedPart + 3 * i + 2];
    }
    block_sum4(a, b, f, z);
    if (threadIdx.x == 0) {
        double *s = red + kRedScal;
        const double q = b > 0.0 ? a / b * s[R_RHOINV] : 0.0;
        s[R_C] = q > 0.0 ? 2.0 * sqrt(q) : 0.0;
        s[R_FF] = f;
    }
}

struct DrAcc {
    DSum num, den, ff;
};

__device__ __forceinline__ void write_partial3(double *red, const DrAcc &acc)
{
    const DSum *a[3] = {&acc.num, &acc.den, &acc.ff};
    double t[3];
    block_sums<3>(a, t);
    if (threadIdx.x == 0) {
        red[kRedPart + 3 * blockIdx.x] = t[0];
        red[kRedPart + 3 * blockIdx.x + 1] = t[1];
        red[kRedPart + 3 * blockIdx.x + 2] = t[2];
    }
}

// one node's contribution to e.Ae (A e = r - F), e.e and ||F||^2
template <typename T>
__device__ __forceinline__ void dr_accumulate(DrAcc &acc, T Fn, T r, T ee)
{
    acc.ff.add(Fn * Fn);
    acc.den.add(ee * ee);
    acc.num.add(ee * (r - Fn));
}

// rows, forward: v^{n+1/2}, e^{n+1} from c^n, F^n; transform chi v
template <typename T, int D>
struct ProDR {
    static constexpr int kFin = 0, kFout = D, kNF = 0, kNB = 1, kStage = 0;
    static constexpr bool kSparse = false;
    T *e, *v;
    const T *F;
    const uint8_t *chi;
    const double *scal;
    int64_t N;
    int n1;
    cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int) const { return nullptr; }
    __device__ cx<T> *spec_out(int f) const { return spec + f * fstride; }
    __device__ const T *nf_src(int) const { return nullptr; }
    __device__ const uint8_t *nb_src(int) const { return chi; }
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *, const T *, T *o0,
                                          T *o1) const
    {
        const T cd = (T)scal[R_C], rinv = (T)scal[R_RHOINV];
        const T a = (T(2) - cd) / (T(2) + cd), bf = T(2) * rinv / (T(2) + cd);
        const T m0 = c.b(0, rl, i1) ? T(1) : T(0), m1 = c.b(0, rl, i1 + 1) ? T(1) : T(0);
        const int64_t p = (c.row0 + rl) * n1 + i1;
        typename vec2<T>::type ev[D], vv[D], fv[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            ev[j] = load2(e + j * N + p);
            vv[j] = load2(v + j * N + p);
            fv[j] = load2(F + j * N + p);
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const T va = a * vv[j].x + bf * fv[j].x, vb = a * vv[j].y + bf * fv[j].y;
            const T ea = ev[j].x + va, eb = ev[j].y + vb;
            store2(v + j * N + p, va, vb);
            store2(e + j * N + p, ea, eb);
            o0[j] = m0 * va;
            o1[j] = m1 * vb;
        }
    }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    __device__ void emit(const RowCtx<T> &, int, int, const T *, const T *, DSum &) const {}
    __device__ void block_done(DSum &) const {}
};

// rows, inverse: L(v) = chi y - G v staged, F^{n+1} = F^n + chi_O L(v), partials
template <typename T, int D>
struct EpiDR {
    static constexpr int kFin = D, kFout = 0, kStage = D, kNF = 0, kNB = 1 + D;
    static constexpr bool kSparse = false;
    using Acc = DrAcc;
    const T *e, *v, *rhs;
    T *F;
    const uint8_t *chi, *co;
    const GEntry<T> *gent;
    const int *gidx;
    double *red;
    int64_t N;
    int n1;
    const cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_out(int) const { return nullptr; }
    __device__ const T *nf_src(int) const { return nullptr; }
    __device__ const uint8_t *nb_src(int k) const { return k == 0 ? chi : co + (k - 1) * N; }
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *in0, const T *in1, T *o0,
                                          T *o1) const
    {
        const T m0 = c.b(0, rl, i1) ? T(1) : T(0), m1 = c.b(0, rl, i1 + 1) ? T(1) : T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            o0[i] = m0 * in0[i];
            o1[i] = m1 * in1[i];
        }
    }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    // L -= G v at a boundary node (entry k of the list)
    __device__ __forceinline__ void fix(int64_t p, int k, T *s) const
    {
        const GEntry<T> g = gent[k];
        T vv[D], Gv[D];
#pragma unroll
        for (int q = 0; q < D; ++q) {
            vv[q] = v[q * N + p];
            Gv[q] = T(0);
        }
        sym_apply<T, D>(g.g, vv, Gv);
#pragma unroll
        for (int i = 0; i < D; ++i) s[i] -= Gv[i];
    }
    __device__ __forceinline__ void emit(const RowCtx<T> &c, int rl, int i1, const T *s0, const T *s1,
                                         DrAcc &acc) const
    {
        const int64_t p = (c.row0 + rl) * n1 + i1;
        const int2 gi = *reinterpret_cast<const int2 *>(gidx + p);
        T a[D], b[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            a[i] = s0[i];
            b[i] = s1[i];
        }
        if (gi.x >= 0) fix(p, gi.x, a);
        if (gi.y >= 0) fix(p + 1, gi.y, b);
        typename vec2<T>::type ev[D], rv[D], fv[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            ev[i] = load2(e + i * N + p);
            rv[i] = load2(rhs + i * N + p);
            fv[i] = load2(F + i * N + p);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const T fa = c.b(1 + i, rl, i1) ? fv[i].x + a[i] : T(0);
            const T fb = c.b(1 + i, rl, i1 + 1) ? fv[i].y + b[i] : T(0);
            store2(F + i * N + p, fa, fb);
            dr_accumulate<T>(acc, fa, rv[i].x, ev[i].x);
            dr_accumulate<T>(acc, fb, rv[i].y, ev[i].y);
        }
    }
    __device__ void block_done(DrAcc &acc) const { write_partial3(red, acc); }
};

// unfused step (state-based operator): v, e update ...
template <typename T>
__global__ void k_dr_pre(T *e, T *v, const T *F, int64_t n, const double *red)
{
    const double *s = red + kRedScal;
    const T cd = (T)s[R_C], rinv = (T)s[R_RHOINV];
    const T a = (T(2) - cd) / (T(2) + cd), bf = T(2) * rinv / (T(2) + cd);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T vn = a * v[i] + bf * F[i];
        v[i] = vn;
        e[i] += vn;
    }
}

// ... and F^{n+1} = F^n + chi_O L(v) with the partials
template <typename T>
__global__ void k_dr_post(const T *L, const T *e, const T *rhs, T *F, const uint8_t *co, int64_t n, double *red)
{
    DrAcc acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T fn = co[i] ? F[i] + L[i] : T(0);
        F[i] = fn;
        dr_accumulate<T>(acc, fn, rhs[i], e[i]);
    }
    write_partial3(red, acc);
}

// Enqueues the relaxation of one specimen; all launches go to one stream
// (which may be capturing into a graph or a conditional body).
struct DrSpec {
    pd_plan *p;
    double *u;
    const double *b, *w;
    int64_t nvec;
    unsigned nb;

    template <typename T>
    T *vec(int k) const
    {
        void *v[4] = {p->cg_e, p->cg_r, p->cg_p, p->cg_q};  // e, r, v, F
        return reinterpret_cast<T *>(v[k]);
    }

    pd_status residual(cudaStream_t st) const
    {
        PD_TRY(force_plain<double>(p, u, nullptr, p->r64, nullptr, st));
        k_residual<<<nb, 256, 0, st>>>(p->r64, b, p->chi_om, nvec, p->red);
        PD_LAUNCH_CHECK();
        k_finish<<<1, 1024, 0, st>>>(p->red, (int)nb, R_RN, 0);
        PD_LAUNCH_CHECK();
        p->launches += 2;
        return PD_OK;
    }

    template <typename T>
    pd_status reset(cudaStream_t st) const
    {
        k_dr_reset<T><<<nb, 256, 0, st>>>(p->r64, vec<T>(1), vec<T>(0), vec<T>(2), vec<T>(3), nvec, p->red);
        PD_LAUNCH_CHECK();
        p->launches++;
        return PD_OK;
    }

    template <typename T, int D>
    pd_status step(cudaStream_t st) const
    {
        T *e = vec<T>(0), *rhs = vec<T>(1), *v = vec<T>(2), *F = vec<T>(3);
        if (p->state_based) {
            k_dr_pre<T><<<nb, 256, 0, st>>>(e, v, F, nvec, p->red);
            PD_LAUNCH_CHECK();
            T *L = reinterpret_cast<T *>(p->r64);  // scratch between refinement residuals
            PD_TRY(force_plain<T>(p, v, nullptr, L, nullptr, st));
            k_dr_post<T><<<nb, 256, 0, st>>>(L, e, rhs, F, p->chi_om, nvec, p->red);
            PD_LAUNCH_CHECK();
            k_dr_finish<<<1, kFinishThreads, 0, st>>>(p->red, (int)nb);
            PD_LAUNCH_CHECK();
            p->launches += 3;
            return PD_OK;
        }
        cx<T> *spec = reinterpret_cast<cx<T> *>(spec_buf<T>(p));
        const int64_t fs = p->N / 2;
        const Model<T> m = model_view<T>(p);
        ProDR<T, D> pro{e, v, F, p->chi, p->red + kRedScal, p->N, p->n1, spec, fs};
        PD_TRY(launch_rows<T>(p, pro, st));
        if (D == 3) PD_TRY((col_pass<T, D>(p, 0, false, st)));
        const int ob = D == 3 ? D : 0;
        CombForce<T, D, false> cmb{m, ob};
        PD_TRY(launch_cols<T>(p, cmb, D == 3 ? 2 : 1, true, D, st));
        if (D == 3) PD_TRY((col_pass<T, D>(p, ob, true, st)));
        EpiDR<T, D> epi{e, v, rhs, F, p->chi, p->chi_om, m.gent, p->gidx, p->red, p->N, p->n1, spec + ob * fs, fs};
        unsigned gepi = 0;
        PD_TRY(launch_rows<T>(p, epi, st, &gepi));
        if (gepi > (unsigned)kDrPart) {
            set_error("dynamic relaxation: %u row blocks exceed the reduction buffer", gepi);
            return PD_ERR_SIZE;
        }
        k_dr_finish<<<1, kFinishThreads, 0, st>>>(p->red, (int)gepi);
        PD_LAUNCH_CHECK();
        p->launches++;
        return PD_OK;
    }

    pd_status steps(cudaStream_t st, int K) const
    {
        for (int k = 0; k < K; ++k) {
            if (p->prob.fp64) {
                if (p->dim == 3)
                    PD_TRY((step<double, 3>(st)));
                else
                    PD_TRY((step<double, 2>(st)));
            } else {
                if (p->dim == 3)
                    PD_TRY((step<float, 3>(st)));
                else
                    PD_TRY((step<float, 2>(st)));
            }
        }
        return PD_OK;
    }

    pd_status ir_update(cudaStream_t st) const
    {
        if (p->prob.fp64)
            k_dr_ir_update<double><<<nb, 256, 0, st>>>(u, vec<double>(0), p->chi_om, nvec, p->red);
        else
            k_dr_ir_update<float><<<nb, 256, 0, st>>>(u, vec<float>(0), p->chi_om, nvec, p->red);
        PD_LAUNCH_CHECK();
        p->launches++;
        return PD_OK;
    }

    pd_status reset_any(cudaStream_t st) const { return p->prob.fp64 ? reset<double>(st) : reset<float>(st); }
};

// add a conditional node at the current capture position of `st` and make it
// the stream's only dependency; returns the body graph
pd_status add_conditional(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                          cudaGraph_t *body)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    PD_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &ndeps));
    if (cs != cudaStreamCaptureStatusActive) {
        set_error("dynamic relaxation: stream is not capturing");
        return PD_ERR_CUDA;
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    PD_CUDA_TRY(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &np));
    PD_CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    *body = np.conditional.phGraph_out[0];
    return PD_OK;
}

pd_status capture_graph_of(cudaStream_t st, cudaGraph_t *g)
{
    cudaStreamCaptureStatus cs;
    PD_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) {
        set_error("dynamic relaxation: stream is not capturing");
        return PD_ERR_CUDA;
    }
    return PD_OK;
}

// Enqueue one specimen's whole solve on `st` (capturing); bs, bs2: idle
// helper streams for the conditional bodies.
struct DrLaunches {
    int64_t pre = 0, chunk = 0, cycle = 0;  // kernels before the loop, per WHILE pass, per refinement block
};

pd_status capture_specimen(const DrSpec &S, double rtol, double max_steps, cudaStream_t st, cudaStream_t bs,
                           cudaStream_t bs2, DrLaunches *cnt)
{
    pd_plan *p = S.p;
    const int64_t l0 = p->launches;
    const double rho_inv = 1.0 / (0.25 * 1.05 * p->lam_max);
    k_dr_start<<<1, 1, 0, st>>>(p->red, rho_inv, max_steps);
    PD_LAUNCH_CHECK();
    PD_CUDA_TRY(cudaMemsetAsync(p->dev_status, 0, sizeof(int), st));
    k_apply_bc<<<S.nb, 256, 0, st>>>(S.u, S.w, S.b, p->chi_om, S.nvec, p->red);
    PD_LAUNCH_CHECK();
    k_finish<<<1, 1024, 0, st>>>(p->red, (int)S.nb, R_BN2, 0);
    PD_LAUNCH_CHECK();
    p->launches += 3;
    PD_TRY(S.residual(st));
    cudaGraph_t top = nullptr;
    PD_TRY(capture_graph_of(st, &top));
    cudaGraphConditionalHandle hw;
    PD_CUDA_TRY(cudaGraphConditionalHandleCreate(&hw, top, 0, 0));
    k_dr_ir_check<<<1, 1, 0, st>>>(p->red, p->dev_status, hw, 1, rtol);
    PD_LAUNCH_CHECK();
    PD_TRY(S.reset_any(st));
    cudaGraph_t wbody = nullptr;
    PD_TRY(add_conditional(st, hw, cudaGraphCondTypeWhile, &wbody));
    cnt->pre = p->launches - l0 + 2;  // + start and check kernels
    const int64_t l1 = p->launches;

    // WHILE body: K steps, cycle check, IF(cycle over) { refinement }
    PD_CUDA_TRY(cudaStreamBeginCaptureToGraph(bs, wbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    pd_status s = S.steps(bs, kDrChunk);
    cudaGraphConditionalHandle hif;
    cudaGraph_t ibody = nullptr;
    if (s == PD_OK && cudaGraphConditionalHandleCreate(&hif, wbody, 0, 0) != cudaSuccess) {
        set_error("dynamic relaxation: conditional handle creation failed");
        s = PD_ERR_CUDA;
    }
    if (s == PD_OK) {
        k_dr_check<<<1, 1, 0, bs>>>(p->red, p->dev_status, hif, hw, kDrChunk);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("dynamic relaxation: check launch failed");
            s = PD_ERR_CUDA;
        }
    }
    cnt->chunk = p->launches - l1 + 1;  // + check kernel
    const int64_t l2 = p->launches;
    if (s == PD_OK) s = add_conditional(bs, hif, cudaGraphCondTypeIf, &ibody);
    if (s == PD_OK) {
        if (cudaStreamBeginCaptureToGraph(bs2, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess) {
            set_error("dynamic relaxation: capture of the refinement block failed");
            s = PD_ERR_CUDA;
        } else {
            s = S.ir_update(bs2);
            if (s == PD_OK) s = S.residual(bs2);
            if (s == PD_OK) {
                k_dr_ir_check<<<1, 1, 0, bs2>>>(p->red, p->dev_status, hw, 0, rtol);
                if (cudaGetLastError() != cudaSuccess) {
                    set_error("dynamic relaxation: check launch failed");
                    s = PD_ERR_CUDA;
                }
            }
            if (s == PD_OK) s = S.reset_any(bs2);
            cudaGraph_t dummy = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(bs2, &dummy);
            if (s == PD_OK && e2 != cudaSuccess) {
                set_error("dynamic relaxation: refinement capture failed: %s", cudaGetErrorString(e2));
                s = PD_ERR_CUDA;
            }
        }
    }
    cnt->cycle = p->launches - l2 + 1;  // + check kernel
    p->launches = l0;                  // captured, not yet run
    cudaGraph_t dummy = nullptr;
    const cudaError_t e1 = cudaStreamEndCapture(bs, &dummy);
    if (s == PD_OK && e1 != cudaSuccess) {
        set_error("dynamic relaxation: body capture failed: %s", cudaGetErrorString(e1));
        s = PD_ERR_CUDA;
    }
    return s;
}

}  // namespace

// Runs the relaxation of a set of specimens as one graph launch. Owns the
// helper streams and the cached executable graph.
struct DrRunner {
    std::vector<pd_plan *> plans;
    cudaStream_t ms = nullptr, bs = nullptr, bs2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_done = nullptr;
    std::vector<cudaEvent_t> ev_join;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> key;
    double key_rtol = 0.0;
    int key_iter = 0;
    double *host = nullptr;  // pinned, plans.size() x R_COUNT
    std::vector<DrLaunches> counts;

    pd_status init(const std::vector<pd_plan *> &ps)
    {
        plans = ps;
        PD_CUDA_TRY(cudaStreamCreateWithFlags(&ms, cudaStreamNonBlocking));
        PD_CUDA_TRY(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
        PD_CUDA_TRY(cudaStreamCreateWithFlags(&bs2, cudaStreamNonBlocking));
        PD_CUDA_TRY(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        PD_CUDA_TRY(cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming));
        ev_join.assign(ps.size(), nullptr);
        for (auto &e : ev_join) PD_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        PD_CUDA_TRY(cudaMallocHost(&host, sizeof(double) * R_COUNT * ps.size()));
        return PD_OK;
    }

    ~DrRunner()
    {
        if (exec) cudaGraphExecDestroy(exec);
        for (auto e : ev_join)
            if (e) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_done) cudaEventDestroy(ev_done);
        for (cudaStream_t s : {ms, bs, bs2})
            if (s) cudaStreamDestroy(s);
        if (host) cudaFreeHost(host);
    }

    pd_status build(double *const *u, const double *const *b, const double *const *w, double rtol, int max_iter)
    {
        const size_t n = plans.size();
        std::vector<const void *> k;
        for (size_t i = 0; i < n; ++i) {
            k.push_back(u[i]);
            k.push_back(b[i]);
            k.push_back(w ? w[i] : nullptr);
        }
        if (exec && k == key && rtol == key_rtol && max_iter == key_iter) return PD_OK;
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        std::vector<int> prof(n);
        counts.assign(n, DrLaunches());
        for (size_t i = 0; i < n; ++i) {
            prof[i] = plans[i]->prof_on;
            plans[i]->prof_on = 0;  // no event nodes inside conditional bodies
            plans[i]->no_fork = 1;  // and no second stream
            plans[i]->pdl = 0;      // nor programmatic launches
        }
        cudaGraph_t graph = nullptr;
        pd_status s = PD_OK;
        if (cudaStreamBeginCapture(ms, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            set_error("dynamic relaxation: capture could not begin");
            s = PD_ERR_CUDA;
        } else {
            if (cudaEventRecord(ev_fork, ms) != cudaSuccess) s = PD_ERR_CUDA;
            const double msteps = std::min<double>(std::max(max_iter, 1), kDrMaxSteps);
            for (size_t i = 0; i < n && s == PD_OK; ++i) {
                pd_plan *p = plans[i];
                if (cudaStreamWaitEvent(p->own_stream, ev_fork, 0) != cudaSuccess) {
                    s = PD_ERR_CUDA;
                    break;
                }
                DrSpec S{p, u[i], b[i], w ? w[i] : nullptr, (int64_t)p->dim * p->N, 0};
                S.nb = (unsigned)std::min<int64_t>(kUpdBlocks, (S.nvec + 255) / 256);
                s = capture_specimen(S, rtol, msteps, p->own_stream, bs, bs2, &counts[i]);
                if (s == PD_OK && (cudaEventRecord(ev_join[i], p->own_stream) != cudaSuccess ||
                                   cudaStreamWaitEvent(ms, ev_join[i], 0) != cudaSuccess))
                    s = PD_ERR_CUDA;
            }
            const cudaError_t ce = cudaStreamEndCapture(ms, &graph);
            if (s == PD_OK && ce != cudaSuccess) {
                set_error("dynamic relaxation: capture failed: %s", cudaGetErrorString(ce));
                s = PD_ERR_CUDA;
            }
        }
        for (size_t i = 0; i < n; ++i) {
            plans[i]->prof_on = prof[i];
            plans[i]->no_fork = 0;
            plans[i]->pdl = 1;
        }
        if (s != PD_OK) {
            if (graph) cudaGraphDestroy(graph);
            if (s == PD_ERR_CUDA && !*pd_last_error_detail()) set_error("dynamic relaxation: graph build failed");
            return s;
        }
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            exec = nullptr;
            set_error("dynamic relaxation: graph instantiation failed: %s", cudaGetErrorString(ie));
            return PD_ERR_CUDA;
        }
        key = k;
        key_rtol = rtol;
        key_iter = max_iter;
        return PD_OK;
    }

    pd_status run(double *const *u, const double *const *b, const double *const *w, double rtol, int max_iter,
                  int *iters_out, double *relres_out, int *status_out, cudaStream_t caller)
    {
        const size_t n = plans.size();
        PD_TRY(build(u, b, w, rtol, max_iter));
        PD_CUDA_TRY(cudaEventRecord(ev_done, caller));
        PD_CUDA_TRY(cudaStreamWaitEvent(ms, ev_done, 0));
        PD_CUDA_TRY(cudaGraphLaunch(exec, ms));
        for (size_t i = 0; i < n; ++i)
            PD_CUDA_TRY(cudaMemcpyAsync(host + i * R_COUNT, plans[i]->red + kRedScal, sizeof(double) * R_COUNT,
                                        cudaMemcpyDeviceToHost, ms));
        PD_CUDA_TRY(cudaStreamSynchronize(ms));
        PD_CUDA_TRY(cudaEventRecord(ev_done, ms));
        PD_CUDA_TRY(cudaStreamWaitEvent(caller, ev_done, 0));
        pd_status worst = PD_OK;
        for (size_t i = 0; i < n; ++i) {
            const double *h = host + i * R_COUNT;
            const int st = (int)h[R_STATUS];
            pd_plan *p = plans[i];
            const DrLaunches &c = counts[i];
            p->launches += c.pre + (int64_t)h[R_STEPS] / kDrChunk * c.chunk + (int64_t)h[R_CYCLES] * c.cycle;
            pd_status r = PD_OK;
            switch (st) {
                case DR_CONVERGED: r = PD_OK; break;
                case DR_NONFINITE: r = PD_ERR_NONFINITE; break;
                case DR_TIMEOUT: r = PD_ERR_TIMEOUT; break;
                default: r = PD_ERR_NOT_CONVERGED; break;
            }
            if (iters_out) iters_out[i] = (int)h[R_STEPS];
            if (relres_out) relres_out[i] = h[R_REL];
            if (status_out) status_out[i] = (int)r;
            if (r != PD_OK && worst == PD_OK) {
                worst = r;
                set_error("dynamic relaxation: specimen %zu: %s (relative residual %.3e after %d steps)", i,
                          pd_status_string(r), h[R_REL], (int)h[R_STEPS]);
            }
        }
        return worst;
    }
};

}  // namespace pd

using namespace pd;

struct pd_batch {
    std::vector<pd_plan *> plans;
    DrRunner runner;
};

static pd_status check_dr_args(const char *who, double rtol, int max_iter)
{
    if (!(rtol > 0) || max_iter < 1) {
        set_error("%s: rtol must be > 0 and max_iter >= 1", who);
        return PD_ERR_ARG;
    }
    return PD_OK;
}

extern "C" pd_status pd_solve_dr(pd_plan *p, double *u, const double *b, const double *w, double rtol, int max_iter,
                                 int *iters_out, double *relres_out, void *stream)
{
    if (!p || !u || !b) {
        set_error("pd_solve_dr: null plan, u or b");
        return PD_ERR_ARG;
    }
    if (p->nonlinear) {
        set_error("pd_solve_dr: the nonlinear bond model is available through pd_force only");
        return PD_ERR_ARG;
    }
    PD_TRY(check_dr_args("pd_solve_dr", rtol, max_iter));
    DrRunner R;
    PD_TRY(R.init({p}));
    const double *wp[1] = {w};
    return R.run(&u, &b, w ? wp : nullptr, rtol, max_iter, iters_out, relres_out, nullptr, (cudaStream_t)stream);
}

extern "C" pd_status pd_plan_create_batched(int nspec, const pd_problem *problems, const uint8_t *const *chi_B,
                                            const uint8_t *const *chi_Omega, void *stream, pd_batch **out)
{
    if (!out || !problems || !chi_B || nspec < 1) {
        set_error("pd_plan_create_batched: null argument or nspec < 1");
        return PD_ERR_ARG;
    }
    *out = nullptr;
    pd_batch *B = new pd_batch();
    for (int i = 0; i < nspec; ++i) {
        pd_plan *p = nullptr;
        const pd_status s = pd_plan_create(&problems[i], chi_B[i], chi_Omega ? chi_Omega[i] : nullptr, stream, &p);
        if (s != PD_OK) {
            const std::string msg = pd_last_error_detail();
            for (pd_plan *q : B->plans) pd_plan_destroy(q);
            delete B;
            set_error("pd_plan_create_batched: specimen %d: %s", i, msg.c_str());
            return s;
        }
        B->plans.push_back(p);
    }
    const pd_status s = B->runner.init(B->plans);
    if (s != PD_OK) {
        pd_batch_destroy(B);
        return s;
    }
    *out = B;
    return PD_OK;
}

extern "C" int pd_batch_size(const pd_batch *B) { return B ? (int)B->plans.size() : 0; }

extern "C" pd_plan *pd_batch_plan(pd_batch *B, int i)
{
    if (!B || i < 0 || i >= (int)B->plans.size()) return nullptr;
    return B->plans[i];
}

extern "C" pd_status pd_solve_dr_batched(pd_batch *B, double *const *u, const double *const *b,
                                         const double *const *w, double rtol, int max_iter, int *iters_out,
                                         double *relres_out, int *status_out, void *stream)
{
    if (!B || !u || !b) {
        set_error("pd_solve_dr_batched: null batch, u or b");
        return PD_ERR_ARG;
    }
    PD_TRY(check_dr_args("pd_solve_dr_batched", rtol, max_iter));
    for (size_t i = 0; i < B->plans.size(); ++i)
        if (!u[i] || !b[i]) {
            set_error("pd_solve_dr_batched: null u or b of specimen %zu", i);
            return PD_ERR_ARG;
        }
    return B->runner.run(u, b, w, rtol, max_iter, iters_out, relres_out, status_out, (cudaStream_t)stream);
}

extern "C" void pd_batch_destroy(pd_batch *B)
{
    if (!B) return;
    if (B->runner.ms) cudaStreamSynchronize(B->runner.ms);
    if (B->runner.exec) {
        cudaGraphExecDestroy(B->runner.exec);
        B->runner.exec = nullptr;
    }
    for (pd_plan *p : B->plans) pd_plan_destroy(p);
    B->plans.clear();
    delete B;
}

// forget the cached graph (the plans' pass configuration changed)
void pd_batch_invalidate(pd_batch *B)
{
    if (B && B->runner.exec) {
        cudaStreamSynchronize(B->runner.ms);
        cudaGraphExecDestroy(B->runner.exec);
        B->runner.exec = nullptr;
        B->runner.key.clear();
    }
}
