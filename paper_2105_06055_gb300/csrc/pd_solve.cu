// pd_solve_static: FCBM-EC elastostatics (Eq. 85-89) by conjugate gradient (§4.3).
//
// The residual of Eq. 89, R(u) = chi_O (L(u) + b), with u = w on Gamma, is zero
// at the solution. Writing u = u0 + e with e = 0 off Omega, the correction
// solves A e = R(u0) with A e = -chi_O L(chi_O e): A is symmetric and positive
// definite on Omega (the bond sum of Eq. 17-18 / 36 with the chi_B cut is a
// weighted graph Laplacian once the constraint removes the rigid motions).
//
// Precision: on an FP32 plan the CG runs on FP32 FFT convolutions with FP64
// inner products, inside an iterative refinement whose residual R(u) is
// recomputed with the FP64 convolution path on the FP64 iterate u. The outer
// loop stops when ||R(u)||_2 <= rtol ||chi_O b||_2 (both in FP64). On an FP64
// plan the same code runs with FP64 everywhere.
//
// All CG scalars (alpha, beta, residual norms) stay on the device; the host
// reads the residual norm every kCheck iterations to decide when to stop.
#include <cmath>
#include <vector>

#include "pd_plan.cuh"

namespace pd {

template <typename T>
pd_status force_plain(pd_plan *p, const T *u, const T *s, T *L, T *W, cudaStream_t st);

namespace {

constexpr int kRedBlocks = 1024;     // partial-sum slots per reduction
constexpr int kCheck = 16;           // CG iterations between host checks
// layout of the plan's reduction buffer (doubles)
constexpr int RED_PART = 0;          // kRedBlocks partials
constexpr int RED_SCAL = 2048;       // scalars below
enum { S_RR = 0, S_PQ, S_ALPHA, S_BETA, S_RRNEW, S_NORM, S_BN, S_FLAG, S_COUNT };

unsigned red_blocks(const pd_plan *p) { return (unsigned)std::min<int64_t>(kRedBlocks, 2 * (int64_t)p->nsm); }

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;
}

// Final reduction of the block partials into scalar `dst`, then the CG scalar
// update selected by `what`:
//   0: store only; 1: alpha = rr / pq; 2: beta = rrnew / rr, rr = rrnew
__global__ void k_finish(double *red, int nparts, int dst, int what)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += red[RED_PART + i];
    v = block_sum(v);
    if (threadIdx.x == 0) {
        double *s = red + RED_SCAL;
        s[dst] = v;
        if (!isfinite(v)) s[S_FLAG] = 1.0;
        if (what == 1) {
            s[S_ALPHA] = (v > 0.0) ? s[S_RR] / v : 0.0;
            if (!(v > 0.0)) s[S_FLAG] = 2.0;  // breakdown: p.Ap <= 0
        } else if (what == 2) {
            s[S_BETA] = (s[S_RR] > 0.0) ? v / s[S_RR] : 0.0;
            s[S_RR] = v;
        }
    }
}

// u = chi_O u + (1 - chi_O) w ; partial ||chi_O b||^2
__global__ void k_apply_bc(double *u, const double *w, const double *b, const uint8_t *co, int64_t n,
                           double *red)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = co[i] ? 1.0 : 0.0;
        u[i] = m * u[i] + (1.0 - m) * (w ? w[i] : 0.0);
        const double bb = m * b[i];
        acc += bb * bb;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) red[RED_PART + blockIdx.x] = acc;
}

// r = chi_O (b + L) in place on L ; partial ||r||^2
__global__ void k_residual(double *r, const double *b, const uint8_t *co, int64_t n, double *red)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = co[i] ? (b[i] + r[i]) : 0.0;
        r[i] = v;
        acc += v * v;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) red[RED_PART + blockIdx.x] = acc;
}

// r = (T) r64, p = r, e = 0 ; partial r.r
template <typename T>
__global__ void k_cg_init(const double *r64, T *r, T *pp, T *e, int64_t n, double *red)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T v = (T)r64[i];
        r[i] = v;
        pp[i] = v;
        e[i] = T(0);
        acc += (double)v * (double)v;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) red[RED_PART + blockIdx.x] = acc;
}

// q = -chi_O L(p) in place ; partial p.q
template <typename T>
__global__ void k_cg_q(T *q, const T *pp, const uint8_t *co, int64_t n, double *red)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T v = co[i] ? -q[i] : T(0);
        q[i] = v;
        acc += (double)pp[i] * (double)v;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) red[RED_PART + blockIdx.x] = acc;
}

// e += alpha p ; r -= alpha q ; partial r.r
template <typename T>
__global__ void k_cg_update(T *e, T *r, const T *pp, const T *q, int64_t n, double *red)
{
    const double a = red[RED_SCAL + S_ALPHA];
    const T at = (T)a;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        e[i] += at * pp[i];
        const T rv = r[i] - at * q[i];
        r[i] = rv;
        acc += (double)rv * (double)rv;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) red[RED_PART + blockIdx.x] = acc;
}

// p = r + beta p
template <typename T>
__global__ void k_cg_dir(T *pp, const T *r, int64_t n, const double *red)
{
    const T bt = (T)red[RED_SCAL + S_BETA];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pp[i] = r[i] + bt * pp[i];
}

// u += e on Omega
template <typename T>
__global__ void k_ir_update(double *u, const T *e, const uint8_t *co, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (co[i]) u[i] += (double)e[i];
}

struct Solver {
    pd_plan *p;
    cudaStream_t st;
    double *hbuf;  // pinned host scalars
    int64_t nvec;
    unsigned nb;

    pd_status finish(int dst, int what)
    {
        k_finish<<<1, 1024, 0, st>>>(p->red, nb, dst, what);
        PD_LAUNCH_CHECK();
        p->launches++;
        return PD_OK;
    }
    pd_status read_scalars()
    {
        PD_CUDA_TRY(cudaMemcpyAsync(hbuf, p->red + RED_SCAL, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        return PD_OK;
    }

    // FP64 residual r64 = chi_O (b + L64(u)); returns ||r64||
    pd_status residual(const double *u, const double *b, double *rn)
    {
        PD_TRY(force_plain<double>(p, u, nullptr, p->r64, nullptr, st));
        k_residual<<<nb, 256, 0, st>>>(p->r64, b, p->chi_om, nvec, p->red);
        PD_LAUNCH_CHECK();
        p->launches++;
        PD_TRY(finish(S_NORM, 0));
        PD_TRY(read_scalars());
        *rn = std::sqrt(hbuf[S_NORM]);
        if (!std::isfinite(*rn)) {
            set_error("pd_solve_static: non-finite residual");
            return PD_ERR_NONFINITE;
        }
        return PD_OK;
    }

    // CG on A e = r64 until ||r|| <= tol_abs or max_it; returns iterations done
    template <typename T>
    pd_status cg(double tol_abs, int max_it, int *done, double *rr_last)
    {
        T *e = (T *)p->cg_e, *r = (T *)p->cg_r, *pp = (T *)p->cg_p, *q = (T *)p->cg_q;
        k_cg_init<T><<<nb, 256, 0, st>>>(p->r64, r, pp, e, nvec, p->red);
        PD_LAUNCH_CHECK();
        p->launches++;
        PD_TRY(finish(S_RR, 0));
        int it = 0;
        double best = HUGE_VAL;
        int since_best = 0;
        while (it < max_it) {
            const int chunk = std::min(kCheck, max_it - it);
            for (int k = 0; k < chunk; ++k) {
                PD_TRY(force_plain<T>(p, pp, nullptr, q, nullptr, st));
                k_cg_q<T><<<nb, 256, 0, st>>>(q, pp, p->chi_om, nvec, p->red);
                PD_LAUNCH_CHECK();
                PD_TRY(finish(S_PQ, 1));
                k_cg_update<T><<<nb, 256, 0, st>>>(e, r, pp, q, nvec, p->red);
                PD_LAUNCH_CHECK();
                PD_TRY(finish(S_RRNEW, 2));
                k_cg_dir<T><<<nb, 256, 0, st>>>(pp, r, nvec, p->red);
                PD_LAUNCH_CHECK();
                p->launches += 3;
            }
            it += chunk;
            PD_TRY(read_scalars());
            const double rn = std::sqrt(hbuf[S_RR]);
            *rr_last = rn;
            if (hbuf[S_FLAG] == 1.0) {
                set_error("pd_solve_static: non-finite CG scalar");
                return PD_ERR_NONFINITE;
            }
            if (hbuf[S_FLAG] == 2.0 || rn <= tol_abs) break;
            // stagnation of the recursive residual (FP32 attainable accuracy)
            if (rn < 0.999 * best) {
                best = rn;
                since_best = 0;
            } else if ((since_best += chunk) >= 8 * kCheck) {
                break;
            }
        }
        *done = it;
        return PD_OK;
    }
};

}  // namespace
}  // namespace pd

using namespace pd;

extern "C" pd_status pd_solve_static(pd_plan *p, double *u, const double *b, const double *w, double rtol,
                                     int max_iter, int *iters_out, double *relres_out, void *stream)
{
    if (!p || !u || !b) {
        set_error("pd_solve_static: null plan, u or b");
        return PD_ERR_ARG;
    }
    if (!(rtol > 0) || max_iter < 1) {
        set_error("pd_solve_static: rtol must be > 0 and max_iter >= 1");
        return PD_ERR_ARG;
    }
    Solver S;
    S.p = p;
    S.st = (cudaStream_t)stream;
    S.nvec = (int64_t)p->dim * p->N;
    S.nb = red_blocks(p);
    PD_CUDA_TRY(cudaMallocHost((void **)&S.hbuf, sizeof(double) * S_COUNT));
    struct HostFree {
        double *h;
        ~HostFree() { cudaFreeHost(h); }
    } hf{S.hbuf};
    PD_CUDA_TRY(cudaMemsetAsync(p->red + RED_SCAL, 0, sizeof(double) * S_COUNT, S.st));
    k_apply_bc<<<S.nb, 256, 0, S.st>>>(u, w, b, p->chi_om, S.nvec, p->red);
    PD_LAUNCH_CHECK();
    p->launches++;
    PD_TRY(S.finish(S_BN, 0));
    PD_TRY(S.read_scalars());
    const double bn = std::sqrt(S.hbuf[S_BN]);
    int total = 0;
    double rel = 0.0;
    pd_status result = PD_ERR_NOT_CONVERGED;
    const double target = rtol * (bn > 0 ? bn : 1.0);
    for (int outer = 0; outer < 64; ++outer) {
        double rn = 0.0;
        PD_TRY(S.residual(u, b, &rn));
        rel = bn > 0 ? rn / bn : rn;
        if (rn <= target) {
            result = PD_OK;
            break;
        }
        if (total >= max_iter) break;
        int done = 0;
        double rlast = 0.0;
        if (p->prob.fp64) {
            PD_TRY(S.cg<double>(0.5 * target, max_iter - total, &done, &rlast));
            total += done;
            k_ir_update<double><<<S.nb, 256, 0, S.st>>>(u, (const double *)p->cg_e, p->chi_om, S.nvec);
        } else {
            // inner FP32 solve: reduce the residual by 1e-3 (the FP32 operator
            // resolves A e to about that accuracy), never below the target
            const double tol = std::max(1e-3 * rn, 0.5 * target);
            PD_TRY(S.cg<float>(tol, max_iter - total, &done, &rlast));
            total += done;
            k_ir_update<float><<<S.nb, 256, 0, S.st>>>(u, (const float *)p->cg_e, p->chi_om, S.nvec);
        }
        PD_LAUNCH_CHECK();
        p->launches++;
        if (done == 0) break;
    }
    PD_CUDA_TRY(cudaStreamSynchronize(S.st));
    if (iters_out) *iters_out = total;
    if (relres_out) *relres_out = rel;
    if (result != PD_OK) set_error("pd_solve_static: relative residual %.3e above rtol %.3e after %d iterations",
                                   rel, rtol, total);
    return result;
}
