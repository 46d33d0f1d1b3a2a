// pd_solve_mirror: the static problem with mirror-based volume constraints.
//
// §5.1 contrasts the naive fictitious-node constraint (u = g on the whole
// boundary layer Gamma) with a mirror-based one that the paper describes but
// whose appendix is not in its text: each Gamma node takes its value from the
// local boundary value g and the solution at its mirror point inside Omega,
//   u(x) = 2 g(x) - u(x_m)      on Gamma,
//   chi_O (L(u) + b) = 0         on Omega   (Eq. 89),
// updated as the solution changes. Written in the Omega values e alone,
// u = E e + h with (E e) = chi_O e - (1 - chi_O) e(mirror) and h = 2 (1 - chi_O) g,
// the problem is the linear system A e = r0 with
//   A e = -chi_O L(E e),   r0 = chi_O (L(h) + b).
// A is not symmetric (the mirror coupling is one-sided), so the solver is
// BiCGStab (van der Vorst 1992) instead of CG. Every matrix-vector product is
// one FCBM-EC force evaluation of the expanded field; inner products and the
// iteration are FP64 (FP64 plans).
#include <algorithm>
#include <cmath>
#include <vector>

#include "pd_force_impl.cuh"

namespace pd {
namespace {

constexpr int kMirBlocks = 512;

// u = E e + (with h) h: Omega values, minus the mirror value on Gamma, 0 off the body
__global__ void k_mir_expand(const double *e, const int *mirror, const uint8_t *co, const uint8_t *chi,
                             const double *g, double *u, int d, int64_t N)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < d; ++c) {
            const int64_t q = c * N + p;
            double v = 0.0;
            if (co[q]) {
                v = e ? e[q] : 0.0;
            } else if (chi[p]) {
                const int m = mirror[q];
                v = (e ? -e[c * N + m] : 0.0) + (g ? 2.0 * g[q] : 0.0);
            }
            u[q] = v;
        }
    }
}

// y = -chi_O L  (or chi_O (L + b) with b) ; partial of y.y
__global__ void k_mir_mask(const double *L, const double *b, const uint8_t *co, double *y, int64_t n, double sign,
                           double *part)
{
    double acc = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const double v = co[q] ? sign * (L[q] + (b ? b[q] : 0.0)) : 0.0;
        y[q] = v;
        acc += v * v;
    }
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// partials of (a, b) and (c, d)
__global__ void k_mir_dot2(const double *a, const double *b, const double *c, const double *dd, int64_t n,
                           double *part)
{
    double x = 0.0, y = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        x += a[q] * b[q];
        if (c) y += c[q] * dd[q];
    }
    x = block_sum_d(x);
    y = block_sum_d(y);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = x;
        part[kMirBlocks + blockIdx.x] = y;
    }
}

// p = r + beta (p - omega v)
__global__ void k_mir_dir(double *p, const double *r, const double *v, int64_t n, double beta, double omega)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        p[q] = r[q] + beta * (p[q] - omega * v[q]);
}

// s = r - alpha v
__global__ void k_mir_axpy(double *s, const double *r, const double *v, int64_t n, double alpha)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        s[q] = r[q] - alpha * v[q];
}

// x += alpha p + omega s ; r = s - omega t
__global__ void k_mir_update(double *x, double *r, const double *p, const double *s, const double *t, int64_t n,
                             double alpha, double omega)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        x[q] += alpha * p[q] + omega * s[q];
        r[q] = s[q] - omega * t[q];
    }
}

// mirror indices: every Gamma node (chi = 1, chi_O = 0) needs one in [0, N)
// whose node is in Omega for that component
__global__ void k_mir_check(const int *mirror, const uint8_t *co, const uint8_t *chi, int d, int64_t N, int *bad)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        if (!chi[p]) continue;
        for (int c = 0; c < d; ++c) {
            if (co[c * N + p]) continue;
            const int m = mirror[c * N + p];
            if (m < 0 || (int64_t)m >= N || !co[c * N + m]) atomicOr(bad, 1);
        }
    }
}

struct Mirror {
    pd_plan *p;
    cudaStream_t st;
    int64_t n;
    double *part;
    std::vector<double> h;

    double sum(int k)
    {
        double s = 0.0;
        for (int i = 0; i < kMirBlocks; ++i) s += h[(size_t)k * kMirBlocks + i];
        return s;
    }
    pd_status fetch(int cnt)
    {
        PD_CUDA_TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * cnt * kMirBlocks, cudaMemcpyDeviceToHost, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        return PD_OK;
    }
    // y = A x = -chi_O L(E x); returns ||y||^2 partials in part
    pd_status apply(const double *x, const int *mirror, double *y, double *ufull, double *L)
    {
        k_mir_expand<<<kMirBlocks, 256, 0, st>>>(x, mirror, p->chi_om, p->chi, nullptr, ufull, p->dim, p->N);
        PD_LAUNCH_CHECK();
        PD_TRY(force_plain<double>(p, ufull, nullptr, L, nullptr, st));
        k_mir_mask<<<kMirBlocks, 256, 0, st>>>(L, nullptr, p->chi_om, y, n, -1.0, part);
        PD_LAUNCH_CHECK();
        p->launches += 2;
        return PD_OK;
    }
    pd_status dot2(const double *a, const double *b, const double *c, const double *d, double *x, double *y)
    {
        k_mir_dot2<<<kMirBlocks, 256, 0, st>>>(a, b, c, d, n, part);
        PD_LAUNCH_CHECK();
        p->launches++;
        PD_TRY(fetch(2));
        *x = sum(0);
        if (y) *y = sum(1);
        return PD_OK;
    }
};

}  // namespace
}  // namespace pd

using namespace pd;

extern "C" pd_status pd_solve_mirror(pd_plan *p, double *u, const double *b, const double *g, const int32_t *mirror,
                                     double rtol, int max_iter, int *iters_out, double *relres_out, void *stream)
{
    if (!p || !u || !mirror) {
        set_error("pd_solve_mirror: null plan, u or mirror");
        return PD_ERR_ARG;
    }
    if (!p->prob.fp64 || p->nonlinear) {
        set_error("pd_solve_mirror: FP64 plans of the linearized models only");
        return PD_ERR_ARG;
    }
    if (!(rtol > 0) || max_iter < 1) {
        set_error("pd_solve_mirror: rtol must be > 0 and max_iter >= 1");
        return PD_ERR_ARG;
    }
    Mirror M;
    M.p = p;
    M.st = (cudaStream_t)stream;
    M.n = (int64_t)p->dim * p->N;
    M.part = p->red + kRedPart;
    M.h.assign(2 * kMirBlocks, 0.0);
    const cudaStream_t st = M.st;
    const int64_t n = M.n;
    {
        int *bad = reinterpret_cast<int *>(p->red + kRedScal);
        PD_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
        k_mir_check<<<kMirBlocks, 256, 0, st>>>(mirror, p->chi_om, p->chi, p->dim, p->N, bad);
        PD_LAUNCH_CHECK();
        int hb = 0;
        PD_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        if (hb) {
            set_error("pd_solve_mirror: every Gamma node needs a mirror node inside Omega");
            return PD_ERR_ARG;
        }
    }
    // vectors (d x N doubles): the plan's solver vectors, its residual and
    // weight-field buffers, and for t one run of FP64 spectrum slots from 14 on
    // (the force passes use slots 0-7 at most); the expanded field lives in u
    double *x = (double *)p->cg_e, *r = (double *)p->cg_r, *pp = (double *)p->cg_p, *v = (double *)p->cg_q;
    double *rh = p->r64, *sv = (double *)p->Gw;
    double *tv = (double *)p->spec64 + (size_t)14 * p->N;
    if (p->spec64_slots < 14 + p->dim) {
        set_error("pd_solve_mirror: plan has too few FP64 spectrum slots");
        return PD_ERR_ARG;
    }
    // r0 = chi_O (L(h) + b), h = 2 (1 - chi_O) g on Gamma
    k_mir_expand<<<kMirBlocks, 256, 0, st>>>(nullptr, mirror, p->chi_om, p->chi, g, u, p->dim, p->N);
    PD_LAUNCH_CHECK();
    PD_TRY(force_plain<double>(p, u, nullptr, r, nullptr, st));
    k_mir_mask<<<kMirBlocks, 256, 0, st>>>(r, b, p->chi_om, r, n, 1.0, M.part);
    PD_LAUNCH_CHECK();
    p->launches += 2;
    PD_TRY(M.fetch(1));
    const double r0n = std::sqrt(M.sum(0));
    if (!std::isfinite(r0n)) {
        set_error("pd_solve_mirror: non-finite right-hand side");
        return PD_ERR_NONFINITE;
    }
    PD_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    PD_CUDA_TRY(cudaMemcpyAsync(rh, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    PD_CUDA_TRY(cudaMemsetAsync(pp, 0, sizeof(double) * n, st));
    PD_CUDA_TRY(cudaMemsetAsync(v, 0, sizeof(double) * n, st));
    double rho = 1.0, alpha = 1.0, omega = 1.0, rn = r0n;
    int it = 0;
    pd_status result = PD_ERR_NOT_CONVERGED;
    const double target = rtol * (r0n > 0 ? r0n : 1.0);
    if (r0n == 0.0) result = PD_OK;
    // BiCGStab
    while (result != PD_OK && it < max_iter) {
        double rho_new = 0.0;
        PD_TRY(M.dot2(rh, r, nullptr, nullptr, &rho_new, nullptr));
        if (!(std::fabs(rho_new) > 0) || !std::isfinite(rho_new)) break;  // breakdown
        const double beta = (rho_new / rho) * (alpha / omega);
        k_mir_dir<<<kMirBlocks, 256, 0, st>>>(pp, r, v, n, beta, omega);
        PD_LAUNCH_CHECK();
        PD_TRY(M.apply(pp, mirror, v, u, v));
        double rv = 0.0;
        PD_TRY(M.dot2(rh, v, nullptr, nullptr, &rv, nullptr));
        if (!(std::fabs(rv) > 0) || !std::isfinite(rv)) break;
        alpha = rho_new / rv;
        k_mir_axpy<<<kMirBlocks, 256, 0, st>>>(sv, r, v, n, alpha);
        PD_LAUNCH_CHECK();
        PD_TRY(M.apply(sv, mirror, tv, u, tv));
        double ts = 0.0, tt = 0.0;
        PD_TRY(M.dot2(tv, sv, tv, tv, &ts, &tt));
        omega = tt > 0 ? ts / tt : 0.0;
        k_mir_update<<<kMirBlocks, 256, 0, st>>>(x, r, pp, sv, tv, n, alpha, omega);
        PD_LAUNCH_CHECK();
        p->launches += 3;
        double rr = 0.0;
        PD_TRY(M.dot2(r, r, nullptr, nullptr, &rr, nullptr));
        rn = std::sqrt(rr);
        rho = rho_new;
        ++it;
        if (!std::isfinite(rn)) {
            set_error("pd_solve_mirror: non-finite residual");
            return PD_ERR_NONFINITE;
        }
        if (rn <= target) result = PD_OK;
        if (!(omega != 0.0)) break;
    }
    // u = E x + h and its true FP64 residual chi_O (L(u) + b), relative to ||r0||
    k_mir_expand<<<kMirBlocks, 256, 0, st>>>(x, mirror, p->chi_om, p->chi, g, u, p->dim, p->N);
    PD_LAUNCH_CHECK();
    PD_TRY(force_plain<double>(p, u, nullptr, r, nullptr, st));
    k_mir_mask<<<kMirBlocks, 256, 0, st>>>(r, b, p->chi_om, r, n, 1.0, M.part);
    PD_LAUNCH_CHECK();
    p->launches += 2;
    PD_TRY(M.fetch(1));
    const double rel = std::sqrt(M.sum(0)) / (r0n > 0 ? r0n : 1.0);
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = rel;
    if (result != PD_OK || !(rel <= 2 * rtol)) {
        set_error("pd_solve_mirror: relative residual %.3e above rtol %.3e after %d iterations", rel, rtol, it);
        return PD_ERR_NOT_CONVERGED;
    }
    return PD_OK;
}
