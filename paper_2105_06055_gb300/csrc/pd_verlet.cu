// pd_step_verlet: FCBM-EC dynamics with energy-based bond breaking.
//
// Per step (Eq. 83-84 for the kinematics, Eq. 63 for the integrity index,
// Eq. 101-102 for L and W with node weight chi_B lam):
//   kick+drift : v <- v + dt/(2 rho) (L^n + b);  u <- chi_O (u + dt v) + (1 - chi_O) w;
//                lam <- lam [W^n <= Wc]  (irreversible; counts 1 -> 0 flips)
//   G^lam      : recomputed on the device only if some lam flipped this step
//   force      : L^{n+1}, W^{n+1} = FFT convolutions with weight chi_B lam
//   kick       : v <- chi_O (v + dt/(2 rho) (L^{n+1} + b))
// The call starts with one force evaluation of the given state, so a run of
// n steps split over several calls gives the same result as one call.
//
// Energy mode 1 (pd_plan_set_energy_mode) evaluates W of Eq. 102 by the plain
// horizon sum of Eq. 47 instead of the three convolutions T1 - 2 u.(C*(v u))
// + u.(C*v) u: the convolutions' rounding error is global, about
// eps lambda_max (rms|u|^2 + 2 |u(x)| rms|u|) at every node, which in FP32
// exceeds Wc once fragments have moved far (|u| ~ 10-100 grid units), while
// the direct sum errs by about eps |u(x)| / |eta| relative to W, locally.
#include <algorithm>
#include <cmath>

#include "pd_ops.cuh"
#include "pd_plan.cuh"

namespace pd {

template <typename T>
pd_status force_any(pd_plan *p, const T *u, const T *s, const uint8_t *lam, const T *G, T *L, T *W,
                    cudaStream_t st);

namespace {

// device counters live in the reduction buffer: [0] flips (int64), [1] flag
struct VerletCounters {
    unsigned long long flips;
    int changed;
};

// Gamma values at the end of the step: w + t_next w1 (w1 null: w, constant)
template <typename T>
__global__ void k_kick_drift(T *u, T *v, uint8_t *lam, const T *L, const T *b, const T *w, const T *w1, T t_next,
                             const T *W, const uint8_t *chi, const uint8_t *co, int d, int64_t N, T hdt_rho, T dt,
                             T Wc, int breaking, VerletCounters *cnt)
{
    unsigned long long flips = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        for (int i = 0; i < d; ++i) {
            const int64_t q = i * N + p;
            const T vh = v[q] + hdt_rho * (L[q] + b[q]);
            v[q] = vh;
            T g = w ? w[q] : T(0);
            if (w1) g = g + t_next * w1[q];
            u[q] = co[q] ? (u[q] + dt * vh) : g;
        }
        if (breaking && chi[p] && lam[p] && !(W[p] <= Wc)) {
            lam[p] = 0;
            ++flips;
        }
    }
    // warp-aggregated counter update
    for (int o = 16; o > 0; o >>= 1) flips += __shfl_down_sync(0xffffffffu, flips, o);
    if ((threadIdx.x & 31) == 0 && flips) {
        atomicAdd(&cnt->flips, flips);
        atomicExch(&cnt->changed, 1);
    }
}

template <typename T>
__global__ void k_kick(T *v, const T *L, const T *b, const uint8_t *co, int64_t n, T hdt_rho)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        v[q] = co[q] ? v[q] + hdt_rho * (L[q] + b[q]) : T(0);
}

// G^lam_c(x) = Σ_H C_c dV (v(x+xi) - v(x)), v = chi lam; skipped unless the
// change flag is set by this step's kick-drift (k_clear_changed resets it).
template <typename T>
__global__ void k_gfield_lam(int n1, int n2, int n3, HorizonDev hz, int ncomp, const uint8_t *chi,
                             const uint8_t *lam, T *G, int64_t N, VerletCounters *cnt, int force)
{
    if (!force && !cnt->changed) return;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N) {
        int i1, i2, i3;
        node_coords(p, n1, n2, i1, i2, i3);
        T acc[6] = {0, 0, 0, 0, 0, 0};
        if (chi[p]) {
            const T vp = lam[p] ? T(1) : T(0);
            for (int c = 0; c < hz.cnt; ++c) {
                const int a = (i1 + hz.off[3 * c]) & (n1 - 1);
                const int bb = (i2 + hz.off[3 * c + 1]) & (n2 - 1);
                const int e = (i3 + hz.off[3 * c + 2]) & (n3 - 1);
                const int64_t q = ((int64_t)e * n2 + bb) * n1 + a;
                const T dv = ((chi[q] && lam[q]) ? T(1) : T(0)) - vp;
                if (dv != T(0))
                    for (int k = 0; k < ncomp; ++k) acc[k] += (T)hz.c[k * hz.cnt + c] * dv;
            }
        }
        for (int k = 0; k < ncomp; ++k) G[k * N + p] = acc[k];
    }
}

__global__ void k_clear_changed(VerletCounters *cnt) { cnt->changed = 0; }

// W(x) = 1/2 chi lam Σ_H chi' lam' eta.C(xi).eta dV, eta = u(x+xi) - u(x)
// (Eq. 47 with the integrity weights of Eq. 44; periodic neighbour offsets).
// The bond tensor is rank one, C(xi) dV = c(xi) xi xi^T / |xi|^2 with
// c = tr C dV, so each bond adds c (xi.eta)^2 / |xi|^2: the projection is
// formed first, and a rigidly rotating neighbourhood (large eta nearly
// normal to xi) does not cancel large quadratic-form terms.
template <typename T, int D>
__global__ void k_energy_direct(int n1, int n2, int n3, HorizonDev hz, double dx1, double dx2, double dx3,
                                const uint8_t *chi, const uint8_t *lam, const T *u, T *W, int64_t N)
{
    constexpr int NC = Sym<D>::n;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *ws = reinterpret_cast<T *>(sm_raw);            // cnt: c / |xi|^2
    T *xs = ws + hz.cnt;                               // D x cnt: xi
    int *os = reinterpret_cast<int *>(xs + D * hz.cnt);  // 3 x cnt
    for (int c = threadIdx.x; c < hz.cnt; c += blockDim.x) {
        const double x[3] = {hz.off[3 * c] * dx1, hz.off[3 * c + 1] * dx2, hz.off[3 * c + 2] * dx3};
        double tr = 0.0, r2 = 0.0;
        for (int k = 0; k < NC; ++k)
            if (Sym<D>::i(k) == Sym<D>::j(k)) tr += hz.c[k * hz.cnt + c];
        for (int j = 0; j < D; ++j) r2 += x[j] * x[j];
        ws[c] = (T)(tr / r2);
        for (int j = 0; j < D; ++j) xs[j * hz.cnt + c] = (T)x[j];
        for (int j = 0; j < 3; ++j) os[3 * c + j] = hz.off[3 * c + j];
    }
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        T acc = T(0);
        if (chi[p] && lam[p]) {
            int i1, i2, i3;
            node_coords(p, n1, n2, i1, i2, i3);
            T up[D];
#pragma unroll
            for (int j = 0; j < D; ++j) up[j] = u[j * N + p];
            for (int c = 0; c < hz.cnt; ++c) {
                const int a = (i1 + os[3 * c]) & (n1 - 1);
                const int b = (i2 + os[3 * c + 1]) & (n2 - 1);
                const int e = (i3 + os[3 * c + 2]) & (n3 - 1);
                const int64_t q = ((int64_t)e * n2 + b) * n1 + a;
                if (!(chi[q] && lam[q])) continue;
                T s = T(0);
#pragma unroll
                for (int j = 0; j < D; ++j) s += xs[j * hz.cnt + c] * (u[j * N + q] - up[j]);
                acc += ws[c] * s * s;
            }
        }
        W[p] = T(0.5) * acc;
    }
}

template <typename T>
pd_status energy_direct(pd_plan *p, const T *u, const uint8_t *lam, T *W, cudaStream_t st)
{
    const int cnt = p->hdev.cnt;
    const size_t smem = (size_t)(1 + p->dim) * cnt * sizeof(T) + (size_t)3 * cnt * sizeof(int);
    const double *dx = p->prob.dx;
    const unsigned ng = (unsigned)std::min<int64_t>(8 * p->nsm, (p->N + 255) / 256);
    if (p->dim == 3) {
        PD_TRY(set_smem_attr((const void *)k_energy_direct<T, 3>, smem));
        k_energy_direct<T, 3><<<ng, 256, smem, st>>>(p->n1, p->n2, p->n3, p->hdev, dx[0], dx[1], dx[2], p->chi, lam,
                                                     u, W, p->N);
    } else {
        PD_TRY(set_smem_attr((const void *)k_energy_direct<T, 2>, smem));
        k_energy_direct<T, 2><<<ng, 256, smem, st>>>(p->n1, p->n2, p->n3, p->hdev, dx[0], dx[1], dx[2], p->chi, lam,
                                                     u, W, p->N);
    }
    PD_LAUNCH_CHECK();
    p->launches++;
    return PD_OK;
}

// one force evaluation of the step, with W in the plan's energy mode
template <typename T>
pd_status step_force(pd_plan *p, const T *u, const uint8_t *lam, const T *G, T *L, T *W, int breaking,
                     cudaStream_t st)
{
    if (breaking && p->energy_direct) {
        PD_TRY(force_any<T>(p, u, nullptr, lam, G, L, nullptr, st));
        return energy_direct<T>(p, u, lam, W, st);
    }
    return force_any<T>(p, u, nullptr, lam, G, L, breaking ? W : nullptr, st);
}

template <typename T>
pd_status verlet_impl(pd_plan *p, T *u, T *v, uint8_t *lam, const T *b, const T *w, const T *w1, double t0,
                      double dt, int nsteps, int64_t *n_broken_out, cudaStream_t st)
{
    const int d = p->dim;
    const int64_t N = p->N;
    T *L = (T *)p->cg_q;
    T *W = (T *)p->theta;
    T *G = lam ? (T *)p->Gw : (sizeof(T) == 8 ? (T *)p->G64 : (T *)p->G32);
    const int breaking = (lam && p->wc > 0) ? 1 : 0;
    VerletCounters *cnt = reinterpret_cast<VerletCounters *>(p->red + kRedVerlet);
    PD_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(VerletCounters), st));
    const unsigned nbl = (unsigned)((N + 127) / 128);
    if (lam) {
        k_gfield_lam<T><<<nbl, 128, 0, st>>>(p->n1, p->n2, p->n3, p->hdev, p->ncomp, p->chi, lam, G, N, cnt, 1);
        PD_LAUNCH_CHECK();
        p->launches++;
    }
    PD_TRY(step_force<T>(p, u, lam, G, L, W, breaking, st));
    const T hdt = (T)(0.5 * dt / p->prob.rho);
    const unsigned ng = (unsigned)std::min<int64_t>(4 * p->nsm, (N + 255) / 256);
    const unsigned ngv = (unsigned)std::min<int64_t>(4 * p->nsm, (d * N + 255) / 256);
    for (int s = 0; s < nsteps; ++s) {
        const T t_next = (T)(t0 + (double)(s + 1) * dt);
        k_kick_drift<T><<<ng, 256, 0, st>>>(u, v, lam, L, b, w, w1, t_next, W, p->chi, p->chi_om, d, N, hdt,
                                            (T)dt, (T)p->wc, breaking, cnt);
        PD_LAUNCH_CHECK();
        p->launches++;
        if (breaking) {
            k_gfield_lam<T><<<nbl, 128, 0, st>>>(p->n1, p->n2, p->n3, p->hdev, p->ncomp, p->chi, lam, G, N, cnt, 0);
            k_clear_changed<<<1, 1, 0, st>>>(cnt);
            PD_LAUNCH_CHECK();
            p->launches += 2;
        }
        PD_TRY(step_force<T>(p, u, lam, G, L, W, breaking, st));
        k_kick<T><<<ngv, 256, 0, st>>>(v, L, b, p->chi_om, d * N, hdt);
        PD_LAUNCH_CHECK();
        p->launches++;
    }
    if (n_broken_out) {
        VerletCounters h;
        PD_CUDA_TRY(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        *n_broken_out = (int64_t)h.flips;
    }
    return PD_OK;
}

}  // namespace
}  // namespace pd

using namespace pd;

static pd_status verlet_entry(pd_plan *p, void *u, void *v, uint8_t *lambda, const void *b, const void *w,
                              const void *w1, double t0, double dt, int nsteps, int64_t *n_broken_out, void *stream,
                              const char *who)
{
    if (!p || !u || !v || !b) {
        set_error("%s: null plan, u, v or b", who);
        return PD_ERR_ARG;
    }
    if (!(dt > 0) || nsteps < 0 || !(p->prob.rho > 0) || !std::isfinite(t0)) {
        set_error("%s: dt and rho must be positive, nsteps >= 0, t0 finite", who);
        return PD_ERR_ARG;
    }
    if (p->state_based || p->nonlinear) {
        set_error("%s: the dynamic driver uses the linearized bond model", who);
        return PD_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (p->prob.fp64)
        return verlet_impl<double>(p, (double *)u, (double *)v, lambda, (const double *)b, (const double *)w,
                                   (const double *)w1, t0, dt, nsteps, n_broken_out, st);
    return verlet_impl<float>(p, (float *)u, (float *)v, lambda, (const float *)b, (const float *)w,
                              (const float *)w1, t0, dt, nsteps, n_broken_out, st);
}

extern "C" pd_status pd_step_verlet(pd_plan *p, void *u, void *v, uint8_t *lambda, const void *b, const void *w,
                                    double dt, int nsteps, int64_t *n_broken_out, void *stream)
{
    return verlet_entry(p, u, v, lambda, b, w, nullptr, 0.0, dt, nsteps, n_broken_out, stream, "pd_step_verlet");
}

extern "C" pd_status pd_step_verlet_ramp(pd_plan *p, void *u, void *v, uint8_t *lambda, const void *b,
                                         const void *w0, const void *w1, double t0, double dt, int nsteps,
                                         int64_t *n_broken_out, void *stream)
{
    if (!w1) {
        set_error("pd_step_verlet_ramp: w1 is required (use pd_step_verlet for a constant w)");
        return PD_ERR_ARG;
    }
    return verlet_entry(p, u, v, lambda, b, w0, w1, t0, dt, nsteps, n_broken_out, stream, "pd_step_verlet_ramp");
}

extern "C" pd_status pd_plan_set_energy_mode(pd_plan *p, int mode)
{
    if (!p || (mode != 0 && mode != 1)) {
        set_error("pd_plan_set_energy_mode: null plan or mode not 0/1");
        return PD_ERR_ARG;
    }
    p->energy_direct = mode;
    return PD_OK;
}
