// pd_verlet_loss_grad: a loss on the final state of FCBM-EC dynamics with bond
// breaking and its gradient with respect to a spatially varying micromodulus.
//
// Forward (Eq. 83-84 with w = 0, the energy-based breaking of Eq. 63, bond
// factor (s lam)(s' lam') with s = sqrt(c / c0), reading R17 of Eq. 44):
//   a^n       = L(u^n; s lam^n) + b  [+ b0 at n = 0]
//   v^h       = v^n + h a^n,  h = dt / (2 rho)
//   u^{n+1}   = chi_O (u^n + dt v^h)
//   lam^{n+1} = lam^n [W(u^n; s lam^n) <= Wc]
//   v^{n+1}   = chi_O (v^h + h a^{n+1})
//   J         = Σ |u^N - u_T|^2
// The breaking decisions are piecewise constant in c, so the gradient is that
// of the dynamics with the integrity history lam^0 .. lam^N held fixed (the
// derivative wherever no decision changes). Reverse sweep, with the two
// adjoint force applications at each state u^n merged (both act on the same
// cotangent v~^n):
//   u~ = 2 chi_O (u^N - u_T),  v~ = 0
//   for n = N-1 .. 0:
//     v~ = chi_O (v~ + dt u~)
//     (g_u, g_s) = adjoint of L(. ; s lam^n) at u^n against k v~   (k = 2h, or h at n = 0)
//     u~ = chi_O (u~ + g_u),   s~ += g_s lam^n
//   dJ/dc = s~ / (2 c0 s)
// The states u^n, lam^n of the reverse sweep come from checkpoints (u, v, lam)
// every K steps, recomputed forward one segment at a time (memory: one state
// per checkpoint plus K states of one segment, in a caller-provided workspace).
// The adjoint of the force is the fused pass of pd_force_adjoint: the operator
// is symmetric for every weight, and its derivative with respect to the weight
// comes from the same transforms.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pd_ops.cuh"
#include "pd_plan.cuh"

namespace pd {

template <typename T>
pd_status force_any(pd_plan *p, const T *u, const T *s, const uint8_t *lam, const T *G, T *L, T *W,
                    cudaStream_t st);
template <typename T>
pd_status adjoint_weighted(pd_plan *p, const T *u, const T *s, const T *pv, const T *G, T *gu, T *gs,
                           cudaStream_t st);

namespace {

struct AdjCounters {
    unsigned long long flips;
    int changed;  // the integrity index changed: the boundary field of the weight is stale
    int bad;      // a micromodulus value was not positive and finite
};

// s = sqrt(c_rel) (bad flag for c_rel <= 0 or non-finite), lam = lam0 or 1
template <typename T>
__global__ void k_adj_init(const T *c_rel, T *s, const uint8_t *lam0, uint8_t *lam, int64_t N, AdjCounters *cnt)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        const T c = c_rel[p];
        if (!(c > T(0)) || !isfinite(c)) atomicOr(&cnt->bad, 1);
        s[p] = c > T(0) ? sqrt(c) : T(0);
        lam[p] = lam0 ? (lam0[p] ? 1 : 0) : 1;
    }
}

// s_eff = s lam
template <typename T>
__global__ void k_adj_weight(const T *s, const uint8_t *lam, T *s_eff, int64_t N)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
        s_eff[p] = lam[p] ? s[p] : T(0);
}

// boundary field of the weight v = chi s_eff (as k_gfield), skipped unless flagged
template <typename T>
__global__ void k_adj_gfield(int n1, int n2, int n3, HorizonDev hz, int ncomp, const uint8_t *chi, const T *s,
                             T *G, int64_t N, const AdjCounters *cnt)
{
    if (!cnt->changed) return;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int i1, i2, i3;
    node_coords(p, n1, n2, i1, i2, i3);
    T acc[6] = {0, 0, 0, 0, 0, 0};
    if (chi[p]) {
        const T vp = s[p];
        for (int c = 0; c < hz.cnt; ++c) {
            const int a = (i1 + hz.off[3 * c]) & (n1 - 1);
            const int b = (i2 + hz.off[3 * c + 1]) & (n2 - 1);
            const int e = (i3 + hz.off[3 * c + 2]) & (n3 - 1);
            const int64_t q = ((int64_t)e * n2 + b) * n1 + a;
            const T dv = (chi[q] ? s[q] : T(0)) - vp;
            if (dv != T(0))
                for (int k = 0; k < ncomp; ++k) acc[k] += (T)hz.c[k * hz.cnt + c] * dv;
        }
    }
    for (int k = 0; k < ncomp; ++k) G[k * N + p] = acc[k];
}

__global__ void k_adj_flag(AdjCounters *cnt, int v) { cnt->changed = v; }

// first half of a step: v^h = v + h (L + b [+ b0]); u = chi_O (u + dt v^h);
// lam <- lam [W <= Wc] (counts flips, flags a change)
template <typename T>
__global__ void k_adj_kick_drift(T *u, T *v, uint8_t *lam, const T *L, const T *b, const T *b0, const T *W,
                                 const uint8_t *chi, const uint8_t *co, int d, int64_t N, T h, T dt, T Wc,
                                 int breaking, AdjCounters *cnt)
{
    unsigned long long flips = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        for (int i = 0; i < d; ++i) {
            const int64_t q = i * N + p;
            T a = L[q];
            if (b) a += b[q];
            if (b0) a += b0[q];
            const T vh = v[q] + h * a;
            v[q] = vh;
            u[q] = co[q] ? u[q] + dt * vh : T(0);
        }
        if (breaking && chi[p] && lam[p] && !(W[p] <= Wc)) {
            lam[p] = 0;
            ++flips;
        }
    }
    for (int o = 16; o > 0; o >>= 1) flips += __shfl_down_sync(0xffffffffu, flips, o);
    if ((threadIdx.x & 31) == 0 && flips) {
        atomicAdd(&cnt->flips, flips);
        atomicExch(&cnt->changed, 1);
    }
}

// second half: v = chi_O (v^h + h (L + b))
template <typename T>
__global__ void k_adj_kick(T *v, const T *L, const T *b, const uint8_t *co, int64_t n, T h)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        v[q] = co[q] ? v[q] + h * (L[q] + (b ? b[q] : T(0))) : T(0);
}

// loss partials Σ (u - u_T)^2 (FP64) and u~ = 2 chi_O (u - u_T)
template <typename T>
__global__ void k_adj_loss(const T *u, const T *ut, const uint8_t *co, T *ubar, int64_t n, double *part)
{
    double acc = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const T e = u[q] - ut[q];
        acc += (double)e * (double)e;
        ubar[q] = co[q] ? T(2) * e : T(0);
    }
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// v~ = chi_O (v~ + dt u~)
template <typename T>
__global__ void k_adj_vbar(T *vbar, const T *ubar, const uint8_t *co, int64_t n, T dt)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        vbar[q] = co[q] ? vbar[q] + dt * ubar[q] : T(0);
}

// u~ = chi_O (u~ + g_u) ; s~ += g_s lam  (g_u, g_s already for the cotangent k v~)
template <typename T>
__global__ void k_adj_acc(T *ubar, const T *gu, T *sbar, const T *gs, const uint8_t *lam, const uint8_t *co,
                          int d, int64_t N)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        for (int i = 0; i < d; ++i) {
            const int64_t q = i * N + p;
            ubar[q] = co[q] ? ubar[q] + gu[q] : T(0);
        }
        if (lam[p]) sbar[p] += gs[p];
    }
}

// x = k x (the cotangent of the adjoint force application)
template <typename T>
__global__ void k_adj_scale(const T *x, T *y, int64_t n, T k)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        y[q] = k * x[q];
}

// dJ/dc_rel = s~ / (2 s)
template <typename T>
__global__ void k_adj_grad_c(const T *sbar, const T *s, T *g, int64_t N)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
        g[p] = s[p] > T(0) ? sbar[p] / (T(2) * s[p]) : T(0);
}

struct AdjLayout {
    size_t s, u, v, ubar, vbar, sbar, lam, ck_u, ck_v, ck_lam, sg_u, sg_lam, total;
    int ncp, K;
};

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

AdjLayout adj_layout(const pd_plan *p, int nsteps, int K)
{
    AdjLayout a{};
    const size_t tb = p->prob.fp64 ? 8 : 4;
    const size_t N = (size_t)p->N, dN = (size_t)p->dim * N;
    a.K = K;
    a.ncp = (nsteps + K - 1) / K;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += up256(bytes);
        return at;
    };
    a.s = take(tb * N);
    a.u = take(tb * dN);
    a.v = take(tb * dN);
    a.ubar = take(tb * dN);
    a.vbar = take(tb * dN);
    a.sbar = take(tb * N);
    a.lam = take(N);
    a.ck_u = take(tb * dN * a.ncp);
    a.ck_v = take(tb * dN * a.ncp);
    a.ck_lam = take(up256(N) * a.ncp);
    a.sg_u = take(tb * dN * K);
    a.sg_lam = take(up256(N) * K);
    a.total = o;
    return a;
}

template <typename T>
struct AdjRun {
    pd_plan *p;
    cudaStream_t st;
    AdjLayout lay;
    unsigned char *w;
    T *s, *u, *v, *ubar, *vbar, *sbar;
    uint8_t *lam;
    T *L, *W, *G, *seff, *gu, *gs;
    const T *b, *b0;
    AdjCounters *cnt;
    T h, dt;
    int breaking;
    unsigned ng, ngv, nbl;

    T *ck_u(int k) const { return (T *)(w + lay.ck_u) + (size_t)k * p->dim * p->N; }
    T *ck_v(int k) const { return (T *)(w + lay.ck_v) + (size_t)k * p->dim * p->N; }
    uint8_t *ck_lam(int k) const { return w + lay.ck_lam + (size_t)k * up256(p->N); }
    T *sg_u(int k) const { return (T *)(w + lay.sg_u) + (size_t)k * p->dim * p->N; }
    uint8_t *sg_lam(int k) const { return w + lay.sg_lam + (size_t)k * up256(p->N); }

    // s_eff and its boundary field for the current lam (G recomputed when flagged
    // or when force_g), then L (and W when breaking) at u
    pd_status force(const T *uu, bool force_g)
    {
        k_adj_weight<T><<<ng, 256, 0, st>>>(s, lam, seff, p->N);
        if (force_g) k_adj_flag<<<1, 1, 0, st>>>(cnt, 1);
        k_adj_gfield<T><<<nbl, 128, 0, st>>>(p->n1, p->n2, p->n3, p->hdev, p->ncomp, p->chi, seff, G, p->N, cnt);
        k_adj_flag<<<1, 1, 0, st>>>(cnt, 0);
        PD_LAUNCH_CHECK();
        p->launches += force_g ? 4 : 3;
        return force_any<T>(p, uu, seff, nullptr, G, L, breaking ? W : nullptr, st);
    }

    // one step from (u, v, lam) with L (and W) of the current state already
    // computed; b0 applies when n == 0
    pd_status step(int n)
    {
        k_adj_kick_drift<T><<<ng, 256, 0, st>>>(u, v, lam, L, b, n == 0 ? b0 : nullptr, W, p->chi, p->chi_om,
                                                p->dim, p->N, h, dt, (T)p->wc, breaking, cnt);
        PD_LAUNCH_CHECK();
        p->launches++;
        PD_TRY(force(u, false));
        k_adj_kick<T><<<ngv, 256, 0, st>>>(v, L, b, p->chi_om, (int64_t)p->dim * p->N, h);
        PD_LAUNCH_CHECK();
        p->launches++;
        return PD_OK;
    }

    pd_status copy(void *dst, const void *src, size_t bytes)
    {
        PD_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
        return PD_OK;
    }
};

template <typename T>
pd_status loss_grad_impl(pd_plan *p, const T *c_rel, const uint8_t *lam0, const T *u0, const T *v0, const T *b,
                         const T *b0, const T *ut, double dt, int nsteps, int K, void *work, double *loss_out,
                         T *grad_c, T *u_final, uint8_t *lam_final, cudaStream_t st)
{
    AdjRun<T> R;
    R.p = p;
    R.st = st;
    R.lay = adj_layout(p, nsteps, K);
    R.w = (unsigned char *)work;
    R.s = (T *)(R.w + R.lay.s);
    R.u = (T *)(R.w + R.lay.u);
    R.v = (T *)(R.w + R.lay.v);
    R.ubar = (T *)(R.w + R.lay.ubar);
    R.vbar = (T *)(R.w + R.lay.vbar);
    R.sbar = (T *)(R.w + R.lay.sbar);
    R.lam = R.w + R.lay.lam;
    R.L = (T *)p->cg_q;
    R.W = (T *)p->theta;
    R.G = (T *)p->Gw;
    R.seff = (T *)p->cg_e;
    R.gu = (T *)p->cg_r;
    R.gs = (T *)p->cg_p;
    R.b = b;
    R.b0 = b0;
    R.cnt = reinterpret_cast<AdjCounters *>(p->red + kRedVerlet);
    R.h = (T)(0.5 * dt / p->prob.rho);
    R.dt = (T)dt;
    R.breaking = p->wc > 0 ? 1 : 0;
    const int64_t N = p->N, dN = (int64_t)p->dim * N;
    R.ng = (unsigned)std::min<int64_t>(4 * p->nsm, (N + 255) / 256);
    R.ngv = (unsigned)std::min<int64_t>(4 * p->nsm, (dN + 255) / 256);
    R.nbl = (unsigned)((N + 127) / 128);
    const size_t vb = sizeof(T) * (size_t)dN;

    PD_CUDA_TRY(cudaMemsetAsync(R.cnt, 0, sizeof(AdjCounters), st));
    k_adj_init<T><<<R.ng, 256, 0, st>>>(c_rel, R.s, lam0, R.lam, N, R.cnt);
    PD_LAUNCH_CHECK();
    if (u0)
        PD_TRY(R.copy(R.u, u0, vb));
    else
        PD_CUDA_TRY(cudaMemsetAsync(R.u, 0, vb, st));
    if (v0)
        PD_TRY(R.copy(R.v, v0, vb));
    else
        PD_CUDA_TRY(cudaMemsetAsync(R.v, 0, vb, st));
    {
        AdjCounters hc;
        PD_CUDA_TRY(cudaMemcpyAsync(&hc, R.cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        if (hc.bad) {
            set_error("pd_verlet_loss_grad: the micromodulus field must be positive and finite");
            return PD_ERR_ARG;
        }
    }
    // forward with checkpoints
    PD_TRY(R.force(R.u, true));
    for (int n = 0; n < nsteps; ++n) {
        if (n % K == 0) {
            const int k = n / K;
            PD_TRY(R.copy(R.ck_u(k), R.u, vb));
            PD_TRY(R.copy(R.ck_v(k), R.v, vb));
            PD_TRY(R.copy(R.ck_lam(k), R.lam, (size_t)N));
        }
        PD_TRY(R.step(n));
    }
    // loss and u~
    constexpr int kLossBlocks = 512;
    k_adj_loss<T><<<kLossBlocks, 256, 0, st>>>(R.u, ut, p->chi_om, R.ubar, dN, p->red + kRedPart);
    PD_LAUNCH_CHECK();
    {
        std::vector<double> part(kLossBlocks);
        PD_CUDA_TRY(cudaMemcpyAsync(part.data(), p->red + kRedPart, sizeof(double) * kLossBlocks,
                                    cudaMemcpyDeviceToHost, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        double J = 0.0;
        for (double x : part) J += x;
        if (loss_out) *loss_out = J;
    }
    if (u_final) PD_TRY(R.copy(u_final, R.u, vb));
    if (lam_final) PD_TRY(R.copy(lam_final, R.lam, (size_t)N));
    if (!grad_c) return PD_OK;

    // reverse sweep, one segment at a time
    PD_CUDA_TRY(cudaMemsetAsync(R.vbar, 0, vb, st));
    PD_CUDA_TRY(cudaMemsetAsync(R.sbar, 0, sizeof(T) * (size_t)N, st));
    for (int seg = R.lay.ncp - 1; seg >= 0; --seg) {
        const int k0 = seg * K, k1 = std::min(nsteps, k0 + K);
        // recompute the segment's states u^n, lam^n (n = k0 .. k1 - 1)
        PD_TRY(R.copy(R.u, R.ck_u(seg), vb));
        PD_TRY(R.copy(R.v, R.ck_v(seg), vb));
        PD_TRY(R.copy(R.lam, R.ck_lam(seg), (size_t)N));
        PD_TRY(R.force(R.u, true));
        for (int n = k0; n < k1; ++n) {
            PD_TRY(R.copy(R.sg_u(n - k0), R.u, vb));
            PD_TRY(R.copy(R.sg_lam(n - k0), R.lam, (size_t)N));
            if (n + 1 < k1) PD_TRY(R.step(n));
        }
        for (int n = k1 - 1; n >= k0; --n) {
            k_adj_vbar<T><<<R.ngv, 256, 0, st>>>(R.vbar, R.ubar, p->chi_om, dN, R.dt);
            const T kf = n == 0 ? R.h : T(2) * R.h;
            k_adj_scale<T><<<R.ngv, 256, 0, st>>>(R.vbar, R.v, dN, kf);  // R.v: the cotangent k v~
            PD_LAUNCH_CHECK();
            p->launches += 2;
            // weight and boundary field of lam^n (without breaking lam never
            // changes: the ones of the recomputed segment are current)
            if (R.breaking) {
                PD_TRY(R.copy(R.lam, R.sg_lam(n - k0), (size_t)N));
                k_adj_weight<T><<<R.ng, 256, 0, st>>>(R.s, R.lam, R.seff, N);
                k_adj_flag<<<1, 1, 0, st>>>(R.cnt, 1);
                k_adj_gfield<T><<<R.nbl, 128, 0, st>>>(p->n1, p->n2, p->n3, p->hdev, p->ncomp, p->chi, R.seff,
                                                       R.G, N, R.cnt);
                PD_LAUNCH_CHECK();
                p->launches += 3;
            }
            PD_TRY(adjoint_weighted<T>(p, R.sg_u(n - k0), R.seff, R.v, R.G, R.gu, R.gs, st));
            k_adj_acc<T><<<R.ng, 256, 0, st>>>(R.ubar, R.gu, R.sbar, R.gs, R.lam, p->chi_om, p->dim, N);
            PD_LAUNCH_CHECK();
            p->launches++;
        }
    }
    k_adj_grad_c<T><<<R.ng, 256, 0, st>>>(R.sbar, R.s, grad_c, N);
    PD_LAUNCH_CHECK();
    p->launches++;
    return PD_OK;
}

}  // namespace
}  // namespace pd

using namespace pd;

extern "C" int64_t pd_verlet_adjoint_workspace(const pd_plan *p, int nsteps, int checkpoint_every)
{
    if (!p || nsteps < 1 || checkpoint_every < 1) return -1;
    return (int64_t)adj_layout(p, nsteps, std::min(checkpoint_every, nsteps)).total;
}

extern "C" pd_status pd_verlet_loss_grad(pd_plan *p, const void *c_rel, const uint8_t *lambda0, const void *u0,
                                         const void *v0, const void *b, const void *b0, const void *u_target,
                                         double dt, int nsteps, int checkpoint_every, void *work,
                                         int64_t work_bytes, double *loss_out, void *grad_c, void *u_final,
                                         uint8_t *lambda_final, void *stream)
{
    if (!p || !c_rel || !u_target || !work) {
        set_error("pd_verlet_loss_grad: null plan, c_rel, u_target or work");
        return PD_ERR_ARG;
    }
    if (p->state_based || p->nonlinear) {
        set_error("pd_verlet_loss_grad: the dynamic driver uses the linearized bond model");
        return PD_ERR_ARG;
    }
    if (!(dt > 0) || nsteps < 1 || checkpoint_every < 1 || !(p->prob.rho > 0)) {
        set_error("pd_verlet_loss_grad: dt and rho must be positive, nsteps and checkpoint_every >= 1");
        return PD_ERR_ARG;
    }
    const int K = std::min(checkpoint_every, nsteps);
    const int64_t need = (int64_t)adj_layout(p, nsteps, K).total;
    if (work_bytes < need) {
        set_error("pd_verlet_loss_grad: workspace of %lld bytes, %lld needed (pd_verlet_adjoint_workspace)",
                  (long long)work_bytes, (long long)need);
        return PD_ERR_ARG;
    }
    if (reinterpret_cast<uintptr_t>(work) % 256) {
        set_error("pd_verlet_loss_grad: the workspace must be 256-byte aligned");
        return PD_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (p->prob.fp64)
        return loss_grad_impl<double>(p, (const double *)c_rel, lambda0, (const double *)u0, (const double *)v0,
                                      (const double *)b, (const double *)b0, (const double *)u_target, dt, nsteps,
                                      K, work, loss_out, (double *)grad_c, (double *)u_final, lambda_final, st);
    return loss_grad_impl<float>(p, (const float *)c_rel, lambda0, (const float *)u0, (const float *)v0,
                                 (const float *)b, (const float *)b0, (const float *)u_target, dt, nsteps, K, work,
                                 loss_out, (float *)grad_c, (float *)u_final, lambda_final, st);
}
