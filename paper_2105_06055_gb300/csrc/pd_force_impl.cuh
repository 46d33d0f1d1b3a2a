// pd_force: one FCBM-EC force evaluation as fused FFT-convolution passes.
//
// Bond model (Eq. 57-58, 75, 100-102), d = 2 or 3, node weight v = chi s:
//   rows   : X_j = FFT_x1(v u_j)            [+ Q_ij = FFT_x1(v u_i u_j) for W]
//   cols   : FFT_x2                          (3D only)
//   last   : FFT_x3 (3D) / FFT_x2 (2D), Y_i = M^_ij X_j [, T = Σ M^_ij Q_ij], inverse
//   cols   : inverse FFT_x2                  (3D only)
//   rows   : inverse FFT_x1, L_i = v (y_i - G_ij u_j) [, W]
// State-based model with 3 kappa != 5 mu (Eq. 92, 95-97) adds the dilatation
// round trip between the two halves (see force_state below).
#pragma once
#include "pd_ops.cuh"

namespace pd {

static inline unsigned nblk_f(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

template <typename T, int D, bool ENERGY>
pd_status force_bond_pipeline(pd_plan *p, const T *u, const T *s, const uint8_t *lam, const T *G, T *L, T *W,
                              cudaStream_t st)
{
    cx<T> *spec = reinterpret_cast<cx<T> *>(spec_buf<T>(p));
    const int64_t fs = p->N / 2;
    constexpr int FI = D + (ENERGY ? Sym<D>::n : 0), FO = D + (ENERGY ? 1 : 0);
    ProForce<T, D, ENERGY> pro{u, s, lam, p->chi, p->N, p->n1, spec, fs};
    PD_TRY(launch_rows<T>(p, pro, FI, st));
    if (D == 3) PD_TRY((col_pass<T, FI>(p, spec, false, st)));
    const int ob = D == 3 ? FI : 0;
    CombForce<T, D, ENERGY> cmb{model_view<T>(p), spec, fs, ob};
    PD_TRY(launch_cols<T>(p, cmb, D == 3 ? 2 : 1, true, FI, st));
    if (D == 3) PD_TRY((col_pass<T, FO>(p, spec + ob * fs, true, st)));
    EpiForce<T, D, ENERGY> epi{u, s, lam, p->chi, G, L, W, p->N, p->n1, spec + ob * fs, fs};
    PD_TRY(launch_rows<T>(p, epi, FO, st));
    return PD_OK;
}

// ---------------------------------------------------------------------------
// State-based solid with dilatation (3D). With g_i = omega xi_i, the plan's
// node field q_i(x) = Σ_H g_i dV chi(x+xi) = -dV (g_i * chi)(x), and the
// correlation Σ_H g_i f(x+xi) dV = -dV (g_i * f)(x) (g is odd):
//   theta = (3 chi / m) Σ chi' omega xi.(u' - u) dV
//         = -(3 chi / m) [ dV g_i*(chi u_i) + q_i u_i ]                   (Eq. 93, 96)
//   L_i   = chi [ conv_M(chi u)_i - G_ij u_j + ka theta q_i - ka dV g_i*theta ]  (Eq. 92, 95)
// with ka = (3 kappa - 5 mu)/m0. The spectrum of g_i is -i gamma_i with
// gamma_i = Σ g_i sin(theta) (odd), so FFT(dV g_i * f)/N = -i ghat_i FFT(f),
// ghat_i = dV gamma_i / N.
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void load_ghat(const Model<T> &m, const SpecIdx<T> &s, T *g)
{
    const T *t = m.ghat + s.idx;
    const int64_t fs = m.fold_sz;
    g[0] = t[0];
    g[1] = s.fy ? -t[fs] : t[fs];
    g[2] = s.fz ? -t[2 * fs] : t[2 * fs];
}

// Slots: 0-2 chi u_j (x1, x2 transformed), 3 S, 4 theta, 5-7 fully transformed
// chi u_j, 0-2 again for the outputs (every 3D last-axis pass writes slots it
// does not read).
// last axis, round 1: transform chi u_j (kept in slots 5-7), S = Σ -i ghat_i X_i
template <typename T>
struct CombTheta {
    static constexpr int kFin = 3, kFout = 1, kMode = 2, kPre = 0;
    static constexpr bool kStoreIn = true;
    Model<T> m;
    cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_aux(int f) const { return spec + (5 + f) * fstride; }
    __device__ cx<T> *spec_out(int) const { return spec + 3 * fstride; }
    __device__ __forceinline__ void combine(int kx, int ky, int kz, const cx<T> *in, cx<T> *out) const
    {
        T g[3];
        load_ghat(m, spec_index(m, kx, ky, kz), g);
        cx<T> acc = mk(T(0), T(0));
#pragma unroll
        for (int i = 0; i < 3; ++i) acc = acc + scale(in[i], g[i]);
        out[0] = mk(acc.y, -acc.x);  // -i acc
    }
};

// rows: inverse of S, theta at the nodes, forward transform of theta
template <typename T>
struct RowTheta {
    static constexpr int kFin = 1, kFout = 1;
    Model<T> m;
    const T *u;
    T *theta;
    cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int) const { return spec + 3 * fstride; }
    __device__ cx<T> *spec_out(int) const { return spec + 4 * fstride; }
    __device__ __forceinline__ void node(int64_t row, int i1, const T *in, T *out) const
    {
        const int64_t p = row * m.n1 + i1;
        T th = T(0);
        if (m.chi[p]) {
            T qu = T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) qu += m.qt[i * m.N + p] * u[i * m.N + p];
            th = -m.m3inv[p] * (in[0] + qu);
        }
        theta[p] = th;
        out[0] = th;
    }
};

// last axis, round 2: Y_i = M^_ij X_j + i ka ghat_i Theta
template <typename T>
struct CombState {
    static constexpr int kFin = 4, kFout = 3, kMode = 2, kPre = 3;
    static constexpr bool kStoreIn = false;
    Model<T> m;
    cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int f) const { return spec + (f < 3 ? 5 + f : 4) * fstride; }
    __device__ cx<T> *spec_out(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_aux(int) const { return nullptr; }
    __device__ __forceinline__ void combine(int kx, int ky, int kz, const cx<T> *in, cx<T> *out) const
    {
        T M[9], g[3];
        const SpecIdx<T> si = spec_index(m, kx, ky, kz);
        load_mhat(m, si, M);
        load_ghat(m, si, g);
        mat_vec<T, 3>(M, in, out);
        const cx<T> it = mul_i(in[3]);
#pragma unroll
        for (int i = 0; i < 3; ++i) out[i] = out[i] + scale(it, m.ka * g[i]);
    }
};

template <typename T>
struct EpiState {
    static constexpr int kFin = 3, kFout = 0;
    Model<T> m;
    const T *u;
    const T *theta;
    T *L;
    const cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_out(int) const { return nullptr; }
    __device__ __forceinline__ void node(int64_t row, int i1, const T *in, T *) const
    {
        const int64_t p = row * m.n1 + i1;
        const int64_t N = m.N;
        if (!m.chi[p]) {
#pragma unroll
            for (int i = 0; i < 3; ++i) L[i * N + p] = T(0);
            return;
        }
        T uu[3], Gu[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int j = 0; j < 3; ++j) uu[j] = u[j * N + p];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int a = Sym<3>::i(c), b = Sym<3>::j(c);
            const T gc = m.G[c * N + p];
            Gu[a] += gc * uu[b];
            if (a != b) Gu[b] += gc * uu[a];
        }
        const T th = theta[p];
#pragma unroll
        for (int i = 0; i < 3; ++i) L[i * N + p] = in[i] - Gu[i] + m.ka * th * m.qt[i * N + p];
    }
};

template <typename T>
pd_status force_state_pipeline(pd_plan *p, const T *u, T *L, T *theta, cudaStream_t st)
{
    cx<T> *spec = reinterpret_cast<cx<T> *>(spec_buf<T>(p));
    const int64_t fs = p->N / 2;
    const Model<T> m = model_view<T>(p);
    ProForce<T, 3, false> pro{u, nullptr, nullptr, p->chi, p->N, p->n1, spec, fs};
    PD_TRY(launch_rows<T>(p, pro, 3, st));
    PD_TRY((col_pass<T, 3>(p, spec, false, st)));
    CombTheta<T> c1{m, spec, fs};
    PD_TRY(launch_cols<T>(p, c1, 2, true, 3, st));
    PD_TRY((col_pass<T, 1>(p, spec + 3 * fs, true, st)));
    RowTheta<T> rt{m, u, theta, spec, fs};
    PD_TRY(launch_rows<T>(p, rt, 1, st));
    PD_TRY((col_pass<T, 1>(p, spec + 4 * fs, false, st)));
    CombState<T> c2{m, spec, fs};
    PD_TRY(launch_cols<T>(p, c2, 2, true, 4, st));
    PD_TRY((col_pass<T, 3>(p, spec, true, st)));
    EpiState<T> epi{m, u, theta, L, spec, fs};
    PD_TRY(launch_rows<T>(p, epi, 3, st));
    return PD_OK;
}

// Boundary field for a node weight (s and/or lam): G = conv_M(chi s lam), direct sum.
template <typename T>
pd_status weight_gfield(pd_plan *p, const T *s, const uint8_t *lam, T *G, cudaStream_t st)
{
    if (s && lam) {
        set_error("weight_gfield: s and lambda together are not supported");
        return PD_ERR_ARG;
    }
    if (s)
        k_gfield<T, T, T><<<nblk_f(p->N, 128), 128, 0, st>>>(p->n1, p->n2, p->n3, p->hdev, p->ncomp, p->chi, s, G,
                                                           p->N);
    else
        k_gfield<T, uint8_t, T><<<nblk_f(p->N, 128), 128, 0, st>>>(p->n1, p->n2, p->n3, p->hdev, p->ncomp, p->chi,
                                                                 lam, G, p->N);
    PD_LAUNCH_CHECK();
    p->launches++;
    return PD_OK;
}

template <typename T>
pd_status force_any(pd_plan *p, const T *u, const T *s, const uint8_t *lam, const T *G, T *L, T *W,
                    cudaStream_t st)
{
    if (p->dim == 2) {
        if (W) return force_bond_pipeline<T, 2, true>(p, u, s, lam, G, L, W, st);
        return force_bond_pipeline<T, 2, false>(p, u, s, lam, G, L, nullptr, st);
    }
    if (W) return force_bond_pipeline<T, 3, true>(p, u, s, lam, G, L, W, st);
    return force_bond_pipeline<T, 3, false>(p, u, s, lam, G, L, nullptr, st);
}

template <typename T>
T *work_theta(pd_plan *p)
{
    if constexpr (sizeof(T) == 8) {
        if (!p->prob.fp64) return reinterpret_cast<T *>(p->theta64);
    }
    return reinterpret_cast<T *>(p->theta);
}

template <typename T>
pd_status force_plain(pd_plan *p, const T *u, const T *s, T *L, T *W, cudaStream_t st)
{
    if (p->state_based) {
        if (s || W) {
            set_error("pd_force: node weight and energy output are for the bond model only");
            return PD_ERR_ARG;
        }
        return force_state_pipeline<T>(p, u, L, work_theta<T>(p), st);
    }
    const T *G = sizeof(T) == 8 ? (const T *)p->G64 : (const T *)p->G32;
    if (s) {
        if (sizeof(T) == 8 && !p->prob.fp64) {
            set_error("pd_force: FP64 node weight on an FP32 plan is not supported");
            return PD_ERR_ARG;
        }
        T *Gs = reinterpret_cast<T *>(p->Gw);
        PD_TRY(weight_gfield<T>(p, s, nullptr, Gs, st));
        G = Gs;
    }
    return force_any<T>(p, u, s, nullptr, G, L, W, st);
}

}  // namespace pd

