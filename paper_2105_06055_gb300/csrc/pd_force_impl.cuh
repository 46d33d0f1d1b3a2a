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

// SPARSE: the epilogue takes the plan's boundary-node list of G (weight chi_B);
// otherwise the dense G passed in (weight chi_B, chi_B s or chi_B lam).
// Fit of the affine split (pd_affine.cuh): block sums over the body, then the
// exact-form coefficients in the plan's coefficient buffer.
template <typename T, int D>
pd_status affine_fit(pd_plan *p, const T *u, cudaStream_t st, AffineView<T> *view)
{
    constexpr int kBlocks = 296;  // 2 x 148 SMs' worth; the sums are a small part of the evaluation
    AffFitArgs fa;
    for (int i = 0; i < 16; ++i) fa.inv[i] = p->aff_inv[i];
    for (int k = 0; k < 3; ++k) fa.emax[k] = p->aff_emax[k];
    fa.nblk = kBlocks;
    const int lg1 = ilog2(p->n1), lg2 = ilog2(p->n2);
    PD_TRY(launch_k(p->pdl != 0, k_aff_sums<T, D>, dim3(kBlocks), dim3(256), 0, st, u, (const uint8_t *)p->chi, lg1,
                    lg2, p->aff_c[0], p->aff_c[1], p->aff_c[2], p->N, p->red));
    T *coef = reinterpret_cast<T *>(p->aff_coef);
    PD_TRY(launch_k(p->pdl != 0, k_aff_fit<T, D>, dim3(1), dim3(256), 0, st, (const double *)p->red, fa, coef));
    p->launches += 2;
    *view = AffineView<T>{coef, p->aff_c[0], p->aff_c[1], p->aff_c[2], lg1, lg2};
    return PD_OK;
}

template <typename T, int D, bool ENERGY, int WM, bool SPARSE = (WM == W_NONE), bool AFF = false>
pd_status force_bond_pipeline(pd_plan *p, const T *u, const T *s, const uint8_t *lam, const T *G, T *L, T *W,
                              cudaStream_t st)
{
    cx<T> *spec = reinterpret_cast<cx<T> *>(spec_buf<T>(p));
    const int64_t fs = p->N / 2;
    constexpr int FI = D + (ENERGY ? Sym<D>::n : 0), FO = D + (ENERGY ? 1 : 0);
    AffineView<T> av{};
    if constexpr (AFF) PD_TRY((affine_fit<T, D>(p, u, st, &av)));
    ProForce<T, D, ENERGY, WM, AFF> pro{u, s, lam, p->chi, p->N, spec, fs, av};
    PD_TRY(launch_rows<T>(p, pro, st));
    if (D == 3) PD_TRY((col_pass<T, FI>(p, 0, false, st)));
    const int ob = D == 3 ? FI : 0;
    CombForce<T, D, ENERGY> cmb{model_view<T>(p), ob};
    PD_TRY(launch_cols<T>(p, cmb, D == 3 ? 2 : 1, true, FI, st));
    if (D == 3) PD_TRY((col_pass<T, FO>(p, ob, true, st)));
    if constexpr (SPARSE) {
        static_assert(WM == W_NONE, "the boundary-node list is for the plan weight chi_B");
        const Model<T> m = model_view<T>(p);
        EpiForceSparse<T, D, ENERGY, AFF> epi{u, p->chi, m.gent, p->gidx, L, W, p->N, p->n1, spec + ob * fs, fs,
                                              av, reinterpret_cast<const T *>(p->aff_tab)};
        PD_TRY(launch_rows<T>(p, epi, st));
    } else {
        EpiForceDense<T, D, ENERGY, WM> epi{u, s, lam, p->chi, G, L, W, p->N, p->n1, spec + ob * fs, fs};
        PD_TRY(launch_rows<T>(p, epi, st));
    }
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

// Slots: 0-2 chi u_j (x1, x2 transformed), 3 S, 4 theta, 5-7 fully transformed
// chi u_j, 0-2 again for the outputs (every 3D last-axis pass writes slots it
// does not read).
// last axis, first combine: transform chi u_j (kept in slots 5-7), S = Σ -i ghat_i X_i
template <typename T>
struct CombTheta {
    static constexpr int kFin = 3, kFout = 1, kMode = 2, kPre = 0, kTab = 3;
    static constexpr bool kStoreIn = true;
    Model<T> m;
    __device__ int slot_in(int f) const { return f; }
    __device__ int slot_aux(int f) const { return 5 + f; }
    __device__ int slot_out(int) const { return 3; }
    __device__ const T *table(int c) const { return m.ghat + c * m.fold_sz; }
    __device__ __forceinline__ void combine(const T *t, int cs, bool fy, bool fz, const cx<T> *in, cx<T> *out) const
    {
        T g[3];
        load_ghat_s(t, cs, fy, fz, g);
        cx<T> acc = mk(T(0), T(0));
#pragma unroll
        for (int i = 0; i < 3; ++i) acc = acc + scale(in[i], g[i]);
        out[0] = mk(acc.y, -acc.x);  // -i acc
    }
};

// rows: inverse of S, theta at the nodes, forward transform of theta
template <typename T>
struct RowTheta {
    static constexpr int kFin = 1, kFout = 1, kNF = 0, kNB = 0, kStage = 0;
    static constexpr bool kSparse = false;
    Model<T> m;
    const T *u;
    T *theta;
    cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int) const { return spec + 3 * fstride; }
    __device__ cx<T> *spec_out(int) const { return spec + 4 * fstride; }
    __device__ const T *nf_src(int) const { return nullptr; }
    __device__ const uint8_t *nb_src(int) const { return nullptr; }
    __device__ __forceinline__ T node1(int64_t p, T in) const
    {
        T th = T(0);
        if (m.chi[p]) {
            T qu = T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) qu += m.qt[i * m.N + p] * u[i * m.N + p];
            th = -m.m3inv[p] * (in + qu);
        }
        return th;
    }
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *in0, const T *in1, T *o0,
                                          T *o1) const
    {
        const int64_t p = (c.row0 + rl) * m.n1 + i1;
        const T t0 = node1(p, in0[0]), t1 = node1(p + 1, in1[0]);
        store2(theta + p, t0, t1);
        o0[0] = t0;
        o1[0] = t1;
    }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    __device__ void emit(const RowCtx<T> &, int, int, const T *, const T *, DSum &) const {}
    __device__ void block_done(DSum &) const {}
};

// last axis, second combine: Y_i = M^_ij X_j + i ka ghat_i Theta
template <typename T>
struct CombState {
    static constexpr int kFin = 4, kFout = 3, kMode = 2, kPre = 3, kTab = 9;
    static constexpr bool kStoreIn = false;
    Model<T> m;
    __device__ int slot_in(int f) const { return f < 3 ? 5 + f : 4; }
    __device__ int slot_out(int f) const { return f; }
    __device__ int slot_aux(int) const { return 0; }
    __device__ const T *table(int c) const { return c < 6 ? m.mhat + c * m.fold_sz : m.ghat + (c - 6) * m.fold_sz; }
    __device__ __forceinline__ void combine(const T *t, int cs, bool fy, bool fz, const cx<T> *in, cx<T> *out) const
    {
        T M[9], g[3];
        load_mhat_s(3, t, cs, fy, fz, M);
        load_ghat_s(t + 6 * cs, cs, fy, fz, g);
        mat_vec<T, 3>(M, in, out);
        const cx<T> it = mul_i(in[3]);
#pragma unroll
        for (int i = 0; i < 3; ++i) out[i] = out[i] + scale(it, m.ka * g[i]);
    }
};

// rows: inverse of Y, L = chi y staged, boundary fix-up
//   L_i -= G_ij u_j - ka theta q_i   (q_i and G vanish off the boundary list)
template <typename T>
struct EpiState {
    static constexpr int kFin = 3, kFout = 0, kNF = 0, kNB = 1, kStage = 3;
    static constexpr bool kSparse = true;
    Model<T> m;
    const T *u;
    const T *theta;
    T *L;
    const cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_out(int) const { return nullptr; }
    __device__ const T *nf_src(int) const { return nullptr; }
    __device__ const uint8_t *nb_src(int) const { return m.chi; }
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *in0, const T *in1, T *o0,
                                          T *o1) const
    {
        const T v0 = c.b(0, rl, i1) ? T(1) : T(0), v1 = c.b(0, rl, i1 + 1) ? T(1) : T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            o0[i] = v0 * in0[i];
            o1[i] = v1 * in1[i];
        }
    }
    __device__ void sparse(const RowCtx<T> &c, int tid, int nthreads) const
    {
        const int64_t N = m.N;
        const int k0 = m.goff[c.row0], k1 = m.goff[c.row0 + c.rows];
        for (int k = k0 + tid; k < k1; k += nthreads) {
            const GEntry<T> e = m.gent[k];
            const int64_t p = e.p;
            const int rl = (int)(p / m.n1 - c.row0), i1 = (int)(p % m.n1);
            T uu[3], Gu[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int j = 0; j < 3; ++j) uu[j] = u[j * N + p];
            sym_apply<T, 3>(e.g, uu, Gu);
            const T th = theta[p];
#pragma unroll
            for (int i = 0; i < 3; ++i) c.stage(i, rl, i1) -= Gu[i] - m.ka * th * m.qt[i * N + p];
        }
    }
    __device__ __forceinline__ void emit(const RowCtx<T> &c, int rl, int i1, const T *s0, const T *s1,
                                         DSum &) const
    {
        const int64_t p = (c.row0 + rl) * m.n1 + i1;
#pragma unroll
        for (int i = 0; i < 3; ++i) store2(L + i * m.N + p, s0[i], s1[i]);
    }
    __device__ void block_done(DSum &) const {}
};

template <typename T>
pd_status force_state_pipeline(pd_plan *p, const T *u, T *L, T *theta, cudaStream_t st)
{
    cx<T> *spec = reinterpret_cast<cx<T> *>(spec_buf<T>(p));
    const int64_t fs = p->N / 2;
    const Model<T> m = model_view<T>(p);
    ProForce<T, 3, false, W_NONE> pro{u, nullptr, nullptr, p->chi, p->N, spec, fs};
    PD_TRY(launch_rows<T>(p, pro, st));
    PD_TRY((col_pass<T, 3>(p, 0, false, st)));
    CombTheta<T> c1{m};
    PD_TRY(launch_cols<T>(p, c1, 2, true, 3, st));
    PD_TRY((col_pass<T, 1>(p, 3, true, st)));
    RowTheta<T> rt{m, u, theta, spec, fs};
    PD_TRY(launch_rows<T>(p, rt, st));
    PD_TRY((col_pass<T, 1>(p, 4, false, st)));
    CombState<T> c2{m};
    PD_TRY(launch_cols<T>(p, c2, 2, true, 4, st));
    PD_TRY((col_pass<T, 3>(p, 0, true, st)));
    EpiState<T> epi{m, u, theta, L, spec, fs};
    PD_TRY(launch_rows<T>(p, epi, st));
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

// Bond-model force with weight chi_B (s = lam = null: sparse plan G), chi_B s
// or chi_B lam (dense G of that weight passed in G).
template <typename T>
pd_status force_any(pd_plan *p, const T *u, const T *s, const uint8_t *lam, const T *G, T *L, T *W,
                    cudaStream_t st)
{
    if (s && lam) {
        set_error("force: s and lambda together are not supported");
        return PD_ERR_ARG;
    }
#define PD_FORCE_CASE(D, E)                                                                         \
    do {                                                                                            \
        if (s) return force_bond_pipeline<T, D, E, W_S>(p, u, s, lam, G, L, W, st);                 \
        if (lam) return force_bond_pipeline<T, D, E, W_LAM>(p, u, s, lam, G, L, W, st);             \
        return force_bond_pipeline<T, D, E, W_NONE>(p, u, s, lam, G, L, W, st);                     \
    } while (0)
    if (p->dim == 2) {
        if (W) PD_FORCE_CASE(2, true);
        PD_FORCE_CASE(2, false);
    }
    if (W) PD_FORCE_CASE(3, true);
    PD_FORCE_CASE(3, false);
#undef PD_FORCE_CASE
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

// pd_force: force_plain, or with the affine split when the plan has it on and
// the call is the plain bond force in the plan's precision (pd_affine.cuh)
template <typename T>
pd_status force_public(pd_plan *p, const T *u, const T *s, T *L, T *W, cudaStream_t st)
{
    const bool aff = p->affine_split && !p->state_based && !s && !W && sizeof(T) == (p->prob.fp64 ? 8 : 4);
    if (!aff) return force_plain<T>(p, u, s, L, W, st);
    if (p->dim == 2) return force_bond_pipeline<T, 2, false, W_NONE, true, true>(p, u, s, nullptr, nullptr, L, W, st);
    return force_bond_pipeline<T, 3, false, W_NONE, true, true>(p, u, s, nullptr, nullptr, L, W, st);
}

}  // namespace pd

