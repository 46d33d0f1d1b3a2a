// pd_force_adjoint: reverse-mode derivative of the weighted bond force.
//
// The paper has no adjoint. Differentiating the quadrature of Eq. 17-18, 75 with
// bond factor v v' (v = chi s) against a cotangent p = dJ/dL gives
//   gu_i = (dL/du)^T p = v [ conv_M(v p)_i - G_ij p_j ]          (the operator is symmetric)
//   gs   = chi { p . conv_M(v u) - p.G.u - Σ_ij conv_M(v p_i u_j)_ij + u . conv_M(v p) }
// (conv_M = FFT convolution with M^ = (K^(k) - K^(0))/N, G = conv_M(v); the P
// terms of C* = conv_M + P cancel exactly). All of it is one fused pass:
//   rows  : FFT_x1 of v u_j (d), v p_j (d), v (p_i u_j + p_j u_i)/2 (d(d+1)/2)
//   cols  : FFT_x2 (3D)
//   last  : FFT, Y1 = M^ (v u), Y2 = M^ (v p), T3 = Σ_ij M^_ij (v p_i u_j), inverse
//   cols  : inverse FFT_x2 (3D)
//   rows  : inverse FFT_x1, gu and gs at each node.
#include "pd_ops.cuh"

namespace pd {

template <typename T>
pd_status weight_gfield(pd_plan *p, const T *s, const uint8_t *lam, T *G, cudaStream_t st);

namespace {

template <typename T, int D>
struct ProAdj {
    static constexpr int NC = Sym<D>::n;
    static constexpr int kFin = 0, kFout = 2 * D + NC, kNF = 0, kNB = 0, kStage = 0;
    static constexpr bool kSparse = false;
    const T *u, *pv, *s;
    const uint8_t *chi;
    int64_t N;
    int n1;
    cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int) const { return nullptr; }
    __device__ cx<T> *spec_out(int f) const { return spec + f * fstride; }
    __device__ const T *nf_src(int) const { return nullptr; }
    __device__ const uint8_t *nb_src(int) const { return nullptr; }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    __device__ void emit(const RowCtx<T> &, int, int, const T *, const T *, DSum &) const {}
    __device__ void block_done(DSum &) const {}
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *, const T *, T *o0,
                                          T *o1) const
    {
        node(c.row0 + rl, i1, o0);
        node(c.row0 + rl, i1 + 1, o1);
    }
    __device__ __forceinline__ void node(int64_t row, int i1, T *out) const
    {
        const int64_t q = row * n1 + i1;
        T v = chi[q] ? T(1) : T(0);
        if (s) v *= s[q];
        T uu[D], pp[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            uu[j] = u[j * N + q];
            pp[j] = pv[j * N + q];
            out[j] = v * uu[j];
            out[D + j] = v * pp[j];
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int a = Sym<D>::i(c), b = Sym<D>::j(c);
            out[2 * D + c] = v * T(0.5) * (pp[a] * uu[b] + pp[b] * uu[a]);
        }
    }
};

template <typename T, int D>
struct CombAdj {
    static constexpr int NC = Sym<D>::n;
    static constexpr int kFin = 2 * D + NC, kFout = 2 * D + 1, kMode = 2, kPre = 0, kTab = NC;
    static constexpr bool kStoreIn = false;
    Model<T> m;
    int obase;  // first output slot (out of place in 3D)
    __device__ int slot_in(int f) const { return f; }
    __device__ int slot_out(int f) const { return obase + f; }
    __device__ int slot_aux(int) const { return 0; }
    __device__ const T *table(int c) const { return m.mhat + c * m.fold_sz; }
    __device__ __forceinline__ void combine(const T *t, int cs, bool fy, bool fz, const cx<T> *in, cx<T> *out) const
    {
        T M[9];
        load_mhat_s(D, t, cs, fy, fz, M);
        mat_vec<T, D>(M, in, out);
        mat_vec<T, D>(M, in + D, out + D);
        cx<T> acc = mk(T(0), T(0));
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int a = Sym<D>::i(c), b = Sym<D>::j(c);
            const T w = (a == b) ? M[3 * a + b] : T(2) * M[3 * a + b];
            acc = acc + scale(in[2 * D + c], w);
        }
        out[2 * D] = acc;
    }
};

template <typename T, int D>
struct EpiAdj {
    static constexpr int NC = Sym<D>::n;
    static constexpr int kFin = 2 * D + 1, kFout = 0, kNF = 0, kNB = 0, kStage = 0;
    static constexpr bool kSparse = false;
    const T *u, *pv, *s, *G;
    const uint8_t *chi;
    T *gu, *gs;
    int64_t N;
    int n1;
    const cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_out(int) const { return nullptr; }
    __device__ const T *nf_src(int) const { return nullptr; }
    __device__ const uint8_t *nb_src(int) const { return nullptr; }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    __device__ void emit(const RowCtx<T> &, int, int, const T *, const T *, DSum &) const {}
    __device__ void block_done(DSum &) const {}
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *in0, const T *in1, T *,
                                          T *) const
    {
        node(c.row0 + rl, i1, in0);
        node(c.row0 + rl, i1 + 1, in1);
    }
    __device__ __forceinline__ void node(int64_t row, int i1, const T *in) const
    {
        const int64_t q = row * n1 + i1;
        const bool inb = chi[q] != 0;
        T v = inb ? T(1) : T(0);
        if (s) v *= s[q];
        T uu[D], pp[D], Gu[D], Gp[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            uu[j] = u[j * N + q];
            pp[j] = pv[j * N + q];
            Gu[j] = Gp[j] = T(0);
        }
        if (inb) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int a = Sym<D>::i(c), b = Sym<D>::j(c);
                const T g = G[c * N + q];
                Gu[a] += g * uu[b];
                Gp[a] += g * pp[b];
                if (a != b) {
                    Gu[b] += g * uu[a];
                    Gp[b] += g * pp[a];
                }
            }
        }
        if (gu) {
#pragma unroll
            for (int i = 0; i < D; ++i) gu[i * N + q] = v * (in[D + i] - Gp[i]);
        }
        if (gs) {
            T acc = -in[2 * D];
#pragma unroll
            for (int i = 0; i < D; ++i) acc += pp[i] * in[i] - pp[i] * Gu[i] + uu[i] * in[D + i];
            gs[q] = inb ? acc : T(0);
        }
    }
};

template <typename T, int D>
pd_status adjoint_pipeline(pd_plan *p, const T *u, const T *s, const T *pv, const T *G, T *gu, T *gs,
                           cudaStream_t st)
{
    cx<T> *spec = reinterpret_cast<cx<T> *>(spec_buf<T>(p));
    const int64_t fs = p->N / 2;
    constexpr int FI = 2 * D + Sym<D>::n, FO = 2 * D + 1;
    ProAdj<T, D> pro{u, pv, s, p->chi, p->N, p->n1, spec, fs};
    PD_TRY(launch_rows<T>(p, pro, st));
    if (D == 3) PD_TRY((col_pass<T, FI>(p, 0, false, st)));
    const int ob = D == 3 ? FI : 0;
    CombAdj<T, D> cmb{model_view<T>(p), ob};
    PD_TRY(launch_cols<T>(p, cmb, D == 3 ? 2 : 1, true, FI, st));
    if (D == 3) PD_TRY((col_pass<T, FO>(p, ob, true, st)));
    EpiAdj<T, D> epi{u, pv, s, G, p->chi, gu, gs, p->N, p->n1, spec + ob * fs, fs};
    PD_TRY(launch_rows<T>(p, epi, st));
    return PD_OK;
}

template <typename T>
pd_status adjoint_any(pd_plan *p, const T *u, const T *s, const T *pv, T *gu, T *gs, cudaStream_t st)
{
    const T *G = sizeof(T) == 8 ? (const T *)p->G64 : (const T *)p->G32;
    if (s) {
        PD_TRY(weight_gfield<T>(p, s, nullptr, (T *)p->Gw, st));
        G = (const T *)p->Gw;
    }
    if (p->dim == 2) return adjoint_pipeline<T, 2>(p, u, s, pv, G, gu, gs, st);
    return adjoint_pipeline<T, 3>(p, u, s, pv, G, gu, gs, st);
}

}  // namespace

// The adjoint passes for node weight s with its boundary field G given (the
// dynamic adjoint keeps G current as the integrity index changes).
template <typename T>
pd_status adjoint_weighted(pd_plan *p, const T *u, const T *s, const T *pv, const T *G, T *gu, T *gs,
                           cudaStream_t st)
{
    if (p->dim == 2) return adjoint_pipeline<T, 2>(p, u, s, pv, G, gu, gs, st);
    return adjoint_pipeline<T, 3>(p, u, s, pv, G, gu, gs, st);
}
template pd_status adjoint_weighted<float>(pd_plan *, const float *, const float *, const float *, const float *,
                                           float *, float *, cudaStream_t);
template pd_status adjoint_weighted<double>(pd_plan *, const double *, const double *, const double *,
                                            const double *, double *, double *, cudaStream_t);

}  // namespace pd

using namespace pd;

extern "C" pd_status pd_force_adjoint(pd_plan *p, const void *u, const void *s, const void *gL, void *gu, void *gs,
                                      void *stream)
{
    if (!p || !u || !gL) {
        set_error("pd_force_adjoint: null plan, u or gL");
        return PD_ERR_ARG;
    }
    if (p->state_based || p->nonlinear) {
        set_error("pd_force_adjoint: linearized bond model only");
        return PD_ERR_ARG;
    }
    if (!gu && !gs) return PD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->prob.fp64)
        return adjoint_any<double>(p, (const double *)u, (const double *)s, (const double *)gL, (double *)gu,
                                   (double *)gs, st);
    return adjoint_any<float>(p, (const float *)u, (const float *)s, (const float *)gL, (float *)gu, (float *)gs, st);
}
