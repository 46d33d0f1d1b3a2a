// pd_force for the nonlinear rotation-invariant bond model (§3.2, Eq. 19-26).
//
// With w = chi_B the node weight, c(xi) = alpha dV / |xi|^3, a_i = c xi_i,
// C_ij = c xi_i xi_j and S(K, f)(x) = Σ_H K(xi) f(x + xi) the correlation with
// the horizon kernel K, the bond force of Eq. 21 summed over the horizon is
// (Eq. 26, written with the node values u = u(x)):
//   L_i / w = S(C_ij, w u_j) - S(C_ij, w) u_j
//           + S(a_j, w u_j u_i) - u_i S(a_j, w u_j) - u_j S(a_j, w u_i) + u_i u_j S(a_j, w)
//           + 1/2 S(a_i, w |u|^2) - u_j S(a_i, w u_j) + 1/2 |u|^2 S(a_i, w)
//           + 1/2 S(c, w |u|^2 u_i) - 1/2 u_i S(c, w |u|^2) - u_j S(c, w u_i u_j)
//           + u_i u_j S(c, w u_j) + 1/2 |u|^2 S(c, w u_i) - 1/2 |u|^2 u_i S(c, w)
// The paper's discrete form (Eq. 59) prints the second correlation without
// the factor u_i; the form here is Eq. 26's, which the oracle's direct sum of
// Eq. 21 confirms. Every correlation of a nodal product is one FFT product:
//   forward:  X_j = F(w u_j), Y_ij = F(w u_i u_j), Z_i = F(w |u|^2 u_i)
//             (2D: 2 + 3 + 2 = 7 fields, 3D: 3 + 6 + 3 = 12)
//   combine:  P_i  = C^_ij X_j + i g_j Y_ji + 1/2 i g_i Σ_j Y_jj + 1/2 c^ Z_i
//             A_mn = i g_m X_n,  B_ij = c^ Y_ij,  Cc_j = c^ X_j
//             (2D: 2 + 4 + 3 + 2 = 11 inverse fields, 3D: 3 + 9 + 6 + 3 = 21)
// with C^, c^ the (real, even) spectra of C and c and i g_m that of the odd a_m
// (a correlation with an odd kernel multiplies by +i Σ a sin(theta)). As for
// the linearized model the kernels enter as differences from their k = 0
// values, C^ - C^(0) and c^ - c^(0) (1/N folded in): the k = 0 parts cancel in
// the sum above, and the plan-time correlations with w alone then vanish in
// the delta-interior (G = S(C, w) - C^(0) w, S(a, w), S(c, w) - c^(0) w are kept
// on the boundary-node list). The epilogue forms L_i per node from the inverse
// fields and the node values.
//
// The model is exactly invariant under rigid translations, so the body mean of
// u is removed first: the expansion in u(x) and u(x + xi) cancels terms of
// order |u|^3 that the bond stretch never carries, and in FP32 a translation
// would otherwise dominate the rounding.
#include "pd_force_impl.cuh"

namespace pd {
namespace {

template <int D>
struct NL {
    static constexpr int NS = Sym<D>::n;
    static constexpr int FWD = 2 * D + NS;           // X (D), Y (NS), Z (D)
    static constexpr int INV = D + D * D + NS + D;   // P (D), A (D^2), B (NS), Cc (D)
    static constexpr int X = 0, Y = D, Z = D + NS;
    static constexpr int P = 0, A = D, B = D + D * D, CC = D + D * D + NS;
};

// the body mean of u (from the affine-fit block sums) as the coefficient t of
// an AffineView with B = 0 (one block)
template <typename T, int D>
__global__ void __launch_bounds__(256) k_nl_mean(const double *red, int nblk, double inv_count, T *coef)
{
    constexpr int NV = D + D * D;
    __shared__ double sums[D];
    pdl_wait();
    for (int v = 0; v < D; ++v) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += red[kRedPart + (int64_t)b * NV + v];
        s = block_sum_d(s);
        if (threadIdx.x == 0) sums[v] = s;
        __syncthreads();
    }
    pdl_trigger();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 9; ++k) coef[k] = T(0);
        for (int j = 0; j < 3; ++j) coef[kAffT + j] = j < D ? (T)(sums[j] * inv_count) : T(0);
    }
}

// Forward prologue: X_j = w u_j, Y_q = w u_a u_b, Z_i = w |u|^2 u_i with u - mean
template <typename T, int D>
struct ProNL {
    using K = NL<D>;
    static constexpr int kFin = 0, kFout = K::FWD, kNF = D, kNB = 1, kStage = 0;
    static constexpr bool kSparse = false;
    const T *u;
    const uint8_t *chi;
    int64_t N;
    cx<T> *spec;
    int64_t fstride;
    AffineView<T> mean;
    __device__ const cx<T> *spec_in(int) const { return nullptr; }
    __device__ cx<T> *spec_out(int f) const { return spec + f * fstride; }
    __device__ const T *nf_src(int k) const { return u + k * N; }
    __device__ const uint8_t *nb_src(int) const { return chi; }
    __device__ __forceinline__ void node1(const RowCtx<T> &c, int rl, int i1, T *out) const
    {
        const T v = c.b(0, rl, i1) ? T(1) : T(0);
        T m[D], uu[D];
        mean.at(i1, c.row0 + rl, D, m);
        T s2 = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            uu[j] = c.f(j, rl, i1) - m[j];
            s2 += uu[j] * uu[j];
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            out[K::X + j] = v * uu[j];
            out[K::Z + j] = v * s2 * uu[j];
        }
#pragma unroll
        for (int q = 0; q < K::NS; ++q) out[K::Y + q] = v * uu[Sym<D>::i(q)] * uu[Sym<D>::j(q)];
    }
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *, const T *, T *o0,
                                          T *o1) const
    {
        node1(c, rl, i1, o0);
        node1(c, rl, i1 + 1, o1);
    }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    __device__ void emit(const RowCtx<T> &, int, int, const T *, const T *, DSum &) const {}
    __device__ void block_done(DSum &) const {}
};

// odd-kernel spectrum g_i from a table slice (component stride cs): the
// components along folded axes change sign
template <typename T, int D>
__device__ __forceinline__ void load_odd(const T *t, int cs, bool fy, bool fz, T *g)
{
    g[0] = t[0];
    g[1] = fy ? -t[cs] : t[cs];
    if (D == 3) g[2] = fz ? -t[2 * cs] : t[2 * cs];
}

// Spectral combination of the seven (2D) or twelve (3D) forward fields into
// the eleven or twenty-one inverse fields
template <typename T, int D>
struct CombNL {
    using K = NL<D>;
    static constexpr int kFin = K::FWD, kFout = K::INV, kMode = 2, kPre = 0, kTab = K::NS + 1 + D;
    static constexpr bool kStoreIn = false;
    const T *mhat, *chat, *ghat;
    int64_t fold_sz;
    int obase;  // first output slot (3D: after the inputs, the pass is out of place)
    __device__ int slot_in(int f) const { return f; }
    __device__ int slot_out(int f) const { return obase + f; }
    __device__ int slot_aux(int) const { return 0; }
    __device__ const T *table(int c) const
    {
        return c < K::NS ? mhat + c * fold_sz : (c == K::NS ? chat : ghat + (c - K::NS - 1) * fold_sz);
    }
    __device__ __forceinline__ void combine(const T *t, int cs, bool fy, bool fz, const cx<T> *in, cx<T> *out) const
    {
        T M[9], g[3];
        load_mhat_s(D, t, cs, fy, fz, M);
        const T ch = t[K::NS * cs];
        load_odd<T, D>(t + (K::NS + 1) * cs, cs, fy, fz, g);
        auto Yf = [&](int i, int j) -> cx<T> {
            const int a = i < j ? i : j, b = i < j ? j : i;
#pragma unroll
            for (int q = 0; q < K::NS; ++q)
                if (Sym<D>::i(q) == a && Sym<D>::j(q) == b) return in[K::Y + q];
            return mk(T(0), T(0));
        };
        cx<T> yt = mk(T(0), T(0));
#pragma unroll
        for (int j = 0; j < D; ++j) yt = yt + in[K::Y + j];  // diagonal Y come first in Sym order
#pragma unroll
        for (int i = 0; i < D; ++i) {
            cx<T> acc = scale(in[K::Z + i], T(0.5) * ch);
            cx<T> ia = scale(yt, T(0.5) * g[i]);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                acc = acc + scale(in[K::X + j], M[3 * i + j]);
                ia = ia + scale(Yf(j, i), g[j]);
            }
            out[K::P + i] = acc + mul_i(ia);
        }
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
            for (int n = 0; n < D; ++n) out[K::A + D * m + n] = mul_i(scale(in[K::X + n], g[m]));
#pragma unroll
        for (int q = 0; q < K::NS; ++q) out[K::B + q] = scale(in[K::Y + q], ch);
#pragma unroll
        for (int j = 0; j < D; ++j) out[K::CC + j] = scale(in[K::X + j], ch);
    }
};

// Inverse epilogue: L_i = w t_i from the inverse fields and the node values
// (dense part staged), then the boundary terms of the plan-time correlations
// with w at the listed nodes
template <typename T, int D>
struct EpiNL {
    using K = NL<D>;
    static constexpr int kFin = K::INV, kFout = 0, kStage = D, kNF = D, kNB = 1;
    static constexpr bool kSparse = false;
    const T *u;
    const uint8_t *chi;
    const GEntry<T> *gent;
    const T *nlb;  // [entry][4]: S(a_j, w) (D), S(c, w) - c^(0) w
    const int *gidx;
    T *L;
    int64_t N;
    int n1;
    const cx<T> *spec;
    int64_t fstride;
    AffineView<T> mean;
    __device__ const cx<T> *spec_in(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_out(int) const { return nullptr; }
    __device__ const T *nf_src(int k) const { return u + k * N; }
    __device__ const uint8_t *nb_src(int) const { return chi; }
    __device__ __forceinline__ void node_u(const RowCtx<T> &c, int rl, int i1, T *uu, T &s2) const
    {
        T m[D];
        mean.at(i1, c.row0 + rl, D, m);
        s2 = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            uu[j] = c.f(j, rl, i1) - m[j];
            s2 += uu[j] * uu[j];
        }
    }
    __device__ __forceinline__ void node1(const RowCtx<T> &c, int rl, int i1, const T *in, T *o) const
    {
        const T v = c.b(0, rl, i1) ? T(1) : T(0);
        T uu[D], s2;
        node_u(c, rl, i1, uu, s2);
        T trA = T(0), trB = T(0), cu = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            trA += in[K::A + D * j + j];
            trB += in[K::B + j];
            cu += in[K::CC + j] * uu[j];
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
            T t = in[K::P + i] - (trA + T(0.5) * trB - cu) * uu[i] + T(0.5) * s2 * in[K::CC + i];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const int q = sym_index(D, i, j);
                t -= (in[K::A + D * j + i] + in[K::A + D * i + j] + in[K::B + q]) * uu[j];
            }
            o[i] = v * t;
        }
    }
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *in0, const T *in1, T *o0,
                                          T *o1) const
    {
        node1(c, rl, i1, in0, o0);
        node1(c, rl, i1 + 1, in1, o1);
    }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    __device__ __forceinline__ void fix(const RowCtx<T> &c, int rl, int i1, int k, T *s) const
    {
        const GEntry<T> e = gent[k];
        const T *nb = nlb + 4 * (int64_t)k;
        T uu[D], s2, Gu[D];
        node_u(c, rl, i1, uu, s2);
        T sau = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            Gu[j] = T(0);
            sau += nb[j] * uu[j];
        }
        sym_apply<T, D>(e.g, uu, Gu);
        const T sc = nb[3];
#pragma unroll
        for (int i = 0; i < D; ++i) s[i] += -Gu[i] + uu[i] * sau + T(0.5) * s2 * (nb[i] - sc * uu[i]);
    }
    __device__ __forceinline__ void emit(const RowCtx<T> &c, int rl, int i1, const T *s0, const T *s1,
                                         DSum &) const
    {
        const int64_t p = (c.row0 + rl) * n1 + i1;
        const int2 gi = *reinterpret_cast<const int2 *>(gidx + p);
        T a[D], b[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            a[i] = s0[i];
            b[i] = s1[i];
        }
        if (gi.x >= 0) fix(c, rl, i1, gi.x, a);
        if (gi.y >= 0) fix(c, rl, i1 + 1, gi.y, b);
#pragma unroll
        for (int i = 0; i < D; ++i) store2(L + i * N + p, a[i], b[i]);
    }
    __device__ void block_done(DSum &) const {}
};

template <typename T, int D>
pd_status force_nl_dim(pd_plan *p, const T *u, T *L, cudaStream_t st)
{
    using K = NL<D>;
    cx<T> *spec = reinterpret_cast<cx<T> *>(spec_buf<T>(p));
    const int64_t fs = p->N / 2;
    T *coef = reinterpret_cast<T *>(p->aff_coef);
    // body mean of u
    {
        constexpr int kBlocks = 296;
        const int lg1 = ilog2(p->n1), lg2 = ilog2(p->n2);
        PD_TRY(launch_k(p->pdl != 0, k_aff_sums<T, D>, dim3(kBlocks), dim3(256), 0, st, u,
                        (const uint8_t *)p->chi, lg1, lg2, p->aff_c[0], p->aff_c[1], p->aff_c[2], p->N, p->red));
        PD_TRY(launch_k(p->pdl != 0, k_nl_mean<T, D>, dim3(1), dim3(256), 0, st, (const double *)p->red, kBlocks,
                        p->body_count > 0 ? 1.0 / p->body_count : 0.0, coef));
        p->launches += 2;
    }
    const AffineView<T> mean{coef, p->aff_c[0], p->aff_c[1], p->aff_c[2], ilog2(p->n1), ilog2(p->n2)};
    ProNL<T, D> pro{u, p->chi, p->N, spec, fs, mean};
    PD_TRY(launch_rows<T>(p, pro, st));
    if (D == 3) PD_TRY((col_pass<T, K::FWD>(p, 0, false, st)));
    const int ob = D == 3 ? K::FWD : 0;
    const T *mhat = sizeof(T) == 8 ? (const T *)p->mhat64 : (const T *)p->mhat32;
    const T *chat = sizeof(T) == 8 ? (const T *)p->chat64 : (const T *)p->chat32;
    const T *ghat = sizeof(T) == 8 ? (const T *)p->ghat64 : (const T *)p->ghat32;
    CombNL<T, D> cmb{mhat, chat, ghat, p->fold_sz, ob};
    PD_TRY(launch_cols<T>(p, cmb, D == 3 ? 2 : 1, true, K::INV, st));
    if (D == 3) PD_TRY((col_pass<T, K::INV>(p, ob, true, st)));
    const Model<T> m = model_view<T>(p);
    EpiNL<T, D> epi{u, p->chi, m.gent, reinterpret_cast<const T *>(p->nlb), p->gidx, L, p->N, p->n1,
                    spec + ob * fs, fs, mean};
    PD_TRY(launch_rows<T>(p, epi, st));
    return PD_OK;
}

}  // namespace

template <typename T>
pd_status force_nl(pd_plan *p, const T *u, T *L, cudaStream_t st)
{
    if (p->dim == 2) return force_nl_dim<T, 2>(p, u, L, st);
    return force_nl_dim<T, 3>(p, u, L, st);
}

template pd_status force_nl<float>(pd_plan *, const float *, float *, cudaStream_t);
template pd_status force_nl<double>(pd_plan *, const double *, double *, cudaStream_t);

}  // namespace pd
