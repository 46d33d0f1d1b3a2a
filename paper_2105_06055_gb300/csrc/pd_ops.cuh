// Per-node and per-mode functors of the FCBM-EC operators (private).
//
// Notation: v = chi_B s is the node weight (s = 1, lambda or sqrt(c/c0)),
// conv_M(f) = IFFT(M^ FFT(f)) = C*f dV - P f with M^ = (K^(k) - K^(0))/N
// (Eq. 56-57; the 1/N of the inverse transform is folded into M^), and
// G_ij = conv_M(v)_ij. Then, algebraically identical to Eq. 100-102,
//   L_i = v [ conv_M(v u_j)_i - G_ij u_j ]
//   W   = 1/2 v [ Σ_ij conv_M(v u_i u_j)_ij - 2 u_i conv_M(v u_j)_i + u_i G_ij u_j ]
// (the P terms cancel exactly), which avoids the cancellation between
// C*(v u) and (C*v) u in finite precision. For v = chi_B, G is zero in the
// delta-interior and is kept as a sparse list of boundary nodes; the dense
// part of the epilogue stages L in shared memory and a sparse fix-up
// subtracts G u at the listed nodes before the rows are written.
#pragma once

#include "pd_affine.cuh"
#include "pd_plan.cuh"

namespace pd {

// component order of symmetric tensors
template <int D>
struct Sym;
template <>
struct Sym<2> {
    static constexpr int n = 3;
    __host__ __device__ static constexpr int i(int c) { return c == 0 ? 0 : c == 1 ? 1 : 0; }
    __host__ __device__ static constexpr int j(int c) { return c == 0 ? 0 : c == 1 ? 1 : 1; }
};
template <>
struct Sym<3> {
    static constexpr int n = 6;
    __host__ __device__ static constexpr int i(int c) { return c < 3 ? c : (c == 5 ? 1 : 0); }
    __host__ __device__ static constexpr int j(int c) { return c < 3 ? c : (c == 3 ? 1 : 2); }
};

template <typename T, int D>
__device__ __forceinline__ void mat_vec(const T *M, const cx<T> *x, cx<T> *y)
{
#pragma unroll
    for (int i = 0; i < D; ++i) {
        cx<T> acc = mk(T(0), T(0));
#pragma unroll
        for (int j = 0; j < D; ++j) acc = acc + scale(x[j], M[3 * i + j]);
        y[i] = acc;
    }
}

// y_i += G_ij x_j for a symmetric tensor stored in Sym order
template <typename T, int D>
__device__ __forceinline__ void sym_apply(const T *g, const T *x, T *y)
{
#pragma unroll
    for (int c = 0; c < Sym<D>::n; ++c) {
        const int a = Sym<D>::i(c), b = Sym<D>::j(c);
        y[a] += g[c] * x[b];
        if (a != b) y[b] += g[c] * x[a];
    }
}

template <typename T>
struct vec2;
template <>
struct vec2<float> {
    using type = float2;
};
template <>
struct vec2<double> {
    using type = double2;
};
template <typename T>
__device__ __forceinline__ typename vec2<T>::type load2(const T *p)
{
    return *reinterpret_cast<const typename vec2<T>::type *>(p);
}

template <typename T>
__device__ __forceinline__ void store2(T *p, T a, T b)
{
    typename vec2<T>::type v;
    v.x = a;
    v.y = b;
    *reinterpret_cast<typename vec2<T>::type *>(p) = v;
}

enum WeightMode { W_NONE = 0, W_S = 1, W_LAM = 2 };

// ---------------------------------------------------------------------------
// Forward prologue: fields v u_j (D) [and v u_i u_j (ncomp) when ENERGY]
// ---------------------------------------------------------------------------
// AFF: transform u - a instead of u, a the exact affine fit (pd_affine.cuh)
template <typename T, int D, bool ENERGY, int WM, bool AFF = false>
struct ProForce {
    static_assert(!AFF || (!ENERGY && WM == W_NONE), "the affine split is for the plain force");
    static constexpr int kFin = 0, kFout = D + (ENERGY ? Sym<D>::n : 0);
    static constexpr int kNF = D + (WM == W_S ? 1 : 0), kNB = 1 + (WM == W_LAM ? 1 : 0), kStage = 0;
    static constexpr bool kSparse = false;
    static constexpr bool kFixedLength = std::is_same_v<T, float> && !ENERGY && WM == W_NONE;
    const T *u;
    const T *s;
    const uint8_t *lam;
    const uint8_t *chi;
    int64_t N;
    cx<T> *spec;
    int64_t fstride;
    AffineView<T> aff;
    __device__ const cx<T> *spec_in(int) const { return nullptr; }
    __device__ cx<T> *spec_out(int f) const { return spec + f * fstride; }
    __device__ const T *nf_src(int k) const { return k < D ? u + k * N : s; }
    __device__ const uint8_t *nb_src(int k) const { return k == 0 ? chi : lam; }
    __device__ __forceinline__ void node1(const RowCtx<T> &c, int rl, int i1, T *out) const
    {
        T v = c.b(0, rl, i1) ? T(1) : T(0);
        if constexpr (WM == W_S) v *= c.f(D, rl, i1);
        if constexpr (WM == W_LAM) v *= c.b(1, rl, i1) ? T(1) : T(0);
        T uu[D];
#pragma unroll
        for (int j = 0; j < D; ++j) uu[j] = c.f(j, rl, i1);
        if constexpr (AFF) {
            T a[D];
            aff.at(i1, c.row0 + rl, D, a);
#pragma unroll
            for (int j = 0; j < D; ++j) uu[j] -= a[j];
        }
#pragma unroll
        for (int j = 0; j < D; ++j) out[j] = v * uu[j];
        if constexpr (ENERGY) {
#pragma unroll
            for (int q = 0; q < Sym<D>::n; ++q) out[D + q] = v * uu[Sym<D>::i(q)] * uu[Sym<D>::j(q)];
        }
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

// ---------------------------------------------------------------------------
// Spectral combine: Y_i = M^_ij X_j [, T = Σ_ij M^_ij Q_ij]
// ---------------------------------------------------------------------------
template <typename T, int D, bool ENERGY>
struct CombForce {
    static constexpr int kFin = D + (ENERGY ? Sym<D>::n : 0);
    static constexpr int kFout = D + (ENERGY ? 1 : 0);
    static constexpr int kMode = 2, kPre = 0, kTab = Sym<D>::n;
    static constexpr bool kStoreIn = false;
    Model<T> m;
    int obase;  // first output slot (kFin in 3D: the pass is out of place)
    __device__ int slot_in(int f) const { return f; }
    __device__ int slot_out(int f) const { return obase + f; }
    __device__ int slot_aux(int) const { return 0; }
    __device__ const T *table(int c) const { return m.mhat + c * m.fold_sz; }
    __device__ __forceinline__ void combine(const T *t, int cs, bool fy, bool fz, const cx<T> *in, cx<T> *out) const
    {
        T M[9];
        load_mhat_s(D, t, cs, fy, fz, M);
        mat_vec<T, D>(M, in, out);
        if constexpr (ENERGY) {
            cx<T> acc = mk(T(0), T(0));
#pragma unroll
            for (int c = 0; c < Sym<D>::n; ++c) {
                const int a = Sym<D>::i(c), b = Sym<D>::j(c);
                const T w = (a == b) ? M[3 * a + b] : T(2) * M[3 * a + b];
                acc = acc + scale(in[D + c], w);
            }
            out[D] = acc;
        }
    }
};

// ---------------------------------------------------------------------------
// Inverse epilogue, plan weight (v = chi_B): sparse boundary field
//   node2 : L_i = chi y_i, W = 1/2 chi (y_T - 2 u.y)  (staged)
//   emit  : at boundary nodes (gidx >= 0) L_i -= G_ij u_j, W += 1/2 u.G.u with
//           G from the boundary list; write the rows
// ---------------------------------------------------------------------------
// AFF: the transforms saw u - a; G applies to u - a and the exact L(a) is
// added from the boundary entry's moment row
template <typename T, int D, bool ENERGY, bool AFF = false>
struct EpiForceSparse {
    static_assert(!AFF || !ENERGY, "the affine split is for the plain force");
    static constexpr int kFin = D + (ENERGY ? 1 : 0), kFout = 0, kStage = D + (ENERGY ? 1 : 0);
    static constexpr int kNF = ENERGY ? D : 0, kNB = 1;
    static constexpr bool kSparse = false;
    static constexpr bool kFixedLength = std::is_same_v<T, float> && !ENERGY;
    const T *u;
    const uint8_t *chi;
    const GEntry<T> *gent;
    const int *gidx;
    T *L;
    T *W;
    int64_t N;
    int n1;
    const cx<T> *spec;
    int64_t fstride;
    AffineView<T> aff;
    const T *atab;  // [entries][Sym<D>::n * D]
    __device__ const cx<T> *spec_in(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_out(int) const { return nullptr; }
    __device__ const T *nf_src(int k) const { return u + k * N; }
    __device__ const uint8_t *nb_src(int) const { return chi; }
    __device__ __forceinline__ void node1(const RowCtx<T> &c, int rl, int i1, const T *in, T *o) const
    {
        const T v = c.b(0, rl, i1) ? T(1) : T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) o[i] = v * in[i];
        if constexpr (ENERGY) {
            T uc = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) uc += c.f(i, rl, i1) * in[i];
            o[D] = T(0.5) * v * (in[D] - T(2) * uc);
        }
    }
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *in0, const T *in1, T *o0,
                                          T *o1) const
    {
        node1(c, rl, i1, in0, o0);
        node1(c, rl, i1 + 1, in1, o1);
    }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    // boundary correction of one node (entry k of the list)
    __device__ __forceinline__ void fix(const RowCtx<T> &c, int rl, int i1, int64_t p, int k, T *s) const
    {
        const GEntry<T> e = gent[k];
        T uu[D], Gu[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            uu[j] = ENERGY ? c.f(j, rl, i1) : u[j * N + p];
            Gu[j] = T(0);
        }
        if constexpr (AFF) {
            T a[D], La[D];
            aff.at(i1, c.row0 + rl, D, a);
#pragma unroll
            for (int j = 0; j < D; ++j) uu[j] -= a[j];
            aff_force<T, D>(aff.coef, atab + (int64_t)k * (Sym<D>::n * D), La);
#pragma unroll
            for (int i = 0; i < D; ++i) s[i] += La[i];
        }
        sym_apply<T, D>(e.g, uu, Gu);
#pragma unroll
        for (int i = 0; i < D; ++i) s[i] -= Gu[i];
        if constexpr (ENERGY) {
            T ugu = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) ugu += uu[i] * Gu[i];
            s[D] += T(0.5) * ugu;
        }
    }
    __device__ __forceinline__ void emit(const RowCtx<T> &c, int rl, int i1, const T *s0, const T *s1,
                                         DSum &) const
    {
        const int64_t p = (c.row0 + rl) * n1 + i1;
        const int2 gi = *reinterpret_cast<const int2 *>(gidx + p);
        constexpr int S = D + (ENERGY ? 1 : 0);
        T a[S], b[S];
#pragma unroll
        for (int i = 0; i < S; ++i) {
            a[i] = s0[i];
            b[i] = s1[i];
        }
        if (gi.x >= 0) fix(c, rl, i1, p, gi.x, a);
        if (gi.y >= 0) fix(c, rl, i1 + 1, p + 1, gi.y, b);
#pragma unroll
        for (int i = 0; i < D; ++i) store2(L + i * N + p, a[i], b[i]);
        if constexpr (ENERGY) {
            if (W) store2(W + p, a[D], b[D]);
        }
    }
    __device__ void block_done(DSum &) const {}
};

// ---------------------------------------------------------------------------
// Inverse epilogue, node weight s or lambda: dense boundary field G^v
//   L_i = v (y_i - G_ij u_j), W = 1/2 v (y_T - 2 u.y + u.G.u)
// ---------------------------------------------------------------------------
template <typename T, int D, bool ENERGY, int WM>
struct EpiForceDense {
    static constexpr int NC = Sym<D>::n;
    static constexpr int kFin = D + (ENERGY ? 1 : 0), kFout = 0, kStage = 0;
    static constexpr int kNF = D + NC + (WM == W_S ? 1 : 0), kNB = 1 + (WM == W_LAM ? 1 : 0);
    static constexpr bool kSparse = false;
    const T *u;
    const T *s;
    const uint8_t *lam;
    const uint8_t *chi;
    const T *G;  // ncomp x N, for the same weight
    T *L;
    T *W;
    int64_t N;
    int n1;
    const cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_out(int) const { return nullptr; }
    __device__ const T *nf_src(int k) const { return k < D ? u + k * N : (k < D + NC ? G + (k - D) * N : s); }
    __device__ const uint8_t *nb_src(int k) const { return k == 0 ? chi : lam; }
    __device__ __forceinline__ void node1(const RowCtx<T> &c, int rl, int i1, const T *in, T *Lo, T &Wo) const
    {
        T v = c.b(0, rl, i1) ? T(1) : T(0);
        if constexpr (WM == W_S) v *= c.f(D + NC, rl, i1);
        if constexpr (WM == W_LAM) v *= c.b(1, rl, i1) ? T(1) : T(0);
        T uu[D], g[NC], Gu[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            uu[j] = c.f(j, rl, i1);
            Gu[j] = T(0);
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) g[q] = (v != T(0)) ? c.f(D + q, rl, i1) : T(0);
        sym_apply<T, D>(g, uu, Gu);
#pragma unroll
        for (int i = 0; i < D; ++i) Lo[i] = v * (in[i] - Gu[i]);
        if constexpr (ENERGY) {
            T uc = T(0), ugu = T(0);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                uc += uu[i] * in[i];
                ugu += uu[i] * Gu[i];
            }
            Wo = T(0.5) * v * (in[D] - T(2) * uc + ugu);
        }
    }
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *in0, const T *in1, T *,
                                          T *) const
    {
        T a[D], b[D], wa = T(0), wb = T(0);
        node1(c, rl, i1, in0, a, wa);
        node1(c, rl, i1 + 1, in1, b, wb);
        const int64_t p = (c.row0 + rl) * n1 + i1;
#pragma unroll
        for (int i = 0; i < D; ++i) store2(L + i * N + p, a[i], b[i]);
        if constexpr (ENERGY) {
            if (W) store2(W + p, wa, wb);
        }
    }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    __device__ void emit(const RowCtx<T> &, int, int, const T *, const T *, DSum &) const {}
    __device__ void block_done(DSum &) const {}
};

}  // namespace pd
