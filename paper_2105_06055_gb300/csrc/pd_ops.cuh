// Per-node and per-mode functors of the FCBM-EC operators (private).
//
// Notation: v = chi_B s is the node weight (s = 1, lambda or sqrt(c/c0)),
// conv_M(f) = IFFT(M^ FFT(f)) = C*f dV - P f with M^ = (K^(k) - K^(0))/N
// (Eq. 56-57; the 1/N of the inverse transform is folded into M^), and
// G_ij = conv_M(v)_ij. Then, algebraically identical to Eq. 100-102,
//   L_i = v [ conv_M(v u_j)_i - G_ij u_j ]
//   W   = 1/2 v [ Σ_ij conv_M(v u_i u_j)_ij - 2 u_i conv_M(v u_j)_i + u_i G_ij u_j ]
// (the P terms cancel exactly), which avoids the cancellation between
// C*(v u) and (C*v) u in finite precision.
#pragma once

#include "pd_plan.cuh"

namespace pd {

// component order of symmetric tensors
template <int D>
struct Sym;
template <>
struct Sym<2> {
    static constexpr int n = 3;
    __device__ static constexpr int i(int c) { return c == 0 ? 0 : c == 1 ? 1 : 0; }
    __device__ static constexpr int j(int c) { return c == 0 ? 0 : c == 1 ? 1 : 1; }
};
template <>
struct Sym<3> {
    static constexpr int n = 6;
    __device__ static constexpr int i(int c) { return c < 3 ? c : (c == 5 ? 1 : 0); }
    __device__ static constexpr int j(int c) { return c < 3 ? c : (c == 3 ? 1 : 2); }
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

// ---------------------------------------------------------------------------
// Forward prologue: fields v u_j (D) [and v u_i u_j (ncomp) when ENERGY]
// ---------------------------------------------------------------------------
template <typename T, int D, bool ENERGY>
struct ProForce {
    static constexpr int kFin = 0;
    static constexpr int kFout = D + (ENERGY ? Sym<D>::n : 0);
    const T *u;
    const T *s;           // node weight or null
    const uint8_t *lam;   // integrity index or null
    const uint8_t *chi;
    int64_t N;
    int n1;
    cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int) const { return nullptr; }
    __device__ cx<T> *spec_out(int f) const { return spec + f * fstride; }
    __device__ __forceinline__ void node(int64_t row, int i1, const T *, T *out) const
    {
        const int64_t p = row * n1 + i1;
        T v = chi[p] ? T(1) : T(0);
        if (s) v *= s[p];
        if (lam) v *= lam[p] ? T(1) : T(0);
        T uu[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            uu[j] = u[j * N + p];
            out[j] = v * uu[j];
        }
        if constexpr (ENERGY) {
#pragma unroll
            for (int c = 0; c < Sym<D>::n; ++c) out[D + c] = v * uu[Sym<D>::i(c)] * uu[Sym<D>::j(c)];
        }
    }
};

// ---------------------------------------------------------------------------
// Spectral combine: Y_i = M^_ij X_j [, T = Σ_ij M^_ij Q_ij]
// ---------------------------------------------------------------------------
template <typename T, int D, bool ENERGY>
struct CombForce {
    static constexpr int kFin = D + (ENERGY ? Sym<D>::n : 0);
    static constexpr int kFout = D + (ENERGY ? 1 : 0);
    static constexpr int kMode = 2, kPre = 0;
    static constexpr bool kStoreIn = false;
    Model<T> m;
    cx<T> *spec;
    int64_t fstride;
    int obase;  // first output slot (kFin in 3D: the pass is out of place)
    __device__ const cx<T> *spec_in(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_out(int f) const { return spec + (obase + f) * fstride; }
    __device__ cx<T> *spec_aux(int) const { return nullptr; }
    __device__ __forceinline__ void combine(int kx, int ky, int kz, const cx<T> *in, cx<T> *out) const
    {
        T M[9];
        const SpecIdx<T> si = spec_index(m, kx, ky, kz);
        load_mhat(m, si, M);
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
// Inverse epilogue: L_i = v (conv_i - G_ij u_j) [, W]
// ---------------------------------------------------------------------------
template <typename T, int D, bool ENERGY>
struct EpiForce {
    static constexpr int kFin = D + (ENERGY ? 1 : 0);
    static constexpr int kFout = 0;
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
    __device__ __forceinline__ void node(int64_t row, int i1, const T *in, T *) const
    {
        const int64_t p = row * n1 + i1;
        T v = chi[p] ? T(1) : T(0);
        if (s) v *= s[p];
        if (lam) v *= lam[p] ? T(1) : T(0);
        T uu[D], g[Sym<D>::n];
#pragma unroll
        for (int j = 0; j < D; ++j) uu[j] = u[j * N + p];
#pragma unroll
        for (int c = 0; c < Sym<D>::n; ++c) g[c] = (v != T(0)) ? G[c * N + p] : T(0);
        T Gu[D];
#pragma unroll
        for (int i = 0; i < D; ++i) Gu[i] = T(0);
#pragma unroll
        for (int c = 0; c < Sym<D>::n; ++c) {
            const int a = Sym<D>::i(c), b = Sym<D>::j(c);
            Gu[a] += g[c] * uu[b];
            if (a != b) Gu[b] += g[c] * uu[a];
        }
#pragma unroll
        for (int i = 0; i < D; ++i) L[i * N + p] = v * (in[i] - Gu[i]);
        if constexpr (ENERGY) {
            if (W) {
                T uc = T(0), ugu = T(0);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    uc += uu[i] * in[i];
                    ugu += uu[i] * Gu[i];
                }
                W[p] = T(0.5) * v * (in[D] - T(2) * uc + ugu);
            }
        }
    }
};

}  // namespace pd
