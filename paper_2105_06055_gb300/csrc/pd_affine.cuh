// Affine split of the FP32 force evaluation (private).
//
// The FFT convolution's rounding error scales with the norm of the field it
// transforms (about eps ||chi u|| lam_max), while the force of an affine field
// a(x) = A x + t is known exactly: L(a)_i(x) = chi Σ_H chi' C_ij(xi) A_jk xi_k dV
// (Eq. 17-18 with u' - u = A xi), zero in the delta-interior, where the odd
// moments of the horizon vanish. A field dominated by its affine part (a
// uniform strain, the x-dependent part of a loading) therefore loses digits in
// FP32 that are not lost to the method itself. With the split,
//   L(u) = L(u - a) + L(a),
// a is the least-squares affine fit of u over the body, the transforms see
// only the remainder u - a, and L(a) is added at the boundary nodes from a
// plan-time table of moments. The fit is made exactly representable: with
// e = i - c the integer offset of a node from the body's centre node,
//   a_j(x) = t_j + Σ_k B_jk e_k,
// and t_j, B_jk rounded to multiples of a power of two q_j small enough that
// every partial sum is an integer multiple of q_j below 2^digits q_j, each
// step of its evaluation is exact in the plan's precision. The prologue and
// the boundary fix-up evaluate the same a and so subtract and add back the
// same field; the only rounding left is that of u - a itself.
#pragma once

#include <limits>

#include "pd_plan.cuh"

namespace pd {

// Coefficient layout (plan precision): B_jk at [3 j + k], t_j at [9 + j].
constexpr int kAffT = 9;

template <typename T>
struct AffineView {
    const T *coef;
    int c0, c1, c2;  // centre node
    int lg1, lg2;    // log2 n1, log2 n2
    // a_j at node (i1, row) with row = i2 + n2 i3; exact by construction
    __device__ __forceinline__ void at(int i1, int64_t row, int D, T *a) const
    {
        const T e0 = (T)(i1 - c0);
        const T e1 = (T)((int)(row & ((1 << lg2) - 1)) - c1);
        const T e2 = (T)((int)(row >> lg2) - c2);
        for (int j = 0; j < D; ++j) {
            T v = coef[kAffT + j] + coef[3 * j] * e0;
            v = v + coef[3 * j + 1] * e1;
            if (D == 3) v = v + coef[3 * j + 2] * e2;
            a[j] = v;
        }
    }
};

// Block partial sums of the fit: Σ chi u_j (D values) and Σ chi e_k u_j
// (D^2 values, index D + D j + k), in compensated FP32 (FP64 for FP64 fields).
template <typename T, int D>
__global__ void __launch_bounds__(256) k_aff_sums(const T *u, const uint8_t *chi, int lg1, int lg2, int c0, int c1,
                                                  int c2, int64_t N, double *red)
{
    constexpr int NV = D + D * D;
    DSum acc[NV];
    pdl_wait();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        if (!chi[p]) continue;
        const T e[3] = {(T)((int)(p & ((1 << lg1) - 1)) - c0), (T)((int)((p >> lg1) & ((1 << lg2) - 1)) - c1),
                        (T)((int)(p >> (lg1 + lg2)) - c2)};
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const T uj = u[j * N + p];
            acc[j].add(uj);
#pragma unroll
            for (int k = 0; k < D; ++k) acc[D + D * j + k].add(e[k] * uj);
        }
    }
    pdl_trigger();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double t = block_sum_d(acc[v].value());
        if (threadIdx.x == 0) red[kRedPart + (int64_t)blockIdx.x * NV + v] = t;
    }
}

struct AffFitArgs {
    double inv[16];   // (D+1)^2 inverse of [[S0, Se^T], [Se, See]]
    double emax[3];   // largest |e_k| over the box
    int nblk;
};

// The least-squares fit from the partial sums, rounded to exact form (one block).
template <typename T, int D>
__global__ void __launch_bounds__(256) k_aff_fit(const double *red, AffFitArgs a, T *coef)
{
    constexpr int NV = D + D * D;
    __shared__ double sums[NV];
    pdl_wait();
    for (int v = 0; v < NV; ++v) {
        double s = 0.0;
        for (int b = threadIdx.x; b < a.nblk; b += blockDim.x) s += red[kRedPart + (int64_t)b * NV + v];
        s = block_sum_d(s);
        if (threadIdx.x == 0) sums[v] = s;
        __syncthreads();
    }
    pdl_trigger();
    if (threadIdx.x != 0) return;
    constexpr int M = D + 1;
    for (int j = 0; j < D; ++j) {
        // normal equations [[S0, Se^T], [Se, See]] [t_j; B_j] = [Σ chi u_j; Σ chi e u_j]
        double rhs[4], sol[4];
        rhs[0] = sums[j];
        for (int k = 0; k < D; ++k) rhs[1 + k] = sums[D + D * j + k];
        for (int r = 0; r < M; ++r) {
            double s = 0.0;
            for (int c = 0; c < M; ++c) s += a.inv[r * M + c] * rhs[c];
            sol[r] = s;
        }
        double amax = fabs(sol[0]);
        for (int k = 0; k < D; ++k) amax += fabs(sol[1 + k]) * a.emax[k];
        bool ok = isfinite(amax) && amax > 0.0;
        double q = 0.0;
        if (ok) {
            // q = 2^(ceil(log2 amax) + 1 - digits): every partial sum of a_j stays a
            // multiple of q below 2^digits q after the rounding below
            int ex = 0;
            frexp(amax, &ex);  // amax < 2^ex
            q = ldexp(1.0, ex + 1 - std::numeric_limits<T>::digits);
        }
        coef[kAffT + j] = ok ? (T)(q * rint(sol[0] / q)) : T(0);
        for (int k = 0; k < 3; ++k) coef[3 * j + k] = (ok && k < D) ? (T)(q * rint(sol[1 + k] / q)) : T(0);
    }
}

// Symmetric-tensor component of (i, j) in Sym order (2D: 11, 22, 12; 3D: 11,
// 22, 33, 12, 13, 23)
__host__ __device__ constexpr int sym_index(int D, int i, int j)
{
    return i == j ? i : (D == 2 ? 2 : (i + j == 1 ? 3 : (i + j == 2 ? 4 : 5)));
}

// L(a)_i at a boundary entry: Σ_jk B_jk M_(ij)k with the table row m
template <typename T, int D>
__device__ __forceinline__ void aff_force(const T *coef, const T *m, T *out)
{
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const int q = sym_index(D, i, j);
#pragma unroll
            for (int k = 0; k < D; ++k) acc += coef[3 * j + k] * m[q * D + k];
        }
        out[i] = acc;
    }
}

}  // namespace pd
