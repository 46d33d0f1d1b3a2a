// Shared device/host definitions of the GB300 FCBM-EC library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "pd.h"

namespace pd {

template <typename T>
struct cx {
    T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b)
{
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> conjg(cx<T> a) { return mk(a.x, -a.y); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> scale(cx<T> a, T s) { return mk(a.x * s, a.y * s); }
// multiply by i
template <typename T>
__host__ __device__ __forceinline__ cx<T> mul_i(cx<T> a) { return mk(-a.y, a.x); }

// Per-thread error detail (host side).
void set_error(const char *fmt, ...);

#define PD_CUDA_TRY(expr)                                                          \
    do {                                                                           \
        cudaError_t e__ = (expr);                                                  \
        if (e__ != cudaSuccess) {                                                  \
            ::pd::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e__), \
                            __FILE__, __LINE__);                                   \
            return PD_ERR_CUDA;                                                    \
        }                                                                          \
    } while (0)

#define PD_LAUNCH_CHECK()                                                          \
    do {                                                                           \
        cudaError_t e__ = cudaGetLastError();                                      \
        if (e__ != cudaSuccess) {                                                  \
            ::pd::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e__), \
                            __FILE__, __LINE__);                                   \
            return PD_ERR_CUDA;                                                    \
        }                                                                          \
    } while (0)

#define PD_TRY(expr)                        \
    do {                                    \
        pd_status s__ = (expr);             \
        if (s__ != PD_OK) return s__;       \
    } while (0)

__host__ __device__ __forceinline__ int ilog2(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

// Grid coordinates of linear node p (x1 fastest; n1, n2 powers of two).
__device__ __forceinline__ void node_coords(int64_t p, int n1, int n2, int &i1, int &i2, int &i3)
{
    const int l1 = __ffs(n1) - 1, l2 = __ffs(n2) - 1;
    i1 = (int)(p & (n1 - 1));
    i2 = (int)((p >> l1) & (n2 - 1));
    i3 = (int)(p >> (l1 + l2));
}

}  // namespace pd
