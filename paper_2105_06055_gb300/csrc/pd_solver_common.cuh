// Vector kernels shared by the static solvers (CG in pd_solve.cu, dynamic
// relaxation in pd_dr.cu): block partial sums into the plan's FP64 reduction
// buffer, their final reduction, the Dirichlet embedding u = w on Gamma
// (Eq. 74, 87), the FP64 residual R(u) = chi_O (b + L(u)) of Eq. 89 and the
// refinement update u += e.
#pragma once

#include "pd_plan.cuh"

namespace pd {
namespace {

constexpr int kUpdBlocks = 1024;  // blocks of the vector kernels
enum { S_RR = 0, S_PQ, S_ALPHA, S_BETA, S_RRNEW, S_NORM, S_BN, S_FLAG, S_COUNT };

// Sum of four doubles per thread over a block of kFinishThreads threads
// (valid in thread 0): warp shuffles, one shared-memory exchange.
constexpr int kFinishThreads = 256;
__device__ __forceinline__ void block_sum4(double &a, double &b, double &c, double &d)
{
    __shared__ double sh[4][kFinishThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
        d += __shfl_down_sync(0xffffffffu, d, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = a;
        sh[1][wid] = b;
        sh[2][wid] = c;
        sh[3][wid] = d;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = b = c = d = 0.0;
        for (int k = 0; k < kFinishThreads / 32; ++k) {
            a += sh[0][k];
            b += sh[1][k];
            c += sh[2][k];
            d += sh[3][k];
        }
    }
}

__device__ __forceinline__ void write_partial(double *red, double v)
{
    const double t = block_sum_d(v);
    if (threadIdx.x == 0) red[kRedPart + blockIdx.x] = t;
}

// the same for a compensated accumulator (FP32 pairs merged per warp)
__device__ __forceinline__ void write_partial(double *red, const DSum &acc)
{
    const DSum *a[1] = {&acc};
    double t[1];
    block_sums<1>(a, t);
    if (threadIdx.x == 0) red[kRedPart + blockIdx.x] = t[0];
}

// Final reduction of nparts block partials into scalar `dst`, then:
//   0: store only; 1: alpha = rr / pq; 2: beta = rrnew / rr, rr = rrnew
__global__ void k_finish(double *red, int nparts, int dst, int what)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += red[kRedPart + i];
    v = block_sum_d(v);
    if (threadIdx.x == 0) {
        double *s = red + kRedScal;
        s[dst] = v;
        if (!isfinite(v)) s[S_FLAG] = 1.0;
        if (what == 1) {
            s[S_ALPHA] = (v > 0.0) ? s[S_RR] / v : 0.0;
            if (!(v > 0.0)) s[S_FLAG] = 2.0;  // breakdown: p.Ap <= 0
        } else if (what == 2) {
            s[S_BETA] = (s[S_RR] > 0.0) ? v / s[S_RR] : 0.0;
            s[S_RR] = v;
        }
    }
}

// u = chi_O u + (1 - chi_O) w ; partial ||chi_O b||^2
__global__ void k_apply_bc(double *u, const double *w, const double *b, const uint8_t *co, int64_t n,
                           double *red)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = co[i] ? 1.0 : 0.0;
        u[i] = m * u[i] + (1.0 - m) * (w ? w[i] : 0.0);
        const double bb = m * b[i];
        acc += bb * bb;
    }
    write_partial(red, acc);
}

// r = chi_O (b + L) in place on L ; partial ||r||^2
__global__ void k_residual(double *r, const double *b, const uint8_t *co, int64_t n, double *red)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = co[i] ? (b[i] + r[i]) : 0.0;
        r[i] = v;
        acc += v * v;
    }
    write_partial(red, acc);
}

// u += e on Omega
template <typename T>
__global__ void k_ir_update(double *u, const T *e, const uint8_t *co, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (co[i]) u[i] += (double)e[i];
}

}  // namespace
}  // namespace pd
