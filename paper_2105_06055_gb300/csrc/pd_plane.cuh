// Plane passes of the fused CG iteration (Eq. 85-89 on the convolution
// operator of Eq. 57-58) for cubic boxes whose x1-x2 plane of one field fits
// in shared memory (FP32, n1 = n2 <= 128: 64 x 128 packed values, 74 KB).
//
// The row/column scheme moves the spectra through global memory between the
// x1 (row) and the x2 (column) transforms, in both directions. Here one block
// owns one field of one x3-plane and runs both transforms on the plane in
// shared memory, so each CG iteration is
//   plane forward  : CG vector update, chi p, x1 R2C, x2 FFT      (one kernel)
//   last axis      : x3 FFT, spectral multiply, inverse x3 FFT   (k_cols)
//   G p            : (G p) per boundary-list entry   (k_gp_entries, beside the last axis)
//   plane inverse  : x2 inverse FFT, x1 C2R, L = chi y - G p, q, inner products
//   finish         : alpha, beta
// and the two column passes along x2 (a read and a write of every spectrum
// each) disappear. A block's field is one displacement component j: the CG
// vector updates act per component and the inner products are sums over
// components, so a block adds its component's share to the partial sums. The
// boundary term G p couples the components at boundary nodes only. It is
// computed per entry of the boundary list on the plan's second stream while
// the last-axis pass runs (p is final once the forward half is done), and the
// inverse block only reads its plane's entries (node, (G p)_j): the boundary
// nodes are far from evenly spread over the planes (every body node of the
// planes inside the body's faces is one), and with the dependent loads of the
// entry and of p at its node inside the inverse blocks, the blocks of those
// planes held up the whole pass.
//
// Same arithmetic as the row ops ProCG / EpiCG and the column passes: the same
// transforms (fft_ct), unpacking formulas and compensated sums.
#pragma once

#include "pd_fft.cuh"
#include "pd_ops.cuh"
#include "pd_plan.cuh"

namespace pd {
namespace {

template <typename T>
struct PlaneArgs {
    T *e, *r, *pv, *q;      // CG vectors: D components of N nodes each
    const uint8_t *bits;    // per node: bit 0 chi, bit 1 + i chi_Omega of component i
    cx<T> *spec;            // spectrum slots (fs complex each): the forward pass writes slots
                            // 0..D-1, the inverse pass reads slots D..2D-1
    int64_t fs, N;
    double *red;            // reduction buffer: partials and scalars
    const T *gpe;           // [D][nent] (G p) per boundary-list entry (k_gp_entries)
    const int *gnode;       // [nent] node of each entry
    const int *goff;        // per row: first entry of the row (nrows + 1 offsets; the list is ordered by node)
    int64_t nent;
    int lgl;                // log2 of the plan's twiddle table length
    int *err;               // device status word
    int *inject;            // failure-handling test hook (see k_rows): kind 5 stalls the inverse plane pass
};

constexpr int cmin(int a, int b) { return a < b ? a : b; }

template <typename T, int LGH, int LG2>
struct PlaneShape {
    static constexpr int H = 1 << LGH, n1 = 2 * H, n2 = 1 << LG2;
    static constexpr int PITCH = H + 8;  // complex per shared row: rows 8 eight-byte bank pairs apart
    static constexpr int NTR = H / kV;   // threads of one row transform
    static constexpr int NTC = n2 / kV;  // threads of one column transform
    static constexpr int THREADS = cmin(256, cmin(n2 * NTR, H * NTC));
    static constexpr int RROUND = THREADS / NTR;  // rows transformed at once, one per thread group
    static constexpr int CROUND = THREADS / NTC;  // columns transformed at once, one per thread group
    // a thread group transforms RF rows (CF columns) per sweep: the barriers
    // of a stage are shared and the transforms give each thread independent work
    static constexpr int RF = n2 / RROUND >= 2 ? 2 : 1;
    static constexpr int CF = H / CROUND >= 2 ? 2 : 1;
    static constexpr int SH = (LGH - kLgV >= 4) ? 4 : 3;  // swizzle shift of the row transforms
    static constexpr int LGT = LGH + 1;  // twiddle table W_n1 (n1 = n2)
    static constexpr size_t kTw = ((size_t)(1 << LGT) * sizeof(cx<T>) + 127) & ~(size_t)127;
    static constexpr size_t kPlane = (size_t)n2 * PITCH * sizeof(cx<T>);
    static constexpr size_t smem = kTw + kPlane + 16;  // + mbarrier
    static_assert(n2 % RROUND == 0 && H % CROUND == 0, "plane shape");
    static_assert(LG2 == LGH + 1, "cubic planes: one twiddle table W_n1 serves rows and columns");
};

// Forward unpack of one packed row after its complex FFT (in place): Z(k) of
// the even/odd split becomes X(k), k in [0, n1/2), slot 0 holding the real
// pair (X(0), X(n1/2)); as in the row passes.
template <typename T, int H>
__device__ __forceinline__ void unpack_fwd(cx<T> *z, int jt, int nt, const cx<T> *tws)
{
    const T half = T(0.5);
    for (int k = jt; k <= H / 2; k += nt) {
        if (k == 0) {
            const cx<T> z0 = z[0];
            z[0] = mk(z0.x + z0.y, z0.x - z0.y);
        } else {
            const int kk = H - k;
            const cx<T> a = z[k], b = z[kk];
            const cx<T> w = tws[k];
            const cx<T> xk = scale((a + conjg(b)) - mul_i(cmul(w, a - conjg(b))), half);
            if (kk != k) z[kk] = scale((b + conjg(a)) + mul_i(cmul(conjg(w), b - conjg(a))), half);
            z[k] = xk;
        }
    }
}

// Inverse unpack of one packed row (in place): X(k) -> conj(Z(k)), ready for
// the forward FFT that yields the real row (IDFT = conj DFT conj).
template <typename T, int H>
__device__ __forceinline__ void unpack_inv(cx<T> *z, int jt, int nt, const cx<T> *tws)
{
    for (int k = jt; k <= H / 2; k += nt) {
        if (k == 0) {
            const cx<T> p = z[0];
            z[0] = conjg(mk(p.x + p.y, p.x - p.y));
        } else {
            const int kk = H - k;
            const cx<T> a = z[k], b = z[kk];
            const cx<T> w = tws[k];
            const cx<T> zk = (a + conjg(b)) + mul_i(cmul(conjg(w), a - conjg(b)));
            if (kk != k) {
                const cx<T> zkk = (b + conjg(a)) - mul_i(cmul(w, b - conjg(a)));
                z[kk] = conjg(zkk);
            }
            z[k] = conjg(zk);
        }
    }
}

// Plane forward pass: pending CG update e += alpha p, r -= alpha q, partial
// r.r, p = r + beta p, then chi p of component j through x1 (R2C) and x2.
// One block per (x3 plane z, component j): blockIdx.x = z D + j.
template <typename T, int D, int LGH, int LG2>
__global__ void __launch_bounds__(PlaneShape<T, LGH, LG2>::THREADS, 3)
    k_plane_cg_fwd(PlaneArgs<T> a, const cx<T> *__restrict__ tw)
{
    using S = PlaneShape<T, LGH, LG2>;
    using V = typename vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cx<T> *tws = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *pl = reinterpret_cast<cx<T> *>(smem_raw + S::kTw);
    const int tid = threadIdx.x;
    const int j = blockIdx.x % D, z = blockIdx.x / D;
    for (int i = tid; i < (1 << S::LGT); i += S::THREADS) tws[i] = tw[i << (a.lgl - S::LGT)];
    pdl_wait();
    pdl_trigger();

    const int64_t base = (int64_t)z * S::n2 * S::n1 + (int64_t)j * a.N;
    const T alpha = (T)a.red[kRedScal + S_ALPHA], beta = (T)a.red[kRedScal + S_BETA];
    T *__restrict__ e = a.e + base;
    T *__restrict__ r = a.r + base;
    T *__restrict__ pv = a.pv + base;
    const T *__restrict__ q = a.q + base;
    const uint8_t *__restrict__ bits = a.bits + (int64_t)z * S::n2 * S::n1;
    DSum acc;
    // nodes 4 k ... 4 k + 3 of the plane: packed slots 2 k, 2 k + 1 of row 2 k >> LGH
    static_assert(std::is_same_v<T, float>, "16-byte vector accesses of FP32 fields");
#pragma unroll 2
    for (int k = tid; k < S::n2 * S::H / 2; k += S::THREADS) {
        const int i = 4 * k;
        const uchar4 b = *reinterpret_cast<const uchar4 *>(bits + i);
        const float4 ee = *reinterpret_cast<const float4 *>(e + i), rr = *reinterpret_cast<const float4 *>(r + i);
        const float4 pp = *reinterpret_cast<const float4 *>(pv + i), qq = *reinterpret_cast<const float4 *>(q + i);
        *reinterpret_cast<float4 *>(e + i) =
            make_float4(ee.x + alpha * pp.x, ee.y + alpha * pp.y, ee.z + alpha * pp.z, ee.w + alpha * pp.w);
        const float4 rn = make_float4(rr.x - alpha * qq.x, rr.y - alpha * qq.y, rr.z - alpha * qq.z,
                                      rr.w - alpha * qq.w);
        *reinterpret_cast<float4 *>(r + i) = rn;
        acc.add_prod(rn.x, rn.x);
        acc.add_prod(rn.y, rn.y);
        acc.add_prod(rn.z, rn.z);
        acc.add_prod(rn.w, rn.w);
        const float4 pn = make_float4(rn.x + beta * pp.x, rn.y + beta * pp.y, rn.z + beta * pp.z,
                                      rn.w + beta * pp.w);
        *reinterpret_cast<float4 *>(pv + i) = pn;
        const int slot = 2 * k;
        *reinterpret_cast<float4 *>(&pl[(slot >> LGH) * S::PITCH + (slot & (S::H - 1))]) =
            make_float4((b.x & 1) ? pn.x : 0.f, (b.y & 1) ? pn.y : 0.f, (b.z & 1) ? pn.z : 0.f, (b.w & 1) ? pn.w : 0.f);
    }
    __syncthreads();

    // x1: packed complex FFTs of the rows, then the R2C unpack
    {
        const int jt = tid % S::NTR, rf = tid / S::NTR;
#pragma unroll 1
        for (int r0 = 0; r0 < S::n2; r0 += S::RF * S::RROUND)
            fft_ct<T, S::RF, LGH, 0, S::SH>(pl + (r0 + rf) * S::PITCH, S::RROUND * S::PITCH, 1, jt, tws, LGH + 1,
                                            false, false);
#pragma unroll 1
        for (int r0 = 0; r0 < S::n2; r0 += S::RROUND)
            unpack_fwd<T, S::H>(pl + (r0 + rf) * S::PITCH, jt, S::NTR, tws);
        __syncthreads();
    }
    // x2: FFTs along the columns (lanes of a warp on consecutive columns)
    {
        const int col = tid % S::CROUND, jt = tid / S::CROUND;
#pragma unroll 1
        for (int c0 = 0; c0 < S::H; c0 += S::CF * S::CROUND)
            fft_ct<T, S::CF, LG2, 0, 0>(pl + c0 + col, S::CROUND, S::PITCH, jt, tws, S::LGT, false, false);
    }
    // store the plane's spectrum (slot j, rows z n2 ... z n2 + n2 - 1), two values per store
    cx<T> *dst = a.spec + (int64_t)j * a.fs + (int64_t)z * S::n2 * S::H;
    for (int idx = tid; idx < S::n2 * S::H / 2; idx += S::THREADS) {
        const int y = idx / (S::H / 2), k = 2 * (idx % (S::H / 2));
        const cx<T> v0 = pl[y * S::PITCH + k], v1 = pl[y * S::PITCH + k + 1];
        store2(reinterpret_cast<T *>(dst + (int64_t)y * S::H + k), v0.x, v0.y);
        store2(reinterpret_cast<T *>(dst + (int64_t)y * S::H + k + 1), v1.x, v1.y);
    }
    write_partial(a.red, acc);
}

// Plane inverse pass: x2 inverse FFT and x1 C2R of field j (slot D + j), then
// L_j = chi y_j - (G p)_j, q_j = -chi_Omega,j L_j and the partials of p.q, r.q,
// q.q. One block per (x3 plane z, component j): blockIdx.x = z D + j.
template <typename T, int D, int LGH, int LG2>
__global__ void __launch_bounds__(PlaneShape<T, LGH, LG2>::THREADS, 3)
    k_plane_cg_inv(PlaneArgs<T> a, const cx<T> *__restrict__ tw)
{
    using S = PlaneShape<T, LGH, LG2>;
    using V = typename vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cx<T> *tws = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *pl = reinterpret_cast<cx<T> *>(smem_raw + S::kTw);
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(smem_raw + S::kTw + S::kPlane);
    const int tid = threadIdx.x;
    const int j = blockIdx.x % D, z = blockIdx.x / D;
    const int64_t pbase = (int64_t)z * S::n2 * S::n1;  // first node of the plane
    if (tid == 0) mbar_init(mbar, 1);
    for (int i = tid; i < (1 << S::LGT); i += S::THREADS) tws[i] = tw[i << (a.lgl - S::LGT)];
    __syncthreads();
    pdl_wait();
    pdl_trigger();
    if (tid == 0) {
        // test hook: one-shot, so a pass captured in a graph stalls on one replay only
        const bool stall = a.inject && blockIdx.x == 0 && atomicCAS(a.inject, 6, 0) == 6;
        if (!stall) {
            const cx<T> *src = a.spec + (int64_t)(D + j) * a.fs + (int64_t)z * S::n2 * S::H;
            mbar_expect_tx(mbar, (unsigned)(S::n2 * S::H * sizeof(cx<T>)));
            for (int y = 0; y < S::n2; ++y)
                bulk_load(pl + y * S::PITCH, src + (int64_t)y * S::H, S::H * sizeof(cx<T>), mbar);
        }
    }
    const bool ok = mbar_wait(mbar, 0, a.err);
    if (__syncthreads_or(!ok)) return;  // no copy in flight: the stalled block issued none
    if (tid == 0) {
        // p_j, r_j and the mask bytes towards L2 while the plane is transformed
        // (issued once the spectrum is in, so they do not compete with it)
        const unsigned nb = (unsigned)(S::n2 * S::n1 * sizeof(T));
        bulk_prefetch_l2(a.pv + (int64_t)j * a.N + pbase, nb);
        bulk_prefetch_l2(a.r + (int64_t)j * a.N + pbase, nb);
        bulk_prefetch_l2(a.bits + pbase, (unsigned)(S::n2 * S::n1));
    }

    // x2: inverse FFTs along the columns (IDFT = conj DFT conj)
    {
        const int col = tid % S::CROUND, jt = tid / S::CROUND;
#pragma unroll 1
        for (int c0 = 0; c0 < S::H; c0 += S::CF * S::CROUND)
            fft_ct<T, S::CF, LG2, 0, 0>(pl + c0 + col, S::CROUND, S::PITCH, jt, tws, S::LGT, true, true);
    }
    // x1: C2R unpack, then the packed complex FFT of each row
    {
        const int jt = tid % S::NTR, rf = tid / S::NTR;
#pragma unroll 1
        for (int r0 = 0; r0 < S::n2; r0 += S::RROUND)
            unpack_inv<T, S::H>(pl + (r0 + rf) * S::PITCH, jt, S::NTR, tws);
        __syncthreads();
#pragma unroll 1
        for (int r0 = 0; r0 < S::n2; r0 += S::RF * S::RROUND)
            fft_ct<T, S::RF, LGH, 0, S::SH>(pl + (r0 + rf) * S::PITCH, S::RROUND * S::PITCH, 1, jt, tws, LGH + 1,
                                            false, false);
    }

    // boundary term: (G p)_j of the plane's boundary entries (contiguous in the
    // list) subtracted from y_j in shared memory; the two nodes of a packed slot
    // are its two halves, so no two entries write the same word
    {
        const int e0 = a.goff[z * S::n2], e1 = a.goff[(z + 1) * S::n2];
        const T *gj = a.gpe + (int64_t)j * a.nent;
        for (int e = e0 + tid; e < e1; e += S::THREADS) {
            const int nd = (int)(a.gnode[e] - pbase);  // node within the plane
            const T g = gj[e];
            cx<T> &w = pl[(nd >> (LGH + 1)) * S::PITCH + ((nd & (S::n1 - 1)) >> 1)];
            if (nd & 1)
                w.y += g;  // the odd node of the slot holds -Im w
            else
                w.x -= g;
        }
        __syncthreads();
    }

    const T *__restrict__ pj = a.pv + (int64_t)j * a.N + pbase;
    const T *__restrict__ rj = a.r + (int64_t)j * a.N + pbase;
    T *__restrict__ qj = a.q + (int64_t)j * a.N + pbase;
    const uint8_t *bits = a.bits + pbase;
    DSum pq, rq, qq;
    // nodes 2 idx, 2 idx + 1 of the plane: L_j = chi (y_j - (G p)_j) = (Re w, -Im w)
    // of packed slot idx where chi = 1 (the boundary list holds chi = 1 nodes only)
#pragma unroll 2
    for (int idx = tid; idx < S::n2 * S::H; idx += S::THREADS) {
        const int i = 2 * idx;
        const cx<T> w = pl[(idx >> LGH) * S::PITCH + (idx & (S::H - 1))];
        const uchar2 b = *reinterpret_cast<const uchar2 *>(bits + i);
        const V pp = __ldg(reinterpret_cast<const V *>(pj + i));
        const V rr = __ldg(reinterpret_cast<const V *>(rj + i));
        const T L0 = (b.x & 1) ? w.x : T(0), L1 = (b.y & 1) ? -w.y : T(0);
        const T qa = ((b.x >> (1 + j)) & 1) ? -L0 : T(0);
        const T qb = ((b.y >> (1 + j)) & 1) ? -L1 : T(0);
        store2(qj + i, qa, qb);
        pq.add_prod(pp.x, qa);
        pq.add_prod(pp.y, qb);
        rq.add_prod(rr.x, qa);
        rq.add_prod(rr.y, qb);
        qq.add_prod(qa, qa);
        qq.add_prod(qb, qb);
    }
    const DSum *acc[3] = {&pq, &rq, &qq};
    double t[3];
    block_sums<3>(acc, t);
    if (tid == 0) {
        double *o = a.red + kRedPart + kPartB + 3 * blockIdx.x;
        o[0] = t[0];
        o[1] = t[1];
        o[2] = t[2];
    }
}

// (G p) of every boundary-list entry, component-major: gpe[j nent + e] (the
// same products and order as the row passes' boundary term).
template <typename T, int D>
__global__ void __launch_bounds__(256) k_gp_entries(const GEntry<T> *__restrict__ gent, int64_t nent,
                                                    const T *__restrict__ pv, int64_t N, T *__restrict__ gpe)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += (int64_t)gridDim.x * blockDim.x) {
        const GEntry<T> ge = gent[e];
        T x[D], y[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            x[k] = pv[(int64_t)k * N + ge.p];
            y[k] = T(0);
        }
        sym_apply<T, D>(ge.g, x, y);
#pragma unroll
        for (int k = 0; k < D; ++k) gpe[(int64_t)k * nent + e] = y[k];
    }
}

}  // namespace
}  // namespace pd
