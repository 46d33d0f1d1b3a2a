// Shared-memory Stockham FFT passes for the FCBM-EC convolutions.
//
// The convolutions of Eq. 57-65 and 95-102 are evaluated with the DFT of
// Eq. 53-54 on the periodic box. A d-dimensional transform is split into
// passes over one axis at a time; every pass moves whole tiles between HBM and
// shared memory once, and the pointwise work of the method (masking by chi,
// products with u, the spectral multiply by the kernel spectrum, the final
// mask and the Verlet/damage updates) is fused into the first and last pass so
// that no field makes an extra round trip:
//
//   row pass     (x1, contiguous):  real -> packed half spectrum or back,
//                                   with a per-node prologue / epilogue;
//   column pass  (x2 or x3, strided): complex FFT over a W-column tile,
//                                   optionally forward FFT, per-mode spectral
//                                   combine of all fields, inverse FFT.
//
// Packed half spectrum: a real row of n1 samples x[0..n1) becomes n1/2
// complex values X(k), k in [0, n1/2), with slot 0 holding the two real
// values (X(0), X(n1/2)). After the column transforms, slot kx = 0 holds
// X^(0,k') + i X^(n1/2,k') for every (k2,k3); the spectral combine unpacks it
// with the mirror mode (-k2,-k3).
//
// The in-register DFTs are radix 2/4/8/16 (radix-2 butterflies with the
// eighth roots of unity as constants); inter-stage data moves through shared
// memory in Stockham autosort order (no bit reversal pass). Each thread owns
// 16 complex values per stage; a transform of length L uses L/16 threads.
// Inverse transforms reuse the forward code: IDFT(x) = conj(DFT(conj(x))).
#pragma once

#include "pd_common.cuh"

namespace pd {

__host__ __device__ constexpr int bit_reverse(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// a * e^{-2 pi i m / 16}, m in [0, 8)
template <typename T>
__device__ __forceinline__ cx<T> rot16(cx<T> a, int m)
{
    const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173);
    const T r2 = T(0.70710678118654752440);
    switch (m) {
        case 0: return a;
        case 1: return cmul(a, mk(c1, -s1));
        case 2: return mk((a.x + a.y) * r2, (a.y - a.x) * r2);
        case 3: return cmul(a, mk(s1, -c1));
        case 4: return mk(a.y, -a.x);
        case 5: return cmul(a, mk(-s1, -c1));
        case 6: return mk((a.y - a.x) * r2, -(a.x + a.y) * r2);
        default: return cmul(a, mk(-c1, -s1));
    }
}

// Forward DFT of R values in registers (natural order in and out).
template <typename T, int R>
__device__ __forceinline__ void dft_reg(cx<T> *v)
{
    constexpr int bits = (R == 2) ? 1 : (R == 4) ? 2 : (R == 8) ? 3 : 4;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = bit_reverse(i, bits);
        if (i < j) {
            cx<T> t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int h = 1; h < R; h <<= 1) {
#pragma unroll
        for (int i = 0; i < R; i += 2 * h) {
#pragma unroll
            for (int k = 0; k < h; ++k) {
                cx<T> a = v[i + k];
                cx<T> b = rot16(v[i + k + h], k * (8 / h));
                v[i + k] = a + b;
                v[i + k + h] = a - b;
            }
        }
    }
}

// One radix-R Stockham stage of a length-n transform stored at s[e * stride].
// Thread jt (of nt = n/16) handles butterflies j = jt + b nt, b < 16/R.
// tw[i] = e^{-2 pi i i / 2^lgl}. Ends with a block-wide barrier.
template <typename T, int R>
__device__ __forceinline__ void fft_stage(cx<T> *s, int stride, int n, int ns, int lgnsr, int jt,
                                          int nt, const cx<T> *__restrict__ tw, int lgl)
{
    constexpr int B = 16 / R;
    cx<T> v[16];
    const int q = n / R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = jt + b * nt;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = s[(j + r * q) * stride];
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = jt + b * nt;
        const int k = j & (ns - 1);
        if (ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], tw[(r * k) << (lgl - lgnsr)]);
        }
        dft_reg<T, R>(&v[b * R]);
        const int o = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) s[(o + r * ns) * stride] = v[b * R + r];
    }
    __syncthreads();
}

// Forward DFT of length 2^lgn (>= 16) in shared memory, in place.
template <typename T>
__device__ __forceinline__ void fft_smem(cx<T> *s, int stride, int lgn, int jt,
                                         const cx<T> *__restrict__ tw, int lgl)
{
    const int n = 1 << lgn, nt = n >> 4;
    int ns = 1, lgns = 0, rem = lgn;
    while (rem > 0) {
        const int lr = rem >= 4 ? 4 : rem;
        switch (lr) {
            case 4: fft_stage<T, 16>(s, stride, n, ns, lgns + 4, jt, nt, tw, lgl); break;
            case 3: fft_stage<T, 8>(s, stride, n, ns, lgns + 3, jt, nt, tw, lgl); break;
            case 2: fft_stage<T, 4>(s, stride, n, ns, lgns + 2, jt, nt, tw, lgl); break;
            default: fft_stage<T, 2>(s, stride, n, ns, lgns + 1, jt, nt, tw, lgl); break;
        }
        ns <<= lr;
        lgns += lr;
        rem -= lr;
    }
}

// ---------------------------------------------------------------------------
// Row pass
// ---------------------------------------------------------------------------

struct RowGeom {
    int lgh;        // log2(n1/2): complex length of a packed row
    int rows;       // rows per block
    int pitch;      // shared-memory pitch of a row (complex elements)
    int64_t nrows;  // n2 * n3 (multiple of rows)
    int lgl;        // log2 of the twiddle table length
};

// Op interface (all device):
//   static constexpr int kFin, kFout;       packed spectra read / written
//   const cx<T>* spec_in(int f) const;      row-major [row][n1/2] packed spectra
//   cx<T>*       spec_out(int f) const;
//   void node(int64_t row, int i1, const T* in, T* out) const;
//        in:  kFin inverse-transformed values at the node (unnormalised IDFT)
//        out: kFout real values to transform forward
// With kFin == 0, node() is a prologue; with kFout == 0, an epilogue.
template <typename T, class Op>
__global__ void __launch_bounds__(256) k_rows(RowGeom g, Op op, const cx<T> *__restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    constexpr int FI = Op::kFin, FO = Op::kFout;
    constexpr int FB = FI > FO ? FI : FO;
    const int H = 1 << g.lgh, nt = H >> 4;
    const int jt = threadIdx.x % nt, rl = threadIdx.x / nt;
    const int64_t row = (int64_t)blockIdx.x * g.rows + rl;
    const int lg1 = g.lgh + 1;  // log2(n1)
    const int tshift1 = g.lgl - lg1;

    if constexpr (FI > 0) {
#pragma unroll
        for (int f = 0; f < FI; ++f) {
            const cx<T> *src = op.spec_in(f) + row * H;
            cx<T> *dst = sm + (f * g.rows + rl) * g.pitch;
            for (int k = jt; k < H; k += nt) dst[k] = src[k];
        }
        __syncthreads();
        // Unpack the half spectrum into Z(k) = E(k) + i O(k) (E, O: DFTs of the
        // even / odd samples, times 2) and store conj(Z) for the inverse.
#pragma unroll
        for (int f = 0; f < FI; ++f) {
            cx<T> *z = sm + (f * g.rows + rl) * g.pitch;
            for (int k = jt; k <= H / 2; k += nt) {
                if (k == 0) {
                    const cx<T> p = z[0];  // (X(0), X(n1/2))
                    z[0] = conjg(mk(p.x + p.y, p.x - p.y));
                } else {
                    const int kk = H - k;
                    const cx<T> a = z[k], b = z[kk];
                    const cx<T> w = tw[k << tshift1];  // W^k, W = e^{-2 pi i / n1}
                    // Z(k)  = (a + conj b) + i conj(W^k) (a - conj b)
                    const cx<T> s1 = a + conjg(b), d1 = a - conjg(b);
                    const cx<T> zk = s1 + mul_i(cmul(conjg(w), d1));
                    if (kk != k) {
                        // Z(H-k) = (b + conj a) - i W^k (b - conj a)
                        const cx<T> s2 = b + conjg(a), d2 = b - conjg(a);
                        const cx<T> zkk = s2 - mul_i(cmul(w, d2));
                        z[kk] = conjg(zkk);
                    }
                    z[k] = conjg(zk);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int f = 0; f < FI; ++f)
            fft_smem<T>(sm + (f * g.rows + rl) * g.pitch, 1, g.lgh, jt, tw, g.lgl);
        // x[2n] = Re w[n], x[2n+1] = -Im w[n]
        for (int n = jt; n < H; n += nt) {
            T in0[FI > 0 ? FI : 1], in1[FI > 0 ? FI : 1];
            T o0[FO > 0 ? FO : 1], o1[FO > 0 ? FO : 1];
#pragma unroll
            for (int f = 0; f < FI; ++f) {
                const cx<T> w = sm[(f * g.rows + rl) * g.pitch + n];
                in0[f] = w.x;
                in1[f] = -w.y;
            }
            op.node(row, 2 * n, in0, o0);
            op.node(row, 2 * n + 1, in1, o1);
#pragma unroll
            for (int f = 0; f < FO; ++f) sm[(f * g.rows + rl) * g.pitch + n] = mk(o0[f], o1[f]);
        }
        __syncthreads();
    } else {
        for (int n = jt; n < H; n += nt) {
            T o0[FO > 0 ? FO : 1], o1[FO > 0 ? FO : 1];
            op.node(row, 2 * n, nullptr, o0);
            op.node(row, 2 * n + 1, nullptr, o1);
#pragma unroll
            for (int f = 0; f < FO; ++f) sm[(f * g.rows + rl) * g.pitch + n] = mk(o0[f], o1[f]);
        }
        __syncthreads();
    }
    (void)FB;

    if constexpr (FO > 0) {
#pragma unroll
        for (int f = 0; f < FO; ++f)
            fft_smem<T>(sm + (f * g.rows + rl) * g.pitch, 1, g.lgh, jt, tw, g.lgl);
        const T half = T(0.5);
#pragma unroll
        for (int f = 0; f < FO; ++f) {
            const cx<T> *z = sm + (f * g.rows + rl) * g.pitch;
            cx<T> *dst = op.spec_out(f) + row * H;
            for (int k = jt; k <= H / 2; k += nt) {
                if (k == 0) {
                    const cx<T> z0 = z[0];
                    dst[0] = mk(z0.x + z0.y, z0.x - z0.y);
                } else {
                    const int kk = H - k;
                    const cx<T> a = z[k], b = z[kk];
                    const cx<T> w = tw[k << tshift1];
                    // X(k) = 1/2 [(a + conj b) - i W^k (a - conj b)]
                    const cx<T> xk = scale((a + conjg(b)) - mul_i(cmul(w, a - conjg(b))), half);
                    dst[k] = xk;
                    if (kk != k) {
                        // X(H-k) = 1/2 [(b + conj a) + i conj(W^k) (b - conj a)]
                        const cx<T> xkk =
                            scale((b + conjg(a)) + mul_i(cmul(conjg(w), b - conjg(a))), half);
                        dst[kk] = xkk;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Column pass
// ---------------------------------------------------------------------------

struct ColGeom {
    int lgl;            // log2 of the transform length (axis length)
    int w;              // tile width (columns, power of two, divides `inner`)
    int pitch;          // shared-memory pitch of a tile row (>= w + 1)
    int mirror;         // 1: 3D last-axis pass, load the mirror of column kx = 0
    int64_t inner;      // number of contiguous columns per outer index
    int64_t rowstride;  // elements between consecutive positions along the axis
    int64_t outerstride;
    int lgh;            // log2(n1/2) (packed row length), for mode coordinates
    int n2;             // n2 (3D mirror of k2)
    int lgtw;           // log2 of the twiddle table length
};

// Op interface:
//   static constexpr int kFin, kFout;
//   static constexpr int kMode;   0: forward FFT only, 1: inverse FFT only,
//                                 2: forward FFT, combine, inverse FFT
//   static constexpr int kPre;    (kMode 2) leading inputs already transformed
//                                 along this axis: loaded without an FFT
//   static constexpr bool kStoreIn; (kMode 2) write the transformed inputs to
//                                 spec_aux(f) before the combine
//   cx<T>* spec_aux(int f) const;
//   const cx<T>* spec_in(int f) const; cx<T>* spec_out(int f) const;
//   void combine(int kx, int ky, int kz, const cx<T>* in, cx<T>* out) const;
//        (kMode 2; called for true modes with kx in [0, n1/2], so both the
//         kx = 0 and kx = n1/2 halves of the packed column are visited)
// Shared memory: max(kFin, kFout) x L x pitch complex.
template <typename T, class Op>
__global__ void __launch_bounds__(512) k_cols(ColGeom g, Op op, const cx<T> *__restrict__ tw,
                                               int axis_is_z)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    constexpr int FI = Op::kFin, FO = Op::kFout, MODE = Op::kMode;
    constexpr int FB = FI > FO ? FI : FO;
    const int L = 1 << g.lgl, nt = L >> 4;
    const int ncol = g.w + g.mirror;
    const int col = threadIdx.x % ncol, jt = threadIdx.x / ncol;
    const int64_t c0 = (int64_t)blockIdx.x * g.w;
    const int64_t obase = (int64_t)blockIdx.y * g.outerstride;
    const int H = 1 << g.lgh;
    const int nthreads = ncol * nt;
    const int fsz = L * g.pitch;  // complex elements per field in smem
    // mirror column (3D last axis): kx = 0 of k2' = (n2 - k2) mod n2
    int64_t mcol = -1;
    int ky_tile = 0;
    if (g.mirror) {
        ky_tile = (int)(c0 >> g.lgh);
        if ((c0 & (H - 1)) == 0) mcol = (int64_t)((g.n2 - ky_tile) & (g.n2 - 1)) << g.lgh;
    }
    const bool conj_in = (MODE == 1);

    // ---- load
#pragma unroll
    for (int f = 0; f < FI; ++f) {
        const cx<T> *src = op.spec_in(f) + obase;
        cx<T> *dst = sm + f * fsz;
        for (int idx = threadIdx.x; idx < L * g.w; idx += nthreads) {
            const int r = idx / g.w, c = idx % g.w;
            cx<T> v = src[(int64_t)r * g.rowstride + c0 + c];
            dst[r * g.pitch + c] = conj_in ? conjg(v) : v;
        }
        if (g.mirror) {
            for (int r = threadIdx.x; r < L; r += nthreads)
                dst[r * g.pitch + g.w] = (mcol >= 0) ? src[(int64_t)r * g.rowstride + mcol] : mk(T(0), T(0));
        }
    }
    __syncthreads();
    constexpr int FPRE = (MODE == 2) ? Op::kPre : 0;
#pragma unroll
    for (int f = FPRE; f < FI; ++f) fft_smem<T>(sm + f * fsz + col, g.pitch, g.lgl, jt, tw, g.lgtw);

    if constexpr (MODE == 2 && Op::kStoreIn) {
#pragma unroll
        for (int f = FPRE; f < FI; ++f) {
            cx<T> *dst = op.spec_aux(f) + obase;
            const cx<T> *srcs = sm + f * fsz;
            for (int idx = threadIdx.x; idx < L * g.w; idx += nthreads) {
                const int r = idx / g.w, c = idx % g.w;
                dst[(int64_t)r * g.rowstride + c0 + c] = srcs[r * g.pitch + c];
            }
        }
    }

    if constexpr (MODE == 2) {
        // ---- spectral combine, writes conj(output) for the inverse
        for (int idx = threadIdx.x; idx < L * g.w; idx += nthreads) {
            const int r = idx / g.w, c = idx % g.w;
            const int64_t ic = c0 + c;
            int kx, ky, kz;
            if (axis_is_z) {
                kz = r;
                ky = (int)(ic >> g.lgh);
                kx = (int)(ic & (H - 1));
            } else {
                kz = 0;
                ky = r;
                kx = (int)ic;
            }
            cx<T> in[FB], out[FB];
            if (kx != 0) {
#pragma unroll
                for (int f = 0; f < FI; ++f) in[f] = sm[f * fsz + r * g.pitch + c];
                op.combine(kx, ky, kz, in, out);
#pragma unroll
                for (int f = 0; f < FO; ++f) sm[f * fsz + r * g.pitch + c] = conjg(out[f]);
            } else if (axis_is_z) {
                // packed column: mirror (-ky, -kz) is row (L - r) of the extra column
                // (or of this column when ky is its own mirror)
                const int rm = (L - r) & (L - 1);
                const int cm = (mcol == c0 + c) ? c : g.w;  // ky == -ky: same column
                cx<T> a[FB], b[FB], ya[FB], yb[FB];
#pragma unroll
                for (int f = 0; f < FI; ++f) {
                    const cx<T> z = sm[f * fsz + r * g.pitch + c];
                    const cx<T> zm = conjg(sm[f * fsz + rm * g.pitch + cm]);
                    a[f] = scale(z + zm, T(0.5));
                    const cx<T> d = scale(z - zm, T(0.5));
                    b[f] = mk(d.y, -d.x);  // d / i
                }
                op.combine(0, ky, kz, a, ya);
                op.combine(H, ky, kz, b, yb);
#pragma unroll
                for (int f = 0; f < FO; ++f) out[f] = ya[f] + mul_i(yb[f]);
                // the mirror reads above are from the extra column or from row rm
                // of this column; rows are rewritten only after the barrier below
                // when the column is its own mirror (handled by the pair rule)
                if (cm == g.w) {
#pragma unroll
                    for (int f = 0; f < FO; ++f) sm[f * fsz + r * g.pitch + c] = conjg(out[f]);
                } else {
                    // self-mirrored column: defer writes through registers + barrier
                    // is not possible inside this loop; use the pair rule instead
#pragma unroll
                    for (int f = 0; f < FO; ++f) in[f] = out[f];
                    // store to the extra column slot as scratch (its data is unused
                    // here since cm == c)
#pragma unroll
                    for (int f = 0; f < FO; ++f) sm[f * fsz + r * g.pitch + g.w] = conjg(in[f]);
                }
            } else {
                // 2D: packed column kx = 0, mirror -ky is row (L - r) of this column.
                // Pair (r, L - r) is handled by the thread with r <= L - r.
                const int rm = (L - r) & (L - 1);
                if (r > rm) continue;
                cx<T> z[FB], zm[FB], a[FB], b[FB], ya[FB], yb[FB];
#pragma unroll
                for (int f = 0; f < FI; ++f) {
                    z[f] = sm[f * fsz + r * g.pitch + c];
                    zm[f] = sm[f * fsz + rm * g.pitch + c];
                }
                // mode r
#pragma unroll
                for (int f = 0; f < FI; ++f) {
                    a[f] = scale(z[f] + conjg(zm[f]), T(0.5));
                    const cx<T> d = scale(z[f] - conjg(zm[f]), T(0.5));
                    b[f] = mk(d.y, -d.x);
                }
                op.combine(0, ky, kz, a, ya);
                op.combine(H, ky, kz, b, yb);
#pragma unroll
                for (int f = 0; f < FO; ++f) out[f] = ya[f] + mul_i(yb[f]);
                if (rm != r) {
                    cx<T> out2[FB];
#pragma unroll
                    for (int f = 0; f < FI; ++f) {
                        a[f] = scale(zm[f] + conjg(z[f]), T(0.5));
                        const cx<T> d = scale(zm[f] - conjg(z[f]), T(0.5));
                        b[f] = mk(d.y, -d.x);
                    }
                    op.combine(0, rm, kz, a, ya);
                    op.combine(H, rm, kz, b, yb);
#pragma unroll
                    for (int f = 0; f < FO; ++f) out2[f] = ya[f] + mul_i(yb[f]);
#pragma unroll
                    for (int f = 0; f < FO; ++f) sm[f * fsz + rm * g.pitch + c] = conjg(out2[f]);
                }
#pragma unroll
                for (int f = 0; f < FO; ++f) sm[f * fsz + r * g.pitch + c] = conjg(out[f]);
            }
        }
        __syncthreads();
        if (g.mirror && mcol == c0) {
            // self-mirrored packed column (ky = 0 or n2/2): results were parked in
            // the extra column; move them into place
            for (int r = threadIdx.x; r < L; r += nthreads) {
#pragma unroll
                for (int f = 0; f < FO; ++f) sm[f * fsz + r * g.pitch] = sm[f * fsz + r * g.pitch + g.w];
            }
            __syncthreads();
        }
#pragma unroll
        for (int f = 0; f < FO; ++f) fft_smem<T>(sm + f * fsz + col, g.pitch, g.lgl, jt, tw, g.lgtw);
    }

    // ---- store (conj for inverse transforms)
    constexpr int FS = (MODE == 2) ? FO : FI;
    const bool conj_out = (MODE != 0);
#pragma unroll
    for (int f = 0; f < FS; ++f) {
        cx<T> *dst = op.spec_out(f) + obase;
        const cx<T> *srcs = sm + f * fsz;
        for (int idx = threadIdx.x; idx < L * g.w; idx += nthreads) {
            const int r = idx / g.w, c = idx % g.w;
            const cx<T> v = srcs[r * g.pitch + c];
            dst[(int64_t)r * g.rowstride + c0 + c] = conj_out ? conjg(v) : v;
        }
    }
}

}  // namespace pd
