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
// The in-register DFTs are radix 2/4/8 (radix-2 butterflies with the eighth
// roots of unity as constants); inter-stage data moves through shared memory
// in Stockham autosort order (no bit reversal pass). Each thread owns kV = 8
// complex values per stage; a transform of length L uses L/8 threads.
// Inverse transforms reuse the forward code: IDFT(x) = conj(DFT(conj(x))).
#pragma once

#include <type_traits>

#include "pd_common.cuh"
#include "pd_tma.cuh"

namespace pd {

#ifndef PD_FFT_LGV
#define PD_FFT_LGV 3
#endif
constexpr int kLgV = PD_FFT_LGV;  // log2(kV)
constexpr int kV = 1 << kLgV;     // complex values per thread and FFT stage

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

// Swizzled element order between the first and second stage: element e is
// stored at e ^ ((e >> sh) & 7) (an involution for sh >= 3). The first
// radix-8 stage writes the 8 outputs of one butterfly to consecutive
// elements, so in natural order the lanes of a warp store 8 elements apart
// and pile onto two of the 16 eight-byte bank pairs; XOR-ing the element's
// low three bits with the butterfly index spreads them over all pairs. With
// 8 butterflies per row (rows 8 bank pairs apart) sh = 3 is conflict-free,
// with 16 or more sh = 4. The row kernels compiled for a fixed row length and
// the plane passes use it; in the column tiles the lanes of a warp differ
// first in the column, the conflicts are at most 2-way at the tile widths the
// passes run with, and the extra index arithmetic on the strided addresses
// cost more than it saved (measured), as it did in the row kernels that read
// the length at run time.
__device__ __forceinline__ int swz(int e, int sh) { return e ^ ((e >> sh) & 7); }

// One radix-R Stockham stage of F length-n transforms, field f stored at
// s[f * fstride + e * stride]. Thread jt (of nt = n/kV) handles butterflies
// j = jt + b nt, b < kV/R, of every field (the twiddles are loaded once for
// all fields). tw[i] = e^{-2 pi i i / 2^lgl}. SI / SO: read / write in the
// swizzled order of shift sh. Ends with a block-wide barrier.
template <typename T, int R, int F, bool SI = false, bool SO = false>
__device__ __forceinline__ void fft_stage(cx<T> *s, int fstride, int stride, int n, int ns, int lgnsr, int jt,
                                          int nt, const cx<T> *__restrict__ tw, int lgl, bool cin, bool cout,
                                          int sh = 0)
{
    static_assert(R <= kV, "radix larger than the values per thread");
    constexpr int B = kV / R;
    cx<T> v[F][kV];
    const int q = n / R;
#pragma unroll
    for (int f = 0; f < F; ++f) {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int j = jt + b * nt;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int e = j + r * q;
                if constexpr (SI) e = swz(e, sh);
                const cx<T> x = s[f * fstride + e * stride];
                v[f][b * R + r] = cin ? conjg(x) : x;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = jt + b * nt;
        const int k = j & (ns - 1);
        const int o = (j - k) * R + k;
        if constexpr (F == 1) {
            if (ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[0][b * R + r] = cmul(v[0][b * R + r], tw[(r * k) << (lgl - lgnsr)]);
            }
            dft_reg<T, R>(&v[0][b * R]);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int e = o + r * ns;
                if constexpr (SO) e = swz(e, sh);
                s[e * stride] = cout ? conjg(v[0][b * R + r]) : v[0][b * R + r];
            }
        } else {
            cx<T> w[R];
            if (ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) w[r] = tw[(r * k) << (lgl - lgnsr)];
            }
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if (ns > 1) {
#pragma unroll
                    for (int r = 1; r < R; ++r) v[f][b * R + r] = cmul(v[f][b * R + r], w[r]);
                }
                dft_reg<T, R>(&v[f][b * R]);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    int e = o + r * ns;
                    if constexpr (SO) e = swz(e, sh);
                    s[f * fstride + e * stride] = cout ? conjg(v[f][b * R + r]) : v[f][b * R + r];
                }
            }
        }
    }
    __syncthreads();
}

// Forward DFTs of length 2^lgn (>= 16) of F fields (field f at s + f *
// fstride) in shared memory, in place: stages of radix 8 and one stage of
// radix 4 or 2 for the remainder, which comes last (schedule 0) or first
// (schedule 1). With cin the input is conjugated as it is read, with cout the
// output as it is written (IDFT(x) = conj(DFT(conj(x))) costs no extra pass).
template <typename T, int F = 1>
__device__ __forceinline__ void fft_smem(cx<T> *s, int fstride, int stride, int lgn, int jt,
                                         const cx<T> *__restrict__ tw, int lgl, bool cin = false,
                                         bool cout = false, int sched = 0)
{
    const int n = 1 << lgn, nt = n >> kLgV;
    int ns = 1, lgns = 0, rem = lgn;
    const int rm = lgn % kLgV;
    while (rem > 0) {
        const int lr = (sched && lgns == 0 && rm) ? rm : (rem >= kLgV ? kLgV : rem);
        const bool first = (lgns == 0), last = (rem == lr);
        const bool ci = cin && first, co = cout && last;
        switch (lr) {
            case 4:
                if constexpr (kV >= 16) fft_stage<T, 16, F>(s, fstride, stride, n, ns, lgns + 4, jt, nt, tw, lgl, ci, co);
                break;
            case 3: fft_stage<T, 8, F>(s, fstride, stride, n, ns, lgns + 3, jt, nt, tw, lgl, ci, co); break;
            case 2: fft_stage<T, 4, F>(s, fstride, stride, n, ns, lgns + 2, jt, nt, tw, lgl, ci, co); break;
            default: fft_stage<T, 2, F>(s, fstride, stride, n, ns, lgns + 1, jt, nt, tw, lgl, ci, co); break;
        }
        ns <<= lr;
        lgns += lr;
        rem -= lr;
    }
}

// fft_smem for a length 2^LGN, stage schedule SCHED and swizzle shift SH
// (0: none) fixed at compile time: the stage sequence unrolls, so the lengths,
// strides, twiddle shifts and conjugation flags fft_stage derives from it are
// constants (shared-memory offsets fold into the load and store instructions
// and no stage dispatch runs). Same arithmetic as fft_smem.
template <typename T, int F, int LGN, int SCHED, int SH, int LGNS = 0, bool SWIN = false>
__device__ __forceinline__ void fft_ct(cx<T> *s, int fstride, int stride, int jt, const cx<T> *__restrict__ tw,
                                       int lgl, bool cin, bool cout)
{
    constexpr int REM = LGN - LGNS, RM = LGN % kLgV;
    constexpr int LR = (SCHED && LGNS == 0 && RM) ? RM : (REM >= kLgV ? kLgV : REM);
    constexpr bool FIRST = LGNS == 0, LAST = REM == LR;
    constexpr bool SWOUT = kV == 8 && SH > 0 && FIRST && !LAST && LR == 3;
    fft_stage<T, (1 << LR), F, SWIN, SWOUT>(s, fstride, stride, 1 << LGN, 1 << LGNS, LGNS + LR, jt,
                                            (1 << LGN) >> kLgV, tw, lgl, cin && FIRST, cout && LAST, SH);
    if constexpr (!LAST) fft_ct<T, F, LGN, SCHED, SH, LGNS + LR, SWOUT>(s, fstride, stride, jt, tw, lgl, cin, cout);
}

// Hooks of fft_fields, called with the index of a sweep's first field and
// its field count before and after the sweep (by all threads).
struct NoHook {
    __device__ __forceinline__ void operator()(int, int) const {}
};

// F transforms in sweeps of up to MG fields at a time (one barrier pair per
// stage and sweep instead of per stage and field; MG x 8 complex values live
// per thread). f0 numbers the first field for the hooks.
template <typename T, int F, int MG, class Before = NoHook, class After = NoHook>
__device__ __forceinline__ void fft_fields(cx<T> *s, int fstride, int stride, int lgn, int jt,
                                           const cx<T> *__restrict__ tw, int lgl, bool cin, bool cout, int sched,
                                           int f0 = 0, const Before &before = {}, const After &after = {})
{
    if constexpr (MG == 1) {
        // one field per sweep: a loop (one copy of the transform code)
#pragma unroll 1
        for (int f = 0; f < F; ++f) {
            before(f0 + f, 1);
            fft_smem<T, 1>(s + f * fstride, fstride, stride, lgn, jt, tw, lgl, cin, cout, sched);
            after(f0 + f, 1);
        }
    } else if constexpr (F > 0) {
        constexpr int G = F < MG ? F : MG;
        before(f0, G);
        fft_smem<T, G>(s, fstride, stride, lgn, jt, tw, lgl, cin, cout, sched);
        after(f0, G);
        if constexpr (F > G)
            fft_fields<T, F - G, MG>(s + G * fstride, fstride, stride, lgn, jt, tw, lgl, cin, cout, sched, f0 + G,
                                     before, after);
    }
}
// column passes: grouped sweeps pay for the spectral-combine passes; the plain
// transforms keep one field per sweep (fewer registers, more resident warps)
constexpr int kCombFieldGroup = kV == 8 ? 3 : 1;

// ---------------------------------------------------------------------------
// Compensated FP32 accumulation (Knuth two-sum): sums carried as an
// unevaluated pair (hi, lo), accurate to about FP32^2, so reductions run on
// FP32 units and only the block totals are combined in FP64. Inner products
// take each FP32 product exactly (the FMA residual a b - fl(a b) is itself a
// float, the error-free two-product), so a dot product of FP32 vectors is
// accumulated to about FP64 accuracy without FP64 arithmetic per element.
// ---------------------------------------------------------------------------
struct DSum {
    float hi = 0.f, lo = 0.f;
    double d = 0.0;  // FP64 operands accumulate here directly
    __device__ __forceinline__ void add(float x)
    {
        const float s = hi + x;
        const float bb = s - hi;
        lo += (hi - (s - bb)) + (x - bb);
        hi = s;
    }
    __device__ __forceinline__ void add(double x) { d += x; }
    // += a b with the product's rounding error kept
    __device__ __forceinline__ void add_prod(float a, float b)
    {
        const float p = a * b;
        lo += __fmaf_rn(a, b, -p);
        add(p);
    }
    __device__ __forceinline__ void add_prod(double a, double b) { d += a * b; }
    __device__ __forceinline__ double value() const { return d + (double)hi + (double)lo; }
};

// Sum of one double per thread over the block (all threads must call).
__device__ __forceinline__ double block_sum_d(double v)
{
    __shared__ double sh_bs[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh_bs[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? sh_bs[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;  // valid in thread 0
}

// Block sums of NV compensated accumulators (valid in thread 0; whole warps).
// The FP32 pairs (hi, lo) are merged across each warp by the two-sum of the
// hi parts, their rounding errors going to lo, so only one lane per warp
// converts to FP64: FP64 runs at a small fraction of the FP32 rate, and a
// per-thread FP64 reduction kept that pipe busy for several microseconds of
// every row pass. FP64 parts are summed in FP64 only in warps that hold any.
template <int NV>
__device__ __forceinline__ void block_sums(const DSum *const (&a)[NV], double (&out)[NV])
{
    __shared__ double sh_bn[NV][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();  // a previous call may still be reading sh_bn
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        float hi = a[v]->hi, lo = a[v]->lo;
        double d = a[v]->d;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            const float s = hi + h2, bb = s - hi;
            lo += l2 + ((hi - (s - bb)) + (h2 - bb));
            hi = s;
        }
        if (__any_sync(0xffffffffu, d != 0.0))
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) sh_bn[v][wid] = d + (double)hi + (double)lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double t = 0.0;
            for (int k = 0; k < nw; ++k) t += sh_bn[v][k];
            out[v] = t;
        }
    }
}

// ---------------------------------------------------------------------------
// Row pass
// ---------------------------------------------------------------------------

struct RowGeom {
    int lgh;        // log2(n1/2): complex length of a packed row
    int rows;       // rows per tile
    int pitch;      // shared-memory pitch of a packed row (complex elements, even)
    int64_t nrows;  // n2 * n3 (multiple of rows)
    int lgl;        // log2 of the global twiddle table length
    int sched;      // FFT stage schedule (fft_smem)
    int nstage;     // 2: the next tile's copies overlap this tile's work; 1: no overlap
    int *err;       // device status word (bounded-wait time-outs)
    int *inject;    // failure-handling test hook (device word or null): when it
                    // holds 1 + this pass's kind (0 forward, 3 inverse), block 0
                    // clears it and issues no copies, so its bounded wait runs out
};

// Bytes of one pipeline stage of a row tile: SB packed-row slots loaded by
// the stage (the inverse passes' spectra; 0 for forward passes), NF node
// fields of T and NB byte fields, rounded up to 128 bytes.
template <typename T>
__host__ __device__ constexpr size_t row_stage_bytes(int SB, int NF, int NB, int rows, int pitch, int n1)
{
    return ((size_t)SB * rows * pitch * sizeof(cx<T>) + (size_t)NF * rows * n1 * sizeof(T) +
            (((size_t)NB * rows * n1 + 15) & ~(size_t)15) + 127) & ~(size_t)127;
}

// Shared memory of a row pass: twiddles, a single transform workspace for
// forward passes (FI = 0), and nstage pipeline stages.
template <typename T>
__host__ __device__ constexpr size_t row_smem_bytes(int FI, int FB, int NF, int NB, int rows, int pitch, int n1,
                                                    int nstage)
{
    return (((size_t)n1 * sizeof(cx<T>) + 127) & ~(size_t)127) +
           (FI > 0 ? 0 : (((size_t)FB * rows * pitch * sizeof(cx<T>) + 127) & ~(size_t)127)) +
           (size_t)nstage * row_stage_bytes<T>(FI > 0 ? FB : 0, NF, NB, rows, pitch, n1) + 16;
}

// Shared-memory views handed to the row ops.
template <typename T>
struct RowCtx {
    int64_t row0;
    int rows, n1, pitch;
    cx<T> *spec;        // [slots][rows][pitch] packed rows (staged outputs after the epilogue)
    const T *nf;        // [kNF][rows][n1] preloaded node fields
    const uint8_t *nb;  // [kNB][rows][n1] preloaded byte fields
    __device__ __forceinline__ T f(int k, int rl, int i1) const { return nf[((size_t)k * rows + rl) * n1 + i1]; }
    __device__ __forceinline__ uint8_t b(int k, int rl, int i1) const
    {
        return nb[((size_t)k * rows + rl) * n1 + i1];
    }
    // staged value of field q at node (rl, i1): one half of packed slot i1/2
    __device__ __forceinline__ T &stage(int q, int rl, int i1) const
    {
        cx<T> &c = spec[(q * rows + rl) * pitch + (i1 >> 1)];
        return (i1 & 1) ? c.y : c.x;
    }
};

// Block accumulator of a row op: Op::Acc when the op declares one, else DSum.
template <class Op, class = void>
struct op_acc {
    using type = DSum;
};
template <class Op>
struct op_acc<Op, std::void_t<typename Op::Acc>> {
    using type = typename Op::Acc;
};

// Row ops whose node2 also accumulates into the block accumulator declare
// kNodeAcc = true and take the accumulator as a last argument.
template <class Op, class = void>
struct op_node_acc : std::false_type {
};
template <class Op>
struct op_node_acc<Op, std::void_t<decltype(Op::kNodeAcc)>> : std::bool_constant<Op::kNodeAcc> {
};

// Op interface (all device unless noted):
//   static constexpr int kFin, kFout;  packed spectra read (inverse) / written (forward)
//   static constexpr int kNF, kNB;     node fields (T / uint8) bulk-loaded for the tile's rows
//   static constexpr int kStage;       outputs staged in shared memory and written by emit()
//   static constexpr bool kSparse;     sparse() runs between node2() and emit()
//   const cx<T>* spec_in(int f); cx<T>* spec_out(int f);   row-major [row][n1/2]
//   const T* nf_src(int k); const uint8_t* nb_src(int k);  row-major [row][n1]
//   void node2(ctx, rl, i1, in0, in1, o0, o1): nodes i1 and i1+1 of tile row rl;
//        in: kFin inverse-transformed values (unnormalised IDFT);
//        o:  max(kFout, kStage) outputs (forward inputs or staged values)
//   void sparse(ctx, tid, nthreads); void emit(ctx, rl, i1, s0, s1, acc)
//   void block_done(acc): called by every thread at the end (block reductions);
//        acc is an Op::Acc if the op declares that type, else a DSum
// Data movement: the kernel is persistent; each block walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... One thread issues the bulk async
// copies (cp.async.bulk) of a tile's spectrum rows and node fields into one of
// two shared-memory stages, completing on that stage's mbarrier: the copies of
// the next tile are in flight while the current one is transformed. Twiddles
// are copied to shared memory once; outputs leave through coalesced stores.
// Block accumulators (acc) run over all tiles of the block.
// Row ops may declare l2_prefetch(row0, rows): called by the thread that
// issues a tile's bulk copies, right after them, to start the node fields the
// op reads with plain loads later (after the tile's transforms) towards L2.
template <class Op, class = void>
struct op_has_l2_prefetch : std::false_type {
};
template <class Op>
struct op_has_l2_prefetch<Op, std::void_t<decltype(&Op::l2_prefetch)>> : std::true_type {
};

// Row ops may declare kMinBlocks (resident 256-thread blocks per SM the
// compiler must allow, i.e. a register cap of 256 / kMinBlocks per thread).
template <class Op, class = void>
struct op_min_blocks : std::integral_constant<int, 1> {
};
template <class Op>
struct op_min_blocks<Op, std::void_t<decltype(Op::kMinBlocks)>> : std::integral_constant<int, Op::kMinBlocks> {
};
// LG > 0: compiled for packed rows of 2^LG complex values (g.lgh == LG) and
// stage schedule SCHED (g.sched == SCHED); LG = 0 reads both from g.
template <typename T, class Op, int LG = 0, int SCHED = 0>
__global__ void __launch_bounds__(256, op_min_blocks<Op>::value) k_rows(RowGeom g, Op op,
                                                                       const cx<T> *__restrict__ tw)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int FI = Op::kFin, FO = Op::kFout, NF = Op::kNF, NB = Op::kNB, ST = Op::kStage;
    constexpr int KO = FO > ST ? FO : ST;
    constexpr int FB = FI > KO ? FI : KO;
    static_assert(!(FO > 0 && ST > 0), "an op either stages outputs or transforms forward");
    constexpr bool kLoad = FI > 0 || NF > 0 || NB > 0;
    const int lgh = LG > 0 ? LG : g.lgh;
    const int H = 1 << lgh, n1 = 2 * H, nt = H >> kLgV, lg1 = lgh + 1;
    const int rows = g.rows, pitch = g.pitch;
    const int64_t ntiles = g.nrows / rows;
    // forward passes (FI = 0) load no spectra: one transform workspace, and
    // the stages hold only the node fields
    constexpr int SB = FI > 0 ? FB : 0;
    const size_t sbytes = row_stage_bytes<T>(SB, NF, NB, rows, pitch, n1);
    cx<T> *tws = reinterpret_cast<cx<T> *>(smem_raw);
    unsigned char *after_tw = smem_raw + (((size_t)n1 * sizeof(cx<T>) + 127) & ~(size_t)127);
    cx<T> *work = reinterpret_cast<cx<T> *>(after_tw);
    unsigned char *stage0 =
        after_tw + (FI > 0 ? 0 : (((size_t)FB * rows * pitch * sizeof(cx<T>) + 127) & ~(size_t)127));
    const int ns = g.nstage;
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(stage0 + ns * sbytes);
    auto stage_spec = [&](int s) {
        return FI > 0 ? reinterpret_cast<cx<T> *>(stage0 + s * sbytes) : work;
    };
    auto stage_nf = [&](int s) { return reinterpret_cast<T *>(stage0 + s * sbytes + SB * rows * pitch * sizeof(cx<T>)); };
    auto stage_nb = [&](int s) { return reinterpret_cast<uint8_t *>(stage_nf(s) + NF * rows * n1); };

    // one thread: bulk copies of tile `tile` into stage s
    auto issue = [&](int64_t tile, int s) {
        const int64_t r0 = tile * rows;
        cx<T> *spec = stage_spec(s);
        T *nf = stage_nf(s);
        uint8_t *nb = stage_nb(s);
        const unsigned bytes = (unsigned)(FI * rows * H * sizeof(cx<T>) + NF * rows * n1 * sizeof(T) + NB * rows * n1);
        mbar_expect_tx(&mbar[s], bytes);
#pragma unroll
        for (int f = 0; f < FI; ++f)
            for (int r = 0; r < rows; ++r)
                bulk_load(spec + (f * rows + r) * pitch, op.spec_in(f) + (r0 + r) * H, H * sizeof(cx<T>), &mbar[s]);
#pragma unroll
        for (int k = 0; k < NF; ++k)
            bulk_load(nf + k * rows * n1, op.nf_src(k) + r0 * n1, rows * n1 * sizeof(T), &mbar[s]);
#pragma unroll
        for (int k = 0; k < NB; ++k) bulk_load(nb + k * rows * n1, op.nb_src(k) + r0 * n1, rows * n1, &mbar[s]);
        if constexpr (op_has_l2_prefetch<Op>::value) op.l2_prefetch(r0, rows);
    };

    if (kLoad && threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        if (ns == 2) mbar_init(&mbar[1], 1);
    }
    for (int i = threadIdx.x; i < n1; i += blockDim.x) tws[i] = tw[i << (g.lgl - lg1)];
    __syncthreads();
    // everything above reads plan constants only; the op's fields come from
    // the preceding pass
    pdl_wait();
    pdl_trigger();
    int64_t t = blockIdx.x;
    // test hook: one-shot, so a pass captured in a graph stalls on one replay only
    bool stall = false;
    if (kLoad && g.inject && blockIdx.x == 0 && threadIdx.x == 0) {
        const int kind = FI > 0 ? 3 : 0;
        stall = atomicCAS(g.inject, kind + 1, 0) == kind + 1;
    }
    if (kLoad && threadIdx.x == 0 && t < ntiles && !stall) issue(t, 0);
    unsigned phase = 0;  // bit s: parity of the next completion of stage s
    const int jt = threadIdx.x % nt, rf = threadIdx.x / nt;  // FFT mapping: nt threads per row
    // the kernels compiled for a row length exchange the first stage's outputs
    // in swizzled order (constant index arithmetic); with the run-time length
    // the extra index arithmetic cost more than the bank conflicts it removes
    // (2D rows of 256 to 1024 nodes: relaxation steps 26% slower)
    auto row_fft = [&](cx<T> *z) {
        if constexpr (LG > 0)
            fft_ct<T, 1, LG, SCHED, (LG - kLgV >= 4 ? 4 : 3)>(z, 0, 1, jt, tws, LG + 1, false, false);
        else
            fft_smem<T>(z, 0, 1, g.lgh, jt, tws, lg1, false, false, g.sched);
    };
    typename op_acc<Op>::type acc;

    for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
        const int s = ns == 2 ? (it & 1) : 0;
        const int64_t tn = t + gridDim.x;
        const bool pre = kLoad && ns == 2 && tn < ntiles && !stall;
        if (pre && threadIdx.x == 0) issue(tn, s ^ 1);
        if (kLoad && ns == 1 && it > 0 && threadIdx.x == 0 && !stall) issue(t, 0);
        if constexpr (kLoad) {
            const bool ok = mbar_wait(&mbar[s], (phase >> s) & 1u, g.err);
            phase ^= 1u << s;
            if (__syncthreads_or(!ok)) {
                // give up: let the prefetch in flight land before the block exits
                if (threadIdx.x == 0 && pre) mbar_wait(&mbar[s ^ 1], (phase >> (s ^ 1)) & 1u, g.err);
                __syncthreads();
                return;
            }
        }
        const int64_t row0 = t * rows;
        cx<T> *spec = stage_spec(s);
        const RowCtx<T> ctx{row0, rows, n1, pitch, spec, stage_nf(s), stage_nb(s)};

        if constexpr (FI > 0) {
            // Unpack the half spectrum into Z(k) = E(k) + i O(k) (E, O: DFTs of the
            // even / odd samples, times 2) and store conj(Z) for the inverse.
#pragma unroll
            for (int f = 0; f < FI; ++f) {
                cx<T> *z = spec + (f * rows + rf) * pitch;
                for (int k = jt; k <= H / 2; k += nt) {
                    if (k == 0) {
                        const cx<T> p = z[0];  // (X(0), X(n1/2))
                        z[0] = conjg(mk(p.x + p.y, p.x - p.y));
                    } else {
                        const int kk = H - k;
                        const cx<T> a = z[k], b = z[kk];
                        const cx<T> w = tws[k];  // W^k, W = e^{-2 pi i / n1}
                        // Z(k)  = (a + conj b) + i conj(W^k) (a - conj b)
                        const cx<T> zk = (a + conjg(b)) + mul_i(cmul(conjg(w), a - conjg(b)));
                        if (kk != k) {
                            // Z(H-k) = (b + conj a) - i W^k (b - conj a)
                            const cx<T> zkk = (b + conjg(a)) - mul_i(cmul(w, b - conjg(a)));
                            z[kk] = conjg(zkk);
                        }
                        z[k] = conjg(zk);
                    }
                }
            }
            __syncthreads();
#pragma unroll 1
            for (int f = 0; f < FI; ++f)
                row_fft(spec + (f * rows + rf) * pitch);
        }

        // per-node work, lanes over consecutive packed slots (2 nodes each)
        for (int idx = threadIdx.x; idx < rows * H; idx += blockDim.x) {
            const int rl = idx >> lgh, n = idx & (H - 1);
            T in0[FI > 0 ? FI : 1], in1[FI > 0 ? FI : 1];
            T o0[KO > 0 ? KO : 1], o1[KO > 0 ? KO : 1];
#pragma unroll
            for (int f = 0; f < FI; ++f) {
                const cx<T> w = spec[(f * rows + rl) * pitch + n];  // x[2n] = Re w, x[2n+1] = -Im w
                in0[f] = w.x;
                in1[f] = -w.y;
            }
            if constexpr (op_node_acc<Op>::value)
                op.node2(ctx, rl, 2 * n, in0, in1, o0, o1, acc);
            else
                op.node2(ctx, rl, 2 * n, in0, in1, o0, o1);
#pragma unroll
            for (int f = 0; f < KO; ++f) spec[(f * rows + rl) * pitch + n] = mk(o0[f], o1[f]);
        }
        __syncthreads();

        if constexpr (Op::kSparse) {
            op.sparse(ctx, threadIdx.x, blockDim.x);
            __syncthreads();
        }
        if constexpr (ST > 0) {
            for (int idx = threadIdx.x; idx < rows * H; idx += blockDim.x) {
                const int rl = idx >> lgh, n = idx & (H - 1);
                T s0[ST], s1[ST];
#pragma unroll
                for (int f = 0; f < ST; ++f) {
                    const cx<T> v = spec[(f * rows + rl) * pitch + n];
                    s0[f] = v.x;
                    s1[f] = v.y;
                }
                op.emit(ctx, rl, 2 * n, s0, s1, acc);
            }
        }

        if constexpr (FO > 0) {
#pragma unroll 1
            for (int f = 0; f < FO; ++f)
                row_fft(spec + (f * rows + rf) * pitch);
            const T half = T(0.5);
#pragma unroll
            for (int f = 0; f < FO; ++f) {
                const cx<T> *z = spec + (f * rows + rf) * pitch;
                cx<T> *dst = op.spec_out(f) + (row0 + rf) * H;
                for (int k = jt; k <= H / 2; k += nt) {
                    if (k == 0) {
                        const cx<T> z0 = z[0];
                        dst[0] = mk(z0.x + z0.y, z0.x - z0.y);
                    } else {
                        const int kk = H - k;
                        const cx<T> a = z[k], b = z[kk];
                        const cx<T> w = tws[k];
                        // X(k) = 1/2 [(a + conj b) - i W^k (a - conj b)]
                        dst[k] = scale((a + conjg(b)) - mul_i(cmul(w, a - conjg(b))), half);
                        // X(H-k) = 1/2 [(b + conj a) + i conj(W^k) (b - conj a)]
                        if (kk != k) dst[kk] = scale((b + conjg(a)) + mul_i(cmul(conjg(w), b - conjg(a))), half);
                    }
                }
            }
        }
        // the stage is rewritten by the async proxy two tiles on
        fence_proxy_async();
        __syncthreads();
    }
    op.block_done(acc);
}

// ---------------------------------------------------------------------------
// Column pass (TMA)
// ---------------------------------------------------------------------------

struct ColGeom {
    int lgl;     // log2 of the transform length L (axis length)
    int w;       // tile width (columns, power of two, divides the inner extent)
    int lgw;     // log2(w)
    int mirror;  // 1: 3D last-axis pass, also loads the mirror of column kx = 0
    int lgh;     // log2(n1/2) (packed row length), for mode coordinates
    int n2;      // n2 (3D mirror of k2)
    int lgtw;    // log2 of the twiddle table length
    int lb;      // rows per TMA box (<= 256, divides L)
    int outer;   // outer extent: n3 for the x2 pass, 1 for the last axis
    int sched;   // FFT stage schedule (fft_smem)
    int tmode;   // tiles: 0 all (c0 = block w), 1 3D last axis without the kx = 0
                 // tiles, 2 3D last axis, only the kx = 0 tiles (with mirror)
    int *err;    // device status word (bounded-wait time-outs)
};

// Op interface:
//   static constexpr int kFin, kFout, kMode, kPre; static constexpr bool kStoreIn;
//   kMode 0: forward FFT only, 1: inverse FFT only,
//         2: forward FFT, combine, inverse FFT (kFout <= kFin)
//   kPre: (kMode 2) leading inputs already transformed along this axis
//   kStoreIn: (kMode 2) store the transformed inputs to slot_aux(f) first
//   int slot_in(int f), slot_out(int f), slot_aux(int f): packed-spectrum slots
//   static constexpr int kTab; const T* table(int c): kTab folded kernel-spectrum
//        components (layout [k3f][k2f][k1], k1 in [0, n1/2]); the tile's slice is
//        prefetched into shared memory while the TMA loads are in flight
//   void combine(const T* t, int cs, bool fy, bool fz, const cx<T>* in, cx<T>* out);
//        (kMode 2; called for true modes with kx in [0, n1/2], so both the
//         kx = 0 and kx = n1/2 halves of the packed column are visited; t points
//         at component 0 of the mode in the slice, cs is the component stride,
//         fy / fz say that k2 / k3 were folded to n - k)
// Tensor maps: tmt covers all slots of the spectrum buffer as
// [outer * slots][L][2 * inner] scalars with box (2w, lb, 1); tmm the same with
// box (4, lb, 1) for the mirror column.
// Shared memory: [L] twiddles, [max(kFin,kFout)][L][w] tiles, [max(kFin,kFout)][L][2] mirror,
// the table slice, mbarriers (one per field for the plain transforms, else one).
template <typename T, class Op>
__global__ void __launch_bounds__(512) k_cols(ColGeom g, Op op, const cx<T> *__restrict__ tw, int axis_is_z,
                                              const __grid_constant__ CUtensorMap tmt,
                                              const __grid_constant__ CUtensorMap tmm)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int FI = Op::kFin, FO = Op::kFout, MODE = Op::kMode;
    constexpr int FB = FI > FO ? FI : FO;
    // the combine reads all inputs of a mode before it writes that mode's
    // outputs, so outputs may outnumber inputs (the tile holds max(kFin, kFout))
    const int lgl = g.lgl;
    const int L = 1 << lgl;
    const int w = g.w, ncol = w + g.mirror;  // threads: ncol x (L / kV)
    const int col = threadIdx.x % ncol, jt = threadIdx.x / ncol;
    const int H = 1 << g.lgh;
    int c0;
    if (g.tmode == 1) {
        const int per = (H >> g.lgw) - 1;  // tiles of a k2 row after its kx = 0 tile
        c0 = ((int)blockIdx.x / per) * H + w * (1 + (int)blockIdx.x % per);
    } else {
        c0 = g.tmode == 2 ? (int)blockIdx.x * H : (int)blockIdx.x * w;
    }
    const int o = blockIdx.y;
    const int nthreads = blockDim.x;
    const int fsz = L * w;
    cx<T> *tws = reinterpret_cast<cx<T> *>(smem_raw);  // W_L^i, i < L
    cx<T> *tile = tws + L;
    cx<T> *mir = tile + FB * fsz;
    constexpr int NTAB = (MODE == 2) ? Op::kTab : 0;
    // table slice [comp][fold row][kx]; the kx = n1/2 column only where the tile holds kx = 0
    const int trows = L / 2 + 1, tcols = w + (g.tmode == 1 ? 0 : 1), tcs = trows * tcols;
    T *tab = reinterpret_cast<T *>(mir + (g.mirror ? FB * L * 2 : 0));  // mirror: inputs in, parked outputs out
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(tab + ((NTAB * tcs + 1) & ~1));

    // mirror column (3D last axis): kx = 0 of k2' = (n2 - k2) mod n2
    int mcol = -1;
    if (g.mirror && (c0 & (H - 1)) == 0) mcol = ((g.n2 - (c0 >> g.lgh)) & (g.n2 - 1)) << g.lgh;

    // every field has its own barrier: a sweep of fields is transformed as
    // soon as they have arrived while the later ones are still in flight,
    // and outputs leave sweep by sweep while the next sweep is transformed
    if (threadIdx.x == 0) {
#pragma unroll
        for (int f = 0; f < FI; ++f) mbar_init(&mbar[f], 1);
    }
    for (int i = threadIdx.x; i < L; i += nthreads) tws[i] = tw[i << (g.lgtw - lgl)];
    __syncthreads();
    // kernel-table slice of this tile (plan constants: fetched before the wait
    // for the preceding pass, overlapping its tail)
    const int kx0 = axis_is_z ? (c0 & (H - 1)) : c0;
    const int kyt = c0 >> g.lgh;  // 3D: the tile's k2
    const bool fyt = axis_is_z && kyt > (g.n2 >> 1);
    if constexpr (NTAB > 0) {
        // flat loop over the slice; the (component, fold row, column) split
        // uses FP32 reciprocals, exact here (indices < 2^15, divisors <= 2^10 + 1)
        const int kyf = fyt ? g.n2 - kyt : kyt;
        const int64_t rstride = axis_is_z ? (int64_t)((g.n2 >> 1) + 1) * (H + 1) : (int64_t)(H + 1);
        const int64_t roff = axis_is_z ? (int64_t)kyf * (H + 1) : 0;
        const float inv_tcs = 1.0f / (float)tcs, inv_tcols = 1.0f / (float)tcols;
#pragma unroll 8
        for (int i = threadIdx.x; i < NTAB * tcs; i += nthreads) {
            const int comp = (int)(((float)i + 0.5f) * inv_tcs);
            const int rem = i - comp * tcs;
            const int rr = (int)(((float)rem + 0.5f) * inv_tcols);
            const int cc = rem - rr * tcols;
            tab[i] = op.table(comp)[rr * rstride + roff + ((cc == w) ? H : kx0 + cc)];
        }
    }
    pdl_trigger();
    if (threadIdx.x == 0) {
        pdl_wait();  // the tiles are the preceding pass's output; only thread 0 touches global data
        const unsigned fbytes = (unsigned)(fsz * sizeof(cx<T>) + (mcol >= 0 ? L * 2 * sizeof(cx<T>) : 0));
#pragma unroll
        for (int f = 0; f < FI; ++f) {
            mbar_expect_tx(&mbar[f], fbytes);
            const int z = o + op.slot_in(f) * g.outer;
            for (int l0 = 0; l0 < L; l0 += g.lb) {
                tma_load_3d(tile + f * fsz + l0 * w, &tmt, 2 * c0, l0, z, &mbar[f]);
                if (mcol >= 0) tma_load_3d(mir + f * L * 2 + l0 * 2, &tmm, 2 * mcol, l0, z, &mbar[f]);
            }
        }
    }

    // per-thread transform: a tile column, or the mirror column
    const bool is_m = col >= w;
    const int cstride = is_m ? 2 : w;
    auto colbase = [&](int f) -> cx<T> * { return is_m ? (mir + f * L * 2) : (tile + f * fsz + col); };
    const int fstr = is_m ? L * 2 : fsz;  // field stride of this thread's column

    constexpr int FPRE = (MODE == 2) ? Op::kPre : 0;
    constexpr int GF = MODE == 2 ? kCombFieldGroup : 1;  // fields per sweep
    // A bounded wait that runs out marks the block failed (all threads agree):
    // it stores nothing, and before it exits it lets the copies in flight land.
    bool failed = false;
    int narrived = 0;  // fields waited for
    auto arrive = [&](int f0, int n) {
        const int upto = f0 + n;
        bool ok = true;
        if (!failed)
            for (int f = narrived; f < upto; ++f) ok = ok && mbar_wait(&mbar[f], 0, g.err);
        narrived = upto;
        failed = __syncthreads_or(failed || !ok);
    };
    auto emit = [&](int f0, int n) {  // store output fields [f0, f0 + n)
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0 && !failed) {
            for (int f = f0; f < f0 + n; ++f)
                for (int l0 = 0; l0 < L; l0 += g.lb)
                    tma_store_3d(&tmt, 2 * c0, l0, o + op.slot_out(f) * g.outer, tile + f * fsz + l0 * w);
            bulk_commit();
        }
    };

    if constexpr (MODE != 2) {
        fft_fields<T, FI, 1>(colbase(0), fstr, cstride, lgl, jt, tws, lgl, MODE == 1, MODE == 1, g.sched, 0, arrive,
                             emit);
    } else {
        if constexpr (FI == FPRE) arrive(0, FI);
        fft_fields<T, FI - FPRE, GF>(colbase(FPRE), fstr, cstride, lgl, jt, tws, lgl, false, false, g.sched, FPRE,
                                     arrive);
    }

    if constexpr (MODE == 2 && Op::kStoreIn) {
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0 && !failed) {
#pragma unroll
            for (int f = FPRE; f < FI; ++f)
                for (int l0 = 0; l0 < L; l0 += g.lb)
                    tma_store_3d(&tmt, 2 * c0, l0, o + op.slot_aux(f) * g.outer, tile + f * fsz + l0 * w);
            bulk_commit();
            bulk_wait_read_all();
        }
        __syncthreads();
    }

    if constexpr (MODE == 2) {
        // ---- spectral combine; writes conj(output) for the inverse
        const bool self_m = (mcol == c0);  // k2 is its own mirror: results parked in mir
        const int half = L >> 1;
        // table position of mode (row r, column c) and of the kx = n1/2 half
        auto tpos = [&](int r, int kxl) { return (r <= half ? r : L - r) * tcols + kxl; };
        for (int idx = threadIdx.x; idx < L * w; idx += nthreads) {
            const int r = idx >> g.lgw, c = idx & (w - 1);
            const int kx = kx0 + c;
            const bool fr = r > half;  // the row's wave number was folded
            const bool fy = axis_is_z ? fyt : fr, fz = axis_is_z && fr;
            cx<T> in[FB], out[FB];
            if (kx != 0) {
#pragma unroll
                for (int f = 0; f < FI; ++f) in[f] = tile[f * fsz + r * w + c];
                op.combine(tab + tpos(r, c), tcs, fy, fz, in, out);
#pragma unroll
                for (int f = 0; f < FO; ++f) tile[f * fsz + r * w + c] = conjg(out[f]);
            } else if (axis_is_z) {
                // packed column: mirror (-ky, -kz) is row (L - r) of the mirror
                // column, or of this column when ky is its own mirror
                const int rm = (L - r) & (L - 1);
                cx<T> a[FB], b[FB], ya[FB], yb[FB];
#pragma unroll
                for (int f = 0; f < FI; ++f) {
                    const cx<T> z = tile[f * fsz + r * w + c];
                    const cx<T> zm = conjg(self_m ? tile[f * fsz + rm * w + c] : mir[f * L * 2 + rm * 2]);
                    a[f] = scale(z + zm, T(0.5));
                    const cx<T> d = scale(z - zm, T(0.5));
                    b[f] = mk(d.y, -d.x);  // d / i
                }
                op.combine(tab + tpos(r, c), tcs, fy, fz, a, ya);
                op.combine(tab + tpos(r, w), tcs, fy, fz, b, yb);
#pragma unroll
                for (int f = 0; f < FO; ++f) {
                    const cx<T> y = conjg(ya[f] + mul_i(yb[f]));
                    if (self_m)
                        mir[f * L * 2 + r * 2] = y;
                    else
                        tile[f * fsz + r * w + c] = y;
                }
            } else {
                // 2D: packed column kx = 0, mirror -ky is row (L - r) of this
                // column. Pair (r, L - r) is handled by the thread with r <= L - r.
                const int rm = (L - r) & (L - 1);
                if (r > rm) continue;
                cx<T> z[FB], zm[FB], a[FB], b[FB], ya[FB], yb[FB];
#pragma unroll
                for (int f = 0; f < FI; ++f) {
                    z[f] = tile[f * fsz + r * w + c];
                    zm[f] = tile[f * fsz + rm * w + c];
                }
#pragma unroll
                for (int f = 0; f < FI; ++f) {
                    a[f] = scale(z[f] + conjg(zm[f]), T(0.5));
                    const cx<T> d = scale(z[f] - conjg(zm[f]), T(0.5));
                    b[f] = mk(d.y, -d.x);
                }
                op.combine(tab + tpos(r, c), tcs, fy, fz, a, ya);
                op.combine(tab + tpos(r, w), tcs, fy, fz, b, yb);
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
                    const bool frm = rm > half;
                    op.combine(tab + tpos(rm, c), tcs, frm, false, a, ya);
                    op.combine(tab + tpos(rm, w), tcs, frm, false, b, yb);
#pragma unroll
                    for (int f = 0; f < FO; ++f) out2[f] = ya[f] + mul_i(yb[f]);
#pragma unroll
                    for (int f = 0; f < FO; ++f) tile[f * fsz + rm * w + c] = conjg(out2[f]);
                }
#pragma unroll
                for (int f = 0; f < FO; ++f) tile[f * fsz + r * w + c] = conjg(out[f]);
            }
        }
        __syncthreads();
        if (self_m) {
            for (int r = threadIdx.x; r < L; r += nthreads) {
#pragma unroll
                for (int f = 0; f < FO; ++f) tile[f * fsz + r * w] = mir[f * L * 2 + r * 2];
            }
            __syncthreads();
        }
        fft_fields<T, FO, GF>(colbase(0), fstr, cstride, lgl, jt, tws, lgl, false, true, g.sched, 0, NoHook{}, emit);
    }

    if (threadIdx.x == 0) {
        if (failed)
            for (int f = 0; f < FI; ++f) mbar_wait(&mbar[f], 0, nullptr);
        bulk_wait_read_all();
    }
}

}  // namespace pd
