// pd_solve_static: FCBM-EC elastostatics (Eq. 85-89) by conjugate gradient (§4.3).
//
// The residual of Eq. 89, R(u) = chi_O (L(u) + b), with u = w on Gamma, is zero
// at the solution. Writing u = u0 + e with e = 0 off Omega, the correction
// solves A e = R(u0) with A e = -chi_O L(chi_O e): A is symmetric and positive
// definite on Omega (the bond sum of Eq. 17-18 / 36 with the chi_B cut is a
// weighted graph Laplacian once the constraint removes the rigid motions).
//
// Precision: on an FP32 plan the CG runs on FP32 FFT convolutions inside an
// iterative refinement whose residual R(u) is recomputed with the FP64
// convolution path on the FP64 iterate u; the outer loop stops when
// ||R(u)||_2 <= rtol ||chi_O b||_2 (both in FP64). On an FP64 plan the same code
// runs in FP64. CG inner products are accumulated per thread in compensated
// FP32 (two-sum) and per block in FP64.
//
// One CG iteration is five fused passes and one small kernel (three passes
// and the small kernel on cubes of up to 128^3 in FP32, where the plane passes
// of pd_plane.cuh fuse the x1 and x2 transforms); the vector
// updates of iteration i are applied in the first pass of iteration i+1, so
// all reductions of an iteration happen in one place (r.q and q.q give the
// next r.r before r is updated: (r - alpha q).(r - alpha q) = rr - 2 alpha rq
// + alpha^2 qq; the true r.r is summed again by the next first pass):
//   rows  : e += alpha p, r -= alpha q, p = r + beta p (stored), partials of
//           r.r, FFT_x1 of chi p
//   cols / last / cols : FFT_x2, M^ multiply with FFT_x3, inverse (3D)
//   rows  : inverse FFT_x1, q = -chi_O L(p) (stored), partials of p.q, r.q, q.q
//   finish: rr, alpha = rr / p.q, beta = (rr - 2 alpha rq + alpha^2 qq) / rr
// After the last iteration one update kernel applies the pending e, r update.
// All CG scalars stay on the device. Chunks of kChunk iterations are captured
// once into a CUDA graph and replayed; the host reads the residual norm after
// each chunk.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pd_force_impl.cuh"
#include "pd_solver_common.cuh"

namespace pd {
namespace {

constexpr int kChunk = 16;       // CG iterations per graph replay
constexpr int kPartB = 14400;    // fused iteration: r.r partials below, (p.q, r.q, q.q) triples above
}  // namespace
}  // namespace pd

#include "pd_plane.cuh"

namespace pd {
namespace {

constexpr int kHostStatus = 32;  // slot of the pinned host scalars that receives the device status word

// rr = sum of the first pass's partials; alpha, beta from the second pass's triples
// rr = sum of the first pass's partials; alpha, beta from the second pass's
// triples (one block of kFinishThreads)
__global__ void __launch_bounds__(kFinishThreads) k_cg_finish_fused(double *red, int na, int nb)
{
    pdl_wait();
    pdl_trigger();
    double rr = 0.0, pq = 0.0, rq = 0.0, qq = 0.0;
    for (int i = threadIdx.x; i < na; i += blockDim.x) rr += red[kRedPart + i];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        pq += red[kRedPart + kPartB + 3 * i];
        rq += red[kRedPart + kPartB + 3 * i + 1];
        qq += red[kRedPart + kPartB + 3 * i + 2];
    }
    block_sum4(rr, pq, rq, qq);
    if (threadIdx.x == 0) {
        double *s = red + kRedScal;
        if (!isfinite(rr) || !isfinite(pq) || !isfinite(rq) || !isfinite(qq)) s[S_FLAG] = 1.0;
        const double a = pq > 0.0 ? rr / pq : 0.0;
        if (!(pq > 0.0) && rr > 0.0) s[S_FLAG] = 2.0;  // breakdown: p.Ap <= 0
        const double rn = fmax(rr - 2.0 * a * rq + a * a * qq, 0.0);
        s[S_ALPHA] = a;
        s[S_BETA] = rr > 0.0 ? rn / rr : 0.0;
        s[S_PQ] = pq;
        s[S_RR] = rn;  // r.r after this iteration's (pending) update
    }
}

// r = (T) r64, p = 0, e = 0, q = 0 ; partial r.r
template <typename T>
__global__ void k_cg_init(const double *r64, T *r, T *pp, T *e, T *q, int64_t n, double *red)
{
    DSum acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T v = (T)r64[i];
        r[i] = v;
        pp[i] = T(0);
        e[i] = T(0);
        q[i] = T(0);
        acc.add_prod(v, v);
    }
    write_partial(red, acc);
}

// e += alpha p ; r -= alpha q ; partial r.r   (n a multiple of 2)
template <typename T>
__global__ void k_cg_update(T *e, T *r, const T *pp, const T *q, int64_t n, double *red)
{
    using V = typename vec2<T>::type;
    const T a = (T)red[kRedScal + S_ALPHA];
    DSum acc;
    const int64_t n2 = n / 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        V ev = reinterpret_cast<V *>(e)[i];
        V rv = reinterpret_cast<V *>(r)[i];
        const V pv = reinterpret_cast<const V *>(pp)[i];
        const V qv = reinterpret_cast<const V *>(q)[i];
        ev.x += a * pv.x;
        ev.y += a * pv.y;
        rv.x -= a * qv.x;
        rv.y -= a * qv.y;
        reinterpret_cast<V *>(e)[i] = ev;
        reinterpret_cast<V *>(r)[i] = rv;
        acc.add_prod(rv.x, rv.x);
        acc.add_prod(rv.y, rv.y);
    }
    write_partial(red, acc);
}

// p = r + beta p (state-based path, unfused)
template <typename T>
__global__ void k_cg_dir(T *pp, const T *r, int64_t n, const double *red)
{
    const T bt = (T)red[kRedScal + S_BETA];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pp[i] = r[i] + bt * pp[i];
}

// q = -chi_O L(p) in place ; partial p.q (state-based path, unfused)
template <typename T>
__global__ void k_cg_q(T *q, const T *pp, const uint8_t *co, int64_t n, double *red)
{
    DSum acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T v = co[i] ? -q[i] : T(0);
        q[i] = v;
        acc.add_prod(pp[i], v);
    }
    write_partial(red, acc);
}

// rows, forward: pending update e += alpha p, r -= alpha q, then
// p = r + beta p (stored), partials of r.r, transform chi p. Node fields come
// straight from global memory (coalesced pairs); only the mask bits are staged.
template <typename T, int D>
struct ProCG {
    static constexpr int kFin = 0, kFout = D, kNF = 0, kNB = 1, kStage = 0;
    static constexpr bool kSparse = false, kNodeAcc = true;
    static constexpr bool kFixedLength = std::is_same_v<T, float>;
    T *e, *r, *pv;
    const T *q;
    const uint8_t *bits;
    double *red;
    int64_t N;
    int n1;
    cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int) const { return nullptr; }
    __device__ cx<T> *spec_out(int f) const { return spec + f * fstride; }
    __device__ const T *nf_src(int) const { return nullptr; }
    __device__ const uint8_t *nb_src(int) const { return bits; }
    // e, r, p and q of the tile's rows start towards L2 while its mask bytes arrive
    __device__ __forceinline__ void l2_prefetch(int64_t row0, int rows) const
    {
        const int64_t base = row0 * n1;
        const unsigned bytes = (unsigned)(rows * n1 * sizeof(T));
#pragma unroll
        for (int j = 0; j < D; ++j) {
            bulk_prefetch_l2(e + j * N + base, bytes);
            bulk_prefetch_l2(r + j * N + base, bytes);
            bulk_prefetch_l2(pv + j * N + base, bytes);
            bulk_prefetch_l2(q + j * N + base, bytes);
        }
    }
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *, const T *, T *o0,
                                          T *o1, DSum &acc) const
    {
        const double *s = red + kRedScal;
        const T alpha = (T)s[S_ALPHA], beta = (T)s[S_BETA];
        const T v0 = (c.b(0, rl, i1) & 1) ? T(1) : T(0), v1 = (c.b(0, rl, i1 + 1) & 1) ? T(1) : T(0);
        const int64_t p = (c.row0 + rl) * n1 + i1;
        typename vec2<T>::type ee[D], rr[D], pp[D], qq[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            ee[j] = load2(e + j * N + p);
            rr[j] = load2(r + j * N + p);
            pp[j] = load2(pv + j * N + p);
            qq[j] = load2(q + j * N + p);
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            store2(e + j * N + p, ee[j].x + alpha * pp[j].x, ee[j].y + alpha * pp[j].y);
            const T ra = rr[j].x - alpha * qq[j].x, rb = rr[j].y - alpha * qq[j].y;
            store2(r + j * N + p, ra, rb);
            acc.add_prod(ra, ra);
            acc.add_prod(rb, rb);
            const T a = ra + beta * pp[j].x;
            const T b = rb + beta * pp[j].y;
            store2(pv + j * N + p, a, b);
            o0[j] = v0 * a;
            o1[j] = v1 * b;
        }
    }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    __device__ void emit(const RowCtx<T> &, int, int, const T *, const T *, DSum &) const {}
    __device__ void block_done(DSum &acc) const { write_partial(red, acc); }
};

static_assert(op_min_blocks<ProCG<float, 3>>::value == 1, "ProCG declares no register cap");

struct CgAcc {
    DSum pq, rq, qq;
};

// rows, inverse: L = chi y - G p (G from the boundary list, looked up per node
// with the p already in registers), q = -chi_O L, block partials of p.q,
// r.q, q.q
template <typename T, int D>
struct EpiCG {
    static constexpr int kFin = D, kFout = 0, kStage = D, kNF = 0, kNB = 1;
    static constexpr bool kSparse = false;
    static constexpr bool kFixedLength = std::is_same_v<T, float>;
    static constexpr int kMinBlocks = 4;  // <= 64 registers: more resident warps
    using Acc = CgAcc;
    // loads of one node pair: p, r and its boundary-list indices (read-only in this pass)
    struct EmitIn {
        typename vec2<T>::type pp[D], rr[D];
        int2 gi;
    };
    const T *pv, *r;
    const uint8_t *bits;
    const GEntry<T> *gent;
    const int *gidx;
    T *q;
    double *red;
    int64_t N;
    int n1;
    const cx<T> *spec;
    int64_t fstride;
    __device__ const cx<T> *spec_in(int f) const { return spec + f * fstride; }
    __device__ cx<T> *spec_out(int) const { return nullptr; }
    __device__ const T *nf_src(int) const { return nullptr; }
    __device__ const uint8_t *nb_src(int) const { return bits; }
    // p, r and the boundary index of the tile's rows start towards L2 while
    // the tile's spectra arrive and are transformed (one bulk prefetch each)
    __device__ __forceinline__ void l2_prefetch(int64_t row0, int rows) const
    {
        const int64_t base = row0 * n1;
        const unsigned bytes = (unsigned)(rows * n1 * sizeof(T));
#pragma unroll
        for (int j = 0; j < D; ++j) {
            bulk_prefetch_l2(pv + j * N + base, bytes);
            bulk_prefetch_l2(r + j * N + base, bytes);
        }
        bulk_prefetch_l2(gidx + base, (unsigned)(rows * n1 * sizeof(int)));
    }
    __device__ __forceinline__ void node2(const RowCtx<T> &c, int rl, int i1, const T *in0, const T *in1, T *o0,
                                          T *o1) const
    {
        const T v0 = (c.b(0, rl, i1) & 1) ? T(1) : T(0), v1 = (c.b(0, rl, i1 + 1) & 1) ? T(1) : T(0);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            o0[i] = v0 * in0[i];
            o1[i] = v1 * in1[i];
        }
    }
    __device__ void sparse(const RowCtx<T> &, int, int) const {}
    __device__ __forceinline__ void load_emit(const RowCtx<T> &c, int rl, int i1, EmitIn &in) const
    {
        using V = typename vec2<T>::type;
        const int64_t p = (c.row0 + rl) * n1 + i1;
        in.gi = __ldg(reinterpret_cast<const int2 *>(gidx + p));
#pragma unroll
        for (int i = 0; i < D; ++i) {
            in.pp[i] = __ldg(reinterpret_cast<const V *>(pv + i * N + p));
            in.rr[i] = __ldg(reinterpret_cast<const V *>(r + i * N + p));
        }
    }
    __device__ __forceinline__ void emit(const RowCtx<T> &c, int rl, int i1, const T *s0, const T *s1,
                                         CgAcc &acc) const
    {
        EmitIn in;
        load_emit(c, rl, i1, in);
        emit_loaded(c, rl, i1, s0, s1, acc, in);
    }
    __device__ __forceinline__ void emit_loaded(const RowCtx<T> &c, int rl, int i1, const T *s0, const T *s1,
                                                CgAcc &acc, const EmitIn &in) const
    {
        const int64_t p = (c.row0 + rl) * n1 + i1;
        const unsigned b0 = c.b(0, rl, i1), b1 = c.b(0, rl, i1 + 1);
        const int2 gi = in.gi;
        const typename vec2<T>::type *pp = in.pp, *rr = in.rr;
        T L0[D], L1[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            L0[i] = s0[i];
            L1[i] = s1[i];
        }
        if (gi.x >= 0) {
            const GEntry<T> e = gent[gi.x];
            T x[D], y[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                x[i] = pp[i].x;
                y[i] = T(0);
            }
            sym_apply<T, D>(e.g, x, y);
#pragma unroll
            for (int i = 0; i < D; ++i) L0[i] -= y[i];
        }
        if (gi.y >= 0) {
            const GEntry<T> e = gent[gi.y];
            T x[D], y[D];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                x[i] = pp[i].y;
                y[i] = T(0);
            }
            sym_apply<T, D>(e.g, x, y);
#pragma unroll
            for (int i = 0; i < D; ++i) L1[i] -= y[i];
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const T a = ((b0 >> (1 + i)) & 1) ? -L0[i] : T(0);
            const T b = ((b1 >> (1 + i)) & 1) ? -L1[i] : T(0);
            store2(q + i * N + p, a, b);
            acc.pq.add_prod(pp[i].x, a);
            acc.pq.add_prod(pp[i].y, b);
            acc.rq.add_prod(rr[i].x, a);
            acc.rq.add_prod(rr[i].y, b);
            acc.qq.add_prod(a, a);
            acc.qq.add_prod(b, b);
        }
    }
    __device__ void block_done(CgAcc &acc) const
    {
        const DSum *a[3] = {&acc.pq, &acc.rq, &acc.qq};
        double t[3];
        block_sums<3>(a, t);
        if (threadIdx.x == 0) {
            double *o = red + kRedPart + kPartB + 3 * blockIdx.x;
            o[0] = t[0];
            o[1] = t[1];
            o[2] = t[2];
        }
    }
};

static_assert(op_min_blocks<EpiCG<float, 3>>::value == EpiCG<float, 3>::kMinBlocks,
              "the row kernel must apply the epilogue's register cap");

// log2(n1 / 2) when the plane passes apply (FP32 cubes of 32^3, 64^3 or 128^3:
// one field of an x1-x2 plane fits in shared memory), else 0
template <typename T, int D>
int plane_lgh(const pd_plan *p)
{
    if (!std::is_same_v<T, float> || D != 3 || p->dim != 3 || p->n1 != p->n2 || !p->plane_passes || !p->gnode)
        return 0;
    if (D * p->n3 > kPartB) return 0;
    return p->n1 == 32 ? 4 : p->n1 == 64 ? 5 : p->n1 == 128 ? 6 : 0;
}

template <typename T, int D, int LGH>
pd_status launch_plane(pd_plan *p, bool fwd, const PlaneArgs<T> &pa, cudaStream_t st)
{
    using S = PlaneShape<T, LGH, LGH + 1>;
    const auto kern = fwd ? k_plane_cg_fwd<T, D, LGH, LGH + 1> : k_plane_cg_inv<T, D, LGH, LGH + 1>;
    PD_TRY(set_smem_attr((const void *)kern, S::smem));
    PD_TRY(prof_begin(p, fwd ? PASS_PLANE_FWD : PASS_PLANE_INV, st));
    PD_TRY(launch_k(p->pdl != 0, kern, dim3((unsigned)(D * p->n3)), dim3(S::THREADS), S::smem, st, pa,
                    tw_buf<T>(p)));
    PD_TRY(prof_end(p, st));
    p->launches++;
    return PD_OK;
}

struct Solver {
    pd_plan *p;
    cudaStream_t st;
    int64_t nvec;
    unsigned nb;

    double *hs() const { return p->host_scal; }

    pd_status finish(int nparts, int dst, int what)
    {
        k_finish<<<1, 1024, 0, st>>>(p->red, nparts, dst, what);
        PD_LAUNCH_CHECK();
        p->launches++;
        return PD_OK;
    }
    pd_status copy_scalars()
    {
        PD_CUDA_TRY(cudaMemcpyAsync(hs(), p->red + kRedScal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
        // the device status word (bounded-wait time-outs) rides along
        PD_CUDA_TRY(cudaMemcpyAsync(hs() + kHostStatus, p->dev_status, sizeof(int), cudaMemcpyDeviceToHost, st));
        return PD_OK;
    }
    int dev_status() const { return *reinterpret_cast<const int *>(hs() + kHostStatus); }
    pd_status read_scalars()
    {
        PD_TRY(copy_scalars());
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        return PD_OK;
    }

    // FP64 residual r64 = chi_O (b + L64(u)); returns ||r64||
    pd_status residual(const double *u, const double *b, double *rn)
    {
        PD_TRY(force_plain<double>(p, u, nullptr, p->r64, nullptr, st));
        k_residual<<<nb, 256, 0, st>>>(p->r64, b, p->chi_om, nvec, p->red);
        PD_LAUNCH_CHECK();
        p->launches++;
        PD_TRY(finish(nb, S_NORM, 0));
        PD_TRY(read_scalars());
        if (dev_status()) {  // a pass that gave up leaves its tiles unwritten: report that first
            set_error("pd_solve_static: a bounded device wait timed out (status %d)", dev_status());
            return PD_ERR_TIMEOUT;
        }
        *rn = std::sqrt(hs()[S_NORM]);
        if (!std::isfinite(*rn)) {
            set_error("pd_solve_static: non-finite residual");
            return PD_ERR_NONFINITE;
        }
        return PD_OK;
    }

    template <typename T, int D>
    pd_status plane_pass(int lgh, bool fwd, const PlaneArgs<T> &pa)
    {
        if constexpr (std::is_same_v<T, float> && D == 3) {
            switch (lgh) {
                case 4: return launch_plane<T, D, 4>(p, fwd, pa, st);
                case 5: return launch_plane<T, D, 5>(p, fwd, pa, st);
                case 6: return launch_plane<T, D, 6>(p, fwd, pa, st);
                default: break;
            }
        }
        set_error("plane pass for an unsupported shape");
        return PD_ERR_SIZE;
    }

    // one CG iteration (enqueued; no host synchronisation)
    template <typename T, int D>
    pd_status iteration()
    {
        T *e = (T *)p->cg_e, *r = (T *)p->cg_r, *pv = (T *)p->cg_p, *q = (T *)p->cg_q;
        if (p->state_based) {
            // state-based solid: the dilatation round trip sits between the
            // halves of the operator, so the vector steps run as own kernels
            k_cg_dir<T><<<nb, 256, 0, st>>>(pv, r, nvec, p->red);
            PD_LAUNCH_CHECK();
            PD_TRY(force_plain<T>(p, pv, nullptr, q, nullptr, st));
            k_cg_q<T><<<nb, 256, 0, st>>>(q, pv, p->chi_om, nvec, p->red);
            PD_LAUNCH_CHECK();
            PD_TRY(finish(nb, S_PQ, 1));
            k_cg_update<T><<<kUpdBlocks, 256, 0, st>>>(e, r, pv, q, nvec, p->red);
            PD_LAUNCH_CHECK();
            p->launches += 3;
            return finish(kUpdBlocks, S_RRNEW, 2);
        }
        cx<T> *spec = reinterpret_cast<cx<T> *>(spec_buf<T>(p));
        const int64_t fs = p->N / 2;
        const Model<T> m = model_view<T>(p);
        unsigned gpro = 0, gepi = 0;
        const int ob = D == 3 ? D : 0;
        const int lgh = plane_lgh<T, D>(p);
        const bool plane_fwd = lgh && (p->plane_passes & 1), plane_inv = lgh && (p->plane_passes & 2);
        const PlaneArgs<T> pa{e, r, pv, q, p->mbits, spec, fs, p->N, p->red, (const T *)p->gpe, p->gnode, p->goff,
                              p->ngent, p->lgl, p->dev_status, p->inject};
        if (plane_fwd) {
            PD_TRY((plane_pass<T, D>(lgh, true, pa)));
            gpro = (unsigned)(D * p->n3);
        } else {
            ProCG<T, D> pro{e, r, pv, q, p->mbits, p->red, p->N, p->n1, spec, fs};
            PD_TRY(launch_rows<T>(p, pro, st, &gpro));
            if (D == 3) PD_TRY((col_pass<T, D>(p, 0, false, st)));
        }
        if (plane_inv && p->ngent > 0) {
            // (G p) per boundary entry for the inverse plane pass, on the second
            // stream beside the last-axis pass (joined by that pass's join)
            const bool fork = p->aux_stream && !p->no_fork;
            cudaStream_t gs = fork ? p->aux_stream : st;
            if (fork) {
                PD_CUDA_TRY(cudaEventRecord(p->ev_fork[0], st));
                PD_CUDA_TRY(cudaStreamWaitEvent(gs, p->ev_fork[0], 0));
            }
            const unsigned gb = (unsigned)std::min<int64_t>((p->ngent + 255) / 256, 4 * (int64_t)p->nsm);
            k_gp_entries<T, D><<<gb, 256, 0, gs>>>(m.gent, p->ngent, (const T *)pv, p->N, (T *)p->gpe);
            PD_LAUNCH_CHECK();
            p->launches++;
        }
        CombForce<T, D, false> cmb{m, ob};
        PD_TRY(launch_cols<T>(p, cmb, D == 3 ? 2 : 1, true, D, st));
        if (plane_inv) {
            PD_TRY((plane_pass<T, D>(lgh, false, pa)));
            gepi = (unsigned)(D * p->n3);
        } else {
            if (D == 3) PD_TRY((col_pass<T, D>(p, ob, true, st)));
            EpiCG<T, D> epi{pv, r, p->mbits, m.gent, p->gidx, q, p->red, p->N, p->n1, spec + ob * fs, fs};
            PD_TRY(launch_rows<T>(p, epi, st, &gepi));
        }
        if (gpro > (unsigned)kPartB || gepi > (unsigned)kPartB) {
            set_error("pd_solve_static: %u / %u row blocks exceed the reduction buffer", gpro, gepi);
            return PD_ERR_SIZE;
        }
        PD_TRY(launch_k(p->pdl != 0, k_cg_finish_fused, dim3(1), dim3(kFinishThreads), 0, st, p->red, (int)gpro,
                        (int)gepi));
        p->launches++;
        return PD_OK;
    }

    // a chunk of kChunk iterations followed by a copy of the scalars to the
    // pinned host buffer, captured once into a CUDA graph per precision
    template <typename T, int D>
    pd_status chunk()
    {
        const int gi = sizeof(T) == 8 ? 1 : 0;
        if (p->cg_graph[gi] && p->cg_graph_prof[gi] != p->prof_on) {
            cudaGraphExecDestroy(p->cg_graph[gi]);
            p->cg_graph[gi] = nullptr;
        }
        if (!p->cg_graph[gi]) {
            if (p->prof_on) PD_TRY(prof_harvest(p));
            const int ev0 = p->ev_used;
            const int64_t l0 = p->launches;  // launches recorded by the capture = launches per replay
            cudaGraph_t graph = nullptr;
            PD_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            pd_status s = PD_OK;
            for (int k = 0; k < kChunk && s == PD_OK; ++k) s = iteration<T, D>();
            if (s == PD_OK) s = copy_scalars();
            const cudaError_t ce = cudaStreamEndCapture(st, &graph);
            if (s != PD_OK) {
                if (graph) cudaGraphDestroy(graph);
                return s;
            }
            if (ce != cudaSuccess) {
                set_error("graph capture failed: %s", cudaGetErrorString(ce));
                return PD_ERR_CUDA;
            }
            const cudaError_t ie = cudaGraphInstantiate(&p->cg_graph[gi], graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                p->cg_graph[gi] = nullptr;
                set_error("graph instantiation failed: %s", cudaGetErrorString(ie));
                return PD_ERR_CUDA;
            }
            p->cg_graph_prof[gi] = p->prof_on;
            p->cg_graph_ev[gi][0] = ev0;
            p->cg_graph_ev[gi][1] = p->ev_used;
            p->cg_graph_launches[gi] = p->launches - l0;
            p->launches = l0;
            p->ev_reserved = p->ev_used;  // keep the graph's event pairs
        }
        PD_CUDA_TRY(cudaGraphLaunch(p->cg_graph[gi], st));
        p->launches += p->cg_graph_launches[gi];
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        if (p->prof_on) PD_TRY(prof_harvest_range(p, p->cg_graph_ev[gi][0], p->cg_graph_ev[gi][1]));
        return PD_OK;
    }

    // CG on A e = r64 until ||r|| <= tol_abs or max_it; returns iterations done
    template <typename T, int D>
    pd_status cg(double tol_abs, int max_it, int *done)
    {
        T *e = (T *)p->cg_e, *r = (T *)p->cg_r, *pv = (T *)p->cg_p, *q = (T *)p->cg_q;
        k_cg_init<T><<<nb, 256, 0, st>>>(p->r64, r, pv, e, q, nvec, p->red);
        PD_LAUNCH_CHECK();
        p->launches++;
        PD_TRY(finish(nb, S_RR, 0));
        PD_CUDA_TRY(cudaMemsetAsync(p->red + kRedScal + S_ALPHA, 0, 2 * sizeof(double), st));  // alpha, beta
        int it = 0;
        double best = HUGE_VAL;
        int since_best = 0;
        while (it < max_it) {
            PD_TRY((chunk<T, D>()));
            it += kChunk;
            const double rn = std::sqrt(hs()[S_RR]);
            if (dev_status()) {
                set_error("pd_solve_static: a bounded device wait timed out (status %d)", dev_status());
                return PD_ERR_TIMEOUT;
            }
            if (hs()[S_FLAG] == 1.0) {
                set_error("pd_solve_static: non-finite CG scalar");
                return PD_ERR_NONFINITE;
            }
            if (hs()[S_FLAG] == 2.0 || rn <= tol_abs) break;
            // stagnation of the recursive residual (FP32 attainable accuracy):
            // no new minimum (by 0.1%) over the last half of the iterations and
            // at least 8 chunks (the CG residual norm is not monotone and can
            // plateau for long stretches on ill-conditioned problems)
            if (rn < 0.999 * best) {
                best = rn;
                since_best = 0;
            } else if ((since_best += kChunk) >= 8 * kChunk && 2 * since_best >= it) {
                break;
            }
        }
        if (!p->state_based) {
            // the fused iteration leaves the last e, r update pending
            k_cg_update<T><<<kUpdBlocks, 256, 0, st>>>(e, r, pv, (const T *)p->cg_q, nvec, p->red);
            PD_LAUNCH_CHECK();
            p->launches++;
        }
        *done = it;
        return PD_OK;
    }
};

}  // namespace
}  // namespace pd

using namespace pd;

namespace pd {
namespace {

// r64 = chi_O sin(2 pi (i1 + 2 i2 + 3 i3) / 64): a fixed right-hand side for timing
__global__ void k_tune_rhs(double *r, const uint8_t *co, int n1, int n2, int64_t N, int d)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)d * N;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = q % N;
        int i1, i2, i3;
        node_coords(p, n1, n2, i1, i2, i3);
        r[q] = co[q] ? sinpi((double)(i1 + 2 * i2 + 3 * i3 + (int)(q / N)) / 32.0) : 0.0;
    }
}

}  // namespace

// Time of one captured chunk of CG iterations (the static solver's unit of
// work) in the plan's current pass configuration; for the autotuner.
pd_status time_cg_chunk(pd_plan *p, cudaEvent_t e0, cudaEvent_t e1, float *ms_out)
{
    Solver S;
    S.p = p;
    S.st = p->own_stream;
    S.nvec = (int64_t)p->dim * p->N;
    S.nb = (unsigned)std::min<int64_t>(kUpdBlocks, (S.nvec + 255) / 256);
    k_tune_rhs<<<S.nb, 256, 0, S.st>>>(p->r64, p->chi_om, p->n1, p->n2, p->N, p->dim);
    PD_LAUNCH_CHECK();
    std::vector<float> t;
    for (int rep = 0; rep < 4; ++rep) {
        // restart from the same state; the first replay also captures the graph
        if (p->prob.fp64) {
            k_cg_init<double><<<S.nb, 256, 0, S.st>>>(p->r64, (double *)p->cg_r, (double *)p->cg_p,
                                                      (double *)p->cg_e, (double *)p->cg_q, S.nvec, p->red);
        } else {
            k_cg_init<float><<<S.nb, 256, 0, S.st>>>(p->r64, (float *)p->cg_r, (float *)p->cg_p,
                                                     (float *)p->cg_e, (float *)p->cg_q, S.nvec, p->red);
        }
        PD_LAUNCH_CHECK();
        PD_TRY(S.finish(S.nb, S_RR, 0));
        PD_CUDA_TRY(cudaMemsetAsync(p->red + kRedScal + S_ALPHA, 0, 2 * sizeof(double), S.st));
        PD_CUDA_TRY(cudaEventRecord(e0, S.st));
        if (p->prob.fp64)
            PD_TRY(p->dim == 3 ? (S.chunk<double, 3>()) : (S.chunk<double, 2>()));
        else
            PD_TRY(p->dim == 3 ? (S.chunk<float, 3>()) : (S.chunk<float, 2>()));
        PD_CUDA_TRY(cudaEventRecord(e1, S.st));
        PD_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        PD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    *ms_out = t[t.size() / 2];
    return PD_OK;
}

}  // namespace pd

extern "C" pd_status pd_solve_static(pd_plan *p, double *u, const double *b, const double *w, double rtol,
                                     int max_iter, int *iters_out, double *relres_out, void *stream)
{
    if (!p || !u || !b) {
        set_error("pd_solve_static: null plan, u or b");
        return PD_ERR_ARG;
    }
    if (!(rtol > 0) || max_iter < 1) {
        set_error("pd_solve_static: rtol must be > 0 and max_iter >= 1");
        return PD_ERR_ARG;
    }
    if (p->nonlinear) {
        set_error("pd_solve_static: the nonlinear bond model is available through pd_force only");
        return PD_ERR_ARG;
    }
    // The solve runs on the plan's own stream (CUDA graphs cannot be captured
    // on the legacy default stream), ordered after the caller's stream.
    cudaStream_t caller = (cudaStream_t)stream;
    PD_CUDA_TRY(cudaEventRecord(p->ev_join[0], caller));
    PD_CUDA_TRY(cudaStreamWaitEvent(p->own_stream, p->ev_join[0], 0));
    Solver S;
    S.p = p;
    S.st = p->own_stream;
    S.nvec = (int64_t)p->dim * p->N;
    S.nb = (unsigned)std::min<int64_t>(kUpdBlocks, (S.nvec + 255) / 256);
    PD_CUDA_TRY(cudaMemsetAsync(p->red + kRedScal, 0, sizeof(double) * S_COUNT, S.st));
    PD_CUDA_TRY(cudaMemsetAsync(p->dev_status, 0, sizeof(int), S.st));
    k_apply_bc<<<S.nb, 256, 0, S.st>>>(u, w, b, p->chi_om, S.nvec, p->red);
    PD_LAUNCH_CHECK();
    p->launches++;
    PD_TRY(S.finish(S.nb, S_BN, 0));
    PD_TRY(S.read_scalars());
    // the residual is relative to ||chi_O b||; a problem driven by the
    // prescribed w alone (b = 0 on Omega) takes the initial residual instead
    double scale = std::sqrt(S.hs()[S_BN]);
    int total = 0;
    double rel = 0.0;
    pd_status result = PD_ERR_NOT_CONVERGED;
    double target = 0.0;
    for (int outer = 0; outer < 64; ++outer) {
        double rn = 0.0;
        PD_TRY(S.residual(u, b, &rn));
        if (outer == 0) {
            if (!(scale > 0)) scale = (rn > 0 && std::isfinite(rn)) ? rn : 1.0;
            target = rtol * scale;
        }
        rel = rn / scale;
        if (rn <= target) {
            result = PD_OK;
            break;
        }
        if (total >= max_iter) break;
        int done = 0;
        if (p->prob.fp64) {
            if (p->dim == 3)
                PD_TRY((S.cg<double, 3>(0.5 * target, max_iter - total, &done)));
            else
                PD_TRY((S.cg<double, 2>(0.5 * target, max_iter - total, &done)));
            k_ir_update<double><<<S.nb, 256, 0, S.st>>>(u, (const double *)p->cg_e, p->chi_om, S.nvec);
        } else {
            // inner FP32 solve: reduce the residual by 1e-3 (the FP32 operator
            // resolves A e to about that accuracy), never below the target
            const double tol = std::max(1e-3 * rn, 0.5 * target);
            if (p->dim == 3)
                PD_TRY((S.cg<float, 3>(tol, max_iter - total, &done)));
            else
                PD_TRY((S.cg<float, 2>(tol, max_iter - total, &done)));
            k_ir_update<float><<<S.nb, 256, 0, S.st>>>(u, (const float *)p->cg_e, p->chi_om, S.nvec);
        }
        PD_LAUNCH_CHECK();
        p->launches++;
        total += done;
        if (done == 0) break;
    }
    PD_CUDA_TRY(cudaStreamSynchronize(S.st));
    PD_CUDA_TRY(cudaEventRecord(p->ev_join[1], S.st));
    PD_CUDA_TRY(cudaStreamWaitEvent(caller, p->ev_join[1], 0));
    int hstat = 0;
    PD_CUDA_TRY(cudaMemcpy(&hstat, p->dev_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (hstat) {
        set_error("pd_solve_static: a bounded device wait timed out (status %d)", hstat);
        return PD_ERR_TIMEOUT;
    }
    if (iters_out) *iters_out = total;
    if (relres_out) *relres_out = rel;
    if (result != PD_OK) set_error("pd_solve_static: relative residual %.3e above rtol %.3e after %d iterations",
                                   rel, rtol, total);
    return result;
}
