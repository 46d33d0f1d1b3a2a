// Plan object and launch helpers of the GB300 FCBM-EC library (private).
#pragma once

#include <algorithm>
#include <utility>

#include <vector>

#include "pd_common.cuh"
#include "pd_fft.cuh"

namespace pd {

// Packed-spectrum slots per plan. The 3D last-axis pass is out of place: its
// blocks read the mirror column k2 -> -k2 of another block's tile, so outputs
// go to slots after the inputs (inputs + outputs <= kMaxSpecFields).
constexpr int kMaxSpecFields = 20;

// One boundary node of the plan's G field (G != 0 only within delta of the
// body's boundary): the ncomp components in Sym order and the node index.
template <typename T>
struct GEntry {
    T g[6];
    int64_t p;
};

// Device-side view of the model used by the per-node and per-mode functors.
template <typename T>
struct Model {
    int dim;
    int n1, n2, n3;
    int h;             // n1 / 2
    int ky_half, kz_half;
    int64_t N;         // nodes
    int64_t nrows;     // n2 * n3
    const T *mhat;     // folded difference spectrum (K^(k) - K^(0)) / N, ncomp fields
    const T *ghat;     // folded dV/N * Σ g_i sin(theta) (state-based), 3 fields, or null
    int64_t fold_sz;   // entries per folded component: (h+1)(n2/2+1)(n3/2+1)
    const uint8_t *chi;
    const uint8_t *chi_om;  // d x N
    const T *G;        // ncomp x N boundary field for v = chi
    const GEntry<T> *gent;  // the same field as a list of boundary nodes, by row
    const int *goff;        // nrows + 1 offsets into gent
    const T *qt;       // 3 x N, state-based q_i(x) = dV (g_i * chi)
    const T *m3inv;    // N, 3/m(x) (0 outside the body)
    T ka;              // (3 kappa - 5 mu)/m0 (state-based)
};

struct HorizonDev {
    const int *off;   // 3 x cnt
    const double *c;  // ncomp x cnt: C_ij(xi) dV
    const double *g;  // 3 x cnt: g_i(xi) dV = omega xi_i dV (state-based), or
                      // a_i(xi) dV = alpha xi_i / |xi|^3 dV (nonlinear bond model)
    const double *w2; // cnt: omega |xi|^2 dV
    const double *cs; // cnt: c(xi) dV = alpha / |xi|^3 dV (nonlinear bond model), or null
    int cnt;
};

// Boundary field of a node weight v = chi s (Eq. 100 with the difference kernel):
//   G_c(x) = Σ_H C_c(xi) dV (v(x+xi) - v(x)),  G = 0 where chi = 0.
// For v = chi this is -(Σ_H C dV (1 - chi(x+xi))): zero in the delta-interior.
template <typename T, typename V, typename Acc>
__global__ void k_gfield(int n1, int n2, int n3, HorizonDev hz, int ncomp, const uint8_t *chi,
                         const V *s, T *G, int64_t N)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int i1, i2, i3;
    node_coords(p, n1, n2, i1, i2, i3);
    Acc acc[6] = {0, 0, 0, 0, 0, 0};
    if (chi[p]) {
        const Acc vp = s ? (Acc)s[p] : Acc(1);
        for (int c = 0; c < hz.cnt; ++c) {
            const int a = (i1 + hz.off[3 * c]) & (n1 - 1);
            const int b = (i2 + hz.off[3 * c + 1]) & (n2 - 1);
            const int e = (i3 + hz.off[3 * c + 2]) & (n3 - 1);
            const int64_t q = ((int64_t)e * n2 + b) * n1 + a;
            const Acc vq = chi[q] ? (s ? (Acc)s[q] : Acc(1)) : Acc(0);
            const Acc dv = vq - vp;
            if (dv != Acc(0))
                for (int k = 0; k < ncomp; ++k) acc[k] += (Acc)hz.c[k * hz.cnt + c] * dv;
        }
    }
    for (int k = 0; k < ncomp; ++k) G[k * N + p] = (T)acc[k];
}

// Kernel-spectrum lookup from a tile's shared-memory slice (component stride cs)
template <typename T>
__device__ __forceinline__ void load_mhat_s(int dim, const T *t, int cs, bool fy, bool fz, T *M /*3x3*/)
{
    if (dim == 2) {
        const T m11 = t[0], m22 = t[cs], m12 = fy ? -t[2 * cs] : t[2 * cs];
        M[0] = m11; M[1] = m12; M[3] = m12; M[4] = m22;
    } else {
        const T m11 = t[0], m22 = t[cs], m33 = t[2 * cs];
        const T m12 = fy ? -t[3 * cs] : t[3 * cs];
        const T m13 = fz ? -t[4 * cs] : t[4 * cs];
        const T m23 = (fy != fz) ? -t[5 * cs] : t[5 * cs];
        M[0] = m11; M[1] = m12; M[2] = m13;
        M[3] = m12; M[4] = m22; M[5] = m23;
        M[6] = m13; M[7] = m23; M[8] = m33;
    }
}

// gamma_i (odd in k_i) from a slice whose components start at t
template <typename T>
__device__ __forceinline__ void load_ghat_s(const T *t, int cs, bool fy, bool fz, T *g)
{
    g[0] = t[0];
    g[1] = fy ? -t[cs] : t[cs];
    g[2] = fz ? -t[2 * cs] : t[2 * cs];
}

struct LaunchCfg {
    dim3 grid, block;
    size_t smem;
};

}  // namespace pd

struct pd_plan {
    pd_problem prob;
    int dim, n1, n2, n3, h, ncomp;
    int64_t N, nrows;
    int lgl;            // log2 twiddle table length
    double dV, alpha;   // bond constant (or 30 mu / m0 for the state-based C)
    double ka, m0;      // state-based constants
    double lam_max;     // largest eigenvalue of the periodic symbol
    double wc = 0.0;    // critical energy density of bond breaking (problem Wc, or from s0)
    int state_based;    // model == PD_LIN_STATE && ka != 0 (dilatation round needed)
    int hcount;
    // device memory
    uint8_t *chi = nullptr, *chi_om = nullptr;
    uint8_t *mbits = nullptr;      // N: bit 0 chi_B, bit 1+c chi_Omega of component c
    int *hoff = nullptr;           // 3 x hcount integer offsets
    double *mhat64 = nullptr;      // ncomp x fold_sz
    float *mhat32 = nullptr;
    double *ghat64 = nullptr;      // 3 x fold_sz (state-based; nonlinear bond model: the a_i spectrum)
    double *chat64 = nullptr;      // fold_sz: (c^(k) - c^(0)) / N (nonlinear bond model)
    float *chat32 = nullptr;
    void *nlb = nullptr;           // nonlinear bond model: per boundary entry S(a_j, chi) (d values) and
                                   // S(c, chi) - c^(0) chi (slot 3), [ngent][4] in the plan's precision
    int nonlinear = 0;             // model == PD_NONLIN_BOND
    double body_count = 0.0;       // Σ chi
    float *ghat32 = nullptr;
    int64_t fold_sz = 0;
    double *G64 = nullptr;         // ncomp x N
    float *G32 = nullptr;
    int *goff = nullptr;           // nrows + 1: boundary-node list offsets per row
    int *gidx = nullptr;           // N: entry of the node in the boundary list, or -1
    int *gnode = nullptr;          // [ngent] node of each boundary entry (plane-pass cubes only)
    void *gpe = nullptr;           // [3][ngent] FP32 (G p) per boundary entry, written by the CG iteration
                                   // while its last-axis pass runs (plane-pass cubes only)
    void *gent64 = nullptr;        // GEntry<double>[ngent]
    void *gent32 = nullptr;        // GEntry<float>[ngent]
    // affine split of pd_force (pd_plan_set_affine_split): per boundary entry the
    // moments M_(ij)k = Σ_H chi(x+xi) C_ij(xi) dV o_k (o = integer offset), in the
    // plan's precision, [ngent][ncomp * dim]; the fitted coefficients; the body's
    // moment inverse and centre (host)
    void *aff_tab = nullptr;
    void *aff_coef = nullptr;      // 32 values of the plan's precision
    int affine_split = 0;
    int aff_ok = 0;                // body moments invertible
    int aff_c[3] = {0, 0, 0};      // centre node (integer grid indices)
    double aff_inv[16] = {};       // inverse of the (d+1)^2 normal matrix of the least-squares fit
    double aff_emax[3] = {0, 0, 0};
    int64_t ngent = 0;
    double *qt64 = nullptr, *m3inv64 = nullptr;  // state-based
    float *qt32 = nullptr, *m3inv32 = nullptr;
    pd::cx<double> *tw64 = nullptr;
    pd::cx<float> *tw32 = nullptr;
    void *spec32 = nullptr;        // spec32_slots x N floats (packed spectra)
    void *spec64 = nullptr;        // spec64_slots x N doubles
    int spec32_slots = 0, spec64_slots = 0;
    int *dev_status = nullptr;     // device status word (bounded-wait time-outs)
    int *inject = nullptr;         // row-pass stall word (pd_plan_inject_stall), next to dev_status
    void *work = nullptr;          // one allocation carved into the scratch fields below
    size_t work_bytes = 0;
    // scratch fields (plan precision T unless noted)
    void *cg_e = nullptr, *cg_r = nullptr, *cg_p = nullptr, *cg_q = nullptr;  // d x N each
    void *theta = nullptr;         // N, dilatation (state-based)
    void *Gw = nullptr;            // ncomp x N, boundary field of a node weight
    double *r64 = nullptr;         // d x N, FP64 residual / force
    double *theta64 = nullptr;     // N, FP64 dilatation for the FP64 residual
    double *red = nullptr;         // reduction partials and scalars
    int64_t bytes = 0;
    int64_t launches = 0;
    int nsm = 148;
    pd::HorizonDev hdev;  // device horizon tables (views into hoff)
    // per-pass timing (diagnostics): event pairs around each FFT-pass launch
    static constexpr int kEvPool = 1024;
    static constexpr int kKinds = 6;
    cudaEvent_t ev[2 * kEvPool] = {};
    int ev_kind[kEvPool] = {};
    int ev_used = 0;
    int ev_reserved = 0;            // pairs [0, ev_reserved) belong to captured graphs
    int prof_on = 0;                // bit k: time pass kind k
    int prof_cur = 0;               // the launch being bracketed is timed
    // cached CUDA graph of a chunk of CG iterations (per precision)
    cudaGraphExec_t cg_graph[2] = {nullptr, nullptr};
    int cg_graph_prof[2] = {0, 0};
    int cg_graph_ev[2][2] = {{0, 0}, {0, 0}};
    int64_t cg_graph_launches[2] = {0, 0};  // kernel launches per replay
    double *host_scal = nullptr;    // pinned host copy of the solver scalars
    cudaStream_t own_stream = nullptr;  // plan stream for captured work (never the legacy stream)
    cudaEvent_t ev_join[2] = {nullptr, nullptr};
    // second stream: the kx = 0 tiles of the 3D last-axis pass run beside the others
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_fork[2] = {nullptr, nullptr};
    int no_fork = 0;  // set while capturing into conditional-node bodies (single stream there)
    int pdl = 1;      // pass kernels launched as programmatic dependents (griddepcontrol)
    int plane_passes = 1;  // FP32 CG on cubes up to 128^3: halves of the iteration whose x1 and x2
                           // transforms run fused in plane passes (bit 0 forward, bit 1 inverse)
    double prof_ms[kKinds] = {};
    // pass configuration picked by pd_plan_autotune (0: built-in heuristic)
    int tune_rows = 0;     // rows per row-pass block
    int tune_w[2] = {0, 0};  // column-tile width of the x2 / last-axis passes
    int tune_sched = 0;    // FFT stage schedule
    int tune_stages = 0;   // row-pass pipeline stages (1 or 2; 0: 2)
    int tune_stages_inv = 0;  // the same for the inverse row passes (0: as tune_stages)
    int energy_direct = 0; // pd_step_verlet: W by a direct horizon sum (pd_plan_set_energy_mode)
    int64_t prof_n[kKinds] = {};
};

namespace pd {

template <typename T>
Model<T> model_view(const pd_plan *p);

template <typename T>
inline T *spec_buf(const pd_plan *p);
template <>
inline float *spec_buf<float>(const pd_plan *p) { return (float *)p->spec32; }
template <>
inline double *spec_buf<double>(const pd_plan *p) { return (double *)p->spec64; }

template <typename T>
inline const cx<T> *tw_buf(const pd_plan *p);
template <>
inline const cx<float> *tw_buf<float>(const pd_plan *p) { return p->tw32; }
template <>
inline const cx<double> *tw_buf<double>(const pd_plan *p) { return p->tw64; }

// Row-pass configuration: FB packed-row slots, NF node fields of T, NB byte
// fields; two pipeline stages. c.grid is the tile count; launch_rows caps it
// at the resident blocks (the kernel is persistent).
template <typename T>
inline void row_cfg(const pd_plan *p, int FI, int FB, int NF, int NB, RowGeom &g, LaunchCfg &c)
{
    const int H = p->h, nt = H >> kLgV, n1 = 2 * H;
    const int pad = nt < 16 ? (nt < 2 ? 2 : nt) : 0;  // keeps rows 16-byte aligned, spreads banks
    const int pitch = H + pad;
    const int ns_fwd = p->tune_stages == 1 ? 1 : 2;
    const int ns = (FI > 0 && p->tune_stages_inv > 0) ? p->tune_stages_inv : ns_fwd;
    auto smem_of = [&](int rows) { return row_smem_bytes<T>(FI, FB, NF, NB, rows, pitch, n1, ns); };
    int rows = p->tune_rows > 0 ? p->tune_rows : 128 / nt;
    if (rows < 1) rows = 1;
    // whole warps: the epilogues' block reductions shuffle over full warps
    // (the heuristic and the autotuner never go below; a pinned value could)
    if (rows * nt < 32) rows = 32 / nt;
    while (rows > 1 && rows * nt > 256) rows >>= 1;  // k_rows launch bound
    while (rows > 1 && smem_of(rows) > 100 * 1024) rows >>= 1;
    while (p->nrows % rows) rows >>= 1;
    g.lgh = ilog2(H);
    g.rows = rows;
    g.pitch = pitch;
    g.nrows = p->nrows;
    g.lgl = p->lgl;
    g.sched = p->tune_sched;
    g.nstage = ns;
    g.err = p->dev_status;
    g.inject = p->inject;
    c.grid = dim3((unsigned)(p->nrows / rows));
    c.block = dim3(rows * nt);
    c.smem = smem_of(rows);
}

// Column-pass configuration: axis 1 = x2, axis 2 = x3 (3D); FB fields in the
// tile, FI of them with a mirror column. The 3D last-axis pass runs as two
// launches with one tile width: tmode 1 (tiles without kx = 0: no mirror
// column, no kx = n1/2 table column) and tmode 2 (the kx = 0 tile of each k2
// row, with the mirror column of -k2).
template <typename T>
inline void col_cfg(const pd_plan *p, int axis, bool last, int FB, int FI, int NTAB, int tmode, ColGeom &g,
                    LaunchCfg &c, int64_t &inner)
{
    const int H = p->h;
    const int L = axis == 1 ? p->n2 : p->n3;
    const int nt = L >> kLgV;
    const bool split = p->dim == 3 && last;
    const int wmirror = split ? 1 : 0;  // the width must also fit the kx = 0 tiles
    const int mirror = (tmode == 2 || (split && tmode == 0)) ? 1 : 0;  // tmode 0 + split: one launch, all tiles
    inner = axis == 1 ? (int64_t)H : (int64_t)p->n2 * H;
    auto smem_of = [&](int w, int mir, int tc) {
        const size_t tab = (((size_t)NTAB * (L / 2 + 1) * tc + 1) & ~(size_t)1) * sizeof(T);
        return (size_t)L * sizeof(cx<T>) + (size_t)FB * L * w * sizeof(cx<T>) +
               (mir ? (size_t)FB * L * 2 * sizeof(cx<T>) : 0) + tab + 8 * ((size_t)FB + 1);
    };
    int w = p->tune_w[last ? 1 : 0] > 0 ? p->tune_w[last ? 1 : 0] : 32;
    while (w > 2 && ((w + wmirror) * nt > 512 || smem_of(w, wmirror, w + 1) > 100 * 1024 || (H % w))) w >>= 1;
    g.lgl = ilog2(L);
    g.w = w;
    g.lgw = ilog2(w);
    g.mirror = mirror;
    g.lgh = ilog2(H);
    g.n2 = p->n2;
    g.lgtw = p->lgl;
    g.lb = L < 256 ? L : 256;
    g.outer = axis == 1 ? p->n3 : 1;
    g.sched = p->tune_sched;
    g.tmode = split ? tmode : 0;
    g.err = p->dev_status;
    unsigned gx = (unsigned)(inner / w);
    if (split && tmode != 0) gx = tmode == 2 ? (unsigned)p->n2 : (unsigned)(p->n2 * (H / w - 1));
    c.grid = dim3(gx, (unsigned)g.outer);
    c.block = dim3((w + mirror) * nt);
    c.smem = smem_of(w, mirror, w + (split && tmode == 1 ? 0 : 1));
}

pd_status set_smem_attr(const void *func, size_t smem);

// pass kinds for the timing facility
enum PassKind { PASS_ROWS_FWD = 0, PASS_COLS = 1, PASS_LAST = 2, PASS_ROWS_INV = 3, PASS_PLANE_FWD = 4, PASS_PLANE_INV = 5 };
pd_status prof_harvest(pd_plan *p);
pd_status prof_harvest_range(pd_plan *p, int b, int e);

// Layout of the plan's FP64 reduction buffer (65536 doubles).
constexpr int kRedPart = 0;       // block partial sums (up to kMaxPart)
constexpr int kMaxPart = 58000;
constexpr int kRedScal = 60000;   // solver scalars
constexpr int kRedVerlet = 62000; // Verlet counters
// the device status word sits in the last 64 bytes
// Events recorded while the stream is being captured must become external
// event nodes of the graph, so that each replay records them.
inline cudaError_t prof_record(cudaEvent_t e, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t r = cudaStreamIsCapturing(st, &cs);
    if (r != cudaSuccess) return r;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal)
                                               : cudaEventRecord(e, st);
}

inline pd_status prof_begin(pd_plan *p, int kind, cudaStream_t st)
{
    p->prof_cur = ((p->prof_on >> kind) & 1) != 0;
    if (!p->prof_cur) return PD_OK;
    if (p->ev_used == pd_plan::kEvPool) PD_TRY(prof_harvest(p));
    if (p->ev_used == pd_plan::kEvPool) {
        set_error("profiling event pool exhausted");
        return PD_ERR_ARG;
    }
    p->ev_kind[p->ev_used] = kind;
    PD_CUDA_TRY(prof_record(p->ev[2 * p->ev_used], st));
    return PD_OK;
}
inline pd_status prof_end(pd_plan *p, cudaStream_t st)
{
    if (!p->prof_cur) return PD_OK;
    PD_CUDA_TRY(prof_record(p->ev[2 * p->ev_used + 1], st));
    p->ev_used++;
    return PD_OK;
}

// Launch with the programmatic-stream-serialization attribute when pdl is set:
// the kernel may start while its predecessor in the stream finishes and waits
// for it with griddepcontrol.wait (every pass kernel does, before it touches
// data of the preceding pass).
template <typename... KArgs, typename... Args>
inline pd_status launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return PD_ERR_CUDA;
    }
    return PD_OK;
}

// Row ops that declare kFixedLength = true also get row kernels compiled for
// the packed row lengths of the 128^3 to 512^3 boxes (64 to 256 values), one
// per stage schedule where the schedule matters; other lengths use the kernel
// that reads the length at run time.
template <class Op, class = void>
struct op_fixed_len : std::false_type {
};
template <class Op>
struct op_fixed_len<Op, std::void_t<decltype(Op::kFixedLength)>> : std::bool_constant<Op::kFixedLength> {
};

template <typename T, class Op>
auto rows_kernel(int lgh, int sched)
{
    using K = decltype(&k_rows<T, Op>);
    if constexpr (op_fixed_len<Op>::value) {
        switch (lgh) {
            case 6: return (K)&k_rows<T, Op, 6, 0>;
            case 7: return sched ? (K)&k_rows<T, Op, 7, 1> : (K)&k_rows<T, Op, 7, 0>;
            case 8: return sched ? (K)&k_rows<T, Op, 8, 1> : (K)&k_rows<T, Op, 8, 0>;
            default: break;
        }
    }
    return (K)&k_rows<T, Op>;
}

// Persistent row pass: as many blocks as fit on the GPU at once (at most one
// per tile). *grid_out receives the block count (the number of block partial
// sums an op with a block accumulator writes).
template <typename T, class Op>
pd_status launch_rows(pd_plan *p, const Op &op, cudaStream_t st, unsigned *grid_out = nullptr)
{
    RowGeom g;
    LaunchCfg c;
    constexpr int KO = Op::kFout > Op::kStage ? Op::kFout : Op::kStage;
    constexpr int FB = Op::kFin > KO ? Op::kFin : KO;
    row_cfg<T>(p, Op::kFin, FB, Op::kNF, Op::kNB, g, c);
    const auto kern = rows_kernel<T, Op>(g.lgh, g.sched);
    PD_TRY(set_smem_attr((const void *)kern, c.smem));
    int per_sm = 0;
    PD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)c.block.x, c.smem));
    const int64_t cap = (int64_t)std::max(per_sm, 1) * p->nsm;
    if ((int64_t)c.grid.x > cap) c.grid.x = (unsigned)cap;
    if (grid_out) *grid_out = c.grid.x;
    PD_TRY(prof_begin(p, Op::kFin > 0 ? PASS_ROWS_INV : PASS_ROWS_FWD, st));
    PD_TRY(launch_k(p->pdl != 0, kern, c.grid, c.block, c.smem, st, g, op, tw_buf<T>(p)));
    PD_TRY(prof_end(p, st));
    p->launches++;
    return PD_OK;
}

template <typename T>
inline int spec_slots(const pd_plan *p) { return sizeof(T) == 8 ? p->spec64_slots : p->spec32_slots; }

template <class Op>
constexpr int op_tab()
{
    if constexpr (Op::kMode == 2)
        return Op::kTab;
    else
        return 0;
}

template <typename T, class Op>
pd_status launch_cols(pd_plan *p, const Op &op, int axis, bool last, int F, cudaStream_t st)
{
    // The 3D last-axis pass runs as two launches: the kx = 0 tiles (one per k2
    // row, with the mirror column) on the plan's second stream beside the
    // other tiles on `st` (fork and join by events; inside a stream capture
    // they become parallel graph branches). Bodies of conditional graph nodes
    // are captured from one stream only (no_fork): there the two launches
    // follow each other.
    const bool split = p->dim == 3 && last;
    const bool fork = split && p->aux_stream && !p->no_fork;
    PD_TRY(prof_begin(p, last ? PASS_LAST : PASS_COLS, st));
    if (fork) {
        PD_CUDA_TRY(cudaEventRecord(p->ev_fork[0], st));
        PD_CUDA_TRY(cudaStreamWaitEvent(p->aux_stream, p->ev_fork[0], 0));
    }
    for (int tmode = split ? 2 : 0; tmode >= (split ? 1 : 0); --tmode) {
        cudaStream_t ls = (fork && tmode == 2) ? p->aux_stream : st;
        ColGeom g;
        LaunchCfg c;
        int64_t inner = 0;
        col_cfg<T>(p, axis, last, F, Op::kFin, Op::kMode == 2 ? op_tab<Op>() : 0, tmode, g, c, inner);
        if (c.grid.x == 0) continue;  // one tile per k2 row: no tmode-1 tiles
        const int L = 1 << g.lgl;
        const unsigned long long dims[3] = {(unsigned long long)(2 * inner), (unsigned long long)L,
                                            (unsigned long long)g.outer * spec_slots<T>(p)};
        const unsigned long long strides[2] = {(unsigned long long)(2 * inner * sizeof(T)),
                                               (unsigned long long)(2 * inner * L * sizeof(T))};
        const unsigned box_t[3] = {(unsigned)(2 * g.w), (unsigned)g.lb, 1u};
        const unsigned box_m[3] = {4u, (unsigned)g.lb, 1u};
        CUtensorMap tmt, tmm;
        PD_TRY(encode_tmap_3d(&tmt, spec_buf<T>(p), sizeof(T) == 8, dims, strides, box_t));
        PD_TRY(encode_tmap_3d(&tmm, spec_buf<T>(p), sizeof(T) == 8, dims, strides, box_m));
        PD_TRY(set_smem_attr((const void *)k_cols<T, Op>, c.smem));
        PD_TRY(launch_k(p->pdl != 0, k_cols<T, Op>, c.grid, c.block, c.smem, ls, g, op, tw_buf<T>(p),
                        axis == 2 ? 1 : 0, tmt, tmm));
        p->launches++;
    }
    if (fork) {
        PD_CUDA_TRY(cudaEventRecord(p->ev_fork[1], p->aux_stream));
        PD_CUDA_TRY(cudaStreamWaitEvent(st, p->ev_fork[1], 0));
    }
    PD_TRY(prof_end(p, st));
    return PD_OK;
}

// Plain column FFT of F packed spectra (slots slot0 ... slot0+F-1) along x2, in place.
template <typename T, int F, int MODE>
struct ColPass {
    static constexpr int kFin = F, kFout = F, kMode = MODE, kPre = 0, kTab = 0;
    static constexpr bool kStoreIn = false;
    int slot0;
    __device__ int slot_in(int f) const { return slot0 + f; }
    __device__ int slot_out(int f) const { return slot0 + f; }
    __device__ int slot_aux(int) const { return 0; }
    __device__ const T *table(int) const { return nullptr; }
    __device__ void combine(const T *, int, bool, bool, const cx<T> *, cx<T> *) const {}
};

template <typename T, int F>
pd_status col_pass(pd_plan *p, int slot0, bool inverse, cudaStream_t st)
{
    if (inverse) {
        ColPass<T, F, 1> op{slot0};
        return launch_cols<T>(p, op, 1, false, F, st);
    }
    ColPass<T, F, 0> op{slot0};
    return launch_cols<T>(p, op, 1, false, F, st);
}

}  // namespace pd
