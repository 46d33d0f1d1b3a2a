// Plan creation: validation, horizon, kernel spectra, boundary fields, twiddles.
//
// Everything here runs once per plan (§4.1.1: "P can be computed once and
// stored as a preprocessing step"); all device memory of the library is
// allocated here so that later calls allocate nothing.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <vector>

#include <map>
#include <mutex>

#include "pd_plan.cuh"

namespace pd {

static thread_local char g_err[512];

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

pd_status encode_tmap_3d(CUtensorMap *m, void *base, bool fp64, const unsigned long long dims[3],
                         const unsigned long long strides[2], const unsigned box[3])
{
    typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                                               cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f) {
            set_error("cuTensorMapEncodeTiled is not available from the driver");
            return PD_ERR_CUDA;
        }
        fn = (EncodeFn)f;
    }
    const cuuint64_t gd[3] = {dims[0], dims[1], dims[2]};
    const cuuint64_t gs[2] = {strides[0], strides[1]};
    const cuuint32_t bx[3] = {box[0], box[1], box[2]};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = fn(m, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, gd, gs,
                          bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d): dims %llu x %llu x %llu, box %u x %u x %u", (int)r, dims[0],
                  dims[1], dims[2], box[0], box[1], box[2]);
        return PD_ERR_CUDA;
    }
    return PD_OK;
}

// The dynamic shared-memory limit is a property of the kernel function, shared
// by every plan and by every kernel node of a captured graph: it only ever
// grows, so plans of different sizes never lower it under each other.
pd_status set_smem_attr(const void *func, size_t smem)
{
    static std::mutex mu;
    static std::map<const void *, size_t> set;
    if (smem <= 48 * 1024) return PD_OK;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = set[func];
    if (smem <= cur) return PD_OK;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        set_error("cudaFuncSetAttribute(%zu bytes): %s", smem, cudaGetErrorString(e));
        return PD_ERR_CUDA;
    }
    cur = smem;
    return PD_OK;
}

pd_status prof_harvest_range(pd_plan *p, int b, int e)
{
    if (e <= b) return PD_OK;
    PD_CUDA_TRY(cudaEventSynchronize(p->ev[2 * e - 1]));
    for (int i = b; i < e; ++i) {
        float ms = 0.f;
        PD_CUDA_TRY(cudaEventElapsedTime(&ms, p->ev[2 * i], p->ev[2 * i + 1]));
        p->prof_ms[p->ev_kind[i]] += ms;
        p->prof_n[p->ev_kind[i]]++;
    }
    return PD_OK;
}

// Harvest the event pairs of direct launches (those above the graph reservation).
pd_status prof_harvest(pd_plan *p)
{
    PD_TRY(prof_harvest_range(p, p->ev_reserved, p->ev_used));
    p->ev_used = p->ev_reserved;
    return PD_OK;
}

template <typename T>
Model<T> model_view(const pd_plan *p)
{
    Model<T> m;
    m.dim = p->dim;
    m.n1 = p->n1;
    m.n2 = p->n2;
    m.n3 = p->n3;
    m.h = p->h;
    m.ky_half = p->n2 / 2;
    m.kz_half = p->n3 / 2;
    m.N = p->N;
    m.nrows = p->nrows;
    m.fold_sz = p->fold_sz;
    m.chi = p->chi;
    m.chi_om = p->chi_om;
    m.goff = p->goff;
    if constexpr (sizeof(T) == 8) {
        m.gent = (const GEntry<T> *)p->gent64;
        m.mhat = (const T *)p->mhat64;
        m.ghat = (const T *)p->ghat64;
        m.G = (const T *)p->G64;
        m.qt = (const T *)p->qt64;
        m.m3inv = (const T *)p->m3inv64;
    } else {
        m.gent = (const GEntry<T> *)p->gent32;
        m.mhat = (const T *)p->mhat32;
        m.ghat = (const T *)p->ghat32;
        m.G = (const T *)p->G32;
        m.qt = (const T *)p->qt32;
        m.m3inv = (const T *)p->m3inv32;
    }
    m.ka = (T)p->ka;
    return m;
}
template Model<float> model_view<float>(const pd_plan *);
template Model<double> model_view<double>(const pd_plan *);

// ---------------------------------------------------------------------------
// Plan-time kernels (FP64)
// ---------------------------------------------------------------------------

// Folded spectra: for kx in [0, h], ky in [0, n2/2], kz in [0, n3/2]:
//   mhat_c(k) = (1/N) Σ_H C_c(xi) dV (cos(theta) - 1) = -(2/N) Σ C_c dV sin^2(theta/2)
//   ghat_i(k) = (1/N) Σ_H g_i(xi) dV sin(theta)
// theta = 2 pi Σ_a k_a o_a / n_a, reduced exactly with integer arithmetic.
//   chat(k)   = (1/N) Σ_H c(xi) dV (cos(theta) - 1)   (nonlinear bond model, when chat is given)
__global__ void k_fold_tables(int dim, int n1, int n2, int n3, int h, HorizonDev hz, int ncomp,
                              double invN, double *mhat, double *ghat, int64_t fold_sz, double *chat = nullptr)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= fold_sz) return;
    const int kx = (int)(t % (h + 1));
    const int ky = (int)((t / (h + 1)) % (n2 / 2 + 1));
    const int kz = (int)(t / ((int64_t)(h + 1) * (n2 / 2 + 1)));
    const int nmax = max(n1, max(n2, n3));
    const int s1 = nmax / n1, s2 = nmax / n2, s3 = nmax / n3;
    double accm[6] = {0, 0, 0, 0, 0, 0}, accg[3] = {0, 0, 0}, accc = 0.0;
    for (int c = 0; c < hz.cnt; ++c) {
        const int o1 = hz.off[3 * c], o2 = hz.off[3 * c + 1], o3 = hz.off[3 * c + 2];
        long long num = (long long)kx * o1 * s1 + (long long)ky * o2 * s2 + (long long)kz * o3 * s3;
        num %= nmax;
        if (num < 0) num += nmax;
        const double frac = (double)num / (double)nmax;  // theta / (2 pi) in [0, 1)
        const double sh = sinpi(frac);                   // sin(theta / 2)
        const double one_minus_cos = 2.0 * sh * sh;
        for (int q = 0; q < ncomp; ++q) accm[q] -= hz.c[q * hz.cnt + c] * one_minus_cos;
        if (chat) accc -= hz.cs[c] * one_minus_cos;
        if (ghat) {
            const double sn = sinpi(2.0 * frac);
            for (int i = 0; i < 3; ++i) accg[i] += hz.g[i * hz.cnt + c] * sn;
        }
    }
    for (int q = 0; q < ncomp; ++q) mhat[q * fold_sz + t] = accm[q] * invN;
    if (chat) chat[t] = accc * invN;
    if (ghat)
        for (int i = 0; i < 3; ++i) ghat[i * fold_sz + t] = accg[i] * invN;
    (void)dim;
}

// Unfolded FP64 kernel spectrum K^_c(k) = Σ_H C_c(xi) dV cos(theta), k1 in [0, n1/2].
__global__ void k_kernel_spectrum(int n1, int n2, int n3, int h, HorizonDev hz, int ncomp, double *out,
                                  int64_t total)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int kx = (int)(t % (h + 1));
    const int ky = (int)((t / (h + 1)) % n2);
    const int kz = (int)(t / ((int64_t)(h + 1) * n2));
    const int nmax = max(n1, max(n2, n3));
    const int s1 = nmax / n1, s2 = nmax / n2, s3 = nmax / n3;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int c = 0; c < hz.cnt; ++c) {
        long long num = (long long)kx * hz.off[3 * c] * s1 + (long long)ky * hz.off[3 * c + 1] * s2 +
                        (long long)kz * hz.off[3 * c + 2] * s3;
        num %= nmax;
        if (num < 0) num += nmax;
        const double cs = cospi(2.0 * (double)num / (double)nmax);
        for (int q = 0; q < ncomp; ++q) acc[q] += hz.c[q * hz.cnt + c] * cs;
    }
    for (int q = 0; q < ncomp; ++q) out[q * total + t] = acc[q];
}

// State-based node fields: q_i(x) = Σ_H g_i dV chi(x+xi), m(x) = chi Σ_H omega|xi|^2 dV chi(x+xi)
// (Eq. 93-94, 96-97), stored as q_i and 3/m (0 outside the body).
__global__ void k_state_fields(int n1, int n2, int n3, HorizonDev hz, const uint8_t *chi, double *qt,
                               double *m3inv, int64_t N)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int i1, i2, i3;
    node_coords(p, n1, n2, i1, i2, i3);
    double q[3] = {0, 0, 0}, m = 0;
    if (chi[p]) {
        for (int c = 0; c < hz.cnt; ++c) {
            const int a = (i1 + hz.off[3 * c]) & (n1 - 1);
            const int b = (i2 + hz.off[3 * c + 1]) & (n2 - 1);
            const int e = (i3 + hz.off[3 * c + 2]) & (n3 - 1);
            const int64_t qi = ((int64_t)e * n2 + b) * n1 + a;
            if (!chi[qi]) continue;
            for (int i = 0; i < 3; ++i) q[i] += hz.g[i * hz.cnt + c];
            m += hz.w2[c];
        }
    }
    for (int i = 0; i < 3; ++i) qt[i * N + p] = chi[p] ? q[i] : 0.0;
    m3inv[p] = (chi[p] && m > 0) ? 3.0 / m : 0.0;
}

// Largest eigenvalue over the folded modes of the periodic symbol
//   M(k) = -N mhat(k) + (3 ka / m0) (N ghat)(N ghat)^T   (state-based term only
// when ghat is given), per-block maxima written to out[blockIdx.x].
__global__ void k_lam_max(int dim, const double *mhat, const double *ghat, double kcoef, double Nd,
                          int64_t fold_sz, double *out)
{
    __shared__ double sm[256];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double lm = 0.0;
    if (t < fold_sz) {
        double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (dim == 2) {
            M[0] = -Nd * mhat[t];
            M[4] = -Nd * mhat[fold_sz + t];
            M[1] = M[3] = -Nd * mhat[2 * fold_sz + t];
        } else {
            M[0] = -Nd * mhat[t];
            M[4] = -Nd * mhat[fold_sz + t];
            M[8] = -Nd * mhat[2 * fold_sz + t];
            M[1] = M[3] = -Nd * mhat[3 * fold_sz + t];
            M[2] = M[6] = -Nd * mhat[4 * fold_sz + t];
            M[5] = M[7] = -Nd * mhat[5 * fold_sz + t];
            if (ghat) {
                double gv[3];
                for (int i = 0; i < 3; ++i) gv[i] = Nd * ghat[i * fold_sz + t];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) M[3 * i + j] += kcoef * gv[i] * gv[j];
            }
        }
        if (dim == 2) {
            const double a = M[0], b = M[1], d = M[4];
            const double tr = 0.5 * (a + d), df = 0.5 * (a - d);
            lm = tr + sqrt(df * df + b * b);
        } else {
            // largest eigenvalue of the symmetric 3x3 matrix, closed form
            // (trigonometric solution of the characteristic cubic)
            const double p1 = M[1] * M[1] + M[2] * M[2] + M[5] * M[5];
            const double q = (M[0] + M[4] + M[8]) / 3.0;
            const double a0 = M[0] - q, a4 = M[4] - q, a8 = M[8] - q;
            const double p2 = a0 * a0 + a4 * a4 + a8 * a8 + 2.0 * p1;
            const double pp = sqrt(p2 / 6.0);
            if (pp == 0.0) {
                lm = q;
            } else {
                const double b0 = a0 / pp, b4 = a4 / pp, b8 = a8 / pp;
                const double b1 = M[1] / pp, b2 = M[2] / pp, b5 = M[5] / pp;
                const double det = b0 * (b4 * b8 - b5 * b5) - b1 * (b1 * b8 - b5 * b2) + b2 * (b1 * b5 - b4 * b2);
                const double rr = fmin(1.0, fmax(-1.0, 0.5 * det));
                const double phi = acos(rr) / 3.0;
                lm = q + 2.0 * pp * cos(phi);
            }
        }
    }
    sm[threadIdx.x] = lm;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sm[0];
}

// Packed masks: bit 0 chi_B, bit 1+c chi_Omega of component c.
__global__ void k_mask_bits(const uint8_t *chi, const uint8_t *chi_om, int d, int64_t N, uint8_t *bits)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        unsigned b = chi[p] ? 1u : 0u;
        for (int k = 0; k < d; ++k)
            if (chi_om[k * N + p]) b |= 2u << k;
        bits[p] = (uint8_t)b;
    }
}

// Body must keep delta away from the box faces (§4.2.2) and chi_Omega <= chi_B.
__global__ void k_check_masks(int n1, int n2, int n3, int r1, int r2, int r3, const uint8_t *chi,
                              const uint8_t *chi_om, int d, int64_t N, int *bad)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int i1, i2, i3;
    node_coords(p, n1, n2, i1, i2, i3);
    const uint8_t c = chi[p];
    if (c > 1) atomicOr(bad, 4);
    if (c) {
        if (i1 < r1 || i1 >= n1 - r1 || i2 < r2 || i2 >= n2 - r2 || (n3 > 1 && (i3 < r3 || i3 >= n3 - r3)))
            atomicOr(bad, 1);
    }
    if (chi_om)
        for (int k = 0; k < d; ++k)
            if (chi_om[k * N + p] > c) atomicOr(bad, 2);
}

// Boundary-node list of G: per row, the nodes with chi = 1 and G != 0.
__global__ void k_gcount(int n1, int64_t nrows, const uint8_t *chi, const double *G, int nc, int64_t N, int *cnt)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrows) return;
    int k = 0;
    for (int i = 0; i < n1; ++i) {
        const int64_t p = row * n1 + i;
        if (!chi[p]) continue;
        bool nz = false;
        for (int c = 0; c < nc; ++c) nz |= (G[c * N + p] != 0.0);
        k += nz;
    }
    cnt[row] = k;
}

__global__ void k_gfill(int n1, int64_t nrows, const uint8_t *chi, const double *G, int nc, int64_t N, const int *off,
                        GEntry<double> *e64, GEntry<float> *e32, int *gidx)
{
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrows) return;
    int k = off[row];
    for (int i = 0; i < n1; ++i) {
        const int64_t p = row * n1 + i;
        if (!chi[p]) continue;
        bool nz = false;
        for (int c = 0; c < nc; ++c) nz |= (G[c * N + p] != 0.0);
        if (!nz) continue;
        GEntry<double> a;
        GEntry<float> b;
        for (int c = 0; c < 6; ++c) {
            a.g[c] = c < nc ? G[c * N + p] : 0.0;
            b.g[c] = (float)a.g[c];
        }
        a.p = b.p = p;
        e64[k] = a;
        e32[k] = b;
        gidx[p] = k;
        ++k;
    }
}

// gnode[e] = node of boundary entry e
__global__ void k_gnode(const GEntry<float> *g, int64_t n, int *gnode)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) gnode[e] = (int)g[e].p;
}

// Body moments about the node (c0, c1, c2): Σ chi, Σ chi e_k, Σ chi e_k e_l
// (e = i - c; order S0, e1, e2, e3, 11, 22, 33, 12, 13, 23), block partials.
// The sums are of integers below 2^53, so they are exact in FP64.
__global__ void __launch_bounds__(256) k_body_moments(int n1, int n2, const uint8_t *chi, int c0, int c1, int c2,
                                                      int64_t N, double *part)
{
    double a[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        if (!chi[p]) continue;
        int i1, i2, i3;
        node_coords(p, n1, n2, i1, i2, i3);
        const double e[3] = {(double)(i1 - c0), (double)(i2 - c1), (double)(i3 - c2)};
        a[0] += 1.0;
        for (int k = 0; k < 3; ++k) a[1 + k] += e[k];
        a[4] += e[0] * e[0];
        a[5] += e[1] * e[1];
        a[6] += e[2] * e[2];
        a[7] += e[0] * e[1];
        a[8] += e[0] * e[2];
        a[9] += e[1] * e[2];
    }
    for (int v = 0; v < 10; ++v) {
        const double t = block_sum_d(a[v]);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * 10 + v] = t;
    }
}

// Affine-split moments per boundary entry: M_(q)k = Σ_H chi(x+xi) C_q(xi) dV o_k
// (C_q in Sym order with its quadrature weight, o the integer offset), FP64 sums.
template <typename T>
__global__ void k_aff_table(int n1, int n2, int n3, HorizonDev hz, int nc, int dim, const uint8_t *chi,
                            const GEntry<double> *gent, int64_t ngent, T *tab)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ngent) return;
    const int64_t p = gent[k].p;
    int i1, i2, i3;
    node_coords(p, n1, n2, i1, i2, i3);
    double acc[18];
    for (int v = 0; v < 18; ++v) acc[v] = 0.0;
    for (int c = 0; c < hz.cnt; ++c) {
        const int o[3] = {hz.off[3 * c], hz.off[3 * c + 1], hz.off[3 * c + 2]};
        const int a = (i1 + o[0]) & (n1 - 1), b = (i2 + o[1]) & (n2 - 1), e = (i3 + o[2]) & (n3 - 1);
        if (!chi[((int64_t)e * n2 + b) * n1 + a]) continue;
        for (int q = 0; q < nc; ++q) {
            const double cq = hz.c[(int64_t)q * hz.cnt + c];
            for (int kk = 0; kk < dim; ++kk) acc[q * dim + kk] += cq * (double)o[kk];
        }
    }
    for (int v = 0; v < nc * dim; ++v) tab[k * nc * dim + v] = (T)acc[v];
}

// Nonlinear bond model, per boundary entry: S(a_j, chi) = Σ_H a_j(xi) dV chi(x+xi)
// and S(c, chi) - c^(0) chi = Σ_H c(xi) dV (chi(x+xi) - 1) (both vanish in the
// delta-interior: a is odd, and there every chi(x+xi) = 1)
template <typename T>
__global__ void k_nl_bfields(int n1, int n2, int n3, HorizonDev hz, int dim, const uint8_t *chi,
                             const GEntry<double> *gent, int64_t ngent, T *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ngent) return;
    const int64_t p = gent[k].p;
    int i1, i2, i3;
    node_coords(p, n1, n2, i1, i2, i3);
    double sa[3] = {0, 0, 0}, sc = 0.0;
    for (int c = 0; c < hz.cnt; ++c) {
        const int a = (i1 + hz.off[3 * c]) & (n1 - 1), b = (i2 + hz.off[3 * c + 1]) & (n2 - 1),
                  e = (i3 + hz.off[3 * c + 2]) & (n3 - 1);
        if (chi[((int64_t)e * n2 + b) * n1 + a]) {
            for (int j = 0; j < dim; ++j) sa[j] += hz.g[j * hz.cnt + c];
        } else {
            sc -= hz.cs[c];
        }
    }
    for (int j = 0; j < 3; ++j) out[4 * k + j] = (T)sa[j];
    out[4 * k + 3] = (T)sc;
}

template <typename Tout>
__global__ void k_convert(const double *in, Tout *out, int64_t n)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = (Tout)in[t];
}

static unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace pd

using namespace pd;

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

template <typename P>
pd_status dalloc(pd_plan *p, P **ptr, size_t bytes)
{
    if (bytes == 0) {
        *ptr = nullptr;
        return PD_OK;
    }
    cudaError_t e = cudaMalloc((void **)ptr, bytes);
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        cudaGetLastError();
        return PD_ERR_NOMEM;
    }
    p->bytes += (int64_t)bytes;
    return PD_OK;
}

struct HostHorizon {
    std::vector<int> off;
    std::vector<double> c, g, w2, cs;
    int cnt = 0;
};

// Reach of the family along axis a in cells: offsets with |xi| <= delta
// (tolerance 1e-12 relative on delta^2), or, with partial volumes, every
// offset whose cell the ball of radius delta still covers in part,
// |xi| < delta + h/2.
int family_radius(const pd_problem *pr, int a)
{
    if (pr->volume_rule == 1) return (int)std::floor((pr->delta + 0.5 * pr->dx[0]) / pr->dx[a] * (1.0 - 1e-12));
    return (int)std::floor(pr->delta / pr->dx[a] + 1e-9);
}

// Horizon offsets and per-bond kernel values (omega = 1/|xi|):
//   C_ij = kc xi_i xi_j / |xi|^3 w, g_i = xi_i / |xi| w, omega|xi|^2 w = |xi| w,
// with the bond's quadrature weight w = dV, or beta(|xi|) dV under the linear
// partial-volume rule (Hu, Ha and Bobaru): beta = min(1, (delta + h/2 - |xi|)/h)
// on cubic cells of side h; the weight is part of the kernel, so every
// convolution stays a convolution (§4.1.1).
HostHorizon make_horizon(const pd_plan *p, double kc)
{
    HostHorizon h;
    const int dim = p->dim;
    const bool pv = p->prob.volume_rule == 1;
    const double hc = p->prob.dx[0];
    const double reach = pv ? p->prob.delta + 0.5 * hc : p->prob.delta;
    int r[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) r[a] = family_radius(&p->prob, a);
    const double d2max = pv ? reach * reach * (1.0 - 1e-12) : p->prob.delta * p->prob.delta * (1.0 + 1e-12);
    const double dV = p->dV;
    std::vector<double> xi;
    for (int k = -r[2]; k <= r[2]; ++k)
        for (int j = -r[1]; j <= r[1]; ++j)
            for (int i = -r[0]; i <= r[0]; ++i) {
                if (!i && !j && !k) continue;
                const double x[3] = {i * p->prob.dx[0], j * p->prob.dx[1], dim == 3 ? k * p->prob.dx[2] : 0.0};
                const double s2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
                if (pv ? !(s2 < d2max) : s2 > d2max) continue;
                h.off.push_back(i);
                h.off.push_back(j);
                h.off.push_back(k);
                xi.push_back(x[0]);
                xi.push_back(x[1]);
                xi.push_back(x[2]);
                h.cnt++;
            }
    const int nc = p->ncomp;
    h.c.assign((size_t)nc * h.cnt, 0.0);
    h.g.assign((size_t)3 * h.cnt, 0.0);
    h.w2.assign((size_t)h.cnt, 0.0);
    h.cs.assign((size_t)h.cnt, 0.0);
    const bool nl = p->prob.model == PD_NONLIN_BOND;
    static const int ci[6] = {0, 1, 2, 0, 0, 1}, cj[6] = {0, 1, 2, 1, 2, 2};
    static const int ci2[3] = {0, 1, 0}, cj2[3] = {0, 1, 1};
    for (int c = 0; c < h.cnt; ++c) {
        const double *x = &xi[3 * c];
        const double rr = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        const double w = pv ? dV * std::min(1.0, (reach - rr) / hc) : dV;
        for (int q = 0; q < nc; ++q) {
            const int a = dim == 3 ? ci[q] : ci2[q], b = dim == 3 ? cj[q] : cj2[q];
            h.c[(size_t)q * h.cnt + c] = kc * x[a] * x[b] / (rr * rr * rr) * w;
        }
        // state-based: g_i = omega xi_i w; nonlinear bond model: a_i = kc xi_i / |xi|^3 w
        for (int i = 0; i < 3; ++i) h.g[(size_t)i * h.cnt + c] = nl ? kc * x[i] / (rr * rr * rr) * w : x[i] / rr * w;
        h.w2[c] = rr * w;
        h.cs[c] = kc / (rr * rr * rr) * w;
    }
    return h;
}

}  // namespace

extern "C" {

const char *pd_last_error_detail(void) { return g_err; }

double pd_plan_critical_energy(const pd_plan *p) { return p ? p->wc : 0.0; }

pd_status pd_plan_set_affine_split(pd_plan *p, int on)
{
    if (!p || (on != 0 && on != 1)) {
        set_error("pd_plan_set_affine_split: null plan or value not 0/1");
        return PD_ERR_ARG;
    }
    if (on && (p->prob.model != PD_LIN_BOND || !p->aff_ok)) {
        set_error("pd_plan_set_affine_split: bond model with a body that spans the grid's dimensions only");
        return PD_ERR_ARG;
    }
    p->affine_split = on;
    return PD_OK;
}

pd_status pd_plan_inject_stall(pd_plan *p, int kind)
{
    if (!p || (kind != 0 && kind != 3 && kind != 5)) {
        set_error("pd_plan_inject_stall: null plan or kind not 0 (forward row pass), 3 (inverse row pass) or 5 "
                  "(inverse plane pass)");
        return PD_ERR_ARG;
    }
    const int v = kind + 1;
    PD_CUDA_TRY(cudaMemcpy(p->inject, &v, sizeof(int), cudaMemcpyHostToDevice));
    return PD_OK;
}

const char *pd_status_string(pd_status s)
{
    switch (s) {
        case PD_OK: return "ok";
        case PD_ERR_ARG: return "invalid argument";
        case PD_ERR_SIZE: return "unsupported size";
        case PD_ERR_NOMEM: return "device allocation failed";
        case PD_ERR_CUDA: return "CUDA error";
        case PD_ERR_NOT_CONVERGED: return "not converged";
        case PD_ERR_TIMEOUT: return "device wait timed out";
        case PD_ERR_NONFINITE: return "non-finite value";
    }
    return "unknown status";
}

int64_t pd_plan_workspace_bytes(const pd_plan *p) { return p ? p->bytes : 0; }

pd_status pd_plan_profile(pd_plan *p, int mask)
{
    if (!p) {
        set_error("pd_plan_profile: null plan");
        return PD_ERR_ARG;
    }
    if (p->prof_on && !mask) PD_TRY(prof_harvest(p));
    p->prof_on = mask & ((1 << pd_plan::kKinds) - 1);
    for (int k = 0; k < pd_plan::kKinds; ++k) {
        p->prof_ms[k] = 0.0;
        p->prof_n[k] = 0;
    }
    // cached graphs hold event nodes of the old setting: rebuild on next use
    for (int k = 0; k < 2; ++k)
        if (p->cg_graph[k]) {
            cudaGraphExecDestroy(p->cg_graph[k]);
            p->cg_graph[k] = nullptr;
        }
    p->ev_used = 0;
    p->ev_reserved = 0;
    return PD_OK;
}

pd_status pd_plan_profile_read(pd_plan *p, int kind, double *ms_total, int64_t *launches)
{
    if (!p || kind < 0 || kind >= pd_plan::kKinds) {
        set_error("pd_plan_profile_read: null plan or kind out of range");
        return PD_ERR_ARG;
    }
    PD_TRY(prof_harvest(p));
    if (ms_total) *ms_total = p->prof_ms[kind];
    if (launches) *launches = p->prof_n[kind];
    return PD_OK;
}
int64_t pd_plan_launch_count(const pd_plan *p) { return p ? p->launches : 0; }
int64_t pd_plan_boundary_nodes(const pd_plan *p) { return p ? p->ngent : 0; }

double pd_stable_dt(const pd_plan *p)
{
    if (!p || p->lam_max <= 0 || p->prob.rho <= 0) return 0.0;
    return 2.0 * std::sqrt(p->prob.rho / p->lam_max);
}

void pd_plan_destroy(pd_plan *p)
{
    if (!p) return;
    void *ptrs[] = {p->chi, p->chi_om, p->mbits, p->hoff, p->mhat64, p->mhat32, p->ghat64, p->ghat32, p->G64, p->G32,
                    p->goff, p->gidx, p->gnode, p->gpe, p->gent64, p->gent32, p->aff_tab, p->aff_coef, p->chat64, p->chat32, p->nlb,
                    p->qt64, p->m3inv64, p->qt32, p->m3inv32, p->tw64, p->tw32, p->spec32, p->spec64,
                    p->work, p->red};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (int i = 0; i < 2 * pd_plan::kEvPool; ++i)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    for (int k = 0; k < 2; ++k)
        if (p->cg_graph[k]) cudaGraphExecDestroy(p->cg_graph[k]);
    if (p->host_scal) cudaFreeHost(p->host_scal);
    for (int k = 0; k < 2; ++k)
        if (p->ev_join[k]) cudaEventDestroy(p->ev_join[k]);
    if (p->own_stream) cudaStreamDestroy(p->own_stream);
    if (p->aux_stream) cudaStreamDestroy(p->aux_stream);
    for (int k = 0; k < 2; ++k)
        if (p->ev_fork[k]) cudaEventDestroy(p->ev_fork[k]);
    delete p;
}

static pd_status plan_create_impl(const pd_problem *pr, const uint8_t *chi_B, const uint8_t *chi_Omega,
                                  cudaStream_t st, pd_plan *p);

pd_status pd_plan_create(const pd_problem *pr, const uint8_t *chi_B, const uint8_t *chi_Omega, void *stream,
                         pd_plan **out)
{
    if (!pr || !chi_B || !out) {
        set_error("pd_plan_create: null problem, chi_B or out");
        return PD_ERR_ARG;
    }
    *out = nullptr;
    pd_plan *p = new pd_plan();
    pd_status s = plan_create_impl(pr, chi_B, chi_Omega, (cudaStream_t)stream, p);
    if (s != PD_OK) {
        pd_plan_destroy(p);
        return s;
    }
    *out = p;
    return PD_OK;
}

// Plan-time part of the affine split of pd_force (pd_affine.cuh): the body's
// centre node and the inverse of the normal matrix of the least-squares
// affine fit, the bound on the node offsets, the coefficient buffer and the
// boundary moment table.
static pd_status affine_setup(pd_plan *p, cudaStream_t st)
{
    const int dim = p->dim;
    constexpr int kBlk = 256;
    double *part = p->red;  // free at plan time
    double mom[10];
    auto moments = [&](int c0, int c1, int c2) -> pd_status {
        k_body_moments<<<kBlk, 256, 0, st>>>(p->n1, p->n2, p->chi, c0, c1, c2, p->N, part);
        PD_LAUNCH_CHECK();
        std::vector<double> h((size_t)kBlk * 10);
        PD_CUDA_TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        for (int v = 0; v < 10; ++v) {
            mom[v] = 0.0;
            for (int b = 0; b < kBlk; ++b) mom[v] += h[(size_t)b * 10 + v];
        }
        return PD_OK;
    };
    PD_TRY(moments(0, 0, 0));
    const int n[3] = {p->n1, p->n2, p->n3};
    for (int k = 0; k < 3; ++k) {
        p->aff_c[k] = (k < dim && mom[0] > 0) ? (int)std::lround(mom[1 + k] / mom[0]) : 0;
        p->aff_emax[k] = k < dim ? (double)std::max(p->aff_c[k], n[k] - 1 - p->aff_c[k]) : 0.0;
    }
    PD_TRY(moments(p->aff_c[0], p->aff_c[1], p->aff_c[2]));
    p->body_count = mom[0];
    // normal matrix [[S0, Se^T], [Se, See]] and its inverse (Gauss-Jordan, partial pivoting)
    const int M = dim + 1;
    const int sidx[3][3] = {{4, 7, 8}, {7, 5, 9}, {8, 9, 6}};
    double a[4][8] = {};
    for (int r = 0; r < M; ++r) {
        for (int c = 0; c < M; ++c)
            a[r][c] = (r == 0 && c == 0) ? mom[0] : (r == 0 ? mom[c] : (c == 0 ? mom[r] : mom[sidx[r - 1][c - 1]]));
        a[r][M + r] = 1.0;
    }
    double scale = 0.0;
    for (int r = 0; r < M; ++r) scale = std::max(scale, std::fabs(a[r][r]));
    p->aff_ok = scale > 0 ? 1 : 0;
    for (int c = 0; c < M && p->aff_ok; ++c) {
        int piv = c;
        for (int r = c + 1; r < M; ++r)
            if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
        if (!(std::fabs(a[piv][c]) > 1e-9 * scale)) {
            p->aff_ok = 0;  // the body spans no full-rank affine space (a line or a point)
            break;
        }
        for (int j = 0; j < 2 * M; ++j) std::swap(a[c][j], a[piv][j]);
        const double d = a[c][c];
        for (int j = 0; j < 2 * M; ++j) a[c][j] /= d;
        for (int r = 0; r < M; ++r) {
            if (r == c) continue;
            const double f = a[r][c];
            for (int j = 0; j < 2 * M; ++j) a[r][j] -= f * a[c][j];
        }
    }
    for (int r = 0; r < M; ++r)
        for (int c = 0; c < M; ++c) p->aff_inv[r * M + c] = a[r][M + c];
    PD_TRY(dalloc(p, &p->aff_coef, sizeof(double) * 32));
    PD_CUDA_TRY(cudaMemsetAsync(p->aff_coef, 0, sizeof(double) * 32, st));
    const int nv = p->ncomp * dim;
    const int64_t ng = std::max<int64_t>(p->ngent, 1);
    if (p->prob.fp64) {
        PD_TRY(dalloc(p, &p->aff_tab, sizeof(double) * nv * ng));
        k_aff_table<double><<<nblk(ng, 128), 128, 0, st>>>(p->n1, p->n2, p->n3, p->hdev, p->ncomp, dim, p->chi,
                                                           (const GEntry<double> *)p->gent64, p->ngent,
                                                           (double *)p->aff_tab);
    } else {
        PD_TRY(dalloc(p, &p->aff_tab, sizeof(float) * nv * ng));
        k_aff_table<float><<<nblk(ng, 128), 128, 0, st>>>(p->n1, p->n2, p->n3, p->hdev, p->ncomp, dim, p->chi,
                                                          (const GEntry<double> *)p->gent64, p->ngent,
                                                          (float *)p->aff_tab);
    }
    PD_LAUNCH_CHECK();
    PD_CUDA_TRY(cudaStreamSynchronize(st));
    return PD_OK;
}

static pd_status plan_create_impl(const pd_problem *pr, const uint8_t *chi_B, const uint8_t *chi_Omega,
                                  cudaStream_t st, pd_plan *p)
{
    p->prob = *pr;
    const int dim = pr->dim;
    if (dim != 2 && dim != 3) {
        set_error("dim must be 2 or 3 (got %d)", dim);
        return PD_ERR_ARG;
    }
    if (pr->model != PD_LIN_BOND && pr->model != PD_LIN_STATE && pr->model != PD_NONLIN_BOND) {
        set_error("unknown model %d", pr->model);
        return PD_ERR_ARG;
    }
    if (pr->model == PD_LIN_STATE && dim != 3) {
        set_error("the state-based model is 3D only");
        return PD_ERR_ARG;
    }
    if (!(pr->delta > 0) || !(pr->E > 0)) {
        set_error("delta and E must be positive");
        return PD_ERR_ARG;
    }
    if (pr->model == PD_LIN_STATE && !(pr->nu > -1.0 && pr->nu < 0.5)) {
        set_error("nu must lie in (-1, 0.5)");
        return PD_ERR_ARG;
    }
    const int n1 = pr->n[0], n2 = pr->n[1], n3 = dim == 3 ? pr->n[2] : 1;
    if (!is_pow2(n1) || n1 < 32 || n1 > 2048 || !is_pow2(n2) || n2 < 16 || n2 > 1024 ||
        (dim == 3 && (!is_pow2(n3) || n3 < 16 || n3 > 1024)) || (dim == 2 && pr->n[2] != 1)) {
        set_error("grid %dx%dx%d unsupported: powers of two, 32<=n0<=2048, 16<=n1,n2<=1024, n2=1 in 2D",
                  pr->n[0], pr->n[1], pr->n[2]);
        return PD_ERR_SIZE;
    }
    if (!(pr->s0 >= 0) || (pr->s0 > 0 && pr->model != PD_LIN_BOND)) {
        set_error("s0 must be >= 0, and is defined for the bond model only (got %g)", pr->s0);
        return PD_ERR_ARG;
    }
    if (pr->volume_rule != 0 && pr->volume_rule != 1) {
        set_error("volume_rule must be 0 (constant dV) or 1 (partial volumes), got %d", pr->volume_rule);
        return PD_ERR_ARG;
    }
    int r[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        if (!(pr->dx[a] > 0)) {
            set_error("dx[%d] must be positive", a);
            return PD_ERR_ARG;
        }
        if (pr->volume_rule == 1 && std::fabs(pr->dx[a] - pr->dx[0]) > 1e-12 * pr->dx[0]) {
            set_error("partial volumes need cubic cells (dx[%d] = %g differs from dx[0] = %g)", a, pr->dx[a],
                      pr->dx[0]);
            return PD_ERR_ARG;
        }
        r[a] = family_radius(pr, a);
    }
    if (r[0] < 1 || 2 * r[0] + 2 > n1 || 2 * r[1] + 2 > n2 || (dim == 3 && 2 * r[2] + 2 > n3)) {
        set_error("horizon of %d x %d x %d cells does not fit the grid", r[0], r[1], r[2]);
        return PD_ERR_SIZE;
    }
    p->dim = dim;
    p->n1 = n1;
    p->n2 = n2;
    p->n3 = n3;
    p->h = n1 / 2;
    p->ncomp = dim == 3 ? 6 : 3;
    p->N = (int64_t)n1 * n2 * n3;
    p->nrows = (int64_t)n2 * n3;
    p->lgl = ilog2(std::max(n1, std::max(n2, n3)));
    p->dV = dim == 3 ? pr->dx[0] * pr->dx[1] * pr->dx[2] : pr->dx[0] * pr->dx[1];
    const double d = pr->delta;
    p->nonlinear = pr->model == PD_NONLIN_BOND ? 1 : 0;
    if (pr->model == PD_LIN_BOND || pr->model == PD_NONLIN_BOND) {
        p->alpha = dim == 2 ? 9.0 * pr->E / (M_PI * d * d * d) : 12.0 * pr->E / (M_PI * d * d * d * d);
        p->ka = 0.0;
        p->m0 = 0.0;
    }
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev);
    }

    // horizon and model constants
    HostHorizon hz0 = make_horizon(p, 1.0);
    if (pr->model == PD_LIN_STATE) {
        double m0 = 0.0;
        for (int c = 0; c < hz0.cnt; ++c) m0 += hz0.w2[c];  // Σ omega |xi|^2 dV
        const double kappa = pr->E / (3.0 * (1.0 - 2.0 * pr->nu));
        const double mu = pr->E / (2.0 * (1.0 + pr->nu));
        p->m0 = m0;
        p->alpha = 30.0 * mu / m0;
        // 3 kappa - 5 mu vanishes at nu = 1/4 (the state-based solid is then the
        // bond form); snap rounding residue to an exact zero
        const double dk = 3.0 * kappa - 5.0 * mu;
        p->ka = (std::fabs(dk) <= 1e-12 * (kappa + mu)) ? 0.0 : dk / m0;
    }
    p->state_based = (pr->model == PD_LIN_STATE && p->ka != 0.0) ? 1 : 0;
    HostHorizon hz = make_horizon(p, p->alpha);
    p->hcount = hz.cnt;
    // critical energy density (Eq. 63): given, or that of a fully bonded node
    // under the isotropic stretch u = s0 x, W = 1/2 Σ_H eta.C.eta w with
    // eta = s0 xi, i.e. 1/2 alpha s0^2 Σ_H |xi| w (omega = 1/|xi|; hz0.w2 holds
    // |xi| w, w = the bond's quadrature weight dV or beta dV)
    if (pr->Wc > 0) {
        p->wc = pr->Wc;
    } else if (pr->s0 > 0) {
        double sl = 0.0;
        for (int c = 0; c < hz0.cnt; ++c) sl += hz0.w2[c];
        p->wc = 0.5 * p->alpha * pr->s0 * pr->s0 * sl;
    }

    const int64_t N = p->N;
    const int nc = p->ncomp;
    // masks
    PD_TRY(dalloc(p, &p->chi, (size_t)N));
    PD_TRY(dalloc(p, &p->chi_om, (size_t)N * dim));
    PD_CUDA_TRY(cudaMemcpyAsync(p->chi, chi_B, (size_t)N, cudaMemcpyDeviceToDevice, st));
    for (int k = 0; k < dim; ++k)
        PD_CUDA_TRY(cudaMemcpyAsync(p->chi_om + k * N, chi_Omega ? chi_Omega + k * N : chi_B, (size_t)N,
                                    cudaMemcpyDeviceToDevice, st));
    PD_TRY(dalloc(p, &p->mbits, (size_t)N));
    k_mask_bits<<<1024, 256, 0, st>>>(p->chi, p->chi_om, dim, N, p->mbits);
    PD_LAUNCH_CHECK();
    // horizon tables on device (one buffer: ints, then doubles)
    int *d_off = nullptr;
    double *d_c = nullptr, *d_g = nullptr, *d_w2 = nullptr, *d_cs = nullptr;
    PD_TRY(dalloc(p, &p->hoff, sizeof(int) * 3 * hz.cnt + sizeof(double) * ((size_t)(nc + 5) * hz.cnt) + 64));
    d_off = p->hoff;
    {
        char *base = (char *)p->hoff;
        size_t o = ((sizeof(int) * 3 * hz.cnt) + 15) / 16 * 16;
        d_c = (double *)(base + o);
        d_g = d_c + (size_t)nc * hz.cnt;
        d_w2 = d_g + (size_t)3 * hz.cnt;
        d_cs = d_w2 + (size_t)hz.cnt;
    }
    PD_CUDA_TRY(cudaMemcpyAsync(d_off, hz.off.data(), sizeof(int) * 3 * hz.cnt, cudaMemcpyHostToDevice, st));
    PD_CUDA_TRY(cudaMemcpyAsync(d_c, hz.c.data(), sizeof(double) * nc * hz.cnt, cudaMemcpyHostToDevice, st));
    PD_CUDA_TRY(cudaMemcpyAsync(d_g, hz.g.data(), sizeof(double) * 3 * hz.cnt, cudaMemcpyHostToDevice, st));
    PD_CUDA_TRY(cudaMemcpyAsync(d_w2, hz.w2.data(), sizeof(double) * hz.cnt, cudaMemcpyHostToDevice, st));
    PD_CUDA_TRY(cudaMemcpyAsync(d_cs, hz.cs.data(), sizeof(double) * hz.cnt, cudaMemcpyHostToDevice, st));
    HorizonDev hd{d_off, d_c, d_g, d_w2, p->nonlinear ? d_cs : nullptr, hz.cnt};
    p->hdev = hd;

    // reduction scratch; the last 64 bytes hold the device status word
    PD_TRY(dalloc(p, &p->red, sizeof(double) * 65536));
    p->dev_status = reinterpret_cast<int *>(p->red + 65536 - 8);  // last 64 bytes
    p->inject = p->dev_status + 1;
    PD_CUDA_TRY(cudaMemsetAsync(p->dev_status, 0, 64, st));

    // mask checks
    {
        int *bad = (int *)p->red;
        PD_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
        k_check_masks<<<nblk(N), 256, 0, st>>>(n1, n2, n3, r[0], r[1], r[2], p->chi, chi_Omega ? p->chi_om : nullptr,
                                               dim, N, bad);
        PD_LAUNCH_CHECK();
        int hbad = 0;
        PD_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        if (hbad & 4) {
            set_error("chi_B must hold 0/1 values");
            return PD_ERR_ARG;
        }
        if (hbad & 1) {
            set_error("the body must stay at least delta (delta + h/2 with partial volumes) away from the box faces");
            return PD_ERR_ARG;
        }
        if (hbad & 2) {
            set_error("chi_Omega must be 0 where chi_B is 0");
            return PD_ERR_ARG;
        }
    }

    // folded spectra
    p->fold_sz = (int64_t)(p->h + 1) * (n2 / 2 + 1) * (n3 / 2 + 1);
    const int64_t fs = p->fold_sz;
    PD_TRY(dalloc(p, &p->mhat64, sizeof(double) * nc * fs));
    PD_TRY(dalloc(p, &p->mhat32, sizeof(float) * nc * fs));
    if (pr->model == PD_NONLIN_BOND) {
        PD_TRY(dalloc(p, &p->chat64, sizeof(double) * fs));
        PD_TRY(dalloc(p, &p->chat32, sizeof(float) * fs));
    }
    if (pr->model == PD_LIN_STATE || pr->model == PD_NONLIN_BOND) {
        PD_TRY(dalloc(p, &p->ghat64, sizeof(double) * 3 * fs));
        PD_TRY(dalloc(p, &p->ghat32, sizeof(float) * 3 * fs));
    }
    k_fold_tables<<<nblk(fs, 128), 128, 0, st>>>(dim, n1, n2, n3, p->h, hd, nc, 1.0 / (double)N, p->mhat64,
                                                p->ghat64, fs, p->chat64);
    PD_LAUNCH_CHECK();
    k_convert<float><<<nblk(nc * fs), 256, 0, st>>>(p->mhat64, p->mhat32, nc * fs);
    PD_LAUNCH_CHECK();
    if (p->chat64) {
        k_convert<float><<<nblk(fs), 256, 0, st>>>(p->chat64, p->chat32, fs);
        PD_LAUNCH_CHECK();
    }
    if (p->ghat64) {
        k_convert<float><<<nblk(3 * fs), 256, 0, st>>>(p->ghat64, p->ghat32, 3 * fs);
        PD_LAUNCH_CHECK();
    }

    // symbol bound for the stable time step
    {
        const unsigned nb = nblk(fs, 256);
        double *tmp = nullptr;
        PD_TRY(dalloc(p, &tmp, sizeof(double) * nb));
        const double kcoef = (pr->model == PD_LIN_STATE) ? 3.0 * p->ka / p->m0 : 0.0;
        k_lam_max<<<nb, 256, 0, st>>>(dim, p->mhat64, p->ghat64, kcoef, (double)N, fs, tmp);
        PD_LAUNCH_CHECK();
        std::vector<double> hm(nb);
        PD_CUDA_TRY(cudaMemcpyAsync(hm.data(), tmp, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(tmp);
        p->bytes -= (int64_t)(sizeof(double) * nb);
        p->lam_max = 0;
        for (double v : hm) p->lam_max = std::max(p->lam_max, v);
    }

    // boundary fields
    PD_TRY(dalloc(p, &p->G64, sizeof(double) * nc * N));
    PD_TRY(dalloc(p, &p->G32, sizeof(float) * nc * N));
    k_gfield<double, double, double><<<nblk(N, 128), 128, 0, st>>>(n1, n2, n3, hd, nc, p->chi, (const double *)nullptr,
                                                                 p->G64, N);
    PD_LAUNCH_CHECK();
    k_convert<float><<<nblk(nc * N), 256, 0, st>>>(p->G64, p->G32, nc * N);
    PD_LAUNCH_CHECK();
    {
        // sparse list of the boundary nodes of G, ordered by row
        const int64_t nr = p->nrows;
        PD_TRY(dalloc(p, &p->goff, sizeof(int) * (size_t)(nr + 1)));
        k_gcount<<<nblk(nr, 128), 128, 0, st>>>(n1, nr, p->chi, p->G64, nc, N, p->goff);
        PD_LAUNCH_CHECK();
        std::vector<int> cnt((size_t)nr + 1, 0);
        PD_CUDA_TRY(cudaMemcpyAsync(cnt.data(), p->goff, sizeof(int) * (size_t)nr, cudaMemcpyDeviceToHost, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
        int64_t acc = 0;
        for (int64_t r = 0; r < nr; ++r) {
            const int c = cnt[(size_t)r];
            cnt[(size_t)r] = (int)acc;
            acc += c;
        }
        cnt[(size_t)nr] = (int)acc;
        p->ngent = acc;
        PD_CUDA_TRY(cudaMemcpyAsync(p->goff, cnt.data(), sizeof(int) * (size_t)(nr + 1), cudaMemcpyHostToDevice, st));
        PD_TRY(dalloc(p, &p->gent64, sizeof(GEntry<double>) * (size_t)std::max<int64_t>(acc, 1)));
        PD_TRY(dalloc(p, &p->gent32, sizeof(GEntry<float>) * (size_t)std::max<int64_t>(acc, 1)));
        PD_TRY(dalloc(p, &p->gidx, sizeof(int) * N));
        PD_CUDA_TRY(cudaMemsetAsync(p->gidx, 0xff, sizeof(int) * N, st));  // -1
        k_gfill<<<nblk(nr, 128), 128, 0, st>>>(n1, nr, p->chi, p->G64, nc, N, p->goff, (GEntry<double> *)p->gent64,
                                              (GEntry<float> *)p->gent32, p->gidx);
        PD_LAUNCH_CHECK();
        if (dim == 3 && !pr->fp64 && n1 == n2 && (n1 == 32 || n1 == 64 || n1 == 128)) {
            // FP32 cubes with plane passes: entry -> node, and the per-entry (G p) buffer
            const int64_t ng = std::max<int64_t>(acc, 1);
            PD_TRY(dalloc(p, &p->gnode, sizeof(int) * (size_t)ng));
            PD_TRY(dalloc(p, &p->gpe, sizeof(float) * 3 * (size_t)ng));
            k_gnode<<<nblk(ng, 256), 256, 0, st>>>((const GEntry<float> *)p->gent32, acc, p->gnode);
            PD_LAUNCH_CHECK();
        }
        PD_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (pr->model == PD_LIN_BOND || pr->model == PD_NONLIN_BOND) PD_TRY(affine_setup(p, st));
    if (pr->model == PD_NONLIN_BOND) {
        const int64_t ng = std::max<int64_t>(p->ngent, 1);
        if (pr->fp64) {
            PD_TRY(dalloc(p, &p->nlb, sizeof(double) * 4 * ng));
            k_nl_bfields<double><<<nblk(ng, 128), 128, 0, st>>>(n1, n2, n3, hd, dim, p->chi,
                                                               (const GEntry<double> *)p->gent64, p->ngent,
                                                               (double *)p->nlb);
        } else {
            PD_TRY(dalloc(p, &p->nlb, sizeof(float) * 4 * ng));
            k_nl_bfields<float><<<nblk(ng, 128), 128, 0, st>>>(n1, n2, n3, hd, dim, p->chi,
                                                              (const GEntry<double> *)p->gent64, p->ngent,
                                                              (float *)p->nlb);
        }
        PD_LAUNCH_CHECK();
        PD_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (pr->model == PD_LIN_STATE) {
        PD_TRY(dalloc(p, &p->qt64, sizeof(double) * 3 * N));
        PD_TRY(dalloc(p, &p->m3inv64, sizeof(double) * N));
        PD_TRY(dalloc(p, &p->qt32, sizeof(float) * 3 * N));
        PD_TRY(dalloc(p, &p->m3inv32, sizeof(float) * N));
        k_state_fields<<<nblk(N, 128), 128, 0, st>>>(n1, n2, n3, hd, p->chi, p->qt64, p->m3inv64, N);
        PD_LAUNCH_CHECK();
        k_convert<float><<<nblk(3 * N), 256, 0, st>>>(p->qt64, p->qt32, 3 * N);
        k_convert<float><<<nblk(N), 256, 0, st>>>(p->m3inv64, p->m3inv32, N);
        PD_LAUNCH_CHECK();
    }

    // twiddles e^{-2 pi i k / L}, L = max(n1, n2, n3), from the eighth-turn symmetric
    // evaluation of cos/sin in FP64 on the host
    {
        const int L = 1 << p->lgl;
        std::vector<cx<double>> t64(L);
        std::vector<cx<float>> t32(L);
        for (int k = 0; k < L; ++k) {
            const double a = 2.0 * M_PI * (double)k / (double)L;
            t64[k] = mk(std::cos(a), -std::sin(a));
        }
        // exact values on the axes and diagonals
        for (int k = 0; k < L; k += L / 8) {
            const int o = (8 * k) / L;
            const double r2 = 0.70710678118654752440;
            const double cs[8] = {1, r2, 0, -r2, -1, -r2, 0, r2};
            const double sn[8] = {0, r2, 1, r2, 0, -r2, -1, -r2};
            t64[k] = mk(cs[o], -sn[o]);
        }
        for (int k = 0; k < L; ++k) t32[k] = mk((float)t64[k].x, (float)t64[k].y);
        PD_TRY(dalloc(p, &p->tw64, sizeof(cx<double>) * L));
        PD_TRY(dalloc(p, &p->tw32, sizeof(cx<float>) * L));
        PD_CUDA_TRY(cudaMemcpyAsync(p->tw64, t64.data(), sizeof(cx<double>) * L, cudaMemcpyHostToDevice, st));
        PD_CUDA_TRY(cudaMemcpyAsync(p->tw32, t32.data(), sizeof(cx<float>) * L, cudaMemcpyHostToDevice, st));
        PD_CUDA_TRY(cudaStreamSynchronize(st));
    }

    // timing events and the pinned solver scalars (created here so that later
    // calls allocate nothing)
    for (int i = 0; i < 2 * pd_plan::kEvPool; ++i) PD_CUDA_TRY(cudaEventCreate(&p->ev[i]));
    PD_CUDA_TRY(cudaMallocHost((void **)&p->host_scal, sizeof(double) * 64));
    PD_CUDA_TRY(cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking));
    PD_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_join[0], cudaEventDisableTiming));
    PD_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_join[1], cudaEventDisableTiming));
    PD_CUDA_TRY(cudaStreamCreateWithFlags(&p->aux_stream, cudaStreamNonBlocking));
    PD_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_fork[0], cudaEventDisableTiming));
    PD_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_fork[1], cudaEventDisableTiming));

    // spectra and scratch
    // the 3D nonlinear bond model's last-axis pass reads 12 and writes 21 spectra (out of place)
    const int slots = (pr->model == PD_NONLIN_BOND && dim == 3) ? 33 : kMaxSpecFields;
    if (!pr->fp64) {
        p->spec32_slots = slots;
        PD_TRY(dalloc(p, &p->spec32, sizeof(float) * (size_t)p->spec32_slots * N));
    }
    p->spec64_slots = pr->fp64 ? slots : 8;
    PD_TRY(dalloc(p, &p->spec64, sizeof(double) * (size_t)p->spec64_slots * N));
    {
        const size_t tb = pr->fp64 ? sizeof(double) : sizeof(float);
        const size_t vec = tb * (size_t)dim * N;  // one vector field
        const size_t sizes[] = {vec, vec, vec, vec, tb * (size_t)N, tb * (size_t)nc * N,
                                sizeof(double) * (size_t)dim * N, sizeof(double) * (size_t)N};
        void **slots[] = {&p->cg_e, &p->cg_r, &p->cg_p, &p->cg_q, &p->theta, &p->Gw, (void **)&p->r64,
                          (void **)&p->theta64};
        size_t total = 0;
        for (size_t b : sizes) total += (b + 255) / 256 * 256;
        p->work_bytes = total;
        PD_TRY(dalloc(p, &p->work, total));
        char *base = (char *)p->work;
        for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i) {
            *slots[i] = base;
            base += (sizes[i] + 255) / 256 * 256;
        }
    }
    PD_CUDA_TRY(cudaStreamSynchronize(st));
    return PD_OK;
}

pd_status pd_kernel_spectrum(pd_plan *p, double *out, void *stream)
{
    if (!p || !out) {
        set_error("pd_kernel_spectrum: null plan or output");
        return PD_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    HorizonDev hd = p->hdev;
    const int64_t total = (int64_t)(p->h + 1) * p->n2 * p->n3;
    k_kernel_spectrum<<<nblk(total, 128), 128, 0, st>>>(p->n1, p->n2, p->n3, p->h, hd, p->ncomp, out, total);
    PD_LAUNCH_CHECK();
    p->launches++;
    return PD_OK;
}

}  // extern "C"
