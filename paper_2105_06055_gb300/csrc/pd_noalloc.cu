// pd_force2d_noalloc: a 2D FP32 force evaluation that allocates no memory.
//
// Who needs it: callers that must not call cudaMalloc at all -- for example
// code running inside a host framework that owns every device allocation
// through its own pool (and forbids the CUDA allocator), a real-time loop that
// may not hit the allocator's locks and device synchronisation, or a
// plug-in loaded where device memory is capped at what its host handed out.
// They cannot create a pd_plan (pd_plan_create allocates the spectra,
// kernel tables and boundary fields), so this entry point runs the same 2D
// bond-model FFT-convolution passes as pd_force with every intermediate in
// one file-scope device array, g_pd_noalloc_scratch, of fixed size. The
// caller still passes chi_B, u and L.
//
// Scratch: kScratchBytes (2 MiB) of __device__ memory, held by every GPU that
// loads the library until the process exits. It fits grids with
// n0 n1 <= 65536 nodes and horizons of at most 512 bonds. On each device the
// first call looks up the array's device address with cudaGetSymbolAddress
// (host code cannot use the symbol itself: on the host it names a stand-in
// object, not device memory); make that first call before any stream capture.
// Every call recomputes everything it reads from the array (horizon table,
// kernel spectrum, boundary field, twiddles, spectra), so nothing depends on
// the previous call's contents; the only values that must start at zero, the
// mask-check flag and the passes' wait-status word, are cleared at the start of
// each call. The call reads the mask-check flag back to the host, so it
// synchronises `stream` once before it enqueues the force passes (a wrong mask
// is then an argument error, not a device fault). All calls share the
// one array: calls that overlap on the GPU (other streams, other host
// threads) race on it and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "pd_force_impl.cuh"

namespace {
constexpr size_t kScratchBytes = size_t(2) << 20;
constexpr int64_t kMaxNodes = 65536;
constexpr int kMaxBonds = 512;
}  // namespace

static __device__ __align__(256) unsigned char g_pd_noalloc_scratch[kScratchBytes];

namespace pd {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
void *g_na_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
pd_status na_scratch(unsigned char **out)
{
    int dev = 0;
    PD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("pd_force2d_noalloc: device ordinal %d out of range", dev);
        return PD_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_pd_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            set_error("pd_force2d_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return PD_ERR_CUDA;
        }
        g_na_ptr[dev] = ptr;
    }
    *out = (unsigned char *)g_na_ptr[dev];
    return PD_OK;
}

// Horizon offsets and C_ij dV per bond (2D order 11, 22, 12), in the same
// order as pd_plan_create: rows of x2 offsets, x1 fastest.
__global__ void k_na_horizon(int r1, int r2, double dx1, double dx2, double delta, double alpha, double dV,
                             int *off, double *c, int cnt)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const double d2max = delta * delta * (1.0 + 1e-12);
    int k = 0;
    for (int j = -r2; j <= r2; ++j)
        for (int i = -r1; i <= r1; ++i) {
            if (!i && !j) continue;
            const double x0 = i * dx1, x1 = j * dx2;
            const double s2 = x0 * x0 + x1 * x1;
            if (s2 > d2max) continue;
            const double r = sqrt(s2);
            off[3 * k] = i;
            off[3 * k + 1] = j;
            off[3 * k + 2] = 0;
            const double a = alpha / (r * r * r) * dV;
            c[k] = a * x0 * x0;
            c[cnt + k] = a * x1 * x1;
            c[2 * cnt + k] = a * x0 * x1;
            ++k;
        }
}

// Folded difference spectrum (K^(k) - K^(0)) / N in FP32, FP64 accumulation.
__global__ void k_na_fold(int n1, int n2, int h, const int *off, const double *c, int cnt, double invN,
                          float *mhat, int64_t fold_sz)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= fold_sz) return;
    const int kx = (int)(t % (h + 1));
    const int ky = (int)(t / (h + 1));
    const int nmax = max(n1, n2);
    double acc[3] = {0, 0, 0};
    for (int b = 0; b < cnt; ++b) {
        long long num = (long long)kx * off[3 * b] * (nmax / n1) + (long long)ky * off[3 * b + 1] * (nmax / n2);
        num %= nmax;
        if (num < 0) num += nmax;
        const double sh = sinpi((double)num / (double)nmax);
        const double omc = 2.0 * sh * sh;  // 1 - cos(theta)
        for (int q = 0; q < 3; ++q) acc[q] -= c[q * cnt + b] * omc;
    }
    for (int q = 0; q < 3; ++q) mhat[q * fold_sz + t] = (float)(acc[q] * invN);
}

__global__ void k_na_twiddle(cx<float> *tw, int L)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)L, &s, &c);
    tw[k] = mk((float)c, (float)-s);
}

// The body must stay delta away from the box faces and chi must be 0/1.
__global__ void k_na_check(int n1, int n2, int r1, int r2, const uint8_t *chi, int64_t N, int *bad)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int i1 = (int)(p % n1), i2 = (int)(p / n1);
    const uint8_t v = chi[p];
    if (v > 1) atomicOr(bad, 2);
    if (v && (i1 < r1 || i1 >= n1 - r1 || i2 < r2 || i2 >= n2 - r2)) atomicOr(bad, 1);
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace pd

using namespace pd;

extern "C" pd_status pd_force2d_noalloc(const pd_problem *pr, const uint8_t *chi_B, const float *u, float *L,
                                        void *stream)
{
    if (!pr || !chi_B || !u || !L) {
        set_error("pd_force2d_noalloc: null problem, chi_B, u or L");
        return PD_ERR_ARG;
    }
    if (pr->dim != 2 || pr->model != PD_LIN_BOND || pr->fp64 != 0) {
        set_error("pd_force2d_noalloc: 2D bond model in FP32 only");
        return PD_ERR_ARG;
    }
    const int n1 = pr->n[0], n2 = pr->n[1];
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (!pow2(n1) || !pow2(n2) || n1 < 32 || n1 > 2048 || n2 < 16 || n2 > 1024 || pr->n[2] != 1) {
        set_error("pd_force2d_noalloc: grid %dx%d unsupported (powers of two, 32<=n0<=2048, 16<=n1<=1024)", n1,
                  n2);
        return PD_ERR_SIZE;
    }
    const int64_t N = (int64_t)n1 * n2;
    if (N > kMaxNodes) {
        set_error("pd_force2d_noalloc: %lld nodes exceed the fixed scratch limit of %lld nodes (%zu bytes); "
                  "use pd_plan_create + pd_force",
                  (long long)N, (long long)kMaxNodes, kScratchBytes);
        return PD_ERR_SIZE;
    }
    if (!(pr->delta > 0) || !(pr->E > 0) || !(pr->dx[0] > 0) || !(pr->dx[1] > 0)) {
        set_error("pd_force2d_noalloc: delta, E and dx must be positive");
        return PD_ERR_ARG;
    }
    if (pr->volume_rule != 0) {
        set_error("pd_force2d_noalloc: constant dV only (volume_rule 0); use pd_plan_create for partial volumes");
        return PD_ERR_ARG;
    }
    const int r1 = (int)std::floor(pr->delta / pr->dx[0] + 1e-9), r2 = (int)std::floor(pr->delta / pr->dx[1] + 1e-9);
    if (r1 < 1 || 2 * r1 + 2 > n1 || 2 * r2 + 2 > n2) {
        set_error("pd_force2d_noalloc: horizon of %d x %d cells does not fit the grid", r1, r2);
        return PD_ERR_SIZE;
    }
    // bond count (same membership rule as pd_plan_create)
    int cnt = 0;
    {
        const double d2max = pr->delta * pr->delta * (1.0 + 1e-12);
        for (int j = -r2; j <= r2; ++j)
            for (int i = -r1; i <= r1; ++i) {
                if (!i && !j) continue;
                const double x0 = i * pr->dx[0], x1 = j * pr->dx[1];
                if (x0 * x0 + x1 * x1 <= d2max) ++cnt;
            }
    }
    if (cnt > kMaxBonds) {
        set_error("pd_force2d_noalloc: %d bonds exceed the limit of %d", cnt, kMaxBonds);
        return PD_ERR_SIZE;
    }
    const int h = n1 / 2;
    const int64_t fold = (int64_t)(h + 1) * (n2 / 2 + 1);
    const int lgl = ilog2(std::max(n1, n2));
    const int L2 = 1 << lgl;
    // carve the scratch array
    const size_t b_spec = up256(sizeof(float) * 2 * (size_t)N);  // two packed spectra (2D pass is in place)
    const size_t b_G = up256(sizeof(float) * 3 * (size_t)N);
    const size_t b_mh = up256(sizeof(float) * 3 * (size_t)fold);
    const size_t b_tw = up256(sizeof(cx<float>) * (size_t)L2);
    const size_t b_off = up256(sizeof(int) * 3 * (size_t)cnt);
    const size_t b_c = up256(sizeof(double) * 3 * (size_t)cnt);
    const size_t b_flag = 256;
    const size_t need = b_spec + b_G + b_mh + b_tw + b_off + b_c + b_flag;
    if (need > kScratchBytes) {
        set_error("pd_force2d_noalloc: needs %zu scratch bytes, the fixed array has %zu", need, kScratchBytes);
        return PD_ERR_SIZE;
    }
    unsigned char *base = nullptr;
    PD_TRY(na_scratch(&base));
    float *spec = (float *)base;
    float *G = (float *)(base + b_spec);
    float *mh = (float *)(base + b_spec + b_G);
    cx<float> *tw = (cx<float> *)(base + b_spec + b_G + b_mh);
    int *off = (int *)(base + b_spec + b_G + b_mh + b_tw);
    double *cc = (double *)(base + b_spec + b_G + b_mh + b_tw + b_off);
    int *flag = (int *)(base + b_spec + b_G + b_mh + b_tw + b_off + b_c);

    cudaStream_t st = (cudaStream_t)stream;
    PD_CUDA_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
    k_na_check<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(n1, n2, r1, r2, chi_B, N, flag);
    PD_LAUNCH_CHECK();
    int hbad = 0;
    PD_CUDA_TRY(cudaMemcpyAsync(&hbad, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    PD_CUDA_TRY(cudaStreamSynchronize(st));
    if (hbad) {
        set_error(hbad & 2 ? "pd_force2d_noalloc: chi_B must hold 0/1 values"
                           : "pd_force2d_noalloc: the body must stay at least delta away from the box faces");
        return PD_ERR_ARG;
    }

    const double dV = pr->dx[0] * pr->dx[1];
    const double alpha = 9.0 * pr->E / (M_PI * pr->delta * pr->delta * pr->delta);
    k_na_horizon<<<1, 32, 0, st>>>(r1, r2, pr->dx[0], pr->dx[1], pr->delta, alpha, dV, off, cc, cnt);
    k_na_fold<<<(unsigned)((fold + 127) / 128), 128, 0, st>>>(n1, n2, h, off, cc, cnt, 1.0 / (double)N, mh, fold);
    k_na_twiddle<<<(L2 + 255) / 256, 256, 0, st>>>(tw, L2);
    PD_LAUNCH_CHECK();
    HorizonDev hd{off, cc, nullptr, nullptr, nullptr, cnt};
    k_gfield<float, double, double><<<(unsigned)((N + 127) / 128), 128, 0, st>>>(n1, n2, 1, hd, 3, chi_B,
                                                                               (const double *)nullptr, G, N);
    PD_LAUNCH_CHECK();

    // a plan description on the host stack pointing into the scratch array
    pd_plan p;
    p.prob = *pr;
    p.dim = 2;
    p.n1 = n1;
    p.n2 = n2;
    p.n3 = 1;
    p.h = h;
    p.ncomp = 3;
    p.N = N;
    p.nrows = n2;
    p.lgl = lgl;
    p.dV = dV;
    p.alpha = alpha;
    p.ka = 0.0;
    p.m0 = 0.0;
    p.lam_max = 0.0;
    p.state_based = 0;
    p.hcount = cnt;
    p.chi = const_cast<uint8_t *>(chi_B);
    p.mhat32 = mh;
    p.fold_sz = fold;
    p.G32 = G;
    p.tw32 = tw;
    p.spec32 = spec;
    p.spec32_slots = 2;
    p.dev_status = flag + 1;
    p.hdev = hd;
    {
        // persistent row-pass grids are sized by the SM count (a query, no allocation)
        int dev = 0;
        PD_CUDA_TRY(cudaGetDevice(&dev));
        PD_CUDA_TRY(cudaDeviceGetAttribute(&p.nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    const pd_status s = force_bond_pipeline<float, 2, false, W_NONE, false>(&p, u, nullptr, nullptr, G, L, nullptr, st);
    // the stack plan owns nothing: detach its views before it goes out of scope
    p.chi = nullptr;
    p.mhat32 = nullptr;
    p.G32 = nullptr;
    p.tw32 = nullptr;
    p.spec32 = nullptr;
    return s;
}
