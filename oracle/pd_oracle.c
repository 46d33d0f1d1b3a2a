/*
 * FP64 direct-sum oracle for the FCBM-EC peridynamic operators
 * (Jafarzadeh, Mousavi, Larios, Bobaru, "A general and fast convolution-based
 * method for peridynamics", arXiv 2105.06055).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg call this code; the GPU library never links or calls it and
 * shares nothing with it.
 *
 * What it computes is the plain definition the fast method reorganises: the
 * one-point (mid-point) quadrature of the PD integrals on the uniform periodic
 * grid of Eq. 52, written as a direct sum over the horizon offsets
 * (Eq. 55, first line; §4.1.1), with the embedded-constraint masks of Eq. 75
 * (bond cut chi_B chi_B'), Eq. 92-94 (state-based), Eq. 100-102 (damage).
 * No FFT, no blocking, no reordering: for every node, loop over the horizon
 * and accumulate in FP64.
 *
 * Readings of the paper where it is silent or garbled (named in the comments):
 *   R1  horizon membership |xi| <= delta (Eq. 48), tested as
 *       sum_k (i_k dx_k)^2 <= delta^2 (1 + 1e-12)
 *   R2  the self-bond xi = 0 is excluded (C is singular there)
 *   R3  quadrature weight dV = dx1 dx2 dx3 (§4.1.1); under the partial-volume
 *       rule (or_set_volume_rule(1), §4.1.1 remark on partially covered cells)
 *       each bond's weight is beta(|xi|) dV with the linear rule of Hu, Ha and
 *       Bobaru (PA-HHB in Seleson's 2014 comparison of one-point quadratures):
 *       beta = min(1, (delta + h/2 - |xi|) / h) for |xi| < delta + h/2, cubic
 *       cells of side h; the family is then every offset with beta > 0
 *   R4  the "P u" / "(C*chi) u" term enters with a minus sign: it comes from
 *       (u'_j - u_j) in Eq. 17-18; Eq. 38, 92, 93 print a plus
 *   R5  state-based kernels use the bulk m0 (Eq. 35 over a full horizon); the
 *       dilatation uses the nodal m(x) of Eq. 94
 *   R9  strain energy density is Eq. 47 literally
 *   R11 damage is normalised by the node's initial in-body bond count
 *   R16 neighbour offsets wrap periodically (the box is periodic, §4.1)
 *
 * Layout: fields are component-major, x1 fastest: f[c][i3][i2][i1],
 * node index (i3*n2 + i2)*n1 + i1. In 2D, n3 = 1. Masks are uint8 0/1.
 */
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int cnt;
    int *o;      /* cnt x 3 integer offsets */
    double *xi;  /* cnt x 3 physical offsets */
    double *len; /* |xi| */
    double *vol; /* quadrature weight of the bond relative to dV: 1, or beta(|xi|) */
} horizon_t;

/* 0: constant dV (the paper's examples); 1: linear partial volumes (R3). */
static int g_volume_rule = 0;

/*
 * Horizon offsets: all lattice vectors xi != 0 with |xi| <= delta (R1, R2), or,
 * under the partial-volume rule, with |xi| < delta + h/2, where a cell of side
 * h centred at x + xi is partly covered by the ball of radius delta (R3).
 */
static int build_horizon(int dim, const double *dx, double delta, horizon_t *h)
{
    const int pv = g_volume_rule == 1;
    const double hc = dx[0];
    const double reach = pv ? delta + 0.5 * hc : delta;
    int r[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a)
        r[a] = pv ? (int)floor(reach / dx[a] * (1.0 - 1e-12)) : (int)floor(delta / dx[a] + 1e-9);
    int cap = (2 * r[0] + 1) * (2 * r[1] + 1) * (2 * r[2] + 1);
    h->o = (int *)malloc(sizeof(int) * 3 * cap);
    h->xi = (double *)malloc(sizeof(double) * 3 * cap);
    h->len = (double *)malloc(sizeof(double) * cap);
    h->vol = (double *)malloc(sizeof(double) * cap);
    h->cnt = 0;
    double d2max = pv ? reach * reach * (1.0 - 1e-12) : delta * delta * (1.0 + 1e-12);
    for (int k = -r[2]; k <= r[2]; ++k)
        for (int j = -r[1]; j <= r[1]; ++j)
            for (int i = -r[0]; i <= r[0]; ++i) {
                if (i == 0 && j == 0 && k == 0) continue;
                double x0 = i * dx[0], x1 = j * dx[1], x2 = (dim == 3) ? k * dx[2] : 0.0;
                double d2 = x0 * x0 + x1 * x1 + x2 * x2;
                if (pv ? !(d2 < d2max) : d2 > d2max) continue;
                int c = h->cnt++;
                h->o[3 * c] = i; h->o[3 * c + 1] = j; h->o[3 * c + 2] = k;
                h->xi[3 * c] = x0; h->xi[3 * c + 1] = x1; h->xi[3 * c + 2] = x2;
                h->len[c] = sqrt(d2);
                h->vol[c] = 1.0;
                if (pv) {
                    double b = (reach - h->len[c]) / hc;
                    h->vol[c] = b < 1.0 ? b : 1.0;
                }
            }
    return h->cnt;
}

static void free_horizon(horizon_t *h)
{
    free(h->o); free(h->xi); free(h->len); free(h->vol);
}

static inline int64_t wrap_index(const int *n, int i1, int i2, int i3, const int *o)
{
    int a = i1 + o[0], b = i2 + o[1], c = i3 + o[2];
    a %= n[0]; if (a < 0) a += n[0];
    b %= n[1]; if (b < 0) b += n[1];
    c %= n[2]; if (c < 0) c += n[2];
    return ((int64_t)c * n[1] + b) * n[0] + a;
}

static inline double dvol(int dim, const double *dx)
{
    return dim == 3 ? dx[0] * dx[1] * dx[2] : dx[0] * dx[1];
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Volume rule of every later call: 0 constant dV, 1 linear partial volumes (R3). */
void or_set_volume_rule(int rule)
{
    g_volume_rule = rule == 1 ? 1 : 0;
}

int or_volume_rule(void)
{
    return g_volume_rule;
}

/* Number of horizon offsets, the offsets, lengths and weights (cap entries max). */
int or_horizon(int dim, const double *dx, double delta, int cap, int *off_out, double *len_out, double *vol_out)
{
    horizon_t h;
    int cnt = build_horizon(dim, dx, delta, &h);
    for (int c = 0; c < cnt && c < cap; ++c) {
        off_out[3 * c] = h.o[3 * c];
        off_out[3 * c + 1] = h.o[3 * c + 1];
        off_out[3 * c + 2] = h.o[3 * c + 2];
        if (len_out) len_out[c] = h.len[c];
        if (vol_out) vol_out[c] = h.vol[c];
    }
    free_horizon(&h);
    return cnt;
}

/*
 * Linearized bond-based force with embedded constraint and node weight
 * (Eq. 17-18 with Eq. 75; Eq. 100 when s = lambda):
 *   L_i(x) = chi s Σ_xi chi' s' C_ij(xi) (u_j' - u_j) dV,
 *   C_ij(xi) = alpha omega(|xi|) xi_i xi_j / |xi|^2,  omega = 1/|xi| (§5.1, §5.2).
 * s == NULL means s = 1. alpha is the bond constant (9E/(pi delta^3) in 2D
 * plane stress, §5.2). Primes denote values at x + xi, wrapped periodically.
 */
void or_force_bond(int dim, const int *n, const double *dx, double delta, double alpha,
                   const uint8_t *chi, const double *s, const double *u, double *L)
{
    horizon_t h;
    build_horizon(dim, dx, delta, &h);
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    const double dV = dvol(dim, dx);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int i1 = (int)(p % n[0]), i2 = (int)((p / n[0]) % n[1]), i3 = (int)(p / ((int64_t)n[0] * n[1]));
        double acc[3] = {0, 0, 0};
        double wx = chi[p] * (s ? s[p] : 1.0);
        if (wx != 0.0) {
            for (int c = 0; c < h.cnt; ++c) {
                int64_t q = wrap_index(n, i1, i2, i3, &h.o[3 * c]);
                double wq = chi[q] * (s ? s[q] : 1.0);
                if (wq == 0.0) continue;
                const double *xi = &h.xi[3 * c];
                double r = h.len[c];
                double coef = alpha * (1.0 / r) / (r * r) * wq * h.vol[c]; /* alpha omega / |xi|^2 */
                double xe = 0.0;                                 /* xi . eta */
                for (int j = 0; j < dim; ++j) xe += xi[j] * (u[j * N + q] - u[j * N + p]);
                for (int i = 0; i < dim; ++i) acc[i] += coef * xi[i] * xe;
            }
        }
        for (int i = 0; i < dim; ++i) L[i * N + p] = wx * acc[i] * dV;
    }
    free_horizon(&h);
}

/*
 * The same sum at selected nodes only (for checks on grids too large for a
 * full evaluation): L[i * nsel + k] = L_i(nodes[k]).
 */
void or_force_bond_at(int dim, const int *n, const double *dx, double delta, double alpha,
                      const uint8_t *chi, const double *u, const int64_t *nodes, int64_t nsel, double *L)
{
    horizon_t h;
    build_horizon(dim, dx, delta, &h);
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    const double dV = dvol(dim, dx);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nsel; ++k) {
        const int64_t p = nodes[k];
        int i1 = (int)(p % n[0]), i2 = (int)((p / n[0]) % n[1]), i3 = (int)(p / ((int64_t)n[0] * n[1]));
        double acc[3] = {0, 0, 0};
        if (chi[p]) {
            for (int c = 0; c < h.cnt; ++c) {
                int64_t q = wrap_index(n, i1, i2, i3, &h.o[3 * c]);
                if (!chi[q]) continue;
                const double *xi = &h.xi[3 * c];
                double r = h.len[c];
                double coef = alpha * (1.0 / r) / (r * r) * h.vol[c];
                double xe = 0.0;
                for (int j = 0; j < dim; ++j) xe += xi[j] * (u[j * N + q] - u[j * N + p]);
                for (int i = 0; i < dim; ++i) acc[i] += coef * xi[i] * xe;
            }
        }
        for (int i = 0; i < dim; ++i) L[i * nsel + k] = chi[p] * acc[i] * dV;
    }
    free_horizon(&h);
}

/*
 * Strain energy density of the linearized bond model with bond breaking
 * (Eq. 47, EC form Eq. 102):  W(x) = 1/2 chi lam Σ_xi chi' lam' eta.C(xi).eta dV.
 * lam == NULL means lam = 1.
 */
void or_energy_bond(int dim, const int *n, const double *dx, double delta, double alpha,
                    const uint8_t *chi, const uint8_t *lam, const double *u, double *W)
{
    horizon_t h;
    build_horizon(dim, dx, delta, &h);
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    const double dV = dvol(dim, dx);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int i1 = (int)(p % n[0]), i2 = (int)((p / n[0]) % n[1]), i3 = (int)(p / ((int64_t)n[0] * n[1]));
        double acc = 0.0;
        int wx = chi[p] && (lam ? lam[p] : 1);
        if (wx) {
            for (int c = 0; c < h.cnt; ++c) {
                int64_t q = wrap_index(n, i1, i2, i3, &h.o[3 * c]);
                if (!(chi[q] && (lam ? lam[q] : 1))) continue;
                const double *xi = &h.xi[3 * c];
                double r = h.len[c];
                double xe = 0.0;
                for (int j = 0; j < dim; ++j) xe += xi[j] * (u[j * N + q] - u[j * N + p]);
                acc += alpha * (1.0 / r) / (r * r) * h.vol[c] * xe * xe; /* eta.C.eta */
            }
        }
        W[p] = 0.5 * acc * dV;
    }
    free_horizon(&h);
}

/*
 * W of Eq. 47 with a real node weight s in place of the integrity index
 * (bond factor s s' instead of lam lam', Eq. 44; reading R17 for a spatially
 * varying micromodulus c = c0 s^2):
 *   W(x) = 1/2 chi s Σ_xi chi' s' eta.C(xi).eta dV.
 */
void or_energy_bond_w(int dim, const int *n, const double *dx, double delta, double alpha,
                      const uint8_t *chi, const double *s, const double *u, double *W)
{
    horizon_t h;
    build_horizon(dim, dx, delta, &h);
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    const double dV = dvol(dim, dx);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int i1 = (int)(p % n[0]), i2 = (int)((p / n[0]) % n[1]), i3 = (int)(p / ((int64_t)n[0] * n[1]));
        double acc = 0.0;
        if (chi[p]) {
            for (int c = 0; c < h.cnt; ++c) {
                int64_t q = wrap_index(n, i1, i2, i3, &h.o[3 * c]);
                if (!chi[q]) continue;
                const double *xi = &h.xi[3 * c];
                double r = h.len[c];
                double xe = 0.0;
                for (int j = 0; j < dim; ++j) xe += xi[j] * (u[j * N + q] - u[j * N + p]);
                acc += s[q] * alpha * (1.0 / r) / (r * r) * h.vol[c] * xe * xe;
            }
        }
        W[p] = 0.5 * s[p] * acc * dV;
    }
    free_horizon(&h);
}

/*
 * Nonlinear, rotation-invariant bond model (§3.2, Eq. 19-22) with the
 * embedded-constraint cut (Eq. 75) and a bond factor lam lam' (Eq. 44):
 *   f(xi, eta) = alpha omega |xi| (s + 3/2 s^2 + 1/2 s^3) (xi + eta)/|xi + eta|,
 *   s = (|xi + eta| - |xi|)/|xi|        (bond strain, Eq. 20),
 * which the paper rewrites (Eq. 21) as
 *   f = c(xi)/2 (|xi + eta|^2 - |xi|^2)(xi + eta),  c = alpha omega / |xi|^2,
 * a polynomial in eta (the form summed here, no square roots of |xi + eta|).
 *   L(x) = chi lam Σ_xi chi' lam' f(xi, u' - u) dV.
 * lam == NULL means lam = 1. omega = 1/|xi|.
 */
void or_force_nl(int dim, const int *n, const double *dx, double delta, double alpha,
                 const uint8_t *chi, const uint8_t *lam, const double *u, double *L)
{
    horizon_t h;
    build_horizon(dim, dx, delta, &h);
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    const double dV = dvol(dim, dx);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int i1 = (int)(p % n[0]), i2 = (int)((p / n[0]) % n[1]), i3 = (int)(p / ((int64_t)n[0] * n[1]));
        double acc[3] = {0, 0, 0};
        int wx = chi[p] && (lam ? lam[p] : 1);
        if (wx) {
            for (int c = 0; c < h.cnt; ++c) {
                int64_t q = wrap_index(n, i1, i2, i3, &h.o[3 * c]);
                if (!(chi[q] && (lam ? lam[q] : 1))) continue;
                const double *xi = &h.xi[3 * c];
                double r = h.len[c];
                double cc = alpha * (1.0 / r) / (r * r) * h.vol[c];
                double y[3] = {0, 0, 0}, yy = 0.0; /* y = xi + eta */
                for (int j = 0; j < dim; ++j) {
                    y[j] = xi[j] + (u[j * N + q] - u[j * N + p]);
                    yy += y[j] * y[j];
                }
                double g = 0.5 * cc * (yy - r * r);
                for (int i = 0; i < dim; ++i) acc[i] += g * y[i];
            }
        }
        for (int i = 0; i < dim; ++i) L[i * N + p] = wx * acc[i] * dV;
    }
    free_horizon(&h);
}

/*
 * Energy density of the same model: f is the gradient in eta of the pairwise
 * potential w(xi, eta) = c/8 (|xi + eta|^2 - |xi|^2)^2, and
 *   W(x) = chi lam Σ_xi chi' lam' w(xi, u' - u) dV,
 * which for small eta is 1/2 Σ eta.C.eta dV, the density of Eq. 47 (R9).
 */
void or_energy_nl(int dim, const int *n, const double *dx, double delta, double alpha,
                  const uint8_t *chi, const uint8_t *lam, const double *u, double *W)
{
    horizon_t h;
    build_horizon(dim, dx, delta, &h);
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    const double dV = dvol(dim, dx);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int i1 = (int)(p % n[0]), i2 = (int)((p / n[0]) % n[1]), i3 = (int)(p / ((int64_t)n[0] * n[1]));
        double acc = 0.0;
        int wx = chi[p] && (lam ? lam[p] : 1);
        if (wx) {
            for (int c = 0; c < h.cnt; ++c) {
                int64_t q = wrap_index(n, i1, i2, i3, &h.o[3 * c]);
                if (!(chi[q] && (lam ? lam[q] : 1))) continue;
                const double *xi = &h.xi[3 * c];
                double r = h.len[c];
                double cc = alpha * (1.0 / r) / (r * r) * h.vol[c];
                double yy = 0.0;
                for (int j = 0; j < dim; ++j) {
                    double yj = xi[j] + (u[j * N + q] - u[j * N + p]);
                    yy += yj * yj;
                }
                double d = yy - r * r;
                acc += 0.125 * cc * d * d;
            }
        }
        W[p] = acc * dV;
    }
    free_horizon(&h);
}

/*
 * Broken-bond count and damage index (Eq. 12 with mu = lam lam' (Eq. 44) and the
 * bond cut of Eq. 75; reading R11):
 *   beta(x) = chi Σ_xi chi'           (initial in-body bonds, integer)
 *   nb(x)   = chi Σ_xi chi' (1 - lam lam')
 *   d(x)    = nb / beta   (0 where beta = 0)
 * The sums run over the family; under the partial-volume rule a partly covered
 * bond still counts as one bond (the counts are integers).
 */
void or_damage(int dim, const int *n, const double *dx, double delta,
               const uint8_t *chi, const uint8_t *lam, int32_t *nb, int32_t *beta, double *d)
{
    horizon_t h;
    build_horizon(dim, dx, delta, &h);
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int i1 = (int)(p % n[0]), i2 = (int)((p / n[0]) % n[1]), i3 = (int)(p / ((int64_t)n[0] * n[1]));
        int b = 0, k = 0;
        if (chi[p]) {
            for (int c = 0; c < h.cnt; ++c) {
                int64_t q = wrap_index(n, i1, i2, i3, &h.o[3 * c]);
                if (!chi[q]) continue;
                ++b;
                if (!(lam[p] && lam[q])) ++k;
            }
        }
        if (nb) nb[p] = k;
        if (beta) beta[p] = b;
        if (d) d[p] = b ? (double)k / (double)b : 0.0;
    }
    free_horizon(&h);
}

/*
 * Linearized state-based (LPS) solid with embedded constraint, 3D
 * (Eq. 33-39 with the chi_B cut of Eq. 92-94; readings R4, R5):
 *   m(x)   = chi Σ chi' omega |xi|^2 dV                                   (Eq. 94)
 *   th(x)  = (3 chi / m) Σ chi' omega xi.(u' - u) dV     (0 where m = 0)   (Eq. 93)
 *   L_i(x) = chi Σ chi' [ ka omega xi_i (th + th')
 *                         + cb omega xi_i xi_j / |xi|^2 (u_j' - u_j) ] dV (Eq. 36, 92)
 * with ka = (3 kappa - 5 mu)/m0 and cb = 30 mu / m0 (Eq. 37).
 * theta and m may be NULL; when given they receive th and m.
 */
void or_force_lps(const int *n, const double *dx, double delta, double ka, double cb,
                  const uint8_t *chi, const double *u, double *L, double *theta_out, double *m_out)
{
    const int dim = 3;
    horizon_t h;
    build_horizon(dim, dx, delta, &h);
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    const double dV = dvol(dim, dx);
    double *th = (double *)calloc((size_t)N, sizeof(double));
    double *mm = (double *)calloc((size_t)N, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int i1 = (int)(p % n[0]), i2 = (int)((p / n[0]) % n[1]), i3 = (int)(p / ((int64_t)n[0] * n[1]));
        double msum = 0.0, tsum = 0.0;
        if (chi[p]) {
            for (int c = 0; c < h.cnt; ++c) {
                int64_t q = wrap_index(n, i1, i2, i3, &h.o[3 * c]);
                if (!chi[q]) continue;
                const double *xi = &h.xi[3 * c];
                double r = h.len[c], om = 1.0 / r;
                msum += om * r * r * h.vol[c];
                double xe = 0.0;
                for (int j = 0; j < dim; ++j) xe += xi[j] * (u[j * N + q] - u[j * N + p]);
                tsum += om * xe * h.vol[c];
            }
        }
        mm[p] = chi[p] ? msum * dV : 0.0;
        th[p] = (chi[p] && mm[p] > 0.0) ? 3.0 / mm[p] * tsum * dV : 0.0;
    }
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int i1 = (int)(p % n[0]), i2 = (int)((p / n[0]) % n[1]), i3 = (int)(p / ((int64_t)n[0] * n[1]));
        double acc[3] = {0, 0, 0};
        if (chi[p]) {
            for (int c = 0; c < h.cnt; ++c) {
                int64_t q = wrap_index(n, i1, i2, i3, &h.o[3 * c]);
                if (!chi[q]) continue;
                const double *xi = &h.xi[3 * c];
                double r = h.len[c], om = 1.0 / r;
                double xe = 0.0;
                for (int j = 0; j < dim; ++j) xe += xi[j] * (u[j * N + q] - u[j * N + p]);
                for (int i = 0; i < dim; ++i)
                    acc[i] += h.vol[c] * (ka * om * xi[i] * (th[p] + th[q]) + cb * om * xi[i] * xe / (r * r));
            }
        }
        for (int i = 0; i < dim; ++i) L[i * N + p] = chi[p] ? acc[i] * dV : 0.0;
    }
    if (theta_out) memcpy(theta_out, th, sizeof(double) * (size_t)N);
    if (m_out) memcpy(m_out, mm, sizeof(double) * (size_t)N);
    free(th);
    free(mm);
    free_horizon(&h);
}

/*
 * Gradient of J = Σ_x p(x).L(x) with respect to the node weight s of the bond
 * model above (the paper has no adjoint; this follows from differentiating the
 * direct sum of Eq. 17-18, 75 with the bond factor s s'):
 *   dJ/ds(y) = chi(y) Σ_xi chi' s' C_ij(xi) (p_i(y) - p_i(y+xi)) (u_j(y+xi) - u_j(y)) dV
 * The gradient with respect to u is the operator itself applied to p (the
 * operator is symmetric), so it needs no routine of its own.
 */
void or_force_bond_grad_s(int dim, const int *n, const double *dx, double delta, double alpha,
                          const uint8_t *chi, const double *s, const double *u, const double *pvec,
                          double *gs)
{
    horizon_t h;
    build_horizon(dim, dx, delta, &h);
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    const double dV = dvol(dim, dx);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < N; ++p) {
        int i1 = (int)(p % n[0]), i2 = (int)((p / n[0]) % n[1]), i3 = (int)(p / ((int64_t)n[0] * n[1]));
        double acc = 0.0;
        if (chi[p]) {
            for (int c = 0; c < h.cnt; ++c) {
                int64_t q = wrap_index(n, i1, i2, i3, &h.o[3 * c]);
                double wq = chi[q] * (s ? s[q] : 1.0);
                if (wq == 0.0) continue;
                const double *xi = &h.xi[3 * c];
                double r = h.len[c];
                double coef = alpha * (1.0 / r) / (r * r) * wq * h.vol[c];
                double xu = 0.0, xp = 0.0;
                for (int j = 0; j < dim; ++j) {
                    xu += xi[j] * (u[j * N + q] - u[j * N + p]);
                    xp += xi[j] * (pvec[j * N + p] - pvec[j * N + q]);
                }
                acc += coef * xp * xu;
            }
        }
        gs[p] = chi[p] ? acc * dV : 0.0;
    }
    free_horizon(&h);
}

/*
 * Fourier symbol of the periodic bond operator (chi = 1, s = 1), from Eq. 57:
 * for u = Re(a e^{i 2 pi k.x/N}) the direct sum gives L = -M(k) u with
 *   M_ij(k) = dV Σ_xi C_ij(xi) (1 - cos(2 pi Σ_a k_a o_a / n_a)).
 * Used by the tests as a closed form for single-mode displacements.
 */
void or_symbol_bond(int dim, const int *n, const double *dx, double delta, double alpha,
                    const double *k, double *M)
{
    horizon_t h;
    build_horizon(dim, dx, delta, &h);
    const double dV = dvol(dim, dx);
    for (int i = 0; i < 9; ++i) M[i] = 0.0;
    for (int c = 0; c < h.cnt; ++c) {
        double ph = 0.0;
        for (int a = 0; a < dim; ++a) ph += k[a] * h.o[3 * c + a] / (double)n[a];
        double w = 1.0 - cos(2.0 * M_PI * ph);
        double r = h.len[c];
        double coef = alpha * (1.0 / r) / (r * r) * w * h.vol[c] * dV;
        for (int i = 0; i < dim; ++i)
            for (int j = 0; j < dim; ++j) M[3 * i + j] += coef * h.xi[3 * c + i] * h.xi[3 * c + j];
    }
    free_horizon(&h);
}
