/*
 * pd.h -- C ABI of the GB300 FCBM-EC peridynamics library.
 *
 * The library evaluates the peridynamic (PD) internal-force operator of the
 * fast convolution-based method with embedded constraint (FCBM-EC;
 * Jafarzadeh, Mousavi, Larios, Bobaru, arXiv 2105.06055) as FFT convolutions
 * on one NVIDIA GB300 (sm_103a), and builds the paper's dynamic (velocity
 * Verlet, §4.2.3) and static (conjugate gradient, §4.3) drivers on it.
 *
 * Conventions shared by every entry point
 *   Grid (Eq. 52): n[0] x n[1] x n[2] nodes (n[2] = 1 in 2D), spacing dx[k],
 *     node (i1,i2,i3) at x = (i1 dx1, i2 dx2, i3 dx3), periodic box (§4.1).
 *     Supported lengths: powers of two, 32 <= n[0] <= 2048, 16 <= n[1], n[2] <= 1024.
 *   Fields: device arrays, component-major and x1 fastest,
 *     f[c][i3][i2][i1]; vector fields have d = dim components; N = n0 n1 n2.
 *     Floating-point fields are float (problem.fp64 == 0) or double
 *     (problem.fp64 == 1). Masks are uint8 0/1.
 *   Ownership: the caller owns every field buffer it passes; the library
 *     owns the plan and all of its workspace, which is allocated in
 *     pd_plan_create only. Later calls allocate nothing.
 *   Streams: every call enqueues its work on `stream` (a cudaStream_t, NULL
 *     for the legacy default stream) and returns without synchronising,
 *     except where a call says it reads back a result. A plan may be used
 *     by one stream at a time.
 *   Errors: no exception crosses the ABI. A non-PD_OK status means nothing
 *     was enqueued (argument errors) or a CUDA call failed (PD_ERR_CUDA);
 *     pd_status_string gives a message, pd_last_error_detail more context.
 *
 * Model constants (omega(|xi|) = 1/|xi| throughout, §5.1, §5.2):
 *   PD_LIN_BOND, 2D: C_ij(xi) = alpha omega xi_i xi_j / |xi|^2 (Eq. 17),
 *     alpha = 9E/(pi delta^3), plane stress, nu = 1/3 (§5.2).
 *   PD_LIN_BOND, 3D: alpha = 12E/(pi delta^4), nu = 1/4 (energy calibration of
 *     an isotropic stretch; the paper prints only the 2D value).
 *   PD_LIN_STATE (3D): linearized state-based solid (Eq. 33-39, 92-97) with
 *     kappa = E/(3(1-2nu)), mu = E/(2(1+nu)), bulk m0 = Σ_H omega|xi|^2 dV
 *     in the kernels (Eq. 37) and the nodal m(x) of Eq. 94 in the dilatation.
 *   PD_NONLIN_BOND (2D/3D): bond force c/2 (|xi+eta|^2 - |xi|^2)(xi+eta) with
 *     c = alpha/|xi|^3 and the alpha of PD_LIN_BOND (§3.2, Eq. 19-22): exactly
 *     invariant under finite rigid motions; its small-eta limit is Eq. 17.
 */
#ifndef PD_H
#define PD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PD_OK = 0,
    PD_ERR_ARG = -1,            /* invalid argument (null pointer, bad enum, bad mask) */
    PD_ERR_SIZE = -2,           /* unsupported grid size or horizon                    */
    PD_ERR_NOMEM = -3,          /* device allocation failed in pd_plan_create          */
    PD_ERR_CUDA = -4,           /* a CUDA runtime call or kernel launch failed         */
    PD_ERR_NOT_CONVERGED = -5,  /* iterative solve hit max_iter before rtol            */
    PD_ERR_TIMEOUT = -6,        /* a bounded device-side wait gave up                  */
    PD_ERR_NONFINITE = -7       /* a NaN or Inf appeared in a reduction                */
} pd_status;

typedef enum {
    PD_LIN_BOND = 0,   /* linearized bond-based solid, Eq. 17-18            */
    PD_LIN_STATE = 1,  /* linearized state-based (LPS) solid, Eq. 33-39, 3D */
    PD_NONLIN_BOND = 2 /* nonlinear rotation-invariant bond model, Eq. 19-26
                          (pd_force only; its linearization is PD_LIN_BOND)  */
} pd_model;

typedef struct {
    int dim;         /* 2 or 3                                                    */
    int n[3];        /* grid nodes per axis (Eq. 52); n[2] = 1 in 2D              */
    double dx[3];    /* grid spacing per axis (dx[2] ignored in 2D)               */
    double delta;    /* horizon radius; bonds are 0 < |xi| <= delta (Eq. 48)      */
    int model;       /* pd_model                                                  */
    double E;        /* Young's modulus                                           */
    double nu;       /* Poisson ratio (PD_LIN_STATE only)                         */
    double rho;      /* mass density (Eq. 1), used by pd_step_verlet              */
    double Wc;       /* critical strain energy density (Eq. 40, 63); <= 0: no damage */
    int fp64;        /* 0: FP32 fields and FFTs; 1: FP64 fields and FFTs          */
    int volume_rule; /* quadrature weight of a bond (§4.1.1, remark on cells only
                        partly covered by the horizon): 0 the constant dV of the
                        paper's examples; 1 linear partial volumes, weight
                        beta(|xi|) dV with beta = min(1, (delta + h/2 - |xi|)/h)
                        for |xi| < delta + h/2 (Hu, Ha and Bobaru's rule), which
                        needs cubic cells (all dx equal to h, else PD_ERR_ARG).
                        Part of the kernel C(xi), so the convolution structure and
                        every entry point are unchanged; the family (and the
                        damage counts of pd_damage) then holds every offset with
                        beta > 0, and the body must stay that far from the faces */
    double s0;       /* critical bond stretch (bond model; used when Wc <= 0 and
                        s0 > 0): the plan takes Wc = 1/2 alpha s0^2 dV Σ_H w|xi|,
                        the Eq. 47 energy density of a fully bonded node under the
                        isotropic stretch u = s0 x (every bond then has
                        eta.C.eta = alpha s0^2 |xi| for omega = 1/|xi|; w is the
                        bond's quadrature weight relative to dV). The paper's
                        failure criterion is energy based (§3.4, Eq. 40-44, 51);
                        this maps a stretch criterion onto it. Negative values,
                        or s0 > 0 with the state-based model: PD_ERR_ARG      */
} pd_problem;

typedef struct pd_plan pd_plan;  /* opaque; owns spectra, masks and workspace */

/*
 * pd_plan_create -- validate a problem, copy its masks and precompute every
 * plan-time quantity (§4.1.1, §4.2.2):
 *   - the horizon offsets and the kernel spectrum K^_ij(k) = dV Σ_H C_ij(xi)
 *     e^{-2 pi i k.xi/n} in FP64 (Eq. 56-57; real and even), kept as the
 *     difference M^ = (K^(k) - K^(0)) / N in FP32 and FP64;
 *   - the boundary field G_ij(x) = dV Σ_H C_ij(xi) chi(x+xi) - P_ij chi(x)
 *     (the (C*chi_B) u_j term of Eq. 100 minus P u, zero in the delta-interior);
 *   - state-based: m(x) (Eq. 94, 97) and q_i(x) = Σ_H g_i(xi) dV chi(x+xi) with
 *     g_i = omega xi_i, and the spectrum of g_i.
 * chi_B:     device, N bytes, 1 inside the body B (Eq. 73). The body must stay
 *            at least delta from the box faces (§4.2.2), else PD_ERR_ARG.
 * chi_Omega: device, d x N bytes (Eq. 74, one mask per component), or NULL
 *            for chi_Omega_i = chi_B. chi_Omega must be 0 where chi_B is 0.
 * stream:    stream for the plan-time kernels; pd_plan_create synchronises it.
 * out:       receives the plan; release it with pd_plan_destroy.
 * The masks are copied; the caller may free its buffers afterwards.
 */
pd_status pd_plan_create(const pd_problem *problem, const uint8_t *chi_B,
                         const uint8_t *chi_Omega, void *stream, pd_plan **out);

/* Release a plan and all of its device memory. NULL is a no-op. */
void pd_plan_destroy(pd_plan *plan);

/*
 * pd_kernel_spectrum -- write the FP64 kernel spectrum (Eq. 56-57)
 *   K^_ij(k) = dV Σ_{xi in H} C_ij(xi) cos(2 pi Σ_a k_a o_a / n_a)
 * for the half-spectrum k1 in [0, n0/2], k2 in [0, n1), k3 in [0, n2), as
 * d(d+1)/2 real arrays in the order 11,22,33,12,13,23 (2D: 11,22,12), each
 * [k3][k2][k1] with k1 fastest. out: device, d(d+1)/2 x (n0/2+1) n1 n2 doubles.
 * K^(0) is the tensor P_ij of Eq. 56.
 */
pd_status pd_kernel_spectrum(pd_plan *plan, double *out, void *stream);

/*
 * pd_force -- one FCBM-EC force evaluation (Eq. 57-58 with the chi_B cut of
 * Eq. 75 and the node weight of Eq. 100):
 *   bond:  L_i = v [ C_ij * (v u_j) - (C_ij * v) u_j ] dV,  v = chi_B s
 *   state: L_i = chi [ -th (a_i*chi) - a_i*(chi th) + C_ij*(chi u_j)
 *                      - (C_ij*chi) u_j ] dV           (Eq. 92, 95-97)
 * computed as FFT convolutions on the device:
 *   L_i = v [ IFFT( M^_ij FFT(v u_j) ) - G_ij u_j ]  (algebraically identical).
 * u:  device, d x N (input displacement).
 * s:  device, N node weight (bond model only), or NULL for s = 1. With s the
 *     G field is formed for v = chi_B s inside the call (extra convolutions).
 * L:  device, d x N (output force density; 0 where chi_B = 0).
 * W:  device, N, or NULL: strain energy density of Eq. 47 / 102 with bond
 *     factor v v' (bond model only).
 * u and L must not overlap.
 * PD_NONLIN_BOND (s and W must be NULL): the force of Eq. 21 with the chi_B
 * cut, L_i = chi Σ_H chi' c/2 (|xi+eta|^2 - |xi|^2)(xi_i+eta_i) dV, evaluated as
 * the correlations of Eq. 26 (the paper's Eq. 59 prints one of its terms
 * without the factor u_i; the form used here is Eq. 26's): forward transforms
 * of chi u_j, chi u_i u_j and chi |u|^2 u_i (2D: 7 fields, 3D: 12), one
 * spectral combination with the kernels C_ij = c xi_i xi_j, a_i = c xi_i and c
 * (2D: 11 inverse fields, 3D: 21), and a per-node epilogue with plan-time
 * boundary fields. The body mean of u is removed first (the model is exactly
 * translation invariant), which keeps the FP32 rounding at the level of the
 * deformation instead of |u|^3.
 */
pd_status pd_force(pd_plan *plan, const void *u, const void *s, void *L, void *W, void *stream);

/*
 * pd_step_verlet -- nsteps of velocity Verlet with embedded constraint and the
 * energy-based bond breaking of §3.4 (bond model):
 *   a^n       = L(u^n, lam^n) + b
 *   u^{n+1}   = chi_O { u^n + dt [v^n + dt/(2 rho) a^n] } + (1 - chi_O) w   (Eq. 83)
 *   lam^{n+1} = lam^n [ W(u^n, lam^n) <= Wc ]  (Eq. 63; irreversible)
 *   v^{n+1}   = chi_O { v^n + dt/(2 rho) (a^n + a^{n+1}) }                  (Eq. 84)
 * with L and W of Eq. 101-102 (node weight chi_B lam). Wc <= 0 disables
 * breaking (lam stays as given).
 * u, v:   device, d x N, updated in place.
 * lambda: device, N bytes (integrity index, Eq. 43), updated in place; NULL
 *         means lam = 1 and no breaking.
 * b, w:   device, d x N: body force density and Gamma values (Eq. 78); w may
 *         be NULL (w = 0).
 * n_broken_out: host pointer or NULL; receives the number of nodes whose lam
 *         went from 1 to 0 during the call (this synchronises the stream).
 */
pd_status pd_step_verlet(pd_plan *plan, void *u, void *v, uint8_t *lambda, const void *b,
                         const void *w, double dt, int nsteps, int64_t *n_broken_out,
                         void *stream);

/*
 * pd_step_verlet_ramp -- pd_step_verlet with a time-varying volume constraint
 * (Eq. 78, 83: the values prescribed on Gamma change with time), linear in
 * time: the step that ends at time t = t0 + (n + 1) dt (n = 0 .. nsteps - 1)
 * sets u = w0 + t w1 on Gamma. This is displacement-controlled loading at a
 * constant rate, run on the device with no per-step host work; a general
 * w(t) is applied by calling pd_step_verlet once per step (or per chunk) with
 * the current field. t0 is the time at the start of the call.
 * w0: device d x N or NULL (= 0); w1: device d x N (required).
 * Other arguments and the result as for pd_step_verlet.
 */
pd_status pd_step_verlet_ramp(pd_plan *plan, void *u, void *v, uint8_t *lambda, const void *b, const void *w0,
                              const void *w1, double t0, double dt, int nsteps, int64_t *n_broken_out,
                              void *stream);

/*
 * pd_plan_set_energy_mode -- how pd_step_verlet evaluates the strain energy
 * density W that decides bond breaking (Eq. 63):
 *   0 (default): the paper's convolution form, Eq. 102 (three FFT
 *      convolutions of nodal products, fused into the force passes);
 *   1: the plain horizon sum of Eq. 47 in the plan's precision.
 * Both compute the same W. The convolutions' rounding error is global, about
 * eps lambda_max (rms|u|^2 + 2|u(x)| rms|u|) at every node; in FP32 it reaches
 * Wc once fragments have moved tens of grid units, and spurious breaking
 * follows. The direct sum's error is local (about eps |u(x)| / |eta| relative
 * to W). Mode 1 is for FP32 runs that go past full separation.
 */
pd_status pd_plan_set_energy_mode(pd_plan *plan, int mode);

/*
 * pd_solve_static -- solve the FCBM-EC static problem (Eq. 85-89)
 *   chi_O (L(u) + b) = 0 on Omega,  u = w on Gamma,
 * by conjugate gradient (§4.3, ref. [50]) on A e = chi_O (b + L(w)),
 * A e = -chi_O L(chi_O e), which is symmetric positive definite on Omega.
 * FP32 plan: the inner CG runs on FP32 FFT convolutions with FP64 inner
 * products; an outer iterative refinement recomputes the residual
 * r = chi_O (b + L(u)) with the FP64 operator and stops when
 * ||r||_2 <= rtol ||chi_O b||_2, or, for a problem driven by w alone
 * (chi_O b = 0), when ||r||_2 <= rtol times the residual of the initial guess
 * (for u = 0 on Omega that is ||chi_O L(w)||_2, the norm of the right-hand
 * side). FP64 plan: plain CG on the FP64 operator.
 * u:  device, d x N, FP64 regardless of the plan's precision; in: initial
 *     guess (values on Gamma are replaced by w), out: solution.
 * b, w: device, d x N, FP64 (w may be NULL for w = 0).
 * max_iter: cap on the total number of CG iterations.
 * iters_out, relres_out: host pointers (may be NULL): CG iterations done and
 *     the final FP64 relative residual. The call synchronises the stream.
 * Returns PD_ERR_NOT_CONVERGED if rtol was not reached.
 */
pd_status pd_solve_static(pd_plan *plan, double *u, const double *b, const double *w,
                          double rtol, int max_iter, int *iters_out, double *relres_out,
                          void *stream);

/*
 * pd_solve_dr -- the static problem of pd_solve_static (same arguments,
 * same FP64 iterative refinement and stopping rule) with dynamic relaxation
 * as the inner solver instead of CG. Dynamic relaxation is not in the paper;
 * the method is adaptive dynamic relaxation (Underwood 1983; the peridynamic
 * form of Kilic and Madenci, Theor. Appl. Fract. Mech. 53 (2010) 194-204):
 * damped central-difference pseudo dynamics with a fictitious density of
 * 1.05/4 of the largest eigenvalue of the periodic symbol (pd_stable_dt),
 * unit pseudo time step and the damping 2 sqrt(e.Ae / (rho e.e)), with A e
 * taken exactly (it is the right-hand side minus the pseudo force) instead
 * of the published diagonal local-stiffness estimate.
 * The whole solve, including its stopping decisions, runs as one CUDA graph
 * launch with device-side conditional nodes.
 * max_iter: cap on the total number of relaxation steps (rounded up to a
 *     multiple of 16; at most 16777216).
 * iters_out: relaxation steps done. The call synchronises the stream.
 */
pd_status pd_solve_dr(pd_plan *plan, double *u, const double *b, const double *w,
                      double rtol, int max_iter, int *iters_out, double *relres_out, void *stream);

/*
 * pd_solve_mirror -- the static problem of §5.1 with mirror-based volume
 * constraints instead of the naive ones: every node of Gamma (chi_B = 1,
 * chi_O = 0 for a component) takes u = 2 g - u(mirror) from the local boundary
 * value g and the solution at its mirror node inside Omega, while
 * chi_O (L(u) + b) = 0 holds on Omega (Eq. 89). The paper describes the method
 * but its appendix is not in the text; this solves the coupled problem at
 * once: in the Omega values e, u = E e + h with E e = chi_O e - (1 - chi_O)
 * e(mirror) and h = 2 (1 - chi_O) g, and A e = -chi_O L(E e) = chi_O (L(h) + b)
 * is solved by BiCGStab (A is not symmetric), one FFT force evaluation per
 * product, FP64 (FP64 plans only).
 * u:      device d x N FP64, out: the solution (E e + h).
 * b, g:   device d x N FP64 or NULL (0); g is read on Gamma.
 * mirror: device d x N int32: for each component the flat node index of the
 *         mirror node of a Gamma node (ignored elsewhere); PD_ERR_ARG unless
 *         every Gamma node has one inside Omega for that component.
 * Stops when ||r|| <= rtol ||r0||, r0 = chi_O (L(h) + b); relres_out is the
 * recomputed FP64 residual of u relative to ||r0||. Synchronises the stream.
 */
pd_status pd_solve_mirror(pd_plan *plan, double *u, const double *b, const double *g, const int32_t *mirror,
                          double rtol, int max_iter, int *iters_out, double *relres_out, void *stream);

/*
 * Batched specimens: nspec independent problems (each its own grid, horizon,
 * masks and material) solved together. pd_plan_create_batched creates one plan
 * per specimen (same rules and arguments as pd_plan_create, element i of each
 * array for specimen i; chi_Omega may be NULL for chi_Omega = chi_B for all,
 * or contain NULL entries) and the batch's streams and events.
 */
typedef struct pd_batch pd_batch;  /* opaque; owns its plans */
pd_status pd_plan_create_batched(int nspec, const pd_problem *problems, const uint8_t *const *chi_B,
                                 const uint8_t *const *chi_Omega, void *stream, pd_batch **out);
int pd_batch_size(const pd_batch *batch);
/* Plan of specimen i (owned by the batch; NULL if i is out of range). */
pd_plan *pd_batch_plan(pd_batch *batch, int i);
/*
 * pd_solve_dr_batched -- pd_solve_dr for every specimen, all in ONE CUDA-graph
 * launch: each specimen is an independent branch of the graph whose loop of
 * relaxation steps and refinement cycles is controlled on the device
 * (conditional WHILE / IF nodes set by the solver's check kernels), so
 * specimens of different sizes converge without host round trips and run
 * concurrently. The executable graph is cached and rebuilt only when the
 * buffers, rtol or max_iter change.
 * u, b, w: host arrays of nspec device pointers (d_i x N_i FP64 each; w may be
 *     NULL, or hold NULL entries, for w = 0).
 * iters_out, relres_out, status_out: host arrays of nspec (each may be NULL):
 *     steps, final FP64 relative residual and pd_status of each specimen.
 * Returns PD_OK if every specimen converged, else the first failure's status.
 * Synchronises the stream.
 */
pd_status pd_solve_dr_batched(pd_batch *batch, double *const *u, const double *const *b,
                              const double *const *w, double rtol, int max_iter, int *iters_out,
                              double *relres_out, int *status_out, void *stream);
/* Release the batch and all of its plans. NULL is a no-op. */
void pd_batch_destroy(pd_batch *batch);

/*
 * Autotuning of the FFT passes. pd_plan_autotune times the plan's force
 * evaluation (on its own workspace; no caller buffer is touched) over the
 * candidate rows per row-pass block, row-pass pipeline depths, column-tile
 * widths of the x2 and last-axis passes and FFT stage schedules (radix-4/2
 * remainder stage first or last), coordinate-wise from the built-in
 * heuristic, and keeps the fastest. Results do not change (the same transforms are computed); later
 * calls use the chosen configuration. Synchronises the stream.
 * pd_batch_autotune tunes one plan per distinct grid/precision/operator of a
 * batch and gives the others the same configuration.
 * pd_plan_tuning writes {rows, x2 width, last-axis width, schedule, stages,
 * inverse-pass stages} (0 = heuristic) to out6.
 */
pd_status pd_plan_autotune(pd_plan *plan, void *stream);
/* The same search timing a chunk of 16 iterations of the static solver's CG
 * (pd_solve_static's unit of work) instead of a force evaluation; uses the
 * plan's solver workspace. */
pd_status pd_plan_autotune_solve(pd_plan *plan, void *stream);
pd_status pd_batch_autotune(pd_batch *batch, void *stream);
pd_status pd_plan_tuning(const pd_plan *plan, int *out6);
/* Pin a pass configuration {rows, x2 width, last-axis width, schedule,
 * stages, inverse-pass stages}: rows and widths 0 or powers of two (rows <=
 * 256, widths 2..32; 0 = heuristic), schedule 0/1, row-pass pipeline stages
 * 0 (= 2), 1 or 2, inverse-pass stages 0 (= as the forward passes), 1 or 2;
 * PD_ERR_ARG otherwise. The pass configuration functions still shrink a value
 * that does not fit the grid or the shared memory, and raise rows to fill at
 * least one warp per row-pass block. */
pd_status pd_plan_set_tuning(pd_plan *plan, const int *in6);

/*
 * pd_force_adjoint -- reverse-mode derivative of pd_force (bond model). The
 * paper has no adjoint; this differentiates the quadrature of Eq. 17-18, 75
 * with bond factor s s'. Given gL = dJ/dL for some scalar J:
 *   gu_i(y) = (dL/du)^T gL = L[gL](y)   (the operator is symmetric, so this is
 *             the same FFT convolution applied to gL)
 *   gs(y)   = chi(y) Σ_xi chi' s' C_ij(xi) (gL_i(y) - gL_i(y+xi)) (u_j(y+xi) - u_j(y)) dV
 *           = chi { gL_i [C_ij*(v u_j)] - gL_i u_j [C_ij*v] - Σ_ij C_ij*(v gL_i u_j)
 *                   + u_j [C_ij*(v gL_i)] } dV,   v = chi s
 * u, s, gL: device inputs (s may be NULL for s = 1); gu: device d x N output
 * (may be NULL); gs: device N output (may be NULL).
 */
pd_status pd_force_adjoint(pd_plan *plan, const void *u, const void *s, const void *gL,
                           void *gu, void *gs, void *stream);

/*
 * pd_verlet_loss_grad -- differentiable FCBM-EC dynamics with bond breaking:
 * a loss on the final state of velocity Verlet (Eq. 83-84 with w = 0) and its
 * gradient with respect to a spatially varying micromodulus c(x). The paper
 * has no adjoint; this differentiates the same discrete dynamics.
 * Dynamics: bond model with bond factor (s lam)(s' lam'), s = sqrt(c_rel)
 * (c = c_rel times the plan's micromodulus), energy-based breaking of Eq. 63
 * when the plan has Wc > 0 (W of Eq. 47 with the same bond factor);
 *   a^n = L(u^n) + b [+ b0 at n = 0],  v^h = v^n + dt/(2 rho) a^n,
 *   u^{n+1} = chi_O (u^n + dt v^h),  lam^{n+1} = lam^n [W^n <= Wc],
 *   v^{n+1} = chi_O (v^h + dt/(2 rho) a^{n+1}),   n = 0 .. nsteps - 1;
 * loss J = Σ_nodes,components (u^N - u_target)^2.
 * Gradient: dJ/dc_rel with the breaking history held fixed (the decisions
 * are piecewise constant in c: this is the derivative wherever none of them
 * changes), by a reverse sweep of adjoint force passes (pd_force_adjoint's)
 * over states recomputed from checkpoints of (u, v, lam) every
 * checkpoint_every steps.
 * c_rel: device N (> 0, else PD_ERR_ARG). lambda0: device N bytes or NULL (1).
 * u0, v0, b, b0: device d x N or NULL (0). u_target: device d x N.
 * work: device, at least pd_verlet_adjoint_workspace(plan, nsteps,
 *   checkpoint_every) bytes, 256-byte aligned; the caller owns it.
 * loss_out: host (may be NULL). grad_c: device N or NULL (no reverse sweep).
 * u_final (device d x N) and lambda_final (device N) may be NULL.
 * Plan precision for every field. Synchronises the stream.
 */
int64_t pd_verlet_adjoint_workspace(const pd_plan *plan, int nsteps, int checkpoint_every);
pd_status pd_verlet_loss_grad(pd_plan *plan, const void *c_rel, const uint8_t *lambda0, const void *u0,
                              const void *v0, const void *b, const void *b0, const void *u_target, double dt,
                              int nsteps, int checkpoint_every, void *work, int64_t work_bytes, double *loss_out,
                              void *grad_c, void *u_final, uint8_t *lambda_final, void *stream);

/*
 * pd_damage -- broken-bond counts and damage index (Eq. 12, 44, 48-49, 65):
 *   beta(x) = chi Σ_H chi',  nb(x) = chi Σ_H chi' (1 - lam lam'),  d = nb / beta.
 * Counts are exact integers (direct integer sums over the horizon).
 * lambda: device N bytes. nb: device N int32 or NULL. d: device N float/double
 * (plan precision) or NULL.
 */
pd_status pd_damage(pd_plan *plan, const uint8_t *lambda, int32_t *nb, void *d, void *stream);

/*
 * pd_force2d_noalloc -- pd_force for a 2D bond-model FP32 problem without a
 * plan and without allocating any memory. The paper has no counterpart: this
 * exists for callers that may not call cudaMalloc (a host framework that owns
 * all device memory through its own pool, a real-time loop that must not hit
 * the allocator, a plug-in with a fixed memory budget) and so cannot create a
 * pd_plan. Same operator and result as pd_plan_create + pd_force with s = NULL
 * and W = NULL.
 *   problem: dim = 2, model = PD_LIN_BOND, fp64 = 0, volume_rule = 0 (else
 *            PD_ERR_ARG); grid rules as for pd_plan_create, and
 *            n[0] * n[1] <= 65536 nodes, horizon <= 512 bonds
 *            (else PD_ERR_SIZE, nothing enqueued).
 *   chi_B:   device, N bytes (0/1, body at least delta from the box faces,
 *            checked: PD_ERR_ARG otherwise). u: device, 2 x N floats.
 *   L:       device, 2 x N floats (output).
 * All intermediates live in one fixed 2 MiB __device__ array inside the
 * library, held by every GPU that loads it until the process exits. The first
 * call on each device looks up that array's device address; make it before
 * any stream capture. The call synchronises `stream` once (it reads the mask
 * check back to the host), then enqueues the force passes and returns. Every call reuses the same array, so
 * calls that overlap on the GPU (from several streams or threads) race; the
 * caller must serialise them.
 */
pd_status pd_force2d_noalloc(const pd_problem *problem, const uint8_t *chi_B, const float *u, float *L,
                             void *stream);

/* Critical strain energy density the plan uses for bond breaking (Eq. 63):
 * problem.Wc when it is > 0, else the value derived from problem.s0 (see
 * pd_problem), else 0 (no breaking). Host FP64. */
double pd_plan_critical_energy(const pd_plan *plan);

/*
 * pd_plan_set_affine_split -- accuracy option of pd_force for FP32 fields
 * with a large affine part (bond model; 1 on, 0 off, the default). The FFT
 * convolution's rounding error grows with the norm of the transformed field
 * (about eps ||chi u|| lam_max), while the force of an affine field
 * a = A x + t is known exactly: chi Σ_H chi' C_ij(xi) A_jk xi_k dV (Eq. 17-18
 * with u' - u = A xi), nonzero only within delta of the body's boundary. With
 * the option on, pd_force (s = NULL, W = NULL) fits a by least squares over
 * the body (one reduction over u), transforms u - a only and adds the force of
 * a at the boundary nodes from a plan-time moment table; the fit's
 * coefficients are rounded so that a is evaluated exactly, and the result is
 * the same operator applied to u. Cost: one extra read of u per call. Other
 * calls (weights, W, the solvers) are unchanged. PD_ERR_ARG for the
 * state-based model or a body without a full-rank set of nodes.
 */
pd_status pd_plan_set_affine_split(pd_plan *plan, int on);

/*
 * pd_plan_set_plane_passes -- pass layout of the FP32 CG iteration of
 * pd_solve_static on cubes of 32^3, 64^3 and 128^3. Bit 0 of mask: the
 * forward half (CG update, x1 and x2 transforms), bit 1: the inverse half
 * (x2 and x1 inverse transforms, CG epilogue) run as plane passes, where the
 * transforms of one field of one x1-x2 plane run in one block
 * (pd_plan_profile kinds 4 and 5) and the spectra make no round trip between
 * them; a clear bit runs that half as a row pass and a column pass along x2
 * (kinds 0, 1, 3), as on every other shape. Same operator either way (the
 * transforms and epilogues do the same arithmetic). Default 1: on the 128^3
 * cube with cavity the forward plane pass makes the solve faster than its row
 * and column passes, while adding the inverse plane pass makes it slower
 * (115.3 against 105.9 ms per solve); pd_plan_autotune_solve times 1 and 0
 * and keeps the faster. PD_ERR_ARG for a null plan or a mask outside 0..3.
 */
pd_status pd_plan_set_plane_passes(pd_plan *plan, int mask);

/*
 * pd_plan_inject_stall -- test hook for the failure handling of bounded
 * device waits. The next pass of the given kind launched on the plan
 * (0: forward row pass, 3: inverse row pass, 5: inverse plane pass of the
 * FP32 CG; see pd_plan_profile) has its first block issue none
 * of its bulk copies, so that block's wait on its copy barrier gives up after
 * the library's limit (2 s), sets the plan's device status word and the block
 * exits; the rest of the pass runs normally. pd_solve_static then returns
 * PD_ERR_TIMEOUT at its next check (after the CG chunk, at most 16
 * iterations). Nothing faults or hangs; the plan stays usable (each solve
 * clears the status word). One-shot: the word is cleared by the block that
 * takes it. Synchronous (writes one word to device memory).
 */
pd_status pd_plan_inject_stall(pd_plan *plan, int kind);

/* Bytes of device memory owned by the plan. */
int64_t pd_plan_workspace_bytes(const pd_plan *plan);

/* Largest stable velocity-Verlet step for the plan's periodic operator:
 * 2 sqrt(rho / max_k max-eig M(k)), M(k) = K^(0) - K^(k) (host FP64). */
double pd_stable_dt(const pd_plan *plan);

/* Number of kernel launches the library has enqueued since the plan was
 * created (for launch accounting). */
int64_t pd_plan_launch_count(const pd_plan *plan);

/* Number of body nodes within delta of the body's boundary, where the
 * boundary field G of pd_plan_create is nonzero (kept as a sparse list). */
int64_t pd_plan_boundary_nodes(const pd_plan *plan);

/*
 * Per-pass timing (diagnostics). pd_plan_profile(plan, mask) selects the pass
 * kinds to time (bit k for kind k, 0 switches timing off): every FFT-pass
 * launch of a selected kind is then bracketed by two CUDA events recorded on
 * the launching stream (the events are created in pd_plan_create; inside the
 * solver's CUDA graphs they are graph event nodes). pd_plan_profile_read
 * returns the summed event time and the launch count of one pass kind since
 * the last pd_plan_profile call:
 *   0 row pass, forward (prologue + x1 transform)
 *   1 column pass along x2 (3D), forward or inverse
 *   2 last-axis pass (forward transform, spectral combine, inverse transform)
 *   3 row pass, inverse (x1 transform + epilogue)
 *   4 plane pass, forward (CG prologue + x1 and x2 transforms; FP32 CG on cubes
 *     of 32^3, 64^3 and 128^3, whose x1-x2 plane of one field fits in shared memory)
 *   5 plane pass, inverse (x2 and x1 transforms + CG epilogue; same cubes)
 * Reading synchronises on the recorded events. Enabling resets the counters.
 */
pd_status pd_plan_profile(pd_plan *plan, int mask);
pd_status pd_plan_profile_read(pd_plan *plan, int kind, double *ms_total, int64_t *launches);

const char *pd_status_string(pd_status status);
const char *pd_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* PD_H */
