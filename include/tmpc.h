/*
 * tmpc.h -- C ABI of the batched, differentiable OCP solver (GB300, sm_103a).
 *
 * The library solves B independent optimal-control problems (the OCP of
 * Section II-A / Appendix A of the paper) with SQP (Algorithm 1): at each SQP
 * iterate the QP of Section III-A / Appendix B is built and solved by the ADMM
 * scheme of Algorithm 3 (Section III-B, Appendix C), whose primal system
 * S x = eta (Eq. admm:schur) is factored once per SQP step and per accepted
 * rho and reused; the next iterate is chosen by the line search of Appendix D.
 * The backward pass is the active-set implicit differentiation of Algorithm 2
 * (Section III-D, Appendix E).
 *
 * Conventions for every call
 *  - Plain C types only.  Array arguments are DEVICE pointers (CUDA global
 *    memory) unless the name of the call ends in _host.  All float arrays are
 *    contiguous, row-major FP32; integer arrays are int32.  The caller owns
 *    every array it passes; the handle owns its workspace.
 *  - Padded batch layout with layout maxima (Nmax, nx, nu, ng) from tmpc_dims:
 *    stage arrays are [B][Nmax+1][...]; an instance i uses stages 0..N[i] and
 *    the leading (nx_i, nu_i, ng_i) entries of its model: a stage vector
 *    z[t] holds the state in z[t][0:nx_i] and the control in
 *    z[t][nx_i:nx_i+nu_i].  Outputs beyond an instance's horizon or dims are
 *    written as 0.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream and return after the
 *    work is enqueued, except where stated.  Argument validation (null
 *    pointers, dims, alignment) is synchronous; a failed validation enqueues
 *    nothing.
 *  - Per-instance outcomes (non-convergence, factorisation failure, NaN) are
 *    reported in the status array, never as a call failure.
 *  - A handle is not thread-safe; one host thread at a time.
 *  - No exceptions cross this ABI.
 */
#ifndef TMPC_H
#define TMPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TMPC_OK = 0,
    TMPC_ERR_INVALID_ARG = 1,   /* null pointer, bad dims, misaligned array     */
    TMPC_ERR_CUDA = 2,          /* a CUDA runtime call failed                   */
    TMPC_ERR_OOM = 3,           /* workspace allocation failed in tmpc_setup    */
    TMPC_ERR_NOT_SETUP = 4,     /* backward without a matching solve, etc.      */
    TMPC_ERR_UNSUPPORTED = 5    /* model/dims combination not compiled in       */
} tmpc_status;

/* per-instance status values written by tmpc_solve / tmpc_backward */
enum {
    TMPC_INST_OK = 0,         /* final SQP KKT residual (Eq. sqp_stop) <= eps_c   */
    TMPC_INST_MAX_ITER = 1,   /* iteration caps reached before eps_c             */
    TMPC_INST_NOT_PD = 2,     /* a pivot block of S was not positive definite    */
    TMPC_INST_NAN = 3,        /* a non-finite value appeared                     */
    TMPC_INST_INVALID = 4,    /* tmpc_solve_static only: N or model of the instance
                                 is out of range for the layout; not solved       */
    TMPC_INST_TIMEOUT = 5     /* a bounded wait for an asynchronous shared-memory copy
                                 gave up; the result of the instance is not valid  */
};

/* model ids (problem families; dynamics as in Appendix A of the paper, Remark A1) */
enum {
    TMPC_MODEL_DOUBLE_INTEGRATOR = 0, /* nx=4 nu=2 ng=4, ZOH.  dyn = [dt]                          */
    TMPC_MODEL_LINEAR = 1,            /* layout nx, nu, ng=nu; x+ = A x + B u + b.  dyn = [A, B, b]
                                         (row-major; b is optional: 0 when n_dyn < nx^2 + nx nu + nx) */
    TMPC_MODEL_BICYCLE = 2,           /* nx=6 nu=2 ng=5, implicit midpoint.  dyn = [dt, L, ds, nt] */
    TMPC_MODEL_QUADROTOR = 3,         /* nx=6 nu=2 ng=2, RK4.  dyn = [dt, m, I, arm, g]            */
    TMPC_MODEL_BICYCLE_TRAP = 4,      /* as 2 with the trapezoidal constraint of Remark A1         */
    TMPC_MODEL_BICYCLE_NEWTON = 5,    /* as 2 with the explicit map x+ = Phi(x, u) that 3 Newton
                                         steps on the midpoint rule define, Jacobians by the
                                         implicit function theorem (generic kernel only)          */
    TMPC_MODEL_SRB = 6                /* single-rigid-body humanoid (App. humanoid SRB dynamics):
                                         nx=12 (p, ZYX Euler angles, v, body rates) nu=6 (foot
                                         forces f_L, f_R, world frame) ng=6 (box on the forces),
                                         RK4.  dyn = [dt, m, Ixx, Iyy, Izz, r_L (3), r_R (3),
                                         gravity] (generic kernel only)                           */
};

/* number of floats per instance in tmpc_solution.stats */
#define TMPC_STATS 10
/* stats[0] SQP iterations, [1] ADMM iterations (total), [2] r_prim and [3] r_dual of
 * the last QP (Eq. admm:residuals), [4] final rho_bar, [5] factorisations of S,
 * [6] KKT residual of Eq. (sqp_stop) at the returned point, [7] last line-search step,
 * [8], [9] line-search history of SQP iterations 0-5 and 6-11: the integer value
 * holds 4 bits per iteration j at bit 4*(j mod 6), k for a step 2^-k (k >= 14 coded
 * 14) and 15 for a zero step. */

typedef struct {
    int32_t batch;   /* B >= 1                                                     */
    int32_t N_max;   /* layout horizon; stage arrays hold N_max+1 stages           */
    int32_t nx, nu;  /* layout state / control sizes                               */
    int32_t ng;      /* layout inequality rows per stage                           */
    int32_t n_dyn;   /* floats of dynamics parameters per instance                 */
    int32_t n_track; /* centreline table intervals per instance (0 = no table)     */
} tmpc_dims;

typedef struct {
    /* ADMM (Section III-B): sigma, initial rho_bar, rho_bar clip range, over-relaxation */
    float sigma, rho0, rho_min, rho_max, alpha;
    /* termination (Eq. admm:termination:slack), SQP stop (Eq. sqp_stop), active-set tolerance */
    float eps_abs, eps_rel, eps_c, eps_g;
    float ls_eta;        /* Armijo constant of Appendix D                             */
    int32_t k_rho_iter;  /* rho_bar is re-evaluated every k_rho_iter ADMM iterations  */
    float k_rho_ratio;   /* ... and accepted if it changes by more than this factor   */
    int32_t max_sqp, max_admm;
    int32_t n_ls;        /* line-search candidates alpha = 2^-k, k < n_ls (<= 16)     */
    int32_t newton_steps;/* Newton steps per stage of the implicit initial rollout    */
    int32_t early_exit;  /* 1: stop ADMM / SQP when converged; 0: fixed counts        */
    int32_t check_every; /* ADMM termination test period when early_exit              */
    /* backward: regularised-KKT refinement (see tmpc_backward) */
    float bwd_rho, bwd_sigma;
    int32_t bwd_iters;
    int32_t threads;     /* CTA size per instance (0 = automatic)                     */
    int32_t solver;      /* 0 automatic, 1 generic kernel (any model; sequential block LDL'
                          * by the CTA, workspace in global memory), 2 block cyclic
                          * reduction (shared-memory arena per instance where it fits, else
                          * global), 3 as 2 with every arena in global memory, 4 sequential
                          * block LDL' swept by one warp (shared-memory arena), 5 as 4 with
                          * every arena in global memory, 6 block cyclic reduction by one
                          * thread-block cluster per instance (long horizons, few
                          * instances), 7 the plain per-phase form (one launch per ADMM
                          * iteration and phase, state in global memory, fixed counts: a
                          * measurement baseline).  2-7 apply to the double integrator,
                          * bicycle and quadrotor; other models use 1.                    */
    /* Failure-path hooks (host-side fault injection; nothing here can fault the GPU):
     * force_pivot_failure: instance index + 1 whose factorisation of S is treated as
     *   failed from the first SQP step on (status TMPC_INST_NOT_PD from tmpc_solve and
     *   tmpc_backward; the arithmetic is unchanged); 0 = none.
     * wait_polls: polls of each bounded wait on an asynchronous shared-memory copy of
     *   the generic kernel before it gives up (status TMPC_INST_TIMEOUT; the instance
     *   finishes on global-memory reads of the same values); 0 = the default, 2^24.
     * force_wait_timeout: nonzero makes every such wait give up at once, as if its
     *   copy had not landed in time (the copies still in flight are then waited for,
     *   bounded, before their shared buffers are reused). */
    int32_t force_pivot_failure;
    int32_t wait_polls;
    int32_t force_wait_timeout;
    /* backward solver.  1 = the iterative refinement preconditioned by an FP32
     * factorisation of the regularised system (bwd_rho, bwd_sigma, bwd_iters); 2 (the
     * default) = one direct FP64 block LDL' factorisation of the interleaved active-set
     * KKT system (exact up to rounding, also when the active rows are nearly
     * dependent); 0 = the refinement, then the direct solve for every instance whose
     * refinement did not converge by its own step test.  The direct solve exists for
     * the small models and, on the generic kernel, when nx + (nx + nu) + ng <= 32;
     * elsewhere 0 and 2 mean 1.  3 = the reduced adjoint QP of Appendix E (the
     * paper's ADMM-based backward, kept for comparison): every hard active row is
     * absorbed into the Hessian as a penalty of weight bwd_gamma, leaving an
     * equality-only QP in eta_x that the refinement solves (multipliers on the
     * dynamics rows only); its gradient is biased by O(1 / bwd_gamma) against the
     * exact adjoint of 0-2, and the multiplier it returns for a hard active row is
     * bwd_gamma G_A eta_x.  Not combinable with exact_hessian. */
    int32_t bwd_solver;
    /* 1: the direct backward uses the exact Lagrangian Hessian H = Hessian of
     * l + y_f' f + y_A' g_A (App. E) at the solution, the constraint curvature by FP64
     * central differences of the analytic Jacobians; 0: the cost Hessian (the paper's
     * Hessian approximation; exact for linear dynamics).  Implies the direct solve
     * (small models). */
    int32_t exact_hessian;
    float bwd_gamma;     /* penalty weight of the hard active rows when bwd_solver = 3   */
} tmpc_options;

/* Problem parameters theta (the OCP of Appendix A with the cost of Eq. (cost)).
 * All DEVICE pointers, layout as in the header comment; optional ones may be NULL
 * (treated as zeros; gamma2 NULL = every row hard).
 *   N [B], model [B]                           horizon and model id of each instance
 *   Qd [B][Nmax+1][nx], Rd [B][Nmax+1][nu]     diagonal cost weights (row N: terminal)
 *   Wd [B][nu]                                 control-rate weights (optional)
 *   ref [B][Nmax+1][nx+nu]                     reference (x_ref, u_ref) (optional)
 *   lin [B][Nmax+1][nx+nu]                     linear cost term (optional)
 *   lo, hi [B][Nmax+1][ng]                     bounds of g_t; +-inf = no bound
 *   gamma2, gamma1 [B][ng]                     L2 / L1 slack weights; gamma2 = +inf: hard row
 *   dyn [B][n_dyn]                             model parameters
 *   track [B][n_track+1][4]                    centreline table (x_c, y_c, psi_c, kappa)
 *   scale [B][nx+nu]                           optional: characteristic magnitude of each state
 *                                              and control (Remark 4, problem rescaling).
 *     When given, every ADMM solve runs on the QP in normalised variables z = D zh, with
 *     D = diag(d) on every stage and d_j the largest power of two not above scale_j (an
 *     entry that is not positive and finite counts as 1; keep the magnitudes within
 *     2^-30 .. 2^30, as the normalised data must stay in FP32 range); the dynamics rows are divided by
 *     the scale of the state they define and a bound row of one variable by that
 *     variable's scale, the other rows are left as they are.  Powers of two make the
 *     change of variables exact.  rho, the ADMM residuals, the termination test and the
 *     rho rule act in the normalised units; the SQP iterate, the line search, the KKT
 *     test, the returned solution and multipliers and tmpc_backward stay in physical
 *     units.  Built on the shared-memory kernels (double integrator, bicycle, quadrotor;
 *     solver 0 or 2..7); a call that would run a scaled instance on the generic kernel,
 *     and tmpc_solve_static with a scale, return TMPC_ERR_INVALID_ARG before any work
 *     is enqueued.  NULL = no rescaling. */
typedef struct {
    const int32_t* N;
    const int32_t* model;
    const float* Qd;
    const float* Rd;
    const float* Wd;
    const float* ref;
    const float* lin;
    const float* lo;
    const float* hi;
    const float* gamma2;
    const float* gamma1;
    const float* dyn;
    const float* track;
    const float* scale;
} tmpc_params;

/* Solution (z, xi, y) of Algorithm 1 and per-instance diagnostics; DEVICE pointers.
 *   z [B][Nmax+1][nx+nu]   primal stage vectors
 *   xi [B][Nmax+1][ng]     slacks (0 on hard rows)
 *   y_eq [B][Nmax+1][nx]   multipliers of x_0 = x_init (row 0) and f_{t} = 0 (row t+1)
 *   y_ineq [B][Nmax+1][ng] multipliers of the inequality rows (>0: upper side active)
 *   status [B], stats [B][TMPC_STATS] (may be NULL) */
typedef struct {
    float* z;
    float* xi;
    float* y_eq;
    float* y_ineq;
    int32_t* status;
    float* stats;
} tmpc_solution;

/* Gradients of a scalar loss with respect to the parameters (same layouts as the
 * parameters; any pointer may be NULL to skip that gradient). */
typedef struct {
    float* x0;      /* [B][nx]   */
    float* Qd;
    float* Rd;
    float* Wd;
    float* ref;
    float* lin;
    float* lo;
    float* hi;
    float* gamma2;
    float* gamma1;
} tmpc_grads;

typedef struct tmpc_handle tmpc_handle;

/* Default options: sigma 1e-6, rho0 0.1, rho in [1e-6, 1e6], alpha 1.6,
 * eps 1e-5, eps_g 1e-4, eta 0.4, k_rho 25 / ratio 5 (Section III-B), 1 SQP step,
 * 200 ADMM iterations, 8 line-search candidates, 3 Newton steps; backward
 * rho_b 1e4 (lowered tenfold, at most three times, if the FP32 factorisation
 * fails), sigma_b 1e-6, 30 refinement sweeps. */
void tmpc_default_options(tmpc_options* o);

/* Create a solver for the given layout and options and the parameter arrays p.
 * Allocates the whole workspace (stage blocks, factors of S, iterates) once;
 * later calls never allocate.  Reads p->N and p->model back to the host once
 * (synchronous) to order the work queue.  On failure *h is set to NULL.
 * Errors: INVALID_ARG (null h/d/o/p or inconsistent dims), OOM, CUDA, UNSUPPORTED. */
tmpc_status tmpc_setup(tmpc_handle** h, const tmpc_dims* d, const tmpc_options* o,
                       const tmpc_params* p);

/* Replace the parameter pointers (same layout, N and model values unchanged). */
tmpc_status tmpc_update_params(tmpc_handle* h, const tmpc_params* p);

/* Replace the options (same layout). */
tmpc_status tmpc_set_options(tmpc_handle* h, const tmpc_options* o);

/* Forward pass (Algorithm 1): solve every instance from x0 [B][nx] (DEVICE).
 * If warm_start != 0, out->z, out->xi, out->y_eq and out->y_ineq are read as
 * the initial primal-dual guess; otherwise the guess is the Newton rollout of
 * the reference controls.  The handle keeps nothing the caller needs: the
 * backward pass takes the solution arrays explicitly. */
tmpc_status tmpc_solve(tmpc_handle* h, const float* x0, tmpc_solution* out,
                       int32_t warm_start, void* stream);

/* Backward pass (Algorithm 2) at the solution sol (DEVICE arrays as written by
 * tmpc_solve for the same parameters and x0): given dL/dz [B][Nmax+1][nx+nu]
 * and optionally dL/dxi [B][Nmax+1][ng] (NULL = 0), writes the requested
 * gradients.  The active-set KKT system of Eq. (bwd:slack_reduced_system) is
 * solved by iterative refinement preconditioned with the regularised
 * block-tridiagonal matrix H + sigma_b I + rho_b (df'df + dgA'dgA) + gamma dgS'dgS,
 * factored by the same block factorisation as the forward S (bwd_iters sweeps).
 * The Hessian is the cost Hessian (the paper's Hessian approximation); it is
 * exact for linear dynamics.  sol->status receives per-instance flags
 * (NOT_PD / NAN) if non-NULL. */
tmpc_status tmpc_backward(tmpc_handle* h, const float* x0, const tmpc_solution* sol,
                          const float* dL_dz, const float* dL_dxi, tmpc_grads* g,
                          void* stream);

/* One entry per model group of tmpc_autotune (groups in the order of the
 * double integrator, bicycle, quadrotor and the generic kernel; unused entries
 * are not written). */
typedef struct {
    int32_t model;       /* model id of the group; -1: the generic kernel (not tuned)  */
    int32_t count;       /* instances in the group                                      */
    int32_t solver;      /* chosen launch form, as the codes of tmpc_options.solver     */
    int32_t threads;     /* threads per CTA                                             */
    int32_t cluster;     /* CTAs per thread-block cluster (form 6), else 0              */
    int32_t candidates;  /* forms timed                                                 */
    float ms;            /* mean device time of the chosen form per trial solve, ms    */
    float ms_default;    /* the same for the form chosen by tmpc_setup; -1 if untimed  */
} tmpc_tune_result;

/* Autotuner of the launch form (the fused, batched solve of Section III-E: one
 * persistent launch per model group).  For every group of the double
 * integrator, bicycle or quadrotor, times the group's forward solve from x0
 * [B][nx] (DEVICE) in each candidate form -- cyclic reduction with shared
 * arenas at 256 and 128 threads per CTA, the one-warp block LDL', cyclic
 * reduction with global arenas at 256 and 128 threads per CTA (the latter four
 * CTAs per SM), the plain per-phase form, and one cluster per
 * instance when the group is at most about one wave of clusters -- and keeps the
 * fastest for later tmpc_solve / tmpc_backward calls.
 *   init       (DEVICE, may be NULL) warm start of the trials: z, xi, y_eq and
 *              y_ineq are copied (not written) before each trial, as tmpc_solve
 *              with warm_start reads them; NULL starts each trial cold.
 *   reps       1..1000 timed passes.  The setup's form first runs until about
 *              20 ms of device time (clocks up); each form then runs once, forms
 *              four times slower than the fastest of these are dropped, and the
 *              rest run reps interleaved passes; a form's time is its fastest
 *              launch (CUDA events on stream, warm-start copy included).
 *   trial_sqp  > 0 caps the SQP iterations of the trials; 0 runs the handle's.
 *   res [4]    (HOST, may be NULL) one entry per group.
 * The choice minimises the forward solve; the backward follows it (shared-memory
 * backward for cyclic-reduction forms, the generic backward for LDL' forms).
 * Trial outputs go to buffers of the handle; caller arrays other than res are
 * not written.  Synchronous; may allocate (larger global arenas, plain-form
 * state, cluster flags).  A handle whose options fix the form (solver != 0) is
 * not changed (candidates = 0).
 * Errors: NOT_SETUP, INVALID_ARG (x0 NULL or misaligned, init incomplete, reps
 * or trial_sqp out of range), CUDA, OOM. */
tmpc_status tmpc_autotune(tmpc_handle* h, const float* x0, const tmpc_solution* init, int32_t reps,
                          int32_t trial_sqp, tmpc_tune_result* res, void* stream);

/* Device time of the last launches of a handle, one entry per model group of the
 * forward (the order of tmpc_tune_result) and, when the generic backward kernel
 * ran for instances outside the generic group, one more entry for it.  The paper
 * has no counterpart: it is the measurement hook of the roofline report, timing
 * each persistent kernel by CUDA events recorded on the stream it is launched on
 * (not recorded while that stream is being captured into a graph). */
typedef struct {
    int32_t model;   /* model id of the group; -1: the generic kernel                    */
    int32_t form;    /* launch form, as the codes of tmpc_options.solver                 */
    int32_t count;   /* instances                                                          */
    float fwd_ms;    /* the group's last forward launch(es), ms; -1 if not timed           */
    float bwd_ms;    /* the group's last backward launch, ms; -1 if not timed or none     */
} tmpc_group_time;

/* out [5] (HOST) receives *n_out entries.  Synchronises on the recorded events.
 * Errors: NOT_SETUP, INVALID_ARG (out or n_out NULL). */
tmpc_status tmpc_group_times(tmpc_handle* h, tmpc_group_time* out, int32_t* n_out);

/* Measurement helper with no counterpart in the paper: the FP32 FMA throughput of
 * the current device (TFLOP/s, an FMA counted as 2 flop), the denominator of the
 * roofline of the solve kernels, which are bound by FP32 issue.  Eight CTAs of 256
 * threads per SM each run eight independent FMA chains; three warm-up launches,
 * then the fastest of five, timed by CUDA events on a private stream.  tflops
 * (HOST, required) receives the rate, ms (HOST, may be NULL) the launch time.
 * Synchronous; allocates and frees a small device buffer.  Errors: INVALID_ARG
 * for a NULL tflops, OOM, CUDA. */
tmpc_status tmpc_fp32_fma_probe(float* tflops, float* ms);

/* End-to-end forward pass from HOST memory: copies the parameter arrays of
 * host_p and x0 (HOST pointers, pinned memory recommended) into device
 * buffers owned by the handle, solves, copies z, xi, y_eq, y_ineq, status and
 * stats back into the HOST arrays of host_out, and synchronises the stream
 * before returning.  z_init [B][Nmax+1][nx+nu] (HOST, may be NULL) is an
 * initial primal guess (slacks and multipliers start at zero); NULL starts
 * from the Newton rollout.  The handle's device parameter pointers are not
 * changed. */
tmpc_status tmpc_solve_host(tmpc_handle* h, const tmpc_params* host_p, const float* x0,
                            const float* z_init, tmpc_solution* host_out, void* stream);

/* Size of the device array that backs tmpc_solve_static (64 MiB per device). */
#define TMPC_STATIC_SCRATCH_BYTES (64u << 20)

/* Forward solve that allocates nothing.  The paper has no counterpart: it is an
 * entry point for callers that may not allocate device memory when they solve,
 * e.g. a control loop that must not block on the CUDA allocator or risk an
 * out-of-memory failure once it runs, or code running while another component
 * owns all device memory.  It computes the same SQP / ADMM solve as tmpc_setup +
 * tmpc_solve with solver 1 (the generic kernel), without a handle.
 *
 * d, o, p, x0, out: as for tmpc_setup / tmpc_solve (device pointers for p, x0
 * and out; out->status is required, out->stats may be NULL).  o->solver must be
 * 0 or 1, and either value runs the generic kernel (the shared-memory kernels
 * need a handle).  Scratch: the instance order, the work-queue counter and one
 * workspace per instance live in a file-scope device array of
 * TMPC_STATIC_SCRATCH_BYTES.  A batch whose scratch does not fit is rejected
 * with TMPC_ERR_INVALID_ARG before anything is enqueued, and so is a layout
 * whose per-instance workspace would exceed 2^31 floats; tmpc_last_error()
 * then gives the bytes it needs (about 81 KB per racing instance of N = 50).
 * Nothing in the scratch has to start at zero: the call's first kernel writes
 * the order and the counter before the solve kernel reads them.
 * Instance checks run on the device: an instance whose N or model does not fit
 * the layout gets status TMPC_INST_INVALID and zero outputs.
 * Set-up: the first call on a device (with that device current) looks up the
 * address of the scratch array once; make that first call before any stream
 * capture.  The scratch is shared by every caller on the device, so calls
 * whose work can overlap (other streams, other host threads) race on it and
 * corrupt each other's results: serialise them on one stream.  Instances run
 * in no fixed order; each instance's result does not depend on it. */
tmpc_status tmpc_solve_static(const tmpc_dims* d, const tmpc_options* o, const tmpc_params* p,
                              const float* x0, tmpc_solution* out, int32_t warm_start, void* stream);

/* Free the handle and its workspace (synchronises its allocations). NULL is a no-op. */
void tmpc_destroy(tmpc_handle* h);

/* Static description of a status code. */
const char* tmpc_status_string(tmpc_status s);

/* Last CUDA error text seen by the library on this thread (for TMPC_ERR_CUDA). */
const char* tmpc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TMPC_H */
