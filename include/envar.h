/*
 * envar.h -- C ABI of the GB300 (sm_103a) EnVar open-cavity library.
 *
 * The library advances an ensemble of forced 2-D incompressible Navier-Stokes
 * open-cavity simulations on one GPU, accumulates each member's fluctuation
 * cost, and projects the cost anomalies onto the control perturbations to give
 * the ensemble-variational (EnVar) gradient of arXiv 2605.23812:
 *
 *   f   = f_e + E w                               Sec. 3.3.1, Eq. (ensemble_representation), f_e = 0
 *   J(w)= 1/2 ||y - H q(E w)||^2 + (N-1)/2 w^T w  Eq. (J_w), R = I, y = 0 (Sec. 4.1)
 *   Y_i ~ (H q(E w + eps E_i) - H q(E w)) / eps   Eq. (fdapprox)
 *   dJ/dw = Y^T (H q - y) + (N-1) w               Eq. (gradient_EnVar)
 *   w  <- w + dw                                  Sec. 3.3.1 (weight update); dw = -alpha g/(N-1)
 *
 * Every call runs its work in the library's own CUDA kernels on the stream
 * given to envar_init; there is no CPU fallback.
 *
 * Conventions shared by all calls
 *  - Return value: 0 on success, a negative ENVAR_E* code on failure.  The
 *    message of the last failure is returned by envar_last_error(h).
 *  - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA memory),
 *    owned by the caller, and must stay valid until the call's stream work has
 *    finished.  Pointers named *_host are host pointers; calls that write them
 *    synchronise the stream before returning.
 *  - Field layouts (row-major, float64): u is [ny][nx+1] (x-velocity on
 *    vertical faces), v is [ny+1][nx] (y-velocity on horizontal faces), p is
 *    [ny][nx] (cell centres).
 *  - Control vectors have n_ctrl = 2 * n_cc entries: [fx over control cells,
 *    fy over control cells]; control cells are the fluid cells whose centre
 *    lies in cfg.region (inclusive), ordered row-major (y outer, x inner).
 *    E is n_ctrl x N, column-major (column k contiguous).
 *  - A handle is not thread-safe; calls on one handle are stream-ordered.
 */
#ifndef ENVAR_H
#define ENVAR_H

#ifdef __cplusplus
extern "C" {
#endif

#define ENVAR_ABI_VERSION 4

enum {
    ENVAR_OK = 0,
    ENVAR_EINVAL = -1,     /* bad argument or configuration */
    ENVAR_ENOMEM = -2,     /* device allocation failed */
    ENVAR_ECUDA = -3,      /* CUDA runtime error */
    ENVAR_ESTATE = -4,     /* call out of order (e.g. envar_cost before a forward run) */
    ENVAR_EDEVICE = -5     /* device is not an sm_103 GPU */
};

/* Precision / batching of the forward ensemble (batching and precision). */
enum {
    ENVAR_FP64_PLAIN = 0,   /* one member at a time, all arithmetic FP64 */
    ENVAR_FP64_BATCHED = 1, /* all N+1 members per launch, all arithmetic FP64 */
    ENVAR_MIXED = 2         /* all members per launch; FP32 tendencies, FP32 multigrid and inner
                               CG vectors, whose dot products accumulate FP32 products (pairs
                               rounded once) in df64; velocity state, predictor, Poisson
                               right-hand side and solution, the outer Poisson residual of the
                               iterative refinement and the Welford cost accumulators in double-float
                               (df64: a pair of floats, about 48 significant bits, on the FP32 pipe);
                               per-block partial sums, member costs and the gradient in FP64.  The
                               outer refinement stops at the same divergence tolerance (div_tol) as
                               the FP64 modes. */
};

/* Observation operator H of Sec. 4.1. */
enum {
    ENVAR_COST_DOMAIN = 0,  /* J = 1/(2 n_w) sum_t sum_cells |u'|^2 dx dy  (Eq. kinenergy / n_w) */
    ENVAR_COST_SENSORS = 1  /* J = 1/2 sum_{sensors, t} |u'(x_s, t)|^2, x_s = 1/5..4/5, y = 0
                               (Eq. specific_cost_function) */
};

/* Per-member status bits (envar_member_status). */
enum {
    ENVAR_ST_NONFINITE = 1,     /* NaN or Inf met in the velocity */
    ENVAR_ST_DIVERGENCE = 2,    /* pressure solve ended above div_tol */
    ENVAR_ST_CFL = 4,           /* |u| dt / h exceeded 1 */
    ENVAR_ST_ADJOINT = 8        /* an adjoint Poisson solve ended above its tolerance */
};

typedef struct envar_config {
    int nx, ny;              /* cells; nx, ny even, nx >= 8, ny >= 4 */
    double x0, x1, y0, y1;   /* box; the cavity is [0,1] x [y0,0] with fluid above y = 0 */
    double Re;               /* Reynolds number U D / nu (Sec. 2) */
    double cfl;              /* dt = cfl * min(dx, dy) / U, U = 1 */
    double inlet_delta;      /* inlet u = erf(y / inlet_delta) above the lip, v = 0 */
    double conv_speed;       /* convective outflow speed */
    int n_steps;             /* time steps per forward evaluation (warm-up + window) */
    int n_window;            /* the last n_window steps form the cost window (Sec. 4.1) */
    int n_members;           /* N_ens, ensemble perturbations; N+1 forward runs */
    double region[4];        /* control region [x0, x1, y0, y1] (Sec. 4.1) */
    double sigma;            /* prior standard deviation (Eq. covarianceB, sigma_i = sigma) */
    double corr_len;         /* a_x = a_y (Eq. covarianceB), c_xy = infinity */
    double eps;              /* finite-difference step of Eq. (fdapprox) */
    unsigned long long seed; /* ensemble seed (Philox4x64-10 key) */
    int precision;           /* ENVAR_FP64_PLAIN / ENVAR_FP64_BATCHED / ENVAR_MIXED */
    int cost_mode;           /* ENVAR_COST_DOMAIN / ENVAR_COST_SENSORS */
    double div_tol;          /* pressure solve stops when max |D u^{n+1}| <= div_tol */
    int max_outer;           /* cap on FP64 residual refinements per time step */
    int max_inner;           /* cap on inner preconditioned-CG iterations per refinement */
    double inner_rtol;       /* inner CG stops when r^T z <= inner_rtol^2 * r0^T z0 */
    int nu_pre, nu_post;     /* red-black Gauss-Seidel sweeps before / after coarse correction */
    int coarse_sweeps;       /* symmetric sweep pairs on the coarsest multigrid level */
    int steps_per_graph;     /* time steps per captured CUDA graph (even) */
    int member_groups;       /* batched runs: member groups whose time steps run as concurrent
                                branches of the captured graph; 0 = automatic (4 from 24 member
                                slots, 2 from 8), 1 .. 8 */
    int lip_slip;            /* 1: the lower wall of the channel (y = 0) is free slip outside
                                noslip_span and no slip inside it (the slip segments of Sec. 4.4);
                                0: no slip everywhere */
    double noslip_span[2];   /* x range of the no-slip part of the lower wall (default -0.4, 1.75) */
    int forcing_y_only;      /* 1: forcing in the y-momentum equation only (Sec. 4.1): the prior
                                variance of the fx entries is zero, so the drawn or eigenvector
                                ensemble has zero fx rows */
    int conditional_refinement; /* 1 (default): in the captured time step the pressure solve's
                                refinement loop is a conditional WHILE graph node, run as often as
                                the slowest member of the group needs (at most max_outer); 0: the
                                loop is unrolled to max_outer refinements */
    int guess_extrapolation; /* MIXED, 1 (default): the pressure increment's initial guess is the
                                linear extrapolation 2 dp^n - dp^(n-1) of the last two increments
                                (both re-centred on their fluid mean) from the third step on, the
                                last increment before; 0: the last increment.  Only the number
                                of refinements changes: every solve still ends at div_tol */
    int nu_coarse;           /* smoothing sweep pairs on the multigrid levels below the finest one
                                (pre- and post-smoothing alike, so the V-cycle stays symmetric);
                                0 (default): nu_pre / nu_post on every level; 1 .. 3 */
} envar_config;

typedef struct envar_handle_s *envar_handle;

/* Fill *cfg with the library defaults for an nx x ny open-cavity grid. */
int envar_default_config(envar_config *cfg, int nx, int ny);

/* Create a handle: checks the device (sm_103), builds the geometry and multigrid
 * hierarchy on the device, allocates all internal buffers (owned by the handle,
 * freed by envar_destroy), and draws the ensemble E from N(0, B) with the
 * seeded white-noise convolution sampler (Sec. 3.3.2, Eq. covarianceB).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream). */
int envar_init(envar_handle *h, const envar_config *cfg, void *cuda_stream);

/* Release every resource of the handle (NULL is accepted). */
int envar_destroy(envar_handle h);

/* Message of the last failure on this handle (or of the last envar_init failure
 * when h is NULL).  Static storage inside the handle; valid until the next call. */
const char *envar_last_error(envar_handle h);

/* Sizes: n_ctrl (= 2 x control cells), number of forward members in flight,
 * multigrid levels, and dt.  Any pointer may be NULL. */
int envar_sizes(envar_handle h, int *n_ctrl, int *n_cc, int *n_levels, double *dt);

/* Initial state shared by all members (raw fields; the library applies the wall,
 * inlet and outlet rules when loading them).  u0_dev [ny][nx+1], v0_dev [ny+1][nx]. */
int envar_set_initial_state(envar_handle h, const double *u0_dev, const double *v0_dev);

/* Replace the ensemble matrix (n_ctrl x N column-major, device). */
int envar_set_ensemble(envar_handle h, const double *E_dev, int n_ctrl, int N);
/* Copy the ensemble matrix out (n_ctrl x N column-major, device). */
int envar_get_ensemble(envar_handle h, double *E_dev);

/* Replace E by the eigenvector ensemble of Sec. 3.3.2: B = U Sigma U^T with U^T M_f U = I and
 * E = U_N Sigma_N^{1/2} sqrt(N-1) (Eq. eigenvm1), B the prior covariance of Eq. (covarianceB) on the
 * control cells (sigma_i = sigma, a_x = a_y = corr_len, c_xy = infinity).  On the uniform grid
 * M_f = dx dy I drops out, so the members are sqrt(lambda_k (N-1)) v_k for the Euclidean eigenpairs
 * of the one-component covariance B_s; both forcing components share B_s, and the members take its
 * eigenvectors in decreasing eigenvalue order, each first as an fx field (member 2r) and then as an
 * fy field (member 2r+1), or, with forcing_y_only, only as fy fields (member r); each eigenvector's
 * largest-magnitude entry is positive.  The eigenpairs
 * come from Lanczos with full reorthogonalisation on B_s applied through its Kronecker factors
 * (B_s is never formed) and a Jacobi diagonalisation of the projected matrix.  lambda_host
 * (nullable): N doubles, the eigenvalue of each member.  Allocates and frees temporary device memory. */
int envar_eigen_ensemble(envar_handle h, double *lambda_host);

/* N+1 forward evaluations of Fig. (envar_loop): member 0 with forcing E w,
 * member i with E w + eps E_i (Eq. fdapprox), each over n_steps from the
 * initial state, accumulating the window cost in-kernel (Welford for DOMAIN,
 * sensor samples for SENSORS).  w_dev: N doubles (device). */
int envar_forward_ensemble(envar_handle h, const double *w_dev);

/* Observation costs of the last forward run: J_host[N+1] (member 0 first) and
 * J_prior = (N-1)/2 w^T w of Eq. (J_w) for the w of that run (either may be NULL). */
int envar_cost(envar_handle h, double *J_host, double *J_prior_host);

/* EnVar gradient of Eq. (gradient_EnVar) for the last forward run: g_host[N],
 *   g = Y^T (Hq_0 - y) + (N-1) w,  Y_i = (H q_i - H q_0)/eps  (Eq. fdapprox),  R = I, y = 0.
 * SENSORS: H q_m = the sensor series of member m minus its window mean; the contraction runs over
 *   the 8 n_window observations.
 * DOMAIN: H q_m = sqrt(dx dy / n_w) (cell-centred velocity minus its window mean) over every fluid
 *   cell and window step; the forward run accumulates, per cell and member, the Welford sums of
 *   d = u_m - u_0, so Y_i^T h_0 = (J_i - J_0 - 1/2 ||h_i - h_0||^2)/eps exactly (no (eps/2)||Y_i||^2
 *   term of the scalar-anomaly form).
 * A perturbed member whose status word is nonzero (envar_member_status) contributes no column of
 * Y: its component is (N-1) w_i; envar_excluded_members counts them.  ENVAR_ESTATE if the
 * unperturbed member 0 failed.  df_dev (nullable, n_ctrl doubles, device) receives E g / (N-1). */
int envar_gradient(envar_handle h, double *g_host, double *df_dev);

/* The scalar-anomaly form of the same gradient, g_i = (J_i - J_0)/eps + (N-1) w_i
 * (= Y_i^T (Hq_0 - y) + (eps/2)||Y_i||^2 + (N-1) w_i), for comparison: g_host[N].  Excluded
 * members as in envar_gradient. */
int envar_gradient_scalar(envar_handle h, double *g_host);

/* Number of perturbed members of the last forward run left out of the gradient (nonzero status). */
int envar_excluded_members(envar_handle h, int *count);

/* One EnVar iteration: forward ensemble at w, costs, gradient (envar_gradient), and the update
 * w <- w - alpha g / (N-1) (Sec. 3.3.1 weight update with the prior-Hessian
 * step).  w_inout_host: N doubles (host, in/out).  J0_out_host (nullable):
 * total cost J(w) = J_obs(member 0) + J_prior before the update.  ENVAR_ESTATE (w unchanged)
 * if the unperturbed member failed. */
int envar_step(envar_handle h, double alpha, double *w_inout_host, double *J0_out_host);

/* envar_step with device-resident w_inout_dev (N doubles) and J0_out_dev (nullable, 1 double):
 * no host copy of the step's inputs or results, and no host synchronisation, so a failed
 * unperturbed member is not detected here: check envar_member_status after the step. */
int envar_step_device(envar_handle h, double alpha, double *w_inout_dev, double *J0_out_dev);

/* Gauss-Newton EnVar iteration (Sec. 3.3.1, Eq. Hessian_EnVar and Eq. update_Newton): forward
 * ensemble at w, the sensor-space Y of Eq. (fdapprox) (members with a nonzero status word give a
 * zero column), H_GN = Y^T R^{-1} Y + (N-1) I with R = I, g of Eq. (gradient_EnVar), and
 * w <- w - alpha H_GN^{-1} g (alpha = 1: the full Gauss-Newton step).  Needs the SENSORS cost.
 * w_inout_host: N doubles (host, in/out).  J0_out_host (nullable): J(w) before the update.
 * ENVAR_ESTATE (w unchanged) if member 0 failed or H_GN is not positive definite. */
int envar_gn_step(envar_handle h, double alpha, double *w_inout_host, double *J0_out_host);

/* H_GN = Y^T Y + (N-1) I of the last forward run (N x N row-major, host); SENSORS cost only. */
int envar_gn_hessian(envar_handle h, double *H_host);

/* Limited-memory BFGS EnVar iteration (Sec. 3.3.1, Eq. update_BFGS): forward ensemble at w and g;
 * the pair (w - w_prev, g - g_prev) of the previous call joins the history when its curvature is
 * positive; the direction p = -H g comes from the two-loop recursion over the newest `memory`
 * pairs on the initial matrix (s^T y / y^T y) I, or (1/(N-1)) I without pairs (the inverse prior
 * Hessian); the step length a = 1, 1/2, 1/4, ... (at most 12 trials) is the first that meets the
 * Armijo condition J(w + a p) <= J(w) + 1e-4 a g^T p, each trial cost J = J_obs + (N-1)/2 w^T w
 * from one forward run of the unperturbed member alone.  Either cost mode.
 * w_inout_host: N doubles (host, in/out).  J0_out_host (nullable): J(w) before the update;
 * alpha_out_host (nullable): the accepted step length, 0 if no trial met the condition (then w is
 * unchanged: it is stationary to the accuracy of J, and no pair is pending); evals_out_host
 * (nullable): trial runs.  ENVAR_ESTATE (w unchanged) if member 0 failed.  Leaves member slot 0
 * holding the last trial run. */
int envar_lbfgs_step(envar_handle h, double *w_inout_host, double *J0_out_host, double *alpha_out_host,
                     int *evals_out_host);

/* Clear the L-BFGS history and set its length (1 .. 64 pairs; the first envar_lbfgs_step uses 8). */
int envar_lbfgs_reset(envar_handle h, int memory);

/* Run ONE member with a given control vector f (n_ctrl doubles, device) over
 * n_steps and return its observation cost (host).  Member slot 0 is used. */
int envar_forward_control(envar_handle h, const double *f_dev, double *J_host);

/* Per-member status words (ENVAR_ST_* bits) of the last forward run: N+1 ints (host). */
int envar_member_status(envar_handle h, int *status_host);

/* Final state of member m of the last forward run (device pointers, compact
 * layouts above; p is mean-zero over fluid cells).  Any pointer may be NULL. */
int envar_get_state(envar_handle h, int member, double *u_dev, double *v_dev, double *p_dev);

/* Sensor samples of member m over the window: [n_window][8] = (u, v) at the 4
 * sensors, host. */
int envar_get_series(envar_handle h, int member, double *series_host);

/* Diagnostics of the last forward run: max |D u| over all members and steps,
 * and total pressure-refinement / inner-CG iterations summed over steps and
 * members (host; any pointer may be NULL). */
int envar_diagnostics(envar_handle h, double *max_div, long long *outer_its, long long *inner_its);

/* Advance the members' current state by n_steps without resetting it (the
 * forcing of the last forward run stays in place).  For step-level timing and
 * trajectory tests: call envar_forward_ensemble(h, w) with n_steps set in the
 * configuration first, or envar_reset_members(h, w) to load the initial state. */
int envar_reset_members(envar_handle h, const double *w_dev);
int envar_advance(envar_handle h, int n_steps);

/* Kernels launched by this library in this process so far: direct launches plus the
 * kernel nodes of every CUDA-graph replay (h is unused and may be NULL). */
int envar_kernel_launches(envar_handle h, long long *count);

/* Time one hot-path kernel over all member slots: two untimed launches, then `reps`
 * launches on the handle's stream, each preceded by a 256 MB write that evicts the L2 and
 * timed alone between CUDA events; *ms_per_launch receives the mean.  The first call
 * allocates the 256 MB eviction buffer (kept by the handle).  which: 0 momentum predictor (in MIXED handles fused
 * with the Poisson right-hand side), 1 level-0 pre-smoothing + restriction,
 * 2 level-0 prolongation + post-smoothing + dot product, 3 inner SpMV, 4 inner AXPY,
 * 5 outer residual (FP64, or df64 in MIXED handles: block partials only, no totals), 6 projection
 * correction with the Welford update, 7 coarse-level
 * block kernel, 8 Poisson right-hand side (MIXED: the fused predictor).  Overwrites the members' state: call
 * envar_reset_members or a forward run before using the state again. */
int envar_time_kernel(envar_handle h, int which, int reps, double *ms_per_launch);

/* Apply the pressure solve's multigrid preconditioner once, z = M r, to a level-0 cell field of
 * member slot 0 (r_dev, z_dev: [ny][nx] float64, device; solid cells of r must be zero).  M is
 * one symmetric V-cycle (red-black Gauss-Seidel, cell-sum restriction, piecewise-constant
 * prolongation) and must be symmetric positive definite on mean-zero fields.  Overwrites the
 * solver's work vectors of every member slot. */
int envar_apply_preconditioner(envar_handle h, const double *r_dev, double *z_dev);

/* Reference gradient by the discrete adjoint (Sec. 3.2, Eq. adjoint_discrete and
 * Eq. gradient_forcing, in their discrete form): the exact gradient of the DOMAIN cost J(f) of one
 * forward run from the handle's initial state, with the steady forcing f on the control cells,
 * with respect to f.  The reverse sweep transposes every step of the FP64 stepper -- AB2
 * predictor with its boundary rules, convective outlet with the flux shift, projection (one
 * adjoint Poisson solve per step, the same multigrid-preconditioned CG) -- and accumulates
 * dJ/dF = sum_n dt lambda_n on the forced faces, then maps it to the control cells (each cell
 * takes half of each of its forced faces, the transpose of the forcing map).
 * f_dev: n_ctrl float64 on the device, [fx over control cells | fy over control cells], the layout
 * of one column of E.  gf_dev: n_ctrl float64 on the device (written).  J_host: the cost, or NULL.
 * max_snapshots >= 1: forward states kept on the device (about 6 (nx+1)(ny+1) doubles each); with
 * fewer than n_steps, the binomial checkpoint schedule recomputes the forward in between (at most
 * r forward passes for n_steps <= C(max_snapshots + r, r)).  Needs an FP64 handle
 * (ENVAR_FP64_PLAIN or ENVAR_FP64_BATCHED), the DOMAIN cost, n_window >= 1 and an initial state.
 * Uses and overwrites member slot 0 (state, Welford planes, cost).  Errors: ENVAR_EINVAL for a
 * wrong handle kind or argument, ENVAR_ENOMEM when the checkpoints do not fit, ENVAR_ESTATE when a
 * forward step or an adjoint solve failed (non-finite state, CFL, unconverged solve). */
int envar_adjoint_gradient(envar_handle h, const double *f_dev, double *gf_dev, int max_snapshots, double *J_host);

/* H^1 smoothing of a control-space gradient (Sec. 4.2, Eq. lsob): (I - l_sob^2 Lap) gs = (1 + l_sob^2) g
 * for each forcing component, Lap the 5-point Laplacian on the control cells with no flux through the
 * boundary of the control set (a neighbour outside it contributes nothing).  g_dev, gs_dev: n_ctrl
 * doubles (device), layout of a column of E.  Conjugate gradients to 1e-13 relative residual; ENVAR_ESTATE
 * if that is not reached. */
int envar_h1_smooth(envar_handle h, const double *g_dev, double *gs_dev, double l_sob);

/* One iteration of the adjoint approach (Sec. 3.2, the paragraph after Eq. gradient_forcing, with the
 * regularisation of Sec. 4.2): J(f) and dJ/df by envar_adjoint_gradient (DOMAIN cost, no prior term:
 * the deterministic statement of the problem), the L2 gradient dJ/df / (dx dy) (M_f = dx dy I on the
 * uniform grid), its H^1 smoothing with length l_sob (Eq. lsob; the paper uses 0.02), and an L-BFGS
 * update of f along p = -H g_H1 from the newest pairs (f - f_prev, g_H1 - g_H1_prev) (at most 8 unless
 * envar_adjoint_lbfgs_reset set otherwise).  The step length is the first of a0, a0/2, ... (at most 12
 * trials, each one forward run of member slot 0) that meets the Armijo condition
 * J(f + a p) <= J(f) + 1e-4 a (dJ/df . p); a0 = 1 with curvature pairs, else the length that moves f
 * by first_step in the max norm.  f_inout_dev: n_ctrl doubles (device, in/out).  J_out_host (nullable):
 * J(f) before the update; alpha_out_host, evals_out_host (nullable): step length (0, with f
 * unchanged, if no trial met the condition: f is stationary to the accuracy of J) and trial runs.
 * Needs what envar_adjoint_gradient needs. */
int envar_adjoint_lbfgs_step(envar_handle h, double *f_inout_dev, int max_snapshots, double l_sob, double first_step,
                             double *J_out_host, double *alpha_out_host, int *evals_out_host);

/* Clear the history of envar_adjoint_lbfgs_step and set its length (1 .. 64 pairs). */
int envar_adjoint_lbfgs_reset(envar_handle h, int memory);

/* Counters of the last envar_adjoint_gradient call: forward steps run (initial sweep included),
 * reverse steps, checkpoint stores and restores. */
int envar_adjoint_stats(envar_handle h, long long *forward_steps, long long *reverse_steps, long long *stores,
                        long long *restores);

/* Host only, no device needed: the checkpoint schedule envar_adjoint_gradient uses for n_steps
 * steps and n_slots snapshots (clamped to n_steps), run dry and checked (every step reversed once,
 * in order, each from its own forward state).  recompute: forward steps beyond the initial sweep;
 * stores, restores: checkpoint copies.  Returns ENVAR_ESTATE if the check fails. */
int envar_revolve_plan(long long n_steps, int n_slots, long long *recompute, long long *stores, long long *restores);

/* Pick the fastest pressure-solve parameters for this handle on this GPU: for each candidate of a
 * fixed list of seventeen (refinement cap, inner-iteration cap and tolerance, smoothing sweep pairs
 * on the finest and on the coarser levels, coarse sweeps) run all member slots probe_steps time steps from the initial state with the current
 * forcing, and keep the fastest candidate under which no member reports a status bit (every solve
 * met div_tol).  The divergence tolerance itself is not a candidate parameter: results change only
 * within it.  *best_ms_per_step (may be NULL): the winner's time per step; chosen (may be NULL,
 * 4 ints): max_outer, max_inner, nu_pre (= nu_post), coarse_sweeps; the rest of the choice
 * (inner_rtol, nu_coarse) is in envar_get_config.  Overwrites the members' state
 * and recaptures the step graphs.  ENVAR_ESTATE (parameters unchanged) if no candidate qualifies. */
int envar_autotune(envar_handle h, int probe_steps, double *best_ms_per_step, int *chosen);

/* The handle's configuration as currently used (after envar_autotune, its solver parameters). */
int envar_get_config(envar_handle h, envar_config *cfg);

/* Batches of uneven member groups (members of uneven grid sizes and horizons advancing
 * together).  A batch advances several batched handles -- each its own grid size, Reynolds
 * number, horizon, ensemble and solver parameters (tune each with envar_autotune first) -- in one
 * captured CUDA graph per chunk, which holds the next c_k time steps of every handle k as parallel
 * branches (each handle's member groups branch further).  c_k = n_steps_k / n_chunks with n_chunks
 * the largest common divisor of the horizons that leaves at least 10 steps per chunk to the shortest
 * one (or all of it if shorter), so every handle ends on the last chunk.  The graph is captured at the
 * first envar_batch_forward; create a new batch after changing a handle's solver parameters. */
typedef struct envar_batch_s *envar_batch;

/* handles: n distinct batched handles (FP64_BATCHED or MIXED), kept by the caller and valid for the
 * batch's lifetime.  cuda_stream: the batch's stream (NULL: a new one).  ENVAR_EINVAL if the
 * horizons share no common step that keeps a chunk under 400 steps of the longest horizon. */
int envar_batch_create(envar_batch *b, envar_handle *handles, int n, void *cuda_stream);
int envar_batch_destroy(envar_batch b);

/* The N_k + 1 forward runs of every handle of the batch (envar_forward_ensemble of each, run
 * together): w_devs[k] is handle k's weights (N_k doubles, device).  Afterwards envar_cost,
 * envar_gradient and the other per-run queries of each handle refer to this run.  Synchronises
 * every handle's stream. */
int envar_batch_forward(envar_batch b, const double *const *w_devs);

/* Chunks per forward run and, per handle (n ints, nullable), time steps per chunk. */
int envar_batch_info(envar_batch b, int *n_chunks, int *steps_per_chunk);

/* Draw the ensemble matrix E without allocating device memory.  The paper has no counterpart:
 * this is for callers that cannot let a library call cudaMalloc (a framework whose caching
 * allocator owns the device, a fixed memory budget, code that must avoid the synchronisation of
 * cudaFree).  It writes the same E as envar_init + envar_get_ensemble for the same configuration
 * (n_ctrl x N column-major, E_dev caller-owned device memory) and uses as scratch a file-scope
 * device array of ENVAR_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until exit.
 * No cudaMalloc / cudaFree or allocating library routine is called.  The first call on a device
 * (with that device current) looks up the array's device address.  Every call copies from host
 * memory and synchronises its stream, so no call may be made while its stream (or, in global
 * capture mode, any stream) is being captured.  All calls share the array: calls that overlap on
 * the GPU race.  Configurations needing
 * more scratch than the maximum are rejected (ENVAR_EINVAL); the message of a failure is returned
 * by envar_last_error(NULL).  Runs on cuda_stream (NULL = legacy default) and synchronises it. */
#define ENVAR_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
int envar_draw_ensemble_noalloc(const envar_config *cfg, double *E_dev, int n_ctrl, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ENVAR_H */
