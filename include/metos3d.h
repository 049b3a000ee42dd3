/*
 * metos3d.h -- C ABI of the GB300 (sm_103a) implementation of the Transport Matrix
 * Method year map of Metos3D (Piwonski & Slawig, arXiv:1410.0204).
 *
 * The library advances marine biogeochemical tracers with the TMM time step of
 * Section 3,
 *     y_{j+1} = A_imp(t_j) ( A_exp(t_j) y_j + q_j(y_j, u) ),   j = 0 .. n_step - 1,
 * where A_exp and A_imp are linear interpolations in time of twelve monthly explicit
 * and implicit transport matrices, and iterates it over one model year (Section 4) as
 * the year map phi, y(T) = phi(y(0)), whose fixed point is the periodic solution.
 * q is the per-water-column source-minus-sink term of Section 5 (here the PO4-DOP
 * model of Section 2.2.1).
 *
 * Conventions shared by every call:
 *   - All arithmetic is IEEE FP64.
 *   - A tracer state is a device array of ntracer * n doubles in the layout
 *     [tracer][cell]; cells are ordered water column by water column, each column
 *     from the surface down (the interface's y(nlayer, ntracer), layer fastest).
 *   - State and parameter pointers passed to metos3d_step / metos3d_year_map are
 *     caller-owned DEVICE pointers; the library never frees them.  Work is enqueued
 *     on the context's stream; the calls return without waiting unless stated.
 *   - Every call returns an m3d_status and never lets an exception cross the ABI.
 *     metos3d_last_error(ctx) gives a message for the last failure on ctx
 *     (metos3d_last_error(NULL) for a failed metos3d_init).
 *   - A context is bound to one CUDA device (the current one at metos3d_init) and to
 *     one stream; it is not thread-safe.
 */
#ifndef METOS3D_H
#define METOS3D_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    M3D_OK = 0,
    M3D_NOT_CONVERGED = 1,      /* an iterative solve stopped before its tolerance */
    M3D_ERR_ARG = -1,           /* invalid argument or inconsistent input */
    M3D_ERR_CUDA = -2,          /* a CUDA runtime call failed */
    M3D_ERR_NONFINITE = -3,     /* a non-finite value appeared in the state */
    M3D_ERR_TIMEOUT = -4,       /* a bounded device-side wait ran out */
    M3D_ERR_UNSUPPORTED = -5    /* a valid request this build does not implement */
} m3d_status;

/*
 * Biogeochemical models (Section 2.2).  A single context (metos3d_init) runs every model: NONE
 * and NDOP with the tiled year kernels (and, for NDOP, the tangent and adjoint), N, PHY and
 * NPZD through a one-member ensemble (year map, steps, spin-up, the tangent year map by a
 * one-member tangent ensemble, Newton-Krylov with finite-difference or tangent products,
 * diagnostics).  Ensembles (metos3d_ensemble_init) run N, NDOP,
 * PHY and NPZD members side by side.  The parameters of each model are listed with the
 * ensemble calls below.
 */
enum {
    M3D_MODEL_NONE = 0,         /* q = 0: pure transport, any number of tracers */
    M3D_MODEL_N = 1,            /* PO4 alone, all production exported: 1 tracer, 5 parameters */
    M3D_MODEL_NDOP = 2,         /* PO4-DOP (Section 2.2.1): 2 tracers, 7 parameters */
    M3D_MODEL_PHY = 3,          /* PO4-DOP-PHY (Section 2.2.2): 3 tracers, 11 parameters */
    M3D_MODEL_NPZD = 5          /* NPZD-DOP: PO4-DOP-PHY with zooplankton grazing (Holling II) and
                                   sinking detritus: 5 tracers, 13 parameters */
};

#define M3D_MAX_LAYERS 64       /* deepest water column accepted */
#define M3D_MAX_TRACERS 8

typedef struct m3d_ctx m3d_ctx;   /* opaque; owned by the library */

/*
 * Ocean grid (host pointers; copied at init).  Water column c holds cells
 * col_start[c] .. col_start[c+1]-1, surface first; its layer count must not exceed
 * M3D_MAX_LAYERS.
 */
typedef struct {
    int n;                      /* wet cells */
    int ncol;                   /* water columns */
    const int *col_start;       /* [ncol+1], col_start[0] = 0, strictly increasing, col_start[ncol] = n */
    const double *h;            /* [n] layer thickness [m], > 0 (the interface's h) */
    const double *zc;           /* [n] depth of the layer centre [m] (the interface's d) */
    const double *vol;          /* [n] cell volume [m^3] (mass diagnostics) */
    const double *lat;          /* [ncol] latitude [degrees], in [-90, 90] */
} m3d_grid;

/*
 * Monthly transport matrices (Section 3; host pointers; copied and re-laid out at init).
 * Explicit: nmonth CSR matrices sharing one pattern (rows sorted, no duplicates).
 * Implicit: block diagonal by water column; month m holds, for each column c in order,
 * its dense L_c x L_c block in row-major order, s_imp = sum_c L_c^2 doubles per month.
 * Month m is centred at t = (m + 1/2) / nmonth of the year; between centres the
 * matrices are interpolated linearly, wrapping from the last month to the first.
 */
typedef struct {
    int nmonth;                 /* monthly matrices, >= 1 (12 in the paper) */
    int nnz;                    /* nonzeros of one explicit matrix */
    const int *exp_rowptr;      /* [n+1] */
    const int *exp_colidx;      /* [nnz] */
    const double *exp_val;      /* [nmonth][nnz] */
    long long s_imp;            /* sum over columns of L_c^2 */
    const double *imp_blk;      /* [nmonth][s_imp] */
} m3d_matrices;

/* Model and time discretisation. */
typedef struct {
    int model_id;               /* M3D_MODEL_* */
    int ntracer;                /* the model's count (N 1, NDOP 2, PHY 3, NPZD 5); 1..M3D_MAX_TRACERS for NONE */
    int nparam;                 /* the model's count (N 5, NDOP 7 -- see metos3d_bgc --, PHY 11, NPZD 13) */
    int nsub;                   /* internal model steps per ocean step, >= 1 (the paper's runs use 8) */
    int nstep;                  /* ocean steps per model year (2880 in the paper) */
} m3d_model;

/*
 * Create a context: validate and copy the grid, the matrices and the model onto the
 * current CUDA device, build the device layouts and the insolation table, and bind
 * the context to `stream` (a cudaStream_t; NULL = the legacy default stream).
 * Synchronous.  Returns M3D_ERR_ARG for inconsistent input (bad sizes, unsorted or
 * out-of-range CSR indices, block sizes not matching col_start, non-finite values).
 * On success *ctx must later be released with metos3d_free.
 */
m3d_status metos3d_init(m3d_ctx **ctx, const m3d_grid *grid, const m3d_matrices *mats,
                        const m3d_model *model, void *stream);

/* Rebind the context to another stream (a cudaStream_t). */
m3d_status metos3d_set_stream(m3d_ctx *ctx, void *stream);

/*
 * One TMM step j (Section 3): y_out = A_imp(t_j) (A_exp(t_j) y_in + q(y_in, u)),
 * t_j = j / nstep of the year, 0 <= j < nstep.  y_in, y_out: device [ntracer][n], must
 * not overlap.  u: device [nparam] model parameters.  Asynchronous.
 */
m3d_status metos3d_step(m3d_ctx *ctx, int j, const double *y_in, double *y_out,
                        const double *u);

/*
 * The year map phi (Section 4): nstep steps from y0, result in y1 (device [ntracer][n];
 * y0 and y1 may be the same array).  u: device [nparam].  Asynchronous; the first call
 * on a context builds its execution plan (do it before any stream capture).
 * A non-finite value in the result is reported by metos3d_check_finite.
 */
m3d_status metos3d_year_map(m3d_ctx *ctx, const double *y0, double *y1, const double *u);

/*
 * The year map with HOST arrays: copies y0 and u to the device, runs metos3d_year_map
 * and copies the result back into y1.  Synchronous.  Pinned host memory gives the
 * fastest copies.
 */
m3d_status metos3d_year_map_host(m3d_ctx *ctx, const double *y0_host, double *y1_host,
                                 const double *u_host);

/*
 * The year map and its tangent-linear map (Section 6 names exact Jacobian-vector products
 * by algorithmic differentiation as the alternative to finite differences):
 * phi_out = phi(y0) and jv_out = phi'(y0) v in one pass over the year, the state and its
 * direction advanced together through every step, so each matrix entry is read once for
 * both.  The source term's tangent is the model code evaluated on dual numbers.  Every
 * model: PO4-DOP by the tiled tangent kernels (or the linearised sweep, M3D_OPT_TANGENT_FORM),
 * N, PO4-DOP-PHY and NPZD-DOP by a one-member tangent ensemble (metos3d_ensemble_init_tangent;
 * synchronous for those, as it hands the parameters to the ensemble).  Device arrays
 * [ntracer][n]; u: device [nparam].  Asynchronous.
 */
m3d_status metos3d_year_tangent(m3d_ctx *ctx, const double *y0, const double *v, const double *u,
                                double *phi_out, double *jv_out);

/*
 * The adjoint of the year map, for gradients (the parameter optimisation of Sections 1 and 9;
 * exact derivatives by algorithmic differentiation, Section 6): for y1 = phi(y0; u) and a
 * cotangent ybar1, ybar0 = phi_y(y0; u)^T ybar1 (device [ntracer][n]; may alias ybar1) and
 * ubar = phi_u(y0; u)^T ybar1 (host [nparam], may be NULL), the gradient of <ybar1, y1>
 * with respect to the state and the model parameters.  The forward sweep keeps one
 * checkpoint every ckpt_every steps (<= 0: 240) and recomputes each segment before its
 * reverse sweep: about four year maps of work and ckpt_every + 1 states of memory,
 * allocated for the call.  ckpt_every >= nstep keeps the whole trajectory (nstep + 1
 * states; 2.4 GB for 52,749 cells and two tracers) and recomputes nothing, about three year
 * maps of work.  PO4-DOP by the tiled reverse kernels (see M3D_OPT_ADJOINT_PLAN); N,
 * PO4-DOP-PHY and NPZD-DOP by the context's one-member ensemble (metos3d_ensemble_year_adjoint,
 * whose checkpoint rule applies).  One internal step and a structurally symmetric explicit
 * pattern only (M3D_ERR_UNSUPPORTED otherwise).  Synchronous.
 */
m3d_status metos3d_year_adjoint(m3d_ctx *ctx, const double *y0, const double *u, const double *ybar1,
                                double *ybar0, double *ubar_host, int ckpt_every);

/*
 * Diagnostics, synchronous, result on the host:
 *   metos3d_mass:     sum over tracers and cells of vol_i y_{tr,i} (total tracer mass);
 *   metos3d_residual: || a - b ||_2 over all ntracer * n entries (the paper's spin-up and
 *                     Newton residual || y - phi(y) ||_2, Section 7);
 *   metos3d_check_finite: M3D_OK, or M3D_ERR_NONFINITE if y holds a NaN or infinity.
 */
m3d_status metos3d_mass(m3d_ctx *ctx, const double *y, double *mass_host);
m3d_status metos3d_residual(m3d_ctx *ctx, const double *a, const double *b, double *norm_host);
m3d_status metos3d_check_finite(m3d_ctx *ctx, const double *y);

/*
 * The biogeochemical model interface of Section 5.2, evaluated by the library's device
 * code on one water column, with HOST arrays (a check and debugging entry; the time
 * step uses the same device code):
 *   bgc(t, dt, lat, insol, dayfrac, ice, wind, ntracer, nlayer, h, d, salt, temp,
 *       y, ybgc, nparam, u)
 * y and ybgc are (nlayer, ntracer) arrays, layer index fastest.  ybgc receives the
 * increment of the model over the ocean step dt: nsub explicit Euler steps of length
 * dt / nsub with the forcing given.  For M3D_MODEL_NDOP, u = (k_w [1/m], alpha [1/d],
 * sigma [-], lambda [1/yr], K_N [mmol P/m^3], K_I [W/m^2], b [-]) and time is in years.
 * lat, dayfrac, wind, salt and temp are accepted and unused by this model; salt and
 * temp may be NULL.  Synchronous.  Returns M3D_ERR_ARG for bad sizes.
 */
m3d_status metos3d_bgc(int model_id, double t, double dt, double lat, double insol,
                       double dayfrac, double ice, double wind, int ntracer, int nlayer,
                       const double *h, const double *d, const double *salt,
                       const double *temp, const double *y, double *ybgc, int nparam,
                       const double *u, int nsub);

/*
 * || a - b ||_2 over len doubles (device arrays a, b), written to the device double
 * *norm_dev, without allocating anything.  The paper has no counterpart: this is the
 * metos3d_residual reduction for callers that cannot call cudaMalloc when they need the
 * norm: a process whose device memory is all handed out by another allocator with a
 * fixed budget (a framework's caching pool, a host application that sized its pools at
 * start-up) has none left to give, and a caller without a library context has no
 * context-owned scratch to lend.  It needs no context.
 * Its per-block partial sums live in one static device array of
 * M3D_RESIDUAL_STATIC_MAX_BLOCKS doubles (512 KiB), which every GPU that loads the
 * library keeps until the process exits; len may be at most
 * M3D_RESIDUAL_STATIC_MAX_BLOCKS * 2048 (about 134 million doubles), larger sizes
 * return M3D_ERR_ARG.  Asynchronous on `stream` (a cudaStream_t).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  All calls share the array, so calls that overlap on
 * the GPU (on different streams) race; calls on one stream are ordered and safe.
 * The message of the last failure is metos3d_residual_static_error().
 */
#define M3D_RESIDUAL_STATIC_MAX_BLOCKS 65536
m3d_status metos3d_residual_static(const double *a, const double *b, long long len, double *norm_dev,
                                   void *stream);
const char *metos3d_residual_static_error(void);

/*
 * Wait for the context's stream and report a failure of the last year map that can only be
 * seen on the device: M3D_ERR_TIMEOUT if the persistent year kernel gave up a bounded
 * wait (its tiles wait only for neighbouring tiles, at most the configured timeout; on
 * time-out they stop and the result is not valid).
 */
m3d_status metos3d_sync(m3d_ctx *ctx);

/*
 * Execution options (tuning and checks; the defaults need no setting):
 *   M3D_OPT_YEAR_PLAN:
 *       M3D_PLAN_RESIDENT (default when it fits): the year map is one cooperative launch;
 *       each tile of water columns keeps its month of matrices in shared memory, reloads
 *       them when the month changes, and synchronises with its neighbouring tiles through
 *       per-tile step counters;
 *       M3D_PLAN_PERSISTENT: the same launch with the matrices read from global memory
 *       every step (default when the matrices do not fit in shared memory);
 *       M3D_PLAN_GRAPH: one kernel launch per step, captured in a CUDA graph.
 *   M3D_OPT_WAIT_TIMEOUT_NS: bound of every device-side wait of the persistent kernel
 *       (default 2 s).
 *   M3D_OPT_TEST_WITHHOLD_TILE: for tests of the timeout path only: the given tile never
 *       announces its progress, so its neighbours' waits run out (-1: off, the default).
 *   M3D_OPT_NTILES (read only): number of tiles (CTAs) of a step.
 *   M3D_OPT_ADJOINT_PLAN: how metos3d_year_adjoint runs: M3D_PLAN_RESIDENT (default when it
 *       fits: the tiles' months of transposed operators in shared memory), or
 *       M3D_PLAN_PERSISTENT (default otherwise, e.g. on a 1-degree grid): a streaming sweep that
 *       reads the transposed operators from HBM every step and applies dense implicit blocks,
 *       its forward segments recomputed one step launch at a time; -1 when neither fits.
 *   M3D_OPT_IMPLICIT_FORM: M3D_IMPLICIT_TRIDIAGONAL (default when every monthly implicit
 *       block is, to 1e-11 relative, the inverse of a tridiagonal matrix, as a vertical
 *       diffusion (I - dt K)^{-1} is, and the plan in use can apply it): the interpolated
 *       implicit part is applied as (1 - w) z0 + w z1 with z_h solved by Thomas' algorithm
 *       from the two monthly tridiagonal factors, which equals the interpolated dense product
 *       up to rounding at a third of its FP64 work.  The resident kernel keeps the factors in
 *       shared memory; the persistent and graph plans read them from global memory (contexts
 *       of at most two tracers).  All plans give the same bits in either form.
 *       M3D_IMPLICIT_DENSE: the dense blocks.
 *   M3D_OPT_STEP_OPERATORS (resident plan): 1 keeps the explicit matrix of every step of the
 *       year, A_m + w_j (A_{m+1} - A_m) (Section 4), in device memory, computed once with the
 *       same fused multiply-add the year kernel would apply; the kernel then streams step j's
 *       values into shared memory (one bulk copy per tile and step, made during the implicit
 *       part of step j-1 from L2, where they were prefetched a step earlier) instead of
 *       interpolating every entry, which saves a third of the explicit part's FP64 work and
 *       gives bit-identical results.  Costs nstep x (explicit slot count) doubles
 *       (16.9 GB on the 128 x 64 x 15 grid).  Default 1 when that is at most an eighth of the
 *       free device memory at init, else 0.  Setting 1 allocates and computes the array
 *       (synchronous; M3D_ERR_CUDA if the allocation fails, M3D_ERR_UNSUPPORTED without the
 *       resident plan); 0 frees it.  The derivative sweeps use it for their forward parts.
 *       The first resident reverse sweep (metos3d_year_adjoint, metos3d_periodic_gradient)
 *       of a context that keeps them also builds the transposed operator of every step,
 *       A_j^T, the same size again, where it takes at most a quarter of the free device
 *       memory (else the sweep interpolates in the kernel); it is kept until 0 is set or the
 *       context is freed.
 *   M3D_OPT_STEP_OPERATOR_BYTES (read only): bytes held by the per-step operators (0 if none).
 *   M3D_OPT_TANGENT_FORM: how metos3d_year_tangent evaluates phi'(y) v.  M3D_TANGENT_DUAL
 *       (default): one sweep of the state and its perturbation together, the source term on
 *       dual numbers.  M3D_TANGENT_LINEARISED (PO4-DOP, one internal step, resident plan): the
 *       year map recording the source term's Jacobian df/dN of every euphotic cell and step
 *       (nstep x euphotic cells doubles, held by the context), then one sweep of the
 *       perturbation alone through the linearised step.  Newton-Krylov with tangent products
 *       uses the linearised sweep wherever it is available, whatever this option says: its
 *       line search records the Jacobian along the trajectory it evaluates anyway.
 *   M3D_OPT_KERNEL_TIMING: 1 records CUDA events on the context's stream around every launch
 *       of the year kernel (resident and persistent plans), default 0.
 *   M3D_OPT_LAST_KERNEL_NS (read only): device time of the last year-kernel launch timed that
 *       way, in nanoseconds; -1 if none was timed or it has not completed (synchronize first).
 * metos3d_get_option returns -1 for an unknown option.
 */
enum {
    M3D_OPT_YEAR_PLAN = 1,
    M3D_OPT_WAIT_TIMEOUT_NS = 2,
    M3D_OPT_TEST_WITHHOLD_TILE = 3,
    M3D_OPT_NTILES = 4,
    M3D_OPT_IMPLICIT_FORM = 5,
    M3D_OPT_ADJOINT_PLAN = 6,
    M3D_OPT_STEP_OPERATORS = 7,
    M3D_OPT_STEP_OPERATOR_BYTES = 8,
    M3D_OPT_KERNEL_TIMING = 9,
    M3D_OPT_LAST_KERNEL_NS = 10,
    M3D_OPT_TANGENT_FORM = 11
};
enum { M3D_TANGENT_DUAL = 0, M3D_TANGENT_LINEARISED = 1 };
enum { M3D_IMPLICIT_DENSE = 0, M3D_IMPLICIT_TRIDIAGONAL = 1 };
enum { M3D_PLAN_PERSISTENT = 0, M3D_PLAN_GRAPH = 1, M3D_PLAN_RESIDENT = 2 };
m3d_status metos3d_set_option(m3d_ctx *ctx, int option, long long value);
long long metos3d_get_option(const m3d_ctx *ctx, int option);

/*
 * Spin-up (Sections 4 and 7): the fixed-point iteration y <- phi(y) for up to nyears model
 * years, stopping early when ||phi(y) - y||_2 <= tol.  y: device [ntracer][n], updated in
 * place; u: device [nparam].  residuals_host (may be NULL) receives ||phi(y) - y||_2 of
 * every year; *years_done the number of years run.  Synchronous.
 */
m3d_status metos3d_spinup(m3d_ctx *ctx, double *y, const double *u, int nyears, double tol,
                          double *residuals_host, int *years_done);

/*
 * Matrix-free Newton-Krylov periodic solve (Sections 6 and 7): Newton's method on
 * F(y) = y - phi(y) = 0, globalised by a backtracking line search on f = |F|^2 / 2 with
 * quadratic (first backtrack) and cubic (later ones) interpolation (Armijo constant 1e-4,
 * steps kept in [0.1, 0.5] of the previous one; the slope of f along the step s is
 * F.J s = -(|F|^2 - rho^2), rho the GMRES residual of the step); each Newton system
 * (I - phi'(y)) s = -F(y) is solved by restarted GMRES with modified Gram-Schmidt
 * orthogonalisation to the Eisenstat-Walker tolerance (choice 2: eta_0 = 0.3,
 * gamma = 0.9, alpha = (1+sqrt 5)/2, safeguarded, kept within [0.5 tol/||F||, 0.9]).
 * A trial step whose residual is not finite (the state left the model's domain) is cut to a
 * tenth and gives the interpolation no point; no step length below 1e-4 is tried: the solve
 * then stops at its iterate (report->line_search_failed).
 * Jacobian-vector products are finite differences, J v = v - (phi(y + h v) - phi(y)) / h
 * with h = fd_eps ||y|| / ||v|| (M3D_JV_FD), or exact, J v = v - phi'(y) v by the tangent
 * year map (M3D_JV_TANGENT, see metos3d_year_tangent).  phi conserves the total mass, so I - phi' is singular and
 * the periodic solution is unique only for a given mass: each Newton step is projected on
 * the zero-mass directions, and the solution keeps the mass of the initial state.
 * y: device [ntracer][n], initial guess on entry and solution on exit; u: device [nparam];
 * opts NULL for the defaults (metos3d_newton_default_options); report may be NULL.
 * Returns M3D_NOT_CONVERGED (with the report filled in) if the tolerance is not met.
 * Synchronous; allocates its Krylov basis ((restart + 11) state vectors) for the call.  The
 * Krylov iterations run on the device (rotations and convergence test included); the host
 * reads their status one iteration late, so the GPU is never left waiting for it.
 */
enum { M3D_JV_FD = 0, M3D_JV_TANGENT = 1 };
typedef struct {
    double tol;                 /* ||y - phi(y)||_2 at which to stop (default 1e-8) */
    int max_newton;             /* Newton steps (default 40) */
    int restart;                /* GMRES restart length (default 200, the paper's) */
    int max_krylov;             /* GMRES iterations per Newton step (default 200) */
    int jv;                     /* M3D_JV_FD (default) or M3D_JV_TANGENT */
    double fd_eps;              /* relative finite-difference step (default 1e-8) */
    int line_search;            /* 1: backtracking line search (default); 0: full Newton steps */
} m3d_newton_opts;

#define M3D_NEWTON_MAX_HIST 64
#define M3D_NEWTON_MAX_TRIALS 512
typedef struct {
    int converged;
    int newton_steps;
    int krylov_total;           /* GMRES iterations over all Newton steps */
    int year_maps;              /* year maps evaluated (model-year equivalents) */
    int tangent_maps;           /* tangent year maps evaluated */
    double residual0, residual; /* ||F|| at the start and at the end */
    double residuals[M3D_NEWTON_MAX_HIST];   /* ||F|| after each Newton step ([0]: initial) */
    int krylov[M3D_NEWTON_MAX_HIST];         /* GMRES iterations of each Newton step */
    double lambdas[M3D_NEWTON_MAX_HIST];     /* accepted line-search step of each Newton step */
    double etas[M3D_NEWTON_MAX_HIST];        /* forcing term (GMRES tolerance) of each Newton step */
    double slopes[M3D_NEWTON_MAX_HIST];      /* slope of |F|^2 / 2 along each Newton step */
    int trials[M3D_NEWTON_MAX_HIST];         /* line-search trials of each Newton step */
    int ntrial;                              /* entries of trial_lambdas */
    double trial_lambdas[M3D_NEWTON_MAX_TRIALS];  /* every step length tried, in order */
    double seconds;
    int line_search_failed;     /* 1: the last step's line search found no decrease with a step
                                   length of 1e-4 or more; the solve stopped at its iterate (that
                                   step's lambda is 0) */
} m3d_newton_report;

void metos3d_newton_default_options(m3d_newton_opts *opts);
m3d_status metos3d_newton_solve(m3d_ctx *ctx, double *y, const double *u, const m3d_newton_opts *opts,
                                m3d_newton_report *report);

/*
 * Gradient at the periodic solution (the parameter optimisation of Sections 1 and 9, where
 * the misfit is evaluated on the periodic state ys(u) = phi(ys(u); u) that Newton's method
 * finds).  phi conserves mass, so ys(u) is defined for a fixed total mass: d ys / d u solves
 * (I - phi_y) dy = phi_u du with vol^T dy = 0 (vol repeated per tracer).  For a misfit J with
 * g = dJ/dy at ys, the implicit function theorem gives dJ/du = dJ/du|_y + (d ys / d u)^T g, and
 * the second term is computed by one adjoint solve:
 *     find lambda with vol^T lambda = 0 and P (I - phi_y^T) lambda = P g,
 *     P x = x - (vol^T x / vol^T vol) vol   (the projection on the zero-mass directions),
 * then ubar = phi_u^T lambda (lambda = 0 and ubar = 0 when ||P g|| <= 1e-13 ||g||: a g along
 * the mass direction alone, up to rounding).  The solve is restarted GMRES with modified Gram-Schmidt on the
 * zero-mass directions (where P (I - phi_y^T) is the adjoint of I - phi_y, invertible there
 * when the periodic solution is unique for its mass); each iteration is one reverse sweep of
 * the adjoint year map at ys, whose forward sweep runs once for the whole solve.
 *
 * ystar: device [ntracer][n], the periodic solution (e.g. from metos3d_newton_solve);
 * u: device [nparam]; g: device [ntracer][n]; lambda: device [ntracer][n] output (may be
 * NULL); ubar_host: host [nparam] output, (d ys / d u)^T g.  opts NULL for the defaults
 * (metos3d_gradient_default_options); report may be NULL.  PO4-DOP contexts only (it drives their
 * tiled reverse sweep; other models give M3D_ERR_UNSUPPORTED).  Returns M3D_NOT_CONVERGED (results and report filled in) if the
 * relative residual tolerance is not met within max_krylov iterations.  Synchronous;
 * allocates the Krylov basis ((restart + 11) state vectors) and the adjoint's trajectory
 * ((ckpt_every + 1) states; the default keeps the whole year, 2.4 GB for 52,749 cells and two
 * tracers) for the call.
 */
typedef struct {
    double tol;                 /* ||P g - P (I - phi_y^T) lambda|| / ||P g|| to reach (default 1e-8) */
    int restart;                /* GMRES restart length (default 200) */
    int max_krylov;             /* GMRES iterations in total (default 1000) */
    int ckpt_every;             /* adjoint checkpoints (default: nstep, the whole trajectory kept) */
} m3d_gradient_opts;

typedef struct {
    int converged;
    int krylov;                 /* GMRES iterations */
    int reverse_sweeps;         /* reverse sweeps of the adjoint year map */
    double forward_years;       /* forward steps run / nstep (1 with the default ckpt_every) */
    double residual;            /* final relative residual, recomputed from lambda */
    double seconds;
} m3d_gradient_report;

void metos3d_gradient_default_options(m3d_gradient_opts *opts);
m3d_status metos3d_periodic_gradient(m3d_ctx *ctx, const double *ystar, const double *u, const double *g,
                                     double *lambda, double *ubar_host, const m3d_gradient_opts *opts,
                                     m3d_gradient_report *report);

/*
 * Batched ensembles.  The paper's parameter studies and optimisations (Sections 1 and 9) run the
 * same transport for many parameter sets; an ensemble advances many members -- each with its
 * own model and parameters -- through the same TMM steps at once, so that every matrix entry
 * is read and interpolated once per step for all of them.  The members share the grid and the
 * matrices and nothing else: member m's result equals its own year map.
 *
 * Parameters of each model (host arrays, this order; rates per day unless stated):
 *   M3D_MODEL_N    (5):  k_w [1/m], alpha, K_N, K_I [W/m^2], b (Martin exponent)
 *   M3D_MODEL_NDOP (7):  as metos3d_bgc (lambda per year)
 *   M3D_MODEL_PHY  (11): mu_1, k_w, K_1, K_I, lambda'_2, sigma_2, lambda_3, kappa_3,
 *                        lambda'_3, sigma_3, b  (the order of the paper's table, Section 2.2.2)
 *   M3D_MODEL_NPZD (13): k_w, mu_P, K_N, K_I, mu_Z, K_P, epsilon, lambda_P, kappa_Z, lambda_Z,
 *                        lambda_D, lambda_DOP, w_D [m/day]
 * N is PO4-DOP without DOP (every production exported with Martin's law); NPZD-DOP grazes
 * phytoplankton by zooplankton (mu_Z Z P/(K_P + P), a fraction epsilon assimilated, the rest to
 * DOP), loses P (lambda_P) and Z (kappa_Z Z^2) to detritus, excretes Z to DOP (lambda_Z),
 * remineralises detritus to DOP (lambda_D) and DOP to PO4 (lambda_DOP), grows P only in the
 * two euphotic layers, and sinks detritus at w_D through the layer interfaces (not the floor).
 *
 * State: device [W][n], W = the members' tracer counts summed; member m's tracers are rows
 * offset_m .. offset_m + ntracer_m - 1 (offsets from metos3d_ensemble_layout), each in the
 * single-context layout.  Internally the tracers are packed into groups of 32 lanes (no
 * member split between groups) and stored cell-major.
 * The implicit matrices must be inverses of tridiagonal matrices (see M3D_IMPLICIT_TRIDIAGONAL);
 * otherwise init returns M3D_ERR_UNSUPPORTED.  An ensemble is bound to one device and one
 * stream and is not thread-safe.
 */
typedef struct m3d_ensemble m3d_ensemble;   /* opaque; owned by the library */
typedef struct {
    int model_id;               /* M3D_MODEL_N, _NDOP, _PHY or _NPZD */
    int nparam;                 /* the model's parameter count (above) */
    const double *u;            /* host [nparam], copied */
} m3d_member;

/*
 * Create an ensemble of nmember members (1 .. 4096) on the current device, bound to `stream`
 * (a cudaStream_t).  grid and mats as for metos3d_init; nsub internal model steps per ocean
 * step; nstep ocean steps per year.  Synchronous.  Chooses a default tiling; see
 * metos3d_ensemble_autotune.
 */
m3d_status metos3d_ensemble_init(m3d_ensemble **ens, const m3d_grid *grid, const m3d_matrices *mats,
                                 int nmember, const m3d_member *members, int nsub, int nstep,
                                 void *stream);

/*
 * A tangent ensemble (Section 6: exact derivatives, the tangent-linear model): every member
 * carries its state and a perturbation of it, and each step advances both, the perturbation
 * through the step's derivative (the models' source terms on dual numbers, the transport as
 * it is).  The state arrays of its calls are [2W][n]: rows 0 .. W-1 the members' states
 * (member m's at offset_m as above), rows W .. 2W-1 their perturbations in the same order.
 * metos3d_ensemble_year_map on it returns [phi(y); phi'(y) v] for every member at once, the
 * Jacobian-vector products of a Newton-Krylov solve per member.  Otherwise as
 * metos3d_ensemble_init (a member takes twice its tracer count of lanes).
 */
m3d_status metos3d_ensemble_init_tangent(m3d_ensemble **ens, const m3d_grid *grid, const m3d_matrices *mats,
                                         int nmember, const m3d_member *members, int nsub, int nstep,
                                         void *stream);

/*
 * Sizes: members, the state rows of the calls (W, the total tracer count; 2W for a tangent
 * ensemble), n, 32-lane groups.  offsets (may be NULL) receives nmember + 1 row offsets of
 * the members' states.
 */
m3d_status metos3d_ensemble_layout(const m3d_ensemble *ens, int *nmember, int *width, int *n,
                                   int *ngroup, int *offsets);

/* Rebind the ensemble to another stream (a cudaStream_t). */
m3d_status metos3d_ensemble_set_stream(m3d_ensemble *ens, void *stream);

/* Replace member m's parameters (host [nparam]); takes effect for the next step. Synchronous. */
m3d_status metos3d_ensemble_set_params(m3d_ensemble *ens, int member, const double *u_host);

/*
 * nsteps TMM steps (Section 3) of every member from step j0 (wrapping around the year):
 * Y1 = steps(Y0); device [W][n] arrays, may be the same.  One kernel launch per step.
 * Asynchronous.
 */
m3d_status metos3d_ensemble_steps(m3d_ensemble *ens, int j0, int nsteps, const double *Y0, double *Y1);

/*
 * The year map of every member (Section 4): nstep steps, one launch per step, the year
 * captured once as a CUDA graph and replayed.  Y0, Y1: device [W][n] (may be the same).
 * Asynchronous; the first call builds the graph (do it before any stream capture).
 */
m3d_status metos3d_ensemble_year_map(m3d_ensemble *ens, const double *Y0, double *Y1);

/*
 * Tiling of the step kernel: each CTA takes cols_per_block consecutive water columns (it
 * interpolates their matrix rows once per step) and warps_per_block warps that take one
 * (column, 32-lane group) at a time.  M3D_ERR_ARG when it does not fit in shared memory.
 */
m3d_status metos3d_ensemble_set_tiling(m3d_ensemble *ens, int cols_per_block, int warps_per_block);
m3d_status metos3d_ensemble_get_tiling(const m3d_ensemble *ens, int *cols_per_block, int *warps_per_block);

/*
 * Autotuner: time nsteps steps from the state Y (device [W][n], not modified) for each
 * candidate tiling (columns per block 1..32, warps per block 4..16, as shared memory allows),
 * keep the fastest and return it with its time per step.  Synchronous.
 */
m3d_status metos3d_ensemble_autotune(m3d_ensemble *ens, const double *Y, int nsteps,
                                     int *cols_per_block, int *warps_per_block, double *ms_per_step);

/*
 * The adjoint of every member's year map (the gradients of the parameter optimisation of
 * Sections 1 and 9, by hand-written reverse models, Section 6): for Y1 = phi(Y0) and the
 * cotangents Ybar1, Ybar0 = phi_y^T Ybar1 per member (device [W][n]; may alias Ybar1) and
 * ubar_host = phi_u^T Ybar1 (host, the members' parameters in member order, each in its
 * model's parameter order, sum of the nparam; may be NULL).  The forward sweep keeps a
 * checkpoint every ckpt_every steps (<= 0: 240); each segment is recomputed before its
 * reverse steps, keeping every state of the segment when that fits in half of the free
 * device memory and otherwise a second level of checkpoints inside it.  Two launches per
 * reverse step (the transposed implicit part; the transposed explicit part with the reverse
 * source terms).  Plain ensembles (not tangent) with one internal model step and a
 * structurally symmetric explicit pattern (M3D_ERR_UNSUPPORTED otherwise).  Allocates its
 * checkpoints for the call.  Synchronous.
 */
m3d_status metos3d_ensemble_year_adjoint(m3d_ensemble *ens, const double *Y0, const double *Ybar1,
                                         double *Ybar0, double *ubar_host, int ckpt_every);

/*
 * The periodic solve of every member of an ensemble (Sections 4, 6, 7): for each member m,
 * Newton-Krylov on F_m(y_m) = y_m - phi_m(y_m) exactly as metos3d_newton_solve states it (its
 * own GMRES(MGS) cycle to its Eisenstat-Walker tolerance, zero-mass projection of its step,
 * its own backtracking line search), all members advancing in lockstep.  One Krylov
 * iteration of all members takes one year map of ens_tan (a tangent ensemble of the same
 * members: metos3d_ensemble_init_tangent) for opts->jv = M3D_JV_TANGENT, or one year map of
 * ens at y + h v for M3D_JV_FD; a line-search trial of all members is one year map of ens.
 * A member that has converged stops iterating while the others go on.  The restart length
 * is min(restart, max_krylov), one cycle per Newton step.  Y: device [W][n] (ens's layout),
 * the initial states on entry and the solutions on exit; vol_host: host [n] cell volumes (for
 * the zero-mass projection); reports: host [nmember] (may be NULL), each with the member's
 * counts (year_maps and tangent_maps count the ensemble year maps, shared by all members).
 * Allocates (restart + 10) ensemble states for the call.  Synchronous; returns
 * M3D_NOT_CONVERGED unless every member reached the tolerance.
 */
m3d_status metos3d_ensemble_newton_solve(m3d_ensemble *ens, m3d_ensemble *ens_tan, double *Y,
                                         const double *vol_host, const m3d_newton_opts *opts,
                                         m3d_newton_report *reports);

/* Kernel launches of the last steps, year-map or adjoint call. */
long long metos3d_ensemble_last_launch_count(const m3d_ensemble *ens);

/* Message for the last failure on ens, or on metos3d_ensemble_init when ens is NULL. */
const char *metos3d_ensemble_last_error(const m3d_ensemble *ens);

/* Release an ensemble and its device memory.  NULL is accepted. */
void metos3d_ensemble_free(m3d_ensemble *ens);

/* Sizes of a context: n, ncol, ntracer, nstep (any pointer may be NULL). */
m3d_status metos3d_info(const m3d_ctx *ctx, int *n, int *ncol, int *ntracer, int *nstep);

/* Number of kernel launches the last metos3d_year_map issued (prologue included). */
long long metos3d_last_launch_count(const m3d_ctx *ctx);

/* Message for the last failure on ctx, or on metos3d_init when ctx is NULL. */
const char *metos3d_last_error(const m3d_ctx *ctx);

/* Release a context and all device memory it owns.  NULL is accepted. */
void metos3d_free(m3d_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* METOS3D_H */
