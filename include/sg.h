/*
 * sg.h -- C ABI of a single-GPU (GB300, sm_103a) RKL-multigrid Poisson solver.
 *
 * Solves the Poisson equation  grad^2 phi = 4 pi G rho  (Sec. 2.2.1, Eq.
 * poisson_eqaution) on a uniform cell-centred Cartesian grid, as the steady
 * state of d phi / dt = grad^2 phi - 4 pi G rho advanced by s-stage
 * Runge-Kutta-Legendre super-time-steps (App. A, Eqs. RKL_intermediate_source),
 * used both as the smoother and as the coarsest-grid solver of a
 * correction-scheme multigrid V-cycle (Sec. 2.1).
 *
 * Conventions shared by every call
 * --------------------------------
 * Layout.   Every 3D array is dense C order [nz][ny][nx] (x fastest), float64,
 *           without ghost cells.  Cell centres are lo + (i + 1/2) h, with
 *           h_d = (hi_d - lo_d) / n_d.
 * Faces.    Dirichlet boundary values (Sec. 2.3, Eq. solution_ghost) come as six
 *           arrays in the order -x, +x, -y, +y, -z, +z; the x faces are
 *           [nz][ny], the y faces [nz][nx], the z faces [ny][nx], sampled at the
 *           centres of the boundary faces.  Unset faces are zero.
 * Memory.   `on_device = 1`: the pointer is CUDA device memory on the grid's
 *           device; `on_device = 0`: host memory (pageable or pinned), moved
 *           by copy-engine transfers (with the option host_copy =
 *           SG_HOST_COPY_KERNEL, pinned memory mapped into the device address
 *           space is read or written by the library's kernels over the CPU-GPU
 *           link instead); a host buffer must hold the whole array.  Caller
 *           buffers are borrowed for the duration of the call only.  All work is
 *           ordered on the CUDA stream given to sg_create_grid; calls that
 *           return data to a host pointer synchronise that stream, calls that
 *           return data to a device pointer do not.
 * Ownership. The grid owns every device buffer it allocates (cudaMalloc at
 *           creation and, for the adjoint, at the first sg_backward); they are
 *           freed by sg_destroy.
 * Errors.   Every call returns an sg_status.  Nothing throws or exits across
 *           the ABI.  On an error the output buffers are left untouched unless
 *           stated otherwise, and sg_last_error() returns a message (thread
 *           local, valid until the next call on the same thread).
 * Threads.  A grid may be used by one host thread at a time.  Different
 *           grids may be created and used from different host threads at the
 *           same time, each on its own stream (the library's one-time setup
 *           and plan caches are locked); their solves then share the device
 *           (sg_residual_restrict_noalloc excepted: see its note).
 */
#ifndef SG_H
#define SG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_grid sg_grid;                 /* opaque solver state */

typedef enum sg_status {
    SG_OK = 0,
    SG_ERR_ARG = 1,              /* invalid argument (sizes, levels, options) */
    SG_ERR_CUDA = 2,             /* a CUDA runtime call failed */
    SG_ERR_OOM = 3,              /* device allocation failed */
    SG_ERR_NOT_CONVERGED = 4,    /* max_cycles reached above the tolerance (result kept) */
    SG_ERR_TIMEOUT = 5,          /* a bounded device wait ran out */
    SG_ERR_NONFINITE = 6,        /* the residual norm became NaN or Inf */
    SG_ERR_STATE = 7             /* call out of order (e.g. potential before solve) */
} sg_status;

typedef enum sg_bc {
    SG_BC_DIRICHLET = 0,         /* Eq. solution_ghost on level 0, Eq. error_ghost below */
    SG_BC_PERIODIC = 1           /* Eq. periodic on every level */
} sg_bc;

typedef enum sg_smoother {
    SG_SMOOTH_RKL = 0,           /* RKL super-steps of s_smooth stages (App. A) */
    SG_SMOOTH_GSRB = 1           /* red-black Gauss-Seidel / SOR sweeps (Sec. 2.2.4, App. B) */
} sg_smoother;

typedef enum sg_staging {
    SG_STAGE_CP_ASYNC = 0,       /* fused super-step planes staged by per-strip asynchronous copies */
    SG_STAGE_TMA = 1             /* ... by tensor-map box copies completing on an mbarrier */
} sg_staging;

typedef enum sg_host_copy {
    SG_HOST_COPY_ENGINE = 0,     /* host buffers moved by copy-engine transfers on the grid's stream */
    SG_HOST_COPY_KERNEL = 1      /* pinned, mapped host buffers read / written by kernels over the link */
} sg_host_copy;

typedef enum sg_precision {
    SG_FP64 = 0,                 /* every sweep in FP64 */
    SG_MIXED = 1                 /* FP32 V-cycle on the error equation inside an FP64
                                    residual / defect-correction loop */
} sg_precision;

/* Solver options.  sg_default_options fills the defaults noted here. */
typedef struct sg_options {
    int    rkl_order;       /* smoother order, 1 or 2                              [2]  */
    int    s_smooth;        /* stages per smoothing super-step; RKL2 needs >= 2     [3]  */
    double tau_frac;        /* smoother tau / tau_max, in (0, 1]                    [1.0]*/
    int    n_pre;           /* smoothing super-steps on the way down (Sec. 4.1)     [2]  */
    int    n_post;          /* smoothing super-steps on the way up                  [1]  */
    double coarse_tol;      /* coarsest solve: stop at this relative residual;
                               0 runs exactly coarse_max_ss super-steps             [1e-2]*/
    int    coarse_max_ss;   /* coarsest solve: cap on super-steps                   [64] */
    double coarse_tau_frac; /* coarsest solve tau / tau_max; 0 = cos^2(pi / 2N)     [0]  */
    int    max_cycles;      /* V-cycle (or single-level super-step / sweep) cap,
                               1 .. 10^7                                        [100]*/
    int    single_s;        /* levels == 1: fixed s; 0 = Legendre-zero schedule
                               (App. A.5); -1 = App. A.4's global s_opt of the
                               grid's largest extent (sg_plan_s_opt)             [0]  */
    double single_tau_frac; /* levels == 1: tau / tau_max; 0 = cos^2(pi / 2N)       [0]  */
    int    fixed_cycles;    /* > 0: run exactly this many cycles (<= 10^7), ignore tol [0] */
    int    use_graph;       /* 1: the whole solve as one CUDA graph, the cycle loop
                               on the device (WHILE nodes); 2: each V-cycle
                               replayed as a captured graph, the loop on the host
                               (a profiler that cannot see into graphs with
                               conditional nodes sees every kernel); 0: kernels
                               launched one by one                               [1]  */
    int    fused;           /* fused multi-stage super-step kernels where possible  [1]  */
    int    smoother;        /* sg_smoother.  With SG_SMOOTH_GSRB one relaxation
                               (n_pre, n_post) is one red-black sweep, every cell
                               solving its own row (Dirichlet ghost folded into the
                               diagonal), the even cells (i + j + k) first; levels == 1
                               runs one sweep per cycle (App. B's single-level GS /
                               SOR); the coarsest level keeps the RKL1 schedule; the
                               fused and cluster kernels are not used; periodic axes
                               need even extents on the swept levels (SG_ERR_ARG
                               from sg_solve otherwise)                        [RKL]*/
    double omega;           /* GS-RB relaxation factor in [0, 2): 1 = Gauss-Seidel,
                               (1, 2) SOR, 0 = App. B's SOR omega of each level:
                               2 / (1 + sqrt(1 - rho_J^2)), rho_J = sum_d cos(pi/n_d)
                               / h_d^2 over sum_d 1 / h_d^2                   [1.0]*/
    double max_residual_tol;/* > 0: stop when max |L phi - f| <= this (App. B's
                               test) instead of the relative L2 test; tol is then
                               ignored                                          [0]  */
    int    tile_rows;       /* rows of the tile of the fused s = 2, 3 super-step:
                               14 or 16; 0 = the launcher's cost model (the plan
                               whose busiest SM has the least work)           [0]  */
    int    inner_n_pre;     /* smoothing super-steps on the way down on levels
                               1 .. L-2; -1 = n_pre (the paper's N_pre on every
                               level)                                           [-1] */
    int    inner_n_post;    /* the same on the way up; -1 = n_post             [-1] */
    int    staging;         /* sg_staging: how the fused s = 2, 3 super-step stages
                               its planes in shared memory.  SG_STAGE_TMA: two
                               tensor-map box copies per field and plane, issued
                               by one thread, completing on an mbarrier (waits
                               bounded), halo cells past a wall rebuilt from
                               their mirrors; it needs no wrap in x and y,
                               nx % 4 == 0 and an even ny (other levels stage by
                               per-strip copies)                  [SG_STAGE_CP_ASYNC]*/
    int    host_copy;       /* sg_host_copy: how host (on_device = 0) buffers cross
                               the CPU-GPU link.  SG_HOST_COPY_ENGINE: copy-engine
                               transfers (the density's 4 pi G scaling then a device
                               pass), which leave every SM to solves running on
                               other streams.  SG_HOST_COPY_KERNEL: pinned, mapped
                               buffers (cudaHostAlloc / cudaHostRegister) are read
                               and written by kernels directly, the scaling in the
                               same pass -- a little faster for one solve at a
                               time, but those kernels hold SMs while the link
                               transfers; pageable buffers use the copy engines
                               either way.  The same bits in both modes
                                                              [SG_HOST_COPY_ENGINE]*/
} sg_options;

#define SG_MAX_HISTORY 256

/* Filled by sg_solve / sg_backward when the pointer is not NULL. */
typedef struct sg_solve_info {
    int    status;                      /* the sg_status of the call */
    int    cycles;                      /* V-cycles (or super-steps when levels == 1) run */
    int    levels;                      /* multigrid levels used */
    int    s_smooth;                    /* smoother stages used */
    int    rkl_order;                   /* smoother order used */
    int    precision;                   /* sg_precision used */
    double r0;                          /* ||L 0 - f||_2 (volume-weighted L2, Sec. 4.1) */
    double rel_residual;                /* final ||L phi - f||_2 / r0 */
    double max_residual;                /* final max |L phi - f| */
    double history[SG_MAX_HISTORY];     /* rel. residual before cycle m (m = 0..cycles;
                                           the first SG_MAX_HISTORY are kept) */
    int    coarse_ss[SG_MAX_HISTORY];   /* coarsest-level super-steps in cycle m (likewise) */
    double elapsed_ms;                  /* device time of the solve (CUDA events) */
    long long stage_cell_updates;       /* sum over levels of cells x RKL stages */
    long long kernel_launches;          /* kernels launched by the solve */
} sg_solve_info;

/* Fill *opt with the defaults listed in sg_options.  Never fails for a non-NULL opt. */
sg_status sg_default_options(sg_options* opt);

/*
 * Create a solver grid of nx x ny x nz cells on the box [lo, hi] (lo[d] < hi[d],
 * order x, y, z) with per-axis boundary kinds bc[3] (sg_bc values) and the
 * given precision, on CUDA stream `cuda_stream` (a cudaStream_t) of the current
 * device.  NULL (the legacy default stream, which cannot be captured into a CUDA
 * graph) makes the grid create and use a private blocking stream, which the
 * legacy default stream orders implicitly.  Sizes: 2 <= n_d <= 4096,
 * total cells <= 2^31 - 1.  Allocates all level buffers for the deepest
 * hierarchy the level rule allows (Sec. 4.1: N / 2^(L-1) even on every axis).
 * Errors: SG_ERR_ARG, SG_ERR_OOM, SG_ERR_CUDA; *out is set only on SG_OK.
 */
sg_status sg_create_grid(int nx, int ny, int nz, const double lo[3], const double hi[3],
                         const int bc[3], int precision, void* cuda_stream, sg_grid** out);

/*
 * Create a two-dimensional solver grid of nx x ny cells on the rectangle
 * [lo, hi] (order x, y), boundary kinds bc[2], for the 2D variants of Sec. 2.2:
 * the five-point Laplacian (Eq. discrete_laplace_2D), the 4-cell restriction
 * (Eqs. restriction_equation_2D, restriction_example_2D) and the 9/3/3/1
 * prolongation (Eq. prolongation_example_2D), with the same V-cycle, RKL
 * stages, coarsest solve and ghost rules (Sec. 2.3) as the 3D grid.  Every
 * other call takes the grid as a 3D grid with nz = 1: arrays are [1][ny][nx]
 * = [ny][nx]; faces -x, +x are [ny], -y, +y are [nx]; the z faces are unused
 * (pass NULL).  Level rule of Sec. 4.1 on x and y.  The fused super-step and
 * cluster kernels are 3D-only; a 2D grid runs the per-stage kernels.  Sizes:
 * 2 <= n_d <= 65536, nx * ny <= 2^31 - 1.  Errors as sg_create_grid.
 */
sg_status sg_create_grid_2d(int nx, int ny, const double lo[2], const double hi[2], const int bc[2], int precision,
                            void* cuda_stream, sg_grid** out);

/* Replace the grid's options (copied).  SG_ERR_ARG if a field is out of range. */
sg_status sg_set_options(sg_grid* g, const sg_options* opt);

/* Read the grid's current options into *opt. */
sg_status sg_get_options(const sg_grid* g, sg_options* opt);

/*
 * Dirichlet boundary potential on the six faces (Sec. 2.3, Eq. solution_ghost:
 * ghost = 2 phi_face - phi_active on the finest level).  faces[f] may be NULL
 * (that face is zero).  Faces of periodic axes are ignored.
 */
sg_status sg_set_boundary(sg_grid* g, const double* const faces[6], int on_device);

/*
 * Source of the solve: f = four_pi_G * rho, with rho -> rho - mean(rho) when
 * every axis is periodic (Sec. 2.3, Eq. source_modification).  rho is
 * [nz][ny][nx].  Resets the initial guess to zero.
 */
sg_status sg_set_density(sg_grid* g, const double* rho, int on_device, double four_pi_G);

/* Optional warm start: initial guess for the next sg_solve (Sec. 4.1 end). */
sg_status sg_set_potential_guess(sg_grid* g, const double* phi, int on_device);

/*
 * Solve (Sec. 2.1): repeat V-cycles until ||L phi - f||_2 / ||L 0 - f||_2 <= tol
 * (Sec. 4.1 norm) or max_cycles.  s > 0 overrides options.s_smooth (for
 * levels == 1: the fixed stage count; 0 = the Legendre-zero schedule of App.
 * A.5).  levels = 0 uses the level rule; 1 <= levels <= that maximum otherwise
 * (SG_ERR_ARG beyond it).  tol must be >= 0.  Returns SG_ERR_NOT_CONVERGED
 * (potential kept) when max_cycles is reached above tol, SG_ERR_NONFINITE on a
 * NaN/Inf residual.  With periodic axes on every side the potential is
 * returned with zero mean.  With use_graph = 1 (the default) and a coarsest
 * level that fits one CTA, the cycles run as one CUDA graph with the loop on
 * the device (the graph is captured once per option set and kept); the host
 * reads the loop's state once when it has finished.
 */
sg_status sg_solve(sg_grid* g, double tol, int s, int levels, sg_solve_info* info);

/* Copy the potential of the last solve into phi_out ([nz][ny][nx]).  SG_ERR_STATE before a solve. */
sg_status sg_potential(sg_grid* g, double* phi_out, int on_device);

/*
 * Gravitational acceleration g = -grad phi by the fourth-order central
 * difference of Sec. 3, Eq. 4thorder_acceleration, along each axis:
 *   g_d = -(4/3) (phi_{+1} - phi_{-1}) / (2 h_d) + (1/3) (phi_{+2} - phi_{-2}) / (4 h_d).
 * phi: NULL for the potential of the last solve (SG_ERR_STATE before one), or
 * a caller potential [nz][ny][nx].  g_out: [3][nz][ny][nx] float64, the x
 * component first.  on_device = 1: phi (when given) and g_out are device
 * pointers and the call is stream-ordered on the grid's stream; 0: host
 * memory, copied in and out (device staging allocated on first use).  The
 * stencil reaches two cells past a wall: on Dirichlet axes both ghost layers
 * reflect through the grid's face values (ghost m = 2 phi_face - the m-th cell
 * from the wall, m = 1, 2; zero faces when none were set), periodic axes wrap.
 * g_out must not overlap phi.
 * Errors: SG_ERR_ARG (NULL g or g_out, overlap), SG_ERR_STATE (phi NULL before any
 * solve), SG_ERR_CUDA (a CUDA call failed, the staging allocation included).
 */
sg_status sg_gravity(sg_grid* g, const double* phi, double* g_out, int on_device);

/*
 * Adjoint of the solve for a loss L(phi): given dL/dphi, return
 * dL/drho = four_pi_G * lambda with L_h lambda = dL/dphi under homogeneous
 * boundaries (the discrete operator is symmetric, so it is its own adjoint; the
 * Dirichlet data do not depend on rho).  Periodic: dL/dphi and the result are
 * projected to zero mean.  Solved to relative residual `tol` with the grid's
 * options and level count of the last solve.  Uses its own buffers: the forward
 * potential is not disturbed.  four_pi_G is the one given to sg_set_density.
 */
sg_status sg_backward(sg_grid* g, const double* dL_dphi, double* dL_drho, int on_device,
                      double tol, sg_solve_info* info);

/*
 * Solve n independent grids (each with its density, boundary and options set;
 * sizes may differ) to tolerance tol, with the levels of each grid's rule.
 * The whole batch is one CUDA graph launch on the first grid's stream: one
 * branch per grid, each its cycle loop on the device (a WHILE node repeating
 * the V-cycle while a one-thread kernel finds the residual above tol), so the
 * kernels of small grids run concurrently, a grid that converges leaves its
 * loop without a host round trip, and the host reads the loop states once at
 * the end.  The graph is kept and launched again while the same grids (with
 * the same options) come back.  Grids whose loop cannot run on the device
 * (one level, a coarsest level too large for one CTA, use_graph != 1,
 * profiling on) are solved one after the other first.
 * Each grid keeps its own stopping rule and info.  infos may be NULL or an
 * array of n entries.  A grid may appear only once.  Returns the first
 * non-OK status.
 */
sg_status sg_solve_batch(sg_grid* const* grids, int n, double tol, sg_solve_info* infos);

/* One candidate of sg_autotune and what it measured. */
typedef struct sg_tune_entry {
    int    rkl_order;          /* smoother order tried */
    int    s_smooth;           /* stages per smoothing super-step tried */
    int    fused;              /* fused (temporally blocked) super-steps on or off */
    double tau_frac;           /* smoother tau / tau_max tried */
    double ms_per_cycle;       /* measured device time per V-cycle */
    double factor;             /* residual reduction per V-cycle: measured over cycles 2..6,
                                  or the smoother's factor on the checkerboard mode raised to
                                  n_pre + n_post when larger (that mode bounds the asymptotic
                                  rate: the coarse grid does not see it) */
    double ms_per_decade;      /* ms_per_cycle / -log10(factor): the score (lower is better) */
    int    n_pre, n_post;      /* smoothing super-steps per V-cycle tried */
    int    tile_rows;          /* tile rows of the fused super-step tried (0: cost model) */
    int    inner_n_pre, inner_n_post;   /* smoothing counts of levels 1 .. L-2 tried (-1: n_pre, n_post) */
} sg_tune_entry;

/*
 * Pick the smoother for this grid and its current density by measurement: for
 * every candidate (RKL order 1 and 2 -- or only the current order when
 * keep_order is 1 --, s = 2..6, a few tau fractions, fused on and off, and
 * (N_pre, N_post) = (2, 1), (3, 2), (4, 3) or (5, 3), on levels 1 .. L-2 the
 * same or (2, 1), and for the fused s = 2, 3 super-step both tile shapes,
 * 32 x 14 and 32 x 16) run
 * two and six V-cycles at `levels` (0 = the level rule), take the difference
 * of their CUDA-event times (so per-solve set-up drops out) and score the time
 * per decade of residual reduction over cycles 2..6, bounded below by the
 * smoother's damping of the checkerboard mode (sg_tune_entry.factor); the best
 * candidate is written into the grid's options (smoother = SG_SMOOTH_RKL).  The trial cycles overwrite the potential
 * (call before sg_solve).  table (may be NULL) receives up to cap entries,
 * *count the number tried.  The App. A.4 spectral analysis motivates the
 * search: the best s balances the cost of s stages against the reduction of
 * the modes the smoother must damp.
 */
sg_status sg_autotune(sg_grid* g, int levels, int keep_order, sg_tune_entry* table, int cap, int* count);

/* Free the grid and its device buffers.  NULL is a no-op. */
void sg_destroy(sg_grid* g);

/* Message for the last error on this thread ("" if none). */
const char* sg_last_error(void);

/* Maximum number of levels the level rule allows for this grid. */
int sg_max_levels(const sg_grid* g);

/* ------------------------------------------------------------------------
 * Host-side planning: the numbers the solver computes on the host before it
 * launches anything.  No device work; callable without a GPU.
 * ------------------------------------------------------------------------ */

/* The first `count` entries of the Legendre-zero schedule of App. A.5 for a
 * level whose largest extent is N: s_k = Round(2.4048 / pi * N / k - 1/2),
 * halves rounded up, for k = N/2 .. 1, a k skipped when its s repeats the
 * previous one, then s_1 repeated (at least 1 each).  The coarsest-level and
 * single-level solves run it.  SG_ERR_ARG for N < 1, count < 0, or s_out NULL
 * with count > 0. */
sg_status sg_plan_schedule(int N, int count, int* s_out);

/* The stage coefficients the kernels run for one s-stage super-step of order 1
 * (RKL1) or 2 (RKL2) (App. A, Eq. RKL_intermediate_source): arrays of s + 1
 * entries, entry j = 1..s (entry 0 unused): mu_j, nu_j, mu~_j (mut) and
 * gamma~_j (gt, zero for RKL1); *tau_max_over_dtpar = tau_max / dt_par.  Any
 * output may be NULL.  SG_ERR_ARG for order not 1 or 2, s < 1 (RKL1), s < 2
 * (RKL2) or s > 100000. */
sg_status sg_plan_stage_coefficients(int order, int s, double* mu, double* nu, double* mut, double* gt,
                                     double* tau_max_over_dtpar);

/* Measurement aid (no counterpart in the paper): the FP64 FMA throughput of
 * the current device in TFLOP/s (2 flops per FMA), from eight independent FMA
 * chains per thread on every SM, timed by CUDA events after a warm-up launch;
 * *ms (may be NULL) receives the timed launch's duration.  It is the ceiling of
 * the FP64 kernels (the FP64 solve's stages, the acceleration), whose
 * roofline is min(HBM, this rate).  Allocates and frees a small buffer;
 * synchronises the device's legacy stream.  SG_ERR_ARG for NULL tflops,
 * SG_ERR_CUDA on a CUDA error. */
sg_status sg_measure_fp64_rate(double* tflops, double* ms);

/* App. A.4's single fixed stage count s_opt for a level whose largest extent is
 * N (Eqs. eigenvalue_RKL, spectral_rad_RKL, sopt_theory and the two-step search
 * that follows them): the s in [first zero of P_s(cos(pi / N)), N] with the
 * smallest spectral radius max_{1 <= k <= min(6, N/2)} |P_s(cos(k pi / N))|, the
 * first such s on ties.  levels == 1 with single_s = -1 runs it.  SG_ERR_ARG
 * for N < 2, N > 10^6 or s_out NULL. */
sg_status sg_plan_s_opt(int N, int* s_out);

/* Largest level count of the level rule (Sec. 4.1: N / 2^(L-1) even on every
 * axis) for nx x ny x nz cells; 0 for a size below 1. */
int sg_plan_levels(int nx, int ny, int nz);

/* App. B's SOR omega = 2 / (1 + sqrt(1 - rho_J^2)) for nx x ny x nz cells on the
 * box [lo, hi], rho_J = sum_d cos(pi / n_d) / h_d^2 over sum_d 1 / h_d^2.
 * SG_ERR_ARG for sizes below 2, lo >= hi on an axis or NULL pointers. */
sg_status sg_plan_sor_omega(int nx, int ny, int nz, const double lo[3], const double hi[3], double* omega);

/* ------------------------------------------------------------------------
 * Optional per-kernel profile.  When enabled, every kernel the grid launches
 * is bracketed by CUDA events on the grid's stream (this adds a few
 * microseconds per launch, so time solves with it disabled) and the totals are
 * kept per kernel class.  `bytes` is the algorithmic traffic of the launches:
 * the compulsory reads and writes of their input and output arrays, each cell
 * counted once, independent of caching.
 * ------------------------------------------------------------------------ */
#define SG_KERNEL_CLASSES 11
typedef struct sg_kernel_stat {
    char      name[24];       /* rkl_stage_l0, rkl_stage_coarse, residual_l0, residual_restrict,
                                 prolong_correct, coarse_solve, update, reduce_misc,
                                 bottom_levels (the two coarsest levels in one launch),
                                 gsrb_sweep (one colour of a GS-RB sweep),
                                 gravity (sg_gravity) */
    long long launches;
    double    ms;             /* summed event time of the launches */
    double    bytes;          /* summed algorithmic bytes */
} sg_kernel_stat;

/* Enable (1) or disable (0) the profile and reset its totals. */
sg_status sg_set_profiling(sg_grid* g, int on);

/* Copy the SG_KERNEL_CLASSES totals into out[].  Launches recorded since the
 * last solve (single operators, sg_gravity) are timed first, which
 * synchronises the grid's stream. */
sg_status sg_kernel_stats(sg_grid* g, sg_kernel_stat* out);

/* ------------------------------------------------------------------------
 * Single operators, for verification and for callers composing their own
 * cycles.  Pointers are device memory holding the level's [nz][ny][nx] array
 * (level l has n_d / 2^l cells per axis) in `dtype` (0 = float64, 1 = float32).
 * They run on the grid's stream and do not synchronise it.  `homogeneous = 1`
 * ignores the Dirichlet faces (Eq. error_ghost); it is forced on levels > 0.
 * ------------------------------------------------------------------------ */

/* One s-stage RKL super-step of order 1 or 2 (App. A, Eq.
 * RKL_intermediate_source) on L u = rhs at `level`, tau = tau_frac * tau_max:
 * out = Y_s.  out must not alias u or rhs.  SG_ERR_ARG for s < 1 (RKL1) or
 * s < 2 (RKL2). */
sg_status sg_op_superstep(sg_grid* g, int level, int dtype, int order, int s, double tau_frac,
                          int homogeneous, const void* u, const void* rhs, void* out);

/* One red-black Gauss-Seidel / SOR sweep (Sec. 2.2.4, App. B) of L u = rhs at
 * `level`, in place on u: the cells with (i + j + k) even, then the odd ones,
 * each u <- u - omega (L u - rhs) / d with d the diagonal of its row (-2 sum
 * 1/h^2, and -1/h_d^2 per Dirichlet wall it touches).  omega in [0, 2); 0 =
 * App. B's SOR omega of the level.  SG_ERR_ARG when a periodic axis of the
 * level has an odd extent (the colouring would not hold across the wrap). */
sg_status sg_op_gsrb_sweep(sg_grid* g, int level, int dtype, int homogeneous, double omega,
                           void* u, const void* rhs);

/* Residual r = rhs - L u at `level` (the negative of Eq. residual), restricted
 * to level + 1 by the 8-cell mean (Eq. restriction_example_3D; the 4-cell mean of Eq.
 * restriction_example_2D on a 2D grid) into coarse_out
 * when it is not NULL.  norms (host, may be NULL) receives
 * {sum r^2 (volume-weighted L2 squared), max |r|}; passing norms synchronises
 * the stream. */
sg_status sg_op_residual_restrict(sg_grid* g, int level, int dtype, int homogeneous,
                                  const void* u, const void* rhs, void* coarse_out,
                                  double norms[2]);

/* The FP64 residual r = rhs - L u of level 0 that confirms a mixed solve
 * (Sec. 2.1; the negative of Eq. residual), with the neighbour sum formed
 * exactly in 64-bit fixed point on a scale common to the level (u and the
 * Dirichlet face data set its largest exponent) and rounded to FP64 once:
 * r into r_out, its FP32 copy (significand truncated) into r32_out.  u, rhs,
 * r_out are device FP64 arrays of level 0 and r32_out a device FP32 one
 * (any grid precision); norms as in sg_op_residual_restrict, of the FP32 copy.
 * Levels whose values lie beyond 2^-900 .. 2^900, or are not finite, and
 * levels that are not strips of four cells (nx % 4 != 0, arrays not 16-byte
 * aligned) take the FP64 stencil. */
sg_status sg_op_residual_exact(sg_grid* g, int homogeneous, const double* u, const double* rhs,
                               double* r_out, float* r32_out, double norms[2]);

/* fine += P(coarse) (Eq. prolongation_example_3D; on a 2D grid Eq.
 * prolongation_example_2D) with coarse ghosts by the boundary rule; `level` is
 * the fine level, coarse is level + 1. */
sg_status sg_op_prolong_correct(sg_grid* g, int level, int dtype, const void* coarse, void* fine);

/* Coarsest-grid style solve of L u = rhs at `level` from u = 0 by the
 * Legendre-zero RKL1 schedule (App. A.5) with the grid's coarse options.
 * ss_done (host, may be NULL) receives the super-steps run and synchronises. */
sg_status sg_op_coarse_solve(sg_grid* g, int level, int dtype, const void* rhs, void* u_out,
                             int* ss_done);

/* ------------------------------------------------------------------------
 * Allocation-free residual.  The paper has no counterpart: this computes what
 * sg_op_residual_restrict computes (r = rhs - L u, the negative of Eq.
 * residual, its 8-cell mean of Eq. restriction_example_3D, and the norms) and
 * only changes where the reduction's scratch lives.
 *
 * For callers that may not allocate device memory while they run -- a job
 * whose device memory is all reserved up front (a caching allocator holding
 * the device, a real-time loop), or a host that owns only its own arrays and
 * wants no grid object (sg_create_grid allocates every multigrid level).  It
 * takes the finest-level geometry directly, runs the same kernels, and keeps
 * the per-block partial norms in one array compiled into this library: 8192
 * block slots, 256 KiB per device.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * nx, ny, nz, lo, hi, bc: as for sg_create_grid (the grid of u).  faces: NULL
 * for the homogeneous rule ghost = -active (Eq. error_ghost), else six DEVICE
 * pointers laid out as for sg_set_boundary (a NULL entry is a zero face;
 * entries of periodic axes are ignored).  dtype: 0 = float64, 1 = float32.
 * u, rhs: device [nz][ny][nx] arrays of dtype on the current device.
 * coarse_out: device (nz/2, ny/2, nx/2) array of dtype receiving the 8-cell
 * mean of r (every size even), or NULL.  norms: host, receives {sum r^2,
 * max |r|} and synchronises the stream, or NULL; coarse_out and norms are not
 * both NULL.  cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 *
 * Limit: one slot per thread block of the launch, about ceil(nx/32) *
 * ceil(ny/8) * (z chunks).  Every cube up to 1024^3 fits; a grid needing more
 * than 8192 slots returns SG_ERR_ARG (with the count) before any launch.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current; this may load the
 * library's kernels onto the device) and caches it.  Make that first call
 * before any stream capture begins.  Nothing in the array needs clearing:
 * each block writes its own slot before the fold reads it, and the fold
 * writes the whole result.
 *
 * The array is shared by every call on a device: calls whose work overlaps
 * on one device (different streams, or threads without ordering) race on it
 * and return wrong norms.  Serialise them (one stream, or an event between).
 * Errors: SG_ERR_ARG, SG_ERR_CUDA.
 */
sg_status sg_residual_restrict_noalloc(int nx, int ny, int nz, const double lo[3], const double hi[3],
                                       const int bc[3], const double* const faces[6], int dtype,
                                       const void* u, const void* rhs, void* coarse_out,
                                       double norms[2], void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SG_H */
