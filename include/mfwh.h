/*
 * mfwh.h -- C ABI of libmfwh: the Multi-Frequency WaveHoltz (MFWH) hot path on
 * one NVIDIA GB300 (sm_103a).
 *
 * MFWH (arXiv 2507.23613) computes N_f Helmholtz solutions
 *     L u_m + omega_m^2 u_m = f_m,  L = c^2 Delta,  u_m = 0 on the boundary
 * (eq. MultipleHelmholtz) by iterating a map Pi that solves ONE wave equation
 * forced by sum_m f_m cos(omega~_m t) (eq. waveEqnCompositeForcings, eq.
 * WaveScheme) and applies N_f time filters to it (eq. pDefQ), followed by an
 * N_f x N_f solve with the filter matrix B at every grid point (eq. filterA,
 * eq. waveHoltzMatrixIteration).  The fixed point of Pi is the discrete
 * Helmholtz solution (eq. discreteHelmholtz); GMRES on A = I - S accelerates
 * it (eq. krylovSystem).  Discretisation: uniform Cartesian grid in 2D or 3D,
 * second-order Laplacian, explicit leapfrog in time (alpha = 0, beta = 1),
 * Dirichlet data zero.
 *
 * Conventions for every call
 *   - Grid functions are dense float64 arrays over ALL grid points, boundary
 *     included, x fastest: index ((k * (ny+1)) + j) * (nx+1) + i.  A stack of
 *     N_f grid functions is N_f such arrays back to back ([N_f][points]).
 *   - Boundary values of inputs are ignored (treated as 0); outputs are 0 there.
 *   - Pointers documented as "host or device" may point to either; the library
 *     asks the CUDA driver which and copies as needed.  Pointers documented as
 *     "device" must be device memory of the handle's current device.
 *   - The caller owns every buffer it passes in; the handle owns its own
 *     workspace, allocated in mfwh_create and released in mfwh_destroy.
 *   - Every call returns an mfwh_status; on failure mfwh_last_error() gives a
 *     message (thread-local, valid until the next call on that thread).
 *   - A handle may be used from one host thread at a time.
 */
#ifndef MFWH_H
#define MFWH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MFWH_MAX_NF 16  /* largest number of frequencies per problem */

typedef enum {
  MFWH_OK = 0,
  MFWH_ERR_INVALID_ARG = 1,   /* bad size, ordering, mode or pointer */
  MFWH_ERR_SINGULAR = 2,      /* B or the optimiser's constraint matrix G is (near) singular */
  MFWH_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has the CUDA error) */
  MFWH_ERR_NOMEM = 4,         /* device or host allocation failed */
  MFWH_ERR_NOT_CONVERGED = 5, /* GMRES reached max_iters above the tolerance */
  MFWH_ERR_SPURIOUS = 6,      /* GMRES converged but the Helmholtz residual check failed */
  MFWH_ERR_NONFINITE = 7,     /* NaN or Inf in an iterate or residual */
  MFWH_ERR_TIMEOUT = 8        /* a bounded wait inside a kernel ran out: a grid-barrier wait of
                                 the implicit step kernel (limit: mfwh_set_wait_limit) or a
                                 tile's tensor copy of the FP32 blocked kernel; that wave solve's
                                 results are invalid, the handle stays usable */
} mfwh_status;

enum { MFWH_FILTER_OPTIMIZED = 0, MFWH_FILTER_TRADITIONAL = 1, MFWH_FILTER_USER = 2 };
/* Arithmetic of the wave solve.  FP64: wave levels, steps and the filter solve in FP64; with
   explicit time stepping the filter sums q_m are unevaluated float pairs (hi + lo, updated
   with two-product/two-sum on the FP32 pipe, about 2^-47 relative per update), so their
   magnitudes must stay below the float range (3.4e38) and keep full accuracy above about
   1e-30.  FP32_KAHAN: wave levels and
   steps in FP32 (increment form of the leapfrog scheme), filter sums with a Kahan update at
   every step; the filter solve B^{-1} q, GMRES and the residual stay FP64.  FP32_BLOCKSUM:
   as FP32_KAHAN, but a blocked launch of T steps sums its T filter terms in plain FP32 and
   folds that partial sum into the Kahan pair once (compensated across launches); with one
   step per launch it is FP32_KAHAN. */
enum { MFWH_PREC_FP64 = 0, MFWH_PREC_FP32_KAHAN = 1, MFWH_PREC_FP32_BLOCKSUM = 2 };
/* How the filter sums become the next iterate (Section "The MFWH algorithm"). */
enum { MFWH_UPDATE_IMPLICIT = 0, MFWH_UPDATE_EXPLICIT = 1 };
enum { MFWH_C_CONST = 0, MFWH_C_TWO_LAYER = 1, MFWH_C_FIELD = 2 };
/* Time stepping of the wave solve (Section "Explicit and implicit time-stepping"). */
enum { MFWH_TIME_EXPLICIT = 0, MFWH_TIME_IMPLICIT = 1 };

typedef struct mfwh_handle_s* mfwh_handle_t;

/* Problem statement (Section "Governing equations", eq. MultipleHelmholtz,
 * eq. gaussianSource inputs; time-step recipe of Section "Time-step determination"). */
typedef struct {
  int dim;                   /* 2 or 3 */
  int64_t n[3];              /* cells per axis, x first; points per axis = n+1; n >= 2 */
  double length[3];          /* domain extent per axis (> 0); h_i = length_i / n_i */
  int nf;                    /* number of frequencies, 1..MFWH_MAX_NF */
  const double* omega;       /* host, [nf], 0 < omega_1 < ... < omega_nf */
  const double* forcing;     /* host or device, [nf][points] values of f_m at the grid points;
                                copied into the handle by mfwh_create (may be NULL: zero forcing) */
  int c_mode;                /* MFWH_C_CONST: c = c_lo everywhere;
                                MFWH_C_TWO_LAYER: c = c_lo where x_axis < interface, c_hi elsewhere;
                                MFWH_C_FIELD: c^2 given per grid point by c2_field (L = c^2 Delta
                                in non-divergence form, L_h W = c_j^2 Delta_h W at point j) */
  double c_lo, c_hi;         /* wave speeds (> 0; c_lo is not used with MFWH_C_FIELD) */
  double interface;          /* coordinate of the layer interface (TWO_LAYER) */
  int layer_axis;            /* 0 = x, 1 = y, 2 = z (TWO_LAYER) */
  int n_p;                   /* N_p: periods of the longest period integrated (>= 1) */
  double cfl;                /* fraction (0, 1] of the explicit von Neumann step limit */
  int filter_mode;           /* MFWH_FILTER_* */
  const double* user_params; /* host, [nf][3] (a, c, s) when filter_mode == MFWH_FILTER_USER */
  int n_delta;               /* N_delta of eq. LambdaRange (paper: 20) */
  double c_delta;            /* c_delta of eq. LambdaRange (paper: 2) */
  int precision;             /* MFWH_PREC_FP64, MFWH_PREC_FP32_KAHAN or MFWH_PREC_FP32_BLOCKSUM */
  int time_block;            /* leapfrog steps per pass over HBM: 0 = library default (3 for
                                FP64 2D problems of up to 8 frequencies with second order,
                                explicit steps and constant or two-layer c, on tile shape 5;
                                1 for the other FP64 problems and for 3D; 16 for FP32 in 2D),
                                1 = one step per kernel launch; 2D: 2, 3, 4 or 8 for FP64, 4, 8
                                or 16 for FP32 = temporal blocking with that depth; 3D: 2 or 4
                                for the FP32 precisions.  Results are bit-identical for every
                                depth (FP32_BLOCKSUM: for every depth with the same partial-sum
                                length). */
  int order;                 /* order p of the spatial operator L_{ph}: 2 (0 means 2) or 4.
                                Order 4: (-W_{j-2} + 16 W_{j-1} - 30 W_j + 16 W_{j+1} - W_{j+2})
                                / (12 h^2) per axis, ghost values W_{-1} = -W_1 and
                                W_{N+1} = -W_{N-1} (odd reflection of homogeneous Dirichlet data),
                                time step limit sqrt(3)/2 of the second-order one, one step
                                per kernel launch (time_block 0 or 1) */
  int filter_update;         /* MFWH_UPDATE_IMPLICIT (0, default): B V^{k+1} = q, the implicit
                                filter of eq. vkUpdate; MFWH_UPDATE_EXPLICIT: B_mm V_m^{k+1} =
                                q_m - sum_{j != m} B_mj V_j^k, the explicit filter of the
                                footnote to eq. filterII (same fixed point) */
  int tile_shape;            /* FP32 blocked kernel tile: 0 = 32x32, 512 threads (default);
                                1 = 32x64, 512 threads; 2 = 64x64, 1024 threads (halved in
                                y above 8 frequencies).  FP64 blocked kernel tile (points x by
                                y): 0 = 32x64, 512 threads; 1 = 32x32, 512 threads; 2 = 32x48,
                                512 threads; 3 = 32x32, 256 threads, two CTAs per SM; 4 =
                                32x16, 512 threads, two CTAs per SM; 5 = 32x16 tiles stepped by
                                persistent CTAs (three per SM) that copy the next tile while
                                stepping one (depths 2 to 4, up to 8 frequencies; the default
                                with time_block 0).  Depths 2 and 3 run shapes 4 and 5 (the
                                others as 1), depth 8 runs shapes 0 to 3 (4 and 5 as 3); above
                                8 frequencies shapes 0 to 3 run as 1 and 5 as 4.  Every tile
                                gives bit-identical results. */
  int time_stepping;         /* MFWH_TIME_EXPLICIT (0, default): leapfrog, alpha = 0, beta = 1;
                                MFWH_TIME_IMPLICIT: trapezoidal scheme alpha = 1/2, beta = 0 of
                                eq. WaveScheme (FP64 results, one step per launch).  Every
                                step solves (I - dt^2/2 L_h) Z = 2 W^n - dt^2 F^n by geometric
                                multigrid on the device; W^{n+1} = Z - W^{n-1} (W^1 = Z/2).
                                Grids must halve (all n_i even, n_i/2 >= 2) down to a level of
                                at most 5000 points.  Order 4 is available for 2D and 3D grids
                                of more than 5000 points (the second-order multigrid
                                preconditions the fourth-order residual). */
  int steps_per_period;      /* implicit: steps over the shortest period 2 pi / omega_nf
                                (0 means 10; >= 5).  N_t = ceil(steps_per_period N_p omega_nf /
                                omega_1); dt solves omega~_1 N_t dt = 2 pi N_p. */
  double mg_tol;             /* implicit: a step's multigrid solve stops when
                                max|rhs - A Z| <= mg_tol max|rhs| (0 means 1e-10) */
  int mg_max_cycles;         /* implicit: V-cycles per step at most (0 means 30; <= 60) */
  const double* c2_field;    /* MFWH_C_FIELD: host or device [points], c^2 at every grid point
                                (all values finite and > 0); copied into the handle by
                                mfwh_create.  c_max^2 = the largest value (all points) sets the
                                explicit time step.  Supported with explicit time stepping and
                                MFWH_PREC_FP64, one step per launch (time_block 0 or 1), second
                                or fourth order; other combinations return
                                MFWH_ERR_INVALID_ARG.  mfwh_plan and the other host-only calls
                                read a device field through the CUDA runtime. */
} mfwh_problem;

/* Everything the set-up derives from a problem (Algorithm 1, first two lines;
 * eq. omegaImplicit, eq. TbarDef, eq. DefNI, Algorithm 2, eq. filterA). */
typedef struct {
  double dt;                                /* time step */
  int n_t;                                  /* N_t: steps per wave solve */
  int nf;
  double h[3];
  double omega_tilde[MFWH_MAX_NF];          /* adjusted frequencies omega~_m */
  int n_pm[MFWH_MAX_NF];                    /* N_{p,m} */
  double t_fm[MFWH_MAX_NF];                 /* T~_{f,m} = N_{p,m} 2 pi / omega~_m */
  double params[MFWH_MAX_NF][3];            /* filter parameters (a, c, s) per frequency */
  double B[MFWH_MAX_NF][MFWH_MAX_NF];       /* B[m][j] = sum_n w_{n,m} cos(omega~_j t^n) */
  double B_inv[MFWH_MAX_NF][MFWH_MAX_NF];
  double lam_max;                           /* right end of Lambda (optimised filters) */
  int n_lambda;                             /* N_lambda (optimised filters) */
  int64_t points;                           /* grid points per grid function */
  int64_t interior_points;
} mfwh_setup;

/* Outcome of mfwh_solve_gmres. */
typedef struct {
  int iterations;              /* Arnoldi steps taken (one homogeneous Pi each) */
  int pi_applications;         /* all applications of Pi (forced and homogeneous) */
  int restarts;                /* restart cycles started */
  double rel_residual;         /* final ||b - A x||_2 / ||b||_2 (Arnoldi estimate) */
  double helmholtz_residual[MFWH_MAX_NF]; /* r_h^{(m)} of the returned solution (eq. errorAndResid) */
  int history_len;             /* entries written to history (<= history_capacity) */
  int history_capacity;        /* set by the caller: capacity of history */
  double* history;             /* host, caller-owned, may be NULL: residual after each Arnoldi step */
  int refinements;             /* mfwh_solve_refined: corrections applied (0 for other solvers) */
} mfwh_solve_info;

/* ---- host-only set-up arithmetic (no GPU needed) ------------------------------ */

/* Full set-up of a problem without touching a GPU (time step, omega~, N_{p,m},
 * quadrature, filter parameters, B and B^{-1}): the first two lines of Algorithm 1, with
 * Section "Time-step determination", eq. omegaImplicit, eq. TbarDef, eq. DefNI, Algorithm 2
 * or eq. origParamAdjust, eq. pDefQ and eq. filterA.  Time step reading: dt_stab =
 * 1/(c_max sqrt(sum 1/h_i^2)); N_t = ceil(N_p (2 pi/omega_1) / (cfl dt_stab));
 * dt = 2 sin(pi N_p / N_t) / omega_1 so that omega~_1 N_t dt = 2 pi N_p.
 * Returns MFWH_ERR_SINGULAR if B has 1-norm condition number > 1e12 or the
 * optimiser's constraint matrix G one > 1e15. */
mfwh_status mfwh_plan(const mfwh_problem* prob, mfwh_setup* out);

/* Filter weights w_{n,m} = (2/T~_{f,m}) sigma_{n,m} K(omega~_m t^n; p_m) (eq. pDefQ)
 * of a planned problem, written to w_out[(n_t+1) * nf] (host, row n, column m). */
mfwh_status mfwh_plan_weights(const mfwh_problem* prob, double* w_out, int64_t capacity);

/* Multigrid hierarchy of an implicit problem (MFWH_TIME_IMPLICIT; the paper solves each implicit
 * step by multigrid, Section "Numerical results and O(N) scaling"; this hierarchy is the
 * library's own), without a GPU: *levels levels, cells[l][0..2] the cells per axis of
 * level l (x first; 0 for z in 2D), *coarse the
 * first level solved by one CTA in shared memory (levels of at most 5000 points).  cells has
 * room for 16 levels.  MFWH_ERR_INVALID_ARG if the problem is invalid, its grid does not
 * halve down to such a level, or it takes the fourth-order operator on a grid of at most 5000
 * points (the cases mfwh_create rejects for the hierarchy). */
mfwh_status mfwh_plan_multigrid(const mfwh_problem* prob, int* levels, int* coarse,
                                int64_t cells[16][3]);

/* Adjusted frequencies of eq. omegaImplicit for scheme weights (alpha, beta):
 * out[m] = acos((1 - beta/2 (omega_m dt)^2) / (1 + alpha (omega_m dt)^2)) / dt.  Host arrays. */
mfwh_status mfwh_adjusted_frequency(int nf, const double* omega, double dt,
                                    double alpha, double beta, double* out);

/* Algorithm 2 (optParameters), discrete form: least-squares filter parameters for
 * frequencies omega[nf] (already adjusted if desired) integrated over N_t equal
 * steps of T_f = max_m T_{f,m} with the trapezoid weights of eq. DefNI.
 * params_out: host [nf][3] (a~, c~, s~).  lam_max / n_lambda may be NULL. */
mfwh_status mfwh_opt_parameters(int nf, const double* omega, int n_p, int n_t,
                                int n_delta, double c_delta, double* params_out,
                                double* lam_max, int* n_lambda);

/* ---- device calls ------------------------------------------------------------ */

/* Plan the problem (the set-up of Algorithm 1, as mfwh_plan) and allocate its device workspace
 * on the current CUDA device.  prob->forcing (host or device) and prob->c2_field are copied.
 * stream: cudaStream_t all work is issued on (NULL = legacy default stream).  *out is NULL on
 * failure (MFWH_ERR_INVALID_ARG, MFWH_ERR_SINGULAR, MFWH_ERR_NOMEM or MFWH_ERR_CUDA). */
mfwh_status mfwh_create(const mfwh_problem* prob, void* stream, mfwh_handle_t* out);

/* Replace the forcings f_m of eq. MultipleHelmholtz: host or device [nf][points], copied.
 * Ordered on the handle's stream. */
mfwh_status mfwh_set_forcing(mfwh_handle_t h, const double* forcing);

/* One application of the MFWH map (the loop body of Algorithm 1):
 * v_out = Pi(v_in) = B^{-1} q(v_in) with the forcing (forced = 1), or
 * v_out = S v_in without it (forced = 0).  v_in may be NULL (zero initial data).
 * v_in, v_out: device [nf][points]; they may alias.  Asynchronous on the stream. */
mfwh_status mfwh_apply_Pi(mfwh_handle_t h, const double* v_in, double* v_out, int forced);

/* Fixed-point iteration of Algorithm 1: v <- Pi(v), `iters` times.
 * v: host or device [nf][points], in: V^0, out: V^iters.  Synchronous. */
mfwh_status mfwh_solve_fpi(mfwh_handle_t h, int iters, double* v);

/* Restarted GMRES(restart), 1 <= restart <= 1023 (restart >= max_iters: no
 * restart, as in the paper), on (I - S) v = Pi(0) (eq. discreteMFWHmapping,
 * eq. krylovSystem): no preconditioner, classical Gram-Schmidt applied twice
 * for the Arnoldi vectors in FP64 on the device, Hessenberg least squares by Givens rotations on the host, stopping
 * when the Arnoldi residual estimate ||b - A v||_2 / ||b||_2 < tol.
 * v: host or device [nf][points]; in: initial guess (warm start), out: solution.
 * The Krylov basis ((restart+1) * nf * points doubles) is allocated on the
 * first call that needs it and kept by the handle.
 * After convergence the Helmholtz residual r_h (eq. errorAndResid) is checked:
 * if max_m r_h^{(m)} > spurious_tol (> 0) the call returns MFWH_ERR_SPURIOUS
 * (convergence to a non-solution, Section "Acceleration by Krylov methods");
 * spurious_tol <= 0 skips the check.  info may be NULL.  Synchronous. */
mfwh_status mfwh_solve_gmres(mfwh_handle_t h, int restart, double tol, int max_iters,
                             double spurious_tol, double* v, mfwh_solve_info* info);

/* Mixed-precision solve: iterative refinement (GMRES-IR) of the MFWH fixed-point system
 * (I - S) v = Pi(0) (eq. discreteMFWHmapping, eq. krylovSystem), whose solution is the
 * discrete Helmholtz solution.  b = Pi(0) and every outer residual r = b - (v - S v) use FP64
 * wave solves; each correction solves (I - S) e = r by GMRES(restart) from zero to the
 * Arnoldi tolerance inner_tol with the handle's wave precision (FP32 wave solves for the FP32
 * precisions, whose products are accurate to about 1e-5 relative) and adds e to v in FP64.
 * The Helmholtz residual r_h (eq. errorAndResid) of v is computed in FP64 before every
 * correction; the solve stops with MFWH_OK once max_m r_h^{(m)} <= target, and with
 * MFWH_ERR_NOT_CONVERGED after max_refinements corrections or max_iters Arnoldi steps in all.
 * v: host or device [nf][points]; in: initial guess (warm start), out: solution.
 * info (may be NULL): Arnoldi steps and Pi applications summed over all corrections,
 * refinements, rel_residual = ||r||_2 / ||b||_2 of the last outer residual, final r_h.
 * Synchronous. */
mfwh_status mfwh_solve_refined(mfwh_handle_t h, int restart, double inner_tol, int max_iters,
                               double target, int max_refinements, double* v,
                               mfwh_solve_info* info);

/* Mixed-precision solve with relaxed products: mfwh_solve_refined whose every inner GMRES
 * starts with FP64 wave solves and switches to the handle's FP32 wave solves once its Arnoldi
 * residual estimate falls below relax_below (0 < relax_below < 1) times the norm of that inner
 * right-hand side; each restart cycle starts again in FP64.  This is an inexact Krylov method
 * whose products may lose accuracy as the residual falls (the relaxation strategies of
 * Simoncini and Szyld, SIAM J. Sci. Comput. 2003, and of Bouras and Fraysse, SIAM J. Matrix
 * Anal. Appl. 2005); the paper itself uses FP64 throughout.  h: an FP32 handle
 * (MFWH_PREC_FP32_KAHAN or MFWH_PREC_FP32_BLOCKSUM), else MFWH_ERR_INVALID_ARG.  Other
 * arguments and results as for mfwh_solve_refined.  Synchronous. */
mfwh_status mfwh_solve_relaxed(mfwh_handle_t h, int restart, double inner_tol, double relax_below,
                               int max_iters, double target, int max_refinements, double* v,
                               mfwh_solve_info* info);

/* ---- many problems: graphs, batches, autotuning (batched workloads; the paper
 * solves one problem at a time) ---------------------------------------------------- */

/* CUDA-graph mode for one handle.  With enable != 0, each variant of the wave solve used by
 * the handle's calls (forced or homogeneous, with or without an input, with or without the
 * v - S v subtraction, FP64 or FP32 arithmetic) is captured once into a CUDA graph on two
 * staging vectors owned by the handle (2 * nf * points doubles, allocated here) and replayed
 * as one graph launch per application of Pi, between a device-to-device copy in and out.
 * Results are bit-identical to direct launches.  enable = 0 drops the graphs.  Synchronises
 * the handle's stream.  Capture happens on the first use of a variant: do not call the
 * handle inside another stream capture then.  Implicit handles (MFWH_TIME_IMPLICIT) accept
 * the call and keep launching directly (N_t + 1 launches per Pi). */
mfwh_status mfwh_set_graphs(mfwh_handle_t h, int enable);

/* Solve count independent problems concurrently: one host thread per handle runs
 * mfwh_solve_gmres(handles[i], restart, tol, max_iters, 0, v[i], &infos[i]) on the handle's
 * own stream (give the handles distinct streams to overlap them on the GPU; handles in graph
 * mode launch one graph per Pi).  seconds[i] (host array, may be NULL) receives the time from
 * the common start to the end of problem i's solve.  Handles must be distinct; infos may be
 * NULL.  Implicit handles share one host thread and are solved one after another (their
 * step kernels are cooperative launches that must not wait on each other's blocks).
 * Returns MFWH_OK when every solve converged, else the first failing status (hard
 * errors before MFWH_ERR_NOT_CONVERGED) with its problem index in mfwh_last_error(). */
mfwh_status mfwh_solve_batch(const mfwh_handle_t* handles, int count, int restart, double tol,
                             int max_iters, double* const* v, mfwh_solve_info* infos,
                             double* seconds);

/* Lockstep batch: GMRES(restart) as mfwh_solve_gmres (spurious_tol 0) on count independent
 * problems whose every application of the map is one CUDA-graph launch across the batch.  The
 * problems advance together: each round applies the map once to every problem that has not
 * finished (b = Pi(0) in the first round, then one product (I - S) u per round: u a problem's
 * newest Arnoldi vector, or its iterate at the start of a restart cycle), all as one launch of a
 * graph whose independent branches are the problems' captured wave solves; between launches
 * each problem's Gram-Schmidt passes and Givens update run on `stream`, with one
 * synchronisation per pass for the whole batch.  The graph is rebuilt when the set of
 * unfinished problems changes.  Handles must be explicit (MFWH_TIME_EXPLICIT), distinct and on
 * the current device; each is put in CUDA-graph mode (mfwh_set_graphs) if it is not.
 * v[i]: host or device [nf][points] of problem i; in: initial guess, out: solution.  infos may
 * be NULL; seconds[i] (host, may be NULL) receives the time from the start to the end of the
 * round in which problem i finished.  stream: cudaStream_t of the batch (NULL = legacy default
 * stream); it waits for each handle's stream at the start, and each handle's stream waits for
 * it at the end.  Returns MFWH_OK when every problem converged, else the first hard error, else
 * MFWH_ERR_NOT_CONVERGED, with the problem index in mfwh_last_error().  Synchronous. */
mfwh_status mfwh_solve_batch_graph(const mfwh_handle_t* handles, int count, int restart,
                                   double tol, int max_iters, double* const* v,
                                   mfwh_solve_info* infos, double* seconds, void* stream);

/* Autotuner for the blocked wave kernels.  Times the first steps (at most 96) of a
 * homogeneous wave solve of prob on the current device for each candidate temporal depth and
 * tile shape (FP32, 2D: depths 4, 8, 16 x tile shapes 0, 1, 2; FP64, 2D: depth 1, and depths
 * 4, 8 x tile shapes 1, 3; FP32, 3D: depths 1, 2, 4; FP64 3D, fourth order and c^2 fields:
 * depth 1), keeping the fastest:
 * *time_block and *tile_shape receive it, *ms_per_step
 * (may be NULL) its time per leapfrog step.  Results are cached per device, grid, number of
 * frequencies and precision for the life of the process.  Allocates (and frees) one handle's
 * workspace per candidate on the given stream; synchronous.  Implicit time stepping has no
 * candidates: depth 1, tile shape 0 and *ms_per_step = 0 without timing. */
mfwh_status mfwh_autotune(const mfwh_problem* prob, void* stream, int* time_block,
                          int* tile_shape, double* ms_per_step);

/* ---- learned warm start (an extension; the paper starts GMRES from zero)
 * A small convolutional network maps one frequency's forcing (and its frequency, as a second
 * constant channel) to an initial iterate V_m^0.  L layers of 3 x 3 "same" convolutions
 * (zero padding) with bias and ReLU after every layer but the last; in_channels inputs,
 * `channels` hidden channels, one output.  Activations and weights in BF16; the convolutions
 * and their input gradients sum products in FP32 on the 5th-generation tensor cores
 * (tcgen05.mma, accumulators in tensor memory), the weight gradients on the FP32 CUDA cores;
 * gradients, master weights and Adam state in FP32.
 * Images are device float32 arrays [B][C][H][W] (x fastest).  Parameters, flat FP32: for each
 * layer l, w_l[Cout][Cin][3][3] (cross-correlation: out[y][x] += w[dy][dx] in[y+dy-1][x+dx-1])
 * then b_l[Cout].  The network owns its workspace, which grows with B * H * W. */
typedef struct mfwh_cnn_s* mfwh_cnn_t;

/* layers 2..16, channels and in_channels 1..32; He-normal weights from `seed`, zero biases. */
mfwh_status mfwh_cnn_create(int layers, int channels, int in_channels, uint64_t seed,
                            void* stream, mfwh_cnn_t* out);
int64_t mfwh_cnn_param_count(mfwh_cnn_t c);
/* Replace the parameters (host, param_count floats) and reset the Adam state.  Synchronous. */
mfwh_status mfwh_cnn_set_params(mfwh_cnn_t c, const float* host, int64_t count);
/* Copy parameters and, if grads_host != NULL, the gradients of the last training step.
 * Synchronous. */
mfwh_status mfwh_cnn_get_params(mfwh_cnn_t c, float* host, float* grads_host, int64_t count);
/* y[B][1][H][W] (device) = network(x[B][in_channels][H][W]) (device).  Asynchronous. */
mfwh_status mfwh_cnn_forward(mfwh_cnn_t c, const float* x, int B, int H, int W, float* y);
/* One Adam step (learning rate lr, betas 0.9 / 0.999, eps 1e-8) on the mean squared error
 * between network(x) and target[B][1][H][W] over the points where mask[H][W] is 1 (device
 * arrays); *loss (host, may be NULL) receives the loss before the step.  Synchronous. */
mfwh_status mfwh_cnn_train_step(mfwh_cnn_t c, const float* x, const float* target,
                                const float* mask, int B, int H, int W, float lr, float* loss);
void mfwh_cnn_destroy(mfwh_cnn_t c);

/* Training pairs of the warm start from a solved 2D problem: for each frequency m, inputs
 * x_out[m][0] = f_m / max|f_m| and x_out[m][1] = omega_m / omega_scale (device float32
 * [nf][2][ny+1][nx+1]) and target t_out[m] = V_m / max|V_m|, the shape of the solution (device
 * float32 [nf][ny+1][nx+1]), from the solution v (device [nf][points]).  Synchronous. */
mfwh_status mfwh_warm_start_data(mfwh_handle_t h, double omega_scale, const double* v,
                                 float* x_out, float* t_out);
/* Initial iterate for GMRES from the network (2D): V_m^0 = alpha_m phi_m, where phi_m is the
 * network's output on the inputs above (0 on the boundary) and alpha_m = <A phi_m, f_m> /
 * <A phi_m, A phi_m> (A = L_h + omega_m^2, interior points) minimises the L2 Helmholtz
 * residual, computed in FP64 on the device.  It is kept only if it lowers GMRES's initial
 * residual, ||b - (V^0 - S V^0)|| < ||b|| with b = Pi(0) (two applications of Pi); otherwise v
 * is set to 0 and the call returns MFWH_ERR_NOT_CONVERGED.  *ratio_out (may be NULL) receives
 * ||b - (V^0 - S V^0)|| / ||b|| of the returned start (1 for zero).  v: host or device
 * [nf][points].  Allocates temporary device buffers.  Synchronous. */
mfwh_status mfwh_warm_start(mfwh_handle_t h, mfwh_cnn_t net, double omega_scale, double* v,
                            double* ratio_out);

/* Helmholtz residual r_h^{(m)} = max_int |f_m - (L_h + omega_m^2) v_m| / max_int |f_m|
 * (eq. errorAndResid, with +omega^2 as in eq. MultipleHelmholtz).
 * v: host or device [nf][points]; r_out: host [nf].  Synchronous. */
mfwh_status mfwh_residual(mfwh_handle_t h, const double* v, double* r_out);

/* Allocation-free Helmholtz residual (no counterpart in the paper).
 * For callers that cannot allocate device memory at the point where they need
 * the residual: code whose device memory belongs to another allocator (a
 * framework's caching allocator, or a pool sized once at start-up) and must
 * not grow outside it, and loops that cannot accept the implicit device
 * synchronisation cudaMalloc / cudaFree may cause.  It computes what
 * mfwh_residual computes, without a handle, and allocates nothing: its
 * reduction scratch is one fixed array of MFWH_NOALLOC_SCRATCH_DOUBLES doubles
 * (256 KiB) in the library's device memory, which every GPU that loads the
 * library holds until the process exits.
 *   prob:    grid (dim, n, length), nf, omega, order and the wave-speed fields, as for
 *            mfwh_create (with MFWH_C_FIELD, c2_field must be device memory of the
 *            current device, values not checked); the other fields are not used
 *   forcing: device [nf][points], the values f_m
 *   v:       device [nf][points]
 *            (forcing and v: device memory of the current device, or managed
 *            memory; other pointers are rejected with MFWH_ERR_INVALID_ARG)
 *   r_out:   host [nf], receives r_h^{(m)}
 *   stream:  cudaStream_t to run on (NULL = legacy default stream); the call
 *            synchronises that stream before it returns.
 * The first call on each device looks up the array's device address (set-up,
 * once per device, with that device current) and keeps it for the life of the
 * process: make that first call before any stream capture.  A cudaDeviceReset
 * of that device unloads the library's device code and leaves the kept address
 * stale, so after one do not call this entry point on that device again.
 * Every call uses the same array, so calls whose work
 * overlaps on the GPU (from other threads or streams) race and must be
 * serialised by the caller.  A call needs 1216 * nf + 2 * nf doubles; a
 * problem needing more than the array holds is rejected (MFWH_ERR_INVALID_ARG). */
#define MFWH_NOALLOC_SCRATCH_DOUBLES 32768
mfwh_status mfwh_residual_noalloc(const mfwh_problem* prob, const double* forcing,
                                  const double* v, double* r_out, void* stream);

/* Copy of the handle's set-up (the quantities of Algorithm 1's set-up, as mfwh_plan). */
mfwh_status mfwh_get_setup(mfwh_handle_t h, mfwh_setup* out);

/* Measurement (no counterpart in the paper).  Timing of the most recent mfwh_apply_Pi /
 * mfwh_solve_fpi / mfwh_solve_gmres /
 * mfwh_residual call, measured with CUDA events on the handle's stream:
 * step_ms = device time of the leapfrog+filter step kernels (the N_t launches of
 * every Pi application, the initial W^0 kernel excluded), step_launches = how
 * many such launches, total_launches = every kernel the call launched.  For
 * mfwh_apply_Pi the call synchronises the stream to read the events.  Any
 * output pointer may be NULL. */
mfwh_status mfwh_last_timing(mfwh_handle_t h, double* step_ms, int64_t* step_launches,
                             int64_t* total_launches);

/* Multigrid statistics of an implicit handle (MFWH_TIME_IMPLICIT; the paper reports multigrid
 * cycles per wave solve in Section "Numerical results and O(N) scaling"), accumulated over every
 * step solve since the handle was created or the counters were last reset:
 * solves = step solves, cycles = V-cycles applied (a solve whose start already meets
 * mg_tol applies none), unconverged = solves that reached mg_max_cycles above mg_tol.
 * levels = levels of the hierarchy (always written).  reset != 0 zeroes the counters after
 * reading them.  Synchronises the stream.  MFWH_ERR_INVALID_ARG for an explicit handle. */
mfwh_status mfwh_mg_stats(mfwh_handle_t h, int64_t* solves, int64_t* cycles,
                          int64_t* unconverged, int* levels, int reset);

/* Time limit of one grid-barrier wait inside the implicit step kernel (MFWH_TIME_IMPLICIT
 * handles whose hierarchy has grid-wide levels; Section "Explicit and implicit time-stepping"),
 * in seconds; seconds <= 0 restores the default of 2 s.  The blocks of that cooperative launch
 * meet at a barrier between multigrid phases.  When one wait runs out, the kernel records it
 * in a device flag and every later barrier of the launch lets its blocks through, so the launch
 * ends (its results are then invalid) and the remaining step launches of the wave solve return
 * at once.  The call that completes the solve (mfwh_solve_fpi, mfwh_solve_gmres,
 * mfwh_solve_refined, mfwh_residual after it, or mfwh_last_timing after mfwh_apply_Pi) then
 * returns MFWH_ERR_TIMEOUT and clears the flag and the barrier state, so the handle can be
 * used again.  Explicit handles accept the call and ignore the limit (no grid barriers). */
mfwh_status mfwh_set_wait_limit(mfwh_handle_t h, double seconds);

/* Index checks of the debugging build (a debugging aid; the paper has none).  The library
 * built with -DMFWH_BOUNDS_CHECK (libmfwh_bc.so) tests the indices of the FP64 step kernels'
 * global and shared-memory accesses against the extents of their arrays; an out-of-range
 * index is skipped, counted in the handle's fault record, and the first one is kept.
 * *count: out-of-range indices met by this handle's kernels so far, or -1 for the normal
 * build (no checks compiled); *index, *extent: the first one and the extent it exceeded;
 * *line: its source line (index, extent, line may be NULL).  Synchronises the stream in the
 * checked build. */
mfwh_status mfwh_debug_bounds(mfwh_handle_t h, int64_t* count, int64_t* index, int64_t* extent,
                              int* line);

/* Release the handle and its device workspace (waits for its stream). */
void mfwh_destroy(mfwh_handle_t h);

/* Error reporting (no counterpart in the paper): the message of the last failed call on this
 * thread (valid until the next call on it), and a fixed description of a status code. */
const char* mfwh_last_error(void);
const char* mfwh_status_string(mfwh_status s);

#ifdef __cplusplus
}
#endif

#endif /* MFWH_H */
