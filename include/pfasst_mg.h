/*
 * pfasst_mg.h -- C ABI of a GB300 (sm_103a) library for batched SDC sweeps with
 * geometric-multigrid sub-step solves, interwoven with two-level PFASST.
 *
 * What it computes ("Interweaving PFASST and Parallel Multigrid", Minion, Speck,
 * Bolten, Emmett, Ruprecht):
 *   the heat equation u_t = nu Lap u on [0,1]^d, d = 1, 2, 3, zero Dirichlet walls,
 *   2nd-order finite differences with n interior points per axis, h = 1/(n+1)
 *   (Sec. 4.1, Sec. 4.2);  time slices of length dt, each integrated by the
 *   collocation method on Gauss-Lobatto nodes (Sec. 2.1, Eq. collocationM);
 *   SDC sweeps with implicit-Euler sub-steps (Sec. 2.2, Eq. sdc-be), whose
 *   sub-step equations (I - dt_m nu Lap_h) u_{m+1} = rhs (Eq. SDCcompactLIII)
 *   are solved by geometric multigrid V-cycles, either a fixed small number of
 *   them (inexact SDC, Sec. 2.3.1) or to a tolerance (Sec. 4.2.1);  two-level
 *   PFASST with an FAS-corrected coarse level (Sec. 2.3, 2.4), where all time
 *   slices, which PFASST treats as parallel, run as one batch on one GPU.
 *
 * Conventions
 *   - Every function returns PMG_OK (0) on success, PMG_NOT_CONVERGED (1) when an
 *     iteration limit was reached, or a negative PMG_ERR_* code.  No C++ exception
 *     crosses this boundary.  pfasst_mg_last_error() gives a message.
 *   - All device work is ordered on the CUDA stream given at creation (NULL = the
 *     legacy default stream).  Functions that return host data synchronise it.
 *   - Grid functions passed in or out use the dense layout [z][y][x], x fastest,
 *     interior points only (n^d doubles); wall values are zero and not stored.
 *   - Pointers are borrowed for the duration of the call only; the handle owns all
 *     device state it allocated.  A caller-provided workspace must outlive the handle.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef PFASST_MG_H
#define PFASST_MG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define PMG_OK                0
#define PMG_NOT_CONVERGED     1   /* max_iter reached before the tolerance       */
#define PMG_ERR_INVALID_ARG  -1   /* bad pointer, size or option                 */
#define PMG_ERR_OOM          -2   /* device allocation failed / workspace short  */
#define PMG_ERR_CUDA         -3   /* a CUDA runtime call or kernel launch failed */
#define PMG_ERR_DIVERGED     -4   /* NaN/Inf or growing residual                 */
#define PMG_ERR_TIMEOUT      -5   /* a bounded device-side wait gave up          */
#define PMG_ERR_UNSUPPORTED  -6   /* valid but not implemented combination       */

/* ---- problem description ------------------------------------------------- */

/* Spatial grid: dim in {1,2,3}; n interior points per axis on the finest level,
 * n = 2^p - 1 with 3 <= n <= 1023 so that the multigrid hierarchy n -> (n-1)/2
 * reaches 3 points (Sec. 4.1.1 "standard geometric multigrid").
 * order: Laplacian stencil of the finest level (Sec. 4.2: second- or fourth-order
 * finite differences).  0 or 2: u_{i-1} - 2u_i + u_{i+1} per axis; 4 (n >= 7):
 * (-u_{i-2} + 16u_{i-1} - 30u_i + 16u_{i+1} - u_{i+2}) / 12 per axis, the point beyond
 * a wall taking the odd reflection -u of its mirror image.  It applies to the fine
 * PFASST level and to the finest grid of its multigrid solves (smoothed by weighted
 * Jacobi, or by Gauss-Seidel in three colours (i+j+k) mod 3 instead of two); coarser
 * PFASST levels and coarser multigrid grids use the second-order stencil. */
typedef struct { int dim; int n; int order; } pmg_grid;

/* Collocation nodes of one level: count = M + 1 nodes in [0,1] including both
 * endpoints.  family 0 = Gauss-Lobatto (Lobatto IIIA collocation); family 1 = the
 * paper's uniform nodes tau_m = m/M with a quadrature rule that does not use the left
 * endpoint (Sec. 3: M = 1 backward Euler, M = 2 midpoint + right endpoint, second
 * order; M = 4 fourth order).  Node 0 (t = 0) carries the slice's initial value. */
typedef struct { int count; int family; } pmg_nodes_desc;

/* Level hierarchy: nlevels = 1 (SDC / parallel SDC), 2 (PFASST / MLSDC) or 3.  Level 1
 * uses coarse_nodes (a subset of the fine nodes, e.g. 3 of 5 Gauss-Lobatto nodes) and
 * the grid (n-1)/2 (Sec. 2.3, spatial and temporal coarsening); with three levels,
 * level 2 uses coarsest_nodes (a subset of coarse_nodes) and the grid (n-3)/4 (needs
 * n >= 15), and the serial coarse chain runs on level 2 while level 1 sweeps every
 * slice at once (multi-level PFASST, Sec. 2.4).  coarsest_nodes is ignored for fewer
 * levels. */
typedef struct { int nlevels; pmg_nodes_desc coarse_nodes; pmg_nodes_desc coarsest_nodes; } pmg_levels;

#define PMG_SMOOTHER_JACOBI 0     /* weighted Jacobi, omega (Sec. 4.1.1)          */
#define PMG_SMOOTHER_RBGS   1     /* red-black Gauss-Seidel (Sec. 4.1.2, 4.2.1)   */
#define PMG_PREC_FP64       0     /* everything in FP64                           */
#define PMG_PREC_MIXED      1     /* V-cycles in FP32, SDC/FAS/residuals in FP64  */

typedef struct {
    int    smoother;      /* PMG_SMOOTHER_*                                          */
    double omega;         /* relaxation weight (2/3 Jacobi, 1 Gauss-Seidel)          */
    int    nu1, nu2;      /* pre-/post-smoothing sweeps per level (V(nu1,nu2))       */
    int    vcycles;       /* > 0: V-cycles per sub-step solve; 0: solve to mg_tol    */
    double mg_tol;        /* full solve: ||b - L u||_inf <= mg_tol * max(1,||b||_inf) */
    double mg_stall;      /* full solve stops when new residual >= mg_stall * old    */
    int    mg_maxcycles;  /* full solve cap on V-cycles                              */
    int    precision;     /* PMG_PREC_*                                              */
    int    interp_order;  /* spatial interpolation between PFASST levels: 2 or 4    */
    int    use_graphs;    /* 1: replay each PFASST iteration as a captured CUDA graph */
    int    autotune;      /* 1: at creation, time the smoother variants of every multigrid
                             level (threads per block; fused, TMA-staged 3D sweeps and
                             their z chunks), each captured into a CUDA graph and replayed
                             as the solver runs it, and keep the fastest; 0: built-in size
                             rules                                                        */
    int    slice_groups;  /* two-level PFASST with fixed V-cycle counts: the slices of an
                             iteration are processed in this many groups so that the serial
                             coarse chain of group g overlaps the fine sweeps of groups
                             > g (same results); 0 or 1 = no overlap, at most 8 (2 groups
                             gain 1.5 % on the 3D workload: every fine kernel already fills
                             the GPU)                                                       */
    int    vcycle_tail;   /* for single grids (the serial coarse chain, members of an uneven
                             batch): 1 = the coarsest multigrid levels (from the first level
                             whose whole remaining V-cycle fits one CTA's shared memory:
                             15^3 in 3D, 63^2 in 2D, all of a 1D hierarchy) run as one kernel
                             launch per V-cycle; 0 = one launch per smoothing sweep,
                             restriction and prolongation; -1 (default) = automatic: one
                             launch in 1D and for red-black Gauss-Seidel, per level for
                             weighted Jacobi in 2D and 3D (the measured-faster choice on the
                             1D, 2D, 3D and uneven workloads)                               */
    int    coarse_vcycles;/* sub-step solves on the coarse PFASST levels (levels >= 1):
                             -1 (default) = vcycles; 0 = solve to mg_tol with the stall
                             rule; > 0 = that many V-cycles.  The paper leaves the coarse
                             level's solver open (Sec. 4.2.1); inexact coarse solves can
                             limit PFASST's convergence with backward Euler on the coarse
                             level.  Any 0 (here or in vcycles) runs the iteration without
                             CUDA graphs (the full solve decides its cycle count on the host) */
    int    single_grid_vcycle;/* 1: the fixed V-cycles of a single-grid sub-step solve (the
                             serial coarse chain) run as one persistent, cooperatively
                             launched kernel -- every smoothing colour, restriction, coarsest
                             solve and prolongation of all cycles, separated by grid-wide
                             barriers, and the update u += e (red-black Gauss-Seidel, 2D/3D,
                             second order; results bitwise those of the per-level kernels);
                             0 (default): one launch per sweep, restriction and prolongation
                             (faster on the 3D workload: 1860 vs 1926 ms per step)          */
} pmg_options;

typedef struct pmg_ctx *pmg_handle;

/* Defaults: Jacobi omega 2/3, V(2,1), 2 V-cycles, tol 1e-12, stall 0.75, cap 50,
 * FP64, 4th-order interpolation, graphs on, autotuning on, slice groups 0 (one group:
 * no overlap), V-cycle tail automatic (-1), coarse levels as the fine level (coarse_vcycles -1),
 * persistent single-grid V-cycles off. */
void pfasst_mg_default_options(pmg_options *opt);

/* Bytes of device workspace pfasst_mg_create needs for this problem.
 * Errors: PMG_ERR_INVALID_ARG for an invalid description. */
int pfasst_mg_workspace_bytes(const pmg_grid *grid, const pmg_nodes_desc *fine_nodes,
                              const pmg_levels *levels, int slices, const pmg_options *opt,
                              size_t *bytes);

/* Create a solver for `slices` consecutive time slices of length dt (the PFASST
 * block [0, slices*dt]) of u_t = nu Lap u.
 *   grid, fine_nodes, levels, opt (NULL = defaults): as above;  nu > 0, dt > 0;
 *   slices >= 1;  stream: a cudaStream_t or NULL;
 *   workspace: device memory of >= pfasst_mg_workspace_bytes() bytes, 256-byte
 *   aligned, owned by the caller, or NULL to let the library cudaMalloc its own.
 * Errors: INVALID_ARG (bad sizes, n not 2^p-1, a level's nodes not a subset of the
 * next finer level's nodes), UNSUPPORTED, OOM, CUDA.  *out is NULL on error. */
int pfasst_mg_create(const pmg_grid *grid, const pmg_nodes_desc *fine_nodes,
                     const pmg_levels *levels, double nu, double dt, int slices,
                     const pmg_options *opt, void *stream, void *workspace,
                     size_t workspace_bytes, pmg_handle *out);

/* Set the initial value u0 (n^d doubles, dense) and spread it to every node of every
 * slice (start of the predictor, Sec. 2.4).  on_device: 1 if u0 is device memory. */
int pfasst_mg_set_initial(pmg_handle h, const double *u0, int on_device);

/* PFASST predictor (Sec. 2.4): FAS-restrict the spread values down to the coarsest
 * level; there, in stage s, every slice p >= s takes the coarsest end value of slice
 * p-1 and does one sweep (slice p does p+1 sweeps); interpolate the corrections level
 * by level up.  With one level the predictor is the spread alone.
 * pfasst_mg_iterate calls it when needed. */
int pfasst_mg_predict(pmg_handle h);

/* One SDC sweep (Eq. sdc-be; sub-steps Eq. SDCcompactLIII solved by V-cycles) on
 * every slice at `level` (0 = fine, batched over slices; the coarsest level of a
 * hierarchy: FAS-corrected, serial chain over slices where slice p first receives the
 * end value of slice p-1 -- the blocking coarse communication of Sec. 2.4; level 1 of
 * three: FAS-corrected, batched over slices). */
int pfasst_mg_sweep(pmg_handle h, int level);

/* PFASST iterations (Sec. 2.4): fine sweep on all slices, FAS restriction (with three
 * levels: a level-1 sweep on all slices and a second FAS restriction), serial chain on
 * the coarsest level, interpolation of the corrections level by level, send-forward
 * of fine end values, collocation residual (Eq. resid).  Runs the predictor first if it has not run.
 * Stops after max_iter iterations or when the max-norm residual of every slice is
 * <= tol.  iters_done / final_res (max over slices) may be NULL.
 * Returns PMG_OK, PMG_NOT_CONVERGED, PMG_ERR_DIVERGED (NaN/Inf) or another error. */
int pfasst_mg_iterate(pmg_handle h, int max_iter, double tol, int *iters_done, double *final_res);

/* Collocation residual r = U_0 + dt Q F(U) - U (Eq. resid) of the fine level,
 * max norm over nodes and points, one value per slice into res_per_slice (host,
 * `slices` doubles).  Synchronises the stream. */
int pfasst_mg_residual(pmg_handle h, double *res_per_slice);

/* Copy the fine solution at (slice, node) into out (n^d doubles, dense).
 * node in [0, M]; node M of slice P-1 is the end of the block. */
int pfasst_mg_get_solution(pmg_handle h, int slice, int node, double *out, int on_device);

/* Copy the whole state of `level` (0 fine, 1 coarse, 2 coarsest): U as
 * [slice][node][n_l^d], dense, into host memory out (slices*nodes*N_l doubles).
 * Synchronises. */
int pfasst_mg_get_state(pmg_handle h, int level, double *out);

/* Start the next block: the end value of the last slice becomes the new initial
 * value and is spread (the predictor runs again on the next iterate). */
int pfasst_mg_advance(pmg_handle h);

/* Number of kernel launches this handle has issued so far (for launch accounting). */
long long pfasst_mg_launch_count(pmg_handle h);

/* Smoother chosen for multigrid level `level` (0 = finest) of the handle's hierarchy,
 * for wide batches (narrow = 0) or a single grid (narrow = 1): *fused = 1 for the fused
 * 3D red-black sweep (then *param = z chunk, 0 = default, and *threads per CTA), 2 for
 * its variant with TMA-staged planes (FP32; two x points per thread), 3 for the same with
 * four x points per thread, 0 for the one-point-per-thread kernels (*param = threads per
 * block). */
int pfasst_mg_tuning(pmg_handle h, int level, int narrow, int *fused, int *param, int *threads);

/* Pin the smoother variant of a level (same encoding as pfasst_mg_tuning; the exact
 * coarsest level has none).  Later iterations use it (captured graphs are rebuilt).
 * Errors: INVALID_ARG, UNSUPPORTED (a variant the level or precision cannot run; the
 * fused and TMA-staged sweeps run the second-order stencil only). */
int pfasst_mg_set_tuning(pmg_handle h, int level, int narrow, int fused, int param, int threads);

/* ---- launch profiling ------------------------------------------------------ */

/* Per-kernel aggregate of CUDA-event timings taken on the handle's stream. */
typedef struct {
    int       kernel;      /* kernel identifier, see pfasst_mg_kernel_name()          */
    int       n;           /* interior points per axis of the grid it ran on          */
    int       precision;   /* 0 FP64, 1 FP32 data                                     */
    long long launches;    /* launches recorded                                       */
    long long points;      /* grid points covered, summed over launches and batch     */
    double    ms;          /* summed launch durations (end event - start event)       */
} pmg_kernel_stat;

/* Record a CUDA event pair around every later launch that covers at least
 * min_points grid points (enable = 1), or stop recording (enable = 0). */
int pfasst_mg_profile(pmg_handle h, int enable, long long min_points);

/* Synchronise, aggregate the recorded launches per (kernel, n, precision) into out
 * (up to capacity entries), set *count to the number of aggregates, and clear the
 * record.  Errors: INVALID_ARG, CUDA. */
int pfasst_mg_profile_read(pmg_handle h, pmg_kernel_stat *out, int capacity, int *count);

/* Name of a kernel identifier ("smooth_rbgs", ...); "unknown" if out of range. */
const char *pfasst_mg_kernel_name(int kernel);

/* Self-check of the library's integer-pipe FP64 -> FP32 rounding (used where mixed
 * precision narrows a value per grid point) against the hardware conversion, on
 * `samples` generated inputs (uniform bit patterns, the float range with subnormal and
 * overflow edges, exact ties).  *mismatches (host) receives the number of differing
 * results (0 expected).  Synchronises the default stream.  Errors: INVALID_ARG, CUDA. */
int pfasst_mg_check_narrowing(long long samples, unsigned long long seed, long long *mismatches);

/* Self-check of the library's integer-pipe FP32 -> FP64 widening (used where an FP32
 * multigrid correction is added to an FP64 iterate) against the hardware conversion on
 * every one of the 2^32 float bit patterns (NaN inputs: both results must be NaN).
 * *mismatches (host) receives the number of differing results (0 expected).
 * Synchronises the default stream.  Errors: INVALID_ARG, CUDA. */
int pfasst_mg_check_widening(long long *mismatches);

/* Measured FP64 FMA throughput of the current device in GFLOP/s (*gflops, host): a
 * probe kernel of independent FMA chains on every SM (8 CTAs of 256 threads per SM, 8
 * chains per thread), warmed up once and then launched `launches` times (1..100) on
 * `stream`, each timed with CUDA events; the best launch counts (FMA = 2 flops).  The
 * roofline denominator of the library's FP64-bound kernels; the paper has no
 * counterpart.  Synchronises the stream.  Errors: INVALID_ARG, CUDA. */
int pfasst_mg_fp64_peak(void *stream, int launches, double *gflops);

/* Release the handle and any device memory it allocated.  NULL is accepted. */
int pfasst_mg_destroy(pmg_handle h);

/* Message of the last error on h (or of the last failed create when h is NULL). */
const char *pfasst_mg_last_error(pmg_handle h);

/* ---- uneven batch of independent problems ------------------------------------ */

/* One problem of an uneven batch: its own grid, Gauss-Lobatto node count, nu and dt. */
typedef struct {
    pmg_grid grid;
    int      nodes;
    double   nu, dt;
} pmg_problem_desc;

/* Bytes of workspace pfasst_mg_create_batch needs.  Errors as pfasst_mg_create;
 * PMG_ERR_UNSUPPORTED if opt->vcycles == 0 (batches run fixed V-cycle counts). */
int pfasst_mg_batch_workspace_bytes(int nprob, const pmg_problem_desc *probs, const pmg_options *opt,
                                    size_t *bytes);

/* Create a solver for nprob independent heat problems of different sizes, each
 * integrated by single-level SDC (Sec. 2.2) with multigrid sub-step solves, one time
 * step of length dt at a time.  All problems advance together: pfasst_mg_batch_run
 * replays one CUDA graph per time step in which every problem is an independent
 * branch.  Arguments and ownership as pfasst_mg_create; probs is copied. */
int pfasst_mg_create_batch(int nprob, const pmg_problem_desc *probs, const pmg_options *opt, void *stream,
                           void *workspace, size_t workspace_bytes, pmg_handle *out);

/* Initial value of problem `prob` (its own n^d doubles, dense layout). */
int pfasst_mg_batch_set_initial(pmg_handle h, int prob, const double *u0, int on_device);

/* Advance every problem by `steps` time steps of `sweeps` SDC sweeps each
 * (Eq. sdc-be with V-cycle sub-step solves); residuals (host, nprob doubles, may be
 * NULL) receives each problem's collocation residual (Eq. resid) after its last sweep.
 * Synchronises the stream. */
int pfasst_mg_batch_run(pmg_handle h, int steps, int sweeps, double *residuals);

/* Current value of problem `prob` (after batch_run: the end of its last time step). */
int pfasst_mg_batch_get_solution(pmg_handle h, int prob, double *out, int on_device);

/* ---- learned multigrid correction network ----------------------------------- */
/*
 * A small convolutional network that stands in for the second pre-smoothing sweep
 * of the V-cycles (the paper has no learned component; this extends its sub-step
 * solver of Sec. 4.1.1):
 *   y = W3 * relu(W2 * relu(W1 * x + b1) + b2) + b3,
 * three 3x3x3 convolutions with zero padding, channels 1 -> 16 -> 16 -> 1.  On a
 * level with operator I - c Lap_h and diagonal D = 1 + 6 c / h^2 the input is the
 * scaled residual x = D^-1 (f - (I - c Lap_h) e) and y is added to e.
 * Parameters: one float vector of pfasst_mg_net_param_count() = 7809 values,
 *   W1[16][27], b1[16], W2[16 out][27][16 in], b2[16], W3[27][16 in], b3[1],
 *   tap index (dz+1)*9 + (dy+1)*3 + (dx+1).
 * The 16 -> 16 layer runs on the tensor cores with BF16 weights and activations and
 * FP32 accumulation; the other layers and all gradients accumulate in FP32.
 * Training loss, per grid b with its own kappa_b in [0, 1/6], for a power p in 0..3:
 *   0.5 * mean over points of (Ahat_b^p (y - t))^2,  Ahat_b v = v - kappa_b * (sum of
 *   the 6 face neighbours of v), kappa = (c/h^2) / (1 + 6 c/h^2),
 * with t the exact remaining error: p = 0 the plain mean squared error, p = 1 the
 * scaled residual left after adding y, p = 2 the error weighted by the squared
 * eigenvalue of Ahat, which ignores the smooth modes that the coarse-grid correction
 * removes.  Grid arrays of a pmg_net handle are dense float [batch][n][n][n], x fastest.
 */
typedef struct pmg_net *pmg_net_handle;

/* Number of parameters (7809). */
int pfasst_mg_net_param_count(void);

/* He-scaled normal weights from a counter-based generator, zero biases, into params
 * (host, 7809 floats). */
int pfasst_mg_net_init(float *params, unsigned long long seed);

/* Create a trainer for batches of `batch` grids of n^3 points (3 <= n <= 255,
 * batch * n^3 <= 2^28); allocates its device memory with cudaMalloc; the parameters
 * start as pfasst_mg_net_init(seed 5).  Errors: INVALID_ARG, OOM. */
int pfasst_mg_net_create(int batch, int n, void *stream, pmg_net_handle *out);

/* Copy parameters in (host, 7809 floats; also resets the Adam state) or out. */
int pfasst_mg_net_set_params(pmg_net_handle h, const float *params);
int pfasst_mg_net_get_params(pmg_net_handle h, float *params);

/* y = net(x) for the handle's batch; x, y dense [batch][n^3] floats, device memory if
 * on_device, else host.  Synchronises. */
int pfasst_mg_net_forward(pmg_net_handle h, const float *x, float *y, int on_device);

/* Loss (power p) of the inputs x and targets t (layout as above) with kappa (host,
 * batch floats) and its gradient with respect to the 7809 parameters, into grad
 * (host) and *loss (may be NULL).  Synchronises. */
int pfasst_mg_net_gradients(pmg_net_handle h, const float *x, const float *t, const float *kappa, int power,
                            int on_device, float *grad, double *loss);

/* Synthetic training pairs: kappa_b uniform in [kappa_lo, kappa_hi]; an error u_b:
 * uniform noise in [-1, 1] (vcycles_max = 0), or (vcycles_max = K in 1..8, n = 2^p - 1)
 * that noise after k_b V(2,1) red-black cycles, k_b uniform in 0..K, of
 * (I - c_b Lap_h) u = 0 with c_b / h^2 = kappa_b / (1 - 6 kappa_b) -- the errors the
 * multigrid iteration leaves -- scaled to max |u_b| = 1; then t = u_b after one
 * red-black Gauss-Seidel sweep of Ahat t = 0 (red = even 1-based index sum first),
 * i.e. the error a first pre-smoothing sweep leaves, and x = Ahat t.  Noise, kappa
 * and k_b come from counter-based generators of `seed`.  Outputs x, t (layout as
 * above) and kappa (host, batch floats).  Errors: INVALID_ARG. */
int pfasst_mg_net_sample(pmg_net_handle h, unsigned long long seed, double kappa_lo, double kappa_hi,
                         int vcycles_max, float *x, float *t, float *kappa, int on_device);

/* Training pairs from the sub-step problems of an SDC sweep: for every grid b of the
 * batch, u0 (dense FP64 [batch][n^3], device memory if on_device) is the initial value
 * and kappa[b] (host, in [0, 1/6)) fixes c_b / h^2 = kappa_b / (1 - 6 kappa_b).  The
 * library's FP64 multigrid (red-black V(2,1), solved to 1e-12) solves the sub-step
 * (I - c_b Lap_h) u = u0 from the initial guess u0; its initial error e0 = u* - u0 --
 * what the first V-cycle of a sweep's sub-step starts from -- scaled to max |e0| = 1,
 * after one red-black Gauss-Seidel sweep of Ahat t = 0 gives the target t, and x =
 * Ahat t the input (layout and Ahat as for pfasst_mg_net_sample).  Needs n = 2^p - 1.
 * Outputs x, t as [batch][n^3] floats.  Errors: INVALID_ARG, CUDA.  Synchronises. */
int pfasst_mg_net_substep_pairs(pmg_net_handle h, const double *u0, const float *kappa, float *x, float *t,
                                int on_device);

/* `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on the loss of
 * power p, each on a fresh batch from pfasst_mg_net_sample(seed + k * golden,
 * kappa_lo, kappa_hi, vcycles_max).  train_bias = 0 keeps the
 * biases fixed (at zero from the default init: the network is then positively
 * homogeneous, net(a x) = a net(x) for a > 0, as residuals shrink by orders of
 * magnitude over an iteration).  loss_history (host, steps doubles, may be NULL)
 * gets every step's loss.  Errors: INVALID_ARG (steps outside 1..4096, lr <= 0, bad
 * kappa range or vcycles_max, power outside 0..3), DIVERGED (non-finite loss).
 * Synchronises. */
int pfasst_mg_net_train(pmg_net_handle h, int steps, double lr, unsigned long long seed, double kappa_lo,
                        double kappa_hi, int vcycles_max, int power, int train_bias, double *loss_history);

/* One Adam step (as pfasst_mg_net_train) on a caller-supplied batch: inputs x, targets
 * t (layout as above, device memory if on_device), kappa (host, batch floats in
 * [0, 1/6]); *loss (may be NULL) gets the batch loss before the step.  Use it to train
 * on error / residual pairs produced elsewhere, e.g. by another multigrid code.
 * Errors: INVALID_ARG, DIVERGED.  Synchronises. */
int pfasst_mg_net_step(pmg_net_handle h, const float *x, const float *t, const float *kappa, int power, double lr,
                       int train_bias, int on_device, double *loss);

/* Kernel launches issued by the trainer so far. */
long long pfasst_mg_net_launch_count(pmg_net_handle h);

/* CUDA-event timing of the trainer's launches, as pfasst_mg_profile /
 * pfasst_mg_profile_read for a solver handle. */
int pfasst_mg_net_profile(pmg_net_handle h, int enable, long long min_points);
int pfasst_mg_net_profile_read(pmg_net_handle h, pmg_kernel_stat *out, int capacity, int *count);

int pfasst_mg_net_destroy(pmg_net_handle h);
const char *pfasst_mg_net_last_error(pmg_net_handle h);

/* Deploy a network (params, host, 7809 floats; copied) in the V-cycles of h: on
 * multigrid levels with n >= min_n (and n >= 7, never the exact coarsest level) the
 * second pre-smoothing sweep becomes e += net(D^-1 r).  calibrate = 1: measure the
 * V-cycle contraction rho on the fine level (uniform noise, f = 0, the max-norm ratio
 * over V-cycles 2..4, worst over the fine sub-step operators) without the network
 * (*rho_plain) and then add levels finest first, keeping a level only when rho drops
 * (*rho_net = the final rho); levels that do not help keep the plain sweep, and with
 * no level kept the handle runs exactly as before.  calibrate = 2: the same search,
 * judged by the handle's own PFASST iteration instead: the max collocation residual after
 * three iterations from the spread initial value (set it first with
 * pfasst_mg_set_initial), without the network (*rho_plain) and with each level added
 * (*rho_net = the final residual); afterwards the state is the spread initial value
 * again.  calibrate = 0: use every eligible level (*rho_plain and *rho_net are still
 * measured as for calibrate = 1).  *level_mask gets bit l set for level l (0 = finest).  params = NULL removes a deployed network.  The correction allocates up to
 * about 1 GiB of scratch (cudaMalloc; grids of a batch are processed in chunks).
 * Errors: UNSUPPORTED unless dim = 3, red-black Gauss-Seidel and nu1 >= 2, and on
 * batch handles; INVALID_ARG if no level qualifies; OOM.  Synchronises. */
int pfasst_mg_set_smoother_net(pmg_handle h, const float *params, int min_n, int calibrate, double *rho_plain,
                               double *rho_net, int *level_mask);

/* ---- standalone multigrid solve ------------------------------------------ */

/* Solve (I - c Lap_h) u = b (the sub-step operator of Eq. SDCcompactLIII with
 * c = dt_m nu) on `batch` independent grids by V(nu1,nu2)-cycles (Sec. 4.1.1):
 * opt->vcycles cycles, or to opt->mg_tol with the stall rule if vcycles == 0.
 * b, u: device pointers, [batch][n^d] dense; u holds the initial guess and
 * receives the result.  cycles_done (host, may be NULL) gets the V-cycles of the
 * slowest grid.  Allocates its scratch with cudaMallocAsync on `stream` and frees
 * it before returning; synchronises the stream.
 * Errors: INVALID_ARG, OOM, CUDA, DIVERGED. */
int pfasst_mg_helmholtz_solve(const pmg_grid *grid, double c, int batch, const double *b,
                              double *u, const pmg_options *opt, void *stream, int *cycles_done);

/* ---- allocation-free multigrid solve -------------------------------------- */

/* Same computation and arguments as pfasst_mg_helmholtz_solve, for callers that
 * cannot allocate device memory: applications that hand all of the GPU's memory to
 * their own pool allocator at start-up (a raw cudaMalloc then fails or fragments the
 * pool), real-time loops in which cudaMalloc / cudaFree would synchronise the device
 * and stall every other stream, and deployments that forbid allocation after
 * initialisation.  The paper has no counterpart; this is a deployment variant of the
 * solve above.
 *   - Scratch comes from one fixed 32 MiB device array inside this library (held
 *     by every GPU that loads the library until the process exits); no device memory
 *     is allocated or freed (no cudaMalloc, cudaMallocAsync or cudaFree).
 *   - Sizes whose scratch (padded b and u plus the multigrid hierarchy) exceeds
 *     32 MiB are rejected with PMG_ERR_INVALID_ARG and a message giving the need;
 *     e.g. a 3D 63^3 grid fits with batch 1 in FP64, a 3D 31^3 grid with batch 16.
 *   - Only a fixed number of V-cycles (opt->vcycles >= 1) is supported; vcycles == 0
 *     returns PMG_ERR_UNSUPPORTED.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before
 *     any stream capture.
 *   - All calls share the one array, which keeps the last call's contents (each call
 *     clears what it uses first).  Calls whose work overlaps on the GPU -- on
 *     different streams, or from different host threads -- race on it; order them.
 *   - The work is queued on `stream`; the call does not synchronise. */
int pfasst_mg_helmholtz_solve_noalloc(const pmg_grid *grid, double c, int batch, const double *b,
                                      double *u, const pmg_options *opt, void *stream, int *cycles_done);

#ifdef __cplusplus
}
#endif
#endif /* PFASST_MG_H */
