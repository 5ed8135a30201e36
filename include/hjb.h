/*
 * hjb.h -- C ABI of the GB300 (sm_103a) solver for the 2-D second-order HJB
 * equation of a stochastic minimum-time problem, discretised by the
 * Markov-chain semi-Lagrangian scheme without self-dependency and solved inside
 * the patchy (dynamic) domain decomposition of Cacace & Falcone, "A dynamic
 * domain decomposition for a class of second order semi-linear equations".
 *
 * Problem (Section 3, eqs. HJB2 and SDE, with a discount):
 *     dX = f(X, a) dt + sigma dW,   f(x, a) = b(x) + c(x) a,   l = const,
 *     u = 0 on the target, value = E[ int_0^tau e^{-lambda t} l dt ].
 *   hjb_create_problem_general adds the general terms of Section 5.3: sigma(x)
 *   per node, the diffusion sigma(x) a along the control, l(x, a) = l(x) + m(a).
 * Scheme (Section 3, eq. SLscheme3; 2-D isotropic form of Section 4.1):
 *     for every free node x_i and control a in the discrete set A,
 *       x_{i,k}^{a,s} = x_i + h f(x_i, a) + s sqrt(2h) sigma e_k   (k = 1,2, s = +-1),
 *       u(x_i) = min_a ( beta Lambda1'(a) + h l ) / ( 1 - beta Lambda0(a) ),
 *     with Q1 interpolation, beta = 1/(1 + lambda h), points projected onto the
 *     square, Lambda0 the self weights and Lambda1' the rest (eq. self-dependency).
 *
 * Grid: n nodes per side on [-1,1]^2, dx = 2/(n-1); node (i, j) sits at
 * (-1 + i dx, -1 + j dx) and every per-node array is row-major with i fastest:
 * element k = j*n + i.
 *
 * Call order (Section 4.3, the patchy algorithm):
 *   hjb_create_problem  -> hjb_coarse_solve -> hjb_build_patches -> hjb_solve_patches
 *   hjb_solve_full (plain full-grid value iteration, the static comparator) may be
 *   called at any time after creation.
 *
 * Conventions shared by every entry point:
 *   - Return value: HJB_OK (0) or a negative HJB_ERR_* code.  The library never
 *     aborts the process; hjb_last_error() gives a one-line message for the
 *     calling thread.  After HJB_ERR_CUDA the problem must be destroyed.
 *   - Host pointers are plain host memory (pageable or pinned); the library
 *     copies inputs at the call and writes outputs into caller-owned buffers
 *     before returning.  The library owns every device buffer it allocates.
 *   - All device work of a problem runs on the stream given at creation (NULL:
 *     a stream the library creates).  Entry points that return host data
 *     synchronise that stream.
 *   - A problem object may be used by one host thread at a time.
 *   - Device memory comes from a stream-ordered pool per device that keeps the
 *     blocks of destroyed problems for the next ones (hjb_trim_memory releases
 *     them).  The per-node input arrays are checked on the device right after
 *     they are uploaded; a bad entry fails the creation with HJB_ERR_INVALID_ARG
 *     and its index in hjb_last_error().
 */
#ifndef HJB_H
#define HJB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HJB_OK                  0
#define HJB_ERR_INVALID_ARG    -1   /* bad size, NULL pointer, NaN/Inf input, non-nesting grids */
#define HJB_ERR_CUDA           -2   /* a CUDA runtime call failed                               */
#define HJB_ERR_OOM            -3   /* device allocation failed                                 */
#define HJB_ERR_STATE          -4   /* call out of order (e.g. solve_patches before build)      */
#define HJB_ERR_NOT_CONVERGED  -5   /* sweep/pass cap reached; the state is valid               */
#define HJB_ERR_TIMEOUT        -6   /* a device-side wait hit its time limit; state is valid   */

#define HJB_MASK_FREE      0
#define HJB_MASK_TARGET    1
#define HJB_MASK_OBSTACLE  2

#define HJB_MAX_CONTROLS 255
#define HJB_MAX_PATCHES  126

typedef struct hjb_problem hjb_problem;

/* Problem description (Section 3 data, Section 4.3 initialisation). */
typedef struct {
    int32_t n;            /* nodes per side of the fine grid G, 3 <= n <= 16385             */
    int32_t n_controls;   /* N_A: points discretising the control set, 1..255              */
    double  h;            /* time step; <= 0 selects h = dx                                  */
    double  lambda;       /* discount rate >= 0; beta = 1/(1 + lambda h)                     */
    double  sigma;        /* diffusion >= 0; points at +-sqrt(2h) sigma e_k                  */
    double  cost;         /* running cost l > 0 (constant)                                   */
    int32_t coarse_n;     /* nodes per side of the coarse grid G_c; (n-1) % (coarse_n-1) == 0;
                             0 = no coarse grid (coarse_solve / build_patches unavailable)    */
    int32_t n_patches;    /* N_P: number of boundary subsets Gamma_p, 1..126                 */
    int32_t scheme;       /* 3: modified scheme SLscheme3 (default), 2: original SLscheme2   */
    double  band_width;   /* width of the causal bands in units of h (<= 0: 1.0)             */
    int32_t band_window;  /* passes > 0 revisit a group of bands if a group within this many
                             bands changed by more than the tolerance (<= 0: 8)               */
    int32_t band_group;   /* band schedule: consecutive bands per grid-wide wave (<= 0: 1)    */
    int32_t wave_warps;   /* warps of the band-wave / tile kernels (<= 0: every co-resident
                             warp)                                                             */
    int32_t resort_passes;/* after each of the first k FP32 passes, re-sort the free nodes by
                             the current value instead of u_hat (0: never)                    */
    int32_t schedule;     /* patch-solve schedule: 0 warp tiles (default; the FP32 phase as
                             in 4 up to n = 3073, as in 3 above), 1 band waves, 2 block
                             tiles, 3 warp tiles from an asynchronous worklist (no grid-wide
                             barrier), 4 warp tiles in barrier-separated steps             */
    int32_t tile_waves;   /* tile schedule: bands per tile wave B (<= 0: automatic, 1 when the
                             diffusion offset sqrt(2h) sigma exceeds one cell, else 2)        */
    int32_t tile_period;  /* tile schedule: period D of the cyclic schedule (<= 0: 1 for warp
                             tiles, 2 for block tiles)                                        */
    int32_t local_sweeps; /* tile schedule: ordered sweeps of a tile per visit (<= 0: automatic,
                             3 with 32-node warp-tile visits, else 1)                        */
    int32_t tile_shape;   /* warp tiles: 0 8x8 nodes, 1 8x4, 2 4x4, -1 automatic (8x8 when the
                             diffusion offset exceeds one cell, n > 2049 or more than 32
                             controls, else 8x4)                                              */
    int32_t visit;        /* warp tiles, FP32: how a warp updates a tile's nodes: 1 one node
                             at a time (a control per lane, warp minimum, Gauss-Seidel through
                             the tile), 2 32 nodes at a time (a node per lane, every control
                             in the lane), 3 two nodes at a time (16 lanes each; interior
                             tiles, 1 elsewhere): four controls a lane with 64 controls closed
                             under quarter turns (a_{m+16} = (-a_m.y, a_m.x), a_{m+32} = -a_m,
                             to 1e-12), two with 32 in opposite pairs (a_{m+16} = -a_m), 1 for
                             other control sets; 4 four nodes at a time (8 lanes each, four
                             controls a lane: 32 controls closed under quarter turns); 0
                             automatic (4 for such 32 controls, 3 for such 64, else 1)        */
} hjb_desc;

/* Per-call statistics; every field is written by the call that receives it. */
typedef struct {
    int32_t sweeps;                /* full sweeps (solve_full, coarse_solve) or passes (solve_patches) */
    int32_t status;                /* the call's return code                                     */
    int64_t node_updates;          /* free-node scheme evaluations performed                     */
    int64_t node_control_updates;  /* node_updates x N_A                                          */
    double  residual;              /* FP64 sup-residual ||T u - u||_inf (eq. SLscheme2), or -1    */
    double  increment;             /* last sup-increment of the iteration                        */
    double  ms_total;              /* device time of the call (CUDA events)                      */
    double  ms_stage[8];           /* per-stage device time, see each entry point                */
    int32_t fp32_passes;           /* solve_patches / solve_full: passes (sweeps) in FP32         */
    int32_t fp64_passes;           /* passes (sweeps) in FP64                                     */
    int64_t fp64_node_updates;     /* the part of node_updates done in FP64                       */
    int32_t residual_evals;        /* FP64 residual evaluations (full-grid operator applications) */
    int32_t corr_sweeps;           /* solve_patches: FP32 sweeps of the FP64 stage's correction
                                      equation (one control per node; part of node_updates)     */
} hjb_stats;

/* Regime of the upwind diffusion-ball condition (Section 4.1, eqs. upper-bound,
 * lower-bound, upper-alpha, lower-alpha, hyperbolicity) for a problem with speed
 * range [f_min, f_max] and diffusion eps (paper's notation; eps = sigma^2 here). */
typedef struct {
    double upsilon;      /* f_max / f_min                                     */
    double omega;        /* f_min / (2 eps)                                    */
    double alpha_lower;  /* 1/(omega dx)                      (eq. lower-alpha) */
    double alpha_upper;  /* 1/Upsilon - (sqrt(1+4 omega dx Upsilon)-1)/(2 omega dx Upsilon^2) (eq. upper-alpha) */
    double alpha;        /* 1/(1+Upsilon), the choice valid whenever the condition holds */
    double tau_dx;       /* dx/(1+Upsilon): the condition is 1/omega < tau_dx (eq. hyperbolicity) */
    double eps_threshold;/* eps below which the condition holds: f_min dx / (2 (1+Upsilon)) */
    double h;            /* alpha dx / f_min                                    */
    int32_t holds;       /* 1 if 1/omega < tau_dx                               */
    int32_t upper_ok;    /* h f_max + sqrt(2 eps h) < dx at h   (eq. upper-bound) */
    int32_t lower_ok;    /* h f_min - sqrt(2 eps h) > 0 at h    (eq. lower-bound) */
    int32_t reach_cells; /* ceil((h f_max + sqrt(2 eps h)) / dx): interpolation reach */
} hjb_regime_info;

/* hjb_regime -- host-only, no GPU needed.  Section 4.1.  dx > 0, 0 < f_min <= f_max,
 * eps >= 0 (eps = 0: omega = +inf, the condition holds).  Returns HJB_OK or
 * HJB_ERR_INVALID_ARG. */
int hjb_regime(double dx, double f_min, double f_max, double eps, hjb_regime_info* out);

/* hjb_create_problem -- Section 4.3 "Initialization": builds G (and G_c when
 * desc->coarse_n > 0), uploads the data and the control set.
 *   speed    : host float[n*n], c(x) >= 0 (finite).
 *   mask     : host uint8[n*n], HJB_MASK_*; target nodes hold u = g = 0, obstacle
 *              nodes hold l/(lambda) + h l (the value of never reaching the target).
 *   sector   : host int8[n*n], the boundary subset Gamma_p of each target node
 *              (0..n_patches-1) or -1; may be NULL when no patches are built.
 *   controls : host double[2*n_controls], a_m = (controls[2m], controls[2m+1]).
 *   drift    : host float[2*n*n] interleaved (b_x, b_y) or NULL (b = 0).
 *   cuda_stream : a cudaStream_t owned by the caller, or NULL.
 *   out      : receives the new problem (NULL on failure).
 * Errors: HJB_ERR_INVALID_ARG (sizes, NULL, NaN/Inf, lambda = 0 with obstacles,
 * non-nesting coarse grid), HJB_ERR_OOM, HJB_ERR_CUDA.  The initial value is
 * u = 0 on free nodes. */
int hjb_create_problem(const hjb_desc* desc, const float* speed, const uint8_t* mask,
                       const int8_t* sector, const double* controls, const float* drift,
                       void* cuda_stream, hjb_problem** out);

/* General terms of Section 5.3 (eqs. s123, l123 and the degenerate diffusion of
 * Section 5.2), all optional:
 *     sigma(x, a) = sqrt(2) sigma(x) I_2  (HJB_DIFFUSION_ISOTROPIC: the four points
 *                   x + h f +- sqrt(2h) sigma(x) e_k, weight 1/4 each), or
 *     sigma(x, a) = sqrt(2) sigma(x) a    (HJB_DIFFUSION_CONTROL: a one-dimensional
 *                   Wiener process along the control, the two points
 *                   x + h f +- sqrt(2h) sigma(x) a, weight 1/2 each),
 *     l(x, a)     = l(x) + m(a).
 * The paper's d_eps(x) = sqrt(2 eps) chi_{x2 >= 0} is sigma(x) = sqrt(eps) chi. */
#define HJB_DIFFUSION_ISOTROPIC 0
#define HJB_DIFFUSION_CONTROL 1
typedef struct {
    const float*  sigma_field;   /* host float[n*n], sigma(x) >= 0 (finite), or NULL: desc->sigma
                                    everywhere; when given, desc->sigma is ignored              */
    int32_t       diffusion;     /* HJB_DIFFUSION_ISOTROPIC or HJB_DIFFUSION_CONTROL            */
    int32_t       reserved;      /* must be 0                                                   */
    const float*  cost_field;    /* host float[n*n], l(x) > 0 (finite), or NULL: desc->cost     */
    const double* control_cost;  /* host double[n_controls], m(a_m) >= 0 (finite), or NULL: 0   */
} hjb_terms;

/* hjb_create_problem_general -- hjb_create_problem with the general terms above
 * (terms may be NULL: the constant-coefficient problem).  The arrays are copied;
 * the coarse grid takes l(x) at its nested nodes (and no diffusion, as always).
 * The obstacle value and the initial coarse value use the largest running cost
 * max l(x) + max m(a).  Every entry point accepts the problem; the kernels
 * evaluate the general terms on the per-node path (the FP32 software-pipelined
 * tile path serves constant coefficients only).  Errors: as hjb_create_problem,
 * plus HJB_ERR_INVALID_ARG for a negative / non-finite sigma(x) or m(a), a
 * non-positive / non-finite l(x), an unknown diffusion or reserved != 0. */
int hjb_create_problem_general(const hjb_desc* desc, const float* speed, const uint8_t* mask,
                               const int8_t* sector, const double* controls, const float* drift,
                               const hjb_terms* terms, void* cuda_stream, hjb_problem** out);

/* hjb_trim_memory -- the problems' device memory comes from a stream-ordered pool
 * per device that keeps the blocks of destroyed problems for the next ones (no
 * device-wide synchronisation on create / destroy).  This releases every cached
 * block that no live problem holds.  Returns HJB_OK or HJB_ERR_CUDA. */
int hjb_trim_memory(void);

/* hjb_create_problem_device -- as hjb_create_problem, but speed, mask, sector and
 * drift are DEVICE pointers (e.g. torch CUDA tensors' data_ptr) on the current
 * device; they are copied device-to-device on cuda_stream.  controls stays a host
 * pointer. */
int hjb_create_problem_device(const hjb_desc* desc, const float* speed, const uint8_t* mask,
                              const int8_t* sector, const double* controls,
                              const float* drift, void* cuda_stream, hjb_problem** out);

/* hjb_coarse_solve -- Section 4.3 "Pre-computation", first item: starting from
 * u_c^0 = l(1/lambda + h) off the target (the paper's "very big value"), iterate
 * SLscheme3 with sigma = 0 on G_c (one cooperative launch: each block keeps a
 * tile of G_c resident and relaxes it in place, a warp per node, between grid
 * barriers -- the paper's "standard (static) domain decomposition" of the coarse
 * solve with one tile per SM) until the sup-increment of the first relaxation
 * after each exchange is <= tol_c (raised to the FP32 floor of the values; without
 * a discount the floor follows the largest value).  stats->sweeps counts global
 * sweeps (each with 4 local relaxations).  G_c is
 * nested in G: coarse node (I,J) is fine node (rI, rJ), r = (n-1)/(coarse_n-1);
 * its speed is the fine speed there; it is a target when a fine target node lies
 * within r/2 fine cells in both axes, else an obstacle when its fine node is one.
 * Time step h_c = h r.  ms_stage[0] = coarse solve.
 * Errors: HJB_ERR_STATE (no coarse grid), HJB_ERR_NOT_CONVERGED (max_sweeps). */
int hjb_coarse_solve(hjb_problem* p, double tol_c, int32_t max_sweeps, hjb_stats* stats);

/* hjb_build_patches -- Section 4.3 "Pre-computation", remaining items:
 *   u_hat = Q1 interpolation of u_c on G (also the initial value of the fine
 *           iteration: "starting from u_hat");
 *   a*    = argmin_a beta u_hat(x_i + h f(x_i,a)) + h l  (eq. discrete-synthesis),
 *           ties to the lowest control index;
 *   labels: winner-take-all reading of eq. discrete-advection -- each free node
 *           takes the patch at the end of its successor chain, the successor being
 *           the heaviest Q1 vertex of the foot x_i + h f(x_i, a*) other than x_i
 *           (foot computed by a fixed FP32 operation sequence); chains ending in a
 *           cycle or at an obstacle get label n_patches ("leftover");
 *   order : free nodes grouped by (causal band, patch), bands by increasing
 *           travel time T(u_hat) = -log(1 - lambda u_hat)/lambda (Section 4.2).
 * ms_stage: [0] interpolation, [1] synthesis + band keys, [2] successors + labels,
 * [3] ordering.  Errors: HJB_ERR_STATE (coarse_solve not run). */
int hjb_build_patches(hjb_problem* p, hjb_stats* stats);

/* hjb_set_uhat -- replace u_hat by the caller's host float[n*n] (finite values on
 * free nodes; the fixed values are taken elsewhere) and redo what follows it in
 * Section 4.3 "Pre-computation": the synthesis a* (eq. discrete-synthesis) with
 * the causal band keys of Section 4.2, successors, labels, ordering, tiles, and
 * the start value u = u_hat.  Lets a caller (a test) run the pre-computation on a
 * u_hat computed elsewhere.  Band key of a value u (exact, FP64): with lambda > 0
 * the number of edges e_k = (1 - exp(-(lambda (k w)))) / lambda, k = 1 .. L-1,
 * that are <= u, with w = band_width h and L = min(2^20, floor(log(1e6)/(lambda w))
 * + 2); with lambda = 0, floor(u / w).  Requires build_patches.
 * Errors: HJB_ERR_INVALID_ARG (NULL, non-finite value), HJB_ERR_STATE. */
int hjb_set_uhat(hjb_problem* p, const float* uhat);

/* hjb_set_feedback -- replace a* by the caller's host uint8[n*n] (values < N_A on
 * free nodes, ignored elsewhere) and recompute successors, labels and ordering
 * from it (the band keys keep u_hat).  Requires build_patches. */
int hjb_set_feedback(hjb_problem* p, const uint8_t* a);

/* hjb_solve_patches -- Section 4.3 "Computation": from the current value (u_hat
 * after build_patches), iterate SLscheme3 (with sigma) in place on the single
 * shared array (sharp interfaces: the transmission condition is the identity),
 * following the causal bands.  Schedules 0 and 2 (tile-pipelined): tiles staged
 * in shared memory -- 0: one warp per 8x8 (or tile_shape) tile visiting the
 * tile's nodes one by one in increasing u_hat; 2: one block per 16x16 tile visiting its bands in
 * order -- tiles grouped into waves by their lowest band and run on a cyclic
 * schedule of period D (one grid-wide barrier per step).  Schedule 0 visits a
 * tile at its wave and afterwards only when a tile within the interpolation
 * reach changed by more than the tolerance (per-step tile queues); schedule 2
 * skips tiles whose neighbourhood did not change.  Converged when no tile
 * visited in the last D steps changed by more than the tolerance ("passes" in
 * the stats count pipeline steps).  Schedule 1
 * (band waves): band_group bands per grid-wide wave, nodes taken in sorted order
 * by the wave_warps warps in flight; passes after the first skip groups whose
 * neighbourhood did not change.  FP32 until a
 * pass's sup-increment is <= tol32 (raised to the FP32 floor
 * 1.01 * 2^-23 * max(1, U) * A, where U bounds the values -- l/lambda + h l, or
 * without a discount four times the largest coarse value -- and A >= 1 is the
 * 1 / (1 - beta Lambda0) amplification of the scheme, about dx / (h mean|f|));
 * then, if tol64 > 0, the FP64 sup-residual
 * ||T2 u - u|| is evaluated; if it exceeds tol64 while tol64 is at least 2^-22
 * max(1, U) A, at most two more FP32 phases run from the current value with
 * the tolerance divided by 4 each time while it stays >= 2^-21 max(1, U) A
 * (schedule 0, every tile visited in the first two steps in checkerboard
 * order); then, for constant coefficients with a discount (lambda > 0) and
 * scheme 3, at most 12 rounds of mixed-precision correction: from the FP64
 * residual r = T2 u - u and its minimising control a per node, FP32 Jacobi
 * sweeps of e = beta P_a e + r (one control per node), u += e in FP64, the FP64
 * residual again (Howard's policy iteration; stops at tol64, after two rounds
 * in a row that do not halve the residual, or if it grows 1e3-fold); then FP64
 * passes until the FP64 sup-residual is <= tol64.  max_passes caps each phase.
 * ms_stage: [0] FP32 passes, [1] promotion + residuals, [2] correction rounds
 * and FP64 passes.  The worklist (schedule 3) stops putting back a tile after
 * min(max_passes, 4096) visits of it (FP32 rounding can keep a few tiles
 * changing by more than a tol32 below what FP32 resolves there); the FP32 phase
 * then counts as not converged.  With tol64 > 0 the FP64 stage runs whether or
 * not the FP32 phase converged, and the FP64 residual decides the status.
 * Errors: HJB_ERR_STATE (build_patches not run), HJB_ERR_NOT_CONVERGED (tol64 = 0
 * and the FP32 phase did not converge, or the FP64 residual stays above tol64),
 * HJB_ERR_TIMEOUT (a grid-wide wait exceeded its limit). */
int hjb_solve_patches(hjb_problem* p, double tol32, double tol64, int32_t max_passes,
                      hjb_stats* stats);

/* hjb_solve_full -- plain full-grid Jacobi value iteration (the static comparator
 * of Section 5.4, without decomposition or ordering): from u = 0, u <- T u on every
 * free node until the sup-increment is <= tol, in FP32 (precision = 32) or FP64
 * (precision = 64).  For precision 32 and tol64 > 0, FP64 Jacobi sweeps follow
 * until the FP64 sup-increment (= residual) is <= tol64.  max_sweeps caps each
 * phase.  ms_stage: [0] FP32 sweeps, [1] FP64 sweeps. */
int hjb_solve_full(hjb_problem* p, int32_t precision, double tol, double tol64,
                   int32_t max_sweeps, hjb_stats* stats);

/* hjb_apply_operator -- one application of the scheme operator to a caller's
 * value: out = T u on free nodes (u on the others), and argmin = the minimising
 * control (-1 on non-free nodes; may be NULL).  precision 32 or 64, scheme 2 or 3.
 * u, out: host double[n*n].  Used to check the operator itself at any size. */
int hjb_apply_operator(hjb_problem* p, int32_t precision, int32_t scheme, const double* u,
                       double* out, int32_t* argmin);

/* hjb_residual -- FP64 sup-residual ||T2 u - u||_inf of the current value. */
int hjb_residual(hjb_problem* p, double* residual);

/* hjb_set_value -- warm start / resume: the current value becomes host double[n*n]
 * (non-free nodes are reset to their fixed values).  Both precisions are set. */
int hjb_set_value(hjb_problem* p, const double* u);

/* hjb_get_value -- the current value (FP64 copy when the last solve ended in
 * FP64, else FP32 widened) into host double[n*n].  Merge of Section 4.3 is
 * implicit: all patches share one array. */
int hjb_get_value(hjb_problem* p, double* u_out);

/* hjb_get_coarse_value -- u_c into host double[coarse_n^2]. */
int hjb_get_coarse_value(hjb_problem* p, double* uc_out);

/* hjb_get_uhat -- u_hat (FP32 widened) into host double[n*n]. */
int hjb_get_uhat(hjb_problem* p, double* uhat_out);

/* hjb_get_feedback -- a* into host uint8[n*n] (255 on non-free nodes). */
int hjb_get_feedback(hjb_problem* p, uint8_t* a_out);

/* hjb_get_successors -- successor of each node into host int32[n*n] (self on
 * non-free nodes). */
int hjb_get_successors(hjb_problem* p, int32_t* succ_out);

/* hjb_get_labels -- patch label of each node into host int8[n*n]: 0..N_P-1, or
 * N_P for leftover / obstacle nodes; target nodes carry their sector. */
int hjb_get_labels(hjb_problem* p, int8_t* label_out);

/* hjb_get_order -- the ordering: band key of each node into host int32[n*n] (-1
 * on non-free nodes, may be NULL), the node list into host int32[n_free] (may be
 * NULL), the band offsets into host int32[n_bands+1] (may be NULL).  *n_free and
 * *n_bands receive the sizes (may be NULL). */
int hjb_get_order(hjb_problem* p, int32_t* keys_out, int32_t* order_out,
                  int32_t* band_off_out, int32_t* n_free, int32_t* n_bands);

/* hjb_device_info -- SM count and the number of co-resident blocks the band-wave
 * kernel runs with (FP32 and FP64), for reporting. */
int hjb_device_info(hjb_problem* p, int32_t* num_sms, int32_t* wave_blocks32,
                    int32_t* wave_blocks64);

/* hjb_residual_noalloc -- the FP64 sup-residual ||T2 u - u||_inf of hjb_residual,
 * for a value field the caller holds, computed without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory where they need the residual -- a loop with a latency
 * budget (cudaMalloc/cudaFree may synchronise the device) or a process whose device
 * memory is wholly owned by another allocator (a caching pool, a fixed budget).
 *   desc     : host; uses n, n_controls, h, lambda, sigma, cost (no coarse grid).
 *   speed, mask, drift (nullable), u : DEVICE arrays with the layouts of
 *              hjb_create_problem (u: double[n*n], 8-byte aligned; drift 8-byte
 *              aligned); controls: DEVICE double[2*n_controls] (16-byte aligned);
 *              residual_out: DEVICE double[1] (written by the call).
 *              u is read at free nodes only: target nodes count as 0 and obstacle
 *              nodes as h l/(1 - beta) (1e6 when lambda = 0), the values the
 *              solver holds there, whatever u contains at those nodes.
 *              A non-finite increment at any free node (NaN or Inf in u, or in
 *              the inputs it meets) makes *residual_out = +Inf.
 *   cuda_stream: the stream the work is queued on (NULL: the legacy default stream);
 *              the call returns before the result is ready.
 * Scratch: one partial maximum per 32x16-node tile, held in a fixed device array of
 * 65536 doubles (512 KiB) that every GPU loading the library keeps until exit; grids
 * with more tiles, ceil(n/32) * ceil(n/16) > 65536 (n >= 5793), are rejected with
 * HJB_ERR_INVALID_ARG before any device work.
 * Every call overwrites the partials it reads, so nothing needs clearing, but all
 * calls share the one array: calls whose work overlaps on the GPU race.  The first
 * call on a device resolves the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 * Errors: HJB_ERR_INVALID_ARG (NULL pointers, sizes, misalignment), HJB_ERR_CUDA. */
int hjb_residual_noalloc(const hjb_desc* desc, const float* speed, const uint8_t* mask,
                         const float* drift, const double* controls, const double* u,
                         double* residual_out, void* cuda_stream);

/* hjb_destroy -- frees every device buffer and the stream the library created.
 * NULL is ignored. */
void hjb_destroy(hjb_problem* p);

/* hjb_status_string -- static text for a return code. */
const char* hjb_status_string(int code);

/* hjb_last_error -- message of the last failure on the calling thread ("" if none). */
const char* hjb_last_error(void);

/* hjb_kernel_launches -- number of CUDA kernels this library has launched since it
 * was loaded (all problems, all threads); a reporting aid for benchmarks. */
long long hjb_kernel_launches(void);

/* FP32 tolerances (tol_c, tol32 and the FP32 Jacobi tolerance) below half an FP32
 * ulp of the largest value, 1.01 * 2^-23 * max(1, u_max), are raised to it: at the
 * FP32 fixed point each node's increment can be that large, so a smaller
 * tolerance could stall until the pass cap.  u_max = l/lambda + h l (the coarse
 * grid's h_c for tol_c). */

/* ===================================================================== batches
 * Many independent problems solved together: the patchy pipeline of Section 4.3
 * (coarse solve -> interpolation -> synthesis -> labels -> ordering -> patch
 * solve -> FP64 residual / polish) with every stage one launch over all the
 * instances, and the patch solve one persistent launch whose steps carry the
 * tiles of every instance.  Each instance has its own grid size, speed, mask,
 * sectors, h, lambda, sigma, coarse grid and patch count; the control set, the
 * scheme and the running cost l are shared.  No drift field. */
typedef struct hjb_batch hjb_batch;

typedef struct {
    int32_t n;            /* nodes per side, 9..16385                                      */
    int32_t coarse_n;     /* coarse nodes per side, >= 5, (n-1) % (coarse_n-1) == 0       */
    int32_t n_patches;    /* sectors Gamma_p, 1..HJB_MAX_PATCHES                           */
    int32_t reserved;     /* must be 0                                                     */
    double h;             /* time step (<= 0: h = dx)                                      */
    double lambda;        /* discount rate, > 0                                            */
    double sigma;         /* diffusion (>= 0)                                              */
} hjb_batch_inst;

typedef struct {
    int32_t n_controls;   /* shared control set, 1..HJB_MAX_CONTROLS                        */
    int32_t scheme;       /* 3 (SLscheme3, default when 0) or 2                            */
    int32_t tile_shape;   /* warp tiles: 0 8x8, 1 8x4, 2 4x4, -1: 8x4 until tuned          */
    int32_t tile_waves;   /* bands per tile wave B (<= 0: 2 until tuned)                   */
    int32_t tile_period;  /* period D of the tile schedule (<= 0: 2)                       */
    int32_t schedule;     /* FP32 passes: 0 barrier-separated steps (hjb_batch_autotune may
                             switch to 3), 3 the asynchronous worklist of hjb_desc.schedule 3,
                             4 barrier-separated steps, never switched                       */
    double cost;          /* running cost l (> 0)                                          */
    double band_width;    /* causal band width in units of h (<= 0: 1)                    */
} hjb_batch_desc;

/* hjb_batch_create -- copies `count` instances to the device.  speed, mask and
 * sector are the instances' n*n arrays (row-major, i fastest) concatenated in
 * instance order; sector may be NULL (every target node in sector 0);
 * controls: n_controls (a_x, a_y) pairs.  Ownership as hjb_create_problem.
 * Errors: HJB_ERR_INVALID_ARG (count < 1, a bad instance: its index is in
 * hjb_last_error), HJB_ERR_OOM, HJB_ERR_CUDA. */
int hjb_batch_create(const hjb_batch_desc* desc, int32_t count, const hjb_batch_inst* insts,
                     const float* speed, const uint8_t* mask, const int8_t* sector,
                     const double* controls, void* cuda_stream, hjb_batch** out);

/* hjb_batch_create_lists -- hjb_batch_create with one host array per instance:
 * speed[i], mask[i] (and sector[i], when sector is not NULL; a NULL sector list
 * or entry gives sector 0 on target nodes, -1 elsewhere) hold instance i's
 * n_i x n_i field.  The library copies each into its place on the device, so the
 * caller never concatenates the instances.  Same checks and errors. */
int hjb_batch_create_lists(const hjb_batch_desc* desc, int32_t count, const hjb_batch_inst* insts,
                           const float* const* speed, const uint8_t* const* mask,
                           const int8_t* const* sector, const double* controls, void* cuda_stream,
                           hjb_batch** out);

/* hjb_batch_solve -- the whole patchy pipeline for every instance: coarse solves
 * until the sup-increment is <= tol_c, pre-computation, FP32 warp-tile passes
 * until no tile changes by more than tol32, the FP64 sup-residual ||T2 u - u||
 * of every instance, then FP64 passes for the instances above tol64 (if tol64 >
 * 0).  residuals (nullable, count doubles) receives each instance's final FP64
 * residual.  stats: node_updates = fine-grid updates of the FP32 and FP64
 * passes, node_control_updates = every scheme evaluation (coarse sweeps, fine
 * passes, residuals) times n_controls, residual = the largest, fp32_passes =
 * pipeline steps; ms_stage: [0] FP32
 * passes, [1] residuals, [2] FP64 passes, [3] coarse solves, [4] pre-computation.
 * An instance above tol64 first gets at most two more FP32 phases (tolerance /4
 * each, while above the FP32 floor), then (scheme 3) at most 12 rounds of the
 * mixed-precision correction of hjb_solve_patches, per instance (an instance
 * leaves after two rounds in a row that do not halve its residual), then FP64
 * passes; the FP32 phases and FP64 passes start warm (that instance's tiles
 * visited once in checkerboard order, then the queues).  stats->corr_sweeps:
 * the correction sweeps (each instance's count, the largest per round, summed).  The
 * worklist schedule caps the visits of one tile as hjb_solve_patches does; with
 * tol64 > 0 the FP64 residuals decide the status.  The FP32 passes update the
 * nodes of interior tiles in groups as hjb_desc.visit 4 (32 controls closed under
 * quarter turns) or 3 (32 in opposite pairs) does, else one at a time.
 * Errors: HJB_ERR_NOT_CONVERGED (a cap was hit, or an FP64 residual stays above
 * tol64; values valid), HJB_ERR_TIMEOUT. */
int hjb_batch_solve(hjb_batch* b, double tol_c, double tol32, double tol64, int32_t max_passes,
                    hjb_stats* stats, double* residuals);

/* hjb_batch_solve_full -- the plain comparator for every instance: full-grid FP32
 * Jacobi sweeps from u = 0 (one launch per sweep over the instances not yet
 * converged) until an instance's sup-increment is <= tol32, then its FP64
 * residual; instances above tol64 continue with the tolerance divided by 4 (at
 * most 3 times).  Same outputs as hjb_batch_solve; fp32_passes = sweeps of the
 * slowest instance. */
int hjb_batch_solve_full(hjb_batch* b, double tol32, double tol64, int32_t max_sweeps,
                         hjb_stats* stats, double* residuals);

/* hjb_batch_autotune -- runs the pre-computation once, then the FP32 patch solve
 * for each candidate schedule (barrier steps with tile shapes 8x8, 8x4, 4x4 x bands
 * per wave 1, 2; with desc.schedule 0 also the asynchronous worklist with each
 * shape), times each with CUDA events and keeps the fastest for later solves.
 * ms_out (nullable, 9 doubles) gets the candidates' times in that order (entries
 * 6..8: the worklist, 0 when not tried); shape_out / waves_out (nullable) the
 * choice (the worklist was chosen when the smallest time is among entries 6..8). */
int hjb_batch_autotune(hjb_batch* b, double tol_c, double tol32, int32_t* shape_out,
                       int32_t* waves_out, double* ms_out);

/* hjb_batch_get_value -- instance `index`'s current value (n*n doubles). */
int hjb_batch_get_value(const hjb_batch* b, int32_t index, double* u_out);

/* hjb_batch_get_values -- every instance's current value in one read-back:
 * u_out (host, caller-owned) holds sum_i n_i^2 doubles, instance i's n_i x n_i
 * field (the layout of hjb_create_problem) starting after those of instances
 * 0 .. i-1.  One device-to-host copy and one stream synchronisation. */
int hjb_batch_get_values(const hjb_batch* b, double* u_out);

/* hjb_batch_get_feedback / hjb_batch_get_labels -- instance `index`'s a*
 * (255 on non-free nodes) and patch labels after a solve. */
int hjb_batch_get_feedback(const hjb_batch* b, int32_t index, uint8_t* a_out);
int hjb_batch_get_labels(const hjb_batch* b, int32_t index, int8_t* label_out);

/* hjb_batch_get_uhat -- instance `index`'s interpolated coarse value u_hat. */
int hjb_batch_get_uhat(const hjb_batch* b, int32_t index, float* uhat_out);

/* hjb_batch_coarse_solve -- the coarse solves alone (Section 4.3 "Pre-computation",
 * sigma = 0) until each instance's sup-increment is <= tol_c; sweeps_out /
 * fallback_out (nullable, count entries): sweeps per instance, 1 where a warm
 * start fell back to the plain start.  stats: node updates, ms_total. */
int hjb_batch_coarse_solve(hjb_batch* b, double tol_c, int32_t max_sweeps, hjb_stats* stats,
                           int32_t* sweeps_out, uint8_t* fallback_out);

/* hjb_batch_precompute -- coarse solves, interpolation, synthesis, labels (no
 * patch solve): u_hat, a* and the coarse values become readable. */
int hjb_batch_precompute(hjb_batch* b, double tol_c, hjb_stats* stats);

/* hjb_batch_get_coarse_value -- instance `index`'s coarse value (coarse_n^2 floats). */
int hjb_batch_get_coarse_value(const hjb_batch* b, int32_t index, float* uc_out);

/* hjb_batch_net_inputs -- the warm-start network's input for every instance (all
 * instances must share one coarse size nc): DEVICE bf16 [count][nc][nc][16],
 * channels speed / 2, target indicator, obstacle indicator, 10 sigma, lambda / 2,
 * then zeros, from the coarse data. */
int hjb_batch_net_inputs(const hjb_batch* b, void* x);

/* hjb_batch_net_targets -- after hjb_batch_precompute: the warm-start network's
 * training targets on every instance's coarse grid (DEVICE, [count][nc][nc]):
 * tval = u_c / u_max, tctrl = a* of the fine node under each coarse node, freem = 1
 * on free coarse nodes (0 elsewhere, where tctrl is 0). */
int hjb_batch_net_targets(const hjb_batch* b, float* tval, uint8_t* tctrl, uint8_t* freem);

/* hjb_batch_coarse_warm -- later coarse solves start the free nodes of instances
 * [first, first + count) from the network output net_out (DEVICE FP32
 * [count][nc][nc][48], image 0 = instance `first`, channel 0 = u / u_max):
 * clamp(o0 * u_max, 0, u_max), u_max = l/lambda + h_c l (instances never given a
 * prediction keep the plain start).  After k_sweeps sweeps from the prediction,
 * if the last sweep changed no node by more than fallback_tol the refined
 * prediction is accepted as the coarse value (the patch builder's u_hat);
 * otherwise that instance restarts from the plain initial value u_max and runs
 * to tol_c (fallback).  u_hat only seeds and orders the fine solve: the fine
 * fixed point does not depend on it (the scheme is a contraction), only the
 * iteration count.  net_out = NULL restores the plain start. */
int hjb_batch_coarse_warm(hjb_batch* b, const float* net_out, int32_t first, int32_t count,
                          int32_t k_sweeps, double fallback_tol);

/* hjb_batch_destroy -- frees the batch; NULL is ignored. */
void hjb_batch_destroy(hjb_batch* b);

/* ======================================================== learned warm start
 * Not in the paper: a 6-layer 3x3 convolutional network (32 channels; input 5
 * channels: speed, target mask, obstacle mask, sigma, lambda, padded to 16;
 * output 33 channels: the coarse value over u_max and 32 control logits, padded
 * to 48; dilations 1, 2, 4, 8, 16, 32 so the receptive field spans a 129^2 grid;
 * ReLU between layers; BF16 weights and activations, FP32 accumulation)
 * whose value channel replaces the coarse solve's initial value (Section 4.3
 * "Initialization" uses a large constant).  Convolutions run as implicit GEMMs
 * on the tcgen05 tensor cores (forward and input gradient); the weight gradient
 * is an FP32 reduction.  Images are NHWC: pixel (b, y, x), channel c at
 * ((b H + y) W + x) C + c.  Parameters (FP32): per layer l = 0..5 the weights
 * w[cout][9][cin_store] (tap t = 3 (dy + 1) + (dx + 1) of the correlation
 * y[p] = sum_t w[., t, .] x[p + dil (dy, dx)], zero outside the image; cin_store = 16
 * for layer 0, 32 after) then the bias b[cout]; cout = 32, 33 for the last layer. */
typedef struct hjb_net hjb_net;

/* hjb_net_param_count -- number of FP32 parameters in the layout above. */
long long hjb_net_param_count(void);

/* hjb_net_create -- buffers for batches of up to max_batch H x W images on the
 * given stream (NULL: the default stream).  Parameters start at zero: call
 * hjb_net_set_params. */
int hjb_net_create(int32_t max_batch, int32_t height, int32_t width, void* cuda_stream, hjb_net** out);

/* hjb_net_set_params / hjb_net_get_params -- host FP32 parameter arrays
 * (hjb_net_param_count() values); set also clears the optimizer state. */
int hjb_net_set_params(hjb_net* net, const float* params);
int hjb_net_get_params(const hjb_net* net, float* params);

/* hjb_net_get_grads -- the parameter gradients of the last hjb_net_train_step
 * (same layout). */
int hjb_net_get_grads(const hjb_net* net, float* grads);

/* hjb_net_forward -- x: DEVICE bf16 [batch][H][W][16]; out_host (nullable): host
 * FP32 [batch][H][W][48] copy of the last layer. */
int hjb_net_forward(hjb_net* net, int32_t batch, const void* x, float* out_host);

/* hjb_net_train_step -- one Adam step (beta 0.9 / 0.999) on a batch: DEVICE
 * inputs x (as above), tval (target value over u_max, FP32 per pixel), tctrl
 * (target control index per pixel), freem (1 on pixels that count); the loss is
 * w_value * mean (o0 - tval)^2 + w_ctrl * mean cross-entropy over the n_free
 * counted pixels.  loss_out (nullable, 2 doubles): the two means. */
int hjb_net_train_step(hjb_net* net, int32_t batch, const void* x, const float* tval, const uint8_t* tctrl,
                       const uint8_t* freem, int64_t n_free, float lr, float w_value, float w_ctrl,
                       double* loss_out);

/* hjb_net_output_device -- the DEVICE FP32 [batch][H][W][48] output of the last
 * hjb_net_forward (owned by the network; valid until its next forward). */
int hjb_net_output_device(const hjb_net* net, const float** out);

/* hjb_net_warm_values -- after hjb_net_forward: image `index`'s value channel x
 * scale, clamped to [0, umax], as a coarse initial value u0 (DEVICE, H*W floats);
 * target nodes 0, obstacle nodes uob (mask: DEVICE H*W codes). */
int hjb_net_warm_values(hjb_net* net, int32_t index, const uint8_t* mask, float scale, float umax, float uob,
                        float* u0);

/* hjb_net_destroy -- NULL is ignored. */
void hjb_net_destroy(hjb_net* net);

/* Single 3x3 layers (dilation dil >= 1) on host buffers, for checking against a
 * reference: x / dy / mask are bf16 bit patterns, NHWC; w is [cout][9][cin] FP32;
 * cin, cout <= 48.
 *   hjb_conv3x3_forward: y = relu?(conv(x, w) + b)          (y: [B][H][W][cout] FP32)
 *   hjb_conv3x3_dgrad:   dx = conv^T(dy, w) * (mask > 0)    (mask nullable; dx: [B][H][W][cin])
 *   hjb_conv3x3_wgrad:   dw = sum_p dy (x) x-neighbourhood, db = sum_p dy (db nullable) */
int hjb_conv3x3_forward(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dil,
                        const uint16_t* x, const float* w, const float* b, int32_t relu, float* y);
int hjb_conv3x3_dgrad(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dil,
                      const uint16_t* dy, const float* w, const uint16_t* mask, float* dx);
int hjb_conv3x3_wgrad(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dil,
                      const uint16_t* x, const uint16_t* dy, float* dw, float* db);

#ifdef __cplusplus
}
#endif

#endif /* HJB_H */
