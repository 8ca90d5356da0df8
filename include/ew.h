/*
 * ew.h -- C ABI of the GB300 (sm_103a) EigenWave filter-operator library.
 *
 * EigenWave (Appelo, Banks, Henshaw, Le, Schwendeman, arXiv 2507.18282)
 * finds eigenpairs  L_h phi = -lambda^2 phi  of the discrete Dirichlet
 * Laplacian near a target frequency omega by applying the filter operator S
 * (one "wave-solve"): step the discrete wave equation w_tt = L_h w from
 * w(0) = v, w_t(0) = 0 over T_f = N_p 2 pi / omega and accumulate the
 * cos(omega t)-weighted trapezoidal time integral (eq. filterQuadrature).
 * S has the eigenvectors of L_h and eigenvalues beta in [-1/2, 1] peaked at
 * lambda = omega (Theorem "Eigenvalues of the EigenWave operator").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Vectors hold the ACTIVE (interior) points only, x fastest, then y, then
 *    z, densely packed (Algorithm matVec, Note 1 of the Arnoldi section).  A
 *    block of `nvec` vectors is nvec such vectors back to back.  Their element
 *    type is the grid's precision (float for EW_FP32, double for EW_FP64)
 *    unless an entry point says otherwise.
 *  - Every pointer named *_dev is device memory owned by the caller; every
 *    pointer named *_host is host memory owned by the caller.  The library
 *    owns grid handles and the scratch it allocates for them (freed by
 *    ew_grid_destroy).  A grid handle is not thread safe: calls that share
 *    one handle must not overlap.
 *  - All GPU work is issued on the caller's `stream`.  Calls return when the
 *    work is queued, except where the comment says the call synchronises.
 *  - Inner products are the unweighted Euclidean sums over active points
 *    (simple Rayleigh quotient, eq. simpleRayleighQuotient) on boxes with
 *    Dirichlet faces; with a Neumann face they carry the trapezoid weights
 *    (the discrete L_2 inner product of eq. discreteRayleighQuotient).
 *  - Errors: every call returns an ew_status; on failure ew_last_error()
 *    returns a message for the calling thread.  No exception crosses the ABI:
 *    a failed host allocation inside a call returns EW_ENOMEM.
 *    Device-side waits are bounded and report EW_ETIMEOUT.  A wave-solve
 *    returns before its kernels run, so a wait that gave up there is reported
 *    by the next call that synchronises (the autotuner, ew_rayleigh and the
 *    solvers built on it); the outputs of that wave-solve are then invalid.
 */
#ifndef EW_H_
#define EW_H_

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EW_OK = 0,
    EW_EINVAL = 1,       /* bad argument (null pointer, size, unsupported combination) */
    EW_ENOMEM = 2,       /* device or host allocation failed */
    EW_ECUDA = 3,        /* a CUDA runtime call failed */
    EW_ENOCONV = 4,      /* an iteration stopped before meeting its tolerance */
    EW_EBREAKDOWN = 5,   /* Krylov breakdown (invariant subspace smaller than asked) */
    EW_ETIMEOUT = 6,     /* a bounded device wait gave up */
    EW_EUNSUPPORTED = 7  /* valid request this build does not implement */
} ew_status;

typedef enum { EW_BC_DIRICHLET = 0, EW_BC_NEUMANN = 1 } ew_bc;
/* EW_FP32X2: 2D boxes only; vectors are FP64 (double) in and out, the wave-solve
 * runs in pairs of FP32 numbers (an unevaluated sum hi + lo, about 48
 * significant bits) on the full-rate FP32 units; ew_filter_apply and
 * ew_filter_apply_batched only (the FP64 filter applications of the
 * mixed-precision eigen-solver, refine_fp64 = 3, use it internally). */
typedef enum { EW_FP32 = 0, EW_FP64 = 1, EW_FP32X2 = 2 } ew_prec;
typedef enum { EW_EXPLICIT = 0, EW_IMPLICIT = 1 } ew_scheme;

typedef struct ew_grid ew_grid; /* opaque, library-owned */

/* Create a Cartesian box grid (Section "Discrete approximations", eq.
 * eigBVPdiscrete, restricted to one Cartesian component grid).
 *   dim         2 or 3
 *   n_interior  interior points per axis (n_interior[2] ignored in 2D), each
 *               >= 1: the vertices strictly between the two walls; at most
 *               2^40 active points in all (EW_EINVAL beyond)
 *   length      box side lengths; h_i = length_i / (n_i + 1)
 *   order       2: the 5/7-point Laplacian; 4: the fourth-order 9/13-point
 *               wide cross.  Both close at a wall by reflection (the paper's
 *               compatibility conditions are not spelled out): odd at a
 *               Dirichlet wall, u_{-j} = -u_{j} (u = 0 and u_xx = 0 there)
 *   bc          six faces (-x, +x, -y, +y, -z, +z); NULL = all Dirichlet.
 *               EW_BC_DIRICHLET: u = 0 on the wall, whose points are not
 *               active.  EW_BC_NEUMANN: a symmetry plane (the paper's Neumann
 *               condition, Section "Numerical results"): the wall points are
 *               active and the points beyond the wall are the even reflection
 *               u_{-j} = u_{j} (centred u_n = 0; order 4 also u_nnn = 0), so
 *               an axis has n_i + (its Neumann faces) active points.  With a
 *               Neumann face L_h is symmetric in the trapezoid-weighted sums
 *               (weight 1/2 per wall coordinate), not in the plain ones;
 *               ew_rayleigh and ew_arnoldi_eigs use those weights.  The
 *               implicit scheme and the multigrid entry points take
 *               Dirichlet boxes only (EW_EUNSUPPORTED otherwise)
 *   prec        field precision of every kernel run on this grid
 * The handle binds to the CUDA device current at creation (or, if none is
 * visible then, to the device current at its first GPU call); later calls
 * must run with that device current (EW_EINVAL otherwise).  No GPU memory is
 * allocated here, so grids and ew_filter_setup work on a host without a GPU. */
ew_status ew_grid_create(int dim, const int64_t n_interior[3], const double length[3], int order,
                         const ew_bc bc[6], ew_prec prec, ew_grid** out);
void ew_grid_destroy(ew_grid* grid);

/* Create a single curvilinear grid by the mapping method (Section "Discrete
 * approximations": a smooth invertible map x = G(r) from the unit square, the
 * equations transformed by the chain rule and discretised by conservative
 * centred differences).  Two dimensions, second order, u = 0 on every
 * boundary vertex.
 *   n_interior  interior vertices per direction (each >= 1); the active points
 *               and the vector layout are those of a 2D box with these counts
 *   xy_host     the (n1 + 2) x (n2 + 2) vertex coordinates, interleaved
 *               (x, y), r1 index fastest, boundary vertices included (host
 *               memory, read during the call and kept for the grid's life)
 *   prec        field precision, EW_FP32 or EW_FP64 (EW_EUNSUPPORTED for EW_FP32X2)
 * The operator: J L u = d_r(A11 u_r + A12 u_s) + d_s(A12 u_r + A22 u_s) with
 * J = x_r y_s - x_s y_r, A11 = (x_s^2 + y_s^2)/J, A22 = (x_r^2 + y_r^2)/J,
 * A12 = -(x_r x_s + y_r y_s)/J from centred differences of the vertex
 * coordinates (second-order one-sided ones on the boundary vertices); the
 * diagonal fluxes at half points (A averaged over two vertices), the cross
 * fluxes centred: a 9-point stencil, symmetric in the J-weighted sums, which
 * ew_rayleigh and ew_arnoldi_eigs use (its eigenvectors come back orthonormal
 * in those weights).  The explicit step limit comes from a Gershgorin bound
 * of rho(-L).  EW_EINVAL if J <= 0 at some vertex.  Like ew_grid_create it
 * needs no GPU; the couplings are copied to the device on first use.
 * ew_filter_apply (explicit scheme, one step per launch; temporal_block is
 * ignored), ew_filter_apply_batched, ew_apply_L, ew_rayleigh,
 * ew_power_iteration and ew_arnoldi_eigs accept such grids; the implicit
 * scheme, multigrid, ew_filter_apply_noalloc and ew_choose_num_periods return
 * EW_EUNSUPPORTED. */
ew_status ew_grid_create_mapped(const int64_t n_interior[2], const double* xy_host, ew_prec prec, ew_grid** out);

/* Multigrid options for the implicit systems M x = b, M = I - (dt^2/2) L_h
 * (eq. impMatrix).  The cycle: damped Jacobi (weight jacobi_weight, constant
 * interior diagonal) or the learned smoother on the finest `learned_levels`
 * levels; full weighting; linear interpolation; coarsening n -> (n-1)/2 while
 * every axis has odd n >= 5; the coarsest level smoothed to convergence. */
typedef struct {
    int pre, post;            /* smoothing steps before / after the coarse correction (V(pre,post)) */
    int max_cycles;           /* cycles per solve (>= 1) */
    double rtol;              /* stop early when ||b - M x||_2 <= rtol ||b||_2 (0: run max_cycles) */
    double jacobi_weight;     /* damped-Jacobi weight (0: 0.8) */
    int learned_levels;       /* 0: plain multigrid */
    const float* weights_dev; /* learned weights, learned_levels x 432 FP32 values (device), each
                                 rounded to BF16 by the kernels; layout [W1 8x27 | W2 8x27],
                                 taps (dz,dy,dx) with dz slowest */
    int red_black;            /* 1: multi-colour Gauss-Seidel smoothing instead of damped Jacobi on
                                 the non-learned levels: each sweep updates the points colour by
                                 colour by x += (b - M x) / M_ii (M_ii of an interior point).
                                 Second order: red-black, colour (i + j + k) mod 2; fourth order:
                                 three colours, (i + j + k) mod 3, so that no stencil offset
                                 joins two points of one colour */
    int guess;                /* initial guess of the implicit wave-solve's systems (the paper does
                                 not state one; 0 or 1, EW_EINVAL otherwise).  The systems are
                                 M W^1 = W^0 and, for n >= 1, M y = 2 W^n with y = W^{n+1} + W^{n-1}.
                                 0: y = rhs (W^0 for the first system, 2 W^n after); its residual
                                 is 2 a L_h W^n, which grows as 1/h^2 for rough W^n.
                                 1: from the third system on, the previous system's solution
                                 W^n + W^{n-2}; when that system was solved exactly its residual
                                 is 2 (W^n - W^{n-1}), independent of h.  ew_implicit_step_mg
                                 ignores it (its x is the guess) */
} ew_mg_params;

/* Filter parameters (Section "Discrete approximations").
 *   omega             target frequency (> 0)
 *   num_periods       N_p >= 1; T_f = N_p 2 pi / omega
 *   steps_per_period  N_its; N_t = N_p * N_its <= 2^31 - 2 (EW_EINVAL beyond),
 *                     dt = T_f / N_t.  0 = derive
 *                     from `cfl` (explicit only): the smallest N_its with
 *                     dt <= cfl * 2 / sqrt(rho(-L_h)), rho the largest
 *                     eigenvalue of -L_h (4 sum 1/h^2, or 16/3 sum 1/h^2)
 *   cfl               used when steps_per_period == 0 (<= 0: 0.8)
 *   scheme            EW_EXPLICIT (leapfrog, eqs. explicitScheme and
 *                     explicitStep1) or EW_IMPLICIT (eqs. implicitScheme,
 *                     implicitStep1, solved by multigrid with `mg`)
 *   adjust_omega      1: replace omega by omega~ of eq. adjustedOmega (needs
 *                     N_its > 4); the filter then peaks at lambda = omega for
 *                     the implicit scheme
 *   temporal_block    explicit steps fused per launch (0: library default)
 *   mg                implicit scheme only: each time step's system gets
 *                     mg->max_cycles V-cycles, or, when mg->rtol > 0, cycles
 *                     until ||b - M x||_2 <= rtol ||b||_2 (at most max_cycles;
 *                     the test synchronises the stream once per cycle) */
typedef struct {
    double omega;
    int num_periods;
    int steps_per_period;
    double cfl;
    ew_scheme scheme;
    int adjust_omega;
    int temporal_block;
    const ew_mg_params* mg;
} ew_filter_params;

/* The derived quantities of one wave-solve (eqs. filterQuadrature, alphad). */
typedef struct {
    double omega_used;   /* omega, or omega~ when adjust_omega */
    double final_time;   /* T_f */
    double dt;
    double alpha_d;      /* tan(omega dt / 2) / tan(omega dt) */
    int64_t num_steps;   /* N_t */
    int steps_per_period;
} ew_filter_info;

/* Compute the wave-solve parameters on the host.  weights_host (may be NULL)
 * receives the N_t + 1 filter weights c_n = (2/T_f) sigma_n (cos(omega t^n) -
 * alpha_d / 2), sigma the trapezoid weights (dt/2 at both ends, dt inside);
 * weights_cap is its capacity (EW_EINVAL if < N_t + 1). */
ew_status ew_filter_setup(const ew_grid* grid, const ew_filter_params* params,
                          ew_filter_info* info_host, double* weights_host, int64_t weights_cap);

/* Number of filter periods N_p for an eigen-solve of n_wanted pairs with a
 * Krylov dimension krylov_dim (Section "Estimating the EigenWave convergence
 * rate based on simultaneous iteration", eq. subSpaceIterationCR: CR =
 * beta_{N_a+1} / beta_{N_r}, N_r = n_wanted, N_a = krylov_dim, beta_j the
 * filter values beta_d of the grid's discrete eigenvalues in decreasing
 * order).  For N_p = 1, 2, 4, ..., max_periods, with the other fields of
 * params as given (omega, scheme, CFL or steps per period, adjust_omega), the
 * estimated cost N_p / (-ln CR) is evaluated from the exact discrete spectrum
 * of the box (tensor sine and cosine modes, by face kind) and the cheapest N_p is written to
 * *num_periods.  cr_host (may be NULL; capacity floor(log2(max_periods)) + 1)
 * receives CR for each candidate; a candidate is skipped (CR = 1), with all
 * longer ones, once its N_t would pass 2^31 - 2.  Each beta_d takes O(1)
 * operations (the trapezoid sum in closed form), over the eigenvalues of a
 * window around omega that is widened until no eigenvalue outside it can
 * enter the top N_a + 1.  Host work only (no GPU, no stream).
 * EW_EUNSUPPORTED if no candidate gives CR < 1, or for a curvilinear grid
 * (its spectrum has no closed form). */
ew_status ew_choose_num_periods(const ew_grid* grid, const ew_filter_params* params, int n_wanted,
                                int krylov_dim, int max_periods, int* num_periods, double* cr_host);

/* v_out = S v_in for each of `nvec` vectors: one wave-solve (Algorithm matVec
 * with the explicit or implicit scheme and the trapezoidal filter).  v_in and
 * v_out are device blocks of nvec vectors in the grid precision (FP64 for
 * EW_FP32X2 grids); they must not overlap.  Scratch (a few fields per vector)
 * is allocated on first use and kept with the grid. */
ew_status ew_filter_apply(const ew_grid* grid, const ew_filter_params* params, const void* v_in_dev,
                          void* v_out_dev, int nvec, cudaStream_t stream);

/* v_out = S v_in for nvec vectors held in HOST memory: the wave-solve of
 * ew_filter_apply (Algorithm matVec) with the copies to and from the device
 * overlapped with the filter applications.  The vectors are cut into chunks of
 * `chunk` vectors (0: at least four a chunk, at most four chunks); chunk k is
 * copied in on a copy stream while chunk k - 1 is filtered on `stream` and
 * chunk k - 2 is copied out on a second copy stream.  The results equal those
 * of ew_filter_apply on the same vectors bit for bit.
 *   v_in_host, v_out_host  nvec vectors each, the layout of ew_filter_apply, in
 *                          the grid precision (FP64 for EW_FP32X2 grids); they
 *                          must not overlap (EW_EINVAL).  Page-locked (pinned)
 *                          memory lets the copies overlap; pageable memory works
 *                          but its copies do not run asynchronously.
 * Stream-ordered like cudaMemcpyAsync: the call returns once the work is
 * queued; work queued on `stream` afterwards sees the outputs, and the host may
 * read v_out_host after synchronising `stream`.  Device buffers of 4 x chunk
 * vectors are allocated on first use and kept with the grid; calls on one grid
 * must not overlap.  EW_EINVAL for chunk < 0 or nvec outside [1, 65535]. */
ew_status ew_filter_apply_host(const ew_grid* grid, const ew_filter_params* params, const void* v_in_host,
                               void* v_out_host, int nvec, int chunk, cudaStream_t stream);

/* v_out[q] = S_q v_in[q] for nprob independent problems (each with its own
 * grid and filter parameters: uneven boxes, their own omega, time step and
 * N_t).  nvec (may be NULL = all 1) gives the vectors per problem; v_in[q]
 * and v_out[q] must not overlap (EW_EINVAL).  2D
 * explicit problems of one precision and one order run together: the work of
 * every problem is cut into rounds of a few time steps, each round is one
 * persistent launch over all unfinished problems' tiles, and the whole
 * sequence is one CUDA graph replayed on `stream`; the tile shape is
 * autotuned once per batch shape.  In FP32, a problem whose N x nvec reaches
 * three waves of 116 x 88 tiles over the GPU's SMs runs alone first, through
 * ew_filter_apply's tuned kernel (the results are the same bits either way).
 * Other mixes run one ew_filter_apply per problem.  The batched workspace is
 * process-wide: calls must not overlap. */
ew_status ew_filter_apply_batched(int nprob, const ew_grid* const* grids, const ew_filter_params* params,
                                  const void* const* v_in_dev, void* const* v_out_dev, const int* nvec,
                                  cudaStream_t stream);

/* ew_filter_apply for callers that cannot allocate device memory (no
 * counterpart in the paper).  Plugins whose host application owns every
 * device allocation, and real-time loops that must not enter the allocator
 * (its latency is unbounded), cannot let the library cudaMalloc scratch on
 * first use, as ew_filter_apply does.
 * This entry point calls no cudaMalloc, cudaFree or other allocating routine:
 * its scratch is one file-scope device array of 16.5 MiB (four time-level
 * fields of up to 16 MiB and up to 512 KiB of filter weights) that every GPU
 * loading the library holds until the process exits.
 *   - One vector (v_in, v_out device, grid precision, not overlapping), the
 *     explicit scheme only (EW_EUNSUPPORTED otherwise).
 *   - Limits: 4 M sizeof(element) <= 16 MiB, with M the points of one
 *     time level: N on 3D grids and (n_x rounded up to 4) n_y on 2D grids,
 *     rounded up to 64; i.e. about 1048576 active points in FP32 and 524288
 *     in FP64.  Also (N_t + 1) sizeof(element) <= 512 KiB.  Larger requests
 *     return EW_EINVAL with the limit in ew_last_error.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) for that device; make that first call before any
 *     stream capture.  The address is kept for the life of the process: do
 *     not call this entry point on a device after cudaDeviceReset of it.
 *   - Every call shares the array (each rewrites all of it that it reads, so
 *     nothing is carried over); calls whose GPU work overlaps race on it.
 *   - temporal_block 0 means a fixed depth of 4 (no autotuning); a negative
 *     one returns EW_EINVAL, as in ew_filter_apply. */
ew_status ew_filter_apply_noalloc(const ew_grid* grid, const ew_filter_params* params, const void* v_in_dev,
                                  void* v_out_dev, cudaStream_t stream);

/* Lu = L_h u for nvec vectors (grid precision, device). */
ew_status ew_apply_L(const ew_grid* grid, const void* u_dev, void* Lu_dev, int nvec,
                     cudaStream_t stream);

/* Stage 2 of the EigenWave approach (Arnoldi section): for each of nvec
 * vectors phi, lambda = sqrt(-sum phi L phi / sum phi^2) (eq.
 * simpleRayleighQuotient; on a box with a Neumann face both sums carry the
 * trapezoid weights, eq. discreteRayleighQuotient) and eig-res =
 * ||L phi + lambda^2 phi||_inf / (lambda^2 ||phi||_inf) (accuracy metrics,
 * Section "Numerical results").  Reductions run on the device in FP64.
 * Synchronises `stream`.  eig_res_host may be NULL. */
ew_status ew_rayleigh(const ew_grid* grid, const void* phi_dev, int nvec, double* lambda_host,
                      double* eig_res_host, cudaStream_t stream);

/* Algorithm EigenWave (power iteration on S): v <- S v, beta = (S v, v),
 * v <- S v / ||S v||, until ||v_new - sign(beta) v_old||_2 < tol or `iters`
 * iterations; then lambda from the Rayleigh quotient of L_h.  v_dev (one
 * vector, grid precision) is normalised first and holds the last iterate on
 * return.  beta_host (may be NULL) receives one beta per iteration done.
 * Synchronises `stream` once per iteration. */
ew_status ew_power_iteration(const ew_grid* grid, const ew_filter_params* params, void* v_dev,
                             int iters, double tol, double* beta_host, int* iters_done,
                             double* lambda_host, cudaStream_t stream);

/* Matrix-free eigen-solver on S (Arnoldi section; Algorithms arnoldi, IRAM,
 * KrylovSchur): block Krylov-Schur with thick restarts.  Wave-solves run in
 * the grid precision; the basis, classical Gram-Schmidt applied twice, the
 * Rayleigh-Ritz projection and all reductions are FP64.  The wanted pairs
 * are the n_wanted largest algebraic eigenvalues beta of S, i.e. the
 * eigenvalues lambda of L_h nearest the filter peak at omega.  lambda is
 * then taken from the Rayleigh quotient of L_h (eq. simpleRayleighQuotient).
 * With refine_fp64 on an FP32 grid the result is refined in FP64 (mixed
 * precision, see refine_fp64).  Convergence is fast when the filter peak holds about
 * krylov_dim eigenvalues: choose num_periods N_p accordingly (the peak is
 * about omega / N_p wide). */
typedef struct {
    int n_wanted;          /* N_r, 1..EW_MAX_EIGS */
    int krylov_dim;        /* N_a: basis size at which the solver restarts (rounded up to a multiple of
                              block); >= n_wanted + block, krylov_dim + 2 block <= 160; 0: 2 N_r + block */
    int block;             /* vectors per expansion, 1..16 (at least the largest multiplicity near omega) */
    double tol;            /* accept a Ritz pair when ||S x - theta x||_2 <= tol (||x|| = 1);
                              0: 1e-4 on FP32 grids (about the FP32 wave-solve noise), 1e-10 on FP64 */
    int max_wave_solves;   /* budget of first-stage filter applications (one per vector); 0: 2000 */
    uint64_t seed;         /* start block from SplitMix64 uniform [-1,1) when start_dev is NULL:
                              element q of the N x block column-major block is draw q of stream seed */
    int refine_fp64;       /* FP32 grids, FP64 refinement of the result (0: none).
                              1: mixed-precision iterative refinement of the invariant subspace of the
                                 n_wanted pairs plus g guard vectors (the next Ritz vectors by beta).
                                 Each outer step (at most 6): a Rayleigh-Ritz with L_h inside span[X]
                                 (separates near-degenerate pairs; pairs ranked by beta_d(lambda));
                                 stop when every wanted eig-res <= refine_tol; else one FP64 wave-solve
                                 per vector gives the exact relation S X = X Theta + E, span[X, E] is
                                 extended by p FP32 block expansions and Rayleigh-Ritz with S picks the
                                 new X.  p = 6 and g = n_wanted where they fit ((p + 2)(n_wanted + g)
                                 <= 128 basis columns), fewer for large n_wanted (n_wanted <= 23); after
                                 the first outer step p is sized by the contraction the last step
                                 achieved (taken as geometric in p) for a 10x margin below refine_tol.
                              2: a second Krylov-Schur run with FP64 full-filter wave-solves started
                                 from the FP32 vectors (block n_wanted, basis 3 n_wanted)
                              3: as 1, with the images S X of each outer step computed in double-FP32
                                 pairs (EW_FP32X2, about 48 significant bits, on the FP32 units) on 2D
                                 boxes; once an outer step cuts the worst eig-res by less than 10x the
                                 remaining images are FP64 */
    double refine_tol;     /* refine_fp64 1, 3: eig-res target of every wanted pair, 0: 5e-9;
                              refine_fp64 2: FP64 Ritz residual target, 0: 1e-10 */
    int lock;              /* 1: lock converged pairs at each thick restart (a wanted Ritz pair whose
                              residual is below tol keeps its vector and value, and its coupling to the
                              residual block is set to zero, so later expansions leave it as it is) */
} ew_eigs_params;

#define EW_MAX_EIGS 64
typedef struct {
    int n_converged;                       /* first-stage pairs that met tol */
    int wave_solves;                       /* first-stage filter applications */
    int wave_solves_fp64;                  /* FP64 refinement filter applications */
    int restarts;
    double seconds;                        /* wall time of the call */
    double beta[EW_MAX_EIGS];              /* Ritz values of S, descending */
    double eig_res[EW_MAX_EIGS];           /* final eig-res (accuracy metrics, Section "Numerical results") */
    double lambda_stage1[EW_MAX_EIGS];     /* lambda from the first-stage vectors */
    double eig_res_stage1[EW_MAX_EIGS];
    double lambda_rel_change[EW_MAX_EIGS]; /* |lambda - nearest first-stage lambda| / lambda */
} ew_eigs_report;

/* lambda_host (n_wanted) receives lambda per pair in the order of descending
 * beta; vecs_dev (may be NULL) receives the FP64 eigenvectors, N x n_wanted
 * column-major, unit 2-norm (with a Neumann face: unit trapezoid-weighted
 * norm, the eigenvectors orthonormal in those weights).  start_dev (may be NULL) is an FP64 N x block
 * start block.  Allocates its own workspace (basis N x (krylov_dim + 2 block)
 * FP64) for the duration of the call and synchronises `stream`.  Returns
 * EW_ENOCONV (results still filled) when the budget ran out first,
 * EW_EBREAKDOWN when the Krylov space became invariant. */
ew_status ew_arnoldi_eigs(const ew_grid* grid, const ew_filter_params* params, const ew_eigs_params* eigs,
                          const double* start_dev, double* lambda_host, double* vecs_dev,
                          ew_eigs_report* report_host, cudaStream_t stream);

/* Eigen-solves of nprob independent problems with their filter applications
 * batched (the paper's method per problem; the batching has no counterpart in
 * the paper).  Problem q runs the solver of ew_arnoldi_eigs with grids[q],
 * params[q] and eigs[q] (random start block from eigs[q].seed) on a host
 * thread and a stream of its own.  Whenever every unfinished solver has asked
 * for a filter application S X, all of them run together as one
 * ew_filter_apply_batched call (its CUDA graph kept per batch and replayed;
 * the tile variant tuned on the first round and then kept); the rest of each
 * solver (orthogonalisation, small eigenproblems, Rayleigh quotients,
 * refinement) runs per problem between those rounds.  At most 1024 problems
 * (one host thread each; EW_EINVAL beyond).
 *   lambda_host[q]  receives problem q's n_wanted eigenvalues (host)
 *   vecs_dev        may be NULL, else vecs_dev[q] (may be NULL) receives
 *                   problem q's eigenvectors as in ew_arnoldi_eigs (device)
 *   reports, statuses  may be NULL, else nprob entries (host)
 *   rounds_host     may be NULL, else the number of batched calls made
 * The problems' work starts after the work already queued on `stream`, and
 * the call returns when all of it is done.  Returns EW_OK when every problem
 * did, else the first other status in problem order, with that problem's
 * message in ew_last_error.  Uses the process-wide batched workspace: calls
 * must not overlap with each other or with ew_filter_apply_batched. */
ew_status ew_arnoldi_eigs_batched(int nprob, const ew_grid* const* grids, const ew_filter_params* params,
                                  const ew_eigs_params* eigs, double* const* lambda_host, double* const* vecs_dev,
                                  ew_eigs_report* reports, ew_status* statuses, int* rounds_host,
                                  cudaStream_t stream);

/* Multigrid solve of one implicit time-step system (eqs. impMatrix,
 * implicitStep1):  (I - half_dt2 L_h) x = rhs, half_dt2 finite and >= 0.
 * x_dev holds the initial guess on entry and the result on return (grid
 * precision, device; must not overlap rhs_dev, EW_EINVAL).  Runs up to
 * mg->max_cycles V-cycles (fewer once ||rhs - M x||_2 <= rtol ||rhs||_2 when
 * rtol > 0).  conv_factor_host (may be NULL) receives the mean residual
 * reduction per cycle, cycles_done_host (may be NULL) the cycles run.  Axis
 * lengths must halve down (n -> (n-1)/2) to at most 2048 coarse points, e.g.
 * n = 2^k - 1 (EW_EUNSUPPORTED otherwise).  Synchronises `stream`; EW_ENOCONV
 * if rtol > 0 was not met. */
ew_status ew_implicit_step_mg(const ew_grid* grid, double half_dt2, const void* rhs_dev, void* x_dev,
                              const ew_mg_params* mg, double* conv_factor_host, int* cycles_done_host,
                              cudaStream_t stream);

/* Learned multigrid smoother (no counterpart in the paper; it replaces the
 * damped-Jacobi step of the V-cycle on the finest levels, see ew_mg_params).
 * The correction of a residual r on a 3D grid, zero outside the active box:
 *   h_c(x) = sum_{o in {-1,0,1}^3} W1[c][o] r(x + o),  c = 0..7
 *   N(r)(x) = sum_c sum_o W2[c][o] h_c(x + o)
 * no bias, no activation (the smoothing step stays linear).  weights_dev: 432
 * FP32 values [W1 8x27 | W2 8x27], taps (dz, dy, dx) with dz slowest; weights,
 * r and h are rounded to BF16 and products accumulated in FP32.
 * ew_smoother_forward: y = N(r).  ew_smoother_backward: grad_dev (432 FP32)
 * = d(loss)/d(weights) for a loss with d(loss)/dy = gy (r, gy grid precision,
 * device).  3D grids only. */
ew_status ew_smoother_forward(const ew_grid* grid, const float* weights_dev, const void* r_dev, void* y_dev,
                              cudaStream_t stream);
ew_status ew_smoother_backward(const ew_grid* grid, const float* weights_dev, const void* r_dev,
                               const void* gy_dev, float* grad_dev, cudaStream_t stream);

/* Train the learned smoother for the system (I - half_dt2 L_h) x = b on this
 * grid (FP32, 3D).  Residual samples come from plain multigrid solves of the
 * same system (random right-hand sides, the residual at the start of the
 * first three V-cycles); each of `steps` Adam steps minimises
 *   1/2 ||M (e - N(r))||^2 = 1/2 ||r - M N(r)||^2    (M e = r)
 * over one sample, with the library's forward and backward kernels.  Plain
 * multigrid decides whether to accept the result: the convergence factors of V(pre, post) cycles
 * with the Jacobi smoother and with the learned one on the finest level are
 * measured on the same system, and the weights are kept only if the learned
 * factor is lower (else weights_dev is restored: plain-multigrid fallback).
 * weights_dev (432 FP32, device) holds the initial weights on entry. */
typedef struct {
    int steps;             /* Adam steps */
    int samples;           /* residual samples kept on the device */
    double lr;             /* Adam learning rate */
    int pre, post;         /* V-cycle shape of the sample generation and of the acceptance test */
    double jacobi_weight;  /* plain smoother weight (0: 0.8) */
    uint64_t seed;         /* right-hand sides: SplitMix64 streams seed, seed + 1, ... */
    int accept_cycles;     /* V-cycles per convergence-factor measurement (0: 6) */
} ew_train_params;
typedef struct {
    double loss_first, loss_last;    /* training loss of the first and the last step */
    double conv_plain, conv_learned; /* residual reduction per V-cycle */
    int accepted;                    /* 1: learned weights kept */
} ew_train_report;
ew_status ew_smoother_train(const ew_grid* grid, double half_dt2, const ew_train_params* params,
                            float* weights_dev, ew_train_report* report_host, cudaStream_t stream);

/* The variant the autotuner chose for the 2D blocked time step on this grid
 * and a block of nvec vectors (no counterpart in the paper; for reports and
 * benchmarks): the kernel's name with its template shape, NUL-terminated in
 * name_host (cap bytes), the time steps per launch (*depth) and the owned
 * tile of a CTA (*tile_x x *tile_y points); depth and tiles may be NULL.
 * EW_EINVAL when no wave-solve of this shape has been tuned in this process,
 * or for a grid other than a 2D box.  Host only. */
ew_status ew_tuned_variant(const ew_grid* grid, int nvec, char* name_host, int cap, int* depth, int* tile_x,
                           int* tile_y);

/* Launch accounting, for benchmarks.  While enabled (process-wide), the
 * library counts every kernel it launches and brackets each launch of its
 * fused time-step kernels (the explicit leapfrog + filter kernels) with a
 * pair of CUDA events recorded on the launching stream.  ew_profile_read
 * waits for the recorded events, returns the totals since the last read and
 * resets them.  Enabling or disabling also resets. */
typedef struct {
    int64_t launches;          /* all kernels launched by the library */
    int64_t fused_launches;    /* launches of the fused time-step kernels */
    double fused_ms;           /* summed event time of those launches */
    int64_t fused_cell_steps;  /* active points x time steps they advanced */
    int64_t fused_points;      /* active points they covered, summed over launches */
    int64_t mg_cycles;         /* V-cycles run by the implicit time steps' multigrid solves */
    int64_t mg_solves;         /* those solves (one per implicit time step) */
} ew_profile;
ew_status ew_profile_enable(int on);
ew_status ew_profile_read(ew_profile* out_host);

/* Message of the last failed call on this thread ("" if none). */
const char* ew_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EW_H_ */
