/*
 * bura.h — C ABI of the GB300 BURA fractional solver.
 *
 * Solves  A^alpha u = f  (0 < alpha < 1) for the scaled SPD finite-difference
 * matrix A = Atilde / Lambda of -div(a grad u) on a uniform 2D/3D interior grid
 * of the unit square/cube with homogeneous Dirichlet data (eq. (algebraic),
 * Sec. 1.2; Lambda = max absolute row sum of Atilde, so spec(A) lies in (0,1]).
 *
 * Method (beta = 1): the best uniform rational approximation r of t^(1-alpha)
 * on [0,1] (Definition def-BURA, Sec. 2.1) is written as
 *     t^{-1} r(t) = sum_{j=0}^k c_j / (t - d_j),  d_0 = 0 > d_1 > ... > d_k,  c_j > 0
 * (eq. (simplified), Sec. 2.2) and
 *     u = sum_{j=0}^k c_j (A - d_j I)^{-1} f            (eq. (Rgeneral), Sec. 2.2).
 * All k+1 shifted SPD systems are solved together by one multi-shift conjugate
 * gradient method preconditioned by geometric multigrid, in CUDA kernels on the
 * current device; the weighted sum is formed in FP64 on the device.
 *
 * Conventions for every entry point
 *  - Return value: BURA_OK (0) or a negative bura_status; nothing aborts and no
 *    exception crosses the ABI.  bura_strerror() describes a code.
 *  - Grid vectors (f, u) have N = nx*ny*nz entries in lexicographic order, x fastest.
 *  - A "device" pointer is CUDA global memory of the current device; a "host"
 *    pointer is ordinary (ideally page-locked) host memory.
 *  - A plan is used by one host thread and one stream at a time.
 *  - There is no CPU fallback: without a usable CUDA device every solve fails
 *    with BURA_ECUDA.
 */
#ifndef BURA_H
#define BURA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BURA_MAX_K 12 /* largest supported BURA degree k (k+1 shifted systems) */

typedef enum {
    BURA_OK = 0,
    BURA_EINVAL = -1,   /* bad argument: alpha not in (0,1), k out of range, bad grid, null pointer */
    BURA_ENOMEM = -2,   /* device or host allocation failed */
    BURA_EREMEZ = -3,   /* the rational approximation did not converge for (alpha, k) */
    BURA_ENOTSPD = -4,  /* CG breakdown: p^T (A - d I) p <= 0 or non-finite values */
    BURA_ENOCONV = -5,  /* tolerance not met within the iteration caps; u holds the last iterate */
    BURA_ETIMEOUT = -6, /* a bounded device-side wait ran out */
    BURA_ECUDA = -7,    /* a CUDA runtime call failed (no device, launch error, ...) */
    BURA_ERANGE = -8    /* a size is above a documented maximum */
} bura_status;

typedef enum { BURA_COEF_CONSTANT = 0, BURA_COEF_FACES = 1 } bura_coef_kind;

typedef enum {
    BURA_PREC_FP64 = 0,  /* every inner iteration in FP64 */
    BURA_PREC_MIXED = 1  /* FP32 multigrid-PCG inner solves inside FP64 iterative refinement */
} bura_precision;

/* Interior grid.  dim = 2 uses n[0] = nx, n[1] = ny (n[2] ignored); dim = 3 uses all three.
 * Mesh sizes are h_x = 1/(nx+1) etc.  Multigrid coarsens while every n is odd and >= 3
 * (n -> (n-1)/2), so sizes 2^m - 1 give the deepest hierarchy. */
typedef struct {
    int dim;
    int n[3];
    int coef_kind; /* bura_coef_kind */
} bura_grid;

/* How the small levels of the multigrid V-cycle are run. */
typedef enum {
    BURA_COARSE_AUTO = 0,    /* FDIAG for 2-D constant coefficients, else CTA (faster than CLUSTER on GB300) */
    BURA_COARSE_CLUSTER = 1, /* levels with <= 16384 points in one thread-block cluster (vectors in L2);
                                bura_setup returns BURA_EINVAL on a device without cluster launch */
    BURA_COARSE_CTA = 2,     /* the levels that fit 200 KB of shared memory in a single CTA */
    BURA_COARSE_NONE = 3,    /* every level as grid-wide kernels; the coarsest level is smoothed only */
    BURA_COARSE_FDIAG = 4    /* 2-D constant coefficients only (else BURA_EINVAL; also without cluster launch):
                                the first level with at most 63 (FP32) or 31 (FP64) points per axis is
                                solved exactly by fast diagonalization, (A - d_j I)^{-1} = S_y (S_y . S_x ./
                                (lambda_x + lambda_y - d_j)) S_x in the sine eigenbasis of the 5-point
                                operator (per axis the eigenpairs of the three-point matrix of Sec. 4.1; the
                                eigen-expansion of eq. (exacalg), Sec. 1.2), and the V-cycle stops there */
} bura_coarse_kernel;

/* How the level sweeps of the large levels are run. */
typedef enum {
    BURA_SWEEP_AUTO = 0, /* TMA-staged tiles (FP32, 2-D, constant coefficients, >= 1 tile per SM), else GRID */
    BURA_SWEEP_GRID = 1  /* grid-stride kernels with direct global loads everywhere */
} bura_sweep_kind;

/* Arithmetic of the iterative refinement of the mixed path (residual, correction, weighted sum). */
typedef enum {
    BURA_REFINE_FP64 = 0, /* IEEE FP64 (default) */
    BURA_REFINE_DF = 1    /* double-float: FP32 pairs hi + lo (about 48 significant bits) with error-free
                             FP32 transformations on the FP32 pipes; tolerances down to about 1e-12 */
} bura_refine;

/* Solver options; bura_default_options() fills the defaults. */
typedef struct {
    int precision;        /* bura_precision; default BURA_PREC_MIXED */
    int smoother_degree;  /* Chebyshev degree of each pre/post smoothing; default 2 */
    double smoother_ratio;/* Chebyshev interval [lmax/ratio, lmax] of D^{-1}(A - d I), ratio > 1; 0 (default) =
                             auto: 4 in 2-D, 8 in 3-D (the band of the spectrum that full coarsening leaves to
                             the smoother is wider for the 7-point operator) */
    int max_iters;        /* cap on PCG iterations per (inner) solve; default 200 */
    int max_outer;        /* cap on FP64 refinement steps (mixed precision); default 12 */
    double inner_rtol;    /* largest relative residual reduction asked of one FP32 inner solve; the FP64
                             refinement plans ceil(log need / log inner_rtol) steps; default 1e-5 */
    int coarse_degree;    /* Chebyshev degree on the coarsest level when it has > 1 point; 0 = auto */
    int block_points;     /* grid points per CTA of the level sweeps (CTA = points x 16-byte chunks); 0 = auto */
    int blocks_per_sm;    /* CTAs per SM of the grid-stride sweeps; 0 = auto */
    int coarse_kernel;    /* bura_coarse_kernel; default BURA_COARSE_AUTO */
    int cluster_size;     /* largest cluster tried for BURA_COARSE_CLUSTER: 2, 4, 8 or 16; 0 = 16.  The
                             size used is the largest power of two <= this that the device co-schedules */
    int sweeps;           /* bura_sweep_kind; default BURA_SWEEP_AUTO */
    int refine;           /* bura_refine (mixed precision only); default BURA_REFINE_FP64 */
    int tma_stages;       /* depth of the shared-memory ring of the TMA-staged sweeps, 1..4 (a kernel whose
                             ring does not fit shared memory uses fewer); 0 = auto (2) */
    int post_smooth_split; /* on the TMA-staged levels (2-D, constant coefficients, FP32) with degree-2
                             smoothing, how the prolongation and both post-smoothing steps run:
                             0 (default): one sweep over TMA tiles (the first step recomputed on a
                             one-point halo of each tile); 1: two sweeps (prolongation + first step, then
                             the second step); 2: one sweep as y-marching strips (no recomputed rows,
                             slower on GB300).  Every point gets the same operations each way; r.z is
                             summed in another grouping, so the iterates may differ in the last bits of
                             the FP32 beta. */
    int unscaled;         /* 0 (default): u solves the scaled problem A^alpha u = f.  1: f is the right-hand
                             side ftilde of the unscaled problem Atilde^alpha utilde = ftilde and u = utilde =
                             Lambda^-alpha (A^-alpha ftilde), since Atilde = Lambda A (eq. (algebraic), Sec. 1.4;
                             Corollary c:BURAerror is stated for the scaled pair).  The stopping rule and
                             bura_stats refer to the scaled solution; the relative error is the same.  Not
                             accepted by bura_setup_shifts (no alpha). */
    long long tma_wait_cycles; /* SM clocks a TMA-staged sweep waits for one stage of its shared-memory ring
                             before it gives up, records a fault and the solve returns BURA_ETIMEOUT; 0 = the
                             default (about 2 s).  Copies still in flight are always drained under the
                             default budget before a kernel exits.  See bura_set_tma_wait_cycles. */
    int smoother_bf16;    /* variable coefficients, mixed precision: 1 stores the face weights that the
                             multigrid V-cycle (smoothing, residuals, coarse levels) reads as bfloat16 (the CG
                             operator and the FP64 refinement keep FP32/FP64 weights, so the solution's
                             accuracy is unchanged; only the preconditioner sees the rounded field); each
                             level's diagonal is summed from its stored weights; default 0 */
} bura_options;

/* Statistics of the last bura_solve*/
typedef struct {
    double Lambda;                   /* Gershgorin scale of Atilde */
    double E;                        /* BURA error E_alpha(k,k;1) of the rational approximation */
    int k;                           /* degree; k+1 systems */
    int levels;                      /* multigrid levels */
    int iters;                       /* PCG iterations in total (sum over refinement steps) */
    int outer;                       /* FP64 refinement steps (mixed precision), 1 for FP64 */
    int shift_iters[BURA_MAX_K + 1]; /* iterations each system stayed active */
    double rel_res[BURA_MAX_K + 1];  /* final ||f - (A - d_j I) v_j|| / ||f|| per system */
    double err_bound;                /* sum_j c_j ||r_j|| / ((lambda_lo - d_j) ||f||): bound on ||u - u_r|| / ||f|| */
    double lambda_lo;                /* lower bound on lambda_min(A) used by the stopping test */
    long long launches;              /* CUDA kernels launched by the last solve */
    size_t device_bytes;             /* device memory the plan holds (all its allocations) */
} bura_stats;

/* Per-kernel timing of the fine-level kernels (see bura_set_profiling). */
typedef struct {
    const char* name;   /* static kernel name, e.g. "cheb_step_f32" */
    long long launches; /* timed launches since profiling was enabled */
    double ms;          /* summed CUDA-event durations of those launches */
    double bytes;       /* summed algorithmic bytes (data a launch must read and write at least) */
} bura_kernel_prof;

typedef struct bura_plan bura_plan;

/* Fill *opt with the defaults listed in bura_options. */
void bura_default_options(bura_options* opt);

/*
 * Best uniform rational approximation of t^(1-alpha) on [0,1] in R(k,k), host only
 * (Sec. 3; the library's own Remez solver, see the implementation notes).
 *   c[0..k], d[0..k]: caller-owned host arrays of k+1 doubles; d[0] = 0 > d[1] > ... > d[k].
 *   E: the equioscillation level (may be NULL).
 * Errors: BURA_EINVAL (alpha not in (0,1), k not in [1, BURA_MAX_K], null c/d),
 *         BURA_EREMEZ (no convergence).
 */
int bura_rational(double alpha, int k, double* c, double* d, double* E);

/*
 * Build a plan for one grid, one operator, one (alpha, k): computes Lambda, the BURA
 * coefficients, the multigrid hierarchy and all device workspaces (cudaMalloc on the
 * current device; the plan owns them until bura_destroy).
 *   faces: NULL for BURA_COEF_CONSTANT; otherwise `dim` HOST arrays of doubles
 *          faces[0] = a on x-faces, shape (nz, ny, nx+1) [2D: (ny, nx+1)],
 *          faces[1] = a on y-faces, shape (nz, ny+1, nx) [2D: (ny+1, nx)],
 *          faces[2] = a on z-faces, shape (nz+1, ny, nx) (3D only),
 *          C order, x fastest; faces[0][.., i] is a between interior nodes i-1 and i
 *          (i = 0 and i = nx are the faces to the boundary).  All values must be > 0.
 *          The arrays are copied; the caller keeps ownership.
 *   opt: NULL for the defaults.
 * Errors: BURA_EINVAL, BURA_ERANGE (N * (k+1) above 2^31), BURA_EREMEZ, BURA_ENOMEM, BURA_ECUDA.
 */
int bura_setup(const bura_grid* grid, const double* const* faces, double alpha, int k,
               const bura_options* opt, bura_plan** out);

/*
 * A plan for a partial-fraction sum with caller-given weights and shifts instead of the BURA:
 *     u = sum_{j=0}^{nsys-1} c[j] (A - d[j] I)^{-1} f,    c[j] > 0, d[j] <= 0,
 * on the same multi-shift multigrid-PCG solve.  This is the form of the sinc quadrature of [BP15] that the
 * paper compares the BURA with (eq. (BonitoPasciak), Sec. 5.3): with A = Atilde / Lambda its nodes are
 * d_l = -e^{-2 l k'} / Lambda with weights c_l = (2 k' sin(pi alpha) / pi) e^{2 (alpha - 1) l k'} Lambda^(alpha - 1)
 * (every term a positive diagonal shift of Atilde).  A quadrature with more than BURA_MAX_K + 1 nodes is
 * split over several plans whose results bura_solve_sum adds.
 *   c, d: HOST arrays of nsys doubles (copied).  The plan stores the systems sorted by descending d;
 *         bura_get_rational returns them in that order with E = 0.
 *   grid, faces, opt: as for bura_setup (opt->unscaled must be 0).
 * Errors: BURA_EINVAL (bad grid, null c/d, nsys < 1, c[j] <= 0, d[j] > 0, non-finite values, unscaled),
 *         BURA_ERANGE (nsys > BURA_MAX_K + 1, or N too large), BURA_ENOMEM, BURA_ECUDA.
 *         bura_retarget rejects such a plan with BURA_EINVAL.
 */
int bura_setup_shifts(const bura_grid* grid, const double* const* faces, int nsys, const double* c, const double* d,
                      const bura_options* opt, bura_plan** out);

/*
 * An assembled SPD matrix Atilde in compressed sparse rows (host arrays, 0-based), for instance the
 * stiffness matrix of conforming P1 finite elements that the paper's 3-D tests use (Sec. 5.4): row i holds
 * its entries val[row_ptr[i] .. row_ptr[i+1]-1] in columns col[...], the diagonal included, in any order.
 */
typedef struct {
    int n;                /* rows = columns */
    long long nnz;        /* entries, row_ptr[n] */
    const int* row_ptr;   /* n + 1 offsets */
    const int* col;       /* nnz column indices */
    const double* val;    /* nnz values */
    double lambda_min;    /* a lower bound (> 0) on the smallest eigenvalue of Atilde, or 0 if none is known */
} bura_csr;

/*
 * A plan for the BURA solve of A^alpha u = f with the sparse matrix A = Atilde / Lambda, Lambda the largest
 * absolute row sum of Atilde (eq. (algebraic), Sec. 1.4), u = sum_j c_j (A - d_j I)^{-1} f (eq. (Rgeneral)).
 * The k+1 shifted systems run as one multi-shift CG on the GPU: the sparse product reads each entry's value
 * and column once for all systems (vectors interleaved by system, as on grids), and the preconditioner is a
 * Chebyshev polynomial in Dinv (A - d_j I) per system (degree opt->coarse_degree, 0 = 8, on the interval
 * [hi_j / ratio, hi_j], hi_j the Gershgorin bound of the scaled rows, ratio = opt->smoother_ratio, 0 = 30):
 * geometric multigrid needs a grid.  lambda_min enters the stopping rule only.
 * Stopping rule: with lambda_min > 0 that of bura_solve; with lambda_min = 0 every system stops at
 * ||f - (A - d_j I) v_j|| <= tol ||f|| (the relative residual criterion of the paper's PCG runs) and
 * bura_stats.err_bound is -1.  The arrays are copied (the caller keeps ownership); bura_solve* and
 * bura_apply_shifted then take vectors of n entries.  Not with opt->refine = BURA_REFINE_DF.
 * Errors: BURA_EINVAL (null pointers, n < 1, offsets not from 0 to nnz or decreasing, a column out of range,
 *         a non-finite value, a row without a positive diagonal, an unsymmetric matrix, lambda_min < 0,
 *         alpha, k or options out of range), BURA_ERANGE (n * 16 or nnz >= 2^31), BURA_EREMEZ, BURA_ENOMEM,
 *         BURA_ECUDA.
 */
int bura_setup_csr(const bura_csr* A, double alpha, int k, const bura_options* opt, bura_plan** out);

/*
 * The scale Lambda of eq. (algebraic) (Sec. 1.4) for a grid and its coefficients, host only: the Gershgorin
 * bound max_P sum_Q |Atilde_PQ| of the unscaled matrix, which every plan of the grid uses (A = Atilde / Lambda).
 * grid and faces as for bura_setup.  Errors: BURA_EINVAL (bad grid or faces, null Lambda), BURA_ERANGE.
 */
int bura_scale(const bura_grid* grid, const double* const* faces, double* Lambda);

/*
 * Nodes of the sinc quadrature of [BP15] in the paper's comparison (eq. (BonitoPasciak), Sec. 5.3) for the
 * scaled operator A = Atilde / Lambda, host only:
 *     Atilde^{-alpha} ftilde ~ (2 k' sin(pi alpha) / pi) sum_{l=-m}^{M} e^{2 (alpha-1) l k'} (e^{-2 l k'} I + Atilde)^{-1} ftilde,
 *     m = ceil(pi^2 / (4 alpha k'^2)), M = ceil(pi^2 / (4 (1 - alpha) k'^2)),
 * returned as the partial-fraction form of A^{-alpha} f:  c[l+m] = (2 k' sin(pi alpha)/pi) e^{2(alpha-1) l k'}
 * Lambda^(alpha-1) > 0 and d[l+m] = -e^{-2 l k'} / Lambda < 0, l = -m..M, for bura_setup_shifts.
 *   cap: capacity of the caller's HOST arrays c, d; *n receives m + M + 1 (also when it exceeds cap).
 * Errors: BURA_EINVAL (alpha not in (0,1), kprime <= 0, Lambda <= 0, null n, null c/d with cap > 0),
 *         BURA_ERANGE (m + M + 1 > cap; nothing written to c, d).
 */
int bura_quadrature_bp15(double alpha, double kprime, double Lambda, int cap, double* c, double* d, int* n);

/*
 * u = sum_j c_j (A - d_j I)^{-1} f, stream-ordered on `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  f and u are DEVICE arrays of N doubles owned by the caller (they
 * may alias each other).  The call returns once the solve has finished (bura_solve_async + bura_solve_wait);
 * u is complete when `stream` reaches this point.
 *   tol: target bound on ||u - u_r|| / ||f||, u_r the exact value of eq. (Rgeneral).  Each system
 *        j stops when c_j ||f - (A - d_j I) v_j|| / (lambda_lo - d_j) <= tol ||f|| / (k+1).
 * Errors: BURA_EINVAL, BURA_ENOTSPD, BURA_ENOCONV (u still written), BURA_ECUDA.
 */
int bura_solve(bura_plan* plan, const double* f, double* u, double tol, void* stream);

/*
 * bura_solve without waiting: the whole solve (the FP64 path, or the mixed path with FP64 refinement) runs
 * as one captured CUDA graph whose controller kernels take every decision on the device (thresholds,
 * refinement plan, convergence), so the call only enqueues work on `stream` and returns BURA_OK (or an
 * argument / CUDA error).  u is complete when `stream` reaches this point; bura_solve_wait returns the
 * solve's status.  The plan's buffers serve this solve until it completes: a later call on the same plan
 * must be ordered after it (the same stream, or an event).  With double-float refinement or profiling on,
 * the solve is host-driven and finishes within the call.  f and u as for bura_solve.
 */
int bura_solve_async(bura_plan* plan, const double* f, double* u, double tol, void* stream);

/*
 * Waits for the plan's last solve and returns its status (BURA_OK, BURA_ENOCONV, BURA_ENOTSPD,
 * BURA_ETIMEOUT, or BURA_ECUDA if waiting failed); bura_get_stats then describes that solve.
 */
int bura_solve_wait(bura_plan* plan);

/*
 * Same as bura_solve with HOST arrays f and u (N doubles each): copies f to the device,
 * solves and copies u back on `stream`; returns after u is in host memory.
 */
int bura_solve_host(bura_plan* plan, const double* f, double* u, double tol, void* stream);

/*
 * The k+1 solutions v_j = (A - d_j I)^{-1} f themselves, written to the DEVICE array V of
 * (k+1)*N doubles, system-major (V[j*N + i]), with the stopping rule of bura_solve.
 */
int bura_solve_systems(bura_plan* plan, const double* f, double* V, double tol, void* stream);

/*
 * y_j = (A - d_j I) x_j for the plan's shifts (the multi-shift operator of the solve, FP64):
 * x and y are DEVICE arrays of (k+1)*N doubles, system-major.  For testing the operator.
 */
int bura_apply_shifted(bura_plan* plan, const double* x, double* y, void* stream);

/*
 * The partial-fraction form of the plan's rational approximation, t^{-1} r(t) = sum_j c_j / (t - d_j)
 * (eq. (simplified), Sec. 2.2): c[0..k] and d[0..k] are caller-owned HOST arrays of k+1 doubles,
 * d[0] = 0 > d[1] > ... > d[k]; E (may be NULL) receives the error E_alpha(k,k;1) of Definition def-BURA
 * (for plans set up with bura_setup_shifts: the caller's weights and shifts, and E = 0).
 * Errors: BURA_EINVAL (null plan, c or d).
 */
int bura_get_rational(const bura_plan* plan, double* c, double* d, double* E);

/*
 * Statistics of the last solve, copied into the caller's HOST struct: the scale Lambda of eq. (algebraic)
 * (Sec. 1.4), E, the iteration counts and the residual-based bound on ||u - u_r|| / ||f|| of the partial-
 * fraction value u_r of eq. (Rgeneral).  Errors: BURA_EINVAL (null plan or stats).
 */
int bura_get_stats(const bura_plan* plan, bura_stats* stats);

/*
 * Enable (1) or disable (0) per-kernel timing: every fine-level kernel launch of later solves is
 * bracketed by CUDA events recorded on the solve stream, and its duration and algorithmic bytes are
 * accumulated per kernel type.  Enabling resets the counters.  Costs one event pair per launch.
 */
int bura_set_profiling(bura_plan* plan, int enable);

/*
 * Copy up to max_entries per-kernel records (kernel types with at least one timed launch) into the
 * host array out; *n_out receives the number written.
 */
int bura_get_profile(const bura_plan* plan, int max_entries, bura_kernel_prof* out, int* n_out);

/*
 * Allocation-free residual norms (no counterpart in the paper; a service for callers that cannot
 * allocate device memory: code that runs under a caller-owned memory pool or a fixed device-memory
 * budget, or a loop that must never enter the allocator because an allocation there can block or fail).
 *   rr[j] = || f - (A - d[j] I) V_j ||_2^2 for j = 0..nsys-1, A the scaled constant-coefficient
 *   operator of `grid` (coef_kind must be BURA_COEF_CONSTANT), computed in FP64.
 *   d: HOST array of nsys shifts.  f: DEVICE array of N doubles.  V: DEVICE array of nsys*N doubles,
 *   system-major (V[j*N + i]).  rr: DEVICE array of nsys doubles (written).  stream: cudaStream_t.
 * Allocates nothing: no cudaMalloc/cudaFree and no allocating library call.  Its scratch is a fixed
 * file-scope device array of BURA_NOALLOC_MAX_BLOCKS * BURA_NOALLOC_MAX_SYSTEMS doubles plus a
 * counter (about 128 KiB), held by every device that loads the library until the process exits.
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  All calls share the one scratch
 * array, so calls whose kernels overlap on the GPU (different streams, or different host threads
 * on one device) race and must be serialised by the caller.  Each call clears the counter it needs
 * (cudaMemsetAsync on the stream) and overwrites the partial sums before reading them.
 * Errors: BURA_EINVAL (null pointer, nsys < 1, bad grid or variable coefficients),
 *         BURA_ERANGE (nsys > BURA_NOALLOC_MAX_SYSTEMS or N >= 2^31), BURA_ECUDA.
 */
#define BURA_NOALLOC_MAX_SYSTEMS 16
#define BURA_NOALLOC_MAX_BLOCKS 1024
int bura_residual_norms_noalloc(const bura_grid* grid, int nsys, const double* d, const double* f,
                                const double* V, double* rr, void* stream);

/*
 * Move the plan to another fractional power alpha in (0, 1), keeping its grid, operator, k and
 * options: recomputes the 1-BURA coefficients (Algorithm 1's best approximation, eq. (simplified)
 * partial fractions) and every table that depends on the shifts d_j (smoother coefficients, coarse
 * inverses, weights c_j), in the plan's existing device buffers.  The multigrid hierarchy, the
 * tensor maps and the captured PCG graph are kept, so this costs a host Remez solve and a few small
 * copies instead of a setup.  The result of a later solve equals that of a plan set up at alpha.
 * Waits for the plan's last solve to finish on the device; the caller must not run a solve of
 * the same plan concurrently.
 * Errors: BURA_EINVAL, BURA_EREMEZ, BURA_ECUDA (the plan keeps its previous alpha unless the
 * error is BURA_ECUDA from a copy).
 */
int bura_retarget(bura_plan* plan, double alpha);

/*
 * Multi-step BURA (Sec. "Multi-step BURA approximation"): with plans of one grid and operator at
 * alpha_1..alpha_n, u = r_{alpha_n}(A) A^{-1} ... r_{alpha_1}(A) A^{-1} f, the approximation of
 * A^{-(alpha_1+...+alpha_n)} f by successive BURA solves (plans[0] first).  f and u are DEVICE arrays
 * of N doubles (they may alias); each step runs in place in u, stream-ordered on `stream`.  Each step
 * meets tol relative to its own input, as bura_solve; a step's error is carried through the later
 * steps, whose operators r_j(A) A^{-1} have norms up to about lambda_min(A)^{-alpha_j}.
 * Errors: BURA_EINVAL (n < 1, a null plan, plans of different grids), those of bura_solve.
 */
int bura_solve_chain(bura_plan* const* plans, int n, const double* f, double* u, double tol, void* stream);

/*
 * Sum of the partial-fraction solves of several plans of one grid and operator:
 *     u = sum_i sum_j c_{i,j} (A - d_{i,j} I)^{-1} f,
 * each plan's weighted sum added into u in FP64 on the device (plans[0] writes u, the others add).  This
 * runs a quadrature whose nodes are spread over several plans of bura_setup_shifts (eq. (BonitoPasciak),
 * Sec. 5.3), or any sum of BURA solves.  f and u are DEVICE arrays of N doubles and must not alias when
 * n > 1; stream-ordered on `stream`.  Each plan meets tol for its own term as bura_solve does.
 * Errors: BURA_EINVAL (n < 1, a null plan, plans of different grids or devices, f == u with n > 1,
 * tol <= 0), those of bura_solve.
 */
int bura_solve_sum(bura_plan* const* plans, int n, const double* f, double* u, double tol, void* stream);

/*
 * Failure detection of the TMA-staged sweeps: set the budget (SM clocks, >= 0; 0 = the default of about 2 s)
 * of their waits on the shared-memory ring for the later solves of this plan.  A budget shorter than a
 * copy's latency makes the first waits give up: the kernel drains its copies in flight under the default
 * budget, records the fault in the plan's CG state, and the solve returns BURA_ETIMEOUT; the plan stays
 * usable.  Errors: BURA_EINVAL (null plan, cycles < 0).
 */
int bura_set_tma_wait_cycles(bura_plan* plan, long long cycles);

/*
 * Frees every device and host resource of the plan (NULL is accepted): the multigrid hierarchy, the
 * shifted-system workspaces of eq. (Rgeneral) and the plan record.  The caller must not use the plan
 * afterwards, and no solve of it may still be running on the device.  Always returns BURA_OK.
 */
int bura_destroy(bura_plan* plan);

/* Batched solves: n independent problems, one per plan, solved concurrently on this GPU; every problem
 * is one BURA solve of eq. (Rgeneral) (its k+1 shifted systems are independent), so many systems x shifts
 * x right-hand sides are in flight together.  When every plan is device-driven (see bura_batch_create) the
 * call captures the batch as one graph, launches it once and waits (nworkers = parallel branches);
 * otherwise worker threads solve the plans on their own streams as described below.
 *   plans[i]  plan of problem i (grid, coefficients, alpha, k, options of its own); a plan may appear
 *             only once in the list (its buffers serve one solve at a time);
 *   f[i]      device FP64 right-hand side of plan i's grid (N_i values, lexicographic, x fastest);
 *   u[i]      device FP64 output, N_i values;
 *   tol       the relative tolerance of bura_solve, for every problem;
 *   nworkers  host worker threads, each with its own non-blocking CUDA stream, taking the problems in
 *             list order (0: 16; at most n);
 *   status    optional, n entries: the status bura_solve returns for each problem.
 * Each problem is solved exactly as bura_solve solves it alone (the plan's own buffers and captured
 * PCG graph, deterministic reductions), so u[i] is bit-for-bit the single-problem result; the workers'
 * streams overlap the problems' kernels on the device.  Blocks until every solve has finished.
 * Returns BURA_OK, BURA_ENOCONV if some problem missed the tolerance (its u still written), the first
 * other error of any problem, or BURA_EINVAL (null pointers, n < 0, a plan listed twice). */
int bura_solve_batch(bura_plan* const* plans, const double* const* f, double* const* u, int n, double tol,
                     int nworkers, int* status);

/*
 * A batch captured once and launched many times: every problem's whole solve (its solve record, ||f||, the
 * device-side controller, the refinement and PCG loops, the weighted sum and the outcome) is one branch of
 * one CUDA graph, `branches` branches in parallel (problem i on branch i % branches; 0 = 64), so one launch
 * solves all n problems of eq. (Rgeneral) with no host step between them.  Each problem runs the kernels
 * and fixed-order reductions of its plan exactly as bura_solve does, so u[i] is bit-for-bit its single-
 * problem result.  plans, f, u as for bura_solve_batch (device arrays; the addresses are part of the graph,
 * so later runs read and write the same buffers); tol as for bura_solve.  Every plan must be device-driven
 * (FP64, or mixed precision with FP64 refinement, profiling off) and on one device.  The plans must outlive
 * the batch and must not be used by another solve while a run is in flight.
 *   bura_batch_run enqueues one run on `stream`; bura_batch_wait waits for it and writes each problem's
 *   status to status[i] (optional); bura_batch_destroy waits for the plans' last solves and frees the graph.
 * Errors: BURA_EINVAL (null pointers, n < 1, a plan listed twice, a plan that is not device-driven, plans on
 *         different devices, tol <= 0), BURA_ENOMEM, BURA_ECUDA; bura_batch_wait as bura_solve_batch.
 */
typedef struct bura_batch bura_batch;

/*
 * Autotuner of one problem class: sets up plans for the grid, coefficients, alpha and k with candidate
 * option sets derived from *base (NULL: the defaults): smoother degree 2 or 3, the Chebyshev interval of
 * the dimension or twice as wide, and on 2-D constant-coefficient grids in mixed precision the TMA-staged
 * tiles or the grid-stride sweeps; times `trials` solves of each (CUDA events around the device-driven
 * solve of a fixed pseudo-random right-hand side at tolerance tol, median) and writes the fastest option
 * set to *best and its median to *best_ms (may be NULL).  A candidate that fails or misses tol is skipped.
 * Allocates two N-vectors, a stream and the candidates' plans (freed before returning).  The paper has no
 * counterpart: this chooses implementation parameters only, every candidate computes eq. (Rgeneral).
 * Errors: BURA_EINVAL (bad arguments), BURA_ENOMEM, BURA_ENOCONV (no candidate converged).
 */
int bura_autotune(const bura_grid* grid, const double* const* faces, double alpha, int k, const bura_options* base,
                  double tol, int trials, bura_options* best, double* best_ms);
int bura_batch_create(bura_plan* const* plans, const double* const* f, double* const* u, int n, double tol,
                      int branches, bura_batch** out);
int bura_batch_run(bura_batch* batch, void* stream);
int bura_batch_wait(bura_batch* batch, int* status);
int bura_batch_destroy(bura_batch* batch);

/*
 * Solve server: a continuous-batching front end for many independent requests (grids, coefficient
 * fields, alpha, k of their own) arriving over time.  Worker threads, each with its own CUDA stream,
 * take requests in arrival order and serve each from a pool of resident plans: a plan of the same
 * class (grid, coefficient field, k) that is idle is reused, moved to the request's alpha with
 * bura_retarget if needed; otherwise a plan is set up, after evicting idle plans (least recently
 * used first) while the resident plans would exceed the device-memory budget, or after waiting for
 * one to become idle.  Requests of one class run concurrently on separate plans.  f and u are HOST
 * arrays owned by the caller until bura_server_wait has reported the request done; the copies and
 * the solve are stream-ordered on the worker's stream.  All functions are thread-safe.
 */
typedef struct bura_server bura_server;

typedef struct {
    int workers;          /* worker threads (streams); 0 = 8 */
    size_t mem_budget;    /* device bytes the resident plans may hold; 0 = 80 % of the free memory at creation */
    bura_options plan;    /* options of every plan the server sets up */
} bura_server_options;

typedef struct {
    bura_grid grid;
    const double* const* faces;  /* BURA_COEF_FACES: dim face arrays as for bura_setup (caller-owned until done) */
    unsigned long long field;    /* caller's id of the coefficient field: requests with the same grid and field
                                    share plans (ignored for BURA_COEF_CONSTANT) */
    double alpha;                /* in (0, 1) */
    int k;                       /* 1 .. BURA_MAX_K */
    double tol;                  /* as for bura_solve */
    const double* f;             /* HOST, N doubles */
    double* u;                   /* HOST, N doubles, written when the request is done */
} bura_request;

typedef struct {
    int status;          /* the solve's status (BURA_OK, BURA_ENOCONV, ...) */
    int built;           /* 1: a plan was set up for this request */
    int retargeted;      /* 1: a resident plan was moved to this request's alpha */
    int iters, outer;    /* PCG iterations and refinement steps of the solve */
    double err_bound;    /* as in bura_stats */
    double queue_ms;     /* submission -> a worker took the request */
    double service_ms;   /* worker took it -> u written (plan setup or retarget, copies, solve) */
    double total_ms;     /* submission -> done */
} bura_request_info;

typedef struct {
    long long submitted, completed, builds, retargets, reuses, evictions;
    int resident_plans;
    size_t resident_bytes;
    size_t mem_budget;
} bura_server_stats;

void bura_server_default_options(bura_server_options* opt);
/* Errors: BURA_EINVAL, BURA_ECUDA (no device), BURA_ENOMEM. */
int bura_server_create(const bura_server_options* opt, bura_server** out);
/* Queue one request; *id identifies it for bura_server_wait.  Errors: BURA_EINVAL (checked here:
 * grid, alpha, k, tol, pointers), BURA_ENOMEM. */
int bura_server_submit(bura_server* srv, const bura_request* req, unsigned long long* id);
/* Wait up to timeout_s seconds (< 0: no limit) for request id.  BURA_OK: done, *info filled and the
 * request forgotten; BURA_ETIMEOUT: not done yet; BURA_EINVAL: unknown id. */
int bura_server_wait(bura_server* srv, unsigned long long id, double timeout_s, bura_request_info* info);
int bura_server_get_stats(bura_server* srv, bura_server_stats* stats);
/* Serves every queued request, joins the workers and frees every plan and request record (NULL is
 * accepted).  No other call on srv may be in progress or follow (a thread blocked in
 * bura_server_wait must have returned first). */
int bura_server_destroy(bura_server* srv);

/* Static description of a status code. */
const char* bura_strerror(int status);

/* Name and description of the CUDA runtime error behind the last BURA_ECUDA / BURA_ENOMEM returned
 * by this library to the calling thread ("no error" if none); a thread-local static string. */
const char* bura_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BURA_H */
