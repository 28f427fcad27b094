/*
 * rve.h -- C ABI of librve, a GB300 (sm_103a) implementation of the
 * representative-volume-element (RVE) corrector method of Khoromskaia,
 * Khoromskij & Otto, arXiv:1903.12227.
 *
 * For each random realization of a two-valued coefficient field on the
 * periodic cell [0,L)^2 (overlapping axis-parallel square inclusions, Sec. 2,
 * Eqs. "Stoch-decomp", "coef_diag") the library
 *   1. generates the field                         (rve_gen_field),
 *   2. solves the two Q1-FEM corrector problems    (rve_solve_correctors)
 *      -div a (e_i + grad phi_i) = 0, i = 1,2 (Eqs. "RHS_grad1",
 *      "Ellipt_variat", "FEM_Galerk") by preconditioned CG with the paper's
 *      preconditioner B = c0 A_Delta + delta I (Sec. 3.4),
 *   3. reduces them to the 2x2 homogenized matrix   (rve_a_hom)
 *      (Eqs. "A_hom_m", "Ahom_m_entry", "wg01"),
 *   4. returns the derivative of sum_ij G_ij A_ij with respect to every cell
 *      value                                        (rve_a_hom_backward).
 *
 * Grid and layout.  A realization has n = L*m0 nodes per axis (grid step
 * h = 1/m0 on the torus [0,L)^2); n must be a power of two with
 * 32 <= n <= 2048 (the preconditioner's radix-2 transforms).  Node (i1,i2)
 * is at (i1 h, i2 h); cell (c1,c2) is the square whose lower-left node is
 * (c1,c2).  Linear index i1*n + i2 (i2 contiguous; the paper's big-endian
 * order, Sec. 3.2).  A batch of realizations is packed back to back in
 * descriptor order; realization b starts at node offset sum_{b'<b} n_b'^2.
 *
 *   mask   uint32 words, n*n/32 per realization: bit (c % 32) of word
 *          (c / 32), c = c1*n + c2, is set iff cell (c1,c2) is covered.
 *   coef   double, n*n per realization: general cell values a_c (may be NULL
 *          where documented; the mask and the two values are used then).
 *   vec    double2 (or float2 for the FP32 helpers), one per node: the two
 *          correctors' values interleaved, x = corrector 1, y = corrector 2.
 *   A      double [batch][4] = (a11, a12, a21, a22).
 *
 * Memory ownership.  The caller allocates every buffer (device memory unless
 * stated otherwise) and keeps it alive until the work on `stream` is done.
 * The library allocates no device memory: solvers take a caller-provided
 * workspace whose size rve_workspace_size() returns, starting on a 256-byte
 * boundary as cudaMalloc's blocks do (another start gives RVE_EINVAL).
 * Every call is
 * asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy
 * default stream) unless stated otherwise.
 *
 * Errors.  Invalid arguments return RVE_EINVAL before anything is launched.
 * A failed launch returns RVE_ECUDA.  Per-realization solver outcomes
 * (non-convergence, NaN, time-out) are reported in rve_solve_info.status and
 * do not fail the call.
 */
#ifndef RVE_H
#define RVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RVE_OK = 0,
    RVE_EINVAL = 1,     /* invalid argument (nothing launched)              */
    RVE_ENOCONV = 2,    /* max_iter reached before the tolerance            */
    RVE_ENAN = 3,       /* NaN/Inf met in a reduction                        */
    RVE_ETIMEOUT = 4,   /* a bounded device-side wait gave up               */
    RVE_ECUDA = 5,      /* a CUDA call failed                               */
    RVE_ENOMEM = 6,     /* workspace smaller than rve_workspace_size()      */
    RVE_ESCRATCH = 7    /* request larger than the fixed scratch of
                           rve_a_hom_noalloc (RVE_NOALLOC_MAX_NODES)         */
} rve_status;

typedef enum {
    RVE_FP64 = 0,       /* every step in FP64                                */
    RVE_MIXED = 1       /* FP32 stencil/transform/vectors; FP64 dots, outer
                           true-residual refinement and A_hom               */
} rve_precision;

typedef enum {
    RVE_Q1_CONSISTENT = 0,  /* Q1 element matrix K1(x)M1 + M1(x)K1, 9-point */
    RVE_Q1_LUMPED = 1       /* trapezoid mass (the paper's I-hat, Eq.
                               "As_Kron"), 5-point                          */
} rve_scheme;

typedef enum {
    RVE_PATH_FUSED = 0,     /* batched fused pipeline (3 passes/iteration)  */
    RVE_PATH_PLAIN = 1,     /* unfused textbook PCG, one kernel per BLAS-1
                               step; FP64 only                              */
    RVE_PATH_PERSISTENT = 2 /* one cooperative persistent launch for the
                               whole batch (uneven sizes allowed)           */
} rve_path;

/* One realization (Sec. 2 and 3.1): L unit cells per axis, m0 grid cells per
 * unit length, n_incl square inclusions of incl_cells x incl_cells grid
 * cells each, lower-left corners uniform on the grid nodes (drawn with
 * SplitMix64 from (seed, index)), overlaps allowed.  Coefficient a_matrix
 * outside and a_incl inside the covered set (Eq. "coef_diag").  48 bytes. */
typedef struct {
    int32_t L, m0, incl_cells, n_incl;
    double a_matrix, a_incl;
    uint64_t seed, index;
} rve_realization;

/* Solver options (Sec. 3.4).  Zero-initialised fields take defaults. */
typedef struct {
    int32_t scheme;      /* rve_scheme                                      */
    int32_t precision;   /* rve_precision                                   */
    int32_t path;        /* rve_path                                        */
    int32_t max_iter;    /* cap on CG iterations per corrector (0 = 20000)  */
    double tol;          /* stop when ||f - A u||_2 <= tol ||f||_2 (0=1e-10)*/
    double delta;        /* preconditioner shift; 0 = drop the constant mode*/
    double inner_tol;    /* mixed: relative reduction per FP32 cycle (0=1e-4)*/
    int32_t tile_rows;   /* stencil tile height in node rows (1..n; n need
                            not be a multiple), 0 = tuned or default       */
    int32_t col_tile;    /* threads of a column-solve block (power of two,
                            32..512); 0 = 128 (mixed) or 512 (FP64)         */
    int32_t check_every; /* host convergence poll period (0 = 8)            */
    int32_t timeout_us;  /* persistent path: bound on each grid-wide wait, in
                            microseconds (0 = 2 s)                          */
    int32_t flags;       /* must be 0                                       */
    int32_t reserved;    /* must be 0                                       */
} rve_solve_opts;

/* Per-realization solver report (device memory, one per realization). */
typedef struct {
    int32_t iters[2];     /* CG iterations (operator applications) per corrector */
    int32_t status;       /* rve_status                                           */
    int32_t refinements;  /* true-residual evaluations (FP64 or double word)      */
    int32_t steps;        /* fused pipeline steps spent iterating (both correctors
                             advance together; plain path: CG iterations)         */
    int32_t reserved;     /* 0                                                    */
    double relres[2];     /* last FP64 true relative residual per corrector       */
} rve_solve_info;         /* 40 bytes */

/* Human-readable name of a status code (static string). */
const char* rve_status_string(int32_t status);

/* Description of the last CUDA failure seen by this host thread (where it
 * happened and CUDA's error string); "" if none. */
const char* rve_last_error(void);

/* Library version: major*10000 + minor*100 + patch. */
int32_t rve_version(void);

/* Number of uint32 mask words / nodes of a batch (host-side arithmetic). */
int64_t rve_mask_words(const rve_realization* r, int32_t batch);
int64_t rve_nodes(const rve_realization* r, int32_t batch);

/* Field generation (Sec. 2 and 3.1, Eq. "Stoch-decomp"): writes the covered
 * set of every realization as a bitmask.  r: host array [batch].
 * mask: device, rve_mask_words() words, fully overwritten. */
rve_status rve_gen_field(const rve_realization* r, int32_t batch, uint32_t* mask,
                         void* stream);

/* Cell values of the coefficient (Eq. "coef_diag": a_matrix outside, a_incl
 * inside the covered set) from the bitmask: coef (device double per cell)
 * is overwritten.  The starting point of an explicit coefficient array
 * (finite differences, the adjoint's inputs). */
rve_status rve_coef_from_mask(const rve_realization* r, int32_t batch, const uint32_t* mask,
                              double* coef, void* stream);

/* Galerkin right-hand sides f_i = -int a d_i psi (Eq. "FEM_discr_RHS"),
 * with the stiffness's quadrature (Sec. 4.3): f[node] = (f_1, f_2).
 * Coefficients from coef (device doubles) if non-NULL, else from mask. */
rve_status rve_rhs(const rve_realization* r, int32_t batch, const uint32_t* mask,
                   const double* coef, double* f, void* stream);

/* y = A x, A the Q1 stiffness of Eq. "FEM_matrix" assembled as in Eq.
 * "As_Kron", applied matrix-free as a 9-point (consistent) or 5-point
 * (lumped) periodic stencil.  precision = RVE_FP64: x, y are double2 per
 * node; RVE_MIXED: float2 per node, FP32 arithmetic. */
rve_status rve_apply_stiffness(const rve_realization* r, int32_t batch,
                               const uint32_t* mask, const double* coef,
                               int32_t scheme, int32_t precision,
                               const void* x, void* y, void* stream);

/* y = M x, M = M1 (x) M1 the Q1 mass matrix of the scheme (1D consistent
 * h [1/6, 2/3, 1/6], lumped h [0, 1, 0]), periodic: turns nodal values of
 * a load function into the Galerkin load vector of the general solve (the
 * FEM convergence test of Sec. 3.5).  x, y: device double2 per node (two
 * loads side by side), must not alias. */
rve_status rve_apply_mass(const rve_realization* r, int32_t batch, int32_t scheme,
                          const double* x, double* y, void* stream);

/* Chebyshev moments for the density of states of the stiffness matrix A
 * (the spectral-density appendix, Eqs. "DOS", "DOS_gauss"): for every
 * realization and each of its two start vectors v (device v[nodes][2]),
 *   mu[b][c][k] = v_c^T T_k(A~) v_c,  A~ = (2 A - (hi + lo) I) / (hi - lo),
 * k = 0 .. K-1, with T_k the Chebyshev polynomials; [lo, hi] must contain
 * the spectrum of A (e.g. lo = 0, hi = 4 w0 max(4 a) by Gershgorin: 16/3
 * a_max consistent, 8 a_max lumped).  The Gaussian-broadened density is a
 * fixed linear combination of these moments (done on the host).  The matrix
 * is applied matrix-free in FP64, one application per two moments.  mu:
 * device doubles [batch][2][K]; ws: rve_cheb_workspace_size() bytes.
 * Errors: RVE_EINVAL (K < 2, hi <= lo, missing pointers), RVE_ENOMEM. */
size_t rve_cheb_workspace_size(const rve_realization* r, int32_t batch);
rve_status rve_cheb_moments(const rve_realization* r, int32_t batch, const uint32_t* mask,
                            const double* coef, int32_t scheme, const double* v, int32_t K,
                            double lo, double hi, double* mu, void* ws, size_t ws_bytes,
                            void* stream);

/* Reconstruction of the broadened density of states from Chebyshev trace
 * moments (host memory, host arithmetic, FP64; the spectral-density
 * appendix, Eq. "DOS_gauss", by the kernel polynomial method).
 * rve_dos_coefficients: c[i][k] (nt x K) = the Chebyshev coefficients of
 *   lambda -> g_eta(t_i - lambda) on [lo, hi], g_eta the Gaussian of
 *   standard deviation eta, by Chebyshev-Gauss quadrature with `quad` nodes
 *   (0 = max(4K, 1024)): c_ik = (2 - [k = 0]) / quad * sum_j g_eta(t_i -
 *   lambda_j) T_k(x_j), x_j = cos(pi (j + 1/2) / quad), lambda_j the image
 *   of x_j on [lo, hi].
 * rve_dos_from_moments: phi[i] = (1/m) sum_k c_ik mu[k] for trace moments
 *   mu[k] = Tr T_k(A~) (or their estimate; see rve_cheb_moments) of a matrix
 *   of order m whose spectrum lies in [lo, hi].
 * Errors: RVE_EINVAL (missing pointers, K < 1, hi <= lo, eta <= 0, m <= 0). */
rve_status rve_dos_coefficients(const double* t, int32_t nt, int32_t K, double lo, double hi,
                                double eta, int32_t quad, double* c);
rve_status rve_dos_from_moments(const double* mu, int32_t K, double m, double lo, double hi,
                                double eta, const double* t, int32_t nt, double* phi);

/* y = B^{-1} x with B = c0 A_Delta + delta I (Sec. 3.4), A_Delta the
 * periodic 5-point Laplacian (Eq. "Lap_Kron"), c0 = (a_matrix + a_incl)/2
 * (Lemma "Cond_Number").  delta = 0 drops the constant mode.  Applied by
 * separable real (Hartley) transforms along each axis.  x, y as in
 * rve_apply_stiffness; x and y may alias.  ws: device workspace of at least
 * rve_workspace_size(r, batch, NULL) bytes. */
rve_status rve_apply_precond(const rve_realization* r, int32_t batch, double delta,
                             int32_t precision, const void* x, void* y,
                             void* ws, size_t ws_bytes, void* stream);

/* Workspace bytes needed by rve_solve_correctors / rve_a_hom /
 * rve_apply_precond for this batch and these options (opts may be NULL for
 * defaults).  Returns 0 for invalid arguments. */
size_t rve_workspace_size(const rve_realization* r, int32_t batch,
                          const rve_solve_opts* opts);

/* Solve both corrector problems of every realization (Sec. 3.4, 4.1):
 * PCG from u = 0 until the FP64 true residual meets opts->tol.
 * mask / coef: as in rve_rhs (coef overrides the mask when non-NULL; c0
 * still comes from a_matrix and a_incl).  u: device double2 per node,
 * overwritten with the correctors (mean zero up to rounding).  info: device
 * rve_solve_info[batch].  ws: device workspace.  With the fused path the
 * call polls convergence every opts->check_every iterations (a stream
 * synchronisation); the persistent path launches once and does not sync. */
rve_status rve_solve_correctors(const rve_realization* r, int32_t batch,
                                const uint32_t* mask, const double* coef,
                                const rve_solve_opts* opts, double* u,
                                rve_solve_info* info, void* ws, size_t ws_bytes,
                                void* stream);

/* A u = f for a caller's pair of load vectors per node instead of the
 * corrector right-hand sides (the general solve of the FEM convergence test,
 * Sec. 3.5, with a load such as sin(2 pi x) cos(6 pi y)): f is device
 * [nodes][2] FP64 (see rve_apply_mass), and each of its two components must
 * sum to zero over every realization (the periodic problem is solvable only
 * then; otherwise the solve ends with RVE_ENOCONV).  Everything else --
 * options, u (mean-zero on exit), info, workspace, paths -- as in
 * rve_solve_correctors. */
rve_status rve_solve_rhs(const rve_realization* r, int32_t batch, const uint32_t* mask,
                         const double* coef, const double* f, const rve_solve_opts* opts,
                         double* u, rve_solve_info* info, void* ws, size_t ws_bytes,
                         void* stream);

/* Homogenized matrix of every realization from its correctors u.
 * A: energy form a_ij = (1/L^2) int (e_j + grad phi_j).a(e_i + grad phi_i)
 * (Eq. "wg01" as rewritten in its symmetry argument), summed cell by cell as
 * (1/L^2) sum_c a_c (xi_i + P_c u_i)^T E (xi_j + P_c u_j) -- equal to the
 * node form mean(a) delta_ij - (f_i.u_j + f_j.u_i - u_i.A u_j)/L^2, but
 * without its cancellation.  A_flux (nullable): flux form of Eq.
 * "Ahom_m_entry", a_ij = mean(a) delta_ij - f_j.u_i / L^2.  Both device
 * double[batch][4].
 * precision: RVE_FP64 sums in double-double arithmetic on the FP64 pipe
 * (differences of u across a cell exact, ~106-bit sums), so A is the
 * correctly rounded energy of the given u up to a few units in the last
 * place; A_lo (nullable, RVE_FP64 only) then receives the low parts, and
 * A + A_lo carries the energy to ~1e-30 relative -- enough to difference two
 * nearby A_hom (finite differences) without FP64 cancellation.
 * RVE_MIXED sums in double words on the FP32 pipe (~1e-14 relative; GB300's
 * FP64 pipe is ~1/64 of FP32), for the mixed-precision pipeline; A_lo must
 * be NULL.  ws: rve_workspace_size() bytes. */
rve_status rve_a_hom(const rve_realization* r, int32_t batch, const uint32_t* mask,
                     const double* coef, int32_t scheme, int32_t precision, const double* u,
                     double* A, double* A_lo, double* A_flux, void* ws, size_t ws_bytes,
                     void* stream);

/* Adjoint of the energy form: grad_coef[cell] = d(sum_ij gradA_ij a_ij)/d a_c
 * = (1/L^2) sum_ij gradA_ij int_cell (e_i + grad phi_i).(e_j + grad phi_j)
 * (the problem is self-adjoint, so no second solve).  gradA: device
 * double[batch][4]; grad_coef: device double per cell, overwritten. */
rve_status rve_a_hom_backward(const rve_realization* r, int32_t batch,
                              int32_t scheme, const double* u, const double* gradA,
                              double* grad_coef, void* stream);

/* Whole pipeline with HOST inputs and outputs: copies the descriptors in,
 * generates the fields, solves, reduces, and copies A (and info) back into
 * host memory; returns after the results are in host memory.  ws: device
 * workspace of rve_homogenize_workspace_size() bytes (holds the masks and
 * correctors too).  A_host: double[batch][4]; info_host nullable. */
size_t rve_homogenize_workspace_size(const rve_realization* r, int32_t batch,
                                     const rve_solve_opts* opts);
rve_status rve_homogenize_host(const rve_realization* r_host, int32_t batch,
                               const rve_solve_opts* opts, double* A_host,
                               rve_solve_info* info_host, void* ws, size_t ws_bytes,
                               void* stream);

/* Plans: the whole pipeline (field, both correctors, A_hom) of a fixed batch
 * (sizes may differ), captured once into a CUDA graph and relaunched; the
 * solve needs no host synchronisation, so one graph launch runs all of it
 * (Sec. 3.4 for the solver itself).  opts->path selects the solve inside
 * the graph:
 *   RVE_PATH_PERSISTENT: ONE cooperative persistent launch over all
 *     realizations, with grid-wide barriers between the pipeline phases;
 *     every barrier wait is bounded by opts->timeout_us, after which the
 *     launch ends and the affected realizations report RVE_ETIMEOUT;
 *   RVE_PATH_FUSED: the fused pipeline kernels inside a conditional WHILE
 *     node of the graph (groups of 4 pipeline steps, re-armed on the device
 *     while a realization is unfinished and the step bound is not reached);
 *     kernel boundaries separate the phases, each kernel at its own
 *     occupancy;
 *   RVE_PATH_PLAIN: RVE_EINVAL.
 * rve_plan_create: validates (host only) and lays out the workspace.
 * rve_plan_execute: A (device double[batch][4], energy form, reduced as
 * rve_a_hom with opts->precision) and info (device rve_solve_info[batch]);
 * ws holds masks, correctors and solver state (rve_plan_workspace_size
 * bytes).  The first call (and any call with different ws/A/info pointers)
 * uploads the descriptors with a host synchronisation and captures the graph
 * on `stream`; later calls only launch the graph.  `stream` must be a
 * created stream (not the legacy default stream, on which CUDA cannot
 * capture; NULL gives RVE_EINVAL).  rve_launch_count() counts the graph's
 * kernel nodes once per execution (a RVE_PATH_FUSED plan's loop body once,
 * however often it ran).  rve_plan_destroy frees the host-side plan. */
typedef struct rve_plan_s* rve_plan;
rve_status rve_plan_create(const rve_realization* r, int32_t batch, const rve_solve_opts* opts,
                           rve_plan* plan);
size_t rve_plan_workspace_size(rve_plan plan);
rve_status rve_plan_execute(rve_plan plan, double* A, rve_solve_info* info, void* ws,
                            size_t ws_bytes, void* stream);
void rve_plan_destroy(rve_plan plan);

/* Autotuner.  For every distinct grid size n of the batch, times short
 * trial solves of up to 16 of its realizations for each candidate tile shape
 * (stencil tile heights; column-block threads 128/256/512 on the fused
 * path, 256 on the persistent path) and records the fastest in the
 * process-wide tuner table, keyed by (n, precision, persistent).  Plans and
 * solves with opts->tile_rows == 0 and opts->col_tile == 0 then use the
 * table.  ws: device scratch for the trials (candidates that do not fit are
 * skipped); synchronises `stream`.  rve_tuner_save / rve_tuner_load write
 * and read the table as text; rve_tuner_lookup returns 1 and the entry if
 * present; rve_tuner_clear empties it. */
rve_status rve_autotune(const rve_realization* r, int32_t batch, const rve_solve_opts* opts,
                        void* ws, size_t ws_bytes, void* stream);
rve_status rve_tuner_save(const char* path);
rve_status rve_tuner_load(const char* path);
int32_t rve_tuner_lookup(int32_t n, int32_t precision, int32_t persistent, int32_t* tile_rows,
                         int32_t* block_threads);
void rve_tuner_clear(void);

/* Ensemble statistics (host memory, host arithmetic, FP64, summed in
 * index order so that results do not depend on how the realizations were
 * distributed).  A: double[N][4] (a11, a12, a21, a22) of N >= 2
 * realizations of RVE size L in d dimensions.  Outputs (each nullable):
 *   mean[4]   empirical mean (Eq. "A_hom_Empir");
 *   var[4]    unbiased sample variance of each entry;
 *   std12     sqrt(mean a12^2) (Eq. "Var1"), stddiff sqrt(mean (a11-a22)^2)
 *             (Eq. "Var2") -- the paper's estimators, no mean subtracted;
 *   Q[16]     L^d/(N-1) sum_n (A_n - mean)(x)(A_n - mean), the 4x4 Kronecker
 *             unfolding of the quartic tensor of Eq. "quartic" (row/column
 *             order a11, a12, a21, a22). */
rve_status rve_statistics(const double* A, int64_t N, double L, int32_t d, double* mean,
                          double* var, double* std12, double* stddiff, double* Q);

/* Allocation-free variant of rve_a_hom, for callers that cannot allocate
 * device memory: programs whose device memory is all owned by their own pool
 * allocator, and latency-critical loops that cannot afford cudaMalloc /
 * cudaFree (which may synchronise the device).  It takes no workspace.  The
 * paper has no counterpart; results equal those of rve_a_hom with precision
 * RVE_MIXED (same double-word sums, same order).
 * Scratch: a fixed library-owned device array of 1 MiB (8 partial sums per
 * 1024 nodes) that every GPU loading the library holds until exit; requests
 * above RVE_NOALLOC_MAX_NODES nodes in total return RVE_ESCRATCH before
 * anything is launched.  The first call on a device does a one-time set-up
 * (it looks up the array's device address with that device current): make
 * that first call before any stream capture.  The set-up is not repeated, so
 * after cudaDeviceReset (or any other teardown of the device's primary
 * context) in the same process the recorded address is stale: do not call
 * this entry point on that device again.  All calls share the array and
 * it keeps the last call's contents; each call writes every partial it reads,
 * so nothing needs clearing, but calls that overlap on the GPU (other streams
 * or host threads) race on it and must be serialised by the caller.
 * Arguments as rve_a_hom. */
#define RVE_NOALLOC_MAX_NODES (1LL << 24)
rve_status rve_a_hom_noalloc(const rve_realization* r, int32_t batch, const uint32_t* mask,
                             const double* coef, int32_t scheme, const double* u,
                             double* A, double* A_flux, void* stream);

/* ---------------------------------------------------------------- 3D --
 * The 3D form of the method (Sec. 2: the setting carries over verbatim to
 * d > 2 with a d x d diagonal coefficient; Sec. 3.2: the rank-3 Kronecker
 * Laplacian A_Delta = A_P (x) I (x) I + I (x) A_P (x) I + I (x) I (x) A_P and
 * Eq. "As_Kron_d"; Sec. 3.1: multilinear functions on cubes).  Realization
 * fields as in 2D with L, m0, incl_cells, n_incl describing the torus
 * [0,L)^3, n = L*m0 nodes per axis, n a power of two, 32 <= n <= 256, and
 * n_incl cubes of incl_cells^3 cells whose lower corners are uniform on the
 * nodes (draws 3k, 3k+1, 3k+2 of the realization's stream for cube k).
 * Node (i1,i2,i3) at linear index (i1 n + i2) n + i3; cell (c1,c2,c3) has
 * lower corner node (c1,c2,c3) and the same index.  Realizations are packed
 * back to back (offset sum_{b'<b} n_b'^3).
 *   mask   uint8, one byte per cell (nonzero = covered by a cube);
 *   coef   double per cell (general values; NULL = mask and the two values);
 *   vectors of three components (u, f, x, y): double [nodes][3].
 * Element matrix: K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1
 * (trilinear Q1, M1 consistent or lumped as in 2D), 27-point stencil.
 * All device pointers; ws: rve3_workspace_size() bytes of device memory,
 * owned by the caller, contents undefined between calls.  Every call is
 * asynchronous on `stream` except rve3_solve_correctors, which polls the
 * convergence flags from the host.  Errors: RVE_EINVAL (sizes outside the
 * range, n not a power of two, non-positive or non-finite coefficients,
 * missing pointers, unknown scheme), RVE_ENOMEM (ws too small), RVE_ECUDA. */
typedef struct {
    int32_t scheme;      /* rve_scheme                                      */
    int32_t precision;   /* RVE_FP64: PCG in FP64.  RVE_MIXED: FP32 PCG
                            cycles restarted on the FP64 true residual
                            (iterative refinement); the stopping test is
                            the same FP64 one                               */
    int32_t max_iter;    /* cap on CG iterations per corrector (0 = 20000)  */
    int32_t check_every; /* host convergence poll period (0 = 8)            */
    double tol;          /* stop when ||f - A u||_2 <= tol ||f||_2 (0=1e-10)*/
    double delta;        /* preconditioner shift; 0 = drop the constant mode*/
    double inner_tol;    /* mixed: relative reduction per FP32 cycle (0=1e-4)*/
} rve3_solve_opts;       /* 40 bytes */

typedef struct {
    int32_t iters[3];     /* PCG iterations per corrector (FP32 ones when mixed) */
    int32_t status;       /* rve_status (first failure of the three)            */
    int32_t refinements;  /* FP64 true residuals evaluated (both pairs)         */
    int32_t reserved;
    double relres[3];     /* FP64 true relative residual per corrector          */
} rve3_solve_info;        /* 48 bytes */

/* Nodes of the batch (sum of n^3), or -1 if a descriptor is invalid. */
int64_t rve3_nodes(const rve_realization* r, int32_t batch);
/* Workspace bytes of every rve3_* call on this batch (0 if invalid). */
size_t rve3_workspace_size(const rve_realization* r, int32_t batch);
/* Cube field: mask[nodes] (bytes) of every realization. */
rve_status rve3_gen_field(const rve_realization* r, int32_t batch, uint8_t* mask,
                          void* stream);
/* Corrector loads f_i = -A (x_i) (the Galerkin right-hand sides of the
 * three cell problems -div a (e_i + grad phi_i) = 0), f[nodes][3].  They do
 * not depend on the scheme (the 1D mass rows sum to h/2 in both; `scheme`
 * is validated only): f_i = (h^2/4) (sum of the 4 cells above the node
 * along axis i - sum of the 4 cells below), exactly 0 where the 8 cells
 * around a node agree. */
rve_status rve3_rhs(const rve_realization* r, int32_t batch, const uint8_t* mask,
                    const double* coef, int32_t scheme, double* f, void* ws,
                    size_t ws_bytes, void* stream);
/* y = A x (27-point stencil), x, y [nodes][3], must not alias. */
rve_status rve3_apply_stiffness(const rve_realization* r, int32_t batch, const uint8_t* mask,
                                const double* coef, int32_t scheme, const double* x,
                                double* y, void* ws, size_t ws_bytes, void* stream);
/* y = B^{-1} x, B = c0 A_Delta + delta I (c0 = (a_matrix + a_incl)/2; with
 * delta = 0 the constant mode of each component is dropped): Hartley
 * transforms along the two inner axes, periodic tridiagonal solves along
 * the outer one.  x, y [nodes][3]; x is read before y is written (x may
 * equal y). */
rve_status rve3_apply_precond(const rve_realization* r, int32_t batch, double delta,
                              const double* x, double* y, void* ws, size_t ws_bytes,
                              void* stream);
/* The three correctors by preconditioned CG from u = 0 (FP64 or mixed
 * precision, opts->precision): u[nodes][3]; info[batch] (device) per
 * realization.  With general cell values the mixed path keeps an FP32 copy
 * of them in ws. */
rve_status rve3_solve_correctors(const rve_realization* r, int32_t batch, const uint8_t* mask,
                                 const double* coef, const rve3_solve_opts* opts, double* u,
                                 rve3_solve_info* info, void* ws, size_t ws_bytes,
                                 void* stream);
/* 3x3 homogenized matrix per realization: A[b][3 i + j] = L^-3 sum_cells
 * a_c v_i^T E v_j (energy form, v_i = x_i + u_i on the cell's corners) and,
 * if A_flux is not NULL, A_flux[b][3 i + j] = L^-3 sum_cells a_c int_c
 * d_j (x_i + u_i) (flux form).  Device doubles [batch][9]. */
rve_status rve3_a_hom(const rve_realization* r, int32_t batch, const uint8_t* mask,
                      const double* coef, int32_t scheme, const double* u, double* A,
                      double* A_flux, void* ws, size_t ws_bytes, void* stream);

/* Ensemble statistics of 3D realizations (host memory, host arithmetic,
 * FP64, summed in index order).  A: double[N][9] (row-major 3x3 A_hom) of
 * N >= 2 realizations of RVE size L.  Outputs (each nullable): mean[9]
 * (Eq. "A_hom_Empir"), var[9] unbiased sample variance of each entry, and
 * Q[81] = L^3/(N-1) sum_n (A_n - mean)(x)(A_n - mean), the 9x9 unfolding of
 * the quartic tensor of Eq. "quartic" in d = 3 (entries in row-major order
 * a11 .. a33).  Errors: RVE_EINVAL (N < 2, L not positive, A NULL). */
rve_status rve3_statistics(const double* A, int64_t N, double L, double* mean, double* var,
                           double* Q);

/* Diagnostics for benchmarks.  The profiler state is process-wide and NOT
 * thread-safe: enable it only while a single host thread solves on a single
 * stream (two streams or threads solving while it is on share, and race
 * on, its event pool and totals).  The launch counter is an atomic and safe
 * to read from any thread.
 * rve_profile_enable(1): the fused solver brackets every launch of its five
 * pipeline kernels with CUDA events on the caller's stream and accumulates
 * their durations.  rve_profile_read(ms[5], launches[5]) returns the totals
 * per kernel -- 0 true-residual (refinement) pass, 1 stencil pass, 2 update
 * + row transform, 3 column transform, 4 control -- and resets them; it
 * returns 5.
 * rve_launch_count() returns the number of kernels the library launched
 * since the previous call. */
void rve_profile_enable(int32_t on);
int32_t rve_profile_read(double* ms, int64_t* launches);
/* The same for the 3D solver (enabled by rve_profile_enable as well): every
 * launch of rve3_solve_correctors bracketed by events, totals per kind --
 * 0 stiffness of the CG steps (27-point stencil, with the p.q partials),
 * 1 line transform (x or y Hartley pass), 2 z tridiagonal solve, 3 CG
 * vector steps (dots, updates), 4 CG scalar steps, 5 FP64 true residual
 * (stiffness with the residual fused) -- reset on read; returns 6. */
int32_t rve3_profile_read(double* ms, int64_t* launches);
int64_t rve_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* RVE_H */
