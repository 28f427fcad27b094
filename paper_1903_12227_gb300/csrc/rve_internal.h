// rve_internal.h -- host-side plan, workspace layout and kernel launchers
// shared by the translation units of librve (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "rve.h"

#include <atomic>

namespace rve {

struct RDesc;

// Kernel launches issued by the library (diagnostics).
extern std::atomic<long long> g_launches;
inline void note_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }
// Workspaces start on a 256-byte boundary (cudaMalloc's alignment): the
// library carves them into 256-byte aligned vectors and moves whole rows of
// them with 16-byte aligned bulk operations.
inline bool ws_misaligned(const void* ws) { return ((uintptr_t)ws & 255) != 0; }

// Solver phases of one realization (fused pipeline).
enum : int32_t { PH_REFINE = 0, PH_ITER = 1, PH_DONE = 2 };

// Per-realization solver state (device), written only by the control kernel
// (and the initialiser); read by the pipeline kernels one launch later.
struct RState {
    int32_t phase, parity, refinements, status;
    int32_t iters[2];
    int32_t active[2];   // corrector still iterating in the current cycle
    int32_t cdone[2];    // corrector met the outer tolerance
    int32_t final_pass, steps;   // steps: pipeline steps spent in ITER
    double fnorm[2];     // ||f_c||
    double s[2];         // scale of the current inner system (||r64|| at restart)
    double rho[2];       // r.z of the current residual
    double alpha[2];     // pending step length (lagged solution update)
    double beta[2];      // direction update factor for the next stencil pass
    double target[2];    // inner-cycle relative residual target
    double relres[2];    // last true relative residual
    double best[2];      // smallest inner residual of the cycle so far
    int32_t stall[2];    // inner steps since it last fell below STALL_FACTOR * best
    int32_t pad_[2];
};

// Tile geometry of one realization for the fused kernels.
struct Tiles {
    int tS;   // node rows per stencil tile
    int tU;   // rows per row-transform block
    int tC;   // columns per column-transform block
};

struct Plan {
    int batch = 0;
    int precision = RVE_FP64;
    int scheme = RVE_Q1_CONSISTENT;
    int path = RVE_PATH_FUSED;
    size_t vbytes = 16;             // bytes of one node pair (float2 / double2)
    int64_t nodes = 0, words = 0;
    int max_log2n = 0;
    std::vector<RDesc> desc;        // host copy
    // startA: tiles of 1024 cells (FP64 A_hom); startA2: strips of
    // a_hom_strip_rows(n) rows (mixed A_hom)
    std::vector<int32_t> startS, startU, startC, startA, startA2;
    int tilesS = 0, tilesU = 0, tilesC = 0, tilesA = 0, tilesA2 = 0;
    size_t smemS = 0, smemU = 0, smemC = 0;
    int blockC = 512;               // threads of a column-solve block
    int persist_grid = 0;           // blocks of the persistent launch (0 = not prepared)
    size_t persist_smem = 0;
    // workspace offsets (bytes)
    size_t o_desc = 0, o_startS = 0, o_startU = 0, o_startC = 0, o_startA = 0, o_startA2 = 0;
    size_t o_tw64 = 0, o_tw32 = 0, o_lap = 0, o_lap32 = 0, o_rho64 = 0, o_rho32 = 0;
    size_t o_state = 0, o_partS = 0, o_partU = 0, o_partC = 0, o_partA = 0, o_ctl = 0;
    size_t o_uscal = 0, o_cnt = 0;
    size_t o_X = 0, o_R = 0, o_Q = 0, o_T = 0, o_P0 = 0, o_P1 = 0;
    size_t total = 0;
};

// Plain FP64 PCG building blocks (rve_plain.cu): vector kernels over the
// nodes of realization b (PL_NODES per block, from desc[b].node_off) on
// corrector pairs, and the per-pair scalar steps.
constexpr int PL_THREADS = 256;
constexpr int PL_NODES = 1024;   // nodes per block (n^2 and n^3 are multiples of 1024)
struct PlainScal {
    double rho[2], alpha[2], beta[2], fnorm[2], relres[2];
    int32_t active[2], iters[2];
    int32_t done, status;
};
enum { SC_FNORM = 0, SC_RHO0, SC_ALPHA, SC_CONV, SC_BETA, SC_RELRES };
__global__ void k_pl_dot(const RDesc* desc, int b, const double2* __restrict__ x,
                         const double2* __restrict__ y, double* part);
__global__ void k_pl_axpy(const RDesc* desc, int b, const PlainScal* sc, double2* __restrict__ u,
                          double2* __restrict__ r, const double2* __restrict__ p,
                          const double2* __restrict__ q, double* part);
__global__ void k_pl_xpby(const RDesc* desc, int b, const PlainScal* sc,
                          const double2* __restrict__ z, double2* __restrict__ p);
__global__ void k_pl_scalar(PlainScal* sc, const double* part, int nb, int what, double tol,
                            int max_iter);
// Fills the lookup tables (twiddles, Laplacian eigenvalues, filter roots)
// for sizes up to 2^max_log2n.
cudaError_t fill_tables(const Tables& tb, int max_log2n, cudaStream_t s);

// Records "<where>: <CUDA error string>" for rve_last_error(); returns RVE_ECUDA.
rve_status note_error(const char* where, cudaError_t e);

// Options with the library defaults filled in.
rve_solve_opts resolved_opts(const rve_solve_opts* o);
// Tuned tile shape of grid size n (false if none recorded).
bool tuned_tiles(int n, int precision, int path, int* tS, int* blockC);
// Kernel attributes and co-resident grid size of the persistent launch.
rve_status prepare_persistent(Plan& p);

// Validates descriptors and fills plan (host only).  opts may be NULL.
rve_status make_plan(const rve_realization* r, int32_t batch, const rve_solve_opts* opts,
                     Plan& plan, bool need_vectors);

// Uploads descriptors/tile tables and fills the lookup tables in ws.
rve_status upload_plan(const Plan& plan, void* ws, cudaStream_t s);
// Device pointers of the lookup tables in the workspace, and the kernel that fills them.
Tables tables_of(const Plan& p, const void* ws);
cudaError_t launch_tables(const Plan& p, void* ws, cudaStream_t s);

// Launchers (return cudaGetLastError()).
cudaError_t launch_gen_field(const Plan& p, void* ws, uint32_t* mask, cudaStream_t s);
cudaError_t launch_rhs(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                       double* f, cudaStream_t s);
cudaError_t launch_coef_from_mask(const Plan& p, const uint32_t* mask, double* coef,
                                  cudaStream_t s);
cudaError_t launch_stiffness(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                             int scheme, int precision, const void* x, void* y, cudaStream_t s);
// Row, column(+scale), row transform passes for realizations
// [b_first, b_first + b_count): y = B^{-1} x, tmp a scratch vector.
template <typename V>
cudaError_t precond_passes(const Plan& p, void* ws, double delta, const V* x, V* y, V* tmp,
                           int b_first, int b_count, cudaStream_t s);
cudaError_t launch_precond(const Plan& p, void* ws, double delta, int precision, const void* x,
                           void* y, cudaStream_t s);
// `f`: device [nodes][2] load vectors; NULL = the corrector right-hand sides.
rve_status run_solve_fused(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                           const rve_solve_opts& o, double* u, rve_solve_info* info,
                           cudaStream_t s, const double* f = nullptr);
rve_status run_solve_persistent(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                                const rve_solve_opts& o, double* u, rve_solve_info* info,
                                cudaStream_t s, const double* f = nullptr);
rve_status upload_descriptors(const Plan& p, void* ws, cudaStream_t s);
rve_status enqueue_solve_persistent(const Plan& p, void* ws, const uint32_t* mask,
                                    const double* coef, const rve_solve_opts& o, double* u,
                                    rve_solve_info* info, cudaStream_t s, const double* f = nullptr);
// The fused pipeline steps inside a CUDA graph conditional WHILE node; only
// while `s` is capturing (RVE_EINVAL otherwise).  prepare_graph_loop sets
// the kernels' shared-memory attributes (call it before the capture).
rve_status prepare_graph_loop(const Plan& p);
rve_status enqueue_solve_graph_loop(const Plan& p, void* ws, const uint32_t* mask,
                                    const double* coef, const rve_solve_opts& o, double* u,
                                    rve_solve_info* info, cudaStream_t s, const double* f = nullptr);
rve_status run_solve_plain(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                           const rve_solve_opts& o, double* u, rve_solve_info* info,
                           cudaStream_t s, const double* f = nullptr);
cudaError_t launch_mass(const Plan& p, int scheme, const double* x, double* y, cudaStream_t s);
size_t cheb_workspace_size(const Plan& p);
cudaError_t launch_cheb(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                        int scheme, const double* v, int K, double lo, double hi, double* mu,
                        cudaStream_t s);
// precision RVE_FP64: double-double sums on the FP64 pipe (A_lo = low
// parts, nullable); RVE_MIXED: double-word sums on the FP32 pipe.
cudaError_t launch_a_hom(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                         int scheme, int precision, const double* u, double* A, double* A_lo,
                         double* A_flux, cudaStream_t s);
constexpr int PROFILE_KERNELS = 5;   // refine, stencil, update, column, control
void profile_enable(bool on);
bool profile_on();
int profile_read(double* ms, long long* launches);
cudaError_t launch_backward(const Plan& p, void* ws, int scheme, const double* u,
                            const double* gradA, double* grad_coef, cudaStream_t s);

}  // namespace rve
