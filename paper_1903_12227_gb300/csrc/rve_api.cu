// rve_api.cu -- the C ABI of librve (declared in include/rve.h): argument
// validation, plan and workspace layout, and dispatch to the launchers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rve_ahom.cuh"
#include "rve_common.cuh"
#include "rve_internal.h"

namespace rve {

static uint64_t host_sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int ilog2(int v) {
    int p = 0;
    while ((1 << p) < v) ++p;
    return p;
}

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

constexpr int MIN_N = 32, MAX_N = 2048;
// Transform groups (2048/n rows each) per update block: the next group's q
// streams in while the current one transforms.
constexpr int U_GROUPS = 4;
constexpr size_t MAX_SMEM = 227 * 1024;

rve_solve_opts resolved_opts(const rve_solve_opts* o) {
    rve_solve_opts r;
    std::memset(&r, 0, sizeof(r));
    if (o) r = *o;
    if (r.max_iter <= 0) r.max_iter = 20000;
    if (!(r.tol > 0.0)) r.tol = 1e-10;
    if (!(r.inner_tol > 0.0)) r.inner_tol = 1e-4;
    if (r.check_every <= 0) r.check_every = 8;
    if (r.timeout_us <= 0) r.timeout_us = 2000000;
    return r;
}

// Tile geometry of one realization.  Row kernels use 256 threads, n/8 per
// row, so a transform group is 2048/n rows; an update block takes U_GROUPS
// groups (tU rows).  The stencil tile keeps tS + 2 padded rows in shared
// memory (see below).  Column blocks use blockC threads, n / col_seg_rows
// per column.
static void default_tiles(int n, size_t vb, int blockC, const rve_solve_opts& o, Tiles& t) {
    const size_t seq = (size_t)seq_stride(n);
    t.tU = std::min(n, U_GROUPS * (2048 / n));   // U_GROUPS transform groups per block
    // stencil tile: tS own rows + 2 halo rows, transformed G = 2048/n rows
    // at a time; choose tS + 2 a multiple of G (no idle row slots) with the
    // tile within ~72 KB (three blocks per SM), tS <= n.  Tiles need not
    // divide n: the last one is shorter.
    const int G = std::max(1, 2048 / n);
    auto smem_of = [&](int ts) {
        return (size_t)(ts + 2) * seq * vb + (size_t)(ts + 1) * (n / 32) * 4;
    };
    auto pick = [&](size_t budget) {
        int best = 1;
        for (int k = 1; k <= 64; ++k) {
            const int ts = std::min(k * G - 2, n);
            if (ts < 1) continue;
            if (smem_of(ts) > budget) break;
            best = ts;
            if (ts == n) break;
        }
        return best;
    };
    t.tS = pick(73728);
    if (t.tS < 4) t.tS = pick(112640);   // large grids: fewer, taller tiles (halo <= 50 %)
    int ts_tuned = 0, bc_tuned = 0;
    if (tuned_tiles(n, o.precision, o.path == RVE_PATH_PERSISTENT ? 1 : 0, &ts_tuned, &bc_tuned))
        t.tS = ts_tuned;
    t.tC = std::min(n, blockC / (n / col_seg_rows(n, (int)vb)));
    if (o.tile_rows > 0) t.tS = o.tile_rows;
    t.tS = std::min(t.tS, n);
}

rve_status make_plan(const rve_realization* r, int32_t batch, const rve_solve_opts* opts,
                     Plan& p, bool need_vectors) {
    if (!r || batch <= 0 || batch > (1 << 22)) return RVE_EINVAL;
    const rve_solve_opts o = resolved_opts(opts);
    if (o.scheme != RVE_Q1_CONSISTENT && o.scheme != RVE_Q1_LUMPED) return RVE_EINVAL;
    if (o.precision != RVE_FP64 && o.precision != RVE_MIXED) return RVE_EINVAL;
    if (o.path != RVE_PATH_FUSED && o.path != RVE_PATH_PLAIN && o.path != RVE_PATH_PERSISTENT)
        return RVE_EINVAL;
    if (o.path == RVE_PATH_PLAIN && o.precision != RVE_FP64) return RVE_EINVAL;
    if (o.flags != 0 || o.reserved != 0) return RVE_EINVAL;
    if (!std::isfinite(o.delta) || o.delta < 0.0 || !(o.tol < 1.0) || !(o.inner_tol < 1.0))
        return RVE_EINVAL;
    p.batch = batch;
    p.precision = o.precision;
    p.scheme = o.scheme;
    p.path = o.path;
    p.vbytes = (o.precision == RVE_MIXED) ? 8 : 16;
    p.desc.resize(batch);
    p.startS.assign(batch + 1, 0);
    p.startU.assign(batch + 1, 0);
    p.startC.assign(batch + 1, 0);
    p.startA.assign(batch + 1, 0);
    p.startA2.assign(batch + 1, 0);
    p.nodes = 0;
    p.words = 0;
    p.max_log2n = 5;
    p.smemS = p.smemU = p.smemC = 0;
    int64_t maxnb = 0;
    int maxn = 0;
    for (int b = 0; b < batch; ++b) {
        const int64_t nn = (int64_t)r[b].L * r[b].m0;
        if (nn > 0 && nn <= MAX_N) maxn = std::max(maxn, (int)nn);
    }
    // column blocks: a segment of up to 32 rows per thread in registers;
    // 128 threads for the mixed path (3 % faster than 256 and 13 % faster
    // than 512 on 512^2 grids, measured), 512 for FP64 (its shorter
    // segments need more threads)
    p.blockC = (p.vbytes == 8) ? 128 : 512;
    {
        int ts_tuned = 0, bc_tuned = 0;
        if (maxn > 0 && tuned_tiles(maxn, o.precision, o.path == RVE_PATH_PERSISTENT ? 1 : 0,
                                    &ts_tuned, &bc_tuned))
            p.blockC = std::min(512, std::max(32, bc_tuned));   // a loaded table may hold anything
    }
    if (o.path == RVE_PATH_PERSISTENT) p.blockC = 256;   // one block shape for all phases
    if (o.col_tile > 0 && o.path != RVE_PATH_PERSISTENT)
        p.blockC = std::min(512, std::max(32, o.col_tile));
    for (int b = 0; b < batch; ++b) {
        const rve_realization& x = r[b];
        if (x.L <= 0 || x.m0 <= 0) return RVE_EINVAL;
        const int64_t n64 = (int64_t)x.L * x.m0;
        if (n64 < MIN_N || n64 > MAX_N || !pow2((int)n64)) return RVE_EINVAL;
        const int n = (int)n64;
        if (x.incl_cells <= 0 || x.incl_cells > n || x.n_incl < 0) return RVE_EINVAL;
        if ((int64_t)x.n_incl * x.incl_cells > (1LL << 30)) return RVE_EINVAL;
        if (!std::isfinite(x.a_matrix) || !std::isfinite(x.a_incl) || !(x.a_matrix > 0.0) ||
            !(x.a_incl > 0.0))
            return RVE_EINVAL;
        Tiles t;
        default_tiles(n, p.vbytes, p.blockC, o, t);
        const int segs = n / col_seg_rows(n, (int)p.vbytes);   // threads per column
        if (t.tS < 1 || t.tS > n || t.tC < 1 || !pow2(t.tC) || n % t.tC ||
            t.tC * segs > p.blockC)
            return RVE_EINVAL;
        RDesc& d = p.desc[b];
        std::memset(&d, 0, sizeof(d));
        d.n = n;
        d.log2n = ilog2(n);
        d.L = x.L;
        d.s = x.incl_cells;
        d.n_incl = x.n_incl;
        d.tS = t.tS;
        d.tU = t.tU;
        d.tC = t.tC;
        d.node_off = p.nodes;
        d.word_off = p.words;
        d.a_matrix = x.a_matrix;
        d.a_incl = x.a_incl;
        d.h = 1.0 / (double)x.m0;
        d.c0 = 0.5 * (x.a_matrix + x.a_incl);
        d.inv_vol = 1.0 / ((double)x.L * (double)x.L);
        d.key = host_sm64_mix(x.seed + (x.index + 1) * 0x9E3779B97F4A7C15ull);
        p.nodes += (int64_t)n * n;
        p.words += ((int64_t)n * n) / 32;
        p.max_log2n = std::max(p.max_log2n, d.log2n);
        p.startS[b + 1] = p.startS[b] + (n + t.tS - 1) / t.tS;
        p.startU[b + 1] = p.startU[b] + n / t.tU;
        p.startC[b + 1] = p.startC[b] + n / t.tC;
        p.startA[b + 1] = p.startA[b] + (int32_t)(((int64_t)n * n) / 1024);
        p.startA2[b + 1] = p.startA2[b] + n / a_hom_strip_rows(n);
        maxnb = std::max<int64_t>(maxnb, ((int64_t)n * n) / 1024);
        const size_t vb = p.vbytes;
        const size_t seq = (size_t)seq_stride(n);
        p.smemS = std::max(p.smemS, (size_t)(t.tS + 2) * seq * vb + (size_t)(t.tS + 1) * (n / 32) * 4);
        // two sets of row buffers (one transform group each) for the update
        // pass's streaming; the preconditioner's row passes use the first
        p.smemU = std::max(p.smemU, (size_t)2 * std::min(t.tU, 2048 / n) * seq * vb);
        // segment end / start values (2 per column segment) and the
        // singular column's sums (2 per segment)
        p.smemC = std::max(p.smemC, (size_t)(2 * t.tC + 2) * segs * vb);
    }
    if (p.smemS > MAX_SMEM || p.smemU > MAX_SMEM || p.smemC > MAX_SMEM) return RVE_EINVAL;
    p.tilesS = p.startS[batch];
    p.tilesU = p.startU[batch];
    p.tilesC = p.startC[batch];
    p.tilesA = p.startA[batch];
    p.tilesA2 = p.startA2[batch];
    // workspace layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o2 = off;
        off = align_up(off + bytes);
        return o2;
    };
    const size_t tab = (size_t)2 << p.max_log2n;
    p.o_desc = take(sizeof(RDesc) * batch);
    p.o_startS = take(sizeof(int32_t) * (batch + 1));
    p.o_startU = take(sizeof(int32_t) * (batch + 1));
    p.o_startC = take(sizeof(int32_t) * (batch + 1));
    p.o_startA = take(sizeof(int32_t) * (batch + 1));
    p.o_startA2 = take(sizeof(int32_t) * (batch + 1));
    p.o_tw64 = take(sizeof(double2) * tab);
    p.o_tw32 = take(sizeof(float2) * tab);
    p.o_lap = take(sizeof(double) * tab);
    p.o_lap32 = take(sizeof(float) * tab);
    p.o_rho64 = take(sizeof(double) * tab);
    p.o_rho32 = take(sizeof(float) * tab);
    p.o_state = take(sizeof(RState) * batch);
    p.o_partS = take(sizeof(double) * 2 * (size_t)std::max<int64_t>(p.tilesS, maxnb));
    p.o_partU = take(sizeof(double) * 2 * (size_t)p.tilesU);
    p.o_partC = take(sizeof(double) * 2 * (size_t)p.tilesC);
    // 8 double-double sums per tile (FP64), or 8 doubles per strip (mixed)
    p.o_partA = take(sizeof(double) * 16 * (size_t)p.tilesA);
    p.o_ctl = take(sizeof(int32_t) * 64);
    p.o_uscal = take(sizeof(double) * 2 * (size_t)batch);
    p.o_cnt = take(sizeof(int32_t) * (size_t)batch);
    if (need_vectors) {
        const size_t vec = (size_t)p.nodes * p.vbytes;
        p.o_X = take(vec);
        p.o_R = take(vec);
        p.o_Q = take(vec);
        p.o_T = take(vec);
        p.o_P0 = take(vec);
        p.o_P1 = take(vec);
    }
    p.total = off;
    return RVE_OK;
}

static thread_local char g_last_error[256] = "";

rve_status note_error(const char* where, cudaError_t e) {
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", where, cudaGetErrorString(e));
    return RVE_ECUDA;
}

}  // namespace rve

using namespace rve;

static cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

extern "C" {

const char* rve_status_string(int32_t status) {
    switch (status) {
        case RVE_OK: return "RVE_OK";
        case RVE_EINVAL: return "RVE_EINVAL: invalid argument";
        case RVE_ENOCONV: return "RVE_ENOCONV: no convergence within max_iter";
        case RVE_ENAN: return "RVE_ENAN: NaN or Inf in a reduction";
        case RVE_ETIMEOUT: return "RVE_ETIMEOUT: a bounded device-side wait gave up";
        case RVE_ECUDA: return "RVE_ECUDA: a CUDA call failed";
        case RVE_ENOMEM: return "RVE_ENOMEM: workspace too small";
        case RVE_ESCRATCH:
            return "RVE_ESCRATCH: more nodes than the fixed scratch of rve_a_hom_noalloc holds "
                   "(RVE_NOALLOC_MAX_NODES)";
        default: return "unknown rve_status";
    }
}

int32_t rve_version(void) { return 100; }

const char* rve_last_error(void) { return g_last_error; }

int64_t rve_mask_words(const rve_realization* r, int32_t batch) {
    Plan p;
    if (make_plan(r, batch, nullptr, p, false) != RVE_OK) return -1;
    return p.words;
}

int64_t rve_nodes(const rve_realization* r, int32_t batch) {
    Plan p;
    if (make_plan(r, batch, nullptr, p, false) != RVE_OK) return -1;
    return p.nodes;
}

rve_status rve_gen_field(const rve_realization* r, int32_t batch, uint32_t* mask, void* stream) {
    Plan p;
    rve_status st = make_plan(r, batch, nullptr, p, false);
    if (st != RVE_OK) return st;
    if (!mask) return RVE_EINVAL;
    return launch_gen_field(p, nullptr, mask, as_stream(stream)) == cudaSuccess ? RVE_OK
                                                                               : RVE_ECUDA;
}

rve_status rve_coef_from_mask(const rve_realization* r, int32_t batch, const uint32_t* mask,
                              double* coef, void* stream) {
    Plan p;
    rve_status st = make_plan(r, batch, nullptr, p, false);
    if (st != RVE_OK) return st;
    if (!mask || !coef) return RVE_EINVAL;
    return launch_coef_from_mask(p, mask, coef, as_stream(stream)) == cudaSuccess ? RVE_OK
                                                                                 : RVE_ECUDA;
}

rve_status rve_rhs(const rve_realization* r, int32_t batch, const uint32_t* mask,
                   const double* coef, double* f, void* stream) {
    Plan p;
    rve_status st = make_plan(r, batch, nullptr, p, false);
    if (st != RVE_OK) return st;
    if (!f || (!mask && !coef)) return RVE_EINVAL;
    return launch_rhs(p, nullptr, mask, coef, f, as_stream(stream)) == cudaSuccess ? RVE_OK
                                                                                  : RVE_ECUDA;
}

rve_status rve_apply_stiffness(const rve_realization* r, int32_t batch, const uint32_t* mask,
                               const double* coef, int32_t scheme, int32_t precision,
                               const void* x, void* y, void* stream) {
    rve_solve_opts o;
    std::memset(&o, 0, sizeof(o));
    o.scheme = scheme;
    o.precision = precision;
    Plan p;
    rve_status st = make_plan(r, batch, &o, p, false);
    if (st != RVE_OK) return st;
    if (!x || !y || x == y || (!mask && !coef)) return RVE_EINVAL;
    return launch_stiffness(p, nullptr, mask, coef, scheme, precision, x, y, as_stream(stream)) ==
                   cudaSuccess
               ? RVE_OK
               : RVE_ECUDA;
}

size_t rve_workspace_size(const rve_realization* r, int32_t batch, const rve_solve_opts* opts) {
    Plan p;
    rve_solve_opts o = resolved_opts(opts);
    if (!opts) o.precision = RVE_FP64;   // large enough for either precision
    if (make_plan(r, batch, &o, p, true) != RVE_OK) return 0;
    return p.total;
}

rve_status rve_apply_precond(const rve_realization* r, int32_t batch, double delta,
                             int32_t precision, const void* x, void* y, void* ws,
                             size_t ws_bytes, void* stream) {
    rve_solve_opts o;
    std::memset(&o, 0, sizeof(o));
    o.precision = precision;
    o.delta = delta;
    Plan p;
    rve_status st = make_plan(r, batch, &o, p, true);
    if (st != RVE_OK) return st;
    if (!x || !y || !ws || ws_misaligned(ws)) return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    return launch_precond(p, ws, delta, precision, x, y, as_stream(stream)) == cudaSuccess
               ? RVE_OK
               : RVE_ECUDA;
}

static rve_status solve_any(const rve_realization* r, int32_t batch, const uint32_t* mask,
                            const double* coef, const double* f, const rve_solve_opts* opts,
                            double* u, rve_solve_info* info, void* ws, size_t ws_bytes,
                            void* stream) {
    const rve_solve_opts o = resolved_opts(opts);
    Plan p;
    rve_status st = make_plan(r, batch, &o, p, true);
    if (st != RVE_OK) return st;
    if (!u || !info || !ws || ws_misaligned(ws) || (!mask && !coef)) return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    if (o.path == RVE_PATH_PLAIN)
        return run_solve_plain(p, ws, mask, coef, o, u, info, as_stream(stream), f);
    if (o.path == RVE_PATH_PERSISTENT)
        return run_solve_persistent(p, ws, mask, coef, o, u, info, as_stream(stream), f);
    return run_solve_fused(p, ws, mask, coef, o, u, info, as_stream(stream), f);
}

rve_status rve_solve_correctors(const rve_realization* r, int32_t batch, const uint32_t* mask,
                                const double* coef, const rve_solve_opts* opts, double* u,
                                rve_solve_info* info, void* ws, size_t ws_bytes, void* stream) {
    return solve_any(r, batch, mask, coef, nullptr, opts, u, info, ws, ws_bytes, stream);
}

rve_status rve_solve_rhs(const rve_realization* r, int32_t batch, const uint32_t* mask,
                         const double* coef, const double* f, const rve_solve_opts* opts,
                         double* u, rve_solve_info* info, void* ws, size_t ws_bytes,
                         void* stream) {
    if (!f) return RVE_EINVAL;
    return solve_any(r, batch, mask, coef, f, opts, u, info, ws, ws_bytes, stream);
}

size_t rve_cheb_workspace_size(const rve_realization* r, int32_t batch) {
    rve_solve_opts o;
    std::memset(&o, 0, sizeof(o));
    Plan p;
    if (make_plan(r, batch, &o, p, false) != RVE_OK) return 0;
    return cheb_workspace_size(p);
}

rve_status rve_cheb_moments(const rve_realization* r, int32_t batch, const uint32_t* mask,
                            const double* coef, int32_t scheme, const double* v, int32_t K,
                            double lo, double hi, double* mu, void* ws, size_t ws_bytes,
                            void* stream) {
    rve_solve_opts o;
    std::memset(&o, 0, sizeof(o));
    o.scheme = scheme;
    Plan p;
    rve_status st = make_plan(r, batch, &o, p, false);
    if (st != RVE_OK) return st;
    if (!v || !mu || !ws || ws_misaligned(ws) || (!mask && !coef) || K < 2 || K > (1 << 20) || !std::isfinite(lo) ||
        !std::isfinite(hi) || !(hi > lo))
        return RVE_EINVAL;
    if (ws_bytes < cheb_workspace_size(p)) return RVE_ENOMEM;
    return launch_cheb(p, ws, mask, coef, scheme, v, K, lo, hi, mu, as_stream(stream)) ==
                   cudaSuccess
               ? RVE_OK
               : RVE_ECUDA;
}

rve_status rve_apply_mass(const rve_realization* r, int32_t batch, int32_t scheme,
                          const double* x, double* y, void* stream) {
    rve_solve_opts o;
    std::memset(&o, 0, sizeof(o));
    o.scheme = scheme;
    Plan p;
    rve_status st = make_plan(r, batch, &o, p, false);
    if (st != RVE_OK) return st;
    if (!x || !y || x == y) return RVE_EINVAL;
    return launch_mass(p, scheme, x, y, as_stream(stream)) == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status rve_a_hom(const rve_realization* r, int32_t batch, const uint32_t* mask,
                     const double* coef, int32_t scheme, int32_t precision, const double* u,
                     double* A, double* A_lo, double* A_flux, void* ws, size_t ws_bytes,
                     void* stream) {
    rve_solve_opts o;
    std::memset(&o, 0, sizeof(o));
    o.scheme = scheme;
    o.precision = precision;
    Plan p;
    rve_status st = make_plan(r, batch, &o, p, false);
    if (st != RVE_OK) return st;
    if (!u || !A || !ws || ws_misaligned(ws) || (!mask && !coef)) return RVE_EINVAL;
    if (A_lo && precision != RVE_FP64) return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    if (upload_plan(p, ws, as_stream(stream)) != RVE_OK) return RVE_ECUDA;
    return launch_a_hom(p, ws, mask, coef, scheme, precision, u, A, A_lo, A_flux,
                        as_stream(stream)) == cudaSuccess
               ? RVE_OK
               : RVE_ECUDA;
}

rve_status rve_a_hom_backward(const rve_realization* r, int32_t batch, int32_t scheme,
                              const double* u, const double* gradA, double* grad_coef,
                              void* stream) {
    rve_solve_opts o;
    std::memset(&o, 0, sizeof(o));
    o.scheme = scheme;
    Plan p;
    rve_status st = make_plan(r, batch, &o, p, false);
    if (st != RVE_OK) return st;
    if (!u || !gradA || !grad_coef) return RVE_EINVAL;
    return launch_backward(p, nullptr, scheme, u, gradA, grad_coef, as_stream(stream)) ==
                   cudaSuccess
               ? RVE_OK
               : RVE_ECUDA;
}

// Host pipeline: [mask | u | A | info | solver workspace] inside ws.
static size_t homog_layout(const Plan& p, size_t* o_mask, size_t* o_u, size_t* o_A,
                           size_t* o_info, size_t* o_ws) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o2 = off;
        off = align_up(off + bytes);
        return o2;
    };
    *o_mask = take(sizeof(uint32_t) * (size_t)p.words);
    *o_u = take(sizeof(double2) * (size_t)p.nodes);
    *o_A = take(sizeof(double) * 4 * (size_t)p.batch);
    *o_info = take(sizeof(rve_solve_info) * (size_t)p.batch);
    *o_ws = take(p.total);
    return off;
}

size_t rve_homogenize_workspace_size(const rve_realization* r, int32_t batch,
                                     const rve_solve_opts* opts) {
    Plan p;
    if (make_plan(r, batch, opts, p, true) != RVE_OK) return 0;
    size_t a, b, c, d, e;
    return homog_layout(p, &a, &b, &c, &d, &e);
}

rve_status rve_homogenize_host(const rve_realization* r_host, int32_t batch,
                               const rve_solve_opts* opts, double* A_host,
                               rve_solve_info* info_host, void* ws, size_t ws_bytes,
                               void* stream) {
    const rve_solve_opts o = resolved_opts(opts);
    Plan p;
    rve_status st = make_plan(r_host, batch, &o, p, true);
    if (st != RVE_OK) return st;
    if (!A_host || !ws || ws_misaligned(ws)) return RVE_EINVAL;
    size_t om, ou, oa, oi, ow;
    const size_t need = homog_layout(p, &om, &ou, &oa, &oi, &ow);
    if (ws_bytes < need) return RVE_ENOMEM;
    char* w = static_cast<char*>(ws);
    cudaStream_t s = as_stream(stream);
    uint32_t* mask = reinterpret_cast<uint32_t*>(w + om);
    double* u = reinterpret_cast<double*>(w + ou);
    double* A = reinterpret_cast<double*>(w + oa);
    rve_solve_info* info = reinterpret_cast<rve_solve_info*>(w + oi);
    if (launch_gen_field(p, nullptr, mask, s) != cudaSuccess) return RVE_ECUDA;
    note_launch();   // the mask clear
    st = rve_solve_correctors(r_host, batch, mask, nullptr, &o, u, info, w + ow, p.total, stream);
    if (st != RVE_OK) return st;
    st = rve_a_hom(r_host, batch, mask, nullptr, o.scheme, o.precision, u, A, nullptr, nullptr,
                   w + ow, p.total, stream);
    if (st != RVE_OK) return st;
    if (cudaMemcpyAsync(A_host, A, sizeof(double) * 4 * (size_t)batch, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return RVE_ECUDA;
    if (info_host &&
        cudaMemcpyAsync(info_host, info, sizeof(rve_solve_info) * (size_t)batch,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return RVE_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status rve_statistics(const double* A, int64_t N, double L, int32_t d, double* mean,
                          double* var, double* std12, double* stddiff, double* Q) {
    if (!A || N < 2 || !(L > 0.0) || d < 1) return RVE_EINVAL;
    double m[4] = {0, 0, 0, 0};
    for (int64_t k = 0; k < N; ++k)
        for (int e = 0; e < 4; ++e) m[e] += A[4 * k + e];
    for (int e = 0; e < 4; ++e) m[e] /= (double)N;
    double c[16];
    for (int e = 0; e < 16; ++e) c[e] = 0.0;
    double s12 = 0.0, sd = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        double dev[4];
        for (int e = 0; e < 4; ++e) dev[e] = A[4 * k + e] - m[e];
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) c[4 * i + j] += dev[i] * dev[j];
        s12 += A[4 * k + 1] * A[4 * k + 1];
        const double df = A[4 * k + 0] - A[4 * k + 3];
        sd += df * df;
    }
    const double Ld = std::pow(L, (double)d);
    for (int e = 0; e < 4; ++e) {
        if (mean) mean[e] = m[e];
        if (var) var[e] = c[5 * e] / (double)(N - 1);
    }
    if (Q)
        for (int e = 0; e < 16; ++e) Q[e] = Ld * c[e] / (double)(N - 1);
    if (std12) *std12 = std::sqrt(s12 / (double)N);
    if (stddiff) *stddiff = std::sqrt(sd / (double)N);
    return RVE_OK;
}

rve_status rve_dos_coefficients(const double* t, int32_t nt, int32_t K, double lo, double hi,
                                double eta, int32_t quad, double* c) {
    if (!t || !c || nt < 0 || K < 1 || K > (1 << 20) || !std::isfinite(lo) ||
        !std::isfinite(hi) || !(hi > lo) || !std::isfinite(eta) || !(eta > 0.0) || quad < 0)
        return RVE_EINVAL;
    const int q = quad > 0 ? quad : std::max(4 * K, 1024);
    const double pi = 3.14159265358979323846;
    const double norm = 1.0 / (std::sqrt(2.0 * pi) * eta);
    std::fill(c, c + (size_t)nt * K, 0.0);
    std::vector<double> g(nt), Tk(K);
    for (int j = 0; j < q; ++j) {
        const double th = pi * ((double)j + 0.5) / (double)q;
        const double x = std::cos(th);
        const double lam = 0.5 * (hi - lo) * x + 0.5 * (hi + lo);
        for (int i = 0; i < nt; ++i) {
            const double s = (t[i] - lam) / eta;
            g[i] = norm * std::exp(-0.5 * s * s);
        }
        // T_k(x) = cos(k th) by the three-term recurrence
        Tk[0] = 1.0;
        if (K > 1) Tk[1] = x;
        for (int k = 2; k < K; ++k) Tk[k] = 2.0 * x * Tk[k - 1] - Tk[k - 2];
        for (int i = 0; i < nt; ++i) {
            double* ci = c + (size_t)i * K;
            const double gi = g[i];
            for (int k = 0; k < K; ++k) ci[k] += gi * Tk[k];
        }
    }
    const double w = 2.0 / (double)q;
    for (int i = 0; i < nt; ++i) {
        double* ci = c + (size_t)i * K;
        for (int k = 0; k < K; ++k) ci[k] *= w;
        ci[0] *= 0.5;
    }
    return RVE_OK;
}

rve_status rve_dos_from_moments(const double* mu, int32_t K, double m, double lo, double hi,
                                double eta, const double* t, int32_t nt, double* phi) {
    if (!mu || !phi || !(m > 0.0)) return RVE_EINVAL;
    std::vector<double> c((size_t)std::max(nt, 0) * std::max(K, 1));
    const rve_status st = rve_dos_coefficients(t, nt, K, lo, hi, eta, 0, c.data());
    if (st != RVE_OK) return st;
    for (int i = 0; i < nt; ++i) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += c[(size_t)i * K + k] * mu[k];
        phi[i] = s / m;
    }
    return RVE_OK;
}

void rve_profile_enable(int32_t on) { profile_enable(on != 0); }

int32_t rve_profile_read(double* ms, int64_t* launches) {
    long long l[PROFILE_KERNELS];
    const int k = profile_read(ms, l);
    if (launches)
        for (int j = 0; j < k; ++j) launches[j] = (int64_t)l[j];
    return k;
}

int64_t rve_launch_count(void) { return (int64_t)g_launches.exchange(0); }

}  // extern "C"
