// rve_solver.cu -- preconditioned CG for the two corrector problems
// (Sec. 3.4 and 4.1), batched over realizations, on sm_103a.
//
// Preconditioner (Sec. 3.4): B = c0 A_Delta + delta I with A_Delta the
// periodic 5-point Laplacian.  On the torus B is diagonalised by the
// separable real Hartley transform H (x) H, (H (x) H)^2 = n^2 I, so
//   B^{-1} r = (H (x) H) diag(1 / (n^2 sigma)) (H (x) H) r,
//   sigma(k1,k2) = c0 (4 sin^2(pi k1/n) + 4 sin^2(pi k2/n)) + delta,
// the constant mode being dropped when delta = 0.  Each 1D Hartley pass
// transforms the two correctors at once: the complex DFT of (r_1 + i r_2)
// along the axis is split into H r_1 and H r_2 (see hartley_pair).  Since
// the transform is orthogonal up to n, r.z = (1/n^2) sum (H(x)H r)^2 / sigma
// is read off in the transform domain.
//
// Fused pipeline (one CG step = three passes over the vectors + a control
// kernel; both correctors of a realization travel together as a pair):
//   R  (REFINE steps only) r64 = f - A(u + s (x + alpha p)), the true
//      residual in double words (FP64 for the FP64 path), partial |r64|^2
//   S  z = inverse row-Hartley(zhat) on the tile + halo rows, p_new = z +
//      beta p_old, x += alpha_prev p_old (the solution update lags one
//      step), q = A p_new, partial p.q; the last block of a realization
//      forms alpha = rho / p.q
//   U  rt -= alpha H q (the residual kept as its row transform rt = H r),
//      partial |r|^2 = |rt|^2 / n (REFINE: u += s (x + alpha p), x = 0,
//      rt = H (r64 / |r64|))
//   C  periodic tridiagonal solve along every column of rt (the row
//      transform diagonalises the row factor of A_Delta), scaled, into
//      zhat; partial rho = r.z
//   K  per realization: reduce the partials in a fixed order, set alpha,
//      beta, convergence and the next phase.
// In MIXED precision x, rt, q, zhat, p are float2 and u is the double-word
// iterate: every REFINE step recomputes the true residual in double words
// and restarts the FP32 inner iteration on the scaled residual equation
// (iterative refinement).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "rve_colsolve.cuh"
#include "rve_common.cuh"
#include "rve_internal.h"

namespace rve {

// Control words (int32) in the workspace: [0] realizations done, then the
// persistent kernel's grid barrier.
enum { CTL_ARRIVE = 8, CTL_GEN = 9, CTL_ERR = 10, CTL_GROUPS = 11 };

struct Ctx {
    int batch;
    const RDesc* __restrict__ desc;
    const int32_t* __restrict__ startS;
    const int32_t* __restrict__ startU;
    const int32_t* __restrict__ startC;
    // written during a solve (by other blocks of the persistent launch too):
    // no __restrict__, so that every read is a coherent load
    RState* st;
    double* partS;
    double* partU;
    double* partC;
    double* uscal;     // [batch][2]: the update kernel's step scalars (see finish_S)
    int* tiles_done;   // [batch]: stencil/refine blocks finished this step
    Tables tb;
    CoefSrc cs;
    double2* u;
    void* X;
    void* R;
    void* Q;
    void* T;
    void* P0;
    void* P1;
    double tol, inner_tol, delta;
    int max_iter;
    int* ndone;
};

// ------------------------------------------------------------- tables --
// tw64[n + m] = exp(-2 pi i m / n), lap[n + m] = 4 sin^2(pi m / n) for every
// n = 2^p <= 2^maxlog, computed with sincospi/sinpi; rho[n + m] the column
// filter root for lambda = lap[n + m] and delta = 0 (1 for the singular
// column m = 0).
__global__ void k_tables(Tables out, int total) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < 2 || idx >= total) return;
    const int p = 31 - __clz(idx);
    const int n = 1 << p, m = idx - n;
    double sn, cs;
    sincospi(-2.0 * (double)m / (double)n, &sn, &cs);
    const_cast<double2*>(out.tw64)[idx] = make_double2(cs, sn);
    const_cast<float2*>(out.tw32)[idx] = make_float2((float)cs, (float)sn);
    const double s1 = sinpi((double)m / (double)n);
    const double lam = 4.0 * s1 * s1;
    const_cast<double*>(out.lap)[idx] = lam;
    const_cast<float*>(out.lap32)[idx] = (float)lam;
    const double rho = (m == 0) ? 1.0 : filter_root(lam);
    const_cast<double*>(out.rho64)[idx] = rho;
    const_cast<float*>(out.rho32)[idx] = (float)rho;
}

Tables tables_of(const Plan& p, const void* ws) {
    const char* w = static_cast<const char*>(ws);
    Tables tb;
    tb.tw64 = reinterpret_cast<const double2*>(w + p.o_tw64);
    tb.tw32 = reinterpret_cast<const float2*>(w + p.o_tw32);
    tb.lap = reinterpret_cast<const double*>(w + p.o_lap);
    tb.lap32 = reinterpret_cast<const float*>(w + p.o_lap32);
    tb.rho64 = reinterpret_cast<const double*>(w + p.o_rho64);
    tb.rho32 = reinterpret_cast<const float*>(w + p.o_rho32);
    return tb;
}

cudaError_t fill_tables(const Tables& tb, int max_log2n, cudaStream_t s) {
    const int total = 2 << max_log2n;
    k_tables<<<(total + 255) / 256, 256, 0, s>>>(tb, total);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tables(const Plan& p, void* ws, cudaStream_t s) {
    return fill_tables(tables_of(p, ws), p.max_log2n, s);
}

// ---------------------------------------------------------- row helpers --
// y + (ax, ay) * x componentwise; the scalars are already in the vector's
// type (no per-element conversion: on GB300 conversions from double run on
// the slow FP64 pipe).
template <typename V>
__device__ __forceinline__ V axpy2(V y, typename ScalarOf<V>::T ax, typename ScalarOf<V>::T ay, V x) {
    V r;
    r.x = y.x + ax * x.x;
    r.y = y.y + ay * x.y;
    return r;
}

template <typename V>
__device__ __forceinline__ int64_t node_of(const RDesc& d, int row, int col) {
    return d.node_off + ((int64_t)row << d.log2n) + col;
}

// Thread layout of the row kernels: T = n/8 threads per row, so
// blockDim/T rows per group; qq = row within the group, t = thread within
// row.  With a compile-time size (LOG2N > 0) T and the divisions fold.
template <int LOG2N>
struct RowLayout {
    Sz<LOG2N> z;
    int qq, t, G;
    __device__ __forceinline__ explicit RowLayout(int log2n) : z(log2n) {
        G = blockDim.x / z.T;
        qq = threadIdx.x / z.T;
        t = threadIdx.x - qq * z.T;
    }
};

template <int LOG2N>
__device__ __forceinline__ int64_t node_at(const RDesc& d, const Sz<LOG2N>& z, int row, int col) {
    return d.node_off + ((int64_t)row << z.log2n) + col;
}

// Calls body.template operator()<LOG2N>() with the realization's size as a
// compile-time constant (n = 32 .. 2048).
template <typename F>
__device__ __forceinline__ void dispatch_size(int log2n, F&& body) {
    switch (log2n) {
        case 5: body.template operator()<5>(); break;
        case 6: body.template operator()<6>(); break;
        case 7: body.template operator()<7>(); break;
        case 8: body.template operator()<8>(); break;
        case 9: body.template operator()<9>(); break;
        case 10: body.template operator()<10>(); break;
        default: body.template operator()<11>(); break;
    }
}

// ----------------------------------------------------------- S kernel --
template <typename V>
__device__ __forceinline__ double2 refine_w(const Ctx& c, const RDesc& d, const RState& s, int i,
                                            int j, const V* P) {
    const int64_t node = d.node_off + ((int64_t)(i & (d.n - 1)) << d.log2n) + (j & (d.n - 1));
    const double2 uu = c.u[node];
    const double2 xx = to_d2(static_cast<const V*>(c.X)[node]);
    const double2 pp = to_d2(P[node]);
    return make_double2(uu.x + s.s[0] * (xx.x + s.alpha[0] * pp.x),
                        uu.y + s.s[1] * (xx.y + s.alpha[1] * pp.y));
}

// Cell value from the shared-memory mask rows of the tile (cell rows
// r0-1 .. r0+TR-1 stored at mrow 0 .. TR) or from the coefficient array.
template <typename T>
struct TileCoef {
    const uint32_t* mrows;   // shared, (TR+1) x (n/32) words, or null
    int wpr;                 // words per row
    T a_incl, a_matrix;      // the two values in the arithmetic type
    __device__ __forceinline__ T cell(const CoefSrc& cs, const RDesc& d, int mrow, int c1,
                                      int c2) const {
        if (mrows) {
            const uint32_t w = mrows[mrow * wpr + (c2 >> 5)];
            return ((w >> (c2 & 31)) & 1u) ? a_incl : a_matrix;
        }
        return (T)cs.cell(d, c1 & (d.n - 1), c2);
    }
};

// Called by every stencil/refine block after it wrote its partial sums of
// realization b.  The block that finishes last (atomic tile counter) sums
// all of them in tile order -- deterministic whichever block is last -- and
// stores the update kernel's scalars: in ITER alpha = rho / p.q (0 for a
// frozen corrector), in REFINE 1/|r64| (0 once the corrector meets the
// tolerance).  The update kernel then starts without any FP64 work.
__device__ void finish_S(const Ctx& c, int b, const RState& s, bool refine) {
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int nt = c.startS[b + 1] - c.startS[b];
        last = (atomicAdd(c.tiles_done + b, 1) == nt - 1);
    }
    __syncthreads();
    if (!last) return;
    if (threadIdx.x < 32) {
        __threadfence();
        const int t0 = c.startS[b], nt = c.startS[b + 1] - t0;
        const double sx = warp_sum_array(c.partS + 2 * (int64_t)t0, nt, 2);
        const double sy = warp_sum_array(c.partS + 2 * (int64_t)t0 + 1, nt, 2);
        if (threadIdx.x == 0) {
            double a0, a1;
            if (!refine) {
                a0 = s.active[0] ? s.rho[0] / sx : 0.0;
                a1 = s.active[1] ? s.rho[1] / sy : 0.0;
            } else {
                const double nx = sqrt(sx), ny = sqrt(sy);
                const bool first = (s.refinements == 0);
                const bool cx = first ? (nx == 0.0) : (nx <= c.tol * s.fnorm[0]);
                const bool cy = first ? (ny == 0.0) : (ny <= c.tol * s.fnorm[1]);
                a0 = cx ? 0.0 : 1.0 / nx;
                a1 = cy ? 0.0 : 1.0 / ny;
            }
            c.uscal[2 * b] = a0;
            c.uscal[2 * b + 1] = a1;
            c.tiles_done[b] = 0;   // ready for the next step
        }
    }
}

// Mixed path: the FP64-accurate iterate lives in the caller's u buffer as a
// double word per node and corrector (float4 = hi.x, hi.y, lo.x, lo.y) until
// the solve ends (k_u_finalize).  The refine and update kernels both form
// the new iterate w = u + s (x + alpha p) with this function -- correction
// in FP32, added to u as a double word -- so that the residual computed for
// w belongs to exactly the w that is stored.
struct DWScal { float sx, sy, ax, ay; };
__device__ __forceinline__ float4 w_new(float4 u, float2 x, float2 p, const DWScal& k) {
    const float dx = __fmul_rn(k.sx, __fmaf_rn(k.ax, p.x, x.x));
    const float dy = __fmul_rn(k.sy, __fmaf_rn(k.ay, p.y, x.y));
    const dword wx = dw_add(dword{u.x, u.z}, dx);
    const dword wy = dw_add(dword{u.y, u.w}, dy);
    return make_float4(wx.hi, wy.hi, wx.lo, wy.lo);
}


// REFINE step of the mixed path: r = f - A w for the tile's rows with
// w = u + s (x + alpha p), in double-word arithmetic on the FP32 pipe (no
// FP64 per node).  The stiffness and the right-hand side are scaled by
// K = 6 (consistent) resp. 2 (lumped) so that every stencil weight is an
// integer multiple of a cell value: K A has centre 2 K w0 (sum of the four
// cells), edges -(sum of the two shared cells), corners -2 K w1 (shared
// cell), and K f_1 = (K h/2)(a_0m + a_00 - a_mm - a_m0).  r_K = K f - K A w
// is accumulated as a compensated dot product, so its absolute error is
// O(eps_32^2) times the size of the stencil terms -- far below the outer
// tolerance -- and r = r_K / K is rounded to FP32 (the inner iteration's
// type).  Each thread walks down one column with a 3 x 3 window of w.
// EXACT: both cell values are integers of magnitude <= 2^20 (the paper's
// two-valued coefficients 1 and the contrast), so every cell sum and scaled
// weight below is exact in one float; the weights are then floats (CW)
// instead of double words, with the same values and so the same results.
template <int SCHEME, bool EXACT>
__device__ void refine_tile_dw(const Ctx& c, int tile, int b, const RState& s, const RDesc& d) {
    typedef std::conditional_t<EXACT, float, dword> CW;
    __shared__ double red[64];
    __shared__ float sc[9];
    const int n = d.n;
    const int r0 = (tile - c.startS[b]) * d.tS;
    const int rows = min(d.tS, n - r0);   // the last tile may be shorter
    if (threadIdx.x == 0) {
        sc[0] = (float)s.s[0];
        sc[1] = (float)s.s[1];
        sc[2] = (float)s.alpha[0];
        sc[3] = (float)s.alpha[1];
        const dword ai = dw_of(d.a_incl), am = dw_of(d.a_matrix);
        sc[4] = ai.hi; sc[5] = ai.lo; sc[6] = am.hi; sc[7] = am.lo;
        sc[8] = (float)d.h;   // 1/m0, a power of two: exact
    }
    __syncthreads();
    const DWScal k{sc[0], sc[1], sc[2], sc[3]};
    const dword aI{sc[4], sc[5]}, aM{sc[6], sc[7]};
    const bool first = (s.refinements == 0);   // u = x = p = 0: r = f
    constexpr float CEN = SCHEME == 0 ? 4.f : 2.f;      // 2 K w0
    constexpr float COR = SCHEME == 0 ? 2.f : 0.f;      // 2 K w1
    constexpr float KH = SCHEME == 0 ? 3.f : 1.f;       // K / 2
    constexpr float INVK = SCHEME == 0 ? (1.f / 6.f) : 0.5f;
    const float kh2 = KH * sc[8];   // K h / 2: exact
    const float4* U = reinterpret_cast<const float4*>(c.u);
    const float2* X = static_cast<const float2*>(c.X);
    const float2* P = static_cast<const float2*>(s.parity ? c.P1 : c.P0);
    float2* Q = static_cast<float2*>(c.Q);
    auto wat = [&](int i, int j) -> float4 {
        if (first) return make_float4(0.f, 0.f, 0.f, 0.f);
        const int64_t node = d.node_off + ((int64_t)(i & (n - 1)) << d.log2n) + (j & (n - 1));
        return w_new(U[node], X[node], P[node], k);
    };
    auto cell = [&](int i, int j) -> CW {
        const int64_t ci = ((int64_t)(i & (n - 1)) << d.log2n) + (j & (n - 1));
        if constexpr (EXACT) {   // mask only (no explicit coefficients)
            const uint32_t w = __ldg(c.cs.mask + d.word_off + (ci >> 5));
            return ((w >> (ci & 31)) & 1u) ? aI.hi : aM.hi;
        } else {
            if (c.cs.coef) return dw_of(__ldg(c.cs.coef + d.node_off + ci));
            const uint32_t w = __ldg(c.cs.mask + d.word_off + (ci >> 5));
            return ((w >> (ci & 31)) & 1u) ? aI : aM;
        }
    };
    // cell-weight arithmetic in CW: exact float operations, or double words
    auto wadd = [](CW x, CW y) -> CW {
        if constexpr (EXACT) return __fadd_rn(x, y); else return dw_add(x, y);
    };
    auto wsub = [](CW x, CW y) -> CW {
        if constexpr (EXACT) return __fsub_rn(x, y); else return dw_add(x, dw_neg(y));
    };
    auto wscale2 = [](CW x, float p2) -> CW {
        if constexpr (EXACT) return x * p2; else return dw_scale2(x, p2);
    };
    auto wmulf = [](CW x, float f) -> dword {
        if constexpr (EXACT) {
            const float p = __fmul_rn(x, f);
            return {p, __fmaf_rn(x, f, -p)};
        } else {
            return dw_mulf(x, f);
        }
    };
    dword nx{0.f, 0.f}, ny{0.f, 0.f};   // |r|^2, double-word per thread
    if (first) {   // u = x = p = 0: r = f, the same arithmetic without the zero terms
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            CW cmm = cell(r0 - 1, j - 1), cm0 = cell(r0 - 1, j);
            for (int q = 0; q < rows; ++q) {
                const int i = r0 + q;
                const CW c0m = cell(i, j - 1), c00 = cell(i, j);
                dword kfx, kfy;   // K f
                if (c.cs.f) {
                    const double2 fl = c.cs.f[d.node_off + ((int64_t)i << d.log2n) + j];
                    kfx = dw_mulf(dw_split(fl.x), 2.f * KH);
                    kfy = dw_mulf(dw_split(fl.y), 2.f * KH);
                } else {
                    const CW top = wadd(cmm, cm0), bot = wadd(c0m, c00);
                    const CW lft = wadd(cmm, c0m), rgt = wadd(cm0, c00);
                    kfx = wmulf(wsub(bot, top), kh2);
                    kfy = wmulf(wsub(rgt, lft), kh2);
                }
                const DotDW rx(kfx), ry(kfy);
                const float2 r = make_float2(rx.value() * INVK, ry.value() * INVK);
                Q[d.node_off + ((int64_t)i << d.log2n) + j] = r;
                nx = dw_add(nx, r.x * r.x);
                ny = dw_add(ny, r.y * r.y);
                cmm = c0m; cm0 = c00;
            }
        }
    }
    for (int j = first ? n : threadIdx.x; j < n; j += blockDim.x) {
        float4 a0 = wat(r0 - 1, j - 1), a1 = wat(r0 - 1, j), a2 = wat(r0 - 1, j + 1);
        float4 b0 = wat(r0, j - 1), b1 = wat(r0, j), b2 = wat(r0, j + 1);
        CW cmm = cell(r0 - 1, j - 1), cm0 = cell(r0 - 1, j);
        for (int q = 0; q < rows; ++q) {
            const int i = r0 + q;
            const float4 e0 = wat(i + 1, j - 1), e1 = wat(i + 1, j), e2 = wat(i + 1, j + 1);
            const CW c0m = cell(i, j - 1), c00 = cell(i, j);
            const CW top = wadd(cmm, cm0);   // cells shared with (i-1, j)
            const CW bot = wadd(c0m, c00);   // with (i+1, j)
            const CW lft = wadd(cmm, c0m);   // with (i, j-1)
            const CW rgt = wadd(cm0, c00);   // with (i, j+1)
            const CW cen = wscale2(wadd(top, bot), -CEN);
            dword kfx, kfy;   // K f
            if (c.cs.f) {
                const double2 fl = c.cs.f[d.node_off + ((int64_t)i << d.log2n) + j];
                kfx = dw_mulf(dw_split(fl.x), 2.f * KH);
                kfy = dw_mulf(dw_split(fl.y), 2.f * KH);
            } else {
                kfx = wmulf(wsub(bot, top), kh2);
                kfy = wmulf(wsub(rgt, lft), kh2);
            }
            DotDW rx(kfx), ry(kfy);
            rx.add(cen, b1.x, b1.z); ry.add(cen, b1.y, b1.w);
            rx.add(top, a1.x, a1.z); ry.add(top, a1.y, a1.w);
            rx.add(bot, e1.x, e1.z); ry.add(bot, e1.y, e1.w);
            rx.add(lft, b0.x, b0.z); ry.add(lft, b0.y, b0.w);
            rx.add(rgt, b2.x, b2.z); ry.add(rgt, b2.y, b2.w);
            if (COR != 0.f) {
                const CW kmm = wscale2(cmm, COR), km0 = wscale2(cm0, COR);
                const CW k0m = wscale2(c0m, COR), k00 = wscale2(c00, COR);
                rx.add(kmm, a0.x, a0.z); ry.add(kmm, a0.y, a0.w);
                rx.add(km0, a2.x, a2.z); ry.add(km0, a2.y, a2.w);
                rx.add(k0m, e0.x, e0.z); ry.add(k0m, e0.y, e0.w);
                rx.add(k00, e2.x, e2.z); ry.add(k00, e2.y, e2.w);
            }
            const float2 r = make_float2(rx.value() * INVK, ry.value() * INVK);
            Q[d.node_off + ((int64_t)i << d.log2n) + j] = r;
            nx = dw_add(nx, r.x * r.x);
            ny = dw_add(ny, r.y * r.y);
            a0 = b0; a1 = b1; a2 = b2;
            b0 = e0; b1 = e1; b2 = e2;
            cmm = c0m; cm0 = c00;
        }
    }
    DotAcc<float> ax, ay;
    ax.hi = nx.hi; ax.lo = nx.lo;
    ay.hi = ny.hi; ay.lo = ny.lo;
    double sx = 0.0, sy = 0.0;
    block_sum2(ax, ay, red, sx, sy);
    if (threadIdx.x == 0) {
        c.partS[2 * (int64_t)tile] = sx;
        c.partS[2 * (int64_t)tile + 1] = sy;
    }
    finish_S(c, b, s, true);
}

// REFINE step: r64 = f - A(u + s (x + alpha p)) for the tile's rows, stored
// (rounded to the vector type) in q, partial |r64|^2 into partS -- in FP64
// for the FP64 path, in double words for the mixed path (refine_tile_dw).
// Launched every step next to k_fused_S; blocks of realizations that are
// not refining return at once.
template <int SCHEME>
__device__ void refine_tile_fp64(const Ctx& c, int tile, int b, const RState& s, const RDesc& d) {
    typedef double2 V;
    __shared__ double red[64];
    const int n = d.n;
    const int r0 = (tile - c.startS[b]) * d.tS;
    const int rows = min(d.tS, n - r0);   // the last tile may be shorter
    const V* Pold = static_cast<const V*>(s.parity ? c.P1 : c.P0);
    V* Q = static_cast<V*>(c.Q);
    const bool first = (s.refinements == 0);   // u = x = p = 0: r = f
    DotAcc<double> a64x, a64y;   // exact FP64 |r64|^2
    for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
        const int i = r0 + (idx >> d.log2n), j = idx & (n - 1);
        const Cells4 a = cells_at(c.cs, d, i, j);
        const double2 f = load_at(c.cs, d, ((int64_t)i << d.log2n) + j, a);
        double2 Aw = make_double2(0.0, 0.0);
        if (!first)
            Aw = stencil_apply<SCHEME, double2>(
                a, refine_w(c, d, s, i - 1, j - 1, Pold), refine_w(c, d, s, i - 1, j, Pold),
                refine_w(c, d, s, i - 1, j + 1, Pold), refine_w(c, d, s, i, j - 1, Pold),
                refine_w(c, d, s, i, j, Pold), refine_w(c, d, s, i, j + 1, Pold),
                refine_w(c, d, s, i + 1, j - 1, Pold), refine_w(c, d, s, i + 1, j, Pold),
                refine_w(c, d, s, i + 1, j + 1, Pold));
        const double2 r64 = make_double2(f.x - Aw.x, f.y - Aw.y);
        Q[node_of<V>(d, i, j)] = from_d2<V>(r64);
        a64x.add(r64.x, r64.x);
        a64y.add(r64.y, r64.y);
    }
    double sx = 0.0, sy = 0.0;
    block_sum2(a64x, a64y, red, sx, sy);
    if (threadIdx.x == 0) {
        c.partS[2 * (int64_t)tile] = sx;
        c.partS[2 * (int64_t)tile + 1] = sy;
    }
    finish_S(c, b, s, true);
}

template <typename V, int SCHEME>
__device__ void fused_R_tile(const Ctx& c, int tile) {
    const int b = find_real(c.startS, c.batch, tile);
    const RState& s = c.st[b];
    if (s.phase != PH_REFINE) return;
    const RDesc d = c.desc[b];
    if constexpr (sizeof(V) == 8) {
        // integer cell values of magnitude <= 2^20: sums of up to four of
        // them, scaled by 2, 4 or 3 h (h a power of two), stay below 2^24
        auto small_int = [](double a) { return a == floor(a) && fabs(a) <= 1048576.0; };
        if (!c.cs.coef && small_int(d.a_incl) && small_int(d.a_matrix))
            refine_tile_dw<SCHEME, true>(c, tile, b, s, d);
        else
            refine_tile_dw<SCHEME, false>(c, tile, b, s, d);
    } else
        refine_tile_fp64<SCHEME>(c, tile, b, s, d);
}

// ITER step: inverse row Hartley of t on the tile + halo rows (z),
// p_new = z + beta p_old, x += alpha p_old (own rows), q = A p_new, p.q.
template <typename V, int SCHEME, int LOG2N>
__device__ __forceinline__ void fused_S_body(const Ctx& c, int tile, int b, const RState& s,
                                             const RDesc& d, double* red,
                                             typename ScalarOf<V>::T* bsc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Sz<LOG2N> z(d.log2n);
    const int n = z.n;
    const int r0 = (tile - c.startS[b]) * d.tS;
    const int TR = min(d.tS, n - r0);   // own rows (the last tile may be shorter)
    const V* Pold = static_cast<const V*>(s.parity ? c.P1 : c.P0);
    V* Pnew = static_cast<V*>(s.parity ? c.P0 : c.P1);
    V* X = static_cast<V*>(c.X);
    V* Q = static_cast<V*>(c.Q);
    typedef typename ScalarOf<V>::T T;

    // ---- ITER ----
    // p_old (own and halo rows) and x (own rows) are read only after the
    // rows' transforms, t group by group: one thread per row asks for them
    // in L2 now, so those loads and copies wait on L2 instead of DRAM
    {
        const unsigned rb = (unsigned)(n * sizeof(V));
        const int k = threadIdx.x;
        if (k < TR + 2) prefetch_l2(Pold + node_at(d, z, (r0 - 1 + k) & (n - 1), 0), rb);
        else if (k >= 64 && k < 64 + TR) prefetch_l2(X + node_at(d, z, r0 + k - 64, 0), rb);
        else if (k >= 128 && k < 128 + TR + 2)
            prefetch_l2(static_cast<const V*>(c.T) + node_at(d, z, (r0 - 1 + k - 128) & (n - 1), 0), rb);
    }
    // scalars of this step, converted once (thread 0) to the vector type
    if (threadIdx.x == 0) {
        bsc[0] = (T)s.beta[0];
        bsc[1] = (T)s.beta[1];
        bsc[2] = (T)s.alpha[0];
        bsc[3] = (T)s.alpha[1];
        bsc[4] = (T)d.a_incl;
        bsc[5] = (T)d.a_matrix;
    }
    const int SEQ = seq_stride(n);
    V* Pt = reinterpret_cast<V*>(smem_raw);            // (TR+2) padded rows
    uint32_t* mrows = reinterpret_cast<uint32_t*>(Pt + (TR + 2) * SEQ);
    const int wpr = n >> 5;
    if (!c.cs.coef) {
        for (int w = threadIdx.x; w < (TR + 1) * wpr; w += blockDim.x) {
            const int mr = w / wpr, col = w - mr * wpr;
            const int row = (r0 - 1 + mr) & (n - 1);
            mrows[w] = __ldg(c.cs.mask + d.word_off + (((int64_t)row << z.log2n) >> 5) + col);
        }
    }
    __syncthreads();
    const TileCoef<T> tc{c.cs.coef ? nullptr : mrows, wpr, bsc[4], bsc[5]};
    const RowLayout<LOG2N> L(z.log2n);
    const T bx = bsc[0], by = bsc[1];
    const T alx = bsc[2], aly = bsc[3];
    const V* Tin = static_cast<const V*>(c.T);
    const V* tw = twiddles<V>(c.tb, n);
    // t of the rows of a transform group goes straight into the rows' own
    // shared slots by asynchronous copies (no registers held), one group
    // ahead: the copies of group g+1 are in flight while group g transforms
    // and while the stencil runs on the rows group g completed
    auto prefetch = [&](int g0) {
        const int q = g0 + L.qq;
        if (g0 < TR + 2 && q < TR + 2) {
            const int row = (r0 - 1 + q) & (n - 1);
            V* buf = Pt + q * SEQ;
#pragma unroll
            for (int m = 0; m < 8; ++m)
                cp_async_v(buf + pidx(L.t + m * L.z.T), Tin + node_at(d, z, row, L.t + m * L.z.T));
        }
        cp_async_commit();   // an empty group past the last: uniform counting
    };
    prefetch(0);
    // q = A p on the own rows, once every row of the tile is transformed:
    // each thread walks down a column keeping the 3 x 3 neighbourhood (and
    // the two cell columns) in registers, so a node costs three shared loads
    // and two cell lookups.
    DotAcc<T> ax, ay;   // p.q
    // a thread walks down two columns j and j + 256 at once (n >= 512, the
    // kernel runs 256 threads): two independent chains of shared loads and
    // multiply-adds per row
    struct Win {
        V u0, u1, u2, m0, m1, m2;
        T cmm, cm0;
        int j, pm, p0, pp;
    };
    auto win_start = [&](Win& w, int j) {
        w.j = j;
        const int jm = (j - 1) & (n - 1), jp = (j + 1) & (n - 1);
        w.pm = pidx(jm); w.p0 = pidx(j); w.pp = pidx(jp);
        w.u0 = Pt[w.pm]; w.u1 = Pt[w.p0]; w.u2 = Pt[w.pp];                    // slot 0
        w.m0 = Pt[SEQ + w.pm]; w.m1 = Pt[SEQ + w.p0]; w.m2 = Pt[SEQ + w.pp];  // slot 1
        w.cmm = tc.cell(c.cs, d, 0, r0 - 1, jm);
        w.cm0 = tc.cell(c.cs, d, 0, r0 - 1, j);
    };
    auto win_step = [&](Win& w, int q) {   // own slot q: node row r0 + q - 1
        const V* dn = Pt + (q + 1) * SEQ;
        const V d0 = dn[w.pm], d1 = dn[w.p0], d2 = dn[w.pp];
        const int jm = (w.j - 1) & (n - 1);
        const T c0m = tc.cell(c.cs, d, q, r0 + q - 1, jm);
        const T c00 = tc.cell(c.cs, d, q, r0 + q - 1, w.j);
        CellsT<T> a;
        a.mm = w.cmm;
        a.m0 = w.cm0;
        a.z0m = c0m;
        a.z00 = c00;
        const V qv = stencil_apply<SCHEME, V>(a, w.u0, w.u1, w.u2, w.m0, w.m1, w.m2, d0, d1, d2);
        Q[node_at(d, z, r0 + q - 1, w.j)] = qv;
        ax.add(w.m1.x, qv.x);
        ay.add(w.m1.y, qv.y);
        w.u0 = w.m0; w.u1 = w.m1; w.u2 = w.m2;
        w.m0 = d0; w.m1 = d1; w.m2 = d2;
        w.cmm = c0m; w.cm0 = c00;
    };
    auto stencil_rows = [&]() {
        constexpr bool TWO = LOG2N >= 9;   // n >= 512 = 2 x 256 threads
        for (int j = threadIdx.x; j < n; j += TWO ? 512 : 256) {
            Win wa, wb;
            win_start(wa, j);
            if (TWO) win_start(wb, j + 256);
            for (int q = 1; q <= TR; ++q) {
                win_step(wa, q);
                if (TWO) win_step(wb, q);
            }
        }
    };
    // every row's transform is done by its own team of n/8 threads: the
    // barriers of the group loop are the team's, so the teams of a block
    // drift independently (one waits on its loads while another transforms)
    const TeamBar team(L.qq, L.z.T);
    for (int g0 = 0; g0 < TR + 2; g0 += L.G) {
        const int q = g0 + L.qq;
        const bool active = q < TR + 2;
        const int row = (r0 - 1 + q) & (n - 1);
        const bool own = active && q >= 1 && q <= TR;
        prefetch(g0 + L.G);
        cp_async_wait<1>();   // this thread's copies of slot q have landed
        team();               // ... and those of the whole team
        V* buf = Pt + (active ? q : 0) * SEQ;
        V v[8];
        if (active) {
#pragma unroll
            for (int m = 0; m < 8; ++m) v[m] = buf[pidx(L.t + m * L.z.T)];
        }
        fft_reg<FFT_TO_BOTH, LOG2N>(v, buf, z.log2n, L.t, tw, active, team);
        V pn[8];
        if (active) {
            // p_new = z + beta p_old; own rows: x += alpha p_old (the lagged
            // solution update) and p_new out.  In two halves of four, the
            // global loads of a half before its stores (the compiler cannot
            // prove Pold, Pnew and X distinct)
#pragma unroll
            for (int h = 0; h < 8; h += 4) {
                V po[4], xo[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) po[m] = Pold[node_at(d, z, row, L.t + (h + m) * L.z.T)];
                if (own) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) xo[m] = X[node_at(d, z, row, L.t + (h + m) * L.z.T)];
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int k = L.t + (h + m) * L.z.T;
                    const V zz = hartley_pair(v[h + m], buf[pidx((n - k) & (n - 1))]);
                    pn[h + m] = axpy2(zz, bx, by, po[m]);
                }
                if (own) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int64_t node = node_at(d, z, row, L.t + (h + m) * L.z.T);
                        Pnew[node] = pn[h + m];
                        X[node] = axpy2(xo[m], alx, aly, po[m]);
                    }
                }
            }
        }
        team();   // the team's mirror reads of this row are done
        if (active) {
#pragma unroll
            for (int m = 0; m < 8; ++m) buf[pidx(L.t + m * L.z.T)] = pn[m];
        }
    }
    cp_async_wait<0>();
    __syncthreads();   // p_new of the whole tile visible
    stencil_rows();
    double sx = 0.0, sy = 0.0;
    block_sum2(ax, ay, red, sx, sy);
    if (threadIdx.x == 0) {
        c.partS[2 * (int64_t)tile] = sx;
        c.partS[2 * (int64_t)tile + 1] = sy;
    }
    finish_S(c, b, s, false);
}

template <typename V, int SCHEME>
__device__ void fused_S_tile(const Ctx& c, int tile) {
    __shared__ double red[64];   // block_sum2 scratch
    __shared__ typename ScalarOf<V>::T bsc[6];
    const int b = find_real(c.startS, c.batch, tile);
    const RState& s = c.st[b];
    if (s.phase != PH_ITER) return;
    const RDesc d = c.desc[b];
    dispatch_size(d.log2n, [&]<int LG>() { fused_S_body<V, SCHEME, LG>(c, tile, b, s, d, red, bsc); });
}

// ----------------------------------------------------------- U kernel --
// Row Hartley pass of the rows held in registers (v[m] = row value at
// t + m T) into `out` (global), through the row's shared buffer.
template <typename V, int LOG2N, typename Out>
__device__ __forceinline__ void row_hartley_out(V (&v)[8], V* buf, const Sz<LOG2N>& z, int row,
                                                int t, const V* tw, bool active, Out&& out) {
    fft_reg<FFT_TO_BOTH, LOG2N>(v, buf, z.log2n, t, tw, active);
    if (active) {
        const int n = z.n;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int k = t + m * z.T;
            out(row, k, hartley_pair(v[m], buf[pidx((n - k) & (n - 1))]));
        }
    }
}

template <typename V, int LOG2N>
__device__ __forceinline__ void row_hartley_store(V (&v)[8], V* buf, const RDesc& d,
                                                  const Sz<LOG2N>& z, int row, int t,
                                                  const V* tw, bool active,
                                                  V* __restrict__ out) {
    row_hartley_out<V, LOG2N>(v, buf, z, row, t, tw, active,
                              [&](int r, int k, V val) { out[node_at(d, z, r, k)] = val; });
}

// The update kernel: tU rows per block, in transform groups of L.G rows
// (n/8 threads per row).  The residual is kept in the row-Hartley domain,
// rt = H r (H the unnormalised Hartley transform along rows, H H = n I):
// that is exactly what the column pass consumes, so the update writes it
// once instead of writing r and t = H r.
//   ITER    rt -= alpha H q  (H q by the row transform of q), |r|^2 = |rt|^2 / n;
//   REFINE  u = w (the new iterate), x = 0, r = r64 / |r64| (|r|^2 from r),
//           rt = H r.
// ITER streams: q of the next group arrives by asynchronous copies into the
// other of two row buffers while the current group transforms, and rt of a
// group is loaded before its transform.
template <typename V, int LOG2N>
__device__ __forceinline__ void fused_U_body(const Ctx& c, int blk, int b, const RState& s,
                                             const RDesc& d, double* red,
                                             typename ScalarOf<V>::T* usc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int phase = s.phase;
    const RowLayout<LOG2N> L(d.log2n);
    const Sz<LOG2N>& z = L.z;
    const int row0 = (blk - c.startU[b]) * d.tU;
    const int ng = (d.tU + L.G - 1) / L.G;   // transform groups of this block
    typedef typename ScalarOf<V>::T T;
    V* Rt = static_cast<V*>(c.R);
    V* X = static_cast<V*>(c.X);
    const V* Qv = static_cast<const V*>(c.Q);
    const int SEQ = seq_stride(z.n);
    V* bufs = reinterpret_cast<V*>(smem_raw);   // two sets of L.G row buffers
    const V* tw = twiddles<V>(c.tb, z.n);
    DotAcc<T> ax, ay;
    double inv_scale = 1.0;   // |r|^2 = (sum of the squares formed here) * inv_scale
    if (phase == PH_ITER) {
        // alpha = rho / p.q, formed by the last stencil block (finish_S)
        if (threadIdx.x == 0) {
            usc[0] = (T)c.uscal[2 * b];
            usc[1] = (T)c.uscal[2 * b + 1];
        }
        // rt of the block's rows is read group by group: one thread per row
        // asks for it in L2 now
        if (threadIdx.x < d.tU)
            prefetch_l2(Rt + node_at(d, z, row0 + threadIdx.x, 0), (unsigned)(z.n * sizeof(V)));
        auto prefetch = [&](int g) {   // q of group g into row buffer set g & 1
            const int q = g * L.G + L.qq;
            if (g < ng && q < d.tU) {
                V* buf = bufs + ((g & 1) * L.G + L.qq) * SEQ;
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    cp_async_v(buf + pidx(L.t + m * z.T), Qv + node_at(d, z, row0 + q, L.t + m * z.T));
            }
            cp_async_commit();
        };
        prefetch(0);
        __syncthreads();
        const T alx = usc[0], aly = usc[1];
        // each row by its own team of n/8 threads, which touches only its own
        // row buffers: team barriers only
        const TeamBar team(L.qq, z.T);
        for (int g = 0; g < ng; ++g) {
            const int q = g * L.G + L.qq;
            const bool active = q < d.tU;
            const int row = row0 + q;
            // the other buffer set was last read by group g-1: the barrier at
            // the end of every group makes it free for group g+1's copies
            prefetch(g + 1);
            V rt[8];
            if (active) {
#pragma unroll
                for (int m = 0; m < 8; ++m) rt[m] = Rt[node_at(d, z, row, L.t + m * z.T)];
            }
            cp_async_wait<1>();
            team();
            V* buf = bufs + ((g & 1) * L.G + (active ? L.qq : 0)) * SEQ;
            V v[8];
            if (active) {
#pragma unroll
                for (int m = 0; m < 8; ++m) v[m] = buf[pidx(L.t + m * z.T)];
            }
            fft_reg<FFT_TO_BOTH, LOG2N>(v, buf, z.log2n, L.t, tw, active, team);
            if (active) {
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int k = L.t + m * z.T;
                    const V qt = hartley_pair(v[m], buf[pidx((z.n - k) & (z.n - 1))]);
                    const V rr = axpy2(rt[m], -alx, -aly, qt);
                    Rt[node_at(d, z, row, k)] = rr;
                    ax.add(rr.x, rr.x);
                    ay.add(rr.y, rr.y);
                }
            }
            team();   // mirror reads of this row buffer are done
        }
        cp_async_wait<0>();
        inv_scale = 1.0 / (double)z.n;
    } else {
        float4* U4 = reinterpret_cast<float4*>(c.u);
        const V* Pold = static_cast<const V*>(s.parity ? c.P1 : c.P0);
        if constexpr (sizeof(T) == 4) {   // the same conversions as refine_tile_dw
            if (threadIdx.x == 0) {
                usc[0] = (float)s.s[0];
                usc[1] = (float)s.s[1];
                usc[2] = (float)s.alpha[0];
                usc[3] = (float)s.alpha[1];
                usc[4] = (float)c.uscal[2 * b];       // 1 / |r| per corrector (0 once
                usc[5] = (float)c.uscal[2 * b + 1];   // converged), from finish_S
            }
            __syncthreads();
        }
        for (int g = 0; g < ng; ++g) {
            const int q = g * L.G + L.qq;
            const bool active = q < d.tU;
            const int row = row0 + q;
            V* buf = bufs + (active ? L.qq : 0) * SEQ;
            V v[8];
            if constexpr (sizeof(T) == 4) {   // REFINE, mixed: u is a double word
                const DWScal k{usc[0], usc[1], usc[2], usc[3]};
                const float ix = usc[4], iy = usc[5];
                if (active) {
#pragma unroll
                    for (int h = 0; h < 8; h += 4) {
                        float4 uu[4];
                        V xx[4], pp[4], qv[4];
#pragma unroll
                        for (int m = 0; m < 4; ++m) {   // loads first, stores after
                            const int64_t node = node_at(d, z, row, L.t + (h + m) * z.T);
                            uu[m] = U4[node];
                            xx[m] = X[node];
                            pp[m] = Pold[node];
                            qv[m] = Qv[node];
                        }
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const int64_t node = node_at(d, z, row, L.t + (h + m) * z.T);
                            U4[node] = w_new(uu[m], xx[m], pp[m], k);
                            X[node] = mk<V>(0.f, 0.f);
                            const V rr = mk<V>(qv[m].x * ix, qv[m].y * iy);
                            v[h + m] = rr;
                            ax.add(rr.x, rr.x);
                            ay.add(rr.y, rr.y);
                        }
                    }
                }
            } else {   // REFINE, FP64
                // 1 / |r64| per corrector (0 once converged), from finish_S
                const double ix = c.uscal[2 * b], iy = c.uscal[2 * b + 1];
                if (active) {
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const int64_t node = node_at(d, z, row, L.t + m * z.T);
                        const double2 xx = to_d2(X[node]);
                        const double2 pp = to_d2(Pold[node]);
                        double2 uu = c.u[node];
                        uu.x += s.s[0] * (xx.x + s.alpha[0] * pp.x);
                        uu.y += s.s[1] * (xx.y + s.alpha[1] * pp.y);
                        c.u[node] = uu;
                        X[node] = from_d2<V>(make_double2(0.0, 0.0));
                        const double2 qq = to_d2(Qv[node]);
                        const V rr = from_d2<V>(make_double2(qq.x * ix, qq.y * iy));
                        v[m] = rr;
                        ax.add(rr.x, rr.x);
                        ay.add(rr.y, rr.y);
                    }
                }
            }
            row_hartley_store<V, LOG2N>(v, buf, d, z, row, L.t, tw, active, Rt);
            __syncthreads();   // mirror reads of the buffer are done
        }
    }
    double sx = 0.0, sy = 0.0;
    block_sum2(ax, ay, red, sx, sy);
    if (threadIdx.x == 0) {
        c.partU[2 * (int64_t)blk] = sx * inv_scale;
        c.partU[2 * (int64_t)blk + 1] = sy * inv_scale;
    }
}

template <typename V>
__device__ void fused_U_tile(const Ctx& c, int blk) {
    __shared__ double red[64];   // block_sum2 scratch: 4 floats per warp (<= 32 warps)
    __shared__ typename ScalarOf<V>::T usc[6];
    const int b = find_real(c.startU, c.batch, blk);
    const RState& s = c.st[b];
    if (s.phase == PH_DONE) return;
    const RDesc d = c.desc[b];
    dispatch_size(d.log2n, [&]<int LG>() { fused_U_body<V, LG>(c, blk, b, s, d, red, usc); });
}

// ----------------------------------------------------------- C kernel --
// (the column solve body is in rve_colsolve.cuh)
// Column pass of one tile (any size): dispatches to the sized body.
// Reads the row transform of the residual (rt) from `in` and writes zhat to
// `out` (in == out allowed: every load of a column segment precedes its
// stores).
template <typename V>
__device__ void col_transform_tile(const V* in, V* out, const RDesc& d,
                                   int c0, V* smem, const Tables& tb, double delta, double* red,
                                   double* rho_part) {
    __shared__ typename ScalarOf<V>::T csc[1];
    dispatch_size(d.log2n, [&]<int LG>() {
        const Sz<LG> z(LG);
        col_solve_body<V, LG>([&](int r, int k) { return in[node_at(d, z, r, k)]; },
                              [&](int r, int k, V val) { out[node_at(d, z, r, k)] = val; }, d,
                              c0, smem, tb, delta, red, rho_part, csc);
    });
}

template <typename V>
__device__ void fused_C_tile(const Ctx& c, int blk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[64];   // block_sum2 scratch: 4 floats per warp (<= 32 warps)
    const int b = find_real(c.startC, c.batch, blk);
    if (c.st[b].phase == PH_DONE) return;
    const RDesc d = c.desc[b];
    col_transform_tile<V>(static_cast<const V*>(c.R), static_cast<V*>(c.T), d,
                          (blk - c.startC[b]) * d.tC,
                          reinterpret_cast<V*>(smem_raw), c.tb, c.delta, red,
                          c.partC + 2 * (int64_t)blk);
}

// One launch per pipeline kernel (the fused path).
template <typename V, int SCHEME>
__global__ void __launch_bounds__(256, sizeof(V) == 8 ? 3 : 2) k_fused_R(const Ctx c) { fused_R_tile<V, SCHEME>(c, blockIdx.x); }
template <typename V, int SCHEME>
__global__ void __launch_bounds__(256, sizeof(V) == 8 ? 3 : 2) k_fused_S(const Ctx c) {
    fused_S_tile<V, SCHEME>(c, blockIdx.x);
}
template <typename V>
__global__ void __launch_bounds__(256, sizeof(V) == 8 ? 4 : 2) k_fused_U(const Ctx c) { fused_U_tile<V>(c, blockIdx.x); }
template <typename V>
__global__ void __launch_bounds__(512) k_fused_C(const Ctx c) {
    fused_C_tile<V>(c, blockIdx.x);
}

// ------------------------------------------------------ control kernel --
__device__ __forceinline__ bool bad(double v) { return !isfinite(v); }

// Stagnation test of an inner cycle: the residual must fall below
// STALL_FACTOR times its best value within STALL_STEPS steps.  Healthy
// preconditioned CG here contracts by ~0.8 per step or better, so only a
// cycle that has reached the attainable accuracy of its precision trips it.
constexpr double STALL_FACTOR = 0.7;
constexpr int STALL_STEPS = 30;

// Control step of realization b, executed by one whole warp.
__device__ void control_one(const Ctx& c, int b) {
    RState& s = c.st[b];
    if (s.phase == PH_DONE) return;
    const int ts0 = c.startS[b], tsn = c.startS[b + 1] - ts0;
    const int tu0 = c.startU[b], tun = c.startU[b + 1] - tu0;
    const int tc0 = c.startC[b], tcn = c.startC[b + 1] - tc0;
    double pS[2], pU[2], pC[2];
    for (int k = 0; k < 2; ++k) {
        pS[k] = warp_sum_array(c.partS + 2 * (int64_t)ts0 + k, tsn, 2);
        pU[k] = warp_sum_array(c.partU + 2 * (int64_t)tu0 + k, tun, 2);
        pC[k] = warp_sum_array(c.partC + 2 * (int64_t)tc0 + k, tcn, 2);
    }
    if ((threadIdx.x & 31) != 0) return;
    if (s.phase == PH_ITER) {
        s.steps += 1;
        bool any_active = false;
        for (int k = 0; k < 2; ++k) {
            if (!s.active[k]) { s.alpha[k] = 0.0; s.beta[k] = 0.0; continue; }
            const double alpha = s.rho[k] / pS[k];
            const double rn = sqrt(pU[k]);
            if (bad(alpha) || bad(rn) || bad(pC[k])) {
                s.status = RVE_ENAN;
                s.phase = PH_DONE;
                atomicAdd(c.ndone, 1);
                return;
            }
            s.alpha[k] = alpha;
            s.iters[k] += 1;
            // a cycle whose residual has stopped falling (the attainable
            // accuracy of the inner precision) ends early: the refinement
            // step then restarts from the true residual
            if (rn < STALL_FACTOR * s.best[k]) {
                s.best[k] = rn;
                s.stall[k] = 0;
            } else {
                s.stall[k] += 1;
            }
            const bool stalled = s.stall[k] >= STALL_STEPS;
            if (rn <= s.target[k] || stalled || s.iters[k] >= c.max_iter) {
                s.active[k] = 0;       // frozen; alpha still pending for x
                s.beta[k] = 0.0;
                if (s.iters[k] >= c.max_iter && rn > s.target[k]) s.final_pass = 1;
            } else {
                s.beta[k] = pC[k] / s.rho[k];
                s.rho[k] = pC[k];
                any_active = true;
            }
        }
        s.parity ^= 1;
        if (!any_active) s.phase = PH_REFINE;   // every corrector ended its cycle
        return;
    }
    // REFINE: true residual of the accumulated solution
    s.refinements += 1;
    bool all_done = true;
    for (int k = 0; k < 2; ++k) {
        const double rn = sqrt(pS[k]);
        if (bad(rn)) {
            s.status = RVE_ENAN;
            s.phase = PH_DONE;
            atomicAdd(c.ndone, 1);
            return;
        }
        if (s.refinements == 1) s.fnorm[k] = rn;
        const bool conv = (s.refinements == 1) ? (rn == 0.0) : (rn <= c.tol * s.fnorm[k]);
        const double prev = s.relres[k];
        s.relres[k] = s.fnorm[k] > 0.0 ? rn / s.fnorm[k] : 0.0;
        s.alpha[k] = 0.0;
        if (conv || s.cdone[k]) {
            s.cdone[k] = 1;
            s.active[k] = 0;
            s.s[k] = 0.0;
            s.beta[k] = 0.0;
            continue;
        }
        all_done = false;
        // each cycle restarts CG from the true residual (p = z): keeping
        // the old direction across the replaced residual loses conjugacy
        // when the FP32 recurrence has drifted (tens of percent here)
        s.beta[k] = 0.0;
        s.s[k] = rn;
        s.active[k] = 1;
        s.best[k] = 1.0;   // the inner system starts from r / |r|
        s.stall[k] = 0;
        // inner target: what the outer tolerance still needs, but no less
        // than the usual inner reduction
        const double want = 0.5 * c.tol * s.fnorm[k] / rn;
        double tgt = fmax(want, c.inner_tol);
        // a cycle gains at most what the rounding of its iterate allows
        // (about eps_inner times the condition of A on the correction): when
        // the last cycle's true residual fell far less than it was asked
        // to, ask the next one for no more than ten times what it achieved
        if (s.refinements >= 2 && prev > 0.0) {
            const double got = s.relres[k] / prev;
            if (got > 10.0 * s.target[k]) tgt = fmax(tgt, 0.1 * got);
        }
        s.target[k] = fmin(0.5, tgt);
        s.rho[k] = pC[k];
        if (s.iters[k] >= c.max_iter) s.final_pass = 1;
    }
    if (all_done || s.final_pass) {
        if (!all_done) s.status = RVE_ENOCONV;
        s.phase = PH_DONE;
        atomicAdd(c.ndone, 1);
        return;
    }
    s.phase = PH_ITER;
}

__global__ void k_control(const Ctx c) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= c.batch) return;
    control_one(c, w);
}

// ------------------------------------------------------ persistent path --
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch.  Every wait is bounded by
// timeout_ns: a block that waits longer sets the error word and leaves; all
// blocks then see the error after their own (bounded) wait and return
// false, so the kernel always ends.
__device__ bool grid_sync(int* ctl, unsigned nblocks, unsigned long long timeout_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int* vgen = ctl + CTL_GEN;
        volatile int* verr = ctl + CTL_ERR;
        const int gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(reinterpret_cast<unsigned*>(ctl + CTL_ARRIVE), 1u);
        if (arrived == nblocks - 1) {
            atomicExch(ctl + CTL_ARRIVE, 0);
            __threadfence();
            atomicAdd(ctl + CTL_GEN, 1);
        } else {
            const unsigned long long t0 = global_ns();
            while (*vgen == gen) {
                if (*verr) break;
                if (global_ns() - t0 > timeout_ns) {
                    atomicExch(ctl + CTL_ERR, 1);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok = (*verr == 0);
    }
    __syncthreads();
    return ok != 0;
}

struct PersistArgs {
    int tilesS, tilesU, tilesC;
    long long max_steps;
    unsigned long long timeout_ns;
};

// The whole solve in one cooperative launch: each pipeline step runs the
// refine/stencil, update, column and control phases over all tiles of the
// batch (any mix of sizes), separated by grid barriers, until every
// realization is done.
// Phases as separate (not inlined) calls, so that each keeps its own register
// allocation inside the one persistent kernel.
template <typename V, int SCHEME>
__device__ __noinline__ void phase_RS(const Ctx& c, int t) {
    fused_R_tile<V, SCHEME>(c, t);
    fused_S_tile<V, SCHEME>(c, t);
}
template <typename V>
__device__ __noinline__ void phase_U(const Ctx& c, int t) { fused_U_tile<V>(c, t); }
template <typename V>
__device__ __noinline__ void phase_C(const Ctx& c, int t) { fused_C_tile<V>(c, t); }

template <typename V, int SCHEME>
__global__ void __launch_bounds__(256, 2) k_persistent(const Ctx c, const PersistArgs a) {
    const unsigned nb = gridDim.x;
    for (long long step = 0; step < a.max_steps; ++step) {
        for (int t = blockIdx.x; t < a.tilesS; t += nb) phase_RS<V, SCHEME>(c, t);
        if (!grid_sync(c.ndone, nb, a.timeout_ns)) return;
        for (int t = blockIdx.x; t < a.tilesU; t += nb) phase_U<V>(c, t);
        if (!grid_sync(c.ndone, nb, a.timeout_ns)) return;
        for (int t = blockIdx.x; t < a.tilesC; t += nb) phase_C<V>(c, t);
        if (!grid_sync(c.ndone, nb, a.timeout_ns)) return;
        const int warps = blockDim.x >> 5;
        for (int r = blockIdx.x * warps + (threadIdx.x >> 5); r < c.batch; r += nb * warps)
            control_one(c, r);
        if (!grid_sync(c.ndone, nb, a.timeout_ns)) return;
        if (*reinterpret_cast<volatile int*>(c.ndone) >= c.batch) return;
    }
}

__global__ void k_init(const Ctx c, int64_t nodes, size_t vbytes) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = gid; k < nodes; k += stride) {
        c.u[k] = make_double2(0.0, 0.0);
        if (vbytes == 16) {
            static_cast<double2*>(c.X)[k] = make_double2(0.0, 0.0);
            static_cast<double2*>(c.P0)[k] = make_double2(0.0, 0.0);
            static_cast<double2*>(c.P1)[k] = make_double2(0.0, 0.0);
        } else {
            static_cast<float2*>(c.X)[k] = make_float2(0.f, 0.f);
            static_cast<float2*>(c.P0)[k] = make_float2(0.f, 0.f);
            static_cast<float2*>(c.P1)[k] = make_float2(0.f, 0.f);
        }
    }
    for (int64_t b = gid; b < c.batch; b += stride) {
        RState z = {};
        z.phase = PH_REFINE;
        z.status = RVE_OK;
        c.st[b] = z;
        c.tiles_done[b] = 0;
    }
    if (gid == 0) {
        c.ndone[0] = 0;                          // realizations done
        c.ndone[CTL_ARRIVE] = 0;                 // grid barrier arrivals
        c.ndone[CTL_GEN] = 0;                    // grid barrier generation
        c.ndone[CTL_ERR] = 0;                    // a bounded wait gave up
        c.ndone[CTL_GROUPS] = 0;                 // loop groups of a captured plan
    }
}

__global__ void k_report(const Ctx c, rve_solve_info* info) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= c.batch) return;
    const RState s = c.st[b];
    rve_solve_info r;
    r.iters[0] = s.iters[0];
    r.iters[1] = s.iters[1];
    r.status = (s.phase == PH_DONE) ? s.status
               : (c.ndone[CTL_ERR] ? RVE_ETIMEOUT : RVE_ENOCONV);
    r.refinements = s.refinements;
    r.steps = s.steps;
    r.reserved = 0;
    r.relres[0] = s.relres[0];
    r.relres[1] = s.relres[1];
    info[b] = r;
}

// (double)f from the IEEE fields of a normal float or a zero, with integer
// instructions (the conversion instruction runs on the narrow FP64 pipe);
// subnormals, infinities and NaNs take the conversion instruction.
__device__ __forceinline__ double f2d(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
    if ((b & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)sgn);
    if (e == 0u || e == 0xFFu) return (double)f;
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// Mixed path: the double-word iterate (float4 per node) becomes the caller's
// FP64 solution, in place (each thread rewrites the 16 bytes it read):
// hi + lo rounded once to double (one FP64 addition per component).
__global__ void k_u_finalize(double2* u, int64_t nodes) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nodes; k += stride) {
        const float4 w = reinterpret_cast<const float4*>(u)[k];
        u[k] = make_double2(f2d(w.x) + f2d(w.z), f2d(w.y) + f2d(w.w));
    }
}

static cudaError_t finalize_u(const Plan& p, const Ctx& c, cudaStream_t s) {
    if (p.precision != RVE_MIXED) return cudaSuccess;
    k_u_finalize<<<std::min<int64_t>((p.nodes + 255) / 256, 8 * 152), 256, 0, s>>>(c.u, p.nodes);
    note_launch();
    return cudaGetLastError();
}

// --------------------------------------------------------------- host --
std::atomic<long long> g_launches{0};

// Per-kernel event timing of the fused pipeline (diagnostics).
// Kernels: 0 refine, 1 stencil, 2 update + row transform, 3 column, 4 control.
struct Profiler {
    static constexpr int K = PROFILE_KERNELS;
    bool on = false;
    double ms[K] = {};
    long long launches[K] = {};
    std::vector<cudaEvent_t> ev;    // K + 1 events per recorded step
    int used = 0;                   // steps recorded since the last harvest
    void ensure(int steps) {
        while ((int)ev.size() < (K + 1) * steps) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            ev.push_back(e);
        }
    }
    void harvest() {   // stream already synchronised
        for (int k = 0; k < used; ++k)
            for (int j = 0; j < K; ++j) {
                float t = 0.f;
                if (cudaEventElapsedTime(&t, ev[(K + 1) * k + j], ev[(K + 1) * k + j + 1]) ==
                    cudaSuccess) {
                    ms[j] += t;
                    launches[j] += 1;
                }
            }
        used = 0;
    }
};
static Profiler g_prof;

void profile_enable(bool on) { g_prof.on = on; }
bool profile_on() { return g_prof.on; }
int profile_read(double* ms, long long* launches) {
    for (int j = 0; j < Profiler::K; ++j) {
        if (ms) ms[j] = g_prof.ms[j];
        if (launches) launches[j] = g_prof.launches[j];
        g_prof.ms[j] = 0.0;
        g_prof.launches[j] = 0;
    }
    return Profiler::K;
}

static Ctx make_ctx(const Plan& p, void* ws, const uint32_t* mask, const double* coef, double* u,
                    const rve_solve_opts& o, const double* f = nullptr) {
    char* w = static_cast<char*>(ws);
    Ctx c;
    c.batch = p.batch;
    c.desc = reinterpret_cast<const RDesc*>(w + p.o_desc);
    c.startS = reinterpret_cast<const int32_t*>(w + p.o_startS);
    c.startU = reinterpret_cast<const int32_t*>(w + p.o_startU);
    c.startC = reinterpret_cast<const int32_t*>(w + p.o_startC);
    c.st = reinterpret_cast<RState*>(w + p.o_state);
    c.partS = reinterpret_cast<double*>(w + p.o_partS);
    c.partU = reinterpret_cast<double*>(w + p.o_partU);
    c.partC = reinterpret_cast<double*>(w + p.o_partC);
    c.uscal = reinterpret_cast<double*>(w + p.o_uscal);
    c.tiles_done = reinterpret_cast<int*>(w + p.o_cnt);
    c.tb = tables_of(p, ws);
    c.cs.mask = mask;
    c.cs.coef = coef;
    c.cs.f = reinterpret_cast<const double2*>(f);
    c.u = reinterpret_cast<double2*>(u);
    c.X = w + p.o_X;
    c.R = w + p.o_R;
    c.Q = w + p.o_Q;
    c.T = w + p.o_T;
    c.P0 = w + p.o_P0;
    c.P1 = w + p.o_P1;
    c.tol = o.tol;
    c.inner_tol = (p.precision == RVE_MIXED) ? o.inner_tol : 0.5 * o.tol;
    c.delta = o.delta;
    c.max_iter = o.max_iter;
    c.ndone = reinterpret_cast<int*>(w + p.o_ctl);
    return c;
}

rve_status upload_plan(const Plan& p, void* ws, cudaStream_t s) {
    char* w = static_cast<char*>(ws);
    cudaError_t e = cudaMemcpyAsync(w + p.o_desc, p.desc.data(), sizeof(RDesc) * p.batch,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + p.o_startS, p.startS.data(), sizeof(int32_t) * (p.batch + 1),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + p.o_startU, p.startU.data(), sizeof(int32_t) * (p.batch + 1),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + p.o_startC, p.startC.data(), sizeof(int32_t) * (p.batch + 1),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + p.o_startA, p.startA.data(), sizeof(int32_t) * (p.batch + 1),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + p.o_startA2, p.startA2.data(), sizeof(int32_t) * (p.batch + 1),
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return RVE_ECUDA;
    return launch_tables(p, ws, s) == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

template <typename V, int SCHEME>
static cudaError_t fused_step(const Plan& p, const Ctx& c, cudaStream_t s, cudaEvent_t* ev) {
    if (ev) cudaEventRecord(ev[0], s);
    k_fused_R<V, SCHEME><<<p.tilesS, 256, 0, s>>>(c);
    if (ev) cudaEventRecord(ev[1], s);
    k_fused_S<V, SCHEME><<<p.tilesS, 256, p.smemS, s>>>(c);
    if (ev) cudaEventRecord(ev[2], s);
    k_fused_U<V><<<p.tilesU, 256, p.smemU, s>>>(c);
    if (ev) cudaEventRecord(ev[3], s);
    k_fused_C<V><<<p.tilesC, p.blockC, p.smemC, s>>>(c);
    if (ev) cudaEventRecord(ev[4], s);
    k_control<<<(p.batch + 7) / 8, 256, 0, s>>>(c);
    if (ev) cudaEventRecord(ev[5], s);
    note_launch(5);
    return cudaGetLastError();
}

template <typename V, int SCHEME>
static cudaError_t set_smem_attrs(const Plan& p) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_S<V, SCHEME>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smemS);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused_U<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p.smemU);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fused_C<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p.smemC);
    return e;
}

template <typename V, int SCHEME>
static rve_status fused_loop(const Plan& p, const Ctx& c, const rve_solve_opts& o,
                             cudaStream_t s) {
    if (set_smem_attrs<V, SCHEME>(p) != cudaSuccess) return RVE_ECUDA;
    // bound on pipeline steps: every cycle costs one REFINE step
    const int64_t max_steps = 2LL * o.max_iter + 64;
    const int every = o.check_every > 0 ? o.check_every : 8;
    int host_done = 0;
    if (g_prof.on) {
        g_prof.ensure(every);
        g_prof.used = 0;
    }
    for (int64_t g = 0; g < max_steps; ++g) {
        cudaEvent_t* ev = nullptr;
        if (g_prof.on && (int)g_prof.ev.size() >= (Profiler::K + 1) * every)
            ev = &g_prof.ev[(Profiler::K + 1) * g_prof.used++];
        if (fused_step<V, SCHEME>(p, c, s, ev) != cudaSuccess) return RVE_ECUDA;
        if ((g + 1) % every == 0) {
            if (cudaMemcpyAsync(&host_done, c.ndone, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return RVE_ECUDA;
            if (g_prof.on) g_prof.harvest();
            if (host_done >= p.batch) break;
        }
    }
    if (g_prof.on) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return RVE_ECUDA;
        g_prof.harvest();
    }
    return RVE_OK;
}

template <typename V, int SCHEME>
static rve_status persistent_prepare_t(Plan& p) {
    const size_t smem = std::max(p.smemS, std::max(p.smemU, p.smemC));
    if (cudaFuncSetAttribute(k_persistent<V, SCHEME>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return RVE_ECUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent<V, SCHEME>, 256,
                                                      smem) != cudaSuccess ||
        per_sm < 1)
        return RVE_ECUDA;
    p.persist_grid = per_sm * sms;   // co-resident: one wave
    p.persist_smem = smem;
    return RVE_OK;
}

rve_status prepare_persistent(Plan& p) {
    if (p.precision == RVE_MIXED)
        return (p.scheme == RVE_Q1_LUMPED) ? persistent_prepare_t<float2, 1>(p)
                                           : persistent_prepare_t<float2, 0>(p);
    return (p.scheme == RVE_Q1_LUMPED) ? persistent_prepare_t<double2, 1>(p)
                                       : persistent_prepare_t<double2, 0>(p);
}

template <typename V, int SCHEME>
static rve_status persistent_launch(const Plan& p, const Ctx& c, const rve_solve_opts& o,
                                    cudaStream_t s) {
    if (p.persist_grid <= 0) return RVE_ECUDA;   // prepare_persistent() first
    PersistArgs a;
    a.tilesS = p.tilesS;
    a.tilesU = p.tilesU;
    a.tilesC = p.tilesC;
    a.max_steps = 2LL * o.max_iter + 64;
    a.timeout_ns = (unsigned long long)o.timeout_us * 1000ull;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.persist_grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = p.persist_smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_persistent<V, SCHEME>, c, a);
    note_launch();
    return e == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

// Persistent path: descriptors must already be in the workspace (upload_plan);
// everything after that is stream-ordered kernel launches (no host sync), so
// the sequence can be captured in a CUDA graph.
rve_status enqueue_solve_persistent(const Plan& p, void* ws, const uint32_t* mask,
                                    const double* coef, const rve_solve_opts& o, double* u,
                                    rve_solve_info* info, cudaStream_t s, const double* f) {
    Ctx c = make_ctx(p, ws, mask, coef, u, o, f);
    if (launch_tables(p, ws, s) != cudaSuccess) return RVE_ECUDA;
    k_init<<<std::min<int64_t>((p.nodes + 255) / 256, 4096), 256, 0, s>>>(c, p.nodes, p.vbytes);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
    rve_status st;
    if (p.precision == RVE_MIXED)
        st = (p.scheme == RVE_Q1_LUMPED) ? persistent_launch<float2, 1>(p, c, o, s)
                                         : persistent_launch<float2, 0>(p, c, o, s);
    else
        st = (p.scheme == RVE_Q1_LUMPED) ? persistent_launch<double2, 1>(p, c, o, s)
                                         : persistent_launch<double2, 0>(p, c, o, s);
    if (st != RVE_OK) return st;
    if (finalize_u(p, c, s) != cudaSuccess) return RVE_ECUDA;
    k_report<<<(p.batch + 127) / 128, 128, 0, s>>>(c, info);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

// Uploads only the descriptors and tile tables (host -> device copies);
// the lookup tables are filled by a kernel in the enqueued sequence.
rve_status upload_descriptors(const Plan& p, void* ws, cudaStream_t s) {
    char* w = static_cast<char*>(ws);
    cudaError_t e = cudaMemcpyAsync(w + p.o_desc, p.desc.data(), sizeof(RDesc) * p.batch,
                                    cudaMemcpyHostToDevice, s);
    const std::vector<int32_t>* tabs[5] = {&p.startS, &p.startU, &p.startC, &p.startA, &p.startA2};
    const size_t offs[5] = {p.o_startS, p.o_startU, p.o_startC, p.o_startA, p.o_startA2};
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(w + offs[k], tabs[k]->data(), sizeof(int32_t) * (p.batch + 1),
                            cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status run_solve_persistent(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                                const rve_solve_opts& o, double* u, rve_solve_info* info,
                                cudaStream_t s, const double* f) {
    Plan q = p;
    rve_status st = (q.persist_grid > 0) ? RVE_OK : prepare_persistent(q);
    if (st == RVE_OK) st = upload_descriptors(q, ws, s);
    if (st != RVE_OK) return st;
    return enqueue_solve_persistent(q, ws, mask, coef, o, u, info, s, f);
}

// ----------------------------------------------- captured loop of steps --
// A plan captured with the fused path: the pipeline steps run inside a CUDA
// graph conditional WHILE node whose body is LOOP_GROUP fused steps (the
// same kernels as the fused path) followed by a one-thread kernel that
// re-arms the node while some realization is unfinished and the step bound
// is not reached.  No host synchronisation, so the whole solve stays inside
// one graph launch; kernel boundaries separate the phases.
constexpr int LOOP_GROUP = 4;

__global__ void k_loop_cond(cudaGraphConditionalHandle h, int* ctl, int batch,
                            long long max_groups) {
    if (threadIdx.x != 0) return;
    const int g = ctl[CTL_GROUPS] + 1;
    ctl[CTL_GROUPS] = g;
    const bool more = *reinterpret_cast<volatile int*>(ctl) < batch && g < max_groups;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

template <typename V, int SCHEME>
static rve_status loop_body(const Plan& p, const Ctx& c, cudaStream_t s,
                            cudaGraphConditionalHandle h, long long max_groups) {
    for (int k = 0; k < LOOP_GROUP; ++k)
        if (fused_step<V, SCHEME>(p, c, s, nullptr) != cudaSuccess) return RVE_ECUDA;
    k_loop_cond<<<1, 32, 0, s>>>(h, c.ndone, p.batch, max_groups);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status prepare_graph_loop(const Plan& p) {
    cudaError_t e;
    if (p.precision == RVE_MIXED)
        e = (p.scheme == RVE_Q1_LUMPED) ? set_smem_attrs<float2, 1>(p) : set_smem_attrs<float2, 0>(p);
    else
        e = (p.scheme == RVE_Q1_LUMPED) ? set_smem_attrs<double2, 1>(p) : set_smem_attrs<double2, 0>(p);
    return e == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status enqueue_solve_graph_loop(const Plan& p, void* ws, const uint32_t* mask,
                                    const double* coef, const rve_solve_opts& o, double* u,
                                    rve_solve_info* info, cudaStream_t s, const double* f) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
        return RVE_EINVAL;   // only inside a stream capture
    Ctx c = make_ctx(p, ws, mask, coef, u, o, f);
    if (launch_tables(p, ws, s) != cudaSuccess) return RVE_ECUDA;
    k_init<<<std::min<int64_t>((p.nodes + 255) / 256, 4096), 256, 0, s>>>(c, p.nodes, p.vbytes);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess)
        return RVE_ECUDA;
    const std::vector<cudaGraphNode_t> dep(deps, deps + nd);   // valid until the next call
    // the conditional node, run at least once per graph launch (default 1,
    // re-assigned on every launch)
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return RVE_ECUDA;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, dep.data(), nullptr, dep.size(), &np) != cudaSuccess)
        return RVE_ECUDA;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                            cudaStreamSetCaptureDependencies) != cudaSuccess)
        return RVE_ECUDA;
    // the body: LOOP_GROUP pipeline steps and the re-arming kernel, captured
    // on a helper stream straight into the node's body graph
    cudaStream_t sb = nullptr;
    if (cudaStreamCreateWithFlags(&sb, cudaStreamNonBlocking) != cudaSuccess) return RVE_ECUDA;
    rve_status st = RVE_OK;
    if (cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = RVE_ECUDA;
    } else {
        const long long max_groups = (2LL * o.max_iter + 64) / LOOP_GROUP + 1;
        if (p.precision == RVE_MIXED)
            st = (p.scheme == RVE_Q1_LUMPED) ? loop_body<float2, 1>(p, c, sb, h, max_groups)
                                             : loop_body<float2, 0>(p, c, sb, h, max_groups);
        else
            st = (p.scheme == RVE_Q1_LUMPED) ? loop_body<double2, 1>(p, c, sb, h, max_groups)
                                             : loop_body<double2, 0>(p, c, sb, h, max_groups);
        cudaGraph_t out = nullptr;
        if (cudaStreamEndCapture(sb, &out) != cudaSuccess) st = RVE_ECUDA;
    }
    cudaStreamDestroy(sb);
    if (st != RVE_OK) return st;
    if (finalize_u(p, c, s) != cudaSuccess) return RVE_ECUDA;
    k_report<<<(p.batch + 127) / 128, 128, 0, s>>>(c, info);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status run_solve_fused(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                           const rve_solve_opts& o, double* u, rve_solve_info* info,
                           cudaStream_t s, const double* f) {
    rve_status st = upload_plan(p, ws, s);
    if (st != RVE_OK) return st;
    Ctx c = make_ctx(p, ws, mask, coef, u, o, f);
    k_init<<<std::min<int64_t>((p.nodes + 255) / 256, 4096), 256, 0, s>>>(c, p.nodes, p.vbytes);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
    if (p.precision == RVE_MIXED) {
        st = (p.scheme == RVE_Q1_LUMPED) ? fused_loop<float2, 1>(p, c, o, s)
                                         : fused_loop<float2, 0>(p, c, o, s);
    } else {
        st = (p.scheme == RVE_Q1_LUMPED) ? fused_loop<double2, 1>(p, c, o, s)
                                         : fused_loop<double2, 0>(p, c, o, s);
    }
    if (st != RVE_OK) return st;
    if (finalize_u(p, c, s) != cudaSuccess) return RVE_ECUDA;
    k_report<<<(p.batch + 127) / 128, 128, 0, s>>>(c, info);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

// --------------------------------------------------- preconditioner apply --
// Standalone transform passes (rve_apply_precond and the plain path): row
// Hartley of `in` into `out`, and the column pair with the scale in place.
// Tiles tile0 .. tile0 + gridDim.x - 1 of the batch's row / column tiling.
template <typename V>
__global__ void __launch_bounds__(256) k_row_hartley(const RDesc* __restrict__ desc,
                                                     const int32_t* __restrict__ startU, int batch,
                                                     int tile0, Tables tb, const V* __restrict__ in,
                                                     V* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int blk = blockIdx.x + tile0;
    const int b = find_real(startU, batch, blk);
    const RDesc d = desc[b];
    dispatch_size(d.log2n, [&]<int LG>() {
        const RowLayout<LG> L(d.log2n);
        const int row0 = (blk - startU[b]) * d.tU;
        for (int g0 = 0; g0 < d.tU; g0 += L.G) {
            const bool active = g0 + L.qq < d.tU;
            const int row = row0 + g0 + L.qq;
            V* buf = reinterpret_cast<V*>(smem_raw) + (active ? L.qq : 0) * seq_stride(L.z.n);
            V v[8];
            if (active) {
#pragma unroll
                for (int m = 0; m < 8; ++m) v[m] = in[node_at(d, L.z, row, L.t + m * L.z.T)];
            }
            row_hartley_store<V, LG>(v, buf, d, L.z, row, L.t, twiddles<V>(tb, L.z.n), active,
                                     out);
            __syncthreads();   // mirror reads of the buffers are done
        }
    });
}

template <typename V>
__global__ void __launch_bounds__(512) k_col_hartley(const RDesc* __restrict__ desc,
                                                      const int32_t* __restrict__ startC, int batch,
                                                      int tile0, Tables tb, double delta,
                                                      V* __restrict__ T) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[64];   // block_sum2 scratch: 4 floats per warp (<= 32 warps)
    const int blk = blockIdx.x + tile0;
    const int b = find_real(startC, batch, blk);
    const RDesc d = desc[b];
    col_transform_tile<V>(T, T, d, (blk - startC[b]) * d.tC, reinterpret_cast<V*>(smem_raw), tb,
                          delta, red, nullptr);
}

template <typename V>
cudaError_t precond_passes(const Plan& p, void* ws, double delta, const V* x, V* y, V* tmp,
                           int b_first, int b_count, cudaStream_t s) {
    char* w = static_cast<char*>(ws);
    const RDesc* desc = reinterpret_cast<const RDesc*>(w + p.o_desc);
    const int32_t* startU = reinterpret_cast<const int32_t*>(w + p.o_startU);
    const int32_t* startC = reinterpret_cast<const int32_t*>(w + p.o_startC);
    const Tables tb = tables_of(p, ws);
    cudaError_t e = cudaFuncSetAttribute(k_row_hartley<V>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smemU);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_col_hartley<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p.smemC);
    if (e != cudaSuccess) return e;
    const int u0 = p.startU[b_first], un = p.startU[b_first + b_count] - u0;
    const int c0 = p.startC[b_first], cn = p.startC[b_first + b_count] - c0;
    k_row_hartley<V><<<un, 256, p.smemU, s>>>(desc, startU, p.batch, u0, tb, x, tmp);
    k_col_hartley<V><<<cn, p.blockC, p.smemC, s>>>(desc, startC, p.batch, c0, tb, delta, tmp);
    k_row_hartley<V><<<un, 256, p.smemU, s>>>(desc, startU, p.batch, u0, tb, tmp, y);
    note_launch(3);
    return cudaGetLastError();
}

template cudaError_t precond_passes<double2>(const Plan&, void*, double, const double2*, double2*,
                                             double2*, int, int, cudaStream_t);
template cudaError_t precond_passes<float2>(const Plan&, void*, double, const float2*, float2*,
                                            float2*, int, int, cudaStream_t);

cudaError_t launch_precond(const Plan& p, void* ws, double delta, int precision, const void* x,
                           void* y, cudaStream_t s) {
    if (upload_plan(p, ws, s) != RVE_OK) return cudaErrorUnknown;
    char* w = static_cast<char*>(ws);
    if (precision == RVE_FP64)
        return precond_passes<double2>(p, ws, delta, static_cast<const double2*>(x),
                                       static_cast<double2*>(y),
                                       reinterpret_cast<double2*>(w + p.o_T), 0, p.batch, s);
    return precond_passes<float2>(p, ws, delta, static_cast<const float2*>(x),
                                  static_cast<float2*>(y), reinterpret_cast<float2*>(w + p.o_T), 0,
                                  p.batch, s);
}

}  // namespace rve
