// rve_colsolve.cuh -- the column pass of the preconditioner: periodic
// tridiagonal solves along one grid axis after the Hartley transforms along
// the others (shared by the 2D pipeline and the 3D solver).
#pragma once

#include "rve_common.cuh"

namespace rve {

// Column pass on t = row-Hartley(r).  The row transform diagonalises the
// row factor of A_Delta, so column k2 of t is left with the periodic
// tridiagonal system
//     M z = t,   M = c0 (T + lambda) + delta,   lambda = 4 sin^2(pi k2 / n),
// T the periodic second difference along the column (the fast Poisson
// scheme of Hockney: Fourier in one direction, tridiagonal solves in the
// other).  With rho + 1/rho = 2 + mu, mu = lambda + delta / c0,
//     M = (c0 / rho) (1 - rho S)(1 - rho S^T),   S the cyclic shift,
// so M^{-1} t = (rho / c0) F^T F t with the causal filter F = (1 - rho S)^{-1}
// (y_i = t_i + rho y_{i-1}, periodic) and its transpose, the anticausal
// filter.  The pass stores zhat = M^{-1} t / n (the row transform in the
// stencil kernel supplies the other factor 1/n of the inverse transform)
// and rho_c = r.z = t.zhat = (rho / (n c0)) |F t|^2.
//
// Each thread holds SEG consecutive rows of one column in registers: it
// runs the filter over its segment from a zero start, the segment's end
// value goes through shared memory, and every thread adds the periodic
// carry-in  sum_{j=1..P} R^{j-1} e_{s-j} / (1 - R^P)  (R = rho^SEG, P
// segments; the sum stops once R^{j-1} is negligible) times rho^{i+1}.
// The anticausal filter runs the same way upwards.  The singular column
// k2 = 0 with delta = 0 (rho = 1) takes the pseudo-inverse: with
// t' = t - mean t, y = cumsum t' made mean-zero, w = reverse cumsum y made
// mean-zero, zhat = w / (n c0), rho_c = |y|^2 / (n c0).
// Block: C columns x P segments, thread (cc, s) with cc fastest so that the
// global accesses of a warp are row segments of C elements.  `rho_part`
// may be null.  rho_of(k2) gives the filter root of column k2 (not called
// for the singular column).  UNROLL: the periodic carries sum all P segment
// values (independent loads, no early exit) instead of stopping once the
// weight is negligible.  SEGO > 0 sets the rows per segment (a divisor of
// n) in place of col_seg_rows.
template <typename V, int LOG2N, bool UNROLL = false, int SEGO = 0, typename Ld, typename St,
          typename RhoOf>
__device__ __forceinline__ void col_solve_core(Ld&& ld, St&& st, RhoOf&& rho_of, const RDesc& d,
                                               int c0, V* smem, const Tables& tb, double delta,
                                               double* red, double* rho_part,
                                               typename ScalarOf<V>::T* csc) {
    typedef typename ScalarOf<V>::T Ts;
    constexpr int n = 1 << LOG2N;
    constexpr int SEG = SEGO > 0 ? SEGO : col_seg_rows(n, (int)sizeof(V));
    constexpr int P = n / SEG;
    // carry terms below this weight are dropped (far below the rounding of Ts)
    constexpr Ts CARRY_EPS = sizeof(Ts) == 4 ? (Ts)1e-10 : (Ts)1e-19;
    const Sz<LOG2N> z(LOG2N);
    const int C = d.tC;
    const int tid = threadIdx.x;
    const int s = tid / C, cc = tid - (tid / C) * C;
    const bool active = s < P;
    const int k2 = c0 + cc;
    const bool zero_block = (c0 == 0 && delta == 0.0);   // block holds the singular column
    const bool zcol = zero_block && cc == 0;
    if (tid == 0) csc[0] = (Ts)(1.0 / ((double)n * d.c0));
    V v[SEG];
#pragma unroll
    for (int i = 0; i < SEG; ++i)
        v[i] = active ? ld(s * SEG + i, k2) : mk<V>((Ts)0, (Ts)0);
    Ts rho = (Ts)1;
    if (active && !zcol) rho = rho_of(k2);
    V* E = smem;                  // [P][C] segment end values (causal pass)
    V* B = smem + P * C;          // [P][C] segment start values (anticausal pass)
    V* Zs = smem + 2 * P * C;     // [2][P] singular column: segment sums
    // causal filter within the segment
#pragma unroll
    for (int i = 1; i < SEG; ++i) {
        v[i].x += rho * v[i - 1].x;
        v[i].y += rho * v[i - 1].y;
    }
    if (active) E[s * C + cc] = v[SEG - 1];
    __syncthreads();   // also publishes csc
    const Ts inv_nc0 = csc[0];
    Ts R = (Ts)0, inv1mRP = (Ts)0;
    if (active && !zcol) {
        R = rho;
#pragma unroll
        for (int k = 1; k < SEG; k <<= 1) R *= R;            // rho^SEG
        Ts RP = R;
#pragma unroll
        for (int k = 1; k < P; k <<= 1) RP *= RP;            // rho^n
        inv1mRP = (Ts)1 / ((Ts)1 - RP);
        V acc = mk<V>((Ts)0, (Ts)0);
        Ts Rj = (Ts)1;
        if (UNROLL) {
#pragma unroll
            for (int j = 1; j <= P; ++j) {
                const V e = E[((s - j) & (P - 1)) * C + cc];
                acc.x += Rj * e.x;
                acc.y += Rj * e.y;
                Rj *= R;
            }
        } else {
            for (int j = 1; j <= P; ++j) {
                const V e = E[((s - j) & (P - 1)) * C + cc];
                acc.x += Rj * e.x;
                acc.y += Rj * e.y;
                Rj *= R;
                if (Rj < CARRY_EPS) break;
            }
        }
        const Ts cx = acc.x * inv1mRP, cy = acc.y * inv1mRP;
        Ts pw = rho;
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            v[i].x += pw * cx;
            v[i].y += pw * cy;
            pw *= rho;
        }
    } else if (active) {   // singular column: y = cumsum(t - mean t)
        V tot = mk<V>((Ts)0, (Ts)0), pre = mk<V>((Ts)0, (Ts)0);
        for (int j = 0; j < P; ++j) {
            const V e = E[j * C];
            tot.x += e.x;
            tot.y += e.y;
            if (j < s) { pre.x += e.x; pre.y += e.y; }
        }
        const Ts mx = tot.x / (Ts)n, my = tot.y / (Ts)n;
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            const Ts k = (Ts)(s * SEG + i + 1);
            v[i].x += pre.x - k * mx;
            v[i].y += pre.y - k * my;
        }
    }
    Ts wbx = (Ts)0, wby = (Ts)0;   // singular column: mean of w
    if (zero_block) {              // block-uniform
        if (zcol && active) {
            V s1 = mk<V>((Ts)0, (Ts)0), s2 = mk<V>((Ts)0, (Ts)0);
#pragma unroll
            for (int i = 0; i < SEG; ++i) {
                const Ts k = (Ts)(s * SEG + i + 1);
                s1.x += v[i].x; s1.y += v[i].y;
                s2.x += k * v[i].x; s2.y += k * v[i].y;
            }
            Zs[s] = s1;
            Zs[P + s] = s2;
        }
        __syncthreads();
        if (zcol && active) {
            V t1 = mk<V>((Ts)0, (Ts)0), t2 = mk<V>((Ts)0, (Ts)0);
            for (int j = 0; j < P; ++j) {
                t1.x += Zs[j].x; t1.y += Zs[j].y;
                t2.x += Zs[P + j].x; t2.y += Zs[P + j].y;
            }
            const Ts ybx = t1.x / (Ts)n, yby = t1.y / (Ts)n;
            const Ts tri = (Ts)0.5 * (Ts)(n + 1);   // (1/n) sum_{j=1..n} j
            wbx = t2.x / (Ts)n - ybx * tri;
            wby = t2.y / (Ts)n - yby * tri;
#pragma unroll
            for (int i = 0; i < SEG; ++i) { v[i].x -= ybx; v[i].y -= yby; }
        }
    }
    // rho partials: (rho / (n c0)) |F t|^2 per corrector
    DotAcc<Ts> ax, ay;
    if (active) {
        Ts qx = (Ts)0, qy = (Ts)0;
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            qx += v[i].x * v[i].x;
            qy += v[i].y * v[i].y;
        }
        const Ts wgt = rho * inv_nc0;
        ax.add(wgt, qx);
        ay.add(wgt, qy);
    }
    // anticausal filter within the segment
#pragma unroll
    for (int i = SEG - 2; i >= 0; --i) {
        v[i].x += rho * v[i + 1].x;
        v[i].y += rho * v[i + 1].y;
    }
    if (active) B[s * C + cc] = v[0];
    __syncthreads();
    if (active) {
        Ts sc, wx, wy;
        if (!zcol) {
            V acc = mk<V>((Ts)0, (Ts)0);
            Ts Rj = (Ts)1;
            if (UNROLL) {
#pragma unroll
                for (int j = 1; j <= P; ++j) {
                    const V e = B[((s + j) & (P - 1)) * C + cc];
                    acc.x += Rj * e.x;
                    acc.y += Rj * e.y;
                    Rj *= R;
                }
            } else {
                for (int j = 1; j <= P; ++j) {
                    const V e = B[((s + j) & (P - 1)) * C + cc];
                    acc.x += Rj * e.x;
                    acc.y += Rj * e.y;
                    Rj *= R;
                    if (Rj < (Ts)1e-18) break;
                }
            }
            wx = acc.x * inv1mRP;
            wy = acc.y * inv1mRP;
            sc = rho * inv_nc0;
        } else {   // w = reverse cumsum of y, then mean-zero
            V suf = mk<V>((Ts)0, (Ts)0);
            for (int j = s + 1; j < P; ++j) { suf.x += B[j * C].x; suf.y += B[j * C].y; }
            wx = suf.x;
            wy = suf.y;
            sc = inv_nc0;
        }
        Ts pw = zcol ? (Ts)0 : rho;
#pragma unroll
        for (int i = SEG - 1; i >= 0; --i) {
            const Ts gx = zcol ? (wx - wbx) : pw * wx;
            const Ts gy = zcol ? (wy - wby) : pw * wy;
            st(s * SEG + i, k2, mk<V>((v[i].x + gx) * sc, (v[i].y + gy) * sc));
            pw *= rho;
        }
    }
    if (rho_part) {
        double sx = 0.0, sy = 0.0;
        block_sum2(ax, ay, red, sx, sy);
        if (tid == 0) { rho_part[0] = sx; rho_part[1] = sy; }
    }
}

// The column pass of the 2D pipeline: the root from the table (delta = 0)
// or, rarely, computed in FP64 for the shift delta.
template <typename V, int LOG2N, typename Ld, typename St>
__device__ __forceinline__ void col_solve_body(Ld&& ld, St&& st, const RDesc& d, int c0,
                                               V* smem, const Tables& tb, double delta,
                                               double* red, double* rho_part,
                                               typename ScalarOf<V>::T* csc) {
    typedef typename ScalarOf<V>::T Ts;
    constexpr int n = 1 << LOG2N;
    col_solve_core<V, LOG2N>(
        ld, st,
        [&](int k2) -> Ts {
            return (delta == 0.0) ? rho_table<Ts>(tb, n)[k2]
                                  : (Ts)filter_root(tb.lap[n + k2] + delta / d.c0);
        },
        d, c0, smem, tb, delta, red, rho_part, csc);
}

}  // namespace rve
