// rve_ahom.cuh -- the homogenized matrices from the correctors, shared by
// rve_a_hom (workspace) and rve_a_hom_noalloc (library-owned scratch).
#pragma once

#include "rve_common.cuh"

namespace rve {

// ---------------------------------------------------------------- A_hom --
// Cell form of both homogenized matrices (Eqs. "Ahom_m_entry", "wg01"):
// with v_i = xi_i + P_c u_i the local values of x_i + phi_i on cell c
// (xi_1 = h(0,0,1,1), xi_2 = h(0,1,0,1) in the local order 00, 01, 10, 11)
// and E the element matrix,
//   energy  a_ij = (1/L^2) sum_c a_c v_i^T E v_j
//   flux    a_ij = mean(a) d_ij - f_j.u_i / L^2,  f_j.u_i = -sum_c a_c xi_j^T E P_c u_i,
// which equal the node forms mean(a) d_ij - (f_i.u_j + f_j.u_i - u_i.A u_j)/L^2
// and mean(a) d_ij - f_j.u_i / L^2.  E has zero row sums and non-positive
// off-diagonals, so x^T E y = sum_{k<l} |E_kl| (x_k - x_l)(y_k - y_l): with
// K = 6 (consistent) or 2 (lumped), K |E_kl| is 1 on the four cell edges and
// q = 2 (resp. 0) on the two diagonals.  The diagonal entries are sums of
// non-negative terms -- nothing cancels -- and the differences of u across a
// cell are formed exactly in double words (u split from its IEEE fields, no
// FP64 instruction), so the partial sums carry ~1e-14 relative error at the
// cost of FP32 arithmetic (GB300's FP64 pipe is ~1/64 of it).
// Per tile of 1024 cells, partial sums (K-scaled, double words per thread):
//   [0] sum a_c   [1] E_11  [2] E_12  [3] E_22  (sum a_c K v_i^T E v_j)
//   [4] P_11 [5] P_12 [6] P_21 [7] P_22  (P_ji = sum a_c K xi_j^T E P_c u_i)
constexpr int AHOM_TILE = 1024;
constexpr int AHOM_NP = 8;

// Double-word difference a - b (exact leading part).
__device__ __forceinline__ dword dw_sub(dword a, dword b) {
    const dword s = two_sum(a.hi, -b.hi);
    return {s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo))};
}

// One cell's contributions to the AHOM_NP partial sums (K-scaled double
// words): cell value a, the corrector pair at the cell's corners 00, 01, 10,
// 11 (local order), already split into double words (u[c][corner]).
template <int SCHEME>
__device__ __forceinline__ void a_hom_cell(dword a, const dword (&u)[2][4], float h,
                                           dword (&acc)[AHOM_NP]) {
    constexpr float Q = SCHEME == 0 ? 2.f : 0.f;   // K |E| on the cell diagonals
    // u differences across the cell, per corrector c: 01-00, 10-00, 11-00,
    // 10-01, 11-01, 11-10
    dword D[2][6];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const dword u00 = u[c][0], u01 = u[c][1], u10 = u[c][2], u11 = u[c][3];
        D[c][0] = dw_sub(u01, u00);
        D[c][1] = dw_sub(u10, u00);
        D[c][2] = dw_sub(u11, u00);
        D[c][3] = dw_sub(u10, u01);
        D[c][4] = dw_sub(u11, u01);
        D[c][5] = dw_sub(u11, u10);
    }
    // differences of v_i = xi_i + u_i: xi_1 = h(0,0,1,1) adds h to pairs
    // 10-00, 11-00, 10-01, 11-01; xi_2 = h(0,1,0,1) adds h to 01-00,
    // 11-00, 11-10 and -h to 10-01
    dword V1[6], V2[6];
    V1[0] = D[0][0];            V2[0] = dw_add(D[1][0], h);
    V1[1] = dw_add(D[0][1], h); V2[1] = D[1][1];
    V1[2] = dw_add(D[0][2], h); V2[2] = dw_add(D[1][2], h);
    V1[3] = dw_add(D[0][3], h); V2[3] = dw_add(D[1][3], -h);
    V1[4] = dw_add(D[0][4], h); V2[4] = D[1][4];
    V1[5] = D[0][5];            V2[5] = dw_add(D[1][5], h);
    dword e11{0.f, 0.f}, e12{0.f, 0.f}, e22{0.f, 0.f};
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        const float wgt = (p == 2 || p == 3) ? Q : 1.f;   // diagonals 00-11, 01-10
        if (wgt == 0.f) continue;
        dw_acc(e11, dw_scale2(dw_mul(V1[p], V1[p]), wgt));
        dw_acc(e12, dw_scale2(dw_mul(V1[p], V2[p]), wgt));
        dw_acc(e22, dw_scale2(dw_mul(V2[p], V2[p]), wgt));
    }
    // xi_j^T (K E) P_c u_i = sum_pairs K|E_kl| (xi_k - xi_l)(u_k - u_l):
    //   xi_1: h (D10 + Q D11 + Q D(10-01) + D(11-01))
    //   xi_2: h (D01 + Q D11 - Q D(10-01) + D(11-10))
    dword F[2][2];   // F[j][i]
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const dword qd11 = dw_scale2(D[c][2], Q), qd1001 = dw_scale2(D[c][3], Q);
        F[0][c] = dw_scale2(dw_add(dw_add(D[c][1], qd11), dw_add(qd1001, D[c][4])), h);
        F[1][c] = dw_scale2(dw_add(dw_add(D[c][0], qd11), dw_add(dw_neg(qd1001), D[c][5])), h);
    }
    dw_acc(acc[0], a);
    dw_acc(acc[1], dw_mul(a, e11));
    dw_acc(acc[2], dw_mul(a, e12));
    dw_acc(acc[3], dw_mul(a, e22));
    dw_acc(acc[4], dw_mul(a, F[0][0]));
    dw_acc(acc[5], dw_mul(a, F[0][1]));
    dw_acc(acc[6], dw_mul(a, F[1][0]));
    dw_acc(acc[7], dw_mul(a, F[1][1]));
}

// The AHOM_NP block sums of the per-thread partials into out[0..AHOM_NP)
// (valid in thread 0).  `red` holds 64 doubles.  Contains barriers.
__device__ __forceinline__ void a_hom_block_sums(const dword (&acc)[AHOM_NP], double* red,
                                                 double* out) {
#pragma unroll
    for (int k = 0; k < AHOM_NP; k += 2) {
        DotAcc<float> ax, ay;
        ax.hi = acc[k].hi; ax.lo = acc[k].lo;
        ay.hi = acc[k + 1].hi; ay.lo = acc[k + 1].lo;
        double sx = 0.0, sy = 0.0;
        block_sum2(ax, ay, red, sx, sy);
        if (threadIdx.x == 0) {
            out[k] = sx;
            out[k + 1] = sy;
        }
    }
}

// The two cell values and h of realization d as floats in sc[0..5)
// (thread 0 writes, then a barrier).
__device__ __forceinline__ void a_hom_scalars(const RDesc& d, float* sc) {
    if (threadIdx.x == 0) {
        const dword ai = dw_split(d.a_incl), am = dw_split(d.a_matrix);
        sc[0] = ai.hi; sc[1] = ai.lo; sc[2] = am.hi; sc[3] = am.lo;
        sc[4] = dw_split(d.h).hi;   // h = 2^-k: exact
    }
    __syncthreads();
}

// Partial sums of tile `tile` (AHOM_TILE cells from cell tile*AHOM_TILE) of
// realization d into out[0..AHOM_NP): valid in thread 0.  `red` holds 64
// doubles, `sc` 5 floats (shared).  Contains barriers.
template <int SCHEME>
__device__ __forceinline__ void a_hom_tile(const RDesc& d, int64_t tile, CoefSrc cs,
                                           const double2* __restrict__ u, double* red,
                                           float* sc, double* out) {
    a_hom_scalars(d, sc);
    const dword aI{sc[0], sc[1]}, aM{sc[2], sc[3]};
    const float h = sc[4];
    const int n = d.n;
    auto at = [&](int i, int j) {   // periodic node access
        return u[d.node_off + ((int64_t)(i & (n - 1)) << d.log2n) + (j & (n - 1))];
    };
    dword acc[AHOM_NP];
#pragma unroll
    for (int k = 0; k < AHOM_NP; ++k) acc[k] = dword{0.f, 0.f};
    const int64_t base = tile * AHOM_TILE;
    for (int t = threadIdx.x; t < AHOM_TILE; t += blockDim.x) {
        const int64_t cidx = base + t;
        const int i = (int)(cidx >> d.log2n), j = (int)(cidx & (n - 1));
        dword a;
        if (cs.coef) {
            a = dw_split(__ldg(cs.coef + d.node_off + cidx));
        } else {
            const uint32_t w = __ldg(cs.mask + d.word_off + (cidx >> 5));
            a = ((w >> (cidx & 31)) & 1u) ? aI : aM;
        }
        const double2 r00 = at(i, j), r01 = at(i, j + 1);
        const double2 r10 = at(i + 1, j), r11 = at(i + 1, j + 1);
        const dword uc[2][4] = {{dw_split(r00.x), dw_split(r01.x), dw_split(r10.x), dw_split(r11.x)},
                                {dw_split(r00.y), dw_split(r01.y), dw_split(r10.y), dw_split(r11.y)}};
        a_hom_cell<SCHEME>(a, uc, h, acc);
    }
    a_hom_block_sums(acc, red, out);
}

// Rows of a strip of a_hom_strip: min(n, AHOM_STRIP / n) rows of n cells.
constexpr int AHOM_STRIP = 8192;
__host__ __device__ constexpr int a_hom_strip_rows(int n) {
    return n < AHOM_STRIP / n ? n : AHOM_STRIP / n;
}

// Partial sums of strip `strip` (rows strip*RT .. +RT of realization d,
// RT = a_hom_strip_rows(n)) into out[0..AHOM_NP), the same cell arithmetic as
// a_hom_tile.  256 threads: min(n, 256) threads across a row band, each
// walking down a column segment of RT / (256 / min(n, 256)) rows (its
// columns j, j + 256, ... for n > 256), so every node is loaded and split
// into double words twice (as the cell below and beside it) instead of four
// times, and a block reduces up to 8192 cells instead of 1024.
template <int SCHEME>
__device__ __forceinline__ void a_hom_strip(const RDesc& d, int strip, CoefSrc cs,
                                            const double2* __restrict__ u, double* red,
                                            float* sc, double* out) {
    a_hom_scalars(d, sc);
    const dword aI{sc[0], sc[1]}, aM{sc[2], sc[3]};
    const float h = sc[4];
    const int n = d.n;
    const int RT = a_hom_strip_rows(n);
    const int W = n < 256 ? n : 256;            // threads across the band
    const int seg = RT / (256 / W);             // rows of a thread's segment
    const int col0 = threadIdx.x & (W - 1);
    const int i0 = strip * RT + (threadIdx.x / W) * seg;
    auto split2 = [&](int i, int j, dword& x, dword& y) {   // periodic node, split
        const double2 r = __ldg(u + d.node_off + ((int64_t)(i & (n - 1)) << d.log2n) + (j & (n - 1)));
        x = dw_split(r.x);
        y = dw_split(r.y);
    };
    dword acc[AHOM_NP];
#pragma unroll
    for (int k = 0; k < AHOM_NP; ++k) acc[k] = dword{0.f, 0.f};
    for (int j = col0; j < n; j += W) {
        dword uc[2][4];   // [corrector][corner 00, 01, 10, 11]
        split2(i0, j, uc[0][0], uc[1][0]);
        split2(i0, j + 1, uc[0][1], uc[1][1]);
        for (int i = i0; i < i0 + seg; ++i) {
            split2(i + 1, j, uc[0][2], uc[1][2]);
            split2(i + 1, j + 1, uc[0][3], uc[1][3]);
            const int64_t cidx = ((int64_t)i << d.log2n) + j;
            dword a;
            if (cs.coef) {
                a = dw_split(__ldg(cs.coef + d.node_off + cidx));
            } else {
                const uint32_t w = __ldg(cs.mask + d.word_off + (cidx >> 5));
                a = ((w >> (cidx & 31)) & 1u) ? aI : aM;
            }
            a_hom_cell<SCHEME>(a, uc, h, acc);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                uc[c][0] = uc[c][2];
                uc[c][1] = uc[c][3];
            }
        }
    }
    a_hom_block_sums(acc, red, out);
}

// FP64 form of a_hom_tile (the A_hom of FP64 solves): the same cell sums in
// double-double arithmetic on the FP64 pipe.  Differences of u across a cell
// are exact (TwoSum), products and sums carry ~106 bits, so the only error
// left in A_hom is that of the correctors themselves -- which enters the
// energy form only quadratically (it is stationary at the exact solution).
// Partials out[2k], out[2k+1] = (hi, lo) of the same eight sums, valid in
// thread 0; `red` holds 32 * AHOM_NP ddouble (shared).  Contains barriers.
template <int SCHEME>
__device__ __forceinline__ void a_hom_tile_dd(const RDesc& d, int64_t tile, CoefSrc cs,
                                              const double2* __restrict__ u, ddouble* red,
                                              double* out) {
    const double h = d.h;
    constexpr double Q = SCHEME == 0 ? 2.0 : 0.0;   // K |E| on the cell diagonals
    const int n = d.n;
    auto at = [&](int i, int j) {   // periodic node access
        return u[d.node_off + ((int64_t)(i & (n - 1)) << d.log2n) + (j & (n - 1))];
    };
    ddouble acc[AHOM_NP];
#pragma unroll
    for (int k = 0; k < AHOM_NP; ++k) acc[k] = ddouble{0.0, 0.0};
    const int64_t base = tile * AHOM_TILE;
    for (int t = threadIdx.x; t < AHOM_TILE; t += blockDim.x) {
        const int64_t cidx = base + t;
        const int i = (int)(cidx >> d.log2n), j = (int)(cidx & (n - 1));
        double a;
        if (cs.coef) {
            a = __ldg(cs.coef + d.node_off + cidx);
        } else {
            const uint32_t w = __ldg(cs.mask + d.word_off + (cidx >> 5));
            a = ((w >> (cidx & 31)) & 1u) ? d.a_incl : d.a_matrix;
        }
        const double2 r00 = at(i, j), r01 = at(i, j + 1);
        const double2 r10 = at(i + 1, j), r11 = at(i + 1, j + 1);
        // exact u differences per corrector: 01-00, 10-00, 11-00, 10-01,
        // 11-01, 11-10
        ddouble D[2][6];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const double u00 = c ? r00.y : r00.x, u01 = c ? r01.y : r01.x;
            const double u10 = c ? r10.y : r10.x, u11 = c ? r11.y : r11.x;
            D[c][0] = dd_sub(u01, u00);
            D[c][1] = dd_sub(u10, u00);
            D[c][2] = dd_sub(u11, u00);
            D[c][3] = dd_sub(u10, u01);
            D[c][4] = dd_sub(u11, u01);
            D[c][5] = dd_sub(u11, u10);
        }
        // differences of v_i = xi_i + u_i (as in a_hom_tile)
        ddouble V1[6], V2[6];
        V1[0] = D[0][0];            V2[0] = dd_add(D[1][0], h);
        V1[1] = dd_add(D[0][1], h); V2[1] = D[1][1];
        V1[2] = dd_add(D[0][2], h); V2[2] = dd_add(D[1][2], h);
        V1[3] = dd_add(D[0][3], h); V2[3] = dd_add(D[1][3], -h);
        V1[4] = dd_add(D[0][4], h); V2[4] = D[1][4];
        V1[5] = D[0][5];            V2[5] = dd_add(D[1][5], h);
        ddouble e11{0.0, 0.0}, e12{0.0, 0.0}, e22{0.0, 0.0};
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            const double wgt = (p == 2 || p == 3) ? Q : 1.0;   // diagonals 00-11, 01-10
            if (wgt == 0.0) continue;
            e11 = dd_add(e11, dd_scale2(dd_mul(V1[p], V1[p]), wgt));
            e12 = dd_add(e12, dd_scale2(dd_mul(V1[p], V2[p]), wgt));
            e22 = dd_add(e22, dd_scale2(dd_mul(V2[p], V2[p]), wgt));
        }
        ddouble F[2][2];   // F[j][i] = xi_j^T (K E) P_c u_i, as in a_hom_tile
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const ddouble qd11 = dd_scale2(D[c][2], Q), qd1001 = dd_scale2(D[c][3], Q);
            F[0][c] = dd_mul(dd_add(dd_add(D[c][1], qd11), dd_add(qd1001, D[c][4])), h);
            F[1][c] = dd_mul(dd_add(dd_add(D[c][0], qd11), dd_add(dd_neg(qd1001), D[c][5])), h);
        }
        acc[0] = dd_add(acc[0], a);
        acc[1] = dd_add(acc[1], dd_mul(e11, a));
        acc[2] = dd_add(acc[2], dd_mul(e12, a));
        acc[3] = dd_add(acc[3], dd_mul(e22, a));
        acc[4] = dd_add(acc[4], dd_mul(F[0][0], a));
        acc[5] = dd_add(acc[5], dd_mul(F[0][1], a));
        acc[6] = dd_add(acc[6], dd_mul(F[1][0], a));
        acc[7] = dd_add(acc[7], dd_mul(F[1][1], a));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < AHOM_NP; ++k) {
        const ddouble v = dd_warp_sum(acc[k]);
        if (lane == 0) red[wid * AHOM_NP + k] = v;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < AHOM_NP; ++k) {
            ddouble v = lane < nw ? red[lane * AHOM_NP + k] : ddouble{0.0, 0.0};
            v = dd_warp_sum(v);
            if (lane == 0) {
                out[2 * k] = v.hi;
                out[2 * k + 1] = v.lo;
            }
        }
    }
    __syncthreads();
}

// Energy and flux forms from the double-double tile partials (16 doubles
// per tile), by one whole warp; lane 0 writes A (rounded to FP64), A_lo (the
// low parts, nullable) and Af (nullable).
template <int SCHEME>
__device__ __forceinline__ void a_hom_finish_dd(const RDesc& d, const double* part, int nt,
                                                double* A, double* Alo, double* Af) {
    const int lane = threadIdx.x & 31;
    ddouble s[AHOM_NP];
#pragma unroll
    for (int k = 0; k < AHOM_NP; ++k) {
        ddouble v{0.0, 0.0};
        for (int t = lane; t < nt; t += 32)
            v = dd_add(v, ddouble{part[(int64_t)t * 2 * AHOM_NP + 2 * k],
                                  part[(int64_t)t * 2 * AHOM_NP + 2 * k + 1]});
        s[k] = dd_warp_sum(v);
    }
    if (lane != 0) return;
    // K L^2 is an integer below 2^53: exact
    const double kvol = (SCHEME == 0 ? 6.0 : 2.0) * (double)d.L * (double)d.L;
    const ddouble e11 = dd_div(s[1], kvol), e12 = dd_div(s[2], kvol), e22 = dd_div(s[3], kvol);
    A[0] = e11.hi;
    A[1] = e12.hi;
    A[2] = e12.hi;
    A[3] = e22.hi;
    if (Alo) {
        Alo[0] = e11.lo;
        Alo[1] = e12.lo;
        Alo[2] = e12.lo;
        Alo[3] = e22.lo;
    }
    if (Af) {
        const double nn = (double)d.n * (double)d.n;   // a power of two
        const ddouble mean_a = dd_scale2(s[0], 1.0 / nn);
        Af[0] = dd_add(mean_a, dd_div(s[4], kvol)).hi;   // P_11
        Af[1] = dd_div(s[6], kvol).hi;                   // a_12: P_21
        Af[2] = dd_div(s[5], kvol).hi;                   // a_21: P_12
        Af[3] = dd_add(mean_a, dd_div(s[7], kvol)).hi;   // P_22
    }
}

// Energy and flux forms of realization d from its nt tile partials, by one
// whole warp (results written by lane 0):
//   energy a_ij = E_ij / (K L^2),   flux a_ij = mean(a) d_ij + P_ji / (K L^2).
template <int SCHEME>
__device__ __forceinline__ void a_hom_finish(const RDesc& d, const double* part, int nt,
                                             double* A, double* Af) {
    double s[AHOM_NP];
#pragma unroll
    for (int k = 0; k < AHOM_NP; ++k) s[k] = warp_sum_array(part + k, nt, AHOM_NP);
    if ((threadIdx.x & 31) != 0) return;
    const double scale = d.inv_vol / (SCHEME == 0 ? 6.0 : 2.0);
    A[0] = s[1] * scale;
    A[1] = s[2] * scale;
    A[2] = s[2] * scale;
    A[3] = s[3] * scale;
    if (Af) {
        const double mean_a = s[0] / ((double)d.n * (double)d.n);
        Af[0] = mean_a + s[4] * scale;   // P_11
        Af[1] = s[6] * scale;            // a_12: P_21 (xi_2 with u_1)
        Af[2] = s[5] * scale;            // a_21: P_12 (xi_1 with u_2)
        Af[3] = mean_a + s[7] * scale;   // P_22
    }
}

}  // namespace rve
