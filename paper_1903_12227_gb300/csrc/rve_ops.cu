// rve_ops.cu -- field generation, right-hand sides, stiffness apply,
// homogenized matrix and its adjoint (sm_103a).
#include <cuda_runtime.h>

#include <algorithm>

#include "rve_ahom.cuh"
#include "rve_common.cuh"
#include "rve_internal.h"

namespace rve {

// uniform integer below n: high word of the 128-bit product (Lemire 2019,
// no rejection)
__device__ __forceinline__ int uniform_below(uint64_t v, uint32_t n) {
    return (int)__umul64hi(v, (uint64_t)n);
}
constexpr uint32_t TAG_CORNER = 1u;

// One thread per (inclusion, row of its square): sets the square's cells of
// that row in the bitmask (Eq. "Stoch-decomp": the covered set is the union
// of the inclusions, overlaps allowed, periodic wrap).
__global__ void k_gen_field(const __grid_constant__ DescChunk ch, uint32_t* __restrict__ mask) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= ch.start[ch.count]) return;
    const int b = find_real(ch.start, ch.count, (int)gid);
    const RDesc& d = ch.d[b];
    const int w = (int)gid - ch.start[b];
    const int k = w / d.s, d1 = w - k * d.s;
    const int c1 = uniform_below(sm64_draw(d.key, TAG_CORNER, 2ull * k), (uint32_t)d.n);
    const int c2 = uniform_below(sm64_draw(d.key, TAG_CORNER, 2ull * k + 1), (uint32_t)d.n);
    const int i1 = (c1 + d1) & (d.n - 1);
    uint32_t* row = mask + d.word_off + (((int64_t)i1 * d.n) >> 5);
    // columns c2 .. c2+s-1 (mod n), split at the wrap, then into words
    int j = c2, left = d.s;
    while (left > 0) {
        const int run = min(left, d.n - j);   // until the wrap
        int jj = j, rl = run;
        while (rl > 0) {
            const int bit = jj & 31;
            const int take = min(rl, 32 - bit);
            const uint32_t m = (take == 32) ? 0xffffffffu : (((1u << take) - 1u) << bit);
            atomicOr(row + (jj >> 5), m);
            jj += take;
            rl -= take;
        }
        left -= run;
        j = 0;
    }
}

// ------------------------------------------------------ RHS / stiffness --
// Work unit = 256 nodes (n*n is a multiple of 1024 for n >= 32).
constexpr int NODE_TILE = 256;

__global__ void k_rhs(const __grid_constant__ DescChunk ch, CoefSrc cs, double2* __restrict__ f) {
    const int b = find_real(ch.start, ch.count, blockIdx.x);
    const RDesc& d = ch.d[b];
    const int64_t node = (int64_t)(blockIdx.x - ch.start[b]) * NODE_TILE + threadIdx.x;
    const int i = (int)(node >> d.log2n), j = (int)(node & (d.n - 1));
    f[d.node_off + node] = rhs_at(cells_at(cs, d, i, j), d.h);
}

// Cell values a_c from the bitmask and the two values (one thread per cell).
__global__ void k_coef_from_mask(const __grid_constant__ DescChunk ch, const uint32_t* __restrict__ mask,
                                 double* __restrict__ coef) {
    const int b = find_real(ch.start, ch.count, blockIdx.x);
    const RDesc& d = ch.d[b];
    const int64_t cell = (int64_t)(blockIdx.x - ch.start[b]) * NODE_TILE + threadIdx.x;
    const uint32_t w = __ldg(mask + d.word_off + (cell >> 5));
    coef[d.node_off + cell] = ((w >> (cell & 31)) & 1u) ? d.a_incl : d.a_matrix;
}

template <typename V>
__device__ __forceinline__ V ldv(const V* __restrict__ x, const RDesc& d, int i, int j) {
    return x[d.node_off + ((int64_t)(i & (d.n - 1)) << d.log2n) + (j & (d.n - 1))];
}

template <int SCHEME, typename V>
__global__ void k_stiffness(const __grid_constant__ DescChunk ch, CoefSrc cs,
                            const V* __restrict__ x, V* __restrict__ y) {
    const int b = find_real(ch.start, ch.count, blockIdx.x);
    const RDesc& d = ch.d[b];
    const int64_t node = (int64_t)(blockIdx.x - ch.start[b]) * NODE_TILE + threadIdx.x;
    const int i = (int)(node >> d.log2n), j = (int)(node & (d.n - 1));
    const CellsT<typename ScalarOf<V>::T> a = cells_as<typename ScalarOf<V>::T>(cells_at(cs, d, i, j));
    y[d.node_off + node] = stencil_apply<SCHEME, V>(
        a, ldv(x, d, i - 1, j - 1), ldv(x, d, i - 1, j), ldv(x, d, i - 1, j + 1),
        ldv(x, d, i, j - 1), ldv(x, d, i, j), ldv(x, d, i, j + 1),
        ldv(x, d, i + 1, j - 1), ldv(x, d, i + 1, j), ldv(x, d, i + 1, j + 1));
}

// y = M x, M = M1 (x) M1 the Q1 mass matrix (1D: consistent h [1/6, 2/3,
// 1/6], lumped h [0, 1, 0]), periodic 9-point (resp. 1-point) stencil: the
// load vector of a nodal load for the general-right-hand-side solve.
template <int SCHEME>
__global__ void k_mass(const __grid_constant__ DescChunk ch, const double2* __restrict__ x,
                       double2* __restrict__ y) {
    const int b = find_real(ch.start, ch.count, blockIdx.x);
    const RDesc& d = ch.d[b];
    const int64_t node = (int64_t)(blockIdx.x - ch.start[b]) * NODE_TILE + threadIdx.x;
    const int i = (int)(node >> d.log2n), j = (int)(node & (d.n - 1));
    const double h2 = d.h * d.h;
    double2 acc = make_double2(0.0, 0.0);
    if (SCHEME == 1) {
        acc = ldv(x, d, i, j);
    } else {
        const double w[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double2 v = ldv(x, d, i + a - 1, j + c - 1);
                acc.x = fma(w[a] * w[c], v.x, acc.x);
                acc.y = fma(w[a] * w[c], v.y, acc.y);
            }
    }
    y[d.node_off + node] = make_double2(h2 * acc.x, h2 * acc.y);
}

// --------------------------------------------------- Chebyshev moments --
// One step of the Chebyshev recurrence of A~ = a0 A - a1 I for both start
// vectors of every realization (the spectral-density appendix):
//   w_{k+1} = 2 A~ w_k - w_{k-1}   (first step: w_1 = A~ w_0),
// written over w_{k-1}; per tile of NODE_TILE nodes the partial sums
// w_k.w_k and w_{k+1}.w_k per start vector, from which the moments follow by
// T_2k = 2 T_k^2 - T_0 and T_{2k+1} = 2 T_{k+1} T_k - T_1 (two moments per
// operator application).  FP64 throughout.
template <int SCHEME>
__global__ void __launch_bounds__(NODE_TILE) k_cheb(const __grid_constant__ DescChunk ch,
                                                    CoefSrc cs, double a0, double a1, int first,
                                                    const double2* __restrict__ wc,
                                                    double2* __restrict__ wp,
                                                    double* __restrict__ part) {
    __shared__ double red[8];
    const int b = find_real(ch.start, ch.count, blockIdx.x);
    const RDesc& d = ch.d[b];
    const int64_t node = (int64_t)(blockIdx.x - ch.start[b]) * NODE_TILE + threadIdx.x;
    const int i = (int)(node >> d.log2n), j = (int)(node & (d.n - 1));
    const Cells4 a = cells_at(cs, d, i, j);
    const double2 Aw = stencil_apply<SCHEME, double2>(
        a, ldv(wc, d, i - 1, j - 1), ldv(wc, d, i - 1, j), ldv(wc, d, i - 1, j + 1),
        ldv(wc, d, i, j - 1), ldv(wc, d, i, j), ldv(wc, d, i, j + 1),
        ldv(wc, d, i + 1, j - 1), ldv(wc, d, i + 1, j), ldv(wc, d, i + 1, j + 1));
    const double2 w = wc[d.node_off + node];
    double2 t = make_double2(a0 * Aw.x - a1 * w.x, a0 * Aw.y - a1 * w.y);
    if (!first) {
        const double2 wm = wp[d.node_off + node];
        t = make_double2(2.0 * t.x - wm.x, 2.0 * t.y - wm.y);
    }
    wp[d.node_off + node] = t;
    const double v[4] = {w.x * w.x, w.y * w.y, t.x * w.x, t.y * w.y};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double sum = block_sum(v[k], red);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * 4 + k] = sum;
    }
}

// Moments of step k from its tile partials, one warp per realization (fixed
// order): mu[b][c][2k] and mu[b][c][2k+1] (k = 0: mu_0 = w_0.w_0, mu_1 = w_1.w_0).
__global__ void k_cheb_moments(const __grid_constant__ DescChunk ch, const double* __restrict__ part,
                               int k, int K, double* __restrict__ mu) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= ch.count) return;
    const int t0 = ch.start[b], nt = ch.start[b + 1] - t0;
    double s[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] = warp_sum_array(part + (int64_t)t0 * 4 + q, nt, 4);
    if ((threadIdx.x & 31) != 0) return;
    for (int c = 0; c < 2; ++c) {
        double* m = mu + ((int64_t)b * 2 + c) * K;
        const double cc = s[c], nc = s[2 + c];
        const double e = (k == 0) ? cc : 2.0 * cc - m[0];
        const double o = (k == 0) ? nc : 2.0 * nc - m[1];
        if (2 * k < K) m[2 * k] = e;
        if (2 * k + 1 < K) m[2 * k + 1] = o;
    }
}

// ------------------------------------------------------------- adjoint --
// grad[c] = (1/L^2) sum_ij G_ij (xi_i + P_c u_i)^T E (xi_j + P_c u_j): the
// explicit derivative of the energy form (the correctors are stationary).
// E (unit coefficient, K1 (x) M1 + M1 (x) K1) has zero row sums, so
//   x^T E y = sum_{k<l} |E_kl| (x_k - x_l)(y_k - y_l)
// with |E_kl| = w0 - w1 on the four cell edges and 2 w1 on the two
// diagonals: the quadratic forms are built from differences across the cell
// (no cancellation between O(|u|) terms, which would cost up to ~1e-10
// relative accuracy where the local energy is small).
template <int SCHEME>
__global__ void k_backward(const __grid_constant__ DescChunk ch, const double2* __restrict__ u,
                           const double* __restrict__ G, double* __restrict__ grad) {
    const int b = find_real(ch.start, ch.count, blockIdx.x);
    const RDesc& d = ch.d[b];
    const int64_t cell = (int64_t)(blockIdx.x - ch.start[b]) * NODE_TILE + threadIdx.x;
    const int c1 = (int)(cell >> d.log2n), c2 = (int)(cell & (d.n - 1));
    const double2 u00 = ldv(u, d, c1, c2), u01 = ldv(u, d, c1, c2 + 1);
    const double2 u10 = ldv(u, d, c1 + 1, c2), u11 = ldv(u, d, c1 + 1, c2 + 1);
    const double h = d.h;
    const double we = Weights<SCHEME>::w0 - Weights<SCHEME>::w1;   // edges
    const double wd = 2.0 * Weights<SCHEME>::w1;                   // diagonals
    // pairs 00-01, 00-10, 00-11, 01-10, 01-11, 10-11 (second minus first) of
    // v_1 = x_1 + phi_1 = (u00, u01, h + u10, h + u11) and
    // v_2 = x_2 + phi_2 = (u00, h + u01, u10, h + u11)
    const double d1[6] = {u01.x - u00.x,       h + (u10.x - u00.x), h + (u11.x - u00.x),
                          h + (u10.x - u01.x), h + (u11.x - u01.x), u11.x - u10.x};
    const double d2[6] = {h + (u01.y - u00.y), u10.y - u00.y,       h + (u11.y - u00.y),
                          (u10.y - u01.y) - h, u11.y - u01.y,       h + (u11.y - u10.y)};
    const double w[6] = {we, we, wd, wd, we, we};
    double e11 = 0.0, e12 = 0.0, e22 = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        e11 = fma(w[k] * d1[k], d1[k], e11);
        e12 = fma(w[k] * d1[k], d2[k], e12);
        e22 = fma(w[k] * d2[k], d2[k], e22);
    }
    const double* Gb = G + 4 * (int64_t)b;   // G is offset to the chunk's first realization
    grad[d.node_off + cell] = d.inv_vol * (Gb[0] * e11 + (Gb[1] + Gb[2]) * e12 + Gb[3] * e22);
}

// ---------------------------------------------------------------- A_hom --
// Cell-form partial sums and the final reduction (rve_ahom.cuh).
// Mixed solves: one block per strip (a_hom_strip).
template <int SCHEME>
__global__ void __launch_bounds__(256, 3)
    k_a_hom_strip(const RDesc* __restrict__ desc, const int32_t* __restrict__ start, int batch,
                  CoefSrc cs, const double2* __restrict__ u, double* __restrict__ part) {
    __shared__ double red[64];
    __shared__ float sc[5];
    const int b = find_real(start, batch, blockIdx.x);
    const RDesc d = desc[b];
    a_hom_strip<SCHEME>(d, blockIdx.x - start[b], cs, u, red, sc,
                        part + (int64_t)blockIdx.x * AHOM_NP);
}

// FP64 solves: double-double partials (16 doubles per tile).
template <int SCHEME>
__global__ void __launch_bounds__(256) k_a_hom_part_dd(const RDesc* __restrict__ desc,
                                                       const int32_t* __restrict__ start, int batch,
                                                       CoefSrc cs, const double2* __restrict__ u,
                                                       double* __restrict__ part) {
    __shared__ ddouble red[32 * AHOM_NP];
    const int b = find_real(start, batch, blockIdx.x);
    const RDesc d = desc[b];
    a_hom_tile_dd<SCHEME>(d, blockIdx.x - start[b], cs, u, red,
                          part + (int64_t)blockIdx.x * 2 * AHOM_NP);
}

template <int SCHEME>
__global__ void k_a_hom_final_dd(const RDesc* __restrict__ desc, const int32_t* __restrict__ start,
                                 int batch, const double* __restrict__ part, double* __restrict__ A,
                                 double* __restrict__ Alo, double* __restrict__ Af) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= batch) return;
    const RDesc d = desc[b];
    a_hom_finish_dd<SCHEME>(d, part + (int64_t)start[b] * 2 * AHOM_NP, start[b + 1] - start[b],
                            A + 4 * (int64_t)b, Alo ? Alo + 4 * (int64_t)b : nullptr,
                            Af ? Af + 4 * (int64_t)b : nullptr);
}

// One warp per realization.
template <int SCHEME>
__global__ void k_a_hom_final(const RDesc* __restrict__ desc, const int32_t* __restrict__ start,
                              int batch, const double* __restrict__ part, double* __restrict__ A,
                              double* __restrict__ Af) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= batch) return;
    const RDesc d = desc[b];
    a_hom_finish<SCHEME>(d, part + (int64_t)start[b] * AHOM_NP, start[b + 1] - start[b],
                         A + 4 * (int64_t)b, Af ? Af + 4 * (int64_t)b : nullptr);
}

// ------------------------------------------------------------- launchers --
// Splits the plan's realizations into chunks and calls `fn(chunk, first)`
// with start[] = prefix sums of units(d) over the chunk.
template <typename UnitsFn, typename LaunchFn>
static cudaError_t for_chunks(const Plan& p, UnitsFn units, LaunchFn fn) {
    for (int b0 = 0; b0 < p.batch; b0 += CHUNK) {
        DescChunk ch;
        ch.count = std::min(CHUNK, p.batch - b0);
        ch.start[0] = 0;
        for (int k = 0; k < ch.count; ++k) {
            ch.d[k] = p.desc[b0 + k];
            ch.start[k + 1] = ch.start[k] + (int32_t)units(ch.d[k]);
        }
        for (int k = ch.count + 1; k <= CHUNK; ++k) ch.start[k] = ch.start[ch.count];
        cudaError_t e = fn(ch, b0);
        if (e != cudaSuccess) return e;
        note_launch();
    }
    return cudaSuccess;
}

cudaError_t launch_gen_field(const Plan& p, void* /*ws*/, uint32_t* mask, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(mask, 0, sizeof(uint32_t) * (size_t)p.words, s);
    if (e != cudaSuccess) return e;
    return for_chunks(p, [](const RDesc& d) { return (int64_t)d.n_incl * d.s; },
                      [&](const DescChunk& ch, int) {
                          const int total = ch.start[ch.count];
                          if (total == 0) return cudaSuccess;
                          k_gen_field<<<(total + 255) / 256, 256, 0, s>>>(ch, mask);
                          return cudaGetLastError();
                      });
}

static int64_t node_tiles(const RDesc& d) { return ((int64_t)d.n * d.n) / NODE_TILE; }

cudaError_t launch_rhs(const Plan& p, void*, const uint32_t* mask, const double* coef, double* f,
                       cudaStream_t s) {
    CoefSrc cs{mask, coef};
    return for_chunks(p, node_tiles, [&](const DescChunk& ch, int) {
        k_rhs<<<ch.start[ch.count], NODE_TILE, 0, s>>>(ch, cs, reinterpret_cast<double2*>(f));
        return cudaGetLastError();
    });
}

cudaError_t launch_coef_from_mask(const Plan& p, const uint32_t* mask, double* coef,
                                  cudaStream_t s) {
    return for_chunks(p, node_tiles, [&](const DescChunk& ch, int) {
        k_coef_from_mask<<<ch.start[ch.count], NODE_TILE, 0, s>>>(ch, mask, coef);
        return cudaGetLastError();
    });
}

cudaError_t launch_stiffness(const Plan& p, void*, const uint32_t* mask, const double* coef,
                             int scheme, int precision, const void* x, void* y, cudaStream_t s) {
    CoefSrc cs{mask, coef};
    return for_chunks(p, node_tiles, [&](const DescChunk& ch, int) {
        const int g = ch.start[ch.count];
        if (precision == RVE_FP64) {
            const double2* xx = static_cast<const double2*>(x);
            double2* yy = static_cast<double2*>(y);
            if (scheme == RVE_Q1_LUMPED) k_stiffness<1, double2><<<g, NODE_TILE, 0, s>>>(ch, cs, xx, yy);
            else k_stiffness<0, double2><<<g, NODE_TILE, 0, s>>>(ch, cs, xx, yy);
        } else {
            const float2* xx = static_cast<const float2*>(x);
            float2* yy = static_cast<float2*>(y);
            if (scheme == RVE_Q1_LUMPED) k_stiffness<1, float2><<<g, NODE_TILE, 0, s>>>(ch, cs, xx, yy);
            else k_stiffness<0, float2><<<g, NODE_TILE, 0, s>>>(ch, cs, xx, yy);
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_mass(const Plan& p, int scheme, const double* x, double* y, cudaStream_t s) {
    return for_chunks(p, node_tiles, [&](const DescChunk& ch, int) {
        const int g = ch.start[ch.count];
        const double2* xx = reinterpret_cast<const double2*>(x);
        double2* yy = reinterpret_cast<double2*>(y);
        if (scheme == RVE_Q1_LUMPED) k_mass<1><<<g, NODE_TILE, 0, s>>>(ch, xx, yy);
        else k_mass<0><<<g, NODE_TILE, 0, s>>>(ch, xx, yy);
        return cudaGetLastError();
    });
}

size_t cheb_workspace_size(const Plan& p) {
    int64_t tiles = 0;   // most node tiles of any launch chunk
    for (int b0 = 0; b0 < p.batch; b0 += CHUNK) {
        int64_t t = 0;
        for (int k = b0; k < std::min(p.batch, b0 + CHUNK); ++k)
            t += ((int64_t)p.desc[k].n * p.desc[k].n) / NODE_TILE;
        tiles = std::max(tiles, t);
    }
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    return 2 * up(sizeof(double2) * (size_t)p.nodes) + up(sizeof(double) * 4 * (size_t)tiles);
}

cudaError_t launch_cheb(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                        int scheme, const double* v, int K, double lo, double hi, double* mu,
                        cudaStream_t s) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* w = static_cast<char*>(ws);
    double2* wa = reinterpret_cast<double2*>(w);
    double2* wb = reinterpret_cast<double2*>(w + up(sizeof(double2) * (size_t)p.nodes));
    double* part = reinterpret_cast<double*>(w + 2 * up(sizeof(double2) * (size_t)p.nodes));
    cudaError_t e = cudaMemcpyAsync(wb, v, sizeof(double2) * (size_t)p.nodes,
                                    cudaMemcpyDeviceToDevice, s);   // w_0
    if (e != cudaSuccess) return e;
    const double a0 = 2.0 / (hi - lo), a1 = (hi + lo) / (hi - lo);
    CoefSrc cs{mask, coef};
    const int steps = (K + 1) / 2;
    return for_chunks(p, node_tiles, [&](const DescChunk& ch, int first_real) {
        const int g = ch.start[ch.count];
        double* m = mu + (int64_t)first_real * 2 * K;
        double2* cur = wb;    // w_k
        double2* oth = wa;    // in: w_{k-1}, out: w_{k+1}
        for (int k = 0; k < steps; ++k) {
            if (scheme == RVE_Q1_LUMPED)
                k_cheb<1><<<g, NODE_TILE, 0, s>>>(ch, cs, a0, a1, k == 0, cur, oth, part);
            else
                k_cheb<0><<<g, NODE_TILE, 0, s>>>(ch, cs, a0, a1, k == 0, cur, oth, part);
            k_cheb_moments<<<(ch.count + 7) / 8, 256, 0, s>>>(ch, part, k, K, m);
            note_launch(2);
            const cudaError_t le = cudaGetLastError();
            if (le != cudaSuccess) return le;
            std::swap(cur, oth);
        }
        return cudaSuccess;
    });
}

cudaError_t launch_backward(const Plan& p, void*, int scheme, const double* u, const double* gradA,
                            double* grad_coef, cudaStream_t s) {
    return for_chunks(p, node_tiles, [&](const DescChunk& ch, int first) {
        const double* G = gradA + 4 * (int64_t)first;
        const double2* uu = reinterpret_cast<const double2*>(u);
        const int g = ch.start[ch.count];
        if (scheme == RVE_Q1_LUMPED) k_backward<1><<<g, NODE_TILE, 0, s>>>(ch, uu, G, grad_coef);
        else k_backward<0><<<g, NODE_TILE, 0, s>>>(ch, uu, G, grad_coef);
        return cudaGetLastError();
    });
}

cudaError_t launch_a_hom(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                         int scheme, int precision, const double* u, double* A, double* A_lo,
                         double* A_flux, cudaStream_t s) {
    char* w = static_cast<char*>(ws);
    const RDesc* desc = reinterpret_cast<const RDesc*>(w + p.o_desc);
    const int32_t* start = reinterpret_cast<const int32_t*>(w + p.o_startA);
    double* part = reinterpret_cast<double*>(w + p.o_partA);
    CoefSrc cs{mask, coef};
    const double2* uu = reinterpret_cast<const double2*>(u);
    const bool lumped = scheme == RVE_Q1_LUMPED;
    const int gf = (p.batch + 7) / 8;
    if (precision == RVE_FP64) {
        if (lumped) k_a_hom_part_dd<1><<<p.tilesA, 256, 0, s>>>(desc, start, p.batch, cs, uu, part);
        else k_a_hom_part_dd<0><<<p.tilesA, 256, 0, s>>>(desc, start, p.batch, cs, uu, part);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (lumped) k_a_hom_final_dd<1><<<gf, 256, 0, s>>>(desc, start, p.batch, part, A, A_lo, A_flux);
        else k_a_hom_final_dd<0><<<gf, 256, 0, s>>>(desc, start, p.batch, part, A, A_lo, A_flux);
    } else {
        const int32_t* start2 = reinterpret_cast<const int32_t*>(w + p.o_startA2);
        if (lumped) k_a_hom_strip<1><<<p.tilesA2, 256, 0, s>>>(desc, start2, p.batch, cs, uu, part);
        else k_a_hom_strip<0><<<p.tilesA2, 256, 0, s>>>(desc, start2, p.batch, cs, uu, part);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (lumped) k_a_hom_final<1><<<gf, 256, 0, s>>>(desc, start2, p.batch, part, A, A_flux);
        else k_a_hom_final<0><<<gf, 256, 0, s>>>(desc, start2, p.batch, part, A, A_flux);
    }
    note_launch(2);
    return cudaGetLastError();
}

}  // namespace rve
