// rve3d.cu -- the 3D extension of the RVE corrector method (the setting of
// Sec. 2 carries over to d = 3; the rank-3 Kronecker Laplacian of Sec. 3.2
// and Eq. "As_Kron_d"; multilinear functions on cubes, Sec. 3.1): cubes on
// the torus [0,L)^3, the trilinear Q1 element K1(x)M1(x)M1 + M1(x)K1(x)M1 +
// M1(x)M1(x)K1, three corrector problems solved by PCG with B = c0 A_Delta +
// delta I (A_Delta the periodic 7-point Laplacian), and the 3x3 homogenized
// matrix.
//
// Grid: n = L m0 nodes per axis, node (i,j,k) at ((i n + j) n + k) within
// the realization; cell (i,j,k) has lower corner node (i,j,k); local corner
// a = 4 a1 + 2 a2 + a3.  The three correctors travel as two pairs: (u_1,
// u_2) and (u_3, 0), so that every kernel -- the stencil, the Hartley
// transforms (pair-packed complex FFT) and the column solve -- works on the
// pair layout of the 2D path.
//
// Units.  The solver's unit of work is one pair of one realization.  Units
// are numbered by grid size (within a size, the pair-0 units first), and
// every launch covers the consecutive units of one size, each unit with its
// own scalars and flags; a unit that has finished makes its blocks return
// at once.  The host polls the flags every few steps.
//
// Preconditioner: the Hartley transforms along x (contiguous lines) and y
// (lines of stride n) diagonalise two factors of A_Delta; along z (lines of
// stride n^2) each (kx, ky) leaves the periodic tridiagonal system
// c0 (T + lambda(kx) + lambda(ky)) + delta, solved by the causal/anticausal
// filter pair of the 2D column pass (rve_colsolve.cuh).  B^{-1} = n^-2 Hx
// Hy M^-1 Hy Hx.
//
// Precision.  GB300 runs FP64 at 1/64 of the FP32 rate, and the 3D stencil
// and transforms carry enough arithmetic per node to be bound by it.  Both
// paths run PCG cycles (Saad, Iterative Methods for Sparse Linear Systems,
// Algorithm 9.1) on A e = r64 / s from e = 0, s = |r64|, between FP64 true
// residuals r64 = f - A u (iterative refinement, u += s e), until |r64| <=
// tol |f|.  FP64: the cycle's vectors are FP64 and it runs to the outer
// tolerance, so one cycle is textbook PCG and a second one is rare.
// Mixed: the cycle's vectors and arithmetic are FP32 and it stops at a
// relative reduction max(tol |f| / (2 |r64|), inner_tol).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>
#include <vector>

#include "rve_colsolve.cuh"
#include "rve_common.cuh"
#include "rve_internal.h"

namespace rve {

// ------------------------------------------------------------ element --
// Entry (a, b) of the element matrix (local corners 4 a1 + 2 a2 + a3).
template <int SCHEME>
__host__ __device__ __forceinline__ double e3(int a, int b, double h) {
    auto m1 = [&](int x, int y) {
        return SCHEME == 0 ? h * (x == y ? 1.0 / 3.0 : 1.0 / 6.0) : (x == y ? 0.5 * h : 0.0);
    };
    auto k1 = [&](int x, int y) { return (x == y ? 1.0 : -1.0) / h; };
    const int a1 = a >> 2, a2 = (a >> 1) & 1, a3 = a & 1;
    const int b1 = b >> 2, b2 = (b >> 1) & 1, b3 = b & 1;
    return k1(a1, b1) * m1(a2, b2) * m1(a3, b3) + m1(a1, b1) * k1(a2, b2) * m1(a3, b3) +
           m1(a1, b1) * m1(a2, b2) * k1(a3, b3);
}

// Descriptor of one unit (a corrector pair of a realization).
struct U3 {
    int32_t n, log2n, pair, pad2;
    int32_t n_incl, s;
    int32_t real;       // realization index
    int32_t partner;    // the realization's other unit
    int64_t off;        // first node of the unit's vectors
    int64_t cell_off;   // first cell (= node) of the realization: mask, coef, ABI vectors
    int64_t part_off;   // first partial (doubles) of the unit
    double am, ai, h, c0, inv_vol;
    float am32, ai32;
    uint64_t key;       // SplitMix64 key of the realization
};

// Blocks of a launch over the units of one grid size (consecutive unit ids
// from `first`): block -> (unit, block within the unit).
struct Grp {
    const U3* __restrict__ desc;
    int first;          // first unit of the launch
    int per_log2;       // log2 of the blocks per unit
};
__device__ __forceinline__ int unit_of(const Grp& g, int& lb) {
    lb = blockIdx.x & ((1 << g.per_log2) - 1);
    return g.first + (blockIdx.x >> g.per_log2);
}

// Local index of node (i, j, k) (periodic) within a realization.
__device__ __forceinline__ int l3(const U3& d, int i, int j, int k) {
    const int m = d.n - 1;
    return ((((i & m) << d.log2n) + (j & m)) << d.log2n) + (k & m);
}

// Cell values in the arithmetic type T: a byte mask with the two values, or
// an explicit array.
template <typename T> struct Cells3T {
    const uint8_t* __restrict__ mask;
    const T* __restrict__ coef;
};
template <typename T> __device__ __forceinline__ T two_values(const U3& d, bool incl);
template <> __device__ __forceinline__ double two_values<double>(const U3& d, bool incl) { return incl ? d.ai : d.am; }
template <> __device__ __forceinline__ float two_values<float>(const U3& d, bool incl) { return incl ? d.ai32 : d.am32; }

constexpr int T3 = 256;   // threads of the node kernels
constexpr int SZ = 4;     // stencil: consecutive planes per thread
constexpr int Z_THREADS = 512;   // z solve

// Block sums of two per-thread values (x, y), valid in thread 0: an xor
// butterfly within each warp in the values' own precision, then the warp
// sums in FP64 in warp order (fixed order: deterministic).  A thread's
// value sums only its own few nodes, so an FP32 tree stays short.
// `red` holds 2 * (blockDim.x / 32) doubles.
template <typename T>
__device__ __forceinline__ void block_pair_sum(T x, T y, double* red, double& sx, double& sy) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[2 * wid] = (double)x;
        red[2 * wid + 1] = (double)y;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[2 * w];
            b += red[2 * w + 1];
        }
        sx = a;
        sy = b;
    }
}

// --------------------------------------------------------------- field --
// One thread per (cube, row d1, d2): sets the s cells along the third axis.
__global__ void k3_gen_field(const U3 d, uint8_t* __restrict__ mask) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t rows = (int64_t)d.n_incl * d.s * d.s;
    if (gid >= rows) return;
    const int kk = (int)(gid / ((int64_t)d.s * d.s));
    const int r = (int)(gid - (int64_t)kk * d.s * d.s);
    const int d1 = r / d.s, d2 = r - d1 * d.s;
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        c[a] = (int)__umul64hi(sm64_draw(d.key, 1u, 3ull * kk + a), (uint64_t)d.n);
    for (int d3 = 0; d3 < d.s; ++d3) mask[d.cell_off + l3(d, c[0] + d1, c[1] + d2, c[2] + d3)] = 1;
}

// ----------------------------------------------------------- stiffness --
// y = A x for one pair.  An entry E[a][b] of the element matrix depends only
// on the number of axes along which the corners a and b differ (K1 and M1
// are symmetric with equal diagonals): e_0 = 3 m0^2 / h, e_1 = (2 m0 m1 -
// m0^2) / h, e_2 = (m1^2 - 2 m0 m1) / h, e_3 = -3 m1^2 / h with M1 = [m0 m1;
// m1 m0].  Consistent (m0 = h/3, m1 = h/6): e_0 = h/3, e_1 = 0, e_2 = e_3 =
// -h/12; lumped (m0 = h/2, m1 = 0): e_0 = 3h/4, e_1 = -h/4, e_2 = e_3 = 0.
// So the assembled row of node i couples neighbour i+o (o in {-1,0,1}^3)
// with e_{|o|} times the sum of a_c over the cells holding both nodes: all 8
// for o = 0, 4 for a face neighbour, 2 for an edge neighbour (a pair sum
// along the axis where o is 0), 1 for a corner neighbour: about 60
// operations per node and pair instead of 144 for the 8 element rows.
// A thread computes two neighbouring nodes (k0, k0 + 1) of one row in SZ
// consecutive planes; a block takes TJ = 512 / n whole rows of those planes.
// It first copies the planes i0-1 .. i0+SZ, rows j0-1 .. j0+TJ of x and the
// cell values of planes i0-1 .. i0+SZ-1, rows j0-1 .. j0+TJ-1 (whole periodic
// rows) into shared memory, every load issued before the first store, then
// each node sums the contributions of its three x-planes: from below (cells
// of plane i-1), in its own plane (both cell planes and the diagonal term)
// and from above (cells of plane i).  Per node pair and row one 16-byte and
// two 8-byte shared loads.
//   MODE_APPLY: y = A x, partials of x.y per component (the p.q of CG);
//   MODE_RESID: y = f - A x (the true residual), partials of |y|^2.
// Blocks of units whose flag (`done`, or `outer_done` for MODE_RESID) is
// set return at once.
enum { MODE_APPLY = 0, MODE_RESID = 1 };
struct MixScal;
__device__ __forceinline__ bool unit_skip(const MixScal* sc, int u, bool outer);

// Shared memory of a stiffness block for grids of n = 2^lg.
template <typename V>
__host__ __device__ constexpr size_t stiff_smem(int lg) {
    return (size_t)(SZ + 2) * (((2 * T3) >> lg) + 2) * ((size_t)1 << lg) * sizeof(V) +
           (size_t)(SZ + 1) * (((2 * T3) >> lg) + 1) * ((size_t)1 << lg) * (sizeof(V) / 2);
}

// Two consecutive elements (16-byte aligned for float2 pairs).
template <typename V> struct Two { V a, b; };
__device__ __forceinline__ Two<float2> ld_two(const float2* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ Two<double2> ld_two(const double2* p) { return {p[0], p[1]}; }
__device__ __forceinline__ void st_two(float2* p, const Two<float2>& t) {
    *reinterpret_cast<float4*>(p) = make_float4(t.a.x, t.a.y, t.b.x, t.b.y);
}
__device__ __forceinline__ void st_two(double2* p, const Two<double2>& t) { p[0] = t.a; p[1] = t.b; }
template <typename T> __device__ __forceinline__ Two<T> ld_two_s(const T* p) { return {p[0], p[1]}; }
template <> __device__ __forceinline__ Two<float> ld_two_s<float>(const float* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return {v.x, v.y};
}

// FP32: three blocks per SM (80 registers, no spills) with the register
// window below.
template <int SCHEME, int MODE, typename V>
__global__ void __launch_bounds__(T3, sizeof(V) == 8 ? (SCHEME == RVE_Q1_LUMPED ? 4 : 3) : 2)
    k3_stiffness(Grp g, Cells3T<typename ScalarOf<V>::T> cs, const V* __restrict__ x,
                 V* __restrict__ y, const V* __restrict__ f, double* part, const MixScal* sc) {
    typedef typename ScalarOf<V>::T T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[16];
    int lb;
    const int u = unit_of(g, lb);
    const U3 d = g.desc[u];   // issued before the flag test
    if (sc && unit_skip(sc, u, MODE == MODE_RESID)) return;
    const int n = d.n, m = n - 1, lg = d.log2n;
    const int TJ = (2 * T3) >> lg;                    // rows of the block
    const int first = lb * (2 * T3);                  // (plane group, j0, 0)
    const int i0 = (first >> (2 * lg)) * SZ;
    const int j0 = (first >> lg) & m;
    const int jl = threadIdx.x >> (lg - 1), k0 = 2 * (threadIdx.x & ((n >> 1) - 1));
    const int RW = TJ + 2, CR = TJ + 1;               // rows of the x and cell tiles
    V* xt = reinterpret_cast<V*>(smem_raw);                          // [SZ+2][RW][n]
    T* ct = reinterpret_cast<T*>(xt + (SZ + 2) * RW * n);            // [SZ+1][CR][n]
    const V* __restrict__ xu = x + d.off;
    const T am = two_values<T>(d, false), ai = two_values<T>(d, true);
    const uint8_t* __restrict__ mk8 = cs.mask + d.cell_off;
    const T* __restrict__ cf = cs.coef ? cs.coef + d.cell_off : nullptr;
    // copy: thread (jl, k0) takes elements k0, k0+1 of tile rows jl, jl + TJ
    // (those below RW, resp. CR) of each plane; x by asynchronous 16-byte
    // copies (no registers held), the cell values through registers (they
    // are converted), every load issued before the first store
    constexpr int CHUNKS = (int)(2 * sizeof(V) / 16);   // 16-byte pieces of two elements
#pragma unroll
    for (int pl = 0; pl < SZ + 2; ++pl) {
        const int gp = ((i0 - 1 + pl) & m) << (2 * lg);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int rr = jl + q * TJ;
            if (rr < RW) {
                const char* gsrc = reinterpret_cast<const char*>(xu + gp + (((j0 - 1 + rr) & m) << lg) + k0);
                const unsigned sdst = (unsigned)__cvta_generic_to_shared(xt + (pl * RW + rr) * n + k0);
#pragma unroll
                for (int c = 0; c < CHUNKS; ++c)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sdst + 16 * c),
                                 "l"(gsrc + 16 * c)
                                 : "memory");
            }
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    Two<T> cr[SZ + 1][2];
#pragma unroll
    for (int pl = 0; pl < SZ + 1; ++pl) {
        const int gp = ((i0 - 1 + pl) & m) << (2 * lg);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int rr = jl + q * TJ;
            if (rr < CR) {
                const int idx = gp + (((j0 - 1 + rr) & m) << lg) + k0;
                if (cf) {
                    cr[pl][q] = ld_two_s(cf + idx);
                } else {
                    const uchar2 mb = *reinterpret_cast<const uchar2*>(mk8 + idx);
                    cr[pl][q] = {mb.x ? ai : am, mb.y ? ai : am};
                }
            }
        }
    }
#pragma unroll
    for (int pl = 0; pl < SZ + 1; ++pl)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int rr = jl + q * TJ;
            if (rr < CR) {
                T* c = ct + (pl * CR + rr) * n + k0;
                c[0] = cr[pl][q].a;
                c[1] = cr[pl][q].b;
            }
        }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    const int kl = (k0 - 1) & m, kr = (k0 + 2) & m;
    const T h = (T)d.h;
    // the cell bit that a neighbour offset fixes on its axis: +1 -> 0, -1 -> 1
    auto cb = [](int o) { return o > 0 ? 0 : 1; };
    const T e0 = SCHEME == RVE_Q1_CONSISTENT ? h * (T)(1.0 / 3.0) : h * (T)0.75;
    const T eo = SCHEME == RVE_Q1_CONSISTENT ? -h * (T)(1.0 / 12.0) : -h * (T)0.25;
    // C[q]: the cell at (j - c2, k - c3) of a cell plane, q = 2 c2 + c3;
    // X[a][b]: x at (j + a - 1, k + b - 1) of an x-plane
    auto side = [&](const V (&X)[3][3], const T (&C)[4]) -> V {   // off-plane couplings
        T sx = 0, sy = 0;
        if (SCHEME == RVE_Q1_CONSISTENT) {
#pragma unroll
            for (int s2 = -1; s2 <= 1; s2 += 2) {
                const T wy = C[cb(s2)] + C[2 + cb(s2)];           // edge (., 0, s2)
                sx = fma(wy, X[1][1 + s2].x, sx);
                sy = fma(wy, X[1][1 + s2].y, sy);
                const T wz = C[2 * cb(s2)] + C[2 * cb(s2) + 1];   // edge (., s2, 0)
                sx = fma(wz, X[1 + s2][1].x, sx);
                sy = fma(wz, X[1 + s2][1].y, sy);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {                          // corners (., o2, o3)
                const int o2 = (c & 2) ? 1 : -1, o3 = (c & 1) ? 1 : -1;
                const T w = C[2 * cb(o2) + cb(o3)];
                sx = fma(w, X[1 + o2][1 + o3].x, sx);
                sy = fma(w, X[1 + o2][1 + o3].y, sy);
            }
        } else {                                                    // face (., 0, 0)
            const T w = (C[0] + C[1]) + (C[2] + C[3]);
            sx = w * X[1][1].x;
            sy = w * X[1][1].y;
        }
        return mk<V>(eo * sx, eo * sy);
    };
    auto inplane = [&](const V (&X)[3][3], const T (&Cm)[4], const T (&C0)[4]) -> V {
        T px[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) px[q] = Cm[q] + C0[q];
        const T A0 = (px[0] + px[1]) + (px[2] + px[3]);
        T sx = 0, sy = 0;
        if (SCHEME == RVE_Q1_CONSISTENT) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {                          // edges (0, s1, s2)
                const int s1 = (c & 2) ? 1 : -1, s2 = (c & 1) ? 1 : -1;
                const T w = px[2 * cb(s1) + cb(s2)];
                sx = fma(w, X[1 + s1][1 + s2].x, sx);
                sy = fma(w, X[1 + s1][1 + s2].y, sy);
            }
        } else {
#pragma unroll
            for (int sg = -1; sg <= 1; sg += 2) {
                const int v0 = cb(sg);
                const T wj = px[2 * v0] + px[2 * v0 + 1];           // face (0, sg, 0)
                sx = fma(wj, X[1 + sg][1].x, sx);
                sy = fma(wj, X[1 + sg][1].y, sy);
                const T wk = px[v0] + px[2 + v0];                   // face (0, 0, sg)
                sx = fma(wk, X[1][1 + sg].x, sx);
                sy = fma(wk, X[1][1 + sg].y, sy);
            }
        }
        const T dA = e0 * A0;
        return mk<V>(fma(eo, sx, dA * X[1][1].x), fma(eo, sy, dA * X[1][1].y));
    };
    // cells of tile plane pl for the two nodes
    auto cells = [&](int pl, T (&c0)[4], T (&c1)[4]) {
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
            const T* r = ct + (pl * CR + jl + 1 - c2) * n;
            const Two<T> M = ld_two_s(r + k0);
            const T Lv = r[kl];
            c0[2 * c2] = M.a;       // node k0: c3 = 0 -> k0, c3 = 1 -> k0 - 1
            c0[2 * c2 + 1] = Lv;
            c1[2 * c2] = M.b;       // node k0 + 1: c3 = 0 -> k0 + 1, c3 = 1 -> k0
            c1[2 * c2 + 1] = M.a;
        }
    };
    T dx = 0, dy = 0;
    // adds the couplings through x-plane t + o1 (X0, X1: [row][k] windows of
    // the two nodes) to acc0, acc1; cell planes t - 1 (Cm*) and t (C0*)
    auto couple = [&](int o1, const V (&X0)[3][3], const V (&X1)[3][3], const T (&Cm0)[4],
                      const T (&Cm1)[4], const T (&C00)[4], const T (&C01)[4], V& acc0, V& acc1) {
        V v0, v1;
        if (o1 < 0) { v0 = side(X0, Cm0); v1 = side(X1, Cm1); }
        else if (o1 == 0) { v0 = inplane(X0, Cm0, C00); v1 = inplane(X1, Cm1, C01); }
        else { v0 = side(X0, C00); v1 = side(X1, C01); }
        acc0.x += v0.x; acc0.y += v0.y;
        acc1.x += v1.x; acc1.y += v1.y;
    };
    // output plane t of the two nodes (xa, xb: their own x values)
    auto emit = [&](int t, V acc0, V acc1, const V& xa, const V& xb) {
        const int64_t node = d.off + ((int64_t)(i0 + t) << (2 * lg)) + ((j0 + jl) << lg) + k0;
        if (MODE == MODE_RESID) {
            const Two<V> ff = ld_two(f + node);
            acc0.x = ff.a.x - acc0.x; acc0.y = ff.a.y - acc0.y;
            acc1.x = ff.b.x - acc1.x; acc1.y = ff.b.y - acc1.y;
            dx = fma(acc0.x, acc0.x, fma(acc1.x, acc1.x, dx));
            dy = fma(acc0.y, acc0.y, fma(acc1.y, acc1.y, dy));
        } else {
            dx = fma(xa.x, acc0.x, fma(xb.x, acc1.x, dx));
            dy = fma(xa.y, acc0.y, fma(xb.y, acc1.y, dy));
        }
        st_two(y + node, Two<V>{acc0, acc1});
    };
    if constexpr (sizeof(T) == 4) {
        // FP32: a window of three x-planes (rows jl .. jl + 2, k0 - 1 ..
        // k0 + 2) and two cell planes rolls down the block's planes in
        // registers, so each tile plane is read from shared memory once
        // instead of three times and each cell plane once instead of twice.
        // The arithmetic and its order are those of the FP64 branch.
        V W[3][3][4];
        auto xplane = [&](int pl, V (&P)[3][4]) {
#pragma unroll
            for (int a2 = 0; a2 < 3; ++a2) {
                const V* r = xt + (pl * RW + jl + a2) * n;
                const Two<V> M = ld_two(r + k0);
                P[a2][0] = r[kl];
                P[a2][1] = M.a;
                P[a2][2] = M.b;
                P[a2][3] = r[kr];
            }
        };
        auto step = [&](int t, const T (&Cm0)[4], const T (&Cm1)[4], const T (&C00)[4],
                        const T (&C01)[4]) {
            V acc0 = mk<V>((T)0, (T)0), acc1 = acc0;
#pragma unroll
            for (int o1 = -1; o1 <= 1; ++o1) {
                const V (&P)[3][4] = W[(t + 1 + o1) % 3];
                V X0[3][3], X1[3][3];
#pragma unroll
                for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        X0[a2][q] = P[a2][q];
                        X1[a2][q] = P[a2][q + 1];
                    }
                couple(o1, X0, X1, Cm0, Cm1, C00, C01, acc0, acc1);
            }
            const V (&P0)[3][4] = W[(t + 1) % 3];
            emit(t, acc0, acc1, P0[1][1], P0[1][2]);
        };
        T Ca0[4], Ca1[4], Cb0[4], Cb1[4];
        xplane(0, W[0]);
        xplane(1, W[1]);
        cells(0, Ca0, Ca1);
#pragma unroll
        for (int t = 0; t < SZ; ++t) {
            xplane(t + 2, W[(t + 2) % 3]);
            if (t % 2 == 0) {
                cells(t + 1, Cb0, Cb1);
                step(t, Ca0, Ca1, Cb0, Cb1);
            } else {
                cells(t + 1, Ca0, Ca1);
                step(t, Cb0, Cb1, Ca0, Ca1);
            }
        }
    } else {
        // FP64: a register window would not fit; each plane step reads its
        // three x-planes and two cell planes from shared memory
#pragma unroll 1
        for (int t = 0; t < SZ; ++t) {
            T Cm0[4], Cm1[4], C00[4], C01[4];
            cells(t, Cm0, Cm1);
            cells(t + 1, C00, C01);
            V acc0 = mk<V>((T)0, (T)0), acc1 = acc0;
#pragma unroll
            for (int o1 = -1; o1 <= 1; ++o1) {
                V X0[3][3], X1[3][3];
#pragma unroll
                for (int a2 = 0; a2 < 3; ++a2) {
                    const V* r = xt + ((t + 1 + o1) * RW + jl + a2) * n;
                    const Two<V> M = ld_two(r + k0);
                    const V Lv = r[kl], Rv = r[kr];
                    X0[a2][0] = Lv;  X0[a2][1] = M.a; X0[a2][2] = M.b;
                    X1[a2][0] = M.a; X1[a2][1] = M.b; X1[a2][2] = Rv;
                }
                couple(o1, X0, X1, Cm0, Cm1, C00, C01, acc0, acc1);
            }
            const Two<V> xc = ld_two(xt + ((t + 1) * RW + jl + 1) * n + k0);
            emit(t, acc0, acc1, xc.a, xc.b);
        }
    }
    if (part) {   // block-uniform
        double tx = 0.0, ty = 0.0;
        block_pair_sum(dx, dy, red, tx, ty);
        if (threadIdx.x == 0) {
            part[d.part_off + 2 * lb] = tx;
            part[d.part_off + 2 * lb + 1] = ty;
        }
    }
}

// ------------------------------------------- double-word true residual --
// The mixed path's true residual r64 = f - A u without FP64 arithmetic per
// node (GB300's FP64 pipe is ~1/64 of FP32): u is split once into double
// words (hi, lo floats from its IEEE fields, k3_split_dw), and the row of
// node i is scaled by K = 12/h (consistent) or 4/h (lumped), which makes
// every Hamming-distance weight an integer multiple of a sum of cell values:
//   consistent  K e = (4, 0, -1, -1)    K r = K f - 4 S8 u_i + sum_edges S2 u + sum_corners S1 u
//   lumped      K e = (3, -1, 0, 0)     K r = K f - 3 S8 u_i + sum_faces S4 u
// (S_m the sum of the m cells the two nodes share).  The sum is a
// compensated dot product of double words (DotDW: the products' rounding
// errors gather in a compensation term), so its absolute error is
// O(eps_32^2) times the size of its terms -- far below the outer tolerance
// -- like the 2D refinement pass.  One node per thread; the neighbours'
// double words come through L1.  Partials: |r|^2 per component (FP32 per
// thread, 256 nodes per block).
__global__ void __launch_bounds__(T3) k3_split_dw(Grp g, const double2* __restrict__ u,
                                                  float4* __restrict__ w, const MixScal* sc) {
    int lb;
    const int un = unit_of(g, lb);
    const U3 d = g.desc[un];
    if (unit_skip(sc, un, true)) return;
    const int64_t node = d.off + (int64_t)lb * T3 + threadIdx.x;
    const double2 v = u[node];
    const dword x = dw_split(v.x), y = dw_split(v.y);
    w[node] = make_float4(x.hi, y.hi, x.lo, y.lo);
}

// EXACT: both cell values are integers of magnitude <= 2^20 (the paper's
// two-valued coefficients), so every cell sum below (at most 8 cells, below
// 2^24) and its power-of-two scalings are exact in one float; the weights
// are then floats instead of double words, with the same values and so the
// same result.
template <int SCHEME, bool EXACT>
__device__ __forceinline__ void resid_dw_body(const U3& d, int lb, Cells3T<double> cs,
                                              const float4* __restrict__ w,
                                              const double2* __restrict__ f,
                                              double2* __restrict__ r, double* part,
                                              double* red) {
    typedef std::conditional_t<EXACT, float, dword> CW;
    auto wadd = [](CW x, CW y) -> CW {
        if constexpr (EXACT) return __fadd_rn(x, y); else return dw_add(x, y);
    };
    auto wneg = [](CW x) -> CW {
        if constexpr (EXACT) return -x; else return dw_neg(x);
    };
    auto wscale2 = [](CW x, float p2) -> CW {
        if constexpr (EXACT) return x * p2; else return dw_scale2(x, p2);
    };
    const int lg = d.log2n;
    const int loc = lb * T3 + threadIdx.x;
    const int i = loc >> (2 * lg), j = (loc >> lg) & (d.n - 1), k = loc & (d.n - 1);
    const float4* __restrict__ wu = w + d.off;
    const dword aI = dw_split(d.ai), aM = dw_split(d.am);
    // the 8 cells around the node: C[4 c1 + 2 c2 + c3] = cell (i - c1, j - c2, k - c3)
    CW C[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int idx = l3(d, i - (q >> 2), j - ((q >> 1) & 1), k - (q & 1));
        if constexpr (EXACT) {   // mask only
            C[q] = __ldg(cs.mask + d.cell_off + idx) ? aI.hi : aM.hi;
        } else {
            if (cs.coef) C[q] = dw_split(__ldg(cs.coef + d.cell_off + idx));
            else C[q] = __ldg(cs.mask + d.cell_off + idx) ? aI : aM;
        }
    }
    // the cell bit an offset fixes on its axis: +1 -> 0, -1 -> 1
    auto cb = [](int o) { return o > 0 ? 0 : 1; };
    // K = 12/h or 4/h: an integer (h = 1/m0)
    const float K = (SCHEME == 0 ? 12.f : 4.f) * rintf((float)(1.0 / d.h));
    const double2 ff = f[d.off + loc];
    DotDW rx(dw_mulf(dw_split(ff.x), K)), ry(dw_mulf(dw_split(ff.y), K));
    auto term = [&](CW wgt, int o1, int o2, int o3) {   // r -= wgt * u(i + o)
        const float4 v = wu[l3(d, i + o1, j + o2, k + o3)];
        const CW nw = wneg(wgt);
        rx.add(nw, v.x, v.z);
        ry.add(nw, v.y, v.w);
    };
    const CW S8 = wadd(wadd(wadd(C[0], C[1]), wadd(C[2], C[3])),
                       wadd(wadd(C[4], C[5]), wadd(C[6], C[7])));
    term(wscale2(S8, SCHEME == 0 ? 4.f : 2.f), 0, 0, 0);
    if (SCHEME != 0) term(S8, 0, 0, 0);   // 3 S8 = 2 S8 + S8 (exact scalings only)
#pragma unroll
    for (int o1 = -1; o1 <= 1; ++o1)
#pragma unroll
        for (int o2 = -1; o2 <= 1; ++o2)
#pragma unroll
            for (int o3 = -1; o3 <= 1; ++o3) {
                const int zeros = (o1 == 0) + (o2 == 0) + (o3 == 0);
                if (zeros == 3) continue;
                if (SCHEME == 0 && zeros == 2) continue;   // faces: K e_1 = 0
                if (SCHEME != 0 && zeros != 2) continue;   // lumped: faces only
                // sum of the cells shared with the neighbour: the bits of
                // the non-zero offsets are fixed, the others run over 0, 1
                CW S{};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int c1 = q >> 2, c2 = (q >> 1) & 1, c3 = q & 1;
                    if (o1 != 0 && c1 != cb(o1)) continue;
                    if (o2 != 0 && c2 != cb(o2)) continue;
                    if (o3 != 0 && c3 != cb(o3)) continue;
                    S = wadd(S, C[q]);
                }
                term(wneg(S), o1, o2, o3);   // K e = -1: r += S u
            }
    const double invK = 1.0 / (double)K;
    const double rxd = ((double)rx.s + (double)rx.comp) * invK;
    const double ryd = ((double)ry.s + (double)ry.comp) * invK;
    r[d.off + loc] = make_double2(rxd, ryd);
    if (part) {
        const float fx = (float)rxd, fy = (float)ryd;
        double tx = 0.0, ty = 0.0;
        block_pair_sum(fx * fx, fy * fy, red, tx, ty);
        if (threadIdx.x == 0) {
            part[d.part_off + 2 * lb] = tx;
            part[d.part_off + 2 * lb + 1] = ty;
        }
    }
}

template <int SCHEME>
__global__ void __launch_bounds__(T3) k3_resid_dw(Grp g, Cells3T<double> cs,
                                                  const float4* __restrict__ w,
                                                  const double2* __restrict__ f,
                                                  double2* __restrict__ r, double* part,
                                                  const MixScal* sc) {
    __shared__ double red[16];
    int lb;
    const int un = unit_of(g, lb);
    const U3 d = g.desc[un];
    if (unit_skip(sc, un, true)) return;
    auto small_int = [](double a) { return a == floor(a) && fabs(a) <= 1048576.0; };
    if (!cs.coef && small_int(d.ai) && small_int(d.am))
        resid_dw_body<SCHEME, true>(d, lb, cs, w, f, r, part, red);
    else
        resid_dw_body<SCHEME, false>(d, lb, cs, w, f, r, part, red);
}

// -------------------------------------------------------------- loads --
// Corrector loads f_i = -sum_c a_c P_c^T E xi_i (xi_i = h x corner bit i).
// Every row of M1 sums to h/2 (both schemes) and every row of K1 to 0, so
// of the three Kronecker terms only the one with K1 along axis i survives,
// and the row of E xi_i at local corner l is (h^2/4) (+1 if l_i = 1, -1
// otherwise).  Summed over the 8 cells around the node (the node is corner
// c of the cell at offset -c):
//     f_i = (h^2/4) (sum_{c_i = 0} a_c - sum_{c_i = 1} a_c),
// which is exactly zero where the 8 cells agree.  Unit pair 0 gets (f_1,
// f_2), pair 1 gets (f_3, 0).  Also the partials of |f|^2.
__global__ void __launch_bounds__(T3) k3_rhs(Grp g, Cells3T<double> cs, double2* __restrict__ f,
                                             double* part) {
    __shared__ double red[32];
    int lb;
    const int u = unit_of(g, lb);
    const U3& d = g.desc[u];
    const int local = lb * T3 + threadIdx.x;
    const int n = d.n;
    const int i = local >> (2 * d.log2n), j = (local >> d.log2n) & (n - 1), k = local & (n - 1);
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int idx = l3(d, i - (c >> 2), j - ((c >> 1) & 1), k - (c & 1));
        a[c] = cs.coef ? cs.coef[d.cell_off + idx] : two_values<double>(d, cs.mask[d.cell_off + idx] != 0);
    }
    const double q = 0.25 * d.h * d.h;
    double v[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        double lo = 0.0, hi = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if ((c >> (2 - ax)) & 1) hi += a[c];
            else lo += a[c];
        }
        v[ax] = q * (lo - hi);
    }
    const double2 out = d.pair == 0 ? make_double2(v[0], v[1]) : make_double2(v[2], 0.0);
    f[d.off + local] = out;
    if (part) {
        DotAcc<double> dx, dy;
        dx.add(out.x, out.x);
        dy.add(out.y, out.y);
        double tx = 0.0, ty = 0.0;
        block_sum2(dx, dy, red, tx, ty);
        if (threadIdx.x == 0) {
            part[d.part_off + 2 * lb] = tx;
            part[d.part_off + 2 * lb + 1] = ty;
        }
    }
}

// ------------------------------------------------------ preconditioner --
// Hartley transform of lines of n nodes (pair-packed complex FFT, register
// Stockham, see rve_device.cuh): dst = scale H src (src may equal dst).
// AXIS 2: x lines (contiguous), threads of a line side by side, one padded
// buffer per line; AXIS 1: y lines (stride n), the G lines of a block side
// by side so that each load instruction reads consecutive nodes, and their
// buffers interleaved element by element so that the lanes of a warp (G
// consecutive lines at the same element) touch consecutive words.  With
// `rd` set, also the block's partials of rd.dst per component (the r.z of
// CG).
template <int LOG2N, int AXIS, typename V>
__global__ void __launch_bounds__(256) k3_lines(Grp g, Tables tb, const V* src, V* dst,
                                                typename ScalarOf<V>::T scale,
                                                const V* __restrict__ rd, double* part,
                                                const MixScal* sc) {
    typedef typename ScalarOf<V>::T T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[16];
    int lb;
    const int u = unit_of(g, lb);
    const U3 d = g.desc[u];   // issued before the flag test
    if (sc && unit_skip(sc, u, false)) return;
    constexpr int n = 1 << LOG2N, TL = n / 8, G = 256 / TL;
    constexpr int BS = AXIS == 2 ? 1 : G;
    int q, t;
    if (AXIS == 2) { q = threadIdx.x / TL; t = threadIdx.x - q * TL; }
    else { t = threadIdx.x / G; q = threadIdx.x - t * G; }
    const int line = lb * G + q;   // < n^2
    int64_t base, stride;
    if (AXIS == 2) { base = d.off + (int64_t)line * n; stride = 1; }
    else { base = d.off + (int64_t)(line / n) * n * n + (line % n); stride = n; }
    V* buf = reinterpret_cast<V*>(smem_raw) + (AXIS == 2 ? q * seq_stride(n) : q);
    V w[8];
#pragma unroll
    for (int mm = 0; mm < 8; ++mm) w[mm] = src[base + (t + mm * TL) * stride];
    fft_reg<FFT_TO_BOTH, LOG2N, BS>(w, buf, LOG2N, t, twiddles<V>(tb, n), true);
    T ax = 0, ay = 0;
#pragma unroll
    for (int mm = 0; mm < 8; ++mm) {
        const int kx = t + mm * TL;
        const V hv = hartley_pair(w[mm], buf[pidx((n - kx) & (n - 1)) * BS]);
        const V o = mk<V>(scale * hv.x, scale * hv.y);
        dst[base + (int64_t)kx * stride] = o;
        if (rd) {
            const V r = rd[base + (int64_t)kx * stride];
            ax = fma(r.x, o.x, ax);
            ay = fma(r.y, o.y, ay);
        }
    }
    if (rd) {   // block-uniform
        double sx = 0.0, sy = 0.0;
        block_pair_sum(ax, ay, red, sx, sy);
        if (threadIdx.x == 0) {
            part[d.part_off + 2 * lb] = sx;
            part[d.part_off + 2 * lb + 1] = sy;
        }
    }
}

// Tridiagonal solves along z after the x and y transforms; writes M^{-1} t
// / n in place.  The n^2 columns (kx, ky) of a unit are numbered kc = ky n +
// kx, so column kc, row r sits at r n^2 + kc; a block takes ZC consecutive
// columns (ZSEG rows per thread, ZC x n / ZSEG = 512 threads).  The filter
// root of (kx, ky) solves rho + 1/rho = 2 + lambda(kx) + lambda(ky) + delta
// / c0, evaluated in the vector's precision; column 0 with delta = 0 is the
// singular one.
constexpr int ZSEG = 16;
template <int LOG2N> __host__ __device__ constexpr int zcols() { return Z_THREADS / ((1 << LOG2N) / ZSEG); }
template <typename T> __device__ __forceinline__ T filter_root_t(T mu) {
    return (T)1 / ((T)1 + (T)0.5 * mu + sqrt(mu * ((T)1 + (T)0.25 * mu)));
}
template <int LOG2N, typename V>
__global__ void __launch_bounds__(Z_THREADS) k3_zsolve(Grp g, Tables tb, double delta,
                                                       V* __restrict__ v, const MixScal* sc) {
    typedef typename ScalarOf<V>::T T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[64];
    __shared__ T csc[1];
    int lb;
    const int u = unit_of(g, lb);
    const U3 d = g.desc[u];   // issued before the flag test
    if (sc && unit_skip(sc, u, false)) return;
    constexpr int n = 1 << LOG2N, NN = n * n, ZC = zcols<LOG2N>();
    RDesc cd;          // the two fields the column solve reads
    cd.tC = ZC;
    cd.c0 = d.c0;
    const int c0 = lb * ZC;
    const T* lapT = lap_table<T>(tb, n);
    const T dc = (T)(delta / d.c0);
    V* vu = v + d.off;
    col_solve_core<V, LOG2N, true, ZSEG>(
        [&](int r, int kc) { return vu[r * NN + kc]; },
        [&](int r, int kc, V val) { vu[r * NN + kc] = val; },
        [&](int kc) -> T {
            const int ky = kc >> LOG2N, kx = kc & (n - 1);
            return (ky == 0 && delta == 0.0) ? rho_table<T>(tb, n)[kx]
                                             : filter_root_t<T>(lapT[kx] + lapT[ky] + dc);
        },
        cd, c0, reinterpret_cast<V*>(smem_raw), tb, delta, red, nullptr, csc);
}

// ------------------------------------------------------------- A_hom --
// Per tile of T3 cells, partial sums of sum a_c, the energy terms
// a_c v_i^T E v_j (ij = 11 12 13 22 23 33) and the flux terms a_c int_c
// d_j (x_i + phi_i) (ij = 11 12 13 21 22 23 31 32 33), v_i = xi_i + P_c u_i.
// Launched over realizations (the pair-0 unit descriptors); u is the ABI
// layout [nodes][3].
constexpr int A3_NP = 16;
template <int SCHEME>
__global__ void __launch_bounds__(T3) k3_a_hom_part(Grp g, Cells3T<double> cs,
                                                    const double* __restrict__ u3,
                                                    double* __restrict__ part) {
    __shared__ double red[8];
    int lb;
    const int un = unit_of(g, lb);
    const U3& d = g.desc[un];
    const int cell = lb * T3 + threadIdx.x;
    const int n = d.n;
    const int i = cell >> (2 * d.log2n), j = (cell >> d.log2n) & (n - 1), k = cell & (n - 1);
    const double h = d.h;
    const double a = cs.coef ? cs.coef[d.cell_off + cell] : two_values<double>(d, cs.mask[d.cell_off + cell] != 0);
    double v[3][8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int64_t gi = 3 * (d.cell_off + l3(d, i + (b >> 2), j + ((b >> 1) & 1), k + (b & 1)));
        v[0][b] = u3[gi] + h * (double)(b >> 2);
        v[1][b] = u3[gi + 1] + h * (double)((b >> 1) & 1);
        v[2][b] = u3[gi + 2] + h * (double)(b & 1);
    }
    double Ev[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < 8; ++b) s = fma(e3<SCHEME>(r, b, h), v[c][b], s);
            Ev[c][r] = s;
        }
    double val[A3_NP];
    val[0] = a;
    int q = 1;
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = x; y < 3; ++y) {
            double s = 0.0;
#pragma unroll
            for (int r = 0; r < 8; ++r) s = fma(v[x][r], Ev[y][r], s);
            val[q++] = a * s;
        }
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < 8; ++b) s += ((b >> (2 - y)) & 1) ? v[x][b] : -v[x][b];
            val[q++] = a * 0.25 * h * h * s;
        }
#pragma unroll
    for (int p = 0; p < A3_NP; ++p) {
        const double s = block_sum(val[p], red);
        if (threadIdx.x == 0) part[d.part_off + (int64_t)lb * A3_NP + p] = s;
    }
}

// One block per realization: fixed-order sums of its partials, then A.
__global__ void k3_a_hom_final(Grp g, const double* __restrict__ part, double* __restrict__ A,
                               double* __restrict__ Af) {
    __shared__ double red[32];
    const int un = g.first + blockIdx.x;
    const U3& d = g.desc[un];
    const int b = d.real;
    const int tiles = (int)(((int64_t)d.n * d.n * d.n) / T3);
    double s[A3_NP];
#pragma unroll
    for (int p = 0; p < A3_NP; ++p) {
        double t = 0.0;
        for (int k = threadIdx.x; k < tiles; k += blockDim.x) t += part[d.part_off + (int64_t)k * A3_NP + p];
        s[p] = block_sum(t, red);
    }
    if (threadIdx.x != 0) return;
    const double iv = d.inv_vol;
    const int sym[3][3] = {{1, 2, 3}, {2, 4, 5}, {3, 5, 6}};
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) {
            A[9 * (int64_t)b + 3 * x + y] = s[sym[x][y]] * iv;
            if (Af) Af[9 * (int64_t)b + 3 * x + y] = s[7 + 3 * x + y] * iv;
        }
}

// ------------------------------------- layout: ABI triples <-> unit pairs --
// Launched over units: unit pair 0 <-> components (1, 2), pair 1 <-> (3, -).
__global__ void __launch_bounds__(T3) k3_split(Grp g, const double* __restrict__ x3,
                                               double2* __restrict__ v) {
    int lb;
    const int un = unit_of(g, lb);
    const U3& d = g.desc[un];
    const int local = lb * T3 + threadIdx.x;
    const int64_t c = 3 * (d.cell_off + local);
    v[d.off + local] = d.pair == 0 ? make_double2(x3[c], x3[c + 1]) : make_double2(x3[c + 2], 0.0);
}

__global__ void __launch_bounds__(T3) k3_join(Grp g, const double2* __restrict__ v,
                                              double* __restrict__ x3) {
    int lb;
    const int un = unit_of(g, lb);
    const U3& d = g.desc[un];
    const int local = lb * T3 + threadIdx.x;
    const int64_t c = 3 * (d.cell_off + local);
    const double2 w = v[d.off + local];
    if (d.pair == 0) { x3[c] = w.x; x3[c + 1] = w.y; }
    else x3[c + 2] = w.x;
}

// Cell values as FP32 for the mixed path's stencil.
__global__ void k3_coef32(const double* __restrict__ coef, float* __restrict__ c32, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) c32[i] = (float)coef[i];
}

// ---------------------------------------------------------- CG cycles --
// Solver state of one unit (device; written by k3_scalar only).
struct MixScal {
    double fnorm[2];    // |f_c|
    double rn_prev[2];  // |r64_c| of the previous refinement
    double s[2];        // scale of the cycle's system (= |r64_c|)
    double target[2];   // relative residual target of the cycle
    double rho[2], alpha[2], beta[2];
    double relres[2];   // last FP64 true relative residual
    float alpha_f[2], beta_f[2], inv_s_f[2];
    int32_t active[2];  // the cycle still iterates on the component
    int32_t cdone[2];   // met the outer tolerance (or f_c = 0), or failed
    int32_t iters[2];
    int32_t stall[2];   // consecutive refinements without a 10x reduction
    int32_t refinements, status;
    int32_t done;       // no component active in the cycle
    int32_t outer_done; // every component finished
};
__device__ __forceinline__ bool unit_skip(const MixScal* sc, int u, bool outer) {
    return outer ? sc[u].outer_done != 0 : sc[u].done != 0;
}
enum { M_FNORM = 0, M_REFINE, M_RHO0, M_ALPHA, M_CONV, M_BETA };
constexpr int MAX_REFINE = 100;
constexpr int MAX_STALL = 4;

// The scalar steps: one block per unit reduces the unit's partial pairs (n^3
// >> pshift of them: one per block of the kernel that wrote them) in a fixed
// order (per-thread strided sums, then the block tree) and thread 0 applies
// `what`.  `tfac`: the cycle target is max(tfac tol |f| /
// |r64|, inner_tol).
struct ScalArgs {
    double tol, inner_tol, tfac;
    int max_iter;
};
__global__ void __launch_bounds__(256) k3_scalar(int first, const U3* __restrict__ desc,
                                                 MixScal* scs,
                                                 const double* __restrict__ part, int what,
                                                 int pshift, ScalArgs a) {
    __shared__ double red[32];
    const int u = first + blockIdx.x;
    MixScal* sc = scs + u;
    const U3& d = desc[u];
    if (what != M_FNORM && what != M_REFINE && sc->done) return;
    if (what == M_REFINE && sc->outer_done) return;
    const int nb = (int)(((int64_t)d.n * d.n * d.n) >> pshift);   // partial pairs written
    const double* pp = part + d.part_off;
    double tx = 0.0, ty = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        tx += pp[2 * k];
        ty += pp[2 * k + 1];
    }
    const double sx = block_sum(tx, red);
    const double sy = block_sum(ty, red);
    if (threadIdx.x != 0) return;
    const double v[2] = {sx, sy};
    switch (what) {
        case M_FNORM:
            for (int k = 0; k < 2; ++k) {
                sc->fnorm[k] = sqrt(v[k]);
                sc->cdone[k] = !(v[k] > 0.0);
                sc->active[k] = 0;
                sc->iters[k] = 0;
                sc->stall[k] = 0;
                sc->relres[k] = 0.0;
                sc->rn_prev[k] = sc->fnorm[k];
            }
            sc->refinements = 0;
            sc->status = RVE_OK;
            sc->done = 1;
            sc->outer_done = sc->cdone[0] && sc->cdone[1];
            break;
        case M_REFINE:
            sc->refinements += 1;
            for (int k = 0; k < 2; ++k) {
                sc->active[k] = 0;
                sc->alpha[k] = sc->beta[k] = 0.0;
                sc->alpha_f[k] = sc->beta_f[k] = 0.f;
                sc->inv_s_f[k] = 0.f;
                if (sc->cdone[k]) continue;
                const double rn = sqrt(v[k]);
                sc->relres[k] = rn / sc->fnorm[k];
                if (!isfinite(rn)) { sc->status = RVE_ENAN; sc->cdone[k] = 1; continue; }
                if (rn <= a.tol * sc->fnorm[k]) { sc->cdone[k] = 1; continue; }
                sc->stall[k] = (rn > 0.1 * sc->rn_prev[k]) ? sc->stall[k] + 1 : 0;
                if (sc->iters[k] >= a.max_iter || sc->refinements > MAX_REFINE ||
                    sc->stall[k] >= MAX_STALL) {
                    sc->status = RVE_ENOCONV;
                    sc->cdone[k] = 1;
                    continue;
                }
                sc->rn_prev[k] = rn;
                sc->s[k] = rn;
                sc->inv_s_f[k] = (float)(1.0 / rn);
                sc->target[k] = fmax(a.tfac * a.tol * sc->fnorm[k] / rn, a.inner_tol);
                sc->active[k] = 1;
            }
            sc->outer_done = sc->cdone[0] && sc->cdone[1];
            sc->done = !(sc->active[0] || sc->active[1]);
            break;
        case M_RHO0:
            for (int k = 0; k < 2; ++k) sc->rho[k] = v[k];
            break;
        case M_ALPHA:
            for (int k = 0; k < 2; ++k) {
                sc->alpha[k] = sc->active[k] ? sc->rho[k] / v[k] : 0.0;
                sc->alpha_f[k] = (float)sc->alpha[k];
                if (sc->active[k]) sc->iters[k] += 1;
            }
            break;
        case M_CONV:   // the cycle's residual starts at norm 1
            for (int k = 0; k < 2; ++k) {
                if (!sc->active[k]) continue;
                const double rn = sqrt(v[k]);
                if (!isfinite(rn)) { sc->status = RVE_ENAN; sc->active[k] = 0; sc->cdone[k] = 1; }
                else if (rn <= sc->target[k] || sc->iters[k] >= a.max_iter) sc->active[k] = 0;
            }
            sc->done = !(sc->active[0] || sc->active[1]);
            break;
        case M_BETA:
            for (int k = 0; k < 2; ++k) {
                sc->beta[k] = sc->active[k] ? v[k] / sc->rho[k] : 0.0;
                sc->beta_f[k] = (float)sc->beta[k];
                sc->rho[k] = v[k];
            }
            break;
    }
}

// The step scalars in the cycle's precision.
template <typename T> __device__ __forceinline__ T alpha_of(const MixScal& s, int k);
template <> __device__ __forceinline__ double alpha_of<double>(const MixScal& s, int k) { return s.alpha[k]; }
template <> __device__ __forceinline__ float alpha_of<float>(const MixScal& s, int k) { return s.alpha_f[k]; }
template <typename T> __device__ __forceinline__ T beta_of(const MixScal& s, int k);
template <> __device__ __forceinline__ double beta_of<double>(const MixScal& s, int k) { return s.beta[k]; }
template <> __device__ __forceinline__ float beta_of<float>(const MixScal& s, int k) { return s.beta_f[k]; }

// Start of a cycle: r = r64 / s, e = 0, p = 0 (components not iterating: 0).
template <typename V>
__global__ void __launch_bounds__(T3) k3_start(Grp g, const MixScal* scs,
                                               const double2* __restrict__ r64, V* __restrict__ r,
                                               V* __restrict__ e, V* __restrict__ p) {
    typedef typename ScalarOf<V>::T T;
    int lb;
    const int u = unit_of(g, lb);
    const U3 d = g.desc[u];   // issued before the flag test
    const MixScal& sc = scs[u];
    if (sc.done) return;
    const int64_t node = d.off + lb * T3 + threadIdx.x;
    const double2 rr = r64[node];
    V o;
    if (sizeof(T) == 8) {
        o.x = (T)(sc.active[0] ? rr.x / sc.s[0] : 0.0);
        o.y = (T)(sc.active[1] ? rr.y / sc.s[1] : 0.0);
    } else {
        o.x = (T)rr.x * (T)sc.inv_s_f[0];
        o.y = (T)rr.y * (T)sc.inv_s_f[1];
    }
    r[node] = o;
    e[node] = mk<V>((T)0, (T)0);
    p[node] = mk<V>((T)0, (T)0);
}

// e += alpha p; r -= alpha q; partials |r|^2.  Four nodes per thread.
template <typename V>
__global__ void __launch_bounds__(T3) k3_axpy(Grp g, const MixScal* scs, V* __restrict__ e,
                                              V* __restrict__ r, const V* __restrict__ p,
                                              const V* __restrict__ q, double* part) {
    typedef typename ScalarOf<V>::T T;
    __shared__ double red[16];
    int lb;
    const int u = unit_of(g, lb);
    const U3 d = g.desc[u];   // issued before the flag test
    const MixScal& sc = scs[u];
    if (sc.done) return;
    const T ax_ = alpha_of<T>(sc, 0), ay_ = alpha_of<T>(sc, 1);
    T sx = 0, sy = 0;
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) {
        const int64_t node = d.off + (int64_t)lb * (4 * T3) + mm * T3 + threadIdx.x;
        const V pp = p[node], qq = q[node];
        V ee = e[node], rr = r[node];
        ee.x = fma(ax_, pp.x, ee.x);
        ee.y = fma(ay_, pp.y, ee.y);
        rr.x = fma(-ax_, qq.x, rr.x);
        rr.y = fma(-ay_, qq.y, rr.y);
        e[node] = ee;
        r[node] = rr;
        sx = fma(rr.x, rr.x, sx);
        sy = fma(rr.y, rr.y, sy);
    }
    double tx = 0.0, ty = 0.0;
    block_pair_sum(sx, sy, red, tx, ty);
    if (threadIdx.x == 0) {
        part[d.part_off + 2 * lb] = tx;
        part[d.part_off + 2 * lb + 1] = ty;
    }
}

// p = z + beta p.  Four nodes per thread.
template <typename V>
__global__ void __launch_bounds__(T3) k3_xpby(Grp g, const MixScal* scs, const V* __restrict__ z,
                                              V* __restrict__ p) {
    typedef typename ScalarOf<V>::T T;
    int lb;
    const int u = unit_of(g, lb);
    const U3 d = g.desc[u];   // issued before the flag test
    const MixScal& sc = scs[u];
    if (sc.done) return;
    const T bx = beta_of<T>(sc, 0), by = beta_of<T>(sc, 1);
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) {
        const int64_t node = d.off + (int64_t)lb * (4 * T3) + mm * T3 + threadIdx.x;
        const V zz = z[node], pp = p[node];
        p[node] = mk<V>(fma(bx, pp.x, zz.x), fma(by, pp.y, zz.y));
    }
}

// End of a cycle: u += s e (components that iterated).
template <typename V>
__global__ void __launch_bounds__(T3) k3_accum(Grp g, const MixScal* scs, const V* __restrict__ e,
                                               double2* __restrict__ uv) {
    int lb;
    const int u = unit_of(g, lb);
    const U3 d = g.desc[u];   // issued before the flag test
    const MixScal& sc = scs[u];
    if (sc.outer_done) return;
    const int64_t node = d.off + lb * T3 + threadIdx.x;
    const double sx = sc.cdone[0] ? 0.0 : sc.s[0], sy = sc.cdone[1] ? 0.0 : sc.s[1];
    const V ee = e[node];
    double2 w = uv[node];
    w.x = fma(sx, (double)ee.x, w.x);
    w.y = fma(sy, (double)ee.y, w.y);
    uv[node] = w;
}

// Per realization: the report of its two units (u_of[b]: the pair-0 unit).
__global__ void k3_report(const MixScal* scs, const U3* __restrict__ desc,
                          const int32_t* __restrict__ u_of, int batch, rve3_solve_info* info) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const int u0 = u_of[b];
    const MixScal& s12 = scs[u0];
    const MixScal& s3 = scs[desc[u0].partner];
    rve3_solve_info r;
    r.iters[0] = s12.iters[0];
    r.iters[1] = s12.iters[1];
    r.iters[2] = s3.iters[0];
    r.status = s12.status != RVE_OK ? s12.status : s3.status;
    r.refinements = s12.refinements + s3.refinements;
    r.reserved = 0;
    r.relres[0] = s12.relres[0];
    r.relres[1] = s12.relres[1];
    r.relres[2] = s3.relres[0];
    info[b] = r;
}

// ------------------------------------------------------------ profile --
// Event timing of every 3D launch by kind (diagnostics, enabled together
// with the fused solver's profiler by rve_profile_enable; process-wide, not
// thread-safe): 0 stiffness of the CG steps, 1 line transform (x or y),
// 2 z solve, 3 vector steps of CG (dots, updates), 4 scalar steps (one block
// per unit), 5 FP64 true residual (the stiffness with the residual fused).
enum { P3_STIFF = 0, P3_LINES, P3_ZSOLVE, P3_VECTOR, P3_SCALAR, P3_RESID, P3_K };
struct Prof3 {
    double ms[P3_K] = {};
    long long launches[P3_K] = {};
    std::vector<cudaEvent_t> pool;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
    }
    void harvest() {   // stream already synchronised
        for (const Rec& r : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
                ms[r.kind] += t;
                launches[r.kind] += 1;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
};
static Prof3 g_prof3;

// Brackets the launches issued during its lifetime with two events.
struct Span3 {
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Span3(cudaStream_t s_, int k) : kind(k), s(s_) {
        if (profile_on() && (a = g_prof3.get()) != nullptr) cudaEventRecord(a, s);
    }
    ~Span3() {
        if (!a) return;
        cudaEvent_t b = g_prof3.get();
        if (!b) { g_prof3.pool.push_back(a); return; }
        cudaEventRecord(b, s);
        g_prof3.pending.push_back({kind, a, b});
    }
};

static void prof3_sync(cudaStream_t s) {
    if (profile_on() && !g_prof3.pending.empty() && cudaStreamSynchronize(s) == cudaSuccess)
        g_prof3.harvest();
}

// ---------------------------------------------------------------- host --
constexpr int N3_MIN = 32, N3_MAX = 256;
constexpr int NVEC = 8;   // unit vectors: f, u, r64, and the cycle's r, z, p, e, q

// The units of one grid size: ids first .. first + count - 1, the pair-0
// units (one per realization) first.
struct Group3 {
    int log2n = 0;
    int first = 0;
    int count = 0;
};

struct Plan3 {
    int batch = 0;
    std::vector<U3> desc;      // 2 * batch units, grouped by size
    std::vector<int32_t> u_of; // pair-0 unit of each realization
    std::vector<Group3> groups;
    int64_t nodes = 0;         // realization nodes (sum n^3)
    int64_t unit_nodes = 0;    // 2 * nodes
    int64_t parts = 0;         // doubles of partials
    int max_log2n = 5;
    size_t o_desc = 0, o_ids = 0, o_tw64 = 0, o_tw32 = 0, o_lap = 0, o_lap32 = 0, o_rho64 = 0,
           o_rho32 = 0, o_sc = 0, o_part = 0, o_c32 = 0, o_vec = 0, total = 0;
};

static rve_status make_plan3(const rve_realization* r, int32_t batch, Plan3& p) {
    if (!r || batch <= 0 || batch > (1 << 16)) return RVE_EINVAL;
    p.batch = batch;
    p.desc.assign(2 * (size_t)batch, U3{});
    p.u_of.assign(batch, 0);
    p.nodes = 0;
    p.parts = 0;
    p.max_log2n = 5;
    std::map<int, std::vector<int32_t>> by_size;   // realizations by log2 n
    std::vector<int64_t> cell_off(batch);
    for (int b = 0; b < batch; ++b) {
        const rve_realization& x = r[b];
        if (x.L <= 0 || x.m0 <= 0) return RVE_EINVAL;
        const int64_t n64 = (int64_t)x.L * x.m0;
        if (n64 < N3_MIN || n64 > N3_MAX || (n64 & (n64 - 1))) return RVE_EINVAL;
        const int n = (int)n64;
        if (x.incl_cells <= 0 || x.incl_cells > n || x.n_incl < 0) return RVE_EINVAL;
        if ((int64_t)x.n_incl * x.incl_cells * x.incl_cells > (1LL << 31)) return RVE_EINVAL;
        if (!std::isfinite(x.a_matrix) || !std::isfinite(x.a_incl) || !(x.a_matrix > 0.0) ||
            !(x.a_incl > 0.0))
            return RVE_EINVAL;
        const int lg = 31 - __builtin_clz((unsigned)n);
        by_size[lg].push_back(b);
        cell_off[b] = p.nodes;
        p.nodes += (int64_t)n * n * n;
        p.max_log2n = std::max(p.max_log2n, lg);
    }
    p.unit_nodes = 2 * p.nodes;
    p.groups.clear();
    int u = 0;
    int64_t off = 0;
    for (auto& kv : by_size) {
        Group3 g;
        g.log2n = kv.first;
        g.first = u;
        g.count = 2 * (int)kv.second.size();
        const int half = (int)kv.second.size();
        const int64_t nn = (int64_t)1 << (3 * kv.first);
        for (int pair = 0; pair < 2; ++pair)
            for (int q = 0; q < half; ++q) {
                const int b = kv.second[q];
                const rve_realization& x = r[b];
                U3& d = p.desc[u];
                std::memset(&d, 0, sizeof(d));
                d.n = 1 << kv.first;
                d.log2n = kv.first;
                d.pair = pair;
                d.n_incl = x.n_incl;
                d.s = x.incl_cells;
                d.real = b;
                d.partner = pair == 0 ? g.first + half + q : g.first + q;
                d.cell_off = cell_off[b];
                d.part_off = p.parts;
                d.am = x.a_matrix;
                d.ai = x.a_incl;
                d.am32 = (float)x.a_matrix;
                d.ai32 = (float)x.a_incl;
                d.h = 1.0 / (double)x.m0;
                d.c0 = 0.5 * (x.a_matrix + x.a_incl);
                d.inv_vol = 1.0 / ((double)x.L * (double)x.L * (double)x.L);
                d.key = sm64_mix(x.seed + (x.index + 1) * 0x9E3779B97F4A7C15ull);
                d.off = off;
                if (pair == 0) p.u_of[b] = u;
                off += nn;
                p.parts += A3_NP * (nn / T3);   // enough for every kernel and for A_hom
                ++u;
            }
        p.groups.push_back(g);
    }
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    size_t woff = 0;
    auto take = [&](size_t bytes) { const size_t o = woff; woff = up(woff + bytes); return o; };
    const size_t tab = (size_t)2 << p.max_log2n;
    p.o_desc = take(sizeof(U3) * p.desc.size());
    p.o_ids = take(sizeof(int32_t) * p.u_of.size());
    p.o_tw64 = take(sizeof(double2) * tab);
    p.o_tw32 = take(sizeof(float2) * tab);
    p.o_lap = take(sizeof(double) * tab);
    p.o_lap32 = take(sizeof(float) * tab);
    p.o_rho64 = take(sizeof(double) * tab);
    p.o_rho32 = take(sizeof(float) * tab);
    p.o_sc = take(sizeof(MixScal) * p.desc.size());
    p.o_part = take(sizeof(double) * (size_t)p.parts);
    p.o_c32 = take(sizeof(float) * (size_t)p.nodes);
    p.o_vec = take(sizeof(double2) * NVEC * (size_t)p.unit_nodes);
    p.total = woff;
    return RVE_OK;
}

struct Ws3 {   // device pointers into the workspace
    const Plan3* p;
    char* w;
    const U3* desc() const { return reinterpret_cast<const U3*>(w + p->o_desc); }
    const int32_t* u_of() const { return reinterpret_cast<const int32_t*>(w + p->o_ids); }
    MixScal* sc() const { return reinterpret_cast<MixScal*>(w + p->o_sc); }
    double* part() const { return reinterpret_cast<double*>(w + p->o_part); }
    float* c32() const { return reinterpret_cast<float*>(w + p->o_c32); }
    template <typename V> V* vec(int k) const {   // unit vector k, 16 bytes per node reserved
        return reinterpret_cast<V*>(w + p->o_vec + (size_t)k * 16 * (size_t)p->unit_nodes);
    }
    Tables tables() const {
        Tables tb;
        tb.tw64 = reinterpret_cast<const double2*>(w + p->o_tw64);
        tb.tw32 = reinterpret_cast<const float2*>(w + p->o_tw32);
        tb.lap = reinterpret_cast<const double*>(w + p->o_lap);
        tb.lap32 = reinterpret_cast<const float*>(w + p->o_lap32);
        tb.rho64 = reinterpret_cast<const double*>(w + p->o_rho64);
        tb.rho32 = reinterpret_cast<const float*>(w + p->o_rho32);
        return tb;
    }
    // launch over the units (or the pair-0 units) of group g, `per` (a power
    // of two) blocks each
    Grp grp(const Group3& g, int per, bool reals = false) const {
        (void)reals;   // the pair-0 units come first in the group
        return Grp{desc(), g.first, 31 - __builtin_clz((unsigned)per)};
    }
};
enum { V_F = 0, V_U, V_R64, V_R, V_Z, V_P, V_E, V_Q };

static unsigned nblocks(const Group3& g, int64_t per, bool reals = false) {
    return (unsigned)((reals ? g.count / 2 : g.count) * per);
}
static int64_t nodes_of(const Group3& g) { return (int64_t)1 << (3 * g.log2n); }

// Setup common to the entry points: descriptors, id lists and tables.
static rve_status setup3(const Plan3& p, char* w, cudaStream_t s, bool tables) {
    if (cudaMemcpyAsync(w + p.o_desc, p.desc.data(), sizeof(U3) * p.desc.size(),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(w + p.o_ids, p.u_of.data(), sizeof(int32_t) * p.u_of.size(),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return RVE_ECUDA;
    if (!tables) return RVE_OK;
    Ws3 ws{&p, w};
    return fill_tables(ws.tables(), p.max_log2n, s) == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

// dst = B^{-1} src for the units of group g; src is read by the first pass
// only (it may equal dst).  With `rd`, the units' partials of rd.dst.
template <int LG, typename V>
static cudaError_t precond3_t(const Ws3& ws, const Group3& g, double delta, const V* src, V* dst,
                              const V* rd, const MixScal* sc, cudaStream_t s) {
    typedef typename ScalarOf<V>::T T;
    constexpr int n = 1 << LG, TL = n / 8;
    const int G = 256 / TL;
    const size_t smem = (size_t)G * seq_stride(n) * sizeof(V);
    const int lines = (n * n) / G;
    constexpr int ZC = zcols<LG>(), ZP = n / ZSEG;
    const size_t zsmem = (size_t)(2 * ZC + 2) * ZP * sizeof(V);
    cudaError_t e = cudaFuncSetAttribute(k3_lines<LG, 2, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k3_lines<LG, 1, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const Tables tb = ws.tables();
    double* part = ws.part();
    const Grp gl = ws.grp(g, lines);
    const unsigned bl = nblocks(g, lines);
    {
        Span3 sp(s, P3_LINES);
        k3_lines<LG, 2, V><<<bl, 256, smem, s>>>(gl, tb, src, dst, (T)1, nullptr, nullptr, sc);
    }
    {
        Span3 sp(s, P3_LINES);
        k3_lines<LG, 1, V><<<bl, 256, smem, s>>>(gl, tb, dst, dst, (T)1, nullptr, nullptr, sc);
    }
    {
        Span3 sp(s, P3_ZSOLVE);
        k3_zsolve<LG, V><<<nblocks(g, n * n / ZC), Z_THREADS, zsmem, s>>>(
            ws.grp(g, n * n / ZC), tb, delta, dst, sc);
    }
    {
        Span3 sp(s, P3_LINES);
        k3_lines<LG, 1, V><<<bl, 256, smem, s>>>(gl, tb, dst, dst, (T)1, nullptr, nullptr, sc);
    }
    {
        Span3 sp(s, P3_LINES);
        k3_lines<LG, 2, V><<<bl, 256, smem, s>>>(gl, tb, dst, dst, (T)(1.0 / (double)n), rd, part, sc);
    }
    note_launch(5);
    return cudaGetLastError();
}

template <typename V>
static cudaError_t precond3(const Ws3& ws, const Group3& g, double delta, const V* src, V* dst,
                            cudaStream_t s, const V* rd = nullptr, const MixScal* sc = nullptr) {
    switch (g.log2n) {
        case 5: return precond3_t<5, V>(ws, g, delta, src, dst, rd, sc, s);
        case 6: return precond3_t<6, V>(ws, g, delta, src, dst, rd, sc, s);
        case 7: return precond3_t<7, V>(ws, g, delta, src, dst, rd, sc, s);
        default: return precond3_t<8, V>(ws, g, delta, src, dst, rd, sc, s);
    }
}

template <int MODE, typename V>
static cudaError_t stiffness3(const Ws3& ws, const Group3& g, Cells3T<typename ScalarOf<V>::T> cs,
                              int scheme, const V* x, V* y, const V* f, bool partials,
                              const MixScal* sc, cudaStream_t s) {
    const int per = (int)(nodes_of(g) / (2 * T3 * SZ));
    const Grp gg = ws.grp(g, per);
    double* part = partials ? ws.part() : nullptr;
    const size_t smem = stiff_smem<V>(g.log2n);
    auto kern = scheme == RVE_Q1_LUMPED ? k3_stiffness<1, MODE, V> : k3_stiffness<0, MODE, V>;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    Span3 sp(s, MODE == MODE_RESID ? P3_RESID : P3_STIFF);
    kern<<<nblocks(g, per), T3, smem, s>>>(gg, cs, x, y, f, part, sc);
    note_launch();
    return cudaGetLastError();
}

// r64 = f - A u of the units of group g in double words (the mixed path):
// u split into double words in the q slot, then the residual pass.
static cudaError_t resid3_dw(const Ws3& ws, const Group3& g, Cells3T<double> cs, int scheme,
                             const double2* u, double2* r, const double2* f, const MixScal* sc,
                             cudaStream_t s) {
    const int per = (int)(nodes_of(g) / T3);
    float4* wdw = reinterpret_cast<float4*>(ws.vec<double2>(V_Q));   // 16 bytes per node
    const Grp gg = ws.grp(g, per);
    Span3 sp(s, P3_RESID);
    k3_split_dw<<<nblocks(g, per), T3, 0, s>>>(gg, u, wdw, ws.sc());
    if (scheme == RVE_Q1_LUMPED)
        k3_resid_dw<1><<<nblocks(g, per), T3, 0, s>>>(gg, cs, wdw, f, r, ws.part(), sc);
    else
        k3_resid_dw<0><<<nblocks(g, per), T3, 0, s>>>(gg, cs, wdw, f, r, ws.part(), sc);
    note_launch(2);
    return cudaGetLastError();
}

// The correctors of every unit: cycles of PCG in the precision of V between
// FP64 true residuals (see the head of the file).
template <typename V>
static rve_status solve_units(const Plan3& p, char* w, Cells3T<double> cs64,
                              Cells3T<typename ScalarOf<V>::T> csV, const rve3_solve_opts& o,
                              cudaStream_t s) {
    const Ws3 ws{&p, w};
    MixScal* sc = ws.sc();
    double* part = ws.part();
    double2* f = ws.vec<double2>(V_F);
    double2* uv = ws.vec<double2>(V_U);
    double2* r64 = ws.vec<double2>(V_R64);
    V* r = ws.vec<V>(V_R);
    V* z = ws.vec<V>(V_Z);
    V* pp = ws.vec<V>(V_P);
    V* e = ws.vec<V>(V_E);
    V* q = ws.vec<V>(V_Q);
    const bool fp64 = sizeof(typename ScalarOf<V>::T) == 8;
    const ScalArgs sa{o.tol, fp64 ? 0.0 : o.inner_tol, fp64 ? 1.0 : 0.5, o.max_iter};
    auto vec_step = [&](auto&& launch) {
        Span3 sp(s, P3_VECTOR);
        launch();
    };
    // partial pairs per unit: n^3 >> shift (rhs: 256 nodes per block; axpy:
    // 1024; stiffness and the last line pass: 2048)
    constexpr int SH_RHS = 8, SH_STIFF = 11, SH_AXPY = 10, SH_LINES = 11;
    static_assert(2 * T3 * SZ == (1 << SH_STIFF) && 4 * T3 == (1 << SH_AXPY) && T3 == (1 << SH_RHS),
                  "partial counts");
    auto scalar = [&](const Group3& g, int what, int shift) {
        Span3 sp(s, P3_SCALAR);
        k3_scalar<<<g.count, 256, 0, s>>>(g.first, ws.desc(), sc, part, what, shift, sa);
        note_launch();
    };
    auto per_group = [&](auto&& fn) -> rve_status {
        for (const Group3& g : p.groups) {
            const rve_status st = fn(g);
            if (st != RVE_OK) return st;
        }
        return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
    };
    std::vector<MixScal> hsc(p.desc.size());
    auto poll = [&](bool outer) -> int {   // -1 error, 1 every unit finished
        if (cudaMemcpyAsync(hsc.data(), sc, sizeof(MixScal) * hsc.size(), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return -1;
        if (profile_on()) g_prof3.harvest();
        for (const MixScal& m : hsc)
            if (!(outer ? m.outer_done : m.done)) return 0;
        return 1;
    };
    rve_status st;
    // loads with |f|^2, u = 0
    st = per_group([&](const Group3& g) {
        const int per = (int)(nodes_of(g) / T3);
        vec_step([&] { k3_rhs<<<nblocks(g, per), T3, 0, s>>>(ws.grp(g, per), cs64, f, part); });
        scalar(g, M_FNORM, SH_RHS);
        note_launch();
        return RVE_OK;
    });
    if (st != RVE_OK) return st;
    if (cudaMemsetAsync(uv, 0, sizeof(double2) * (size_t)p.unit_nodes, s) != cudaSuccess ||
        cudaMemcpyAsync(r64, f, sizeof(double2) * (size_t)p.unit_nodes, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
        return RVE_ECUDA;
    const int every = o.check_every;
    for (int cycle = 0; cycle <= MAX_REFINE + 1; ++cycle) {
        // FP64 true residual r64 = f - A u and the refinement step
        st = per_group([&](const Group3& g) {
            int shift = SH_RHS;   // u = 0: r64 = f, the partials of |f|^2 are still in place
            if (cycle > 0 && fp64) {
                if (stiffness3<MODE_RESID, double2>(ws, g, cs64, o.scheme, uv, r64, f, true, sc, s) !=
                    cudaSuccess)
                    return RVE_ECUDA;
                shift = SH_STIFF;
            } else if (cycle > 0) {   // mixed: the double-word residual
                if (resid3_dw(ws, g, cs64, o.scheme, uv, r64, f, sc, s) != cudaSuccess)
                    return RVE_ECUDA;
                shift = SH_RHS;
            }
            scalar(g, M_REFINE, shift);
            return RVE_OK;
        });
        if (st != RVE_OK) return st;
        const int pr = poll(true);
        if (pr < 0) return RVE_ECUDA;
        if (pr == 1) break;
        // a cycle: r = r64 / s, z = B^-1 r, p = z
        st = per_group([&](const Group3& g) {
            const int per = (int)(nodes_of(g) / T3);
            vec_step([&] { k3_start<V><<<nblocks(g, per), T3, 0, s>>>(ws.grp(g, per), sc, r64, r, e, pp); });
            if (precond3<V>(ws, g, o.delta, r, z, s, r, sc) != cudaSuccess) return RVE_ECUDA;
            scalar(g, M_RHO0, SH_LINES);
            const int per4 = per / 4;
            vec_step([&] { k3_xpby<V><<<nblocks(g, per4), T3, 0, s>>>(ws.grp(g, per4), sc, z, pp); });
            note_launch(2);
            return RVE_OK;
        });
        if (st != RVE_OK) return st;
        for (int it = 1;; ++it) {
            st = per_group([&](const Group3& g) {
                const int per = (int)(nodes_of(g) / T3), per4 = per / 4;
                if (stiffness3<MODE_APPLY, V>(ws, g, csV, o.scheme, pp, q, nullptr, true, sc, s) !=
                    cudaSuccess)
                    return RVE_ECUDA;
                scalar(g, M_ALPHA, SH_STIFF);
                vec_step([&] {
                    k3_axpy<V><<<nblocks(g, per4), T3, 0, s>>>(ws.grp(g, per4), sc, e, r, pp, q, part);
                });
                scalar(g, M_CONV, SH_AXPY);
                if (precond3<V>(ws, g, o.delta, r, z, s, r, sc) != cudaSuccess) return RVE_ECUDA;
                scalar(g, M_BETA, SH_LINES);
                vec_step([&] { k3_xpby<V><<<nblocks(g, per4), T3, 0, s>>>(ws.grp(g, per4), sc, z, pp); });
                note_launch(2);
                return RVE_OK;
            });
            if (st != RVE_OK) return st;
            if (it % every == 0) {
                const int pi = poll(false);
                if (pi < 0) return RVE_ECUDA;
                if (pi == 1) break;
            }
        }
        st = per_group([&](const Group3& g) {
            const int per = (int)(nodes_of(g) / T3);
            vec_step([&] { k3_accum<V><<<nblocks(g, per), T3, 0, s>>>(ws.grp(g, per), sc, e, uv); });
            note_launch();
            return RVE_OK;
        });
        if (st != RVE_OK) return st;
    }
    return RVE_OK;
}

static rve3_solve_opts resolved3(const rve3_solve_opts* opts) {
    rve3_solve_opts o = {};
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 20000;
    if (!(o.tol > 0.0)) o.tol = 1e-10;
    if (!(o.inner_tol > 0.0)) o.inner_tol = 1e-4;
    if (o.check_every <= 0) o.check_every = 8;
    return o;
}

static bool valid_scheme(int s) { return s == RVE_Q1_CONSISTENT || s == RVE_Q1_LUMPED; }

}  // namespace rve

using namespace rve;

extern "C" {

int64_t rve3_nodes(const rve_realization* r, int32_t batch) {
    Plan3 p;
    return make_plan3(r, batch, p) == RVE_OK ? p.nodes : -1;
}

size_t rve3_workspace_size(const rve_realization* r, int32_t batch) {
    Plan3 p;
    return make_plan3(r, batch, p) == RVE_OK ? p.total : 0;
}

rve_status rve3_gen_field(const rve_realization* r, int32_t batch, uint8_t* mask, void* stream) {
    Plan3 p;
    rve_status st = make_plan3(r, batch, p);
    if (st != RVE_OK) return st;
    if (!mask) return RVE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(mask, 0, (size_t)p.nodes, s) != cudaSuccess) return RVE_ECUDA;
    for (int b = 0; b < p.batch; ++b) {
        const U3& d = p.desc[p.u_of[b]];
        const int64_t rows = (int64_t)d.n_incl * d.s * d.s;
        if (rows == 0) continue;
        k3_gen_field<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(d, mask);
        note_launch();
    }
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status rve3_rhs(const rve_realization* r, int32_t batch, const uint8_t* mask, const double* coef,
                    int32_t scheme, double* f, void* ws, size_t ws_bytes, void* stream) {
    Plan3 p;
    rve_status st = make_plan3(r, batch, p);
    if (st != RVE_OK) return st;
    if ((!mask && !coef) || !f || !ws || ws_misaligned(ws) || !valid_scheme(scheme)) return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    if ((st = setup3(p, w, s, false)) != RVE_OK) return st;
    const Ws3 W{&p, w};
    const Cells3T<double> cs{mask, coef};
    for (const Group3& g : p.groups) {
        const int per = (int)(nodes_of(g) / T3);
        k3_rhs<<<nblocks(g, per), T3, 0, s>>>(W.grp(g, per), cs, W.vec<double2>(V_F), nullptr);
        k3_join<<<nblocks(g, per), T3, 0, s>>>(W.grp(g, per), W.vec<double2>(V_F), f);
        note_launch(2);
    }
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status rve3_apply_stiffness(const rve_realization* r, int32_t batch, const uint8_t* mask,
                                const double* coef, int32_t scheme, const double* x, double* y,
                                void* ws, size_t ws_bytes, void* stream) {
    Plan3 p;
    rve_status st = make_plan3(r, batch, p);
    if (st != RVE_OK) return st;
    if ((!mask && !coef) || !x || !y || x == y || !ws || ws_misaligned(ws) || !valid_scheme(scheme))
        return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    if ((st = setup3(p, w, s, false)) != RVE_OK) return st;
    const Ws3 W{&p, w};
    const Cells3T<double> cs{mask, coef};
    for (const Group3& g : p.groups) {
        const int per = (int)(nodes_of(g) / T3);
        k3_split<<<nblocks(g, per), T3, 0, s>>>(W.grp(g, per), x, W.vec<double2>(V_R));
        note_launch();
        if (stiffness3<MODE_APPLY, double2>(W, g, cs, scheme, W.vec<double2>(V_R), W.vec<double2>(V_Q),
                                            nullptr, false, nullptr, s) != cudaSuccess)
            return RVE_ECUDA;
        k3_join<<<nblocks(g, per), T3, 0, s>>>(W.grp(g, per), W.vec<double2>(V_Q), y);
        note_launch();
    }
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status rve3_apply_precond(const rve_realization* r, int32_t batch, double delta,
                              const double* x, double* y, void* ws, size_t ws_bytes,
                              void* stream) {
    Plan3 p;
    rve_status st = make_plan3(r, batch, p);
    if (st != RVE_OK) return st;
    if (!x || !y || !ws || ws_misaligned(ws) || !std::isfinite(delta) || delta < 0.0) return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    if ((st = setup3(p, w, s, true)) != RVE_OK) return st;
    const Ws3 W{&p, w};
    double2* v = W.vec<double2>(V_R);
    for (const Group3& g : p.groups) {
        const int per = (int)(nodes_of(g) / T3);
        k3_split<<<nblocks(g, per), T3, 0, s>>>(W.grp(g, per), x, v);
        note_launch();
    }
    for (const Group3& g : p.groups)
        if (precond3<double2>(W, g, delta, v, v, s) != cudaSuccess) return RVE_ECUDA;
    for (const Group3& g : p.groups) {
        const int per = (int)(nodes_of(g) / T3);
        k3_join<<<nblocks(g, per), T3, 0, s>>>(W.grp(g, per), v, y);
        note_launch();
    }
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status rve3_solve_correctors(const rve_realization* r, int32_t batch, const uint8_t* mask,
                                 const double* coef, const rve3_solve_opts* opts, double* u,
                                 rve3_solve_info* info, void* ws, size_t ws_bytes,
                                 void* stream) {
    const rve3_solve_opts o = resolved3(opts);
    if (!valid_scheme(o.scheme)) return RVE_EINVAL;
    if (o.precision != RVE_FP64 && o.precision != RVE_MIXED) return RVE_EINVAL;
    if (!std::isfinite(o.delta) || o.delta < 0.0 || !(o.tol < 1.0) || !(o.inner_tol < 1.0))
        return RVE_EINVAL;
    Plan3 p;
    rve_status st = make_plan3(r, batch, p);
    if (st != RVE_OK) return st;
    if ((!mask && !coef) || !u || !info || !ws || ws_misaligned(ws)) return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    if ((st = setup3(p, w, s, true)) != RVE_OK) return st;
    const Ws3 W{&p, w};
    const Cells3T<double> cs64{mask, coef};
    if (o.precision == RVE_MIXED) {
        if (coef) {
            k3_coef32<<<(unsigned)((p.nodes + 255) / 256), 256, 0, s>>>(coef, W.c32(), p.nodes);
            note_launch();
        }
        const Cells3T<float> cs32{mask, coef ? W.c32() : nullptr};
        st = solve_units<float2>(p, w, cs64, cs32, o, s);
    } else {
        st = solve_units<double2>(p, w, cs64, cs64, o, s);
    }
    if (st != RVE_OK) return st;
    for (const Group3& g : p.groups) {
        const int per = (int)(nodes_of(g) / T3);
        k3_join<<<nblocks(g, per), T3, 0, s>>>(W.grp(g, per), W.vec<double2>(V_U), u);
        note_launch();
    }
    k3_report<<<(p.batch + 127) / 128, 128, 0, s>>>(W.sc(), W.desc(), W.u_of(), p.batch, info);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
    prof3_sync(s);
    return RVE_OK;
}

rve_status rve3_a_hom(const rve_realization* r, int32_t batch, const uint8_t* mask,
                      const double* coef, int32_t scheme, const double* u, double* A,
                      double* A_flux, void* ws, size_t ws_bytes, void* stream) {
    Plan3 p;
    rve_status st = make_plan3(r, batch, p);
    if (st != RVE_OK) return st;
    if ((!mask && !coef) || !u || !A || !ws || ws_misaligned(ws) || !valid_scheme(scheme)) return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    if ((st = setup3(p, w, s, false)) != RVE_OK) return st;
    const Ws3 W{&p, w};
    const Cells3T<double> cs{mask, coef};
    for (const Group3& g : p.groups) {
        const int per = (int)(nodes_of(g) / T3);
        const Grp gr = W.grp(g, per, true);
        if (scheme == RVE_Q1_LUMPED)
            k3_a_hom_part<1><<<nblocks(g, per, true), T3, 0, s>>>(gr, cs, u, W.part());
        else
            k3_a_hom_part<0><<<nblocks(g, per, true), T3, 0, s>>>(gr, cs, u, W.part());
        k3_a_hom_final<<<g.count / 2, 256, 0, s>>>(W.grp(g, 1, true), W.part(), A, A_flux);
        note_launch(2);
    }
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status rve3_statistics(const double* A, int64_t N, double L, double* mean, double* var,
                           double* Q) {
    if (!A || N < 2 || !(L > 0.0) || !std::isfinite(L)) return RVE_EINVAL;
    double m[9] = {};
    for (int64_t k = 0; k < N; ++k)
        for (int e = 0; e < 9; ++e) m[e] += A[9 * k + e];
    for (int e = 0; e < 9; ++e) m[e] /= (double)N;
    std::vector<double> c(81, 0.0);
    for (int64_t k = 0; k < N; ++k) {
        double dev[9];
        for (int e = 0; e < 9; ++e) dev[e] = A[9 * k + e] - m[e];
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) c[9 * i + j] += dev[i] * dev[j];
    }
    const double L3 = L * L * L;
    for (int e = 0; e < 9; ++e) {
        if (mean) mean[e] = m[e];
        if (var) var[e] = c[10 * e] / (double)(N - 1);
    }
    if (Q)
        for (int e = 0; e < 81; ++e) Q[e] = L3 * c[e] / (double)(N - 1);
    return RVE_OK;
}

int32_t rve3_profile_read(double* ms, int64_t* launches) {
    for (int j = 0; j < P3_K; ++j) {
        if (ms) ms[j] = g_prof3.ms[j];
        if (launches) launches[j] = (int64_t)g_prof3.launches[j];
        g_prof3.ms[j] = 0.0;
        g_prof3.launches[j] = 0;
    }
    return P3_K;
}

}  // extern "C"
