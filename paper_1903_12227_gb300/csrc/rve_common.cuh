// rve_common.cuh -- device-side batch descriptors, coefficient access and the
// matrix-free Q1 stencil shared by the kernels of librve.
//
// The stiffness of Eq. "FEM_matrix", assembled in the paper from local
// Kronecker products a_c (K1 (x) M1 + M1 (x) K1) (Sec. 3.2-3.3, Eq.
// "As_Kron"), is applied here straight from the cell values: node (i,j)
// touches the four cells mm = (i-1,j-1), m0 = (i-1,j), 0m = (i,j-1),
// 00 = (i,j), and with the 1D mass weights w0 = M1[0][0]/h, w1 = M1[0][1]/h
// (consistent: 1/3, 1/6; trapezoid-lumped: 1/2, 0) its row reads
//   centre  2 w0 (a_mm + a_m0 + a_0m + a_00)
//   edge    (w1 - w0) (sum of the two cells the edge neighbour shares)
//   corner  -2 w1 (the one shared cell).
// The right-hand side of Eq. "FEM_discr_RHS" with the same quadrature is
//   f_1 = h/2 (a_0m + a_00 - a_mm - a_m0),  f_2 = h/2 (a_m0 + a_00 - a_mm - a_0m).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rve_device.cuh"

namespace rve {

// Per-realization descriptor, built on the host and copied into the
// workspace.
struct RDesc {
    int32_t n, log2n, L, s;
    int32_t n_incl;
    int32_t tS, tU, tC; // fused-kernel tile geometry (rows, rows, columns)
    int64_t node_off;   // first node of this realization in packed vectors
    int64_t word_off;   // first mask word
    double a_matrix, a_incl;
    double h;           // 1/m0
    double c0;          // (a_matrix + a_incl)/2, the preconditioner's scale
    double inv_vol;     // 1/L^2
    uint64_t key;       // SplitMix64 key of the realization
};

// Descriptors passed by value to the launches that take no workspace
// (at most CHUNK realizations per launch; larger batches are split).
constexpr int CHUNK = 96;
struct DescChunk {
    int32_t count;
    int32_t start[CHUNK + 1];   // prefix sum of the launch's work units
    RDesc d[CHUNK];
};

// Realization owning tile `t` of a launch whose tiles are prefix-summed in
// start[0..batch] (start[b] = first tile of realization b).  `start` may
// live in global memory or in the kernel's parameter space, so it is read
// with ordinary (generic) loads.
__device__ __forceinline__ int find_real(const int32_t* start, int batch, int t) {
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------ SplitMix64 --
// Steele, Lea & Flood (OOPSLA 2014): output k (k >= 1) of the stream seeded
// with s is mix(s + k * GAMMA).  Realization key = output (index+1) of the
// run seed's stream; draw `ctr` under `tag` = output ((tag << 40) + ctr + 1)
// of the key's stream.
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t sm64_draw(uint64_t key, uint32_t tag, uint64_t ctr) {
    return sm64_mix(key + (((uint64_t)tag << 40) + ctr + 1) * 0x9E3779B97F4A7C15ull);
}
// Cell-coefficient source: bitmask + the two values, or an explicit array;
// and the right-hand side: the corrector loads f_1, f_2 formed from the cells
// (f == NULL), or a caller's load vector pair per node.
struct CoefSrc {
    const uint32_t* __restrict__ mask;   // packed over the batch
    const double* __restrict__ coef;     // packed over the batch (or NULL)
    const double2* __restrict__ f;       // packed load vectors (or NULL)
    __device__ __forceinline__ double cell(const RDesc& d, int c1, int c2) const {
        const int64_t c = (int64_t)c1 * d.n + c2;
        if (coef) return __ldg(coef + d.node_off + c);
        const uint32_t w = __ldg(mask + d.word_off + (c >> 5));
        return ((w >> (c & 31)) & 1u) ? d.a_incl : d.a_matrix;
    }
};

// The four cells around node (i,j) with periodic wrap, in arithmetic type T.
template <typename T> struct CellsT { T mm, m0, z0m, z00; };
typedef CellsT<double> Cells4;
template <typename T> __device__ __forceinline__ CellsT<T> cells_as(const Cells4& a) {
    return CellsT<T>{(T)a.mm, (T)a.m0, (T)a.z0m, (T)a.z00};
}

__device__ __forceinline__ Cells4 cells_at(const CoefSrc& cs, const RDesc& d, int i, int j) {
    const int im = (i - 1) & (d.n - 1), jm = (j - 1) & (d.n - 1);
    Cells4 c;
    c.mm = cs.cell(d, im, jm);
    c.m0 = cs.cell(d, im, j);
    c.z0m = cs.cell(d, i, jm);
    c.z00 = cs.cell(d, i, j);
    return c;
}

template <int SCHEME> struct Weights;
template <> struct Weights<0> {   // consistent Q1
    static constexpr double w0 = 1.0 / 3.0, w1 = 1.0 / 6.0;
};
template <> struct Weights<1> {   // trapezoid-lumped (paper's I-hat)
    static constexpr double w0 = 0.5, w1 = 0.0;
};

// q(i,j) = (A p)(i,j) for both correctors (V = float2 or double2), with the
// nine neighbours supplied by the caller.  T is the arithmetic type.
template <int SCHEME, typename V>
__device__ __forceinline__ V stencil_apply(const CellsT<typename ScalarOf<V>::T>& a, V pmm, V pm0,
                                           V pmp, V p0m, V p00, V p0p, V ppm, V pp0, V ppp) {
    typedef typename ScalarOf<V>::T T;
    const T w0 = (T)Weights<SCHEME>::w0, w1 = (T)Weights<SCHEME>::w1;
    const T amm = a.mm, am0 = a.m0, a0m = a.z0m, a00 = a.z00;
    const T cc = (T)2 * w0 * ((amm + am0) + (a0m + a00));
    const T e = w1 - w0;
    const T en = e * (amm + am0);   // edge to (i-1, j)
    const T ew = e * (amm + a0m);   // edge to (i, j-1)
    const T ee = e * (am0 + a00);   // edge to (i, j+1)
    const T es = e * (a0m + a00);   // edge to (i+1, j)
    V q;
    q.x = cc * p00.x + en * pm0.x + ew * p0m.x + ee * p0p.x + es * pp0.x;
    q.y = cc * p00.y + en * pm0.y + ew * p0m.y + ee * p0p.y + es * pp0.y;
    if (SCHEME == 0) {
        const T g = (T)(-2) * w1;
        q.x += g * (amm * pmm.x + am0 * pmp.x + a0m * ppm.x + a00 * ppp.x);
        q.y += g * (amm * pmm.y + am0 * pmp.y + a0m * ppm.y + a00 * ppp.y);
    }
    return q;
}

// Galerkin right-hand sides at a node from its four cells.
__device__ __forceinline__ double2 rhs_at(const Cells4& a, double h) {
    const double hh = 0.5 * h;
    return make_double2(hh * ((a.z0m + a.z00) - (a.mm + a.m0)), hh * ((a.m0 + a.z00) - (a.mm + a.z0m)));
}

// Right-hand side at a node: the caller's load vector, or the corrector
// loads from the node's four cells.
__device__ __forceinline__ double2 load_at(const CoefSrc& cs, const RDesc& d, int64_t node,
                                           const Cells4& a) {
    return cs.f ? cs.f[d.node_off + node] : rhs_at(a, d.h);
}

// Reciprocal of the preconditioner's symbol: the approximate hardware
// reciprocal in FP32 (a preconditioner needs no correct rounding), exact
// division in FP64.
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

// Conversions between the FP64 and FP32 pair types.
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2((double)v.x, (double)v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
template <typename V> __device__ __forceinline__ V from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) { return to_f2(v); }

// Lookup tables shared by all sizes n = 2^p, p <= 11: entry m of the table
// for n sits at index n + m.
struct Tables {
    const double2* __restrict__ tw64;   // exp(-2 pi i m/n)
    const float2* __restrict__ tw32;
    const double* __restrict__ lap;     // 4 sin^2(pi m/n)
    const float* __restrict__ lap32;
    const double* __restrict__ rho64;   // column-filter root for lambda = lap[m], delta = 0
    const float* __restrict__ rho32;    // (1 at m = 0: the singular column)
};
template <typename T> __device__ __forceinline__ const T* rho_table(const Tables& tb, int n);
template <> __device__ __forceinline__ const double* rho_table<double>(const Tables& tb, int n) { return tb.rho64 + n; }
template <> __device__ __forceinline__ const float* rho_table<float>(const Tables& tb, int n) { return tb.rho32 + n; }

// Root rho < 1 of rho + 1/rho = 2 + mu (mu > 0), the decay of the periodic
// tridiagonal inverse; written without cancellation.
__host__ __device__ __forceinline__ double filter_root(double mu) {
    return 1.0 / (1.0 + 0.5 * mu + sqrt(mu * (1.0 + 0.25 * mu)));
}

// Column solve geometry: a thread holds one segment of `col_seg_rows` rows
// of one column in registers (n/16 rows up to n = 512, then 32; at most 16
// for FP64 pairs), so a column spans n / col_seg_rows threads.
__host__ __device__ constexpr int col_seg_rows(int n, int vbytes) {
    return (vbytes == 16) ? ((n <= 512 ? n / 16 : 32) < 16 ? (n <= 512 ? n / 16 : 32) : 16)
                          : (n <= 512 ? n / 16 : 32);
}
template <typename T> __device__ __forceinline__ const T* lap_table(const Tables& tb, int n);
template <> __device__ __forceinline__ const double* lap_table<double>(const Tables& tb, int n) { return tb.lap + n; }
template <> __device__ __forceinline__ const float* lap_table<float>(const Tables& tb, int n) { return tb.lap32 + n; }
template <typename V> __device__ __forceinline__ const V* twiddles(const Tables& tb, int n);
template <> __device__ __forceinline__ const double2* twiddles<double2>(const Tables& tb, int n) { return tb.tw64 + n; }
template <> __device__ __forceinline__ const float2* twiddles<float2>(const Tables& tb, int n) { return tb.tw32 + n; }

}  // namespace rve
