// rve3d.cu -- the 3D extension of the RVE corrector method (the paper's
// remark that the scheme extends to 3D): cubes on the torus [0,L)^3, the
// trilinear Q1 element K1(x)M1(x)M1 + M1(x)K1(x)M1 + M1(x)M1(x)K1, three
// corrector problems solved by PCG with B = c0 A_Delta + delta I (A_Delta
// the periodic 7-point Laplacian), and the 3x3 homogenized matrix.  FP64.
//
// Grid: n = L m0 nodes per axis, node (i,j,k) at ((i n + j) n + k) within
// the realization; cell (i,j,k) has lower corner node (i,j,k); local corner
// a = 4 a1 + 2 a2 + a3.  The three correctors travel as two pairs (double2):
// (u_1, u_2) and (u_3, 0), so that every kernel -- the stencil, the
// Hartley transforms (pair-packed complex FFT) and the column solve -- is
// shared with the pair layout of the 2D path.
//
// Preconditioner: the Hartley transforms along x (contiguous lines) and y
// (lines of stride n) diagonalise two factors of A_Delta; along z (lines of
// stride n^2) each (kx, ky) leaves the periodic tridiagonal system
// c0 (T + lambda(kx) + lambda(ky)) + delta, solved by the causal/anticausal
// filter pair of the 2D column pass (rve_colsolve.cuh) with the shift
// c0 lambda(ky) folded into delta.  B^{-1} = n^-2 Hx Hy M^-1 Hy Hx.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rve_colsolve.cuh"
#include "rve_common.cuh"
#include "rve_internal.h"

namespace rve {

// ------------------------------------------------------------ element --
// Entry (a, b) of the element matrix (local corners 4 a1 + 2 a2 + a3); the
// loops that call it unroll, so every entry folds to a constant times 1/h.
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

__device__ __forceinline__ int64_t n3(const RDesc& d, int i, int j, int k) {
    const int m = d.n - 1;
    return d.node_off + ((((int64_t)(i & m) << d.log2n) + (j & m)) << d.log2n) + (k & m);
}

// Cell values: a byte mask with the two values, or an explicit array.
struct Cells3 {
    const uint8_t* __restrict__ mask;
    const double* __restrict__ coef;
    __device__ __forceinline__ double at(const RDesc& d, int i, int j, int k) const {
        const int64_t c = n3(d, i, j, k);
        if (coef) return coef[c];
        return mask[c] ? d.a_incl : d.a_matrix;
    }
};

constexpr int T3 = 256;   // threads of the node kernels

// --------------------------------------------------------------- field --
// One thread per (cube, row d1, d2): sets the s cells along the third axis.
__global__ void k3_gen_field(const RDesc d, uint8_t* __restrict__ mask) {
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
    for (int d3 = 0; d3 < d.s; ++d3) mask[n3(d, c[0] + d1, c[1] + d2, c[2] + d3)] = 1;
}

// ------------------------------------------------- stiffness and loads --
// y = A x for one pair: for each of the 8 cells around the node, a_c times
// the element row of the node's local corner against the cell's corners.
// With `part` set, also the block's partials of x.y per component (the
// p.q of CG), two doubles per block.
template <int SCHEME>
__global__ void __launch_bounds__(T3) k3_stiffness(const RDesc d, Cells3 cs,
                                                   const double2* __restrict__ x,
                                                   double2* __restrict__ y, double* part) {
    const int64_t node = (int64_t)blockIdx.x * T3 + threadIdx.x;
    const int n = d.n;
    const int i = (int)(node >> (2 * d.log2n)), j = (int)((node >> d.log2n) & (n - 1)),
              k = (int)(node & (n - 1));
    double2 w[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) w[o] = x[n3(d, i + o / 9 - 1, j + (o / 3) % 3 - 1, k + o % 3 - 1)];
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {   // cell offset (-c1, -c2, -c3), c = 4 c1 + 2 c2 + c3
        const int c1 = c >> 2, c2 = (c >> 1) & 1, c3 = c & 1;
        const double a = cs.at(d, i - c1, j - c2, k - c3);
        const int l = c;   // the node is corner (c1, c2, c3) of that cell
        double2 s = make_double2(0.0, 0.0);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int o = (((b >> 2) - c1 + 1) * 3 + (((b >> 1) & 1) - c2 + 1)) * 3 + ((b & 1) - c3 + 1);
            const double e = e3<SCHEME>(l, b, d.h);
            s.x = fma(e, w[o].x, s.x);
            s.y = fma(e, w[o].y, s.y);
        }
        acc.x = fma(a, s.x, acc.x);
        acc.y = fma(a, s.y, acc.y);
    }
    y[d.node_off + node] = acc;
    if (part) {   // block-uniform
        __shared__ double red[8];
        const double sx = block_sum(w[13].x * acc.x, red);
        const double sy = block_sum(w[13].y * acc.y, red);
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = sx;
            part[2 * blockIdx.x + 1] = sy;
        }
    }
}

// Corrector loads f_i = -sum_c a_c P_c^T E xi_i (xi_i = h x corner bit i).
// Every row of M1 sums to h/2 (both schemes) and every row of K1 to 0, so
// of the three Kronecker terms only the one with K1 along axis i survives,
// and the row of E xi_i at local corner l is (h^2/4) (+1 if l_i = 1, -1
// otherwise).  Summed over the 8 cells around the node (the node is corner
// c of the cell at offset -c):
//     f_i = (h^2/4) (sum_{c_i = 0} a_c - sum_{c_i = 1} a_c),
// which is exactly zero where the 8 cells agree.  Pair 0 gets (f_1, f_2),
// pair 1 gets (f_3, 0).
__global__ void __launch_bounds__(T3) k3_rhs(const RDesc d, Cells3 cs, int pair,
                                             double2* __restrict__ f) {
    const int64_t node = (int64_t)blockIdx.x * T3 + threadIdx.x;
    const int n = d.n;
    const int i = (int)(node >> (2 * d.log2n)), j = (int)((node >> d.log2n) & (n - 1)),
              k = (int)(node & (n - 1));
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = cs.at(d, i - (c >> 2), j - ((c >> 1) & 1), k - (c & 1));
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
    f[d.node_off + node] = pair == 0 ? make_double2(v[0], v[1]) : make_double2(v[2], 0.0);
}

// r = f - q (true residual) and its partial |r|^2 per component.
__global__ void __launch_bounds__(T3) k3_resid(const RDesc d, const double2* __restrict__ f,
                                               const double2* __restrict__ q, double2* __restrict__ r,
                                               double* part) {
    __shared__ double red[8];
    const int64_t node = d.node_off + (int64_t)blockIdx.x * T3 + threadIdx.x;
    const double2 v = make_double2(f[node].x - q[node].x, f[node].y - q[node].y);
    r[node] = v;
    const double sx = block_sum(v.x * v.x, red);
    const double sy = block_sum(v.y * v.y, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sx;
        part[2 * blockIdx.x + 1] = sy;
    }
}

// ------------------------------------------------------ preconditioner --
// Hartley transform of lines of n nodes (pair-packed complex FFT, register
// Stockham, see rve_device.cuh): dst = scale H src (src may equal dst).
// AXIS 2: x lines (contiguous), threads of a line side by side; AXIS 1: y
// lines (stride n), the lines of a block side by side so that each load
// instruction reads consecutive nodes.  With `rd` set, also the block's
// partials of rd.dst per component (the r.z of CG), two doubles per block.
template <int LOG2N, int AXIS>
__global__ void __launch_bounds__(256) k3_lines(const RDesc d, Tables tb,
                                                const double2* src, double2* dst,
                                                double scale, const double2* __restrict__ rd,
                                                double* part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[8];
    constexpr int n = 1 << LOG2N, T = n / 8;
    const int G = blockDim.x / T;
    int q, t;
    if (AXIS == 2) { q = threadIdx.x / T; t = threadIdx.x - q * T; }
    else { t = threadIdx.x / G; q = threadIdx.x - t * G; }
    const int64_t line = (int64_t)blockIdx.x * G + q;   // < n^2
    int64_t base, stride;
    if (AXIS == 2) { base = d.node_off + line * n; stride = 1; }
    else { base = d.node_off + (line / n) * (int64_t)n * n + (line % n); stride = n; }
    double2* buf = reinterpret_cast<double2*>(smem_raw) + q * seq_stride(n);
    double2 w[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) w[m] = src[base + (t + m * T) * stride];
    fft_reg<FFT_TO_BOTH, LOG2N>(w, buf, LOG2N, t, twiddles<double2>(tb, n), true);
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int kx = t + m * T;
        const double2 hv = hartley_pair(w[m], buf[pidx((n - kx) & (n - 1))]);
        const double2 o = make_double2(scale * hv.x, scale * hv.y);
        dst[base + (int64_t)kx * stride] = o;
        if (rd) {
            const double2 r = rd[base + (int64_t)kx * stride];
            ax = fma(r.x, o.x, ax);
            ay = fma(r.y, o.y, ay);
        }
    }
    if (rd) {   // block-uniform
        const double sx = block_sum(ax, red);
        const double sy = block_sum(ay, red);
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = sx;
            part[2 * blockIdx.x + 1] = sy;
        }
    }
}

// Tridiagonal solves along z for the lines (kx = c0 .. c0+C-1, ky =
// blockIdx.y) after the x and y transforms; writes M^{-1} t / n in place.
template <int LOG2N>
__global__ void __launch_bounds__(512) k3_zsolve(const RDesc d, Tables tb, double delta,
                                                 double2* __restrict__ v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[64];
    __shared__ double csc[1];
    constexpr int n = 1 << LOG2N;
    const int ky = blockIdx.y, c0 = blockIdx.x * d.tC;
    const double delta_eff = delta + d.c0 * tb.lap[n + ky];   // the y shift folded in
    col_solve_body<double2, LOG2N>(
        [&](int r, int kx) { return v[d.node_off + (((int64_t)r * n + ky) * n) + kx]; },
        [&](int r, int kx, double2 val) { v[d.node_off + (((int64_t)r * n + ky) * n) + kx] = val; },
        d, c0, reinterpret_cast<double2*>(smem_raw), tb, delta_eff, red, nullptr, csc);
}

// ------------------------------------------------------------- A_hom --
// Per tile of T3 cells, partial sums of sum a_c, the energy terms
// a_c v_i^T E v_j (ij = 11 12 13 22 23 33) and the flux terms a_c int_c
// d_j (x_i + phi_i) (ij = 11 12 13 21 22 23 31 32 33), v_i = xi_i + P_c u_i.
constexpr int A3_NP = 16;
template <int SCHEME>
__global__ void __launch_bounds__(T3) k3_a_hom_part(const RDesc d, Cells3 cs,
                                                    const double2* __restrict__ u12,
                                                    const double2* __restrict__ u3,
                                                    double* __restrict__ part) {
    __shared__ double red[8];
    const int64_t cell = (int64_t)blockIdx.x * T3 + threadIdx.x;
    const int n = d.n;
    const int i = (int)(cell >> (2 * d.log2n)), j = (int)((cell >> d.log2n) & (n - 1)),
              k = (int)(cell & (n - 1));
    const double h = d.h;
    const double a = cs.at(d, i, j, k);
    double v[3][8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int64_t g = n3(d, i + (b >> 2), j + ((b >> 1) & 1), k + (b & 1));
        const double2 p = u12[g], s = u3[g];
        v[0][b] = p.x + h * (double)(b >> 2);
        v[1][b] = p.y + h * (double)((b >> 1) & 1);
        v[2][b] = s.x + h * (double)(b & 1);
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
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * A3_NP + p] = s;
    }
}

__global__ void k3_a_hom_final(const RDesc d, const double* __restrict__ part, int tiles,
                               double* __restrict__ A, double* __restrict__ Af) {
    double s[A3_NP];
#pragma unroll
    for (int p = 0; p < A3_NP; ++p) s[p] = warp_sum_array(part + p, tiles, A3_NP);
    if (threadIdx.x != 0) return;
    const double iv = d.inv_vol;
    const int sym[3][3] = {{1, 2, 3}, {2, 4, 5}, {3, 5, 6}};
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) {
            A[3 * x + y] = s[sym[x][y]] * iv;
            if (Af) Af[3 * x + y] = s[7 + 3 * x + y] * iv;
        }
}

// ------------------------------------------- layout: triples <-> pairs --
__global__ void k3_split(const RDesc d, const double* __restrict__ x3, double2* __restrict__ p12,
                         double2* __restrict__ p3) {
    const int64_t node = d.node_off + (int64_t)blockIdx.x * T3 + threadIdx.x;
    p12[node] = make_double2(x3[3 * node], x3[3 * node + 1]);
    p3[node] = make_double2(x3[3 * node + 2], 0.0);
}

__global__ void k3_join(const RDesc d, const double2* __restrict__ p12,
                        const double2* __restrict__ p3, double* __restrict__ x3) {
    const int64_t node = d.node_off + (int64_t)blockIdx.x * T3 + threadIdx.x;
    x3[3 * node] = p12[node].x;
    x3[3 * node + 1] = p12[node].y;
    x3[3 * node + 2] = p3[node].x;
}

__global__ void k3_report(const PlainScal* s12, const PlainScal* s3, rve3_solve_info* info) {
    rve3_solve_info r;
    r.iters[0] = s12->iters[0];
    r.iters[1] = s12->iters[1];
    r.iters[2] = s3->iters[0];
    r.status = s12->status != RVE_OK ? s12->status : s3->status;
    r.relres[0] = s12->relres[0];
    r.relres[1] = s12->relres[1];
    r.relres[2] = s3->relres[0];
    *info = r;
}

// ------------------------------------------------------------ profile --
// Event timing of every 3D launch by kind (diagnostics, enabled together
// with the fused solver's profiler by rve_profile_enable; process-wide, not
// thread-safe): 0 stiffness, 1 line transform (x or y), 2 z solve,
// 3 vector steps of CG (dots, updates), 4 scalar steps (one warp each).
enum { P3_STIFF = 0, P3_LINES, P3_ZSOLVE, P3_VECTOR, P3_SCALAR, P3_K };
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
struct Plan3 {
    int batch = 0;
    std::vector<RDesc> desc;
    int64_t nodes = 0;
    int max_log2n = 5;
    // workspace: descriptors, tables, two scalar blocks, partials, 7 pair vectors
    size_t o_desc = 0, o_tw64 = 0, o_tw32 = 0, o_lap = 0, o_lap32 = 0, o_rho64 = 0, o_rho32 = 0;
    size_t o_sc = 0, o_part = 0, o_vec = 0, total = 0;
    int64_t max_nodes_one = 0;
};

constexpr int N3_MIN = 32, N3_MAX = 256;
constexpr int Z_THREADS = 512;

static int col_tile3(int n) {   // columns of a z-solve block (FP64 segments)
    const int P = n / col_seg_rows(n, 16);
    return std::min(n, Z_THREADS / P);
}

static rve_status make_plan3(const rve_realization* r, int32_t batch, Plan3& p) {
    if (!r || batch <= 0 || batch > (1 << 16)) return RVE_EINVAL;
    p.batch = batch;
    p.desc.assign(batch, RDesc{});
    p.nodes = 0;
    p.max_log2n = 5;
    p.max_nodes_one = 0;
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
        RDesc& d = p.desc[b];
        std::memset(&d, 0, sizeof(d));
        d.n = n;
        d.log2n = 31 - __builtin_clz((unsigned)n);
        d.L = x.L;
        d.s = x.incl_cells;
        d.n_incl = x.n_incl;
        d.tC = col_tile3(n);
        d.node_off = p.nodes;
        d.a_matrix = x.a_matrix;
        d.a_incl = x.a_incl;
        d.h = 1.0 / (double)x.m0;
        d.c0 = 0.5 * (x.a_matrix + x.a_incl);
        d.inv_vol = 1.0 / ((double)x.L * (double)x.L * (double)x.L);
        d.key = sm64_mix(x.seed + (x.index + 1) * 0x9E3779B97F4A7C15ull);
        const int64_t nn = (int64_t)n * n * n;
        p.nodes += nn;
        p.max_nodes_one = std::max(p.max_nodes_one, nn);
        p.max_log2n = std::max(p.max_log2n, d.log2n);
    }
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = up(off + bytes); return o; };
    const size_t tab = (size_t)2 << p.max_log2n;
    p.o_desc = take(sizeof(RDesc) * batch);
    p.o_tw64 = take(sizeof(double2) * tab);
    p.o_tw32 = take(sizeof(float2) * tab);
    p.o_lap = take(sizeof(double) * tab);
    p.o_lap32 = take(sizeof(float) * tab);
    p.o_rho64 = take(sizeof(double) * tab);
    p.o_rho32 = take(sizeof(float) * tab);
    p.o_sc = take(sizeof(PlainScal) * 2);
    p.o_part = take(sizeof(double) * A3_NP * (size_t)(p.max_nodes_one / T3 + 1));
    p.o_vec = take(sizeof(double2) * 7 * (size_t)p.nodes);
    p.total = off;
    return RVE_OK;
}

static Tables tables3(const Plan3& p, char* w) {
    Tables tb;
    tb.tw64 = reinterpret_cast<const double2*>(w + p.o_tw64);
    tb.tw32 = reinterpret_cast<const float2*>(w + p.o_tw32);
    tb.lap = reinterpret_cast<const double*>(w + p.o_lap);
    tb.lap32 = reinterpret_cast<const float*>(w + p.o_lap32);
    tb.rho64 = reinterpret_cast<const double*>(w + p.o_rho64);
    tb.rho32 = reinterpret_cast<const float*>(w + p.o_rho32);
    return tb;
}

static double2* vec3(const Plan3& p, char* w, int k) {
    return reinterpret_cast<double2*>(w + p.o_vec) + (size_t)k * (size_t)p.nodes;
}

static int64_t blocks3(const RDesc& d) { return ((int64_t)d.n * d.n * d.n) / T3; }

// dst = B^{-1} src for one realization (one pair); src is read by the first
// pass only (it may equal dst).  With `rd`, part receives the partials of
// rd.dst (n^3 / 2048 blocks of two doubles).
template <int LG>
static cudaError_t precond3_t(const RDesc& d, const Tables& tb, double delta, const double2* src,
                              double2* dst, const double2* rd, double* part, cudaStream_t s) {
    constexpr int n = 1 << LG, T = n / 8;
    const int G = 256 / T;
    const size_t smem = (size_t)G * seq_stride(n) * sizeof(double2);
    const unsigned lines = (unsigned)(((int64_t)n * n) / G);
    const int P = n / col_seg_rows(n, 16);
    const size_t zsmem = (size_t)(2 * d.tC + 2) * P * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k3_lines<LG, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k3_lines<LG, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    {
        Span3 sp(s, P3_LINES);
        k3_lines<LG, 2><<<lines, 256, smem, s>>>(d, tb, src, dst, 1.0, nullptr, nullptr);
    }
    {
        Span3 sp(s, P3_LINES);
        k3_lines<LG, 1><<<lines, 256, smem, s>>>(d, tb, dst, dst, 1.0, nullptr, nullptr);
    }
    {
        Span3 sp(s, P3_ZSOLVE);
        k3_zsolve<LG><<<dim3((unsigned)(n / d.tC), (unsigned)n), Z_THREADS, zsmem, s>>>(d, tb, delta, dst);
    }
    {
        Span3 sp(s, P3_LINES);
        k3_lines<LG, 1><<<lines, 256, smem, s>>>(d, tb, dst, dst, 1.0, nullptr, nullptr);
    }
    {
        Span3 sp(s, P3_LINES);
        k3_lines<LG, 2><<<lines, 256, smem, s>>>(d, tb, dst, dst, 1.0 / (double)n, rd, part);
    }
    note_launch(5);
    return cudaGetLastError();
}

static cudaError_t precond3(const RDesc& d, const Tables& tb, double delta, const double2* src,
                            double2* dst, cudaStream_t s, const double2* rd = nullptr,
                            double* part = nullptr) {
    switch (d.log2n) {
        case 5: return precond3_t<5>(d, tb, delta, src, dst, rd, part, s);
        case 6: return precond3_t<6>(d, tb, delta, src, dst, rd, part, s);
        case 7: return precond3_t<7>(d, tb, delta, src, dst, rd, part, s);
        default: return precond3_t<8>(d, tb, delta, src, dst, rd, part, s);
    }
}

// Blocks of the last line pass (its partials): n^2 / G lines of G per block.
static int lines_blocks(const RDesc& d) {
    const int T = d.n / 8, G = 256 / T;
    return (int)(((int64_t)d.n * d.n) / G);
}

static cudaError_t stiffness3(const RDesc& d, Cells3 cs, int scheme, const double2* x, double2* y,
                              cudaStream_t s, double* part = nullptr) {
    Span3 sp(s, P3_STIFF);
    if (scheme == RVE_Q1_LUMPED) k3_stiffness<1><<<(unsigned)blocks3(d), T3, 0, s>>>(d, cs, x, y, part);
    else k3_stiffness<0><<<(unsigned)blocks3(d), T3, 0, s>>>(d, cs, x, y, part);
    note_launch();
    return cudaGetLastError();
}

// The loads are the same for both schemes (the mass rows sum to h/2 in each).
static cudaError_t rhs3(const RDesc& d, Cells3 cs, int pair, double2* f, cudaStream_t s) {
    k3_rhs<<<(unsigned)blocks3(d), T3, 0, s>>>(d, cs, pair, f);
    note_launch();
    return cudaGetLastError();
}

// Setup common to every 3D entry point: descriptors and tables into ws.
static rve_status setup3(const Plan3& p, char* w, cudaStream_t s) {
    if (cudaMemcpyAsync(w + p.o_desc, p.desc.data(), sizeof(RDesc) * p.batch,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return RVE_ECUDA;
    return fill_tables(tables3(p, w), p.max_log2n, s) == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

// PCG (Saad, Iterative Methods for Sparse Linear Systems, Algorithm 9.1)
// for one pair of one realization: A u = f with f given, u from 0.  Per
// iteration: q = A p with the p.q partials, the step, u and r updates with
// |r|^2, z = B^{-1} r with the r.z partials, the new direction.
static rve_status pcg3_pair(const Plan3& p, char* w, int b, Cells3 cs, const rve3_solve_opts& o,
                            const double2* f, double2* u, PlainScal* sc, cudaStream_t s) {
    const RDesc& d = p.desc[b];
    const RDesc* desc = reinterpret_cast<const RDesc*>(w + p.o_desc);
    const Tables tb = tables3(p, w);
    double2* r = vec3(p, w, 2);
    double2* z = vec3(p, w, 3);
    double2* pp = vec3(p, w, 4);
    double2* q = vec3(p, w, 5);
    double* part = reinterpret_cast<double*>(w + p.o_part);
    const int nb = (int)(((int64_t)d.n * d.n * d.n) / PL_NODES);   // vector kernels
    const int ns = (int)blocks3(d);                                  // stiffness
    const int nl = lines_blocks(d);                                  // last line pass
    const size_t bytes = sizeof(double2) * (size_t)d.n * d.n * d.n;
    auto vec_step = [&](auto&& launch) {
        Span3 sp(s, P3_VECTOR);
        launch();
    };
    auto scalar_step = [&](auto&& launch) {
        Span3 sp(s, P3_SCALAR);
        launch();
    };
    // u = 0, r = f, p = 0
    if (cudaMemcpyAsync(r + d.node_off, f + d.node_off, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(u + d.node_off, 0, bytes, s) != cudaSuccess ||
        cudaMemsetAsync(pp + d.node_off, 0, bytes, s) != cudaSuccess)
        return RVE_ECUDA;
    vec_step([&] { k_pl_dot<<<nb, PL_THREADS, 0, s>>>(desc, b, r, r, part); });
    scalar_step([&] { k_pl_scalar<<<1, 32, 0, s>>>(sc, part, nb, SC_FNORM, o.tol, o.max_iter); });
    if (precond3(d, tb, o.delta, r, z, s, r, part) != cudaSuccess) return RVE_ECUDA;
    scalar_step([&] { k_pl_scalar<<<1, 32, 0, s>>>(sc, part, nl, SC_RHO0, o.tol, o.max_iter); });
    vec_step([&] { k_pl_xpby<<<nb, PL_THREADS, 0, s>>>(desc, b, sc, z, pp); });   // p = z
    note_launch(4);
    const int every = o.check_every > 0 ? o.check_every : 8;
    PlainScal hsc;
    for (int it = 0; it < o.max_iter; ++it) {
        if (stiffness3(d, cs, o.scheme, pp, q, s, part) != cudaSuccess) return RVE_ECUDA;
        scalar_step([&] { k_pl_scalar<<<1, 32, 0, s>>>(sc, part, ns, SC_ALPHA, o.tol, o.max_iter); });
        vec_step([&] { k_pl_axpy<<<nb, PL_THREADS, 0, s>>>(desc, b, sc, u, r, pp, q, part); });
        scalar_step([&] { k_pl_scalar<<<1, 32, 0, s>>>(sc, part, nb, SC_CONV, o.tol, o.max_iter); });
        if (precond3(d, tb, o.delta, r, z, s, r, part) != cudaSuccess) return RVE_ECUDA;
        scalar_step([&] { k_pl_scalar<<<1, 32, 0, s>>>(sc, part, nl, SC_BETA, o.tol, o.max_iter); });
        vec_step([&] { k_pl_xpby<<<nb, PL_THREADS, 0, s>>>(desc, b, sc, z, pp); });
        note_launch(5);
        if ((it + 1) % every == 0 || it == 0) {
            if (cudaMemcpyAsync(&hsc, sc, sizeof(PlainScal), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return RVE_ECUDA;
            if (profile_on()) g_prof3.harvest();
            if (hsc.done) break;
        }
    }
    // true residual
    if (stiffness3(d, cs, o.scheme, u, q, s) != cudaSuccess) return RVE_ECUDA;
    k3_resid<<<(unsigned)blocks3(d), T3, 0, s>>>(d, f, q, r, part);
    k_pl_scalar<<<1, 32, 0, s>>>(sc, part, (int)blocks3(d), SC_RELRES, o.tol, o.max_iter);
    note_launch(2);
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

static rve3_solve_opts resolved3(const rve3_solve_opts* opts) {
    rve3_solve_opts o = {};
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 20000;
    if (!(o.tol > 0.0)) o.tol = 1e-10;
    if (o.check_every <= 0) o.check_every = 8;
    return o;
}

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
    for (const RDesc& d : p.desc) {
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
    if ((!mask && !coef) || !f || !ws || (scheme != RVE_Q1_CONSISTENT && scheme != RVE_Q1_LUMPED))
        return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    Cells3 cs{mask, coef};
    for (const RDesc& d : p.desc) {
        if (rhs3(d, cs, 0, vec3(p, w, 0), s) != cudaSuccess ||
            rhs3(d, cs, 1, vec3(p, w, 1), s) != cudaSuccess)
            return RVE_ECUDA;
        k3_join<<<(unsigned)blocks3(d), T3, 0, s>>>(d, vec3(p, w, 0), vec3(p, w, 1), f);
        note_launch();
    }
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status rve3_apply_stiffness(const rve_realization* r, int32_t batch, const uint8_t* mask,
                                const double* coef, int32_t scheme, const double* x, double* y,
                                void* ws, size_t ws_bytes, void* stream) {
    Plan3 p;
    rve_status st = make_plan3(r, batch, p);
    if (st != RVE_OK) return st;
    if ((!mask && !coef) || !x || !y || x == y || !ws ||
        (scheme != RVE_Q1_CONSISTENT && scheme != RVE_Q1_LUMPED))
        return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    Cells3 cs{mask, coef};
    for (const RDesc& d : p.desc) {
        k3_split<<<(unsigned)blocks3(d), T3, 0, s>>>(d, x, vec3(p, w, 0), vec3(p, w, 1));
        note_launch();
        if (stiffness3(d, cs, scheme, vec3(p, w, 0), vec3(p, w, 2), s) != cudaSuccess ||
            stiffness3(d, cs, scheme, vec3(p, w, 1), vec3(p, w, 3), s) != cudaSuccess)
            return RVE_ECUDA;
        k3_join<<<(unsigned)blocks3(d), T3, 0, s>>>(d, vec3(p, w, 2), vec3(p, w, 3), y);
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
    if (!x || !y || !ws || !std::isfinite(delta) || delta < 0.0) return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    if ((st = setup3(p, w, s)) != RVE_OK) return st;
    const Tables tb = tables3(p, w);
    for (const RDesc& d : p.desc) {
        k3_split<<<(unsigned)blocks3(d), T3, 0, s>>>(d, x, vec3(p, w, 0), vec3(p, w, 1));
        note_launch();
        if (precond3(d, tb, delta, vec3(p, w, 0), vec3(p, w, 0), s) != cudaSuccess ||
            precond3(d, tb, delta, vec3(p, w, 1), vec3(p, w, 1), s) != cudaSuccess)
            return RVE_ECUDA;
        k3_join<<<(unsigned)blocks3(d), T3, 0, s>>>(d, vec3(p, w, 0), vec3(p, w, 1), y);
        note_launch();
    }
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status rve3_solve_correctors(const rve_realization* r, int32_t batch, const uint8_t* mask,
                                 const double* coef, const rve3_solve_opts* opts, double* u,
                                 rve3_solve_info* info, void* ws, size_t ws_bytes,
                                 void* stream) {
    const rve3_solve_opts o = resolved3(opts);
    if (o.scheme != RVE_Q1_CONSISTENT && o.scheme != RVE_Q1_LUMPED) return RVE_EINVAL;
    if (!std::isfinite(o.delta) || o.delta < 0.0 || !(o.tol < 1.0)) return RVE_EINVAL;
    Plan3 p;
    rve_status st = make_plan3(r, batch, p);
    if (st != RVE_OK) return st;
    if ((!mask && !coef) || !u || !info || !ws) return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    if ((st = setup3(p, w, s)) != RVE_OK) return st;
    Cells3 cs{mask, coef};
    PlainScal* sc = reinterpret_cast<PlainScal*>(w + p.o_sc);
    for (int b = 0; b < p.batch; ++b) {
        const RDesc& d = p.desc[b];
        double2* f = vec3(p, w, 0);
        double2* upair[2] = {vec3(p, w, 1), vec3(p, w, 6)};
        for (int pair = 0; pair < 2; ++pair) {
            if (rhs3(d, cs, pair, f, s) != cudaSuccess) return RVE_ECUDA;
            if ((st = pcg3_pair(p, w, b, cs, o, f, upair[pair], sc + pair, s)) != RVE_OK) return st;
        }
        k3_join<<<(unsigned)blocks3(d), T3, 0, s>>>(d, upair[0], upair[1], u);
        k3_report<<<1, 1, 0, s>>>(sc, sc + 1, info + b);
        note_launch(2);
        if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
    }
    prof3_sync(s);
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

rve_status rve3_a_hom(const rve_realization* r, int32_t batch, const uint8_t* mask,
                      const double* coef, int32_t scheme, const double* u, double* A,
                      double* A_flux, void* ws, size_t ws_bytes, void* stream) {
    Plan3 p;
    rve_status st = make_plan3(r, batch, p);
    if (st != RVE_OK) return st;
    if ((!mask && !coef) || !u || !A || !ws ||
        (scheme != RVE_Q1_CONSISTENT && scheme != RVE_Q1_LUMPED))
        return RVE_EINVAL;
    if (ws_bytes < p.total) return RVE_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    Cells3 cs{mask, coef};
    double* part = reinterpret_cast<double*>(w + p.o_part);
    for (int b = 0; b < p.batch; ++b) {
        const RDesc& d = p.desc[b];
        const unsigned tiles = (unsigned)blocks3(d);
        k3_split<<<tiles, T3, 0, s>>>(d, u, vec3(p, w, 0), vec3(p, w, 1));
        if (scheme == RVE_Q1_LUMPED)
            k3_a_hom_part<1><<<tiles, T3, 0, s>>>(d, cs, vec3(p, w, 0), vec3(p, w, 1), part);
        else
            k3_a_hom_part<0><<<tiles, T3, 0, s>>>(d, cs, vec3(p, w, 0), vec3(p, w, 1), part);
        k3_a_hom_final<<<1, 32, 0, s>>>(d, part, (int)tiles, A + 9 * (int64_t)b,
                                        A_flux ? A_flux + 9 * (int64_t)b : nullptr);
        note_launch(3);
        if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
    }
    return RVE_OK;
}

}  // extern "C"
