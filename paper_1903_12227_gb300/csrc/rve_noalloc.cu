// rve_noalloc.cu -- rve_a_hom_noalloc: the homogenized-matrix reduction for
// callers that cannot allocate device memory.
//
// Who needs it: host programs whose device memory is entirely owned by their
// own pool allocator (a second allocator, or a stray cudaMalloc, would fail
// or fragment the reserved pool), and latency-critical loops that cannot
// afford cudaMalloc/cudaFree, which may synchronise the device.  Such
// callers also may not be able to hand over a per-call workspace.  This
// entry point needs neither: its only scratch is the fixed array below,
// which the library owns.
//
// The scratch holds 8 partial sums per tile of 1024 nodes for at most
// RVE_NOALLOC_MAX_NODES nodes per call (1 MiB).  Every GPU that loads the
// library keeps the array until the process exits.  The first call on a
// device looks up the array's device address (cudaGetSymbolAddress) with that
// device current; make that first call before any stream capture.  All calls
// share the array and it keeps the last call's contents: every partial it
// reads is written earlier in the same call, so nothing needs clearing, but
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "rve_common.cuh"
#include "rve_internal.h"

namespace rve {

constexpr int NA_TILE = 1024;                       // nodes per partial-sum tile
constexpr int NA_NP = 8;                            // partial sums per tile
constexpr int64_t NA_MAX_TILES = RVE_NOALLOC_MAX_NODES / NA_TILE;
constexpr int NA_MAX_DEVICES = 64;

// The fixed scratch (1 MiB).  Host code must not pass its name to a kernel:
// on the host this is only a stand-in symbol; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_TILES * NA_NP];

static std::mutex g_na_lock;
static double* g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch on the current device (set-up on first use).
static cudaError_t noalloc_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_na_lock);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

template <typename V>
__device__ __forceinline__ V na_ld(const V* __restrict__ x, const RDesc& d, int i, int j) {
    return x[d.node_off + ((int64_t)(i & (d.n - 1)) << d.log2n) + (j & (d.n - 1))];
}

// Partial sums of one tile (same quantities as the workspace entry point):
//   [0] sum a_c, [1..4] f_i.u_j, [5] u_1.A u_1, [6] u_1.A u_2, [7] u_2.A u_2.
template <int SCHEME>
__global__ void __launch_bounds__(256) k_na_part(const __grid_constant__ DescChunk ch, CoefSrc cs,
                                                 const double2* __restrict__ u,
                                                 double* __restrict__ part) {
    __shared__ double red[8];
    const int b = find_real(ch.start, ch.count, blockIdx.x);
    const RDesc& d = ch.d[b];
    const int64_t base = (int64_t)(blockIdx.x - ch.start[b]) * NA_TILE;
    double acc[NA_NP];
#pragma unroll
    for (int k = 0; k < NA_NP; ++k) acc[k] = 0.0;
    for (int t = threadIdx.x; t < NA_TILE; t += blockDim.x) {
        const int64_t node = base + t;
        const int i = (int)(node >> d.log2n), j = (int)(node & (d.n - 1));
        const Cells4 a = cells_at(cs, d, i, j);
        const double2 f = rhs_at(a, d.h);
        const double2 q = stencil_apply<SCHEME, double2>(
            a, na_ld(u, d, i - 1, j - 1), na_ld(u, d, i - 1, j), na_ld(u, d, i - 1, j + 1),
            na_ld(u, d, i, j - 1), na_ld(u, d, i, j), na_ld(u, d, i, j + 1),
            na_ld(u, d, i + 1, j - 1), na_ld(u, d, i + 1, j), na_ld(u, d, i + 1, j + 1));
        const double2 uu = na_ld(u, d, i, j);
        acc[0] += a.z00;
        acc[1] = fma(f.x, uu.x, acc[1]);
        acc[2] = fma(f.x, uu.y, acc[2]);
        acc[3] = fma(f.y, uu.x, acc[3]);
        acc[4] = fma(f.y, uu.y, acc[4]);
        acc[5] = fma(uu.x, q.x, acc[5]);
        acc[6] = fma(uu.x, q.y, acc[6]);
        acc[7] = fma(uu.y, q.y, acc[7]);
    }
#pragma unroll
    for (int k = 0; k < NA_NP; ++k) {
        const double s = block_sum(acc[k], red);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * NA_NP + k] = s;
    }
}

// One warp per realization of the chunk: fixed-order sum of its partials,
// then the energy and flux forms (as rve_a_hom).
__global__ void k_na_final(const __grid_constant__ DescChunk ch, const double* __restrict__ part,
                           double* __restrict__ A, double* __restrict__ Af) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= ch.count) return;
    const RDesc& d = ch.d[b];
    const int t0 = ch.start[b], nt = ch.start[b + 1] - ch.start[b];
    double s[NA_NP];
#pragma unroll
    for (int k = 0; k < NA_NP; ++k) s[k] = warp_sum_array(part + (int64_t)t0 * NA_NP + k, nt, NA_NP);
    if ((threadIdx.x & 31) != 0) return;
    const double mean_a = s[0] / ((double)d.n * (double)d.n);
    const double iv = d.inv_vol;
    A[4 * b + 0] = mean_a - (2.0 * s[1] - s[5]) * iv;
    A[4 * b + 1] = -(s[2] + s[3] - s[6]) * iv;
    A[4 * b + 2] = -(s[3] + s[2] - s[6]) * iv;
    A[4 * b + 3] = mean_a - (2.0 * s[4] - s[7]) * iv;
    if (Af) {
        Af[4 * b + 0] = mean_a - s[1] * iv;
        Af[4 * b + 1] = -s[3] * iv;
        Af[4 * b + 2] = -s[2] * iv;
        Af[4 * b + 3] = mean_a - s[4] * iv;
    }
}

}  // namespace rve

using namespace rve;

extern "C" rve_status rve_a_hom_noalloc(const rve_realization* r, int32_t batch,
                                        const uint32_t* mask, const double* coef, int32_t scheme,
                                        const double* u, double* A, double* A_flux, void* stream) {
    rve_solve_opts o = {};
    o.scheme = scheme;
    Plan p;
    rve_status st = make_plan(r, batch, &o, p, false);   // host-side checks only
    if (st != RVE_OK) return st;
    if (!u || !A || (!mask && !coef)) return RVE_EINVAL;
    if (p.nodes > RVE_NOALLOC_MAX_NODES) return RVE_ESCRATCH;
    double* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return RVE_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CoefSrc cs{mask, coef};
    const double2* uu = reinterpret_cast<const double2*>(u);
    int64_t tile_off = 0;
    for (int b0 = 0; b0 < p.batch; b0 += CHUNK) {
        DescChunk ch;
        ch.count = std::min(CHUNK, p.batch - b0);
        ch.start[0] = 0;
        for (int k = 0; k < ch.count; ++k) {
            ch.d[k] = p.desc[b0 + k];
            ch.start[k + 1] = ch.start[k] + (int32_t)(((int64_t)ch.d[k].n * ch.d[k].n) / NA_TILE);
        }
        for (int k = ch.count + 1; k <= CHUNK; ++k) ch.start[k] = ch.start[ch.count];
        double* part = scratch + tile_off * NA_NP;
        const int tiles = ch.start[ch.count];
        if (scheme == RVE_Q1_LUMPED) k_na_part<1><<<tiles, 256, 0, s>>>(ch, cs, uu, part);
        else k_na_part<0><<<tiles, 256, 0, s>>>(ch, cs, uu, part);
        k_na_final<<<(ch.count + 7) / 8, 256, 0, s>>>(ch, part, A + 4 * (int64_t)b0,
                                                      A_flux ? A_flux + 4 * (int64_t)b0 : nullptr);
        if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
        note_launch(2);
        tile_off += tiles;
    }
    return RVE_OK;
}
