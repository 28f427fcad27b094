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
// device current; make that first call before any stream capture.  The
// address is not looked up again: a device reset (cudaDeviceReset, or any
// teardown of the primary context) leaves it stale, and the entry point must
// not be called on that device afterwards.  All calls
// share the array and it keeps the last call's contents: every partial it
// reads is written earlier in the same call, so nothing needs clearing, but
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "rve_ahom.cuh"
#include "rve_common.cuh"
#include "rve_internal.h"

namespace rve {

constexpr int NA_TILE = 1024;                       // nodes per partial-sum tile
constexpr int NA_NP = 8;                            // partial sums per tile
constexpr int64_t NA_MAX_TILES = RVE_NOALLOC_MAX_NODES / NA_TILE;
static_assert(NA_TILE == AHOM_TILE && NA_NP == AHOM_NP, "tiles of rve_ahom.cuh");
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

// Partial sums of one tile and the final forms: the same cell-form
// arithmetic as the workspace entry point (rve_ahom.cuh).
template <int SCHEME>
__global__ void __launch_bounds__(256) k_na_part(const __grid_constant__ DescChunk ch, CoefSrc cs,
                                                 const double2* __restrict__ u,
                                                 double* __restrict__ part) {
    __shared__ double red[64];
    __shared__ float sc[5];
    const int b = find_real(ch.start, ch.count, blockIdx.x);
    a_hom_tile<SCHEME>(ch.d[b], blockIdx.x - ch.start[b], cs, u, red, sc,
                       part + (int64_t)blockIdx.x * NA_NP);
}

// One warp per realization of the chunk.
template <int SCHEME>
__global__ void k_na_final(const __grid_constant__ DescChunk ch, const double* __restrict__ part,
                           double* __restrict__ A, double* __restrict__ Af) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= ch.count) return;
    a_hom_finish<SCHEME>(ch.d[b], part + (int64_t)ch.start[b] * NA_NP, ch.start[b + 1] - ch.start[b],
                         A + 4 * (int64_t)b, Af ? Af + 4 * (int64_t)b : nullptr);
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
        if (scheme == RVE_Q1_LUMPED)
            k_na_final<1><<<(ch.count + 7) / 8, 256, 0, s>>>(ch, part, A + 4 * (int64_t)b0,
                                                      A_flux ? A_flux + 4 * (int64_t)b0 : nullptr);
        else
            k_na_final<0><<<(ch.count + 7) / 8, 256, 0, s>>>(ch, part, A + 4 * (int64_t)b0,
                                                      A_flux ? A_flux + 4 * (int64_t)b0 : nullptr);
        if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
        note_launch(2);
        tile_off += tiles;
    }
    return RVE_OK;
}
