// rve_plain.cu -- the plain FP64 path: textbook preconditioned CG (Saad,
// Iterative Methods for Sparse Linear Systems, Algorithm 9.1) for one
// realization at a time, one kernel per operation (stencil, dot, axpy,
// preconditioner passes, scalar update).  It is the reference point for
// the fused and mixed-precision paths; every kernel is a straightforward
// GPU implementation of its step, with the same stencil and transforms.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "rve_common.cuh"
#include "rve_internal.h"

namespace rve {


__device__ __forceinline__ double2 ld2(const double2* x, const RDesc& d, int i, int j) {
    return x[d.node_off + ((int64_t)(i & (d.n - 1)) << d.log2n) + (j & (d.n - 1))];
}

__device__ __forceinline__ void store_part(double* part, double a, double b, double* red) {
    const double sa = block_sum(a, red);
    const double sb = block_sum(b, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sa;
        part[2 * blockIdx.x + 1] = sb;
    }
}

// r = f, u = 0, partial |f|^2
__global__ void k_pl_init(const RDesc* desc, int b, CoefSrc cs, double2* u, double2* r,
                          double* part) {
    __shared__ double red[8];
    const RDesc d = desc[b];
    DotAcc<double> ax, ay;
    for (int t = threadIdx.x; t < PL_NODES; t += blockDim.x) {
        const int64_t node = (int64_t)blockIdx.x * PL_NODES + t;
        const int i = (int)(node >> d.log2n), j = (int)(node & (d.n - 1));
        const double2 f = load_at(cs, d, node, cells_at(cs, d, i, j));
        r[d.node_off + node] = f;
        u[d.node_off + node] = make_double2(0.0, 0.0);
        ax.add(f.x, f.x);
        ay.add(f.y, f.y);
    }
    store_part(part, ax.value(), ay.value(), red);
}

template <int SCHEME>
__global__ void k_pl_stencil(const RDesc* desc, int b, CoefSrc cs, const double2* __restrict__ p,
                             double2* __restrict__ q) {
    const RDesc d = desc[b];
    for (int t = threadIdx.x; t < PL_NODES; t += blockDim.x) {
        const int64_t node = (int64_t)blockIdx.x * PL_NODES + t;
        const int i = (int)(node >> d.log2n), j = (int)(node & (d.n - 1));
        const Cells4 a = cells_at(cs, d, i, j);
        q[d.node_off + node] = stencil_apply<SCHEME, double2>(
            a, ld2(p, d, i - 1, j - 1), ld2(p, d, i - 1, j),
            ld2(p, d, i - 1, j + 1), ld2(p, d, i, j - 1),
            ld2(p, d, i, j), ld2(p, d, i, j + 1),
            ld2(p, d, i + 1, j - 1), ld2(p, d, i + 1, j),
            ld2(p, d, i + 1, j + 1));
    }
}

__global__ void k_pl_dot(const RDesc* desc, int b, const double2* __restrict__ x,
                         const double2* __restrict__ y, double* part) {
    __shared__ double red[8];
    const RDesc d = desc[b];
    DotAcc<double> ax, ay;
    for (int t = threadIdx.x; t < PL_NODES; t += blockDim.x) {
        const int64_t node = d.node_off + (int64_t)blockIdx.x * PL_NODES + t;
        const double2 a = x[node], c = y[node];
        ax.add(a.x, c.x);
        ay.add(a.y, c.y);
    }
    store_part(part, ax.value(), ay.value(), red);
}

// u += alpha p; r -= alpha q; partial |r|^2
__global__ void k_pl_axpy(const RDesc* desc, int b, const PlainScal* sc, double2* __restrict__ u,
                          double2* __restrict__ r, const double2* __restrict__ p,
                          const double2* __restrict__ q, double* part) {
    __shared__ double red[8];
    const RDesc d = desc[b];
    const double ax_ = sc->alpha[0], ay_ = sc->alpha[1];
    DotAcc<double> ax, ay;
    for (int t = threadIdx.x; t < PL_NODES; t += blockDim.x) {
        const int64_t node = d.node_off + (int64_t)blockIdx.x * PL_NODES + t;
        const double2 pp = p[node], qq = q[node];
        double2 uu = u[node], rr = r[node];
        uu.x = fma(ax_, pp.x, uu.x);
        uu.y = fma(ay_, pp.y, uu.y);
        rr.x = fma(-ax_, qq.x, rr.x);
        rr.y = fma(-ay_, qq.y, rr.y);
        u[node] = uu;
        r[node] = rr;
        ax.add(rr.x, rr.x);
        ay.add(rr.y, rr.y);
    }
    store_part(part, ax.value(), ay.value(), red);
}

// p = z + beta p
__global__ void k_pl_xpby(const RDesc* desc, int b, const PlainScal* sc,
                          const double2* __restrict__ z, double2* __restrict__ p) {
    const RDesc d = desc[b];
    const double bx = sc->beta[0], by = sc->beta[1];
    for (int t = threadIdx.x; t < PL_NODES; t += blockDim.x) {
        const int64_t node = d.node_off + (int64_t)blockIdx.x * PL_NODES + t;
        const double2 zz = z[node], pp = p[node];
        p[node] = make_double2(fma(bx, pp.x, zz.x), fma(by, pp.y, zz.y));
    }
}

// r_true = f - A u, partial |r_true|^2
template <int SCHEME>
__global__ void k_pl_resid(const RDesc* desc, int b, CoefSrc cs, const double2* __restrict__ u,
                           double* part) {
    __shared__ double red[8];
    const RDesc d = desc[b];
    DotAcc<double> ax, ay;
    for (int t = threadIdx.x; t < PL_NODES; t += blockDim.x) {
        const int64_t node = (int64_t)blockIdx.x * PL_NODES + t;
        const int i = (int)(node >> d.log2n), j = (int)(node & (d.n - 1));
        const Cells4 a = cells_at(cs, d, i, j);
        const double2 f = load_at(cs, d, node, a);
        const double2 Au = stencil_apply<SCHEME, double2>(
            a, ld2(u, d, i - 1, j - 1), ld2(u, d, i - 1, j),
            ld2(u, d, i - 1, j + 1), ld2(u, d, i, j - 1),
            ld2(u, d, i, j), ld2(u, d, i, j + 1),
            ld2(u, d, i + 1, j - 1), ld2(u, d, i + 1, j),
            ld2(u, d, i + 1, j + 1));
        const double rx = f.x - Au.x, ry = f.y - Au.y;
        ax.add(rx, rx);
        ay.add(ry, ry);
    }
    store_part(part, ax.value(), ay.value(), red);
}

// Scalar steps of Algorithm 9.1 (one warp): reduce `nb` partials in a fixed
// order and apply `what` (SC_* in rve_internal.h).

__global__ void k_pl_scalar(PlainScal* sc, const double* part, int nb, int what, double tol,
                            int max_iter) {
    const double sx = warp_sum_array(part, nb, 2);
    const double sy = warp_sum_array(part + 1, nb, 2);
    if (threadIdx.x != 0) return;
    const double v[2] = {sx, sy};
    switch (what) {
        case SC_FNORM:
            for (int k = 0; k < 2; ++k) {
                sc->fnorm[k] = sqrt(v[k]);
                sc->active[k] = v[k] > 0.0;
                sc->iters[k] = 0;
                sc->alpha[k] = sc->beta[k] = 0.0;
            }
            sc->done = !(sc->active[0] || sc->active[1]);
            sc->status = RVE_OK;
            break;
        case SC_RHO0:
            for (int k = 0; k < 2; ++k) sc->rho[k] = v[k];
            break;
        case SC_ALPHA:
            for (int k = 0; k < 2; ++k) {
                sc->alpha[k] = sc->active[k] ? sc->rho[k] / v[k] : 0.0;
                if (sc->active[k]) sc->iters[k] += 1;
            }
            break;
        case SC_CONV:
            for (int k = 0; k < 2; ++k) {
                if (!sc->active[k]) continue;
                const double rn = sqrt(v[k]);
                if (!isfinite(rn)) { sc->status = RVE_ENAN; sc->active[0] = sc->active[1] = 0; }
                else if (rn <= tol * sc->fnorm[k]) sc->active[k] = 0;
                else if (sc->iters[k] >= max_iter) { sc->status = RVE_ENOCONV; sc->active[k] = 0; }
            }
            sc->done = !(sc->active[0] || sc->active[1]);
            break;
        case SC_BETA:
            for (int k = 0; k < 2; ++k) {
                sc->beta[k] = sc->active[k] ? v[k] / sc->rho[k] : 0.0;
                sc->rho[k] = v[k];
            }
            break;
        case SC_RELRES:
            for (int k = 0; k < 2; ++k) sc->relres[k] = sc->fnorm[k] > 0.0 ? sqrt(v[k]) / sc->fnorm[k] : 0.0;
            break;
    }
}

__global__ void k_pl_report(const PlainScal* sc, rve_solve_info* info, int b) {
    rve_solve_info r;
    r.iters[0] = sc->iters[0];
    r.iters[1] = sc->iters[1];
    r.status = sc->status;
    r.refinements = 1;
    r.steps = max(sc->iters[0], sc->iters[1]);
    r.reserved = 0;
    r.relres[0] = sc->relres[0];
    r.relres[1] = sc->relres[1];
    info[b] = r;
}

template <int SCHEME>
static rve_status plain_one(const Plan& p, char* w, int b, CoefSrc cs, double2* u,
                            const rve_solve_opts& o, rve_solve_info* info, cudaStream_t s) {
    const RDesc& d = p.desc[b];
    const RDesc* desc = reinterpret_cast<const RDesc*>(w + p.o_desc);
    double2* r = reinterpret_cast<double2*>(w + p.o_R);
    double2* z = reinterpret_cast<double2*>(w + p.o_X);
    double2* pp = reinterpret_cast<double2*>(w + p.o_P0);
    double2* q = reinterpret_cast<double2*>(w + p.o_Q);
    double2* t = reinterpret_cast<double2*>(w + p.o_T);
    double* part = reinterpret_cast<double*>(w + p.o_partS);
    PlainScal* sc = reinterpret_cast<PlainScal*>(w + p.o_state);
    const int nb = (int)(((int64_t)d.n * d.n) / PL_NODES);
    auto precond = [&](const double2* in, double2* out) {
        precond_passes<double2>(p, w, o.delta, in, out, t, b, 1, s);
    };
    k_pl_init<<<nb, PL_THREADS, 0, s>>>(desc, b, cs, u, r, part);
    k_pl_scalar<<<1, 32, 0, s>>>(sc, part, nb, SC_FNORM, o.tol, o.max_iter);
    precond(r, z);
    k_pl_dot<<<nb, PL_THREADS, 0, s>>>(desc, b, r, z, part);
    k_pl_scalar<<<1, 32, 0, s>>>(sc, part, nb, SC_RHO0, o.tol, o.max_iter);
    cudaMemsetAsync(pp + d.node_off, 0, sizeof(double2) * (size_t)d.n * d.n, s);
    k_pl_xpby<<<nb, PL_THREADS, 0, s>>>(desc, b, sc, z, pp);   // beta = 0: p = z
    const int every = o.check_every > 0 ? o.check_every : 8;
    PlainScal hsc;
    for (int it = 0; it < o.max_iter; ++it) {
        k_pl_stencil<SCHEME><<<nb, PL_THREADS, 0, s>>>(desc, b, cs, pp, q);
        k_pl_dot<<<nb, PL_THREADS, 0, s>>>(desc, b, pp, q, part);
        k_pl_scalar<<<1, 32, 0, s>>>(sc, part, nb, SC_ALPHA, o.tol, o.max_iter);
        k_pl_axpy<<<nb, PL_THREADS, 0, s>>>(desc, b, sc, u, r, pp, q, part);
        k_pl_scalar<<<1, 32, 0, s>>>(sc, part, nb, SC_CONV, o.tol, o.max_iter);
        precond(r, z);
        k_pl_dot<<<nb, PL_THREADS, 0, s>>>(desc, b, r, z, part);
        k_pl_scalar<<<1, 32, 0, s>>>(sc, part, nb, SC_BETA, o.tol, o.max_iter);
        k_pl_xpby<<<nb, PL_THREADS, 0, s>>>(desc, b, sc, z, pp);
        note_launch(10);
        if ((it + 1) % every == 0 || it == 0) {
            if (cudaMemcpyAsync(&hsc, sc, sizeof(PlainScal), cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return RVE_ECUDA;
            if (hsc.done) break;
        }
    }
    k_pl_resid<SCHEME><<<nb, PL_THREADS, 0, s>>>(desc, b, cs, u, part);
    k_pl_scalar<<<1, 32, 0, s>>>(sc, part, nb, SC_RELRES, o.tol, o.max_iter);
    k_pl_report<<<1, 1, 0, s>>>(sc, info, b);
    note_launch(14);   // set-up, final residual and report
    return cudaGetLastError() == cudaSuccess ? RVE_OK : RVE_ECUDA;
}

rve_status run_solve_plain(const Plan& p, void* ws, const uint32_t* mask, const double* coef,
                           const rve_solve_opts& o, double* u, rve_solve_info* info,
                           cudaStream_t s, const double* f) {
    rve_status st = upload_plan(p, ws, s);
    if (st != RVE_OK) return st;
    char* w = static_cast<char*>(ws);
    CoefSrc cs{mask, coef, reinterpret_cast<const double2*>(f)};
    double2* uu = reinterpret_cast<double2*>(u);
    for (int b = 0; b < p.batch; ++b) {
        st = (p.scheme == RVE_Q1_LUMPED) ? plain_one<1>(p, w, b, cs, uu, o, info, s)
                                         : plain_one<0>(p, w, b, cs, uu, o, info, s);
        if (st != RVE_OK) return st;
    }
    return RVE_OK;
}

}  // namespace rve
