"""Ensemble studies on the GPU path.

* ``variance``: the random error of the RVE method versus L (Sec. 4.2,
  Eq. "var"): for each L the empirical mean, variances and quartic tensor of
  A_hom over N seeded realizations; L^2 var(a_12) should be roughly constant.
* ``fem``: the FEM approximation test of Sec. 3.5 (Table 1): one fixed
  inclusion configuration (L^2 squares of side 2 alpha = 1, values lambda =
  0.1 outside and 1 inside, corners on the coarsest grid) solved with the
  load f = sin(2 pi x/L) cos(6 pi y/L) on dyadic refinements n = 64 .. 1024;
  reported are |u_p - u_{p-1}|_2 / |u_{p-1}|_2 on the coarser grid's nodes
  and their decay factors (the paper expects about 2 sqrt(2));
* ``dos``: the spectral-density appendix: Gaussian-broadened densities of
  states of the stiffness matrix for N realizations at L = 4 and 8 (lambda =
  0.5, alpha = 1/4, m0 = 8, the paper's lumped operator), their sample
  averages, the spread around them, the distance between the two L (the
  paper observes practically identical shapes) and the distance to the DOS
  of the operator with the homogenized coefficient;
* ``paper``: the statistics of Sec. 5 with the paper's own model parameters
  (overlap alpha = 1/4, i.e. inclusions of side 1/2; L^2 inclusions; matrix
  value 0.4 and inclusion value 1; m0 = 4; the lumped (trapezoid) scheme;
  tolerance 1e-8): the standard deviations of a_12 and a_11 - a_22 (Eqs.
  "Var1", "Var2", Table 6) and the systematic error <a_11>_L - <a_11>_2L
  (Table 5).

    python -m paper_1903_12227_gb300.studies variance --Ls 32 64 128 256 --N 256
    python -m paper_1903_12227_gb300.studies paper --Ls 8 16 32 64 --N 10000
    python -m paper_1903_12227_gb300.studies fem --Ls 2 4 8
    python -m paper_1903_12227_gb300.studies dos --Ls 4 8 --N 20
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import rve, workloads


def solve_ensemble(descs: list, opts, batch: int, device=None):
    """A_hom [N,2,2] (host) and infos of the realizations, in batches on the GPU."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    out, infos = [], []
    ws = None
    for s in range(0, len(descs), batch):
        ds = descs[s:s + batch]
        b = rve.Batch(ds)
        nb = rve.workspace_size(b, opts)
        if ws is None or ws.numel() < nb:
            ws = rve.workspace(nb, dev)
        mask = rve.gen_field(b, device=dev)
        u, info = rve.solve(b, mask=mask, opts=opts, ws=ws)
        out.append(rve.a_hom(b, u, mask=mask, scheme=opts.scheme,
                             precision=opts.precision).cpu().numpy())
        infos.extend(rve.info_to_dicts(info, b.count))
    return np.concatenate(out), infos


def variance_study(Ls=(32, 64, 128, 256), N=256, contrast=100.0, m0=8, seed=0,
                   precision=rve.MIXED, tol=1e-10, batch_nodes=1 << 26) -> list:
    rows = []
    for L in Ls:
        descs = workloads.batch(L, m0, contrast, seed, N)
        n = L * m0
        t0 = time.perf_counter()
        A, infos = solve_ensemble(descs, rve.make_opts(precision=precision, tol=tol),
                                  batch=max(1, batch_nodes // (n * n)))
        dt = time.perf_counter() - t0
        st = rve.statistics(A, L)
        bad = sum(1 for i in infos if i["status"] != rve.RVE_OK)
        rows.append({"L": L, "n": n, "N": N, "seconds": dt, "failed": bad,
                     "mean": st["mean"].tolist(), "var": st["var"].tolist(),
                     "L2_var_a12": float(L * L * st["var"][0, 1]),
                     "L2_var_a11": float(L * L * st["var"][0, 0]),
                     "Q": st["Q"].tolist(), "std12_paper": st["std12_paper"],
                     "stddiff_paper": st["stddiff_paper"]})
    return rows


def paper_descs(L: int, N: int, seed: int = 0, count: str = "fixed") -> list:
    """The paper's statistics model: m0 = 4, inclusions of side 1/2 (alpha =
    1/4), values 0.4 (matrix) and 1 (inclusions); L^2 inclusions per
    realization (count="fixed"), or a Poisson number of mean L^2
    (count="poisson", one reading of Sec. 2's placement)."""
    ds = [workloads.realization(L, 4, 1.0 / 0.4, seed, k, density=1.0, side_units=0.5,
                                a_matrix=0.4) for k in range(N)]
    if count == "poisson":
        g = np.random.default_rng([seed, L, 11])
        for d, m in zip(ds, g.poisson(L * L, size=N)):
            d["n_incl"] = int(m)
    return ds


def paper_study(Ls=(8, 16, 32, 64), N=10000, seed=0, batch_nodes=1 << 26,
                count: str = "fixed") -> list:
    rows = []
    opts = rve.make_opts(scheme=rve.LUMPED, precision=rve.MIXED, tol=1e-8)
    for L in Ls:
        n = 4 * L
        t0 = time.perf_counter()
        A, infos = solve_ensemble(paper_descs(L, N, seed, count), opts,
                                  batch=max(1, batch_nodes // (n * n)))
        dt = time.perf_counter() - t0
        st = rve.statistics(A, L)
        Q = st["Q"]
        rows.append({"L": L, "N": N, "count": count, "seconds": dt,
                     "failed": sum(1 for i in infos if i["status"] != rve.RVE_OK),
                     "mean_a11": float(st["mean"][0, 0]), "mean_a22": float(st["mean"][1, 1]),
                     "mean_a12": float(st["mean"][0, 1]),
                     "std12_paper": st["std12_paper"], "stddiff_paper": st["stddiff_paper"],
                     "sem_a11": float(np.sqrt(st["var"][0, 0] / N)),
                     # Eq. "quartic" with the Kronecker-product unfolding of
                     # (A - mean)(x)(A - mean): q_11 = L^2 var a11 and
                     # q_14 = L^2 var a12 (entry (1,1),(2,2) of X (x) X is
                     # X_12 X_12); q_14 of the vec unfolding = L^2 cov(a11, a22)
                     "q11": float(Q[0, 0]), "q14_kron": float(Q[1, 1]),
                     "q14_vec": float(Q[0, 3]),
                     "Q": Q.tolist()})
    for a, b in zip(rows, rows[1:]):
        if b["L"] == 2 * a["L"]:
            # Table 5 / Fig. 7: <a11>_L - <a11>_2L, with its sampling error
            # (independent ensembles: the two standard errors in quadrature)
            a["systematic_a11_L_minus_2L"] = a["mean_a11"] - b["mean_a11"]
            a["systematic_sem"] = float(np.hypot(a["sem_a11"], b["sem_a11"]))
            # Fig. 9: q_L - q_2L
            a["q11_L_minus_2L"] = a["q11"] - b["q11"]
            a["q14_kron_L_minus_2L"] = a["q14_kron"] - b["q14_kron"]
    return rows


def fem_convergence(Ls=(2, 4, 8), ns=(64, 128, 256, 512, 1024), alpha=0.5, lam=0.1, seed=0,
                    scheme=rve.CONSISTENT, precision=rve.FP64, tol=1e-10) -> list:
    """Sec. 3.5: differences of solutions on dyadic refinements of one fixed
    coefficient configuration.  The configuration is drawn on the coarsest
    grid (L^2 corners, squares of side 2*alpha units) and refined by
    splitting every coarse cell, so that all grids see the same geometry.
    Loads: component 1 the paper's sin(2 pi x/L) cos(6 pi y/L), component 2
    the transposed cos(6 pi x/L) sin(2 pi y/L); load vectors through the
    scheme's mass matrix.  tol = 1e-10: the differences are ~1e-4 and, for
    this smooth load, FP64 CG cannot reach much below ~1e-12 at n = 1024
    (|A| |u| / |A u| ~ 1e4)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    rows = []
    n0 = min(ns)
    for L in Ls:
        m0c = n0 // L
        coarse = workloads.realization(L, m0c, 1.0 / lam, seed, 0, density=1.0,
                                       side_units=2 * alpha, a_matrix=lam)
        mask = rve.gen_field([coarse], device=dev)
        bits = torch.as_tensor(rve.unpack_mask(mask, [coarse])[0], device=dev)   # [n0, n0] bool
        sols = []
        for n in ns:
            fct = n // n0
            m0 = n // L
            d = workloads.realization(L, m0, 1.0 / lam, seed, 0, density=1.0,
                                      side_units=2 * alpha, a_matrix=lam)
            fine = bits.repeat_interleave(fct, 0).repeat_interleave(fct, 1)
            coef = torch.where(fine, torch.tensor(1.0, dtype=torch.float64, device=dev),
                               torch.tensor(lam, dtype=torch.float64, device=dev)).reshape(-1)
            x = torch.arange(n, dtype=torch.float64, device=dev) / m0
            g1 = torch.outer(torch.sin(2 * np.pi * x / L), torch.cos(6 * np.pi * x / L))
            g2 = torch.outer(torch.cos(6 * np.pi * x / L), torch.sin(2 * np.pi * x / L))
            g = torch.stack([g1.reshape(-1), g2.reshape(-1)], dim=1).contiguous()
            f = rve.apply_mass([d], g, scheme=scheme)
            t0 = time.perf_counter()
            u, info = rve.solve([d], coef=coef, opts=rve.make_opts(scheme=scheme, precision=precision,
                                                                   tol=tol), f=f)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            inf = rve.info_to_dicts(info, 1)[0]
            u = u.reshape(n, n, 2)
            u = u - u.mean(dim=(0, 1), keepdim=True)
            sols.append((n, u, inf, dt))
        row = {"L": L, "ns": list(ns), "iters": [s[2]["iters"] for s in sols],
               "status": [s[2]["status"] for s in sols], "seconds": [s[3] for s in sols],
               "rel_diff": [], "decay": []}
        for (na, ua, _, _), (nb, ub, _, _) in zip(sols, sols[1:]):
            step = nb // na
            ub_c = ub[::step, ::step]   # the fine solution at the coarse nodes
            diff = [float((ub_c[..., c] - ua[..., c]).norm() / ua[..., c].norm()) for c in range(2)]
            row["rel_diff"].append(diff)
        for a, b in zip(row["rel_diff"], row["rel_diff"][1:]):
            row["decay"].append([a[c] / b[c] for c in range(2)])
        rows.append(row)
    return rows


def dos_study(Ls=(4, 8), N=20, lam=0.5, alpha=0.25, m0=8, eta=0.05, K=512, vectors=32,
              seed=0, scheme=rve.LUMPED) -> dict:
    """DOS of A for N realizations per L (stochastic Chebyshev moments on the
    GPU, Gaussian broadening eta), on a common grid t in [0, hi]."""
    from . import spectral
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"Ls": list(Ls), "N": N, "eta": eta, "K": K, "vectors": vectors, "per_L": []}
    hi = None
    t = None
    means = []
    for L in Ls:
        ds = [workloads.realization(L, m0, 1.0 / lam, seed, k, density=1.0, side_units=2 * alpha,
                                    a_matrix=lam) for k in range(N)]
        lo, hi = spectral.spectral_bounds(ds[0], scheme)
        t = np.linspace(0.0, hi, 401)
        dt = t[1] - t[0]
        mask = rve.gen_field(ds, device=dev)
        words = (L * m0) ** 2 // 32
        phis = []
        for k, d in enumerate(ds):
            mk = mask[k * words:(k + 1) * words]
            phis.append(spectral.dos(d, mk, t, eta, K=K, vectors=vectors, seed=seed * 1000 + k,
                                     scheme=scheme))
        phis = np.array(phis)
        mean = phis.mean(axis=0)
        means.append(mean)
        # homogenized operator: constant A_hom (sample mean), lumped symbol
        u, _ = rve.solve(ds, mask=mask, opts=rve.make_opts(scheme=scheme, precision=rve.MIXED))
        A = rve.a_hom(ds, u, mask=mask, scheme=scheme, precision=rve.MIXED).cpu().numpy().mean(axis=0)
        n = L * m0
        th = 2 * np.pi * np.arange(n) / n
        kk = 2.0 - 2.0 * np.cos(th)
        if scheme == rve.CONSISTENT:
            mm = (4.0 + 2.0 * np.cos(th)) / 6.0
            ev = (A[0, 0] * np.outer(kk, mm) + A[1, 1] * np.outer(mm, kk)).ravel()
        else:
            ev = (A[0, 0] * kk[:, None] + A[1, 1] * kk[None, :]).ravel()
        g = spectral.gauss(t[:, None] - ev[None, :], eta).sum(axis=1) / ev.size
        running = [float(np.abs(phis[:j].mean(axis=0) - mean).sum() * dt) for j in range(1, N + 1)]
        out["per_L"].append({"L": L, "mean": mean.tolist(),
                             "spread_L1": [float(np.abs(p - mean).sum() * dt) for p in phis],
                             "running_mean_L1": running, "A_hom": A.tolist(),
                             "homogenized_L1": float(np.abs(g - mean).sum() * dt)})
    out["t"] = t.tolist()
    if len(means) >= 2:
        dt = t[1] - t[0]
        out["L_pair_L1"] = float(np.abs(means[0] - means[-1]).sum() * dt)
    return out


# Algorithmic bytes per node of one launch of each 3D kernel kind: the
# stencil reads x (a pair, 16 B) and the cell byte and writes y (16 B); a
# line pass reads and writes a pair (the last one also reads r: 48 B, so
# 36 B on average over the four passes); the z solve reads and writes a
# pair; the CG vector steps of one iteration move 144 B (u, r, p, q read and
# u, r written; z, p read and p written) over two launches; the scalar
# launches move nothing; the FP64 true residual reads u, f and the cells and
# writes r (49 B).  FP32 vectors (the mixed path's cycles) halve the vector
# bytes.
CUBE_BYTES = {"stiffness": 33.0, "lines": 36.0, "zsolve": 32.0, "vector": 72.0, "scalar": 0.0,
              "resid64": 49.0}
CUBE_BYTES_FP32 = {"stiffness": 17.0, "lines": 18.0, "zsolve": 16.0, "vector": 36.0,
                   "scalar": 0.0, "resid64": 49.0}


def _measured_hbm():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def cubes_study(Ls=(2, 4, 8, 16), m0=16, N=None, contrast=10.0, seed=0, tol=1e-10,
                scheme=rve.CONSISTENT, precisions=(rve.FP64, rve.MIXED)) -> list:
    """3D extension: N realizations of round(0.7 L^3) unit cubes on
    [0,L)^3 (n = L m0 nodes per axis) per L: time per realization (field,
    three correctors, A_hom; CUDA events), iterations, per-kernel-kind
    launch times with their algorithmic bandwidth, and the mean and spread
    of the diagonal of the 3x3 A_hom.  N defaults to about 64 M nodes per
    batch (at least 2 realizations): all of a batch run in the same launches."""
    import torch
    from . import rve3
    peak = _measured_hbm()
    rows = []
    for L, prec in [(L, p) for L in Ls for p in precisions]:
        n = L * m0
        NL = N or max(2, (64 << 20) // n ** 3)
        descs = [workloads.realization3(L, m0, contrast, seed, k) for k in range(NL)]
        nodes = n ** 3
        rve3.homogenize(descs[:1], scheme=scheme, tol=tol, precision=prec)   # warm-up
        torch.cuda.synchronize()
        rve.profile_enable(True)
        rve3.profile_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        A, infos = rve3.homogenize(descs, scheme=scheme, tol=tol, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        rve.profile_enable(False)
        prof = rve3.profile_read()
        ms = e0.elapsed_time(e1)
        # a launch covers every unit (pair of a realization) of the batch, but
        # the blocks of units that have converged return at once: scale the
        # bytes by the fraction of unit-steps that did work (CG steps of the
        # units over stiffness launches x units)
        units = 2 * NL
        unit_steps = sum(max(i["iters"][0], i["iters"][1]) + i["iters"][2] for i in infos)
        stiff_launches = max(prof["stiffness"][1], 1)
        active = min(1.0, unit_steps / (stiff_launches * units))
        kinds = {}
        for kind, (t, cnt) in prof.items():
            # mixed: nearly every launch is an FP32 one (a few FP64 refinements)
            per = (CUBE_BYTES if prec == rve.FP64 else CUBE_BYTES_FP32)[kind]
            nodes_launch = units * nodes * active
            gbs = per * nodes_launch * cnt / (t * 1e-3) / 1e9 if t > 0 and per else None
            kinds[kind] = {"ms": round(t, 3), "launches": cnt,
                           "us_per_launch": round(1e3 * t / cnt, 2) if cnt else None,
                           "GBs": round(gbs, 1) if gbs else None,
                           "frac_of_measured": round(gbs / peak, 3) if gbs and peak else None}
        Ad = A.diagonal(dim1=1, dim2=2).cpu().numpy()
        st = rve3.statistics(A, L) if NL >= 2 else None
        rows.append({"L": L, "m0": m0, "n": n, "N": NL, "contrast": contrast, "tol": tol,
                     "precision": "fp64" if prec == rve.FP64 else "mixed",
                     "refinements_mean": float(np.mean([i["refinements"] for i in infos])),
                     "ms_per_realization": round(ms / NL, 3),
                     "realizations_per_s": round(1e3 * NL / ms, 3),
                     "iters_mean": float(np.mean([np.mean(i["iters"]) for i in infos])),
                     "max_relres": float(max(max(i["relres"]) for i in infos)),
                     "status": sorted({i["status"] for i in infos}),
                     "A_diag_mean": float(Ad.mean()), "A_diag_std": float(Ad.std()),
                     "offdiag_max": float(np.abs(A.cpu().numpy() - np.einsum(
                         "bi,ij->bij", Ad, np.eye(3))).max()),
                     "active_unit_fraction": round(active, 3),
                     "L3_var_diag": [float(st["Q"][4 * k, 4 * k]) for k in range(3)] if st else None,
                     "kernels": kinds, "hbm_peak_GBs": peak})
    return rows


# FP64 instructions per node pair of the two study kernels, counted from
# their formulas: the mass stencil 9 FMA per component (consistent) plus the
# h^2 scaling; the Chebyshev step the 9-point stiffness (cell sums and 9
# multiply-adds per component), the three-term update and four partial-sum
# products.
MASS_FP64_PER_NODE = 20
CHEB_FP64_PER_NODE = 40


def kernel_rates(L=32, m0=16, batch=64, K=64, reps=10) -> list:
    """Measured rates of the study kernels of the FEM convergence test
    (rve_apply_mass) and the density of states (rve_cheb_moments, one
    stiffness application per two moments) on `batch` realizations of
    (L m0)^2 nodes: algorithmic bytes against the measured HBM peak and
    FP64 instructions against GB300's FP64 issue rate (152 SMs x 2 per clock
    x the clock)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    ds = workloads.batch(L, m0, 10.0, 0, batch)
    b = rve.Batch(ds)
    nodes = b.nodes
    peak = _hbm_peak()
    mhz = 2070.0
    fp64_peak = 152 * 2 * mhz * 1e6
    x = torch.randn(nodes, 2, dtype=torch.float64, device=dev)
    mask = rve.gen_field(b, device=dev)
    rows = []

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    t = timed(lambda: rve.apply_mass(b, x))
    rows.append({"kernel": "k_mass (rve_apply_mass, consistent)", "nodes": nodes,
                 "us_per_launch": t * 1e6, "bytes_per_node": 32,
                 "GBs": 32 * nodes / t / 1e9, "frac_hbm": 32 * nodes / t / 1e9 / peak,
                 "fp64_inst_per_node": MASS_FP64_PER_NODE,
                 "frac_fp64_issue": MASS_FP64_PER_NODE * nodes / t / fp64_peak})
    lo, hi = 0.0, 16.0 / 3.0 * 10.0
    steps = (K + 1) // 2
    t = timed(lambda: rve.cheb_moments(b, x, K, lo, hi, mask=mask)) / steps
    rows.append({"kernel": "k_cheb (rve_cheb_moments, per stiffness application)", "nodes": nodes,
                 "us_per_launch": t * 1e6, "bytes_per_node": 48.125,
                 "GBs": 48.125 * nodes / t / 1e9, "frac_hbm": 48.125 * nodes / t / 1e9 / peak,
                 "fp64_inst_per_node": CHEB_FP64_PER_NODE,
                 "frac_fp64_issue": CHEB_FP64_PER_NODE * nodes / t / fp64_peak})
    rows.append(refine_rate(L, m0))
    return rows


def refine_rate(L=32, m0=16, copies=32) -> dict:
    """The double-word true-residual pass (k_fused_R) of the mixed solver on
    `copies` copies of one realization, so that every refining launch works
    on all of them at once: its CUDA-event time per launch over one solve
    (idle launches of the iteration steps included) from the library's
    per-kernel profiler."""
    dev = torch.device("cuda", torch.cuda.current_device())
    ds = [workloads.realization(L, m0, 10.0, 0, 5)] * copies
    opts = rve.make_opts(precision=rve.MIXED, tol=1e-10)
    mask = rve.gen_field(ds, device=dev)
    ws = rve.workspace(rve.workspace_size(ds, opts), dev)
    rve.solve(ds, mask=mask, opts=opts, ws=ws)   # warm-up
    torch.cuda.synchronize()
    rve.profile_enable(True)
    rve.profile_read()
    u, info = rve.solve(ds, mask=mask, opts=opts, ws=ws)
    torch.cuda.synchronize()
    prof = rve.profile_read()["refine"]
    rve.profile_enable(False)
    d = rve.info_to_dicts(info, copies)[0]
    return {"kernel": "k_fused_R (double-word true residual, mixed solver)",
            "nodes": (L * m0) ** 2 * copies, "launches": prof["launches"],
            "refining_launches": d["refinements"], "steps": d["steps"],
            "ms_total": prof["ms"], "us_per_launch": 1e3 * prof["ms"] / max(prof["launches"], 1)}


def _hbm_peak() -> float:
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        return float(json.load(open(os.path.join(here, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["variance", "paper", "fem", "dos", "cubes", "kernels"])
    ap.add_argument("--Ls", type=int, nargs="+")
    ap.add_argument("--N", type=int)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--count", choices=["fixed", "poisson"], default="fixed")
    ap.add_argument("--json")
    ap.add_argument("--prec", choices=["both", "fp64", "mixed"], default="both",
                    help="cubes: which solver precision(s) to measure")
    a = ap.parse_args(argv)
    if a.study == "kernels":
        rows = kernel_rates()
    elif a.study == "cubes":
        precs = {"both": (rve.FP64, rve.MIXED), "fp64": (rve.FP64,), "mixed": (rve.MIXED,)}[a.prec]
        rows = cubes_study(Ls=tuple(a.Ls or (2, 4, 8, 16)), N=a.N, seed=a.seed, precisions=precs)
    elif a.study == "dos":
        rows = dos_study(Ls=tuple(a.Ls or (4, 8)), N=a.N or 20, seed=a.seed)
    elif a.study == "fem":
        rows = fem_convergence(Ls=tuple(a.Ls or (2, 4, 8)), seed=a.seed)
    elif a.study == "variance":
        rows = variance_study(Ls=tuple(a.Ls or (32, 64, 128, 256)), N=a.N or 256, seed=a.seed)
    else:
        rows = paper_study(Ls=tuple(a.Ls or (8, 16, 32, 64)), N=a.N or 10000, seed=a.seed,
                           count=a.count)
    txt = json.dumps({"study": a.study, "rows": rows})
    if a.json:
        with open(a.json, "w") as f:
            f.write(txt + "\n")
    print(txt)


if __name__ == "__main__":
    main()
