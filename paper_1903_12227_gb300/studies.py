"""Ensemble studies on the GPU path.

* ``variance``: the random error of the RVE method versus L (Sec. 4.2,
  Eq. "var"): for each L the empirical mean, variances and quartic tensor of
  A_hom over N seeded realizations; L^2 var(a_12) should be roughly constant.
* ``paper``: the statistics of Sec. 5 with the paper's own model parameters
  (overlap alpha = 1/4, i.e. inclusions of side 1/2; L^2 inclusions; matrix
  value 0.4 and inclusion value 1; m0 = 4; the lumped (trapezoid) scheme;
  tolerance 1e-8): the standard deviations of a_12 and a_11 - a_22 (Eqs.
  "Var1", "Var2", Table 6) and the systematic error <a_11>_L - <a_11>_2L
  (Table 5).

    python -m paper_1903_12227_gb300.studies variance --Ls 32 64 128 256 --N 256
    python -m paper_1903_12227_gb300.studies paper --Ls 8 16 32 64 --N 10000
"""
from __future__ import annotations

import argparse
import json
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
        out.append(rve.a_hom(b, u, mask=mask, scheme=opts.scheme).cpu().numpy())
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
        rows.append({"L": L, "N": N, "count": count, "seconds": dt,
                     "failed": sum(1 for i in infos if i["status"] != rve.RVE_OK),
                     "mean_a11": float(st["mean"][0, 0]), "mean_a22": float(st["mean"][1, 1]),
                     "mean_a12": float(st["mean"][0, 1]),
                     "std12_paper": st["std12_paper"], "stddiff_paper": st["stddiff_paper"],
                     "sem_a11": float(np.sqrt(st["var"][0, 0] / N)),
                     "Q": st["Q"].tolist()})
    for a, b in zip(rows, rows[1:]):
        if b["L"] == 2 * a["L"]:
            a["systematic_a11_L_minus_2L"] = a["mean_a11"] - b["mean_a11"]
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["variance", "paper"])
    ap.add_argument("--Ls", type=int, nargs="+")
    ap.add_argument("--N", type=int)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--count", choices=["fixed", "poisson"], default="fixed")
    ap.add_argument("--json")
    a = ap.parse_args(argv)
    if a.study == "variance":
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
