"""GPU checks at the full sizes of the other workloads, on sampled outputs the
oracle computes one by one or through properties that hold at any size.

* uneven batch: 4096 realizations, L in {8,16,32,64}, h = 1/8, contrast in
  {10, 100}, mixed precision, one persistent launch captured in a CUDA graph
  after autotuning; sampled realizations against the oracle;
* adjoint: L = 64, h = 1/16 (1024^2 nodes), contrast 100, batch 64, FP64;
  Euler homogeneity for every realization, the oracle's gradient formula on
  the GPU correctors, and central differences (step 1e-6) on sampled cells;
* large: L = 256, h = 1/8 (2048^2 nodes), contrast 100, mixed precision
  against FP64 on 8 of the 256 realizations.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_12227_gb300 import rve, workloads

pytestmark = pytest.mark.gpu
CUDA = torch.device("cuda", 0)


def _rel_err_A(A, ref):
    return np.abs(np.asarray(A) - ref).max() / max(abs(ref[0, 0]), abs(ref[1, 1]))


def test_uneven_4096_plan_full_batch():
    ds = workloads.config_batch("uneven_4096", seed=0)
    assert len(ds) == 4096
    opts = rve.make_opts(precision=rve.MIXED, path=rve.PATH_PERSISTENT, tol=1e-10)
    rve.tuner_clear()
    rve.autotune(ds[:256], opts, device=CUDA)
    plan = rve.Plan(ds, opts, device=CUDA)
    A, info = plan.execute()
    torch.cuda.synchronize()
    A = A.cpu().numpy()
    inf = rve.info_to_dicts(info, len(ds))
    assert all(d["status"] == rve.RVE_OK for d in inf)
    assert max(max(d["relres"]) for d in inf) <= 1e-10 * 1.0001
    # energy form exactly symmetric; Voigt-Reuss bounds for every realization
    assert np.array_equal(A[:, 0, 1], A[:, 1, 0])
    ev = np.linalg.eigvalsh(A)
    lam = np.array([d["a_incl"] for d in ds])
    assert (ev[:, 0] > 1.0).all() and (ev[:, 1] < lam).all()
    # sampled realizations against the oracle (every size, both contrasts)
    picks = {}
    for k, d in enumerate(ds):
        picks.setdefault((d["L"], d["a_incl"]), k)
    for (L, lam_), k in sorted(picks.items()):
        if L == 64 and lam_ == 100.0:
            continue      # the 512^2 / contrast-100 oracle solve is the slowest; one 512^2 case suffices
        ref = oracle.solve_realization(ds[k], tol=1e-12, want_u=False)
        assert _rel_err_A(A[k], ref["A_energy"]) < 1e-7, (ds[k], A[k], ref["A_energy"])
    plan.close()
    rve.tuner_clear()


def _oracle_grad_roundoff(u, G, h, vol, scheme):
    """Per-cell bound on the rounding of the oracle's plain quadratic forms
    sum_ij G_ij v_i^T E v_j / vol: 32 eps times the sum of the absolute values
    of their terms (v_i = x_i + phi_i on the cell's corners, order 00, 01,
    10, 11)."""
    E = np.abs(oracle.element_matrix(scheme, h))
    n = u.shape[1]
    idx = np.arange(n)
    nx = (idx + 1) % n
    v = []
    for i in range(2):
        ui = u[i]
        c = [ui, ui[:, nx], ui[nx, :], ui[nx][:, nx]]
        if i == 0:
            c = [c[0], c[1], c[2] + h, c[3] + h]
        else:
            c = [c[0], c[1] + h, c[2], c[3] + h]
        v.append(np.abs(np.stack(c, axis=-1)))
    S = np.zeros((n, n))
    for i in range(2):
        Ev = v[i] @ E
        for j in range(2):
            S += abs(G[i, j]) * np.einsum("abk,abk->ab", Ev, v[j])
    return 32 * np.finfo(float).eps * S / vol


def test_adjoint_L64_batch64_euler_oracle_gradient_and_central_differences():
    """Configuration: L = 64, h = 1/16 (1024^2 nodes), contrast 100, batch
    64, FP64, solve tolerance 1e-13.

    * Euler homogeneity sum_c a_c dF/da_c = F for all 64 realizations;
    * the oracle's exact-formula gradient, evaluated on the GPU correctors of
      two realizations, cell by cell within 1e-10 relative plus the rounding
      of the oracle's own plain quadratic forms;
    * central differences with an absolute step of 1e-6 on 32 random cells
      of each of four realizations.  The derivatives here are ~1e-6 (matrix
      cells) to ~1e-10 (inclusion cells), so A moves by 2e-12 .. 2e-16 out of
      ~25: below FP64's resolution of A.  The differences are therefore
      formed from the double-double A_hom (A + A_lo) of the FP64 reduction;
      the energy form is stationary, so the solve error (relative residual
      1e-13) enters only squared (below 1e-19 of A), and the quotient agrees
      with the adjoint to ~1e-7 relative.
    """
    ds = workloads.config_batch("adjoint_L64", seed=0)
    assert len(ds) == 64 and ds[0]["L"] * ds[0]["m0"] == 1024
    n = 1024
    nn = n * n
    h, L = 1.0 / ds[0]["m0"], float(ds[0]["L"])
    b = rve.Batch(ds)
    mask = rve.gen_field(b, device=CUDA)
    bits = rve.unpack_mask(mask, b)
    coef = torch.tensor(np.concatenate([np.where(m, d["a_incl"], d["a_matrix"]).ravel()
                                        for d, m in zip(ds, bits)]), device=CUDA,
                        requires_grad=True)
    opts = rve.make_opts(precision=rve.FP64, tol=1e-13)
    A = rve.AHom.apply(coef, b, opts)
    G = torch.tensor(np.random.default_rng(4).standard_normal((64, 2, 2)), device=CUDA)
    (A * G).sum().backward()
    g = coef.grad.detach()
    # Euler: sum_c a_c dF/da_c = F for F = sum_ij G_ij A_ij (A is 1-homogeneous)
    euler = (coef.detach() * g).view(64, nn).sum(1)
    F = (A.detach() * G).sum((1, 2))
    assert torch.allclose(euler, F, rtol=1e-10, atol=1e-12)
    Gn = G.cpu().numpy()
    # the oracle's gradient formula on the GPU correctors of two realizations
    for r in (0, 37):
        d = ds[r]
        cr = coef.detach()[r * nn:(r + 1) * nn].contiguous()
        u, info = rve.solve([d], coef=cr, opts=opts)
        assert rve.info_to_dicts(info, 1)[0]["status"] == rve.RVE_OK
        gr = rve.a_hom_backward([d], u, G[r:r + 1]).cpu().numpy().reshape(n, n)
        # the autograd path solved the same system with the same kernels
        assert np.array_equal(gr, g[r * nn:(r + 1) * nn].cpu().numpy().reshape(n, n))
        un = u.cpu().numpy().reshape(n, n, 2).transpose(2, 0, 1).copy()
        gref = oracle.a_hom_grad(un, Gn[r], h, L)
        bound = 1e-10 * np.abs(gref) + _oracle_grad_roundoff(un, Gn[r], h, L * L, 0)
        err = np.abs(gr - gref)
        assert (err <= bound).all(), (r, float(err.max()), float((err / np.abs(gref)).max()))
    # central differences, step 1e-6, from double-double A_hom
    eps = 1e-6
    for r in (0, 21, 37, 63):
        d = ds[r]
        base = coef.detach()[r * nn:(r + 1) * nn]
        cells = workloads.fd_cells(n, 32, seed=0, index=r)
        ks = [int(c1) * n + int(c2) for c1, c2 in cells]
        stack = base.repeat(2 * len(ks), 1)
        for q, k in enumerate(ks):
            stack[2 * q, k] += eps
            stack[2 * q + 1, k] -= eps
        stack = stack.view(-1)
        dd = [d] * (2 * len(ks))
        u, info = rve.solve(dd, coef=stack, opts=opts)
        assert all(x["status"] == rve.RVE_OK for x in rve.info_to_dicts(info, len(dd)))
        Ahi, Alo = rve.a_hom(dd, u, coef=stack, precision=rve.FP64, want_lo=True)
        Ahi, Alo = Ahi.cpu().numpy(), Alo.cpu().numpy()
        dA = ((Ahi[0::2] - Ahi[1::2]) + (Alo[0::2] - Alo[1::2])) / (2 * eps)
        fd = (dA * Gn[r]).sum(axis=(1, 2))
        gk = g[r * nn:(r + 1) * nn].cpu().numpy()[ks]
        scale = g[r * nn:(r + 1) * nn].abs().max().item()
        err = np.abs(fd - gk)
        assert (err <= 1e-6 * np.abs(gk) + 1e-9 * scale).all(), \
            (r, float(err.max()), float((err / np.abs(gk)).max()), scale)
        del u, stack


def test_large_L256_mixed_against_fp64_sample():
    ds = workloads.config_batch("large_L256", seed=0, count=8)
    mask = rve.gen_field(ds, device=CUDA)
    u32, i32 = rve.solve(ds, mask=mask, opts=rve.make_opts(precision=rve.MIXED, tol=1e-10))
    A32 = rve.a_hom(ds, u32, mask=mask, precision=rve.MIXED).cpu().numpy()
    del u32
    u64, i64 = rve.solve(ds, mask=mask, opts=rve.make_opts(precision=rve.FP64, tol=1e-10))
    A64 = rve.a_hom(ds, u64, mask=mask).cpu().numpy()
    for k in range(len(ds)):
        assert rve.info_to_dicts(i32, len(ds))[k]["status"] == rve.RVE_OK
        assert rve.info_to_dicts(i64, len(ds))[k]["status"] == rve.RVE_OK
        assert _rel_err_A(A32[k], A64[k]) < 1e-7
        ev = np.linalg.eigvalsh(A32[k])
        assert 1.0 < ev[0] <= ev[1] < 100.0
