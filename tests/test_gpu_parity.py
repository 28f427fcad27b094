"""GPU parity: every step of the CUDA path through the C ABI against the FP64
CPU oracle on the same seeded inputs.

Tolerances: integer work (the field) bit-exact; FP64 kernels 1e-12 relative
(rounding order only); A_hom of the FP64 solve 1e-10 relative per entry
(relative to max(|a11|, |a22|)); mixed precision 1e-7 on the same measure.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_12227_gb300 import rve, workloads

pytestmark = pytest.mark.gpu

CUDA = torch.device("cuda", 0)


def _rel_err_A(A, ref):
    scale = max(abs(ref[0, 0]), abs(ref[1, 1]))
    return np.abs(np.asarray(A) - ref).max() / scale


def _coef_np(d, mask):
    return np.where(mask, d["a_incl"], d["a_matrix"]).astype(np.float64)


def _pack(arrs):
    return torch.tensor(np.concatenate([a.reshape(-1, *a.shape[2:]) if a.ndim > 2 else a.reshape(-1)
                                        for a in arrs]), device=CUDA)


def _u_oracle_to_nodes(u):   # [2, n, n] -> [n*n, 2]
    return np.stack([u[0].ravel(), u[1].ravel()], axis=1)


# ------------------------------------------------------------------ field --
FIELD_CASES = [
    [workloads.realization(4, 8, 10.0, 0, 0)],                          # 32^2, 11 inclusions
    [workloads.realization(32, 16, 10.0, 5, k) for k in range(3)],     # 512^2, 717 inclusions
    workloads.config_batch("uneven_4096", seed=1, count=24),            # uneven sizes
    [workloads.realization(8, 8, 100.0, 2, 7, side_units=5.0)],         # s = 40 > 32: multi-word rows
    [dict(workloads.realization(4, 8, 10.0, 0, 0), n_incl=0)],          # empty field
    [dict(workloads.realization(4, 8, 10.0, 0, 0), incl_cells=32, n_incl=1)],   # s = n: full cover
    [workloads.realization(256, 8, 100.0, 0, 0)],                       # 2048^2, 45875 inclusions
]


@pytest.mark.parametrize("case", range(len(FIELD_CASES)))
def test_gen_field_bit_exact(case):
    ds = FIELD_CASES[case]
    mask = rve.gen_field(ds, device=CUDA)
    torch.cuda.synchronize()
    got = rve.unpack_mask(mask, ds)
    for d, m in zip(ds, got):
        np.testing.assert_array_equal(m, oracle.gen_field(d).astype(bool))


def test_coef_from_mask_bit_exact():
    ds = FIELD_CASES[1] + FIELD_CASES[2][:6]
    mask = rve.gen_field(ds, device=CUDA)
    coef = rve.coef_from_mask(ds, mask).cpu().numpy()
    off = 0
    for d in ds:
        n = d["L"] * d["m0"]
        ref = oracle.coef_from_mask(oracle.gen_field(d), d["a_matrix"], d["a_incl"])
        np.testing.assert_array_equal(coef[off:off + n * n].reshape(n, n), ref)
        off += n * n


# ------------------------------------------------------- rhs / stiffness --
def _setup(ds):
    mask = rve.gen_field(ds, device=CUDA)
    masks = rve.unpack_mask(mask, ds)
    coefs = [_coef_np(d, m) for d, m in zip(ds, masks)]
    return mask, coefs


SMALL = [workloads.realization(4, 8, 10.0, 3, k) for k in range(2)] + \
    [workloads.realization(8, 8, 100.0, 3, 9)]


@pytest.mark.parametrize("use_coef", [False, True])
def test_rhs_matches_oracle(use_coef):
    mask, coefs = _setup(SMALL)
    coef_t = torch.tensor(np.concatenate([c.ravel() for c in coefs]), device=CUDA)
    f = rve.rhs(SMALL, mask=None if use_coef else mask, coef=coef_t if use_coef else None)
    f = f.cpu().numpy()
    off = 0
    for d, c in zip(SMALL, coefs):
        n = c.shape[0]
        ref = oracle.rhs(c, 1.0 / d["m0"])
        got = f[off:off + n * n].reshape(n, n, 2)
        assert np.abs(got[..., 0] - ref[0]).max() < 1e-14
        assert np.abs(got[..., 1] - ref[1]).max() < 1e-14
        off += n * n


@pytest.mark.parametrize("scheme", [rve.CONSISTENT, rve.LUMPED])
def test_stiffness_matches_oracle_csr(scheme):
    mask, coefs = _setup(SMALL)
    g = np.random.default_rng(1)
    xs = [g.standard_normal((c.shape[0] ** 2, 2)) for c in coefs]
    x = torch.tensor(np.concatenate(xs), device=CUDA)
    y64 = rve.apply_stiffness(SMALL, x, mask=mask, scheme=scheme).cpu().numpy()
    y32 = rve.apply_stiffness(SMALL, x.float(), mask=mask, scheme=scheme).cpu().numpy()
    off = 0
    for d, c, xx in zip(SMALL, coefs, xs):
        n = c.shape[0]
        csr = oracle.assemble(c, 1.0 / d["m0"], scheme)
        for k in range(2):
            ref = oracle.spmv(csr, xx[:, k])
            sc = np.abs(ref).max()
            assert np.abs(y64[off:off + n * n, k] - ref).max() < 1e-13 * sc
            assert np.abs(y32[off:off + n * n, k] - ref).max() < 5e-6 * sc
        off += n * n


@pytest.mark.parametrize("delta", [0.0, 0.25])
def test_precond_matches_oracle(delta):
    ds = [workloads.realization(4, 8, 10.0, 0, 0), workloads.realization(16, 8, 100.0, 0, 1),
          workloads.realization(64, 8, 10.0, 0, 2), workloads.realization(8, 8, 10.0, 0, 3)]
    g = np.random.default_rng(2)
    xs = []
    for d in ds:
        n = d["L"] * d["m0"]
        r = g.standard_normal((n * n, 2))
        if delta == 0.0:
            r -= r.mean(axis=0)
        xs.append(r)
    x = torch.tensor(np.concatenate(xs), device=CUDA)
    z64 = rve.apply_precond(ds, x, delta=delta).cpu().numpy()
    z32 = rve.apply_precond(ds, x.float(), delta=delta).cpu().numpy()
    off = 0
    for d, r in zip(ds, xs):
        n = d["L"] * d["m0"]
        c0 = 0.5 * (d["a_matrix"] + d["a_incl"])
        for k in range(2):
            ref = oracle.precond(r[:, k].reshape(n, n), c0, delta).ravel()
            sc = np.abs(ref).max()
            assert np.abs(z64[off:off + n * n, k] - ref).max() < 1e-12 * sc
            assert np.abs(z32[off:off + n * n, k] - ref).max() < 2e-5 * sc
        off += n * n


# ---------------------------------------------------------- A_hom kernels --
@pytest.mark.parametrize("scheme", [rve.CONSISTENT, rve.LUMPED])
def test_a_hom_and_backward_kernels_on_oracle_correctors(scheme):
    ds = SMALL
    mask, coefs = _setup(ds)
    refs = [oracle.solve_coef(c, d["L"], d["m0"], 0.5 * (d["a_matrix"] + d["a_incl"]),
                              scheme=scheme, tol=1e-13) for d, c in zip(ds, coefs)]
    u = torch.tensor(np.concatenate([_u_oracle_to_nodes(r["u"]) for r in refs]), device=CUDA)
    A, Af = rve.a_hom(ds, u, mask=mask, scheme=scheme, want_flux=True)
    G = np.array([[[0.7, -0.3], [0.2, 1.1]]] * len(ds))
    grad = rve.a_hom_backward(ds, u, torch.tensor(G, device=CUDA), scheme=scheme).cpu().numpy()
    off = 0
    for k, (d, c, r) in enumerate(zip(ds, coefs, refs)):
        Ae, Afl = oracle.a_hom(c, r["u"], 1.0 / d["m0"], d["L"], scheme)
        assert _rel_err_A(A[k].cpu().numpy(), Ae) < 1e-12
        assert _rel_err_A(Af[k].cpu().numpy(), Afl) < 1e-12
        n = c.shape[0]
        gref = oracle.a_hom_grad(r["u"], G[k], 1.0 / d["m0"], d["L"], scheme)
        assert np.abs(grad[off:off + n * n].reshape(n, n) - gref).max() < 1e-12 * np.abs(gref).max()
        off += n * n


# -------------------------------------------------------------- solvers --
def _solve_and_hom(ds, opts, mask=None):
    if mask is None:
        mask = rve.gen_field(ds, device=CUDA)
    u, info = rve.solve(ds, mask=mask, opts=opts)
    A = rve.a_hom(ds, u, mask=mask, scheme=opts.scheme, precision=opts.precision).cpu().numpy()
    return mask, u, A, rve.info_to_dicts(info, len(ds))


SOLVE_CASES = {
    "single_L4": [workloads.realization(4, 8, 10.0, 0, 0)],
    "mixed_sizes": [workloads.realization(4, 8, 10.0, 1, 0), workloads.realization(16, 8, 100.0, 1, 1),
                    workloads.realization(8, 8, 10.0, 1, 2), workloads.realization(4, 16, 100.0, 1, 3)],
}


@pytest.mark.parametrize("case", sorted(SOLVE_CASES))
@pytest.mark.parametrize("scheme", [rve.CONSISTENT, rve.LUMPED])
@pytest.mark.parametrize("precision,path,bound", [(rve.FP64, rve.PATH_FUSED, 1e-10),
                                                  (rve.MIXED, rve.PATH_FUSED, 1e-7),
                                                  (rve.FP64, rve.PATH_PLAIN, 1e-10)])
def test_solve_matches_oracle(case, scheme, precision, path, bound):
    ds = SOLVE_CASES[case]
    tol = 1e-12 if precision == rve.FP64 else 1e-10
    opts = rve.make_opts(scheme=scheme, precision=precision, path=path, tol=tol)
    mask, u, A, info = _solve_and_hom(ds, opts)
    un = u.cpu().numpy()
    off = 0
    for k, d in enumerate(ds):
        # same tolerance as the GPU solve, so that iteration counts compare
        ref = oracle.solve_realization(d, scheme=scheme, tol=tol)
        assert info[k]["status"] == rve.RVE_OK, info[k]
        assert max(info[k]["relres"]) <= tol * 1.0001
        assert _rel_err_A(A[k], ref["A_energy"]) < bound, (A[k], ref["A_energy"])
        n = d["L"] * d["m0"]
        for c in range(2):
            ug = un[off:off + n * n, c]
            ug = ug - ug.mean()
            sc = np.abs(ref["u"][c]).max()
            assert np.abs(ug - ref["u"][c].ravel()).max() < (1e-8 if precision == rve.FP64 else 1e-6) * sc
        # iteration counts close to the oracle's: the rounding order differs,
        # and near tol = 1e-12 the CG tail drifts by a few iterations
        if precision == rve.FP64:
            for c in range(2):
                assert abs(info[k]["iters"][c] - ref["iters"][c]) <= max(3, 0.05 * ref["iters"][c])
        off += n * n


@pytest.mark.parametrize("scheme", [rve.CONSISTENT, rve.LUMPED])
def test_mixed_refine_integer_cells_same_bits_as_double_words(scheme):
    """With integer cell values (1 and the contrast) the mixed refinement
    forms its cell weights as exact floats instead of double words: the same
    values, so the same solve, bit for bit, as through the explicit
    coefficient input, which always takes the double-word weights."""
    ds = SOLVE_CASES["mixed_sizes"]
    opts = rve.make_opts(scheme=scheme, precision=rve.MIXED, tol=1e-10)
    mask = rve.gen_field(ds, device=CUDA)
    coef = rve.coef_from_mask(ds, mask)
    u1, i1 = rve.solve(ds, mask=mask, opts=opts)
    u2, i2 = rve.solve(ds, coef=coef, opts=opts)
    np.testing.assert_array_equal(u1.cpu().numpy(), u2.cpu().numpy())
    d1, d2 = rve.info_to_dicts(i1, len(ds)), rve.info_to_dicts(i2, len(ds))
    assert [d["iters"] for d in d1] == [d["iters"] for d in d2]
    assert [d["refinements"] for d in d1] == [d["refinements"] for d in d2]
    assert all(d["status"] == rve.RVE_OK for d in d1)


# ------------------------------------------ general load (Sec. 3.5) --
def _nodal_loads(ds):
    """Per realization the nodal loads sin(2 pi x/L) cos(6 pi y/L) and
    cos(2 pi x/L) sin(4 pi y/L) (both mean-zero on the torus), [nodes, 2]."""
    out = []
    for d in ds:
        n, h, L = d["L"] * d["m0"], 1.0 / d["m0"], d["L"]
        x = np.arange(n) * h
        g1 = np.outer(np.sin(2 * np.pi * x / L), np.cos(6 * np.pi * x / L))
        g2 = np.outer(np.cos(2 * np.pi * x / L), np.sin(4 * np.pi * x / L))
        out.append(np.stack([g1.ravel(), g2.ravel()], axis=1))
    return out


@pytest.mark.parametrize("scheme", [rve.CONSISTENT, rve.LUMPED])
def test_apply_mass_matches_oracle(scheme):
    ds = [workloads.realization(4, 8, 10.0, 0, 0), workloads.realization(8, 16, 10.0, 0, 1)]
    g = np.random.default_rng(5)
    xs = [g.standard_normal(((d["L"] * d["m0"]) ** 2, 2)) for d in ds]
    y = rve.apply_mass(ds, torch.tensor(np.concatenate(xs), device=CUDA), scheme=scheme).cpu().numpy()
    off = 0
    for d, x in zip(ds, xs):
        n, h = d["L"] * d["m0"], 1.0 / d["m0"]
        for c in range(2):
            ref = oracle.apply_mass(x[:, c].reshape(n, n), h, scheme).ravel()
            assert np.abs(y[off:off + n * n, c] - ref).max() < 1e-14 * np.abs(ref).max()
        off += n * n


@pytest.mark.parametrize("scheme", [rve.CONSISTENT, rve.LUMPED])
@pytest.mark.parametrize("precision,path,bound", [(rve.FP64, rve.PATH_FUSED, 1e-8),
                                                  (rve.MIXED, rve.PATH_FUSED, 1e-6),
                                                  (rve.MIXED, rve.PATH_PERSISTENT, 1e-6),
                                                  (rve.FP64, rve.PATH_PLAIN, 1e-8)])
def test_solve_rhs_matches_oracle(scheme, precision, path, bound):
    # the general solve A u = M g (the paper's FEM convergence test) on
    # mixed sizes, against the oracle's assembled solve with the same loads
    ds = [workloads.realization(2, 16, 10.0, 3, 0), workloads.realization(4, 16, 10.0, 3, 1),
          workloads.realization(8, 8, 100.0, 3, 2)]
    mask, coefs = _setup(ds)
    g = _nodal_loads(ds)
    f = rve.apply_mass(ds, torch.tensor(np.concatenate(g), device=CUDA), scheme=scheme)
    tol = 1e-12 if precision == rve.FP64 else 1e-10
    opts = rve.make_opts(scheme=scheme, precision=precision, path=path, tol=tol)
    u, info = rve.solve(ds, mask=mask, opts=opts, f=f)
    un = u.cpu().numpy()
    inf = rve.info_to_dicts(info, len(ds))
    off = 0
    # the plain path stops on the CG recurrence residual (textbook PCG, no
    # refinement): its true residual at exit may exceed tol by a few percent
    slack = 1.1 if path == rve.PATH_PLAIN else 1.0001
    for k, (d, c) in enumerate(zip(ds, coefs)):
        n, h = d["L"] * d["m0"], 1.0 / d["m0"]
        assert inf[k]["status"] == rve.RVE_OK, inf[k]
        assert max(inf[k]["relres"]) <= tol * slack
        for comp in range(2):
            b = oracle.apply_mass(g[k][:, comp].reshape(n, n), h, scheme)
            ref, _, _ = oracle.solve_load(c, d["L"], d["m0"], 0.5 * (d["a_matrix"] + d["a_incl"]),
                                          b, scheme=scheme, tol=1e-13)
            ug = un[off:off + n * n, comp] - un[off:off + n * n, comp].mean()
            assert np.abs(ug - ref.ravel()).max() < bound * np.abs(ref).max()
        off += n * n


# ---------------------------------------- spectral density (appendix) --
@pytest.mark.parametrize("scheme", [rve.CONSISTENT, rve.LUMPED])
def test_cheb_moments_match_dense_recurrence(scheme):
    from paper_1903_12227_gb300 import spectral
    ds = [workloads.realization(4, 8, 2.0, 6, 0, a_matrix=0.5),
          workloads.realization(8, 8, 10.0, 6, 1)]
    mask, coefs = _setup(ds)
    g = np.random.default_rng(8)
    vs = [g.standard_normal(((d["L"] * d["m0"]) ** 2, 2)) for d in ds]
    K = 64
    los_his = [spectral.spectral_bounds(d, scheme) for d in ds]
    lo = 0.0
    hi = max(h for _, h in los_his)
    mu = rve.cheb_moments(ds, torch.tensor(np.concatenate(vs), device=CUDA), K, lo, hi,
                          mask=mask, scheme=scheme).cpu().numpy()
    for k, (d, c, v) in enumerate(zip(ds, coefs, vs)):
        n = d["L"] * d["m0"]
        A = oracle.csr_to_dense(oracle.assemble(c, 1.0 / d["m0"], scheme), n * n)
        At = (2.0 * A - (hi + lo) * np.eye(n * n)) / (hi - lo)
        for comp in range(2):
            x = v[:, comp]
            w0, w1 = x, At @ x
            ref = [x @ w0, x @ w1]
            for _ in range(2, K):
                w0, w1 = w1, 2.0 * (At @ w1) - w0
                ref.append(x @ w1)
            ref = np.array(ref)
            assert np.abs(mu[k, comp] - ref).max() < 1e-10 * abs(ref[0])


def test_dos_exact_trace_matches_dense_spectrum():
    # unit start vectors e_0 .. e_{m-1} give the trace exactly, so the
    # Chebyshev density equals the oracle's dense-spectrum density up to the
    # (tiny) truncation of the Gaussian's expansion
    from paper_1903_12227_gb300 import spectral
    d = workloads.realization(4, 8, 2.0, 9, 0, density=1.0, side_units=0.5, a_matrix=0.5)
    n = d["L"] * d["m0"]
    m = n * n
    mask, coefs = _setup([d])
    lo, hi = spectral.spectral_bounds(d, rve.LUMPED)
    pairs = m // 2
    v = torch.zeros(pairs * m, 2, dtype=torch.float64, device=CUDA)
    idx = torch.arange(pairs, device=CUDA)
    v[idx * m + 2 * idx, 0] = 1.0
    v[idx * m + 2 * idx + 1, 1] = 1.0
    K = 400
    mu = rve.cheb_moments([d] * pairs, v, K, lo, hi, mask=mask.repeat(pairs), scheme=rve.LUMPED)
    tr = mu.sum(dim=(0, 1)).cpu().numpy()
    t = np.linspace(lo, hi, 301)
    eta = 0.1
    phi = spectral.dos_from_moments(tr, t, lo, hi, eta, m)
    ref = oracle.dos_gauss(oracle.spectrum(coefs[0], 1.0 / d["m0"], rve.LUMPED), t, eta)
    assert np.abs(phi - ref).max() < 1e-6 * ref.max()




def test_full_size_plain_L32_fp64_and_mixed():
    # the benchmark's workload size (512^2 nodes), one realization each way
    d = workloads.realization(32, 16, 10.0, 0, 0)
    ref = oracle.solve_realization(d, tol=1e-12, want_u=False)
    for precision, bound in ((rve.FP64, 1e-10), (rve.MIXED, 1e-7)):
        opts = rve.make_opts(precision=precision, tol=1e-10)
        _, _, A, info = _solve_and_hom([d], opts)
        assert info[0]["status"] == rve.RVE_OK
        assert _rel_err_A(A[0], ref["A_energy"]) < bound


def test_large_2048_properties():
    # 2048^2 nodes: f sums to zero, A annihilates constants, symmetry
    d = workloads.realization(256, 8, 100.0, 0, 0)
    mask = rve.gen_field([d], device=CUDA)
    f = rve.rhs([d], mask=mask)
    assert abs(f[:, 0].sum().item()) < 1e-9 and abs(f[:, 1].sum().item()) < 1e-9
    ones = torch.ones(2048 * 2048, 2, dtype=torch.float64, device=CUDA)
    y = rve.apply_stiffness([d], ones, mask=mask)
    assert y.abs().max().item() < 1e-12
    g = torch.randn(2048 * 2048, 2, dtype=torch.float64, device=CUDA)
    h = torch.randn(2048 * 2048, 2, dtype=torch.float64, device=CUDA)
    lhs = (g * rve.apply_stiffness([d], h, mask=mask)).sum(0)
    rhs_ = (h * rve.apply_stiffness([d], g, mask=mask)).sum(0)
    assert torch.allclose(lhs, rhs_, rtol=1e-10)


# ------------------------------------------------------------ edge cases --
def test_constant_field_gives_cI_and_zero_iterations():
    for d in (dict(workloads.realization(4, 8, 10.0, 0, 0), n_incl=0),
              dict(workloads.realization(4, 8, 10.0, 0, 0), incl_cells=32, n_incl=1),
              dict(workloads.realization(8, 8, 1.0, 0, 0))):
        for precision in (rve.FP64, rve.MIXED):
            _, u, A, info = _solve_and_hom([d], rve.make_opts(precision=precision))
            mask = oracle.gen_field(d)
            a = d["a_incl"] if mask.all() else d["a_matrix"]
            if d["a_incl"] == d["a_matrix"] or mask.all() or not mask.any():
                assert np.abs(A[0] - a * np.eye(2)).max() < 1e-14
                assert info[0]["iters"] == (0, 0)
                assert u.abs().max().item() == 0.0


def test_max_iter_reports_no_convergence():
    d = workloads.realization(8, 8, 100.0, 0, 0)
    for precision in (rve.FP64, rve.MIXED):
        _, _, _, info = _solve_and_hom([d], rve.make_opts(precision=precision, max_iter=2))
        assert info[0]["status"] == rve.RVE_ENOCONV
    _, _, _, info = _solve_and_hom([d], rve.make_opts(path=rve.PATH_PLAIN, max_iter=2))
    assert info[0]["status"] == rve.RVE_ENOCONV


def test_invalid_arguments_rejected_before_launch():
    d = workloads.realization(4, 8, 10.0, 0, 0)
    with pytest.raises(rve.RveError):
        rve.solve([d], mask=rve.gen_field([d], device=CUDA), opts=rve.make_opts(precision=7))
    with pytest.raises(rve.RveError):
        rve.gen_field([dict(d, m0=6)], device=CUDA)


def test_homogenize_host_matches_device_path():
    ds = [workloads.realization(4, 8, 10.0, 4, k) for k in range(5)]
    opts = rve.make_opts(precision=rve.MIXED)
    A_host, info = rve.homogenize_host(ds, opts, device=CUDA)
    _, _, A_dev, _ = _solve_and_hom(ds, opts)
    np.testing.assert_array_equal(A_host, A_dev)


def test_repeat_runs_bit_identical():
    ds = SOLVE_CASES["mixed_sizes"]
    opts = rve.make_opts(precision=rve.MIXED)
    _, u1, A1, _ = _solve_and_hom(ds, opts)
    _, u2, A2, _ = _solve_and_hom(ds, opts)
    np.testing.assert_array_equal(A1, A2)
    assert torch.equal(u1, u2)


# --------------------------------------------------------------- adjoint --
def test_autograd_matches_central_differences():
    d = workloads.realization(4, 8, 10.0, 6, 0)
    mask = oracle.gen_field(d)
    coef = torch.tensor(_coef_np(d, mask).ravel(), device=CUDA, requires_grad=True)
    opts = rve.make_opts(tol=1e-13)
    A = rve.AHom.apply(coef, [d], opts)
    G = torch.tensor([[[0.6, -0.2], [0.4, 1.3]]], dtype=torch.float64, device=CUDA)
    (A * G).sum().backward()
    g = coef.grad.cpu().numpy()
    cells = workloads.fd_cells(32, 8, seed=6, index=0)
    eps = 1e-6
    base = coef.detach().clone()
    for c1, c2 in cells:
        k = c1 * 32 + c2
        cp, cm = base.clone(), base.clone()
        cp[k] += eps
        cm[k] -= eps
        fp = (rve.AHom.apply(cp, [d], opts) * G).sum().item()
        fm = (rve.AHom.apply(cm, [d], opts) * G).sum().item()
        fd = (fp - fm) / (2 * eps)
        assert abs(fd - g[k]) < 1e-6 * max(abs(g).max(), 1e-12) + 1e-9
    # Euler identity: sum_c a_c dA_ij/da_c = A_ij (1-homogeneity)
    assert abs((g * base.cpu().numpy()).sum() - (A * G).sum().item()) < 1e-11
