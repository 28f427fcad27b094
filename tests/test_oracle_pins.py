"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
generator outputs, quadrature of the bilinear forms from their definitions,
closed forms (constant coefficient, laminates), a dense direct solve, the
paper's identities (symmetry, Voigt-Reuss bounds, Euler homogeneity) and
finite differences.  CPU only.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1903_12227_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers --
def _gauss2():
    g = 1.0 / np.sqrt(3.0)
    return [(0.5 - 0.5 * g, 0.5), (0.5 + 0.5 * g, 0.5)]   # (point, weight) on [0,1]


def _bilinear_grad(v4, t1, t2, h):
    """Gradient of the bilinear interpolant of local values (00,01,10,11) at (t1,t2) in [0,1]^2."""
    v00, v01, v10, v11 = v4
    d1 = ((v10 - v00) * (1 - t2) + (v11 - v01) * t2) / h
    d2 = ((v01 - v00) * (1 - t1) + (v11 - v10) * t1) / h
    return d1, d2


def _cell_vals(x, c1, c2):
    n = x.shape[0]
    p1, p2 = (c1 + 1) % n, (c2 + 1) % n
    return (x[c1, c2], x[c1, p2], x[p1, c2], x[p1, p2])


def _quad_energy(coef, u, v, h, scheme):
    """int a grad(u_h).grad(v_h) by quadrature, cell by cell (no element matrix).

    consistent: 2x2 Gauss (exact for Q1); lumped: the d1.d1 term with the
    trapezoid rule in x2 and the d2.d2 term with the trapezoid rule in x1."""
    n = coef.shape[0]
    total = 0.0
    g = _gauss2()
    trap = [(0.0, 0.5), (1.0, 0.5)]
    for c1 in range(n):
        for c2 in range(n):
            uu, vv = _cell_vals(u, c1, c2), _cell_vals(v, c1, c2)
            s = 0.0
            if scheme == oracle.SCHEME_CONSISTENT:
                for t1, w1 in g:
                    for t2, w2 in g:
                        du, dv = _bilinear_grad(uu, t1, t2, h), _bilinear_grad(vv, t1, t2, h)
                        s += w1 * w2 * (du[0] * dv[0] + du[1] * dv[1])
            else:
                for t1, w1 in g:
                    for t2, w2 in trap:
                        du, dv = _bilinear_grad(uu, t1, t2, h), _bilinear_grad(vv, t1, t2, h)
                        s += w1 * w2 * du[0] * dv[0]
                for t1, w1 in trap:
                    for t2, w2 in g:
                        du, dv = _bilinear_grad(uu, t1, t2, h), _bilinear_grad(vv, t1, t2, h)
                        s += w1 * w2 * du[1] * dv[1]
            total += coef[c1, c2] * s * h * h
    return total


def _random_coef(n, seed, lo=1.0, hi=10.0):
    g = np.random.default_rng(seed)
    return np.where(g.random((n, n)) < 0.45, hi, lo)


# ------------------------------------------------------------------ field --
def test_splitmix64_published_vectors():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    assert [oracle.splitmix64_output(1234567, k) for k in range(1, 6)] == vals


def test_field_union_matches_predicate():
    # brute force: cell covered iff some inclusion's (wrapped) square contains it
    for d in [workloads.realization(4, 8, 10.0, 3, 0), workloads.realization(3, 4, 10.0, 5, 2),
              workloads.realization(2, 16, 10.0, 9, 1, side_units=0.5)]:
        n = d["L"] * d["m0"]
        s = d["incl_cells"]
        c = oracle.corners(d)
        assert c.min() >= 0 and c.max() < n
        i1, i2 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        cov = np.zeros((n, n), dtype=bool)
        for k in range(d["n_incl"]):
            cov |= (((i1 - c[k, 0]) % n) < s) & (((i2 - c[k, 1]) % n) < s)
        np.testing.assert_array_equal(oracle.gen_field(d).astype(bool), cov)


def test_field_coverage_statistics():
    # E[covered fraction] = 1 - (1 - s^2/n^2)^N_inc for independent uniform corners
    fr = []
    for k in range(400):
        d = workloads.realization(8, 4, 10.0, 11, k)
        fr.append(oracle.gen_field(d).mean())
    d = workloads.realization(8, 4, 10.0, 11, 0)
    n, s, N = 32, d["incl_cells"], d["n_incl"]
    expect = 1.0 - (1.0 - s * s / (n * n)) ** N
    fr = np.asarray(fr)
    assert abs(fr.mean() - expect) < 4 * fr.std() / np.sqrt(len(fr)) + 1e-3


def test_corner_marginals_uniform():
    d = workloads.realization(64, 8, 10.0, 1, 0)   # n = 512, 2867 inclusions
    c = oracle.corners(d).ravel()
    hist = np.bincount(c // 64, minlength=8)
    expect = c.size / 8
    chi2 = ((hist - expect) ** 2 / expect).sum()
    assert chi2 < 30.0      # 7 dof: p ~ 1e-4


def _splitmix64_stream(seed, k):
    """Output k >= 1 of the SplitMix64 stream seeded with `seed`, restated
    from the generator's published definition (Steele, Lea & Flood 2014):
    the state advances by the golden-ratio gamma and each output is the
    state put through the variant-13 finaliser."""
    M = (1 << 64) - 1
    z = (seed + k * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


@pytest.mark.parametrize("seed,index,L,m0", [(0, 0, 4, 8), (7, 123456, 32, 16),
                                             (2**63 + 5, 3, 8, 8), (1234567, 2**40 + 9, 64, 16)])
def test_corner_draws_restated_from_reading_R1(seed, index, L, m0):
    """Reading R1 written out independently of the oracle: the realization key
    is output index+1 of the run seed's stream; draw ctr under tag 1 is output
    (2^40 + ctr + 1) of the key's stream; inclusion k takes draws 2k (row)
    and 2k+1 (column); a corner is the high word of draw * n (Lemire's
    multiply-high, no rejection).  A slip in bit order, counter packing or
    draw pairing in the oracle fails this bit for bit."""
    d = workloads.realization(L, m0, 10.0, seed, index)
    n = L * m0
    key = _splitmix64_stream(seed, index + 1)
    want = np.array([[(_splitmix64_stream(key, (1 << 40) + 2 * k + a + 1) * n) >> 64
                      for a in (0, 1)] for k in range(d["n_incl"])], dtype=np.int64)
    np.testing.assert_array_equal(oracle.corners(d).astype(np.int64), want)


# --------------------------------------------------------------- assembly --
@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_element_matrix_equals_quadrature(scheme):
    h = 0.125
    E = oracle.element_matrix(scheme, h)
    for a in range(4):
        for b in range(4):
            ea = np.zeros(4); ea[a] = 1
            eb = np.zeros(4); eb[b] = 1
            # one cell of a 2x2 torus would wrap; use the local formula directly
            s = 0.0
            g = _gauss2()
            trap = [(0.0, 0.5), (1.0, 0.5)]
            if scheme == oracle.SCHEME_CONSISTENT:
                for t1, w1 in g:
                    for t2, w2 in g:
                        du, dv = _bilinear_grad(ea, t1, t2, h), _bilinear_grad(eb, t1, t2, h)
                        s += w1 * w2 * (du[0] * dv[0] + du[1] * dv[1])
            else:
                for t1, w1 in g:
                    for t2, w2 in trap:
                        du, dv = _bilinear_grad(ea, t1, t2, h), _bilinear_grad(eb, t1, t2, h)
                        s += w1 * w2 * du[0] * dv[0]
                for t1, w1 in trap:
                    for t2, w2 in g:
                        du, dv = _bilinear_grad(ea, t1, t2, h), _bilinear_grad(eb, t1, t2, h)
                        s += w1 * w2 * du[1] * dv[1]
            assert abs(E[a, b] - s * h * h) < 1e-14


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_stiffness_equals_quadrature_bilinear_form(scheme):
    n, h = 6, 0.25
    coef = _random_coef(n, 1)
    csr = oracle.assemble(coef, h, scheme)
    g = np.random.default_rng(2)
    for _ in range(3):
        u = g.standard_normal((n, n))
        v = g.standard_normal((n, n))
        lhs = float(u.ravel() @ oracle.spmv(csr, v))
        rhs = _quad_energy(coef, u, v, h, scheme)
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(rhs))


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_stiffness_structure(scheme):
    n, h = 8, 0.5
    coef = _random_coef(n, 4)
    A = oracle.csr_to_dense(oracle.assemble(coef, h, scheme), n * n)
    assert np.abs(A - A.T).max() < 1e-14
    assert np.abs(A.sum(axis=1)).max() < 1e-13            # constants in the kernel
    ev = np.linalg.eigvalsh(A)
    assert ev[0] > -1e-12 and ev[1] > 1e-6                  # PSD, one-dimensional kernel
    rowptr = oracle.assemble(coef, h, scheme)[0]
    width = np.diff(rowptr)
    assert (width == (9 if scheme == oracle.SCHEME_CONSISTENT else 5)).all() or \
        (scheme == oracle.SCHEME_LUMPED and (width <= 9).all())


def test_lumped_constant_is_fd_laplacian():
    # the paper's lumped scheme with a = 1 is exactly its 5-point A_Delta
    n = 8
    A = oracle.csr_to_dense(oracle.assemble(np.ones((n, n)), 0.5, oracle.SCHEME_LUMPED), n * n)
    D = _paper_A_Delta(n)
    assert np.abs(A - D).max() < 1e-14


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_rhs_equals_quadrature(scheme):
    # f_i . v = -int a d_i v_h, by Gauss quadrature of the bilinear interpolant
    n, h = 6, 0.25
    coef = _random_coef(n, 5)
    f = oracle.rhs(coef, h, scheme)
    v = np.random.default_rng(6).standard_normal((n, n))
    for i in range(2):
        s = 0.0
        for c1 in range(n):
            for c2 in range(n):
                vv = _cell_vals(v, c1, c2)
                for t1, w1 in _gauss2():
                    for t2, w2 in _gauss2():
                        s += coef[c1, c2] * w1 * w2 * _bilinear_grad(vv, t1, t2, h)[i] * h * h
        assert abs(float((f[i] * v).sum()) + s) < 1e-13
        assert abs(f[i].sum()) < 1e-13


# ---------------------------------------------------------- preconditioner --
def _paper_A_Delta(n):
    """A_Delta = (-Delta_P) (x) I + I (x) (-Delta_P), Delta_P of Eq. "BC_Neu_peri"."""
    DP = -2 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    DP[0, -1] = DP[-1, 0] = 1
    I = np.eye(n)
    return np.kron(-DP, I) + np.kron(I, -DP)


def test_laplacian_eigenvalues_closed_form():
    n = 8
    ev = np.sort(np.linalg.eigvalsh(_paper_A_Delta(n)))
    cf = np.sort([oracle.laplacian_eig(n, k1, k2) for k1 in range(n) for k2 in range(n)])
    assert np.abs(ev - cf).max() < 1e-12


@pytest.mark.parametrize("delta", [0.0, 0.3])
def test_precond_inverts_B(delta):
    n, c0 = 16, 5.5
    r = np.random.default_rng(7).standard_normal((n, n))
    if delta == 0.0:
        r -= r.mean()
    z = oracle.precond(r, c0, delta)
    B = c0 * _paper_A_Delta(n) + delta * np.eye(n * n)
    assert np.abs(B @ z.ravel() - r.ravel()).max() < 1e-12
    if delta == 0.0:
        assert abs(z.mean()) < 1e-14


# ------------------------------------------------------------------ solver --
@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_pcg_matches_dense_direct_solve(scheme):
    for n, m0, seed in [(8, 4, 1), (16, 8, 2)]:
        L = n // m0
        h = 1.0 / m0
        coef = _random_coef(n, seed)
        csr = oracle.assemble(coef, h, scheme)
        A = oracle.csr_to_dense(csr, n * n)
        f = oracle.rhs(coef, h, scheme)
        ones = np.ones(n * n) / n
        for i in range(2):
            u, it, rr = oracle.pcg(csr, f[i], 5.5, 1e-14, 2000)
            # bordered system fixes the mean to zero (textbook dense solve)
            K = np.block([[A, ones[:, None]], [ones[None, :], np.zeros((1, 1))]])
            x = np.linalg.solve(K, np.concatenate([f[i].ravel(), [0.0]]))[:-1]
            assert np.abs(u.ravel() - x).max() < 1e-10 * max(1.0, np.abs(x).max())
            assert rr < 1e-12
        Ae, Af = oracle.a_hom(coef, np.stack([oracle.pcg(csr, f[i], 5.5, 1e-14, 2000)[0]
                                              for i in range(2)]), h, L, scheme)
        assert np.abs(Ae - Af).max() < 1e-11


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_constant_coefficient_gives_cI(scheme):
    n, m0 = 16, 4
    r = oracle.solve_coef(np.full((n, n), 3.25), n // m0, m0, c0=3.25, scheme=scheme)
    assert (r["iters"] == 0).all()
    assert np.abs(r["A_energy"] - 3.25 * np.eye(2)).max() < 1e-13
    assert np.abs(r["A_flux"] - 3.25 * np.eye(2)).max() < 1e-13


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
@pytest.mark.parametrize("axis", [0, 1])
def test_laminate_harmonic_and_arithmetic_means(scheme, axis):
    # coefficient varying along x_{axis+1} only: A along that axis is the harmonic
    # mean, across it the arithmetic mean, off-diagonals zero (exact for Q1)
    n, m0 = 32, 4
    prof = np.array([1.0, 1.0, 7.0, 2.5, 2.5, 2.5, 10.0, 1.0] * 4)
    coef = np.repeat(prof[:, None], n, axis=1) if axis == 0 else np.repeat(prof[None, :], n, axis=0)
    r = oracle.solve_coef(coef, n // m0, m0, c0=5.5, scheme=scheme, tol=1e-14)
    harm, arith = 1.0 / np.mean(1.0 / prof), np.mean(prof)
    expect = np.diag([harm, arith]) if axis == 0 else np.diag([arith, harm])
    for key in ("A_energy", "A_flux"):
        assert np.abs(r[key] - expect).max() < 1e-12 * arith


def test_symmetry_and_flux_asymmetry_trend():
    # energy form symmetric by construction; flux asymmetry shrinks with the
    # tolerance (the trend of the paper's symmetry-vs-tolerance table)
    d = workloads.realization(4, 8, 5.0, 2, 0, side_units=0.5)   # contrast 5
    asym = []
    for tol in (1e-4, 1e-7, 1e-10, 1e-13):
        r = oracle.solve_realization(d, tol=tol, want_u=False)
        assert abs(r["A_energy"][0, 1] - r["A_energy"][1, 0]) < 1e-14
        asym.append(abs(r["A_flux"][0, 1] - r["A_flux"][1, 0]))
    assert asym[-1] < 1e-11
    assert asym[0] > asym[-1]


def test_voigt_reuss_bounds():
    for k in range(3):
        d = workloads.realization(4, 8, 10.0, 21, k)
        r = oracle.solve_realization(d, tol=1e-12)
        coef = np.where(r["mask"] == 1, d["a_incl"], d["a_matrix"])
        harm, arith = 1.0 / np.mean(1.0 / coef), np.mean(coef)
        ev = np.linalg.eigvalsh(r["A_energy"])
        assert harm < ev[0] <= ev[1] < arith
        assert abs(r["mean_a"] - arith) < 1e-14


def test_energy_form_above_converged_for_inexact_solve():
    d = workloads.realization(4, 8, 10.0, 5, 0)
    ref = oracle.solve_realization(d, tol=1e-13, want_u=False)["A_energy"]
    for tol in (1e-2, 1e-3, 1e-5):
        A = oracle.solve_realization(d, tol=tol, want_u=False)["A_energy"]
        assert A[0, 0] >= ref[0, 0] - 1e-15 and A[1, 1] >= ref[1, 1] - 1e-15


# ---------------------------------------------------------------- gradient --
def _solve_u(coef, m0, scheme=oracle.SCHEME_CONSISTENT, c0=5.5):
    n = coef.shape[0]
    return oracle.solve_coef(coef, n // m0, m0, c0=c0, scheme=scheme, tol=1e-14, max_iter=5000)


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_gradient_euler_identity(scheme):
    # A is 1-homogeneous in a: sum_c a_c dA_ij/da_c = A_ij
    n, m0 = 16, 4
    coef = _random_coef(n, 8)
    r = _solve_u(coef, m0, scheme)
    for i in range(2):
        for j in range(2):
            G = np.zeros((2, 2)); G[i, j] = 1
            g = oracle.a_hom_grad(r["u"], G, 1.0 / m0, n // m0, scheme)
            assert abs((coef * g).sum() - r["A_energy"][i, j]) < 1e-12
            if i == j:
                assert g.min() >= 0.0


def test_gradient_constant_field_closed_form():
    n, m0 = 8, 4
    r = _solve_u(np.full((n, n), 2.0), m0)
    h, L = 1.0 / m0, n // m0
    for i in range(2):
        for j in range(2):
            G = np.zeros((2, 2)); G[i, j] = 1
            g = oracle.a_hom_grad(r["u"], G, h, L)
            assert np.abs(g - (1.0 if i == j else 0.0) * h * h / L ** 2).max() < 1e-15


def test_gradient_matches_central_differences():
    n, m0 = 8, 4
    coef = _random_coef(n, 9)
    r = _solve_u(coef, m0)
    G = np.array([[0.7, -0.4], [0.25, 1.3]])
    g = oracle.a_hom_grad(r["u"], G, 1.0 / m0, n // m0)
    eps = 1e-5
    for c in [(0, 0), (3, 5), (7, 7), (2, 6)]:
        cp, cm = coef.copy(), coef.copy()
        cp[c] += eps
        cm[c] -= eps
        fd = ((G * _solve_u(cp, m0)["A_energy"]).sum() -
              (G * _solve_u(cm, m0)["A_energy"]).sum()) / (2 * eps)
        assert abs(fd - g[c]) < 1e-8 * max(1.0, abs(g[c])) + 1e-9


# -------------------------------------------------------------- statistics --
def test_statistics_match_numpy():
    g = np.random.default_rng(3)
    A = g.standard_normal((50, 2, 2))
    A[:, 1, 0] = A[:, 0, 1]
    L = 16
    s = oracle.statistics(A, L)
    flat = A.reshape(50, 4)
    np.testing.assert_allclose(s["mean"].ravel(), flat.mean(axis=0), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(s["Q"], L ** 2 * np.cov(flat, rowvar=False, ddof=1), rtol=1e-12,
                               atol=1e-13)
    np.testing.assert_allclose(s["var"].ravel(), flat.var(axis=0, ddof=1), rtol=1e-12)
    assert abs(s["std12_paper"] - np.sqrt((flat[:, 1] ** 2).mean())) < 1e-14
    assert abs(s["stddiff_paper"] - np.sqrt(((flat[:, 0] - flat[:, 3]) ** 2).mean())) < 1e-14
    # symmetric A => the paper's identities among Q's entries hold exactly
    Q = s["Q"]
    assert abs(Q[1, 1] - Q[1, 2]) < 1e-12 and abs(Q[2, 2] - Q[1, 2]) < 1e-12


def test_workload_inclusion_counts():
    assert workloads.realization(4, 8, 10, 0, 0)["n_incl"] == 11
    assert workloads.realization(32, 16, 10, 0, 0)["n_incl"] == 717
    assert workloads.realization(64, 16, 100, 0, 0)["n_incl"] == 2867
    assert workloads.realization(256, 8, 100, 0, 0)["n_incl"] == 45875
    assert workloads.realization(8, 8, 10, 0, 0)["n_incl"] == 45
    assert workloads.realization(16, 8, 10, 0, 0)["n_incl"] == 179
    # 3D: round(0.7 L^3) unit cubes
    assert [workloads.realization3(L, 16, 10, 0, 0)["n_incl"] for L in (2, 4, 8, 16)] == \
        [6, 45, 358, 2867]
    assert workloads.realization3(4, 16, 10, 0, 0)["incl_cells"] == 16


# ------------------------------------------------- general load (Sec. 3.5) --
def _bilinear_basis(t1, t2):
    """Q1 shape functions in local order 00, 01, 10, 11 at (t1, t2) in [0,1]^2."""
    return np.array([(1 - t1) * (1 - t2), (1 - t1) * t2, t1 * (1 - t2), t1 * t2])


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_mass_element_equals_quadrature(scheme):
    # consistent: int phi_a phi_b over the cell (2x2 Gauss is exact for these
    # degree-2 products); lumped: the trapezoid rule in both directions
    h = 0.25
    M = oracle.mass_element(scheme, h)
    pts = _gauss2() if scheme == oracle.SCHEME_CONSISTENT else [(0.0, 0.5), (1.0, 0.5)]
    ref = np.zeros((4, 4))
    for t1, w1 in pts:
        for t2, w2 in pts:
            phi = _bilinear_basis(t1, t2)
            ref += w1 * w2 * np.outer(phi, phi) * h * h
    np.testing.assert_allclose(M, ref, atol=1e-16)


def _symbols(theta, h, scheme):
    """1D stiffness and mass symbols of a Fourier mode with phase theta per node."""
    k = (2.0 - 2.0 * np.cos(theta)) / h
    m = h * (4.0 + 2.0 * np.cos(theta)) / 6.0 if scheme == oracle.SCHEME_CONSISTENT else h
    return k, m


def _mode_load(L, m0):
    n, h = L * m0, 1.0 / m0
    x = np.arange(n) * h
    return np.outer(np.sin(2 * np.pi * x / L), np.cos(6 * np.pi * x / L))


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_load_solve_constant_coefficient_fourier_mode(scheme):
    # a = c: K and M are diagonal on the torus's product Fourier modes, so the
    # discrete solution of c K u = M g for g = sin(2 pi x/L) cos(6 pi y/L) is
    # g times m1 m2 / (c (k1 m2 + m1 k2)) with the 1D symbols k, m
    L, m0, c = 4, 8, 2.5
    n, h = L * m0, 1.0 / m0
    g = _mode_load(L, m0)
    b = oracle.apply_mass(g, h, scheme)
    u, it, rr = oracle.solve_load(np.full((n, n), c), L, m0, c, b, scheme=scheme, tol=1e-13)
    k1, m1 = _symbols(2 * np.pi * h / L, h, scheme)
    k2, m2 = _symbols(6 * np.pi * h / L, h, scheme)
    exact = g * (m1 * m2) / (c * (k1 * m2 + m1 * k2))
    assert rr <= 1e-13
    assert np.abs(u - exact).max() < 1e-11 * np.abs(exact).max()


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_load_solve_second_order_convergence(scheme):
    # constant coefficient: the nodal error against -c Lap u = g, u = g / (c |w|^2),
    # falls by ~4 per grid halving (second-order FEM)
    L, c = 2, 1.5
    w2 = (2 * np.pi / L) ** 2 + (6 * np.pi / L) ** 2
    errs = []
    for m0 in (16, 32, 64):
        n, h = L * m0, 1.0 / m0
        g = _mode_load(L, m0)
        u, _, _ = oracle.solve_load(np.full((n, n), c), L, m0, c, oracle.apply_mass(g, h, scheme),
                                    scheme=scheme, tol=1e-13)
        errs.append(np.abs(u - g / (c * w2)).max())
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.7 < e0 / e1 < 4.3, errs


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_load_solve_matches_dense_direct_solve(scheme):
    # jumping coefficient on a tiny torus: PCG against a direct solve of the
    # bordered system [A 1; 1^T 0] [u; s] = [b; 0] (mean-zero solution)
    L, m0 = 2, 4
    n, h = L * m0, 1.0 / m0
    coef = _random_coef(n, 7, lo=0.1, hi=1.0)
    b = oracle.apply_mass(_mode_load(L, m0), h, scheme)
    A = oracle.csr_to_dense(oracle.assemble(coef, h, scheme), n * n)
    Bord = np.zeros((n * n + 1, n * n + 1))
    Bord[:-1, :-1] = A
    Bord[:-1, -1] = 1.0
    Bord[-1, :-1] = 1.0
    ref = np.linalg.solve(Bord, np.concatenate([b.ravel(), [0.0]]))[:-1]
    u, _, rr = oracle.solve_load(coef, L, m0, 0.55, b, scheme=scheme, tol=1e-14)
    assert np.abs(u.ravel() - ref).max() < 1e-11 * np.abs(ref).max()


# ------------------------------------------- spectral density (appendix) --
@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_spectrum_constant_coefficient_closed_form(scheme):
    # a = c: the eigenvalues of A are the Fourier symbols
    # c (k(t1) m(t2) + m(t1) k(t2)), k = 2 - 2 cos t and m the 1D mass symbol
    # over h (consistent (4 + 2 cos t)/6, lumped 1; the factors h cancel),
    # t = 2 pi p / n
    n, h, c = 16, 0.25, 1.7
    ev = oracle.spectrum(np.full((n, n), c), h, scheme)
    t = 2 * np.pi * np.arange(n) / n
    k = 2.0 - 2.0 * np.cos(t)
    m = (4.0 + 2.0 * np.cos(t)) / 6.0 if scheme == oracle.SCHEME_CONSISTENT else np.ones(n)
    ref = np.sort((c * (np.outer(k, m) + np.outer(m, k))).ravel())
    np.testing.assert_allclose(ev, ref, atol=1e-12 * ref.max())


def test_dos_gauss_normalised_and_centred():
    # the broadened density integrates to one and its mean is Tr(A)/m
    n, h = 16, 0.25
    coef = _random_coef(n, 3, lo=0.5, hi=1.0)
    ev = oracle.spectrum(coef, h)
    t = np.linspace(ev.min() - 1.0, ev.max() + 1.0, 4001)
    phi = oracle.dos_gauss(ev, t, 0.05)
    dt = t[1] - t[0]
    assert abs(phi.sum() * dt - 1.0) < 1e-6
    A = oracle.csr_to_dense(oracle.assemble(coef, h), n * n)
    assert abs((t * phi).sum() * dt - np.trace(A) / (n * n)) < 1e-6


@pytest.mark.parametrize("eta", [0.05, 0.3])
def test_dos_gauss_width_from_second_moment(eta):
    """The broadened density's second central moment is the spectrum's
    variance plus eta^2 (a Gaussian of standard deviation eta convolved with
    the eigenvalue distribution), with the spectrum's moments taken from the
    matrix itself: mean Tr(A)/m and second moment ||A||_F^2 / m = Tr(A^2)/m.
    A width misread as a variance (eta instead of eta^2) or a wrong
    normalisation of the exponent fails this."""
    n, h = 16, 0.25
    coef = _random_coef(n, 4, lo=0.5, hi=1.0)
    ev = oracle.spectrum(coef, h)
    t = np.linspace(ev.min() - 12 * eta, ev.max() + 12 * eta, 20001)
    phi = oracle.dos_gauss(ev, t, eta)
    dt = t[1] - t[0]
    A = oracle.csr_to_dense(oracle.assemble(coef, h), n * n)
    m = n * n
    mean = np.trace(A) / m
    var = (A * A).sum() / m - mean ** 2
    mom2 = ((t - mean) ** 2 * phi).sum() * dt
    assert abs(mom2 - (var + eta ** 2)) < 1e-6 * (var + eta ** 2)


# ---------------------------------------------------------------- 3D --
def _trilinear_grad(e8, t, h):
    """Gradient of the trilinear interpolant of local values (a = 4a1+2a2+a3) at t in [0,1]^3."""
    g = np.zeros(3)
    for a in range(8):
        bits = ((a >> 2) & 1, (a >> 1) & 1, a & 1)
        for ax in range(3):
            prod = 1.0
            for k in range(3):
                if k == ax:
                    prod *= (1.0 if bits[k] else -1.0) / h
                else:
                    prod *= t[k] if bits[k] else (1.0 - t[k])
            g[ax] += e8[a] * prod
    return g


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_element_matrix3_equals_quadrature(scheme):
    # consistent: 2-point Gauss in every direction (exact); lumped: Gauss in
    # the derivative's direction, trapezoid in the other two
    h = 0.5
    E = oracle.element_matrix3(scheme, h)
    gauss, trap = _gauss2(), [(0.0, 0.5), (1.0, 0.5)]
    for a in range(8):
        for b in range(8):
            ea, eb = np.eye(8)[a], np.eye(8)[b]
            s = 0.0
            for ax in range(3):
                rules = [gauss if (scheme == oracle.SCHEME_CONSISTENT or k == ax) else trap
                         for k in range(3)]
                for t1, w1 in rules[0]:
                    for t2, w2 in rules[1]:
                        for t3, w3 in rules[2]:
                            ga = _trilinear_grad(ea, (t1, t2, t3), h)
                            gb = _trilinear_grad(eb, (t1, t2, t3), h)
                            s += w1 * w2 * w3 * ga[ax] * gb[ax]
            assert abs(E[a, b] - s * h ** 3) < 1e-14


def test_stiffness3_structure():
    n, h = 4, 0.5
    coef = np.random.default_rng(3).uniform(0.5, 2.0, (n, n, n))
    A = oracle.csr_to_dense(oracle.assemble3(coef, h), n ** 3)
    assert np.abs(A - A.T).max() < 1e-14
    assert np.abs(A.sum(axis=1)).max() < 1e-13
    ev = np.linalg.eigvalsh(A)
    assert abs(ev[0]) < 1e-12 and ev[1] > 1e-6      # PSD, one-dimensional kernel
    # the trilinear element couples edge-adjacent corners with weight 0, so
    # the six axis neighbours drop out: 1 + 12 + 8 = 21 entries per row
    assert all(np.count_nonzero(np.abs(A[r]) > 1e-15) == 21 for r in range(n ** 3))


def test_field3_union_matches_predicate():
    d = {"L": 2, "m0": 4, "incl_cells": 3, "n_incl": 5, "a_matrix": 1.0, "a_incl": 5.0,
         "seed": 77, "index": 3}
    n = 8
    L = oracle.lib()
    key = L.orc_realization_key(77, 3)
    ref = np.zeros((n, n, n), dtype=np.uint8)
    for k in range(5):
        c = [(L.orc_draw(key, 1, 3 * k + a) * n) >> 64 for a in range(3)]
        for d1 in range(3):
            for d2 in range(3):
                for d3 in range(3):
                    ref[(c[0] + d1) % n, (c[1] + d2) % n, (c[2] + d3) % n] = 1
    np.testing.assert_array_equal(oracle.gen_field3(d), ref)


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_constant_coefficient3_gives_cI(scheme):
    n, c = 8, 2.5
    coef = np.full((n, n, n), c)
    assert np.abs(oracle.rhs3(coef, 0.25, scheme)).max() < 1e-14
    r = oracle.solve_coef3(coef, 2, 4, c, scheme)
    np.testing.assert_allclose(r["A_energy"], c * np.eye(3), atol=1e-13)
    np.testing.assert_allclose(r["A_flux"], c * np.eye(3), atol=1e-13)


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_laminate3_harmonic_and_arithmetic_means(scheme):
    # a depends on the first coordinate only: a_11 = harmonic mean, a_22 =
    # a_33 = arithmetic mean, off-diagonals zero (exact for the Q1 scheme)
    n = 8
    prof = np.array([1.0, 1.0, 7.0, 7.0, 7.0, 2.0, 1.0, 3.0])
    coef = np.broadcast_to(prof[:, None, None], (n, n, n)).copy()
    r = oracle.solve_coef3(coef, 2, 4, 4.0, scheme, tol=1e-13)
    harm, arith = 1.0 / np.mean(1.0 / prof), np.mean(prof)
    ref = np.diag([harm, arith, arith])
    np.testing.assert_allclose(r["A_energy"], ref, atol=1e-11)
    np.testing.assert_allclose(r["A_flux"], ref, atol=1e-10)


def test_precond3_inverts_B():
    # B = c0 A_Delta + delta I with the periodic 7-point Laplacian, built densely
    n, c0 = 8, 1.5
    N = n ** 3
    idx = np.arange(N).reshape(n, n, n)
    Ad = np.zeros((N, N))
    for ax in range(3):
        for sh in (-1, 1):
            nb = np.roll(idx, sh, axis=ax).ravel()
            Ad[np.arange(N), nb] -= 1.0
    Ad[np.arange(N), np.arange(N)] += 6.0
    r = np.random.default_rng(4).standard_normal((n, n, n))
    for delta in (0.0, 0.3):
        rr = r - r.mean() if delta == 0.0 else r
        z = oracle.precond3(rr, c0, delta)
        np.testing.assert_allclose((c0 * Ad + delta * np.eye(N)) @ z.ravel(), rr.ravel(), atol=1e-11)


def test_pcg3_matches_dense_direct_solve():
    n, h = 4, 0.5
    coef = np.where(np.random.default_rng(6).random((n, n, n)) < 0.4, 8.0, 1.0)
    A = oracle.csr_to_dense(oracle.assemble3(coef, h), n ** 3)
    f = oracle.rhs3(coef, h)
    r = oracle.solve_coef3(coef, 2, 2, 4.5, tol=1e-14)
    Bord = np.zeros((n ** 3 + 1, n ** 3 + 1))
    Bord[:-1, :-1] = A
    Bord[:-1, -1] = Bord[-1, :-1] = 1.0
    for i in range(3):
        ref = np.linalg.solve(Bord, np.concatenate([f[i].ravel(), [0.0]]))[:-1]
        assert np.abs(r["u"][i].ravel() - ref).max() < 1e-11 * np.abs(ref).max()


def test_voigt_reuss3_bounds():
    d = {"L": 2, "m0": 4, "incl_cells": 4, "n_incl": 6, "a_matrix": 1.0, "a_incl": 10.0,
         "seed": 5, "index": 0}
    r = oracle.solve_realization3(d)
    mask = r["mask"]
    a = np.where(mask, 10.0, 1.0)
    ev = np.linalg.eigvalsh(0.5 * (r["A_energy"] + r["A_energy"].T))
    assert 1.0 / np.mean(1.0 / a) <= ev[0] and ev[-1] <= np.mean(a)


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_a_hom3_permutes_with_the_axes(scheme):
    # relabelling the coordinate axes of the coefficient relabels A_hom:
    # A(a o P) = P^T A(a) P; an axis treated differently from the others (a
    # wrong offset, sign or corner bit on one axis) in the loads, the
    # stiffness or either A_hom form breaks this
    n = 8
    coef = np.exp(np.random.default_rng(12).normal(0.0, 0.8, size=(n, n, n)))
    ref = oracle.solve_coef3(coef, 2, 4, 2.0, scheme, tol=1e-13)
    for perm in ((1, 0, 2), (2, 1, 0), (1, 2, 0)):
        r = oracle.solve_coef3(np.ascontiguousarray(coef.transpose(perm)), 2, 4, 2.0, scheme,
                               tol=1e-13)
        P = np.eye(3)[list(perm)]
        for form in ("A_energy", "A_flux"):
            np.testing.assert_allclose(r[form], P @ ref[form] @ P.T, atol=1e-11)


def test_a_hom3_energy_equals_flux_at_convergence():
    # at the discrete solution v_j^T E v_i = int a d_j(x_i + phi_i) summed over
    # cells (the Galerkin orthogonality of the corrector), so both forms agree
    # to the solver tolerance, and the energy form is symmetric positive definite
    d = {"L": 2, "m0": 8, "incl_cells": 5, "n_incl": 9, "a_matrix": 1.0, "a_incl": 20.0,
         "seed": 9, "index": 2}
    r = oracle.solve_realization3(d, tol=1e-13)
    A, F = r["A_energy"], r["A_flux"]
    np.testing.assert_allclose(A, A.T, atol=1e-13)
    assert np.linalg.eigvalsh(A)[0] > 0.0
    np.testing.assert_allclose(F, A, atol=1e-9 * np.abs(A).max())


def test_statistics3_match_numpy():
    g = np.random.default_rng(8)
    A = g.standard_normal((40, 3, 3))
    A = 0.5 * (A + A.transpose(0, 2, 1))
    L = 8
    s = oracle.statistics3(A, L)
    flat = A.reshape(40, 9)
    np.testing.assert_allclose(s["mean"].ravel(), flat.mean(axis=0), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(s["Q"], L ** 3 * np.cov(flat, rowvar=False, ddof=1), rtol=1e-12,
                               atol=1e-13)
    np.testing.assert_allclose(s["var"].ravel(), flat.var(axis=0, ddof=1), rtol=1e-12)
    # symmetric A: the rows and columns of a_ij and a_ji coincide
    Q = s["Q"]
    for i, j in ((0, 1), (0, 2), (1, 2)):
        np.testing.assert_allclose(Q[3 * i + j], Q[3 * j + i], atol=1e-12)


@pytest.mark.parametrize("scheme", [oracle.SCHEME_CONSISTENT, oracle.SCHEME_LUMPED])
def test_rhs3_equals_the_row_sum_closed_form(scheme):
    # the rows of M1 sum to h/2 (both schemes) and those of K1 to 0, so only
    # the K1 term along axis i survives in E xi_i and
    #   f_i(node) = (h^2/4) (sum of the 4 cells above along i - the 4 below)
    n, h = 6, 0.3
    a = np.random.default_rng(13).uniform(0.5, 4.0, size=(n, n, n))
    f = oracle.rhs3(a, h, scheme)
    ref = np.zeros_like(f)
    for ax in range(3):
        above = a                                   # cells whose lower corner is the node
        below = np.roll(a, 1, axis=ax)              # the cells one step down along ax
        s_above = sum(np.roll(np.roll(above, o1, axis=(ax + 1) % 3), o2, axis=(ax + 2) % 3)
                      for o1 in (0, 1) for o2 in (0, 1))
        s_below = sum(np.roll(np.roll(below, o1, axis=(ax + 1) % 3), o2, axis=(ax + 2) % 3)
                      for o1 in (0, 1) for o2 in (0, 1))
        ref[ax] = 0.25 * h * h * (s_above - s_below)
    np.testing.assert_allclose(f, ref, atol=1e-14 * np.abs(ref).max())


# ------------------------------------------- statistical identities (Sec. 4) --
def test_ensemble_isotropy_and_zero_mean_off_diagonal():
    # the inclusion law is invariant under swapping the axes and under
    # reflections, so E a_11 = E a_22 and E a_12 = 0; the Q entries of
    # Eq. "quartic" inherit the swap symmetry: Q_1111 = Q_2222 (sampling error)
    ds = [workloads.realization(4, 4, 10.0, 17, k) for k in range(240)]
    A, _, _ = oracle.solve_batch(ds, tol=1e-10)
    a11, a22, a12 = A[:, 0, 0], A[:, 1, 1], A[:, 0, 1]
    se = lambda x: x.std(ddof=1) / np.sqrt(len(x))
    assert abs(a11.mean() - a22.mean()) < 4 * se(a11 - a22)
    assert abs(a12.mean()) < 4 * se(a12)
    s = oracle.statistics(A, 4.0)
    Q = s["Q"]
    # var(a11) = var(a22) within the sampling error of a variance (~sqrt(2/N))
    assert abs(Q[0, 0] - Q[3, 3]) < 4 * np.sqrt(2.0 / len(A)) * max(Q[0, 0], Q[3, 3])


def test_ensemble_isotropy3():
    ds = [{"L": 2, "m0": 4, "incl_cells": 4, "n_incl": 6, "a_matrix": 1.0, "a_incl": 8.0,
           "seed": 23, "index": k} for k in range(120)]
    A = np.array([oracle.solve_realization3(d, tol=1e-10, want_u=False)["A_energy"] for d in ds])
    se = lambda x: x.std(ddof=1) / np.sqrt(len(x))
    diag = [A[:, i, i] for i in range(3)]
    for i in range(3):
        for j in range(i + 1, 3):
            assert abs(diag[i].mean() - diag[j].mean()) < 4 * se(diag[i] - diag[j])
            assert abs(A[:, i, j].mean()) < 4 * se(A[:, i, j])
