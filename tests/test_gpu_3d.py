"""GPU parity of the 3D extension (cubes on [0,L)^3, trilinear Q1, three
correctors, 3x3 A_hom) through the C ABI against the FP64 CPU oracle.

Tolerances as in 2D: the field bit-exact; the loads, the stiffness, the
preconditioner and A_hom of a given corrector 1e-12 relative (rounding order
only); A_hom of the solve 1e-10 relative to max |A_ii| (both solves stop at
a 1e-12 relative residual); the correctors themselves 1e-8 relative.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from paper_1903_12227_gb300 import rve, rve3, workloads

pytestmark = pytest.mark.gpu

CUDA = torch.device("cuda", 0)
SCHEMES = [rve.CONSISTENT, rve.LUMPED]


def _coef_np(d, mask):
    return np.where(mask, d["a_incl"], d["a_matrix"]).astype(np.float64)


def _nodes3(v):   # oracle [3, n, n, n] -> [n^3, 3]
    return np.stack([v[i].ravel() for i in range(3)], axis=1)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _rel_A(A, ref):
    return np.abs(np.asarray(A) - ref).max() / max(abs(ref[0, 0]), abs(ref[1, 1]), abs(ref[2, 2]))


def _split(vals, ds):
    out, o = [], 0
    for d in ds:
        n = d["L"] * d["m0"]
        out.append(vals[o:o + n ** 3])
        o += n ** 3
    return out


# ------------------------------------------------------------------ field --
FIELD_CASES = [
    [workloads.realization3(4, 8, 10.0, 0, 0, side_units=0.5)],                  # 32^3
    [workloads.realization3(2, 32, 10.0, 3, k) for k in range(2)],              # 64^3, s = 32
    [workloads.realization3(4, 8, 10.0, 1, 0), workloads.realization3(8, 16, 100.0, 1, 1),
     workloads.realization3(2, 16, 10.0, 1, 2)],                                # 32, 128, 32
    [dict(workloads.realization3(4, 8, 10.0, 0, 0), n_incl=0)],                  # empty
    [dict(workloads.realization3(4, 8, 10.0, 0, 0), incl_cells=32, n_incl=1)],   # full cover
    [workloads.realization3(16, 16, 10.0, 2, 5)],                               # 256^3, 2867 cubes
]


@pytest.mark.parametrize("case", range(len(FIELD_CASES)))
def test_gen_field3_bit_exact(case):
    ds = FIELD_CASES[case]
    mask = rve3.gen_field(ds, device=CUDA)
    torch.cuda.synchronize()
    for d, m in zip(ds, _split(mask.cpu().numpy(), ds)):
        n = d["L"] * d["m0"]
        np.testing.assert_array_equal(m.reshape(n, n, n) != 0, oracle.gen_field3(d) != 0)


# --------------------------------------------------- loads and stiffness --
OP_CASES = [
    [workloads.realization3(4, 8, 10.0, 4, 0, side_units=0.5)],                          # 32^3
    [workloads.realization3(2, 16, 10.0, 4, 1), workloads.realization3(4, 16, 100.0, 4, 2)],   # 32 + 64
]


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("case", range(len(OP_CASES)))
@pytest.mark.parametrize("general", [False, True])
def test_rhs3_and_stiffness3(case, scheme, general):
    ds = OP_CASES[case]
    rng = np.random.default_rng(11 + case)
    mask = rve3.gen_field(ds, device=CUDA)
    masks = _split(mask.cpu().numpy(), ds)
    coefs = []
    for d, m in zip(ds, masks):
        n = d["L"] * d["m0"]
        c = rng.uniform(0.5, 3.0, size=n ** 3) if general else _coef_np(d, m != 0)
        coefs.append(c.reshape(n, n, n))
    coef_t = torch.tensor(np.concatenate([c.ravel() for c in coefs]), device=CUDA) if general else None
    mask_t = None if general else mask
    f = rve3.rhs(ds, mask=mask_t, coef=coef_t, scheme=scheme).cpu().numpy()
    x = rng.standard_normal((sum(d["L"] ** 3 * d["m0"] ** 3 for d in ds), 3))
    y = rve3.apply_stiffness(ds, torch.tensor(x, device=CUDA), mask=mask_t, coef=coef_t,
                             scheme=scheme).cpu().numpy()
    for d, c, fb, xb, yb in zip(ds, coefs, _split(f, ds), _split(x, ds), _split(y, ds)):
        h = 1.0 / d["m0"]
        ref_f = _nodes3(oracle.rhs3(c, h, scheme))
        assert _rel(fb, ref_f) < 1e-12
        rowptr, colidx, vals = oracle.assemble3(c, h, scheme)
        N = c.size
        A = sp.csr_matrix((vals, colidx, rowptr), shape=(N, N))
        assert _rel(yb, A @ xb) < 1e-12


# --------------------------------------------------------- preconditioner --
@pytest.mark.parametrize("delta", [0.0, 0.3])
@pytest.mark.parametrize("sizes", [[(4, 8)], [(2, 16), (4, 16), (8, 16)]])   # 32; 32, 64, 128
def test_precond3(sizes, delta):
    ds = [workloads.realization3(L, m0, 10.0, 6, k) for k, (L, m0) in enumerate(sizes)]
    rng = np.random.default_rng(5)
    N = sum((L * m0) ** 3 for L, m0 in sizes)
    x = rng.standard_normal((N, 3))
    y = rve3.apply_precond(ds, torch.tensor(x, device=CUDA), delta=delta).cpu().numpy()
    for d, xb, yb in zip(ds, _split(x, ds), _split(y, ds)):
        n = d["L"] * d["m0"]
        c0 = 0.5 * (d["a_matrix"] + d["a_incl"])
        for i in range(3):
            ref = oracle.precond3(xb[:, i].reshape(n, n, n).copy(), c0, delta).ravel()
            assert _rel(yb[:, i], ref) < 1e-12


# ------------------------------------------------------- solve and A_hom --
@pytest.mark.parametrize("scheme", SCHEMES)
def test_a_hom3_of_oracle_correctors(scheme):
    d = workloads.realization3(4, 8, 10.0, 8, 0, side_units=0.5)
    ref = oracle.solve_realization3(d, scheme=scheme, tol=1e-12)
    mask = rve3.gen_field([d], device=CUDA)
    u = torch.tensor(_nodes3(ref["u"]), device=CUDA)
    A, Af = rve3.a_hom([d], u, mask=mask, scheme=scheme, want_flux=True)
    assert _rel_A(A[0].cpu().numpy(), ref["A_energy"]) < 1e-12
    assert _rel_A(Af[0].cpu().numpy(), ref["A_flux"]) < 1e-12


SOLVE_CASES = [
    ([workloads.realization3(4, 8, 10.0, 9, 0, side_units=0.5)], rve.CONSISTENT),            # 32^3
    ([workloads.realization3(4, 8, 10.0, 9, 1, side_units=0.5)], rve.LUMPED),
    ([workloads.realization3(2, 16, 100.0, 9, 2), workloads.realization3(4, 16, 10.0, 9, 3)],
     rve.CONSISTENT),                                                                       # 32 + 64
]


@pytest.mark.parametrize("case", range(len(SOLVE_CASES)))
def test_solve3_matches_oracle(case):
    ds, scheme = SOLVE_CASES[case]
    tol = 1e-12
    mask = rve3.gen_field(ds, device=CUDA)
    u, info = rve3.solve(ds, mask=mask, opts=rve3.make_opts3(scheme=scheme, tol=tol))
    A, Af = rve3.a_hom(ds, u, mask=mask, scheme=scheme, want_flux=True)
    infos = rve3.decode_info(info)
    un = u.cpu().numpy()
    for k, (d, ub) in enumerate(zip(ds, _split(un, ds))):
        ref = oracle.solve_realization3(d, scheme=scheme, tol=tol)
        assert infos[k]["status"] == rve.RVE_OK
        assert max(infos[k]["relres"]) <= tol * 1.1
        assert _rel(ub, _nodes3(ref["u"])) < 1e-8
        assert _rel_A(A[k].cpu().numpy(), ref["A_energy"]) < 1e-10
        assert _rel_A(Af[k].cpu().numpy(), ref["A_flux"]) < 1e-10
        # PCG iteration counts agree up to rounding near the stopping test
        for i in range(3):
            assert abs(infos[k]["iters"][i] - ref["iters"][i]) <= 2


def test_solve3_constant_coefficient_closed_form():
    # no cubes: f = 0, u = 0, A = a_matrix I exactly in both forms
    d = dict(workloads.realization3(4, 8, 10.0, 0, 0), n_incl=0, a_matrix=2.5)
    A, infos = rve3.homogenize([d])
    assert infos[0]["status"] == rve.RVE_OK and infos[0]["iters"] == [0, 0, 0]
    np.testing.assert_allclose(A[0].cpu().numpy(), 2.5 * np.eye(3), rtol=0, atol=1e-14)


def test_solve3_with_shift_delta():
    # delta > 0 changes the preconditioner only, not the solution
    d = workloads.realization3(4, 8, 10.0, 12, 0, side_units=0.5)
    mask = rve3.gen_field([d], device=CUDA)
    u0, _ = rve3.solve([d], mask=mask, opts=rve3.make_opts3(tol=1e-12))
    u1, info = rve3.solve([d], mask=mask, opts=rve3.make_opts3(tol=1e-12, delta=0.05))
    assert rve3.decode_info(info)[0]["status"] == rve.RVE_OK
    A0 = rve3.a_hom([d], u0, mask=mask)[0].cpu().numpy()
    A1 = rve3.a_hom([d], u1, mask=mask)[0].cpu().numpy()
    assert _rel_A(A1, A0) < 1e-10


def test_rve3_rejects_bad_sizes():
    d = workloads.realization3(4, 8, 10.0, 0, 0)
    with pytest.raises(rve.RveError):
        rve3.gen_field([dict(d, m0=4)])          # n = 16 < 32
    b = rve3.Batch3([d])
    x = torch.zeros(32 ** 3, 3, dtype=torch.float64, device=CUDA)
    y = torch.empty_like(x)
    small = torch.empty(256, dtype=torch.uint8, device=CUDA)
    st = rve3.lib().rve3_apply_precond(b.ptr, 1, 0.0, rve._ptr(x), rve._ptr(y), rve._ptr(small),
                                       small.numel(), rve._stream())
    assert st == rve.RVE_ENOMEM


def test_solve3_profile_counts_every_kind():
    d = workloads.realization3(4, 8, 10.0, 13, 0, side_units=0.5)
    mask = rve3.gen_field([d], device=CUDA)
    rve.profile_enable(True)
    try:
        rve3.profile_read()
        u, info = rve3.solve([d], mask=mask, opts=rve3.make_opts3(tol=1e-10))
        torch.cuda.synchronize()
        prof = rve3.profile_read()
    finally:
        rve.profile_enable(False)
    iters = rve3.decode_info(info)[0]["iters"]
    # both pairs advance in the same launches: at least as many steps as the
    # slower pair took iterations
    steps = max(iters)
    # four line passes and one z solve per preconditioner application
    assert prof["zsolve"][1] >= steps
    assert prof["lines"][1] == 4 * prof["zsolve"][1]
    assert prof["stiffness"][1] >= steps
    assert all(ms > 0 for ms, cnt in prof.values())


# ------------------------------------------------------- mixed precision --
MIXED_CASES = [
    ([workloads.realization3(4, 8, 10.0, 9, 0, side_units=0.5)], rve.CONSISTENT, 1e-10),
    ([workloads.realization3(4, 8, 10.0, 9, 1, side_units=0.5)], rve.LUMPED, 1e-10),
    ([workloads.realization3(2, 16, 100.0, 9, 2), workloads.realization3(4, 16, 10.0, 9, 3)],
     rve.CONSISTENT, 1e-11),
]


@pytest.mark.parametrize("case", range(len(MIXED_CASES)))
def test_solve3_mixed_matches_oracle(case):
    # FP32 cycles on the FP64 true residual: the same FP64 stopping test, so
    # A_hom agrees with the FP64 oracle to the mixed path's bar (1e-7)
    ds, scheme, tol = MIXED_CASES[case]
    mask = rve3.gen_field(ds, device=CUDA)
    u, info = rve3.solve(ds, mask=mask, opts=rve3.make_opts3(scheme=scheme, tol=tol,
                                                             precision=rve.MIXED))
    A = rve3.a_hom(ds, u, mask=mask, scheme=scheme)
    infos = rve3.decode_info(info)
    for k, d in enumerate(ds):
        ref = oracle.solve_realization3(d, scheme=scheme, tol=1e-12)
        assert infos[k]["status"] == rve.RVE_OK
        assert max(infos[k]["relres"]) <= tol
        assert infos[k]["refinements"] >= 4          # at least two cycles per pair
        assert _rel_A(A[k].cpu().numpy(), ref["A_energy"]) < 1e-7


def test_solve3_general_coefficients_both_precisions():
    d = workloads.realization3(4, 8, 10.0, 14, 0)
    n = 32
    rng = np.random.default_rng(3)
    coef = rng.uniform(0.5, 4.0, size=(n, n, n))
    ct = torch.tensor(coef.ravel(), device=CUDA)
    ref = oracle.solve_coef3(coef, d["L"], d["m0"], c0=2.25, tol=1e-12)
    for prec, bar in ((rve.FP64, 1e-10), (rve.MIXED, 1e-7)):
        u, info = rve3.solve([d], coef=ct, opts=rve3.make_opts3(tol=1e-11, precision=prec))
        assert rve3.decode_info(info)[0]["status"] == rve.RVE_OK
        A = rve3.a_hom([d], u, coef=ct)[0].cpu().numpy()
        assert _rel_A(A, ref["A_energy"]) < bar


@pytest.mark.parametrize("scheme", [rve.CONSISTENT, rve.LUMPED])
def test_mixed3_integer_cells_same_bits_as_double_words(scheme):
    """With integer cell values (1 and the contrast) the mixed true residual
    forms its cell weights as exact floats instead of double words: the same
    values, so the same solve, bit for bit, as through the explicit
    coefficient input, which always takes the double-word weights."""
    ds = [workloads.realization3(4, 8, 10.0, 21, k) for k in range(2)]
    mask = rve3.gen_field(ds, device=CUDA)
    coef = torch.where(mask.bool(), torch.tensor(ds[0]["a_incl"], dtype=torch.float64, device=CUDA),
                       torch.tensor(ds[0]["a_matrix"], dtype=torch.float64, device=CUDA))
    opts = rve3.make_opts3(tol=1e-10, precision=rve.MIXED, scheme=scheme)
    u1, i1 = rve3.solve(ds, mask=mask, opts=opts)
    u2, i2 = rve3.solve(ds, coef=coef, opts=opts)
    np.testing.assert_array_equal(u1.cpu().numpy(), u2.cpu().numpy())
    d1, d2 = rve3.decode_info(i1), rve3.decode_info(i2)
    assert [x["iters"] for x in d1] == [x["iters"] for x in d2]
    assert all(x["status"] == rve.RVE_OK for x in d1)


def test_solve3_mixed_constant_coefficient():
    d = dict(workloads.realization3(4, 8, 10.0, 0, 0), n_incl=0, a_matrix=2.5)
    A, infos = rve3.homogenize([d], precision=rve.MIXED)
    assert infos[0]["status"] == rve.RVE_OK and infos[0]["iters"] == [0, 0, 0]
    np.testing.assert_allclose(A[0].cpu().numpy(), 2.5 * np.eye(3), rtol=0, atol=1e-14)


@pytest.mark.parametrize("prec", [rve.FP64, rve.MIXED])
def test_solve3_batch_matches_single_solves(prec):
    # units of a batch are independent: the batched launches reproduce each
    # realization's lone solve exactly, whatever the mix of sizes
    ds = [workloads.realization3(4, 8, 10.0, 21, 0, side_units=0.5),
          workloads.realization3(4, 16, 10.0, 21, 1),
          workloads.realization3(2, 16, 100.0, 21, 2),
          workloads.realization3(4, 8, 10.0, 21, 3, side_units=0.5)]
    opts = rve3.make_opts3(tol=1e-10, precision=prec)
    mask = rve3.gen_field(ds, device=CUDA)
    u, info = rve3.solve(ds, mask=mask, opts=opts)
    A = rve3.a_hom(ds, u, mask=mask).cpu().numpy()
    infos = rve3.decode_info(info)
    for k, d in enumerate(ds):
        m1 = rve3.gen_field([d], device=CUDA)
        u1, i1 = rve3.solve([d], mask=m1, opts=opts)
        A1 = rve3.a_hom([d], u1, mask=m1).cpu().numpy()
        assert infos[k]["status"] == rve.RVE_OK
        assert rve3.decode_info(i1)[0]["iters"] == infos[k]["iters"]
        np.testing.assert_array_equal(A[k], A1[0])


def test_a_hom3_gpu_permutes_with_the_axes():
    # the GPU path on its own: relabelling the axes of the cell values
    # relabels A_hom (x lines, y lines and z solves, and the three stencil
    # axes, all enter differently)
    d = workloads.realization3(2, 16, 10.0, 15, 0)
    n = 32
    coef = np.exp(np.random.default_rng(21).normal(0.0, 0.7, size=(n, n, n)))
    opts = rve3.make_opts3(tol=1e-12)

    def A_of(c):
        ct = torch.tensor(np.ascontiguousarray(c).ravel(), device=CUDA)
        u, info = rve3.solve([d], coef=ct, opts=opts)
        assert rve3.decode_info(info)[0]["status"] == rve.RVE_OK
        return rve3.a_hom([d], u, coef=ct)[0].cpu().numpy()

    A = A_of(coef)
    for perm in ((1, 0, 2), (2, 1, 0), (1, 2, 0)):
        P = np.eye(3)[list(perm)]
        assert _rel_A(A_of(coef.transpose(perm)), P @ A @ P.T) < 1e-10
