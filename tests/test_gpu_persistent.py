"""GPU: the persistent single-launch path over uneven sizes, plans captured in
a CUDA graph (one persistent launch, or the fused kernels in a conditional
while node), the autotuner, and the bounded grid-barrier wait."""
import numpy as np
import pytest
import torch

import oracle
from paper_1903_12227_gb300 import rve, workloads

pytestmark = pytest.mark.gpu
CUDA = torch.device("cuda", 0)


def _rel_err_A(A, ref):
    return np.abs(np.asarray(A) - ref).max() / max(abs(ref[0, 0]), abs(ref[1, 1]))


# uneven sizes 32..512 and both contrasts (the oracle's n=512 solve is the slow one:
# keep one of those)
UNEVEN = ([d for d in workloads.config_batch("uneven_4096", seed=5, count=40) if d["L"] <= 32][:9]
          + [workloads.realization(4, 8, 100.0, 5, 99), workloads.realization(32, 16, 10.0, 5, 98)])


@pytest.mark.parametrize("precision,bound", [(rve.MIXED, 1e-7), (rve.FP64, 1e-10)])
def test_persistent_uneven_batch_matches_oracle(precision, bound):
    ds = UNEVEN
    opts = rve.make_opts(precision=precision, path=rve.PATH_PERSISTENT,
                         tol=1e-10 if precision == rve.MIXED else 1e-12)
    mask = rve.gen_field(ds, device=CUDA)
    u, info = rve.solve(ds, mask=mask, opts=opts)
    A = rve.a_hom(ds, u, mask=mask).cpu().numpy()
    inf = rve.info_to_dicts(info, len(ds))
    for k, d in enumerate(ds):
        assert inf[k]["status"] == rve.RVE_OK, inf[k]
        ref = oracle.solve_realization(d, tol=1e-12, want_u=False)
        assert _rel_err_A(A[k], ref["A_energy"]) < bound


def test_plan_graph_replays_and_matches_fused_path():
    ds = UNEVEN[:8]
    plan = rve.Plan(ds, rve.make_opts(precision=rve.MIXED, path=rve.PATH_PERSISTENT), device=CUDA)
    A1, info1 = plan.execute()
    A1 = A1.cpu().numpy().copy()
    A2, info2 = plan.execute()          # graph relaunch
    A2 = A2.cpu().numpy()
    np.testing.assert_array_equal(A1, A2)
    assert all(d["status"] == rve.RVE_OK for d in rve.info_to_dicts(info2, len(ds)))
    mask = rve.gen_field(ds, device=CUDA)
    u, _ = rve.solve(ds, mask=mask, opts=rve.make_opts(precision=rve.MIXED))
    Af = rve.a_hom(ds, u, mask=mask).cpu().numpy()
    for k in range(len(ds)):
        assert _rel_err_A(A1[k], Af[k]) < 1e-9
    plan.close()


@pytest.mark.parametrize("precision", [rve.MIXED, rve.FP64])
def test_plan_graph_loop_equals_fused_path(precision):
    """A plan on the fused path runs the fused kernels inside a conditional
    while node of the graph (no host polling): the same kernels on the same
    data, so the same bits as a fused solve; the graph relaunches; and the
    results match the oracle."""
    ds = UNEVEN[:8]
    opts = rve.make_opts(precision=precision, path=rve.PATH_FUSED,
                         tol=1e-10 if precision == rve.MIXED else 1e-12)
    plan = rve.Plan(ds, opts, device=CUDA)
    A1, info1 = plan.execute()
    A1 = A1.cpu().numpy().copy()
    inf1 = rve.info_to_dicts(info1, len(ds))
    A2, info2 = plan.execute()          # graph relaunch
    np.testing.assert_array_equal(A1, A2.cpu().numpy())
    assert all(d["status"] == rve.RVE_OK for d in rve.info_to_dicts(info2, len(ds)))
    mask = rve.gen_field(ds, device=CUDA)
    u, info = rve.solve(ds, mask=mask, opts=opts)
    Af = rve.a_hom(ds, u, mask=mask, precision=precision).cpu().numpy()
    np.testing.assert_array_equal(A1, Af)
    assert [d["iters"] for d in inf1] == [d["iters"] for d in rve.info_to_dicts(info, len(ds))]
    for k in (0, len(ds) - 1):
        ref = oracle.solve_realization(ds[k], tol=1e-12, want_u=False)
        assert _rel_err_A(A1[k], ref["A_energy"]) < (1e-7 if precision == rve.MIXED else 1e-10)
    plan.close()


def test_autotuner_records_shapes_and_solves_still_match():
    rve.tuner_clear()
    ds = [workloads.realization(8, 8, 10.0, 3, k) for k in range(4)] + \
         [workloads.realization(32, 16, 10.0, 3, 10 + k) for k in range(2)]
    rve.autotune(ds, rve.make_opts(precision=rve.MIXED), device=CUDA)
    for n in (64, 512):
        assert rve.tuner_lookup(n, rve.MIXED, False) is not None
    mask = rve.gen_field(ds, device=CUDA)
    u, info = rve.solve(ds, mask=mask, opts=rve.make_opts(precision=rve.MIXED))
    A = rve.a_hom(ds, u, mask=mask).cpu().numpy()
    for k, d in enumerate(ds):
        ref = oracle.solve_realization(d, tol=1e-12, want_u=False)
        assert _rel_err_A(A[k], ref["A_energy"]) < 1e-7
    rve.tuner_clear()


def test_grid_barrier_wait_is_bounded():
    # a 1 us bound on each grid-barrier wait runs out at once: the launch
    # must end by itself and report the time-out, and the GPU stays usable
    ds = [workloads.realization(32, 16, 10.0, 7, k) for k in range(8)]
    mask = rve.gen_field(ds, device=CUDA)
    opts = rve.make_opts(precision=rve.MIXED, path=rve.PATH_PERSISTENT, timeout_us=1)
    u, info = rve.solve(ds, mask=mask, opts=opts)
    torch.cuda.synchronize()
    st = {d["status"] for d in rve.info_to_dicts(info, len(ds))}
    assert rve.RVE_ETIMEOUT in st
    # the device still works: a normal solve afterwards succeeds
    u, info = rve.solve(ds[:2], mask=rve.gen_field(ds[:2], device=CUDA),
                        opts=rve.make_opts(precision=rve.MIXED, path=rve.PATH_PERSISTENT))
    assert all(d["status"] == rve.RVE_OK for d in rve.info_to_dicts(info, 2))
