"""rve_a_hom_noalloc: the homogenized-matrix reduction for callers that cannot
allocate device memory (programs whose device memory is all owned by their
own pool allocator, or latency-critical loops that cannot afford cudaMalloc
/ cudaFree).  It keeps its scratch in a fixed library-owned array instead of
a workspace.  Checked through the C ABI against the workspace entry point
rve_a_hom (its double-word form, precision RVE_MIXED), on two calls in a row
with different inputs (the second call must not see the first call's
leftovers), from the bitmask and from an explicit array of cell values.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1903_12227_gb300 import rve, workloads

pytestmark = pytest.mark.gpu

CUDA = torch.device("cuda", 0)


def _noalloc_fn():
    f = rve.lib().rve_a_hom_noalloc
    vp = ctypes.c_void_p
    f.restype = ctypes.c_int32
    f.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.c_int32, vp, vp, vp, vp]
    return f


def _call_noalloc(batch, mask, u, scheme, coef=None):
    b = rve.as_batch(batch)
    A = torch.full((b.count, 4), float("nan"), dtype=torch.float64, device=CUDA)
    Af = torch.full((b.count, 4), float("nan"), dtype=torch.float64, device=CUDA)
    st = _noalloc_fn()(b.ptr, b.count, rve._ptr(mask), rve._ptr(coef), scheme, rve._ptr(u),
                       rve._ptr(A), rve._ptr(Af), rve._stream())
    return st, A.view(b.count, 2, 2), Af.view(b.count, 2, 2)


@pytest.mark.parametrize("scheme", [rve.CONSISTENT, rve.LUMPED])
def test_noalloc_a_hom_matches_workspace_entry_point(scheme):
    calls = [
        [workloads.realization(4, 8, 10.0, 11, k) for k in range(3)] +
        [workloads.realization(32, 16, 10.0, 11, 3)],                        # 32^2 .. 512^2
        [workloads.realization(16, 8, 100.0, 12, k) for k in range(2)] +
        [workloads.realization(8, 4, 10.0, 12, 2)],                          # different sizes
    ]
    for ds in calls:                                                         # two calls in a row
        mask = rve.gen_field(ds, device=CUDA)
        u, _ = rve.solve(ds, mask=mask, opts=rve.make_opts(scheme=scheme, precision=rve.MIXED))
        A_ref, Af_ref = rve.a_hom(ds, u, mask=mask, scheme=scheme, want_flux=True,
                                  precision=rve.MIXED)
        st, A, Af = _call_noalloc(ds, mask, u, scheme)
        torch.cuda.synchronize()
        assert st == rve.RVE_OK, rve.lib().rve_status_string(st)
        scale = torch.maximum(A_ref[:, 0, 0].abs(), A_ref[:, 1, 1].abs()).view(-1, 1, 1)
        assert ((A - A_ref).abs() / scale).max().item() < 1e-12
        assert ((Af - Af_ref).abs() / scale).max().item() < 1e-12


@pytest.mark.parametrize("scheme", [rve.CONSISTENT, rve.LUMPED])
def test_noalloc_a_hom_general_cell_values(scheme):
    """The explicit coefficient-array branch: general positive cell values
    (no mask), two calls in a row with different sizes."""
    g = np.random.default_rng(5)
    calls = [[workloads.realization(8, 8, 10.0, 21, k) for k in range(2)],      # 64^2
             [workloads.realization(4, 8, 10.0, 22, 0),
              workloads.realization(16, 16, 10.0, 22, 1)]]                      # 32^2, 256^2
    for ds in calls:
        b = rve.as_batch(ds)
        coef = torch.tensor(g.uniform(0.5, 20.0, size=b.nodes), device=CUDA)
        u, info = rve.solve(ds, coef=coef,
                            opts=rve.make_opts(scheme=scheme, precision=rve.MIXED))
        assert all(x["status"] == rve.RVE_OK for x in rve.info_to_dicts(info, b.count))
        A_ref, Af_ref = rve.a_hom(ds, u, coef=coef, scheme=scheme, want_flux=True,
                                  precision=rve.MIXED)
        st, A, Af = _call_noalloc(ds, None, u, scheme, coef=coef)
        torch.cuda.synchronize()
        assert st == rve.RVE_OK, rve.lib().rve_status_string(st)
        scale = torch.maximum(A_ref[:, 0, 0].abs(), A_ref[:, 1, 1].abs()).view(-1, 1, 1)
        assert ((A - A_ref).abs() / scale).max().item() < 1e-12
        assert ((Af - Af_ref).abs() / scale).max().item() < 1e-12


def test_noalloc_rejects_requests_above_its_scratch():
    # 65 realizations of 512^2 nodes = 17,039,360 nodes > 2^24
    ds = [workloads.realization(32, 16, 10.0, 0, k) for k in range(65)]
    b = rve.Batch(ds)
    dummy = torch.zeros(4, dtype=torch.float64, device=CUDA)
    st = _noalloc_fn()(b.ptr, b.count, rve._ptr(dummy), None, 0, rve._ptr(dummy),
                       rve._ptr(dummy), None, rve._stream())
    assert st == rve.RVE_ESCRATCH
    assert b"RVE_ESCRATCH" in rve.lib().rve_status_string(st)
