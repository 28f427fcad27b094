"""librve loads and exports every symbol include/rve.h declares; host-only
argument validation (no GPU needed: these calls launch nothing)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rve.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(rve3?_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def librve():
    from paper_1903_12227_gb300 import build, rve
    build.build()
    return rve.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("rve_gen_field", "rve_solve_correctors", "rve_a_hom", "rve_a_hom_backward",
                     "rve_workspace_size", "rve_status_string", "rve3_solve_correctors",
                     "rve3_a_hom"):
        assert required in names


def test_library_exports_every_declared_symbol(librve):
    for name in _declared_functions():
        assert hasattr(librve, name), f"librve.so does not export {name}"


def test_struct_sizes_match_header(librve):
    from paper_1903_12227_gb300 import rve
    assert ctypes.sizeof(rve.Realization) == 48
    assert ctypes.sizeof(rve.SolveInfo) == 40
    assert ctypes.sizeof(rve.SolveOpts) == 64
    from paper_1903_12227_gb300 import rve3
    assert ctypes.sizeof(rve3.Solve3Opts) == 40
    assert ctypes.sizeof(rve3.Solve3Info) == 48


def test_host_validation_without_gpu(librve):
    from paper_1903_12227_gb300 import rve, workloads
    ok = rve.Batch([workloads.realization(4, 8, 10.0, 0, 0)])
    assert librve.rve_nodes(ok.ptr, 1) == 32 * 32
    assert librve.rve_mask_words(ok.ptr, 1) == 32
    assert librve.rve_workspace_size(ok.ptr, 1, None) > 0
    # n not a power of two, n too small, non-positive coefficient
    for bad in (workloads.realization(3, 16, 10.0, 0, 0), workloads.realization(1, 8, 10.0, 0, 0),
                dict(workloads.realization(4, 8, 10.0, 0, 0), a_matrix=0.0),
                dict(workloads.realization(4, 8, 10.0, 0, 0), incl_cells=64)):
        b = rve.Batch([bad])
        assert librve.rve_workspace_size(b.ptr, 1, None) == 0
        assert librve.rve_gen_field(b.ptr, 1, None, None) == rve.RVE_EINVAL
    assert librve.rve_gen_field(ok.ptr, 0, None, None) == rve.RVE_EINVAL
    opts = rve.make_opts(precision=rve.MIXED, path=rve.PATH_PLAIN)
    assert librve.rve_workspace_size(ok.ptr, 1, ctypes.byref(opts)) == 0
    assert b"RVE_OK" in librve.rve_status_string(0)


def test_host_validation_3d_without_gpu(librve):
    from paper_1903_12227_gb300 import rve, rve3, workloads
    L3 = rve3.lib()
    ds = [workloads.realization3(4, 8, 10.0, 0, 0), workloads.realization3(2, 32, 10.0, 0, 1),
          workloads.realization3(16, 16, 10.0, 0, 2)]
    b = rve3.Batch3(ds)
    assert L3.rve3_nodes(b.ptr, 3) == 32 ** 3 + 64 ** 3 + 256 ** 3
    # seven pair vectors of 16 bytes per node dominate the workspace
    assert L3.rve3_workspace_size(b.ptr, 3) >= 7 * 16 * (32 ** 3 + 64 ** 3 + 256 ** 3)
    for bad in (workloads.realization3(32, 16, 10.0, 0, 0),             # n = 512 > 256
                workloads.realization3(2, 8, 10.0, 0, 0),               # n = 16 < 32
                workloads.realization3(3, 16, 10.0, 0, 0),              # n = 48
                dict(workloads.realization3(4, 8, 10.0, 0, 0), a_incl=float("nan")),
                dict(workloads.realization3(4, 8, 10.0, 0, 0), incl_cells=33)):
        bb = rve3.Batch3([bad])
        assert L3.rve3_nodes(bb.ptr, 1) == -1
        assert L3.rve3_workspace_size(bb.ptr, 1) == 0
        assert L3.rve3_gen_field(bb.ptr, 1, None, None) == rve.RVE_EINVAL
    assert L3.rve3_workspace_size(b.ptr, 0) == 0
    # missing pointers are rejected before any launch
    ws = ctypes.c_void_p(None)
    assert L3.rve3_solve_correctors(b.ptr, 3, None, None, None, None, None, ws, 0, None) == rve.RVE_EINVAL
    bad_opts = rve3.make_opts3(scheme=7)
    assert L3.rve3_solve_correctors(b.ptr, 3, None, None, ctypes.byref(bad_opts), None, None, ws, 0,
                                    None) == rve.RVE_EINVAL
    bad_prec = rve3.make_opts3(precision=5)
    assert L3.rve3_solve_correctors(b.ptr, 3, None, None, ctypes.byref(bad_prec), None, None, ws, 0,
                                    None) == rve.RVE_EINVAL


def test_solve3_option_validation_without_gpu(librve):
    # every check below returns before the first CUDA call: the pointers are
    # never dereferenced on the host
    from paper_1903_12227_gb300 import rve, rve3, workloads
    L3 = rve3.lib()
    b = rve3.Batch3([workloads.realization3(4, 8, 10.0, 0, 0)])
    fake = ctypes.c_void_p(256)
    need = L3.rve3_workspace_size(b.ptr, 1)

    def call(opts, ws_bytes=need):
        return L3.rve3_solve_correctors(b.ptr, 1, fake, None, ctypes.byref(opts), fake, fake, fake,
                                        ws_bytes, None)

    for bad in (rve3.make_opts3(delta=-1.0), rve3.make_opts3(delta=float("inf")),
                rve3.make_opts3(tol=2.0), rve3.make_opts3(inner_tol=1.5),
                rve3.make_opts3(precision=7), rve3.make_opts3(scheme=-1)):
        assert call(bad) == rve.RVE_EINVAL
    assert call(rve3.make_opts3(precision=rve.MIXED), ws_bytes=need - 1) == rve.RVE_ENOMEM
    # the other 3D entry points check their workspace the same way
    assert L3.rve3_rhs(b.ptr, 1, fake, None, 0, fake, fake, need - 1, None) == rve.RVE_ENOMEM
    assert L3.rve3_rhs(b.ptr, 1, fake, None, 5, fake, fake, need, None) == rve.RVE_EINVAL
    assert L3.rve3_apply_stiffness(b.ptr, 1, fake, None, 0, fake, fake, fake, need, None) == rve.RVE_EINVAL
    assert L3.rve3_apply_precond(b.ptr, 1, -0.5, fake, fake, fake, need, None) == rve.RVE_EINVAL
    assert L3.rve3_a_hom(b.ptr, 1, None, None, 0, fake, fake, None, fake, need, None) == rve.RVE_EINVAL


def test_misaligned_workspace_rejected_without_gpu(librve):
    # a workspace must start on a 256-byte boundary; the check precedes the
    # first CUDA call, so fake device pointers are never dereferenced
    from paper_1903_12227_gb300 import rve, rve3, workloads
    b = rve.Batch([workloads.realization(4, 8, 10.0, 0, 0)])
    opts = rve.make_opts(precision=rve.MIXED)
    need = librve.rve_workspace_size(b.ptr, 1, ctypes.byref(opts))
    fake, mis = ctypes.c_void_p(256), ctypes.c_void_p(256 + 16)
    assert librve.rve_solve_correctors(b.ptr, 1, fake, None, ctypes.byref(opts), fake, fake, mis,
                                       need, None) == rve.RVE_EINVAL
    assert librve.rve_solve_correctors(b.ptr, 1, fake, None, ctypes.byref(opts), fake, fake, fake,
                                       need - 1, None) == rve.RVE_ENOMEM
    assert librve.rve_a_hom(b.ptr, 1, fake, None, 0, rve.MIXED, fake, fake, None, None, mis, need,
                            None) == rve.RVE_EINVAL
    L3 = rve3.lib()
    b3 = rve3.Batch3([workloads.realization3(4, 8, 10.0, 0, 0)])
    need3 = L3.rve3_workspace_size(b3.ptr, 1)
    o3 = rve3.make_opts3(precision=rve.MIXED)
    assert L3.rve3_solve_correctors(b3.ptr, 1, fake, None, ctypes.byref(o3), fake, fake, mis,
                                    need3, None) == rve.RVE_EINVAL


def test_statistics3_host_matches_oracle(librve):
    import numpy as np

    import oracle
    from paper_1903_12227_gb300 import rve, rve3
    g = np.random.default_rng(5)
    A = 3.0 + 0.1 * g.standard_normal((64, 3, 3))
    s = rve3.statistics(A, 4.0)
    o = oracle.statistics3(A, 4.0)
    for k in ("mean", "var", "Q"):
        np.testing.assert_allclose(s[k], o[k], rtol=1e-13, atol=1e-16)
    with pytest.raises(rve.RveError):
        rve3.statistics(A[:1], 4.0)


def test_uneven_batch_sizes_add_up(librve):
    from paper_1903_12227_gb300 import rve, workloads
    ds = workloads.config_batch("uneven_4096", seed=3, count=40)
    b = rve.Batch(ds)
    assert librve.rve_nodes(b.ptr, b.count) == sum((d["L"] * d["m0"]) ** 2 for d in ds)


def test_tuner_table_save_load_roundtrip(librve, tmp_path):
    # host-only: the tuner table is a process-wide map written/read as text
    from paper_1903_12227_gb300 import rve
    rve.tuner_clear()
    assert rve.tuner_lookup(512, rve.MIXED, False) is None
    path = tmp_path / "tune.txt"
    path.write_text("# n precision persistent tile_rows block_threads\n512 1 0 4 512\n64 0 1 8 256\n")
    rve.tuner_load(str(path))
    assert rve.tuner_lookup(512, rve.MIXED, False) == (4, 512)
    assert rve.tuner_lookup(64, rve.FP64, True) == (8, 256)
    out = tmp_path / "out.txt"
    rve.tuner_save(str(out))
    rve.tuner_clear()
    rve.tuner_load(str(out))
    assert rve.tuner_lookup(512, rve.MIXED, False) == (4, 512)
    # the tuned shape changes the plan (tile counts, hence the partial-sum arrays)
    from paper_1903_12227_gb300 import workloads
    b = rve.Batch([workloads.realization(32, 16, 10.0, 0, 0)])
    tuned = rve.workspace_size(b, rve.make_opts(precision=rve.MIXED))
    rve.tuner_clear()
    default = rve.workspace_size(b, rve.make_opts(precision=rve.MIXED))
    assert tuned != default
