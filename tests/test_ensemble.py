"""Ensemble layer on CPU: statistics against the oracle's and numpy's,
sharding over gloo ranks (world size 2) with an index-ordered merge that is
bit-identical to a single-process run, and checkpoint/resume with a failure
injected on the host."""
import json
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1903_12227_gb300 import ensemble, rve


def _fake_A(indices):
    # deterministic stand-in for solved realizations (symmetric 2x2)
    out = []
    for k in indices:
        r = np.random.default_rng(int(k) + 17).standard_normal(3)
        out.append([[2.9 + 0.05 * r[0], 0.01 * r[1]], [0.01 * r[1], 2.9 + 0.05 * r[2]]])
    return np.array(out)


@pytest.fixture(scope="module")
def librve():
    from paper_1903_12227_gb300 import build
    build.build()
    return rve.lib()


def test_statistics_match_oracle_and_numpy(librve):
    A = _fake_A(range(200))
    s = rve.statistics(A, L=32.0)
    o = oracle.statistics(A, 32.0)
    for k in ("mean", "var", "Q"):
        np.testing.assert_allclose(s[k], o[k], rtol=1e-13, atol=1e-16)
    assert abs(s["std12_paper"] - o["std12_paper"]) < 1e-15
    assert abs(s["stddiff_paper"] - o["stddiff_paper"]) < 1e-15
    flat = A.reshape(-1, 4)
    np.testing.assert_allclose(s["Q"], 32.0 ** 2 * np.cov(flat, rowvar=False, ddof=1), rtol=1e-12,
                               atol=1e-16)


def test_shard_ranges_cover_indices_once():
    for total in (0, 1, 7, 1000, 4096):
        for world in (1, 2, 3, 8):
            got = [k for r in range(world) for k in ensemble.shard_range(total, r, world)]
            assert got == list(range(total))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, total, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = list(ensemble.shard_range(total, rank, world))
    merged = ensemble.gather_a_hom(idx, _fake_A(idx), total)
    if rank == 0:
        np.save(out_path, merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_bit_identical(tmp_path):
    total = 37
    out = str(tmp_path / "merged.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), total, out), nprocs=2,
                       start_method="spawn")
    merged = np.load(out)
    single = _fake_A(range(total))
    np.testing.assert_array_equal(merged, single)


def _real_shard_rank(rank, world, port, total, out_path):
    """One rank of a sharded ensemble of real realizations: its contiguous
    index range is solved by the oracle (L = 4, h = 1/8, contrast 10), the
    A_hom gathered to rank 0 and merged in index order."""
    import torch.distributed as dist
    from paper_1903_12227_gb300 import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = list(ensemble.shard_range(total, rank, world))
    ds = [workloads.realization(4, 8, 10.0, 3, k) for k in idx]
    A, _, _ = oracle.solve_batch(ds, tol=1e-12, threads=1) if ds else (np.zeros((0, 2, 2)), 0, 0)
    merged = ensemble.gather_a_hom(idx, A, total)
    if rank == 0:
        np.save(out_path, merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_real_realizations_bit_identical(tmp_path):
    """Each rank solves its shard (the oracle stands in for one GPU per rank);
    the merged A_hom and their statistics equal a single-process run bit for
    bit, because every realization is a pure function of (seed, index)."""
    from paper_1903_12227_gb300 import workloads
    total = 23
    out = str(tmp_path / "merged_real.npy")
    mp.start_processes(_real_shard_rank, args=(2, _free_port(), total, out), nprocs=2,
                       start_method="spawn")
    merged = np.load(out)
    single, _, _ = oracle.solve_batch([workloads.realization(4, 8, 10.0, 3, k)
                                       for k in range(total)], tol=1e-12, threads=1)
    np.testing.assert_array_equal(merged, single)
    s_m, s_s = oracle.statistics(merged, 4.0), oracle.statistics(single, 4.0)
    for k in ("mean", "var", "Q"):
        np.testing.assert_array_equal(s_m[k], s_s[k])


def test_checkpoint_resume_after_injected_failure(tmp_path):
    ck = ensemble.Checkpoint(str(tmp_path / "run.jsonl"))
    calls = []

    def failing_solve(chunk):
        calls.append(list(chunk))
        if len(calls) == 3:
            raise RuntimeError("injected failure")
        return _fake_A(chunk), [{"iters": (5, 5), "status": 0}] * len(chunk)

    with pytest.raises(RuntimeError):
        ensemble.run_ensemble(range(20), failing_solve, batch=4, checkpoint=ck)
    assert sorted(ck.done()) == list(range(8))
    # a torn last line (process killed mid-write) is ignored
    with open(ck.path, "a") as f:
        f.write('{"index": 99, "A": [1, 2')
    calls.clear()

    def ok_solve(chunk):
        calls.append(list(chunk))
        return _fake_A(chunk), [{"iters": (5, 5), "status": 0}] * len(chunk)

    recs = ensemble.run_ensemble(range(20), ok_solve, batch=4, checkpoint=ck)
    assert [k for c in calls for k in c] == list(range(8, 20))   # resumed, nothing redone
    A = ensemble.records_to_array(recs, range(20))
    np.testing.assert_array_equal(A, _fake_A(range(20)))


def test_oracle_thread_count_is_per_call():
    """A one-thread oracle call (the single-thread baseline) leaves later
    calls on the default team: the thread count is a property of the call,
    not of the process.  Results do not depend on the thread count."""
    import os
    from paper_1903_12227_gb300 import workloads
    ds = [workloads.realization(4, 8, 10.0, 5, k) for k in range(4)]
    A_all, _, used_all = oracle.solve_batch(ds, tol=1e-10)
    A_one, _, used_one = oracle.solve_batch(ds[:1], tol=1e-10, threads=1)
    A_again, _, used_again = oracle.solve_batch(ds, tol=1e-10)
    assert used_one == 1
    assert used_again == used_all
    if (os.cpu_count() or 1) > 1 and "OMP_NUM_THREADS" not in os.environ:
        assert used_all > 1
    np.testing.assert_array_equal(A_one[0], A_all[0])
    np.testing.assert_array_equal(A_again, A_all)
