"""Ensembles of realizations: sharding over ranks, index-ordered merge,
checkpoint/resume, and the statistics of Secs. 4.2-4.3 and 5.

Realizations are independent (each is a pure function of (seed, index)), so
a run over N realizations shards the index range contiguously across ranks
with no collective on the data path; results are merged in index order, so
statistics are identical whatever the number of ranks.  Per-realization
records go to an append-only JSONL file; a resumed run skips the indices
already recorded.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Iterable, Sequence

import numpy as np


def shard_range(total: int, rank: int, world: int) -> range:
    """Contiguous block of realization indices owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("invalid shard")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def merge_by_index(parts: Iterable[tuple[Sequence[int], np.ndarray]], total: int) -> np.ndarray:
    """Assemble per-rank (indices, A[k,2,2]) into A[total,2,2] in index order."""
    out = np.full((total, 2, 2), np.nan)
    seen = np.zeros(total, dtype=bool)
    for idx, A in parts:
        idx = np.asarray(idx, dtype=np.int64)
        if seen[idx].any():
            raise ValueError("realization recorded twice")
        out[idx] = np.asarray(A).reshape(-1, 2, 2)
        seen[idx] = True
    if not seen.all():
        raise ValueError(f"{int((~seen).sum())} realizations missing")
    return out


def gather_a_hom(indices: Sequence[int], A: np.ndarray, total: int, group=None) -> np.ndarray | None:
    """torch.distributed gather of every rank's (indices, A) to rank 0, merged
    in index order (None on the other ranks).  Host-side exchange of a few
    doubles per realization; the solves themselves never communicate."""
    import torch.distributed as dist
    payload = (list(map(int, indices)), np.asarray(A, dtype=np.float64).reshape(-1, 4).tolist())
    world = dist.get_world_size(group)
    gathered = [None] * world if dist.get_rank(group) == 0 else None
    dist.gather_object(payload, gathered, dst=0, group=group)
    if gathered is None:
        return None
    return merge_by_index(((p[0], np.asarray(p[1])) for p in gathered), total)


class Checkpoint:
    """Append-only JSONL of finished realizations: {"index", "A", "iters", "status"}."""

    def __init__(self, path: str):
        self.path = path

    def done(self) -> dict:
        out = {}
        if not os.path.exists(self.path):
            return out
        with open(self.path) as f:
            for line in f:
                line = line.strip()
                if not line:
                    continue
                try:
                    rec = json.loads(line)
                except json.JSONDecodeError:
                    continue          # a torn last line from an interrupted run
                out[int(rec["index"])] = rec
        return out

    def append(self, records: Iterable[dict]) -> None:
        with open(self.path, "a") as f:
            for r in records:
                f.write(json.dumps(r) + "\n")
            f.flush()
            os.fsync(f.fileno())


def run_ensemble(indices: Sequence[int], solve_batch: Callable[[list], tuple], batch: int,
                 checkpoint: Checkpoint | None = None) -> dict:
    """Solve the given realization indices in batches, skipping those already
    in the checkpoint.  solve_batch(list_of_indices) -> (A[k,2,2], infos).
    Returns {index: record} for all requested indices."""
    have = checkpoint.done() if checkpoint else {}
    todo = [k for k in indices if k not in have]
    for s in range(0, len(todo), batch):
        chunk = todo[s:s + batch]
        A, infos = solve_batch(chunk)
        recs = [{"index": int(k), "A": np.asarray(A[j]).reshape(4).tolist(),
                 "iters": list(infos[j].get("iters", (0, 0))),
                 "status": int(infos[j].get("status", 0))} for j, k in enumerate(chunk)]
        if checkpoint:
            checkpoint.append(recs)
        for r in recs:
            have[r["index"]] = r
    return {k: have[k] for k in indices}


def records_to_array(records: dict, indices: Sequence[int]) -> np.ndarray:
    return np.array([records[k]["A"] for k in indices], dtype=np.float64).reshape(-1, 2, 2)
