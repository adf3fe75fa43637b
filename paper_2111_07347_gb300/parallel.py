"""Multi-GPU layout of the indexing path (one process per GPU).

Patterns are independent (the paper maps the indexation over images with Dask, Section
2.2), so the default is pattern sharding: each rank indexes a contiguous range of the scan
with the libraries replicated, and no collective is needed on the data path.

For a library too large for one GPU the templates can be sharded instead: every rank
scores all patterns against its template range and returns per-pattern top-N lists; one
all-gather and a merge under the total order (Q desc, template asc) give exactly the
single-GPU answer, because every template's score and best shift are computed the same
way on every rank.
"""
from __future__ import annotations

import numpy as np


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [start, stop) of n items for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def merge_topn(template: np.ndarray, shift: np.ndarray, score: np.ndarray, N: int):
    """Merge per-shard top-N lists of the same patterns.

    template/shift/score: [shards][n][N_s] with global template indices (-1 padding and
    -inf scores for missing rows).  Returns ([n][N], [n][N], [n][N]) ordered by
    (score desc, template asc), padded with -1 / -inf."""
    S, n, Ns = template.shape
    t = template.transpose(1, 0, 2).reshape(n, S * Ns)
    s = shift.transpose(1, 0, 2).reshape(n, S * Ns)
    q = score.transpose(1, 0, 2).reshape(n, S * Ns).astype(np.float64)
    valid = t >= 0
    key_q = np.where(valid, -q, np.inf)
    key_t = np.where(valid, t, np.iinfo(np.int64).max)
    out_t = np.full((n, N), -1, dtype=np.int64)
    out_s = np.full((n, N), -1, dtype=np.int64)
    out_q = np.full((n, N), -np.inf)
    for p in range(n):
        order = np.lexsort((key_t[p], key_q[p]))[:N]
        order = order[valid[p][order]]
        k = len(order)
        out_t[p, :k], out_s[p, :k], out_q[p, :k] = t[p, order], s[p, order], q[p, order]
    return out_t, out_s, out_q


def allgather_topn(template, shift, score, N: int):
    """All-gather per-rank top-N lists (torch.distributed must be initialised; tensors on
    the backend's device) and merge them; returns numpy arrays."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size()
    parts = []
    for x in (template, shift, score):
        bufs = [torch.empty_like(x) for _ in range(world)]
        dist.all_gather(bufs, x)
        parts.append(torch.stack(bufs).cpu().numpy())
    return merge_topn(parts[0], parts[1], parts[2], N)
