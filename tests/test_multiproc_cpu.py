"""Multi-process paths on CPU (gloo, world size 2).

- Pattern sharding: the ranks' ranges cover the scan exactly once.
- Template sharding: each rank scores all patterns against its template range with the
  FP64 oracle; all-gather + merge under (Q desc, template asc) equals the single-process
  top-N over all templates.
- A rank that fails is seen by the other on the host (no GPU involved)."""
import os
import socket

import numpy as np
import pytest

from paper_2111_07347_gb300 import parallel


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_range_covers_once():
    for n in (0, 1, 7, 16384, 16385):
        for world in (1, 2, 3, 8):
            seen = np.zeros(n, dtype=int)
            for r in range(world):
                a, b = parallel.shard_range(n, r, world)
                seen[a:b] += 1
                assert b - a in (n // world, n // world + 1)
            assert np.all(seen == 1)


def test_merge_topn_total_order():
    t = np.array([[[3, 1, -1]], [[2, 5, 0]]])
    s = np.array([[[7, 8, -1]], [[9, 1, 2]]])
    q = np.array([[[0.9, 0.5, -np.inf]], [[0.9, 0.7, 0.1]]])
    mt, ms, mq = parallel.merge_topn(t, s, q, 4)
    assert list(mt[0]) == [2, 3, 5, 1] and list(ms[0]) == [9, 7, 1, 8]


def _worker(rank, world, port, frames, ts_dict, N, outq, fail_rank):
    import torch.distributed as dist
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if rank == fail_rank:
            raise RuntimeError("injected failure on the host")
        from oracle import oracle as O
        from paper_2111_07347_gb300 import synth
        ts = synth.TemplateSet(**ts_dict)
        lib = O.prepare_library(ts, 60, 180)
        a, b = parallel.shard_range(lib.K, rank, world)
        P = O.polar(frames, 60, 180)
        act = np.zeros((frames.shape[0], lib.K), dtype=bool)
        act[:, a:b] = True
        q, s = O.scores(P, lib, act)
        tk, tsh, tq = O.top_n(q, s, N, act)
        mt, ms, mq = parallel.allgather_topn(torch.from_numpy(tk), torch.from_numpy(tsh), torch.from_numpy(tq), N)
        if rank == 0:
            outq.put(("ok", mt, ms, mq))
    except Exception as e:                      # reported to the parent through the queue
        outq.put(("error", rank, str(e)))
    finally:
        dist.destroy_process_group()


def test_template_shard_merge_equals_single_process():
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from paper_2111_07347_gb300 import synth
    ts, scan, prm = synth.tiny_workload(n_side=3)
    frames = scan.frames
    ts_dict = dict(offsets=ts.offsets, a=ts.a, b=ts.b, intensity=ts.intensity, coords=ts.coords)
    ctx = mp.get_context("spawn")
    outq = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, frames, ts_dict, 5, outq, -1)) for r in range(2)]
    for p in procs:
        p.start()
    res = outq.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
    assert res[0] == "ok", res
    _, mt, ms, mq = res
    ref = O.index(frames, O.prepare_library(ts, 60, 180), N=5)
    assert np.array_equal(mt, ref["template"]) and np.array_equal(ms, ref["shift"])
    assert np.allclose(mq, ref["score"], rtol=1e-12)


def test_failed_rank_is_reported_on_the_host():
    import torch.multiprocessing as mp
    from paper_2111_07347_gb300 import synth
    ts, scan, prm = synth.tiny_workload(n_side=1)
    ts_dict = dict(offsets=ts.offsets, a=ts.a, b=ts.b, intensity=ts.intensity, coords=ts.coords)
    ctx = mp.get_context("spawn")
    outq = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, scan.frames[:2], ts_dict, 3, outq, 1)) for r in range(2)]
    for p in procs:
        p.start()
    msgs = []
    try:
        while len(msgs) < 2:
            msgs.append(outq.get(timeout=60))
            if any(m[0] == "error" for m in msgs):
                break
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    assert any(m[0] == "error" and m[1] == 1 for m in msgs)
