"""GPU tests of the serving loop (continuous batching of scan lines and maps).

Failure paths are injected on the host: a paused dispatcher (a stalled producer), a
cancelled request, a full admission budget and an oversized request.  No test faults,
traps or hangs the GPU; every wait has a timeout."""
import numpy as np
import pytest

from paper_2111_07347_gb300 import synth
from paper_2111_07347_gb300 import tmgb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2111_07347_gb300 import build
    build.build()
    ctx = tmgb.Context(0)
    rng = synth.make_rng(4)
    a = synth.kinematic_library("fcc", step_deg=2.0)
    b = synth.kinematic_library("hcp", step_deg=2.0)
    la, lb = ctx.load_library(a, 128, 360), ctx.load_library(b, 128, 360)
    scan = synth.render_scan(rng, b, 1500, 256, 256, n_theta=360)
    frames = scan.frames
    yield ctx, la, lb, frames
    ctx.close()


def _direct(ctx, frames, lids, **kw):
    import torch
    t = torch.from_numpy(frames.view(np.int16)).cuda().view(torch.uint16)
    out = ctx.index(t, lids, **kw)
    torch.cuda.synchronize()
    return tmgb.hits_to_numpy(out)


def test_alone_equals_in_mix(env):
    ctx, la, lb, frames = env
    srv = tmgb.Server(ctx, slots=3, tile_patterns=256, max_libs=2)
    line = np.ascontiguousarray(frames[100:420])
    t = srv.submit(line, [la, lb], top_n=5, priority=1)
    alone, st = srv.wait(t, timeout_ms=60000)
    assert st["status"] == tmgb.TM_OK
    assert np.array_equal(alone, _direct(ctx, line, [la, lb], top_n=5))
    # the same line again, now in a mix of maps and other lines on several slots
    tickets = []
    tickets.append(("map", srv.submit(np.ascontiguousarray(frames[:1024]), [la, lb], top_n=5, priority=0)))
    tickets.append(("line", srv.submit(line, [la, lb], top_n=5, priority=1)))
    tickets.append(("other", srv.submit(np.ascontiguousarray(frames[900:1400]), [la, lb], top_n=5, priority=1)))
    tickets.append(("map2", srv.submit(np.ascontiguousarray(frames[200:1200]), [lb], top_n=5, priority=0)))
    res = {}
    for name, tk in tickets:
        out, st = srv.wait(tk, timeout_ms=60000)
        assert st["status"] == tmgb.TM_OK, (name, st)
        res[name] = out
    assert np.array_equal(res["line"], alone)
    assert np.array_equal(res["map"], _direct(ctx, frames[:1024], [la, lb], top_n=5))
    assert np.array_equal(res["map2"], _direct(ctx, frames[200:1200], [lb], top_n=5))
    srv.close()


def test_bf16_path_through_server(env):
    ctx, la, lb, frames = env
    srv = tmgb.Server(ctx, slots=2, tile_patterns=128, max_libs=1)
    x = np.ascontiguousarray(frames[:300])
    t = srv.submit(x, [lb], top_n=5, priority=1, path=tmgb.TM_PATH_BF16_RESCORE, rescore_k=64)
    out, st = srv.wait(t, timeout_ms=60000)
    assert st["status"] == tmgb.TM_OK
    assert np.array_equal(out, _direct(ctx, x, [lb], top_n=5, path=tmgb.TM_PATH_BF16_RESCORE, rescore_k=64))
    srv.close()
    ctx.check()


def test_stalled_dispatch_times_out_then_completes(env):
    ctx, la, lb, frames = env
    srv = tmgb.Server(ctx, slots=2, tile_patterns=128)
    srv.pause(True)
    t = srv.submit(np.ascontiguousarray(frames[:200]), [la], top_n=3, priority=1)
    with pytest.raises(tmgb.TmError) as e:
        srv.wait(t, timeout_ms=150)
    assert e.value.code == tmgb.TM_ERR_TIMEOUT
    srv.pause(False)
    out, st = srv.wait(t, timeout_ms=60000)
    assert st["status"] == tmgb.TM_OK and st["tiles"] == 2
    srv.close()


def test_cancel_before_dispatch(env):
    ctx, la, lb, frames = env
    srv = tmgb.Server(ctx, slots=1, tile_patterns=64)
    srv.pause(True)
    t = srv.submit(np.ascontiguousarray(frames[:256]), [la], top_n=3)
    srv.cancel(t)
    srv.pause(False)
    out, st = srv.wait(t, timeout_ms=60000)
    assert st["status"] == tmgb.TM_ERR_CANCELLED
    with pytest.raises(tmgb.TmError) as e:
        srv.wait(t, timeout_ms=10)
    assert e.value.code == tmgb.TM_ERR_NOT_FOUND
    srv.close()


def test_admission_budget_busy(env):
    ctx, la, lb, frames = env
    x = np.ascontiguousarray(frames[:128])
    srv = tmgb.Server(ctx, slots=1, tile_patterns=64, queue_bytes=x.nbytes + 1, blocking_submit=False)
    srv.pause(True)
    t1 = srv.submit(x, [la], top_n=3)
    with pytest.raises(tmgb.TmError) as e:
        srv.submit(x, [la], top_n=3)
    assert e.value.code == tmgb.TM_ERR_BUSY
    srv.pause(False)
    out, st = srv.wait(t1, timeout_ms=60000)
    assert st["status"] == tmgb.TM_OK
    t2 = srv.submit(x, [la], top_n=3)           # room again once the first finished
    out2, st2 = srv.wait(t2, timeout_ms=60000)
    assert np.array_equal(out, out2)
    srv.close()


def test_rejects_requests_beyond_limits(env):
    ctx, la, lb, frames = env
    srv = tmgb.Server(ctx, slots=1, tile_patterns=64, max_H=128, max_W=128)
    with pytest.raises(tmgb.TmError) as e:
        srv.submit(np.ascontiguousarray(frames[:4]), [la], top_n=3)
    assert e.value.code == tmgb.TM_ERR_INVALID_ARG
    srv.close()


def test_scan_lines_do_not_wait_for_map_tiles(env):
    """With a slot reserved for requests of priority > 0, a scan line submitted behind two
    maps (whose tiles fill the other slot) finishes before them, with the same hits as a
    direct call."""
    ctx, la, lb, frames = env
    srv = tmgb.Server(ctx, slots=2, tile_patterns=128, max_libs=2, priority_slots=1)
    maps = [srv.submit(np.ascontiguousarray(frames[:1500]), [la, lb], top_n=5, priority=0) for _ in range(2)]
    line = np.ascontiguousarray(frames[10:138])
    t = srv.submit(line, [la, lb], top_n=5, priority=1)
    out, st_line = srv.wait(t, timeout_ms=60000)
    st_maps = [srv.wait(m, timeout_ms=120000)[1] for m in maps]
    assert st_line["status"] == tmgb.TM_OK and all(s["status"] == tmgb.TM_OK for s in st_maps)
    assert st_line["done_ms"] < min(s["done_ms"] for s in st_maps)
    assert np.array_equal(out, _direct(ctx, line, [la, lb], top_n=5))
    srv.close()


def test_hbm_budget_admission_and_device_frames(env):
    """Admission by the device budget: every admitted request holds its hits in the server's
    arena; a non-blocking submit that finds no room gets TM_ERR_BUSY, a request larger than the
    whole arena is refused, and room returns once a request finishes.  A map whose frames are
    already on the device (frames_dev) gives the same hits as a direct call, with no frame copy
    in its timeline; a scan line from host memory records copy and kernel time."""
    import torch
    ctx, la, lb, frames = env
    x = np.ascontiguousarray(frames[:200])
    hits_bytes = 2 * 200 * 5 * 20                      # [n_libs][n][top_n] tm_hit
    srv = tmgb.Server(ctx, slots=2, tile_patterns=64, max_libs=2, blocking_submit=False,
                      hbm_budget_bytes=hits_bytes + 512, priority_slots=1)
    srv.pause(True)
    t1 = srv.submit(x, [la, lb], top_n=5, priority=1)
    with pytest.raises(tmgb.TmError) as e:
        srv.submit(x, [la, lb], top_n=5, priority=1)
    assert e.value.code == tmgb.TM_ERR_BUSY
    with pytest.raises(tmgb.TmError) as e:
        srv.submit(np.ascontiguousarray(frames[:1000]), [la, lb], top_n=5)
    assert e.value.code == tmgb.TM_ERR_INVALID_ARG
    srv.pause(False)
    out1, st1 = srv.wait(t1, timeout_ms=60000)
    assert st1["status"] == tmgb.TM_OK
    assert st1["h2d_ms"] > 0 and st1["kernels_ms"] > 0 and st1["d2h_ms"] > 0
    assert st1["submit_ms"] <= st1["admit_ms"] <= st1["first_dispatch_ms"] <= st1["done_ms"]
    assert np.array_equal(out1, _direct(ctx, x, [la, lb], top_n=5))
    dev = torch.from_numpy(x.view(np.int16)).cuda().view(torch.uint16)
    t2 = srv.submit(dev, [la, lb], top_n=5, priority=0)
    out2, st2 = srv.wait(t2, timeout_ms=60000)
    assert st2["status"] == tmgb.TM_OK and st2["kernels_ms"] > 0
    assert st2["h2d_ms"] < 0.05
    assert np.array_equal(out2, out1)
    srv.close()
