"""The whole path from host buffers (tm_index_patterns_host): chunks alternate between two
streams, so copies overlap kernels.  Its hits must equal the device-buffer call bit for bit
(a pattern's result does not depend on its batch), for ragged chunks, pageable and
page-locked inputs, several libraries and per-pattern centres; and, through the device path,
they agree with the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_07347_gb300 import synth
from paper_2111_07347_gb300 import tmgb
from tests._compare import compare_hits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2111_07347_gb300 import build
    build.build()
    c = tmgb.Context(0)
    yield c
    c.close()


def _dev(a):
    import torch
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(a).cuda()


def _device_hits(ctx, frames, lids, **kw):
    return tmgb.hits_to_numpy(ctx.index(_dev(frames), lids, **kw))


def test_host_equals_device_ragged_chunks_pageable(ctx):
    ts, scan, prm = synth.tiny_workload()
    lid = ctx.load_library(ts, 60, 180)
    ref = _device_hits(ctx, scan.frames, lid, top_n=5)
    for chunk in (37, 256, 0, 1000):
        out = ctx.index_host(scan.frames, lid, top_n=5, chunk=chunk)
        assert np.array_equal(tmgb.hits_to_numpy(out), ref), chunk
    assert ctx.last_stats["patterns"] == scan.frames.shape[0]
    oracle_ref = O.index(scan.frames, O.prepare_library(ts, 60, 180), N=5)
    compare_hits(tmgb.hits_to_numpy(out)[0], oracle_ref, O.prepare_library(ts, 60, 180))
    ctx.unload_library(lid)


def test_host_pinned_multilib_centres_and_prefilter(ctx):
    import torch
    a = synth.kinematic_library("fcc", step_deg=3.0)
    b = synth.kinematic_library("hcp", step_deg=3.0)
    rng = synth.make_rng(4)
    scan = synth.render_scan(rng, a, 96, 256, 256, n_theta=360)
    la, lb = ctx.load_library(a, 128, 360), ctx.load_library(b, 128, 360)
    cen = (np.array([127.5, 127.5]) + rng.uniform(-3.0, 3.0, size=(96, 2))).astype(np.float32)
    kw = dict(top_n=5, prefilter=0.5)
    ref = tmgb.hits_to_numpy(ctx.index(_dev(scan.frames), [la, lb], centres=_dev(cen), **kw))
    pinned = torch.from_numpy(scan.frames.view(np.int16)).view(torch.uint16).pin_memory()
    out = torch.empty((2, 96, 5, 5), dtype=torch.int32).pin_memory()
    ctx.index_host(pinned, [la, lb], out=out, chunk=40, centres=cen, **kw)
    assert np.array_equal(tmgb.hits_to_numpy(out), ref)
    # the BF16 path through the host entry point as well
    ref16 = _device_hits(ctx, scan.frames, la, top_n=5, path=tmgb.TM_PATH_BF16_RESCORE)
    out16 = ctx.index_host(scan.frames, la, top_n=5, path=tmgb.TM_PATH_BF16_RESCORE, chunk=50)
    assert np.array_equal(tmgb.hits_to_numpy(out16), ref16)
    ctx.unload_library(la)
    ctx.unload_library(lb)


def test_host_empty_and_bad_arguments(ctx):
    ts, scan, prm = synth.tiny_workload(n_side=2)
    lid = ctx.load_library(ts, 60, 180)
    out = ctx.index_host(scan.frames[:0], lid, top_n=3)
    assert out.shape == (1, 0, 3, 5)
    with pytest.raises(ValueError):
        ctx.index_host(scan.frames, lid, top_n=3, out=np.empty((1, 1, 3, 5), dtype=np.int32))
    with pytest.raises(tmgb.TmError) as e:
        ctx.index_host(scan.frames, lid, top_n=3, chunk=-1)
    assert e.value.code == tmgb.TM_ERR_INVALID_ARG
    with pytest.raises(tmgb.TmError) as e:
        ctx.index_host(scan.frames, [lid + 1000], top_n=3)
    assert e.value.code == tmgb.TM_ERR_NOT_FOUND
    ctx.unload_library(lid)
