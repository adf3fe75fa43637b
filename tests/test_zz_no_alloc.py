"""GPU test of tm_index_patterns_noalloc, the whole-path call for callers that cannot
allocate device memory while indexing (its scratch lives in a static device array).

It must give the same hits as tm_index_patterns, on two calls in a row (the second call
finds the first call's data in the shared scratch and must not depend on it), for f32
frames and for u16 frames with a pixel mask and a threshold; it must refuse a misaligned
mask, the BF16 path and a pre-filter on the host, and a batch whose scratch does not fit.  The file is named to be collected last."""
import ctypes

import numpy as np
import pytest

from paper_2111_07347_gb300 import synth
from paper_2111_07347_gb300 import tmgb
from tests._compare import tol

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    f = tmgb.library().tm_index_patterns_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(tmgb.tm_index_params), ctypes.c_void_p, ctypes.c_int32,
                  ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    return f


def _same_hits(a, b):
    """Identical templates and shifts; scores within the parity tolerance."""
    assert np.array_equal(a["template_index"], b["template_index"])
    assert np.array_equal(a["shift"], b["shift"])
    q = b["score"].astype(np.float64)
    ok = np.isneginf(q) | (np.abs(a["score"] - q) <= tol(q, np.max(np.abs(q[np.isfinite(q)]))))
    assert np.all(ok)


def test_noalloc_matches_index_patterns_twice():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2111_07347_gb300 import build
    build.build()
    ctx = tmgb.Context(0)
    f = _noalloc_fn()
    ts, scan, prm = synth.tiny_workload(n_side=12)             # 144 frames, 128 x 128 f32
    lid = ctx.load_library(ts, 60, 180)
    stream = torch.cuda.current_stream().cuda_stream
    p = tmgb.make_params(top_n=5)
    for frames in (scan.frames, np.ascontiguousarray(scan.frames[::-1][:100])):
        fd = torch.from_numpy(frames).cuda()
        n = frames.shape[0]
        ref = tmgb.hits_to_numpy(ctx.index(fd, lid, top_n=5))[0]
        out = torch.empty((n, 5, 5), dtype=torch.int32, device="cuda")
        rc = f(ctx.handle, ctypes.byref(p), fd.data_ptr(), tmgb.TM_DTYPE_F32, n, 128, 128, lid, out.data_ptr(), stream)
        assert rc == tmgb.TM_OK, tmgb.tm_last_error()
        torch.cuda.synchronize()
        _same_hits(tmgb.hits_to_numpy(out), ref)
    # u16 frames with a pixel mask (16-byte aligned, as tm_index_patterns requires) and a
    # threshold: the staged u16 path with both applied while the frame is staged
    ts2, scan2, _ = synth.single_phase_workload(n_patterns=96, step_deg=3.0)
    lid2 = ctx.load_library(ts2, 128, 360)
    fd = torch.from_numpy(scan2.frames.view(np.int16)).cuda().view(torch.uint16)
    mask = torch.ones((256, 256), dtype=torch.uint8, device="cuda")
    mask[100:156, 100:156] = 0
    assert mask.data_ptr() % 16 == 0
    p2 = tmgb.make_params(top_n=5, mask=mask, threshold=2.0)
    for _ in range(2):
        ref = tmgb.hits_to_numpy(ctx.index(fd, lid2, top_n=5, mask=mask, threshold=2.0))[0]
        out = torch.empty((96, 5, 5), dtype=torch.int32, device="cuda")
        rc = f(ctx.handle, ctypes.byref(p2), fd.data_ptr(), tmgb.TM_DTYPE_U16, 96, 256, 256, lid2, out.data_ptr(), stream)
        assert rc == tmgb.TM_OK, tmgb.tm_last_error()
        torch.cuda.synchronize()
        _same_hits(tmgb.hits_to_numpy(out), ref)
    # parameters the entry point refuses on the host, before anything is launched
    bad = tmgb.make_params(top_n=5)
    bad.pixel_mask = mask.data_ptr() + 1
    for prm, needle in ((bad, "pixel_mask"), (tmgb.make_params(top_n=5, path=tmgb.TM_PATH_BF16_RESCORE), "FP32"),
                        (tmgb.make_params(top_n=5, prefilter=0.5), "FP32")):
        rc = f(ctx.handle, ctypes.byref(prm), fd.data_ptr(), tmgb.TM_DTYPE_U16, 96, 256, 256, lid2, out.data_ptr(),
               stream)
        assert rc == tmgb.TM_ERR_INVALID_ARG and needle in tmgb.tm_last_error()
    ctx.unload_library(lid2)
    # a batch whose scratch cannot fit is refused with a message, and nothing runs
    big = 4000
    fd = torch.zeros((big, 128, 128), dtype=torch.float32, device="cuda")
    out = torch.empty((big, 5, 5), dtype=torch.int32, device="cuda")
    rc = f(ctx.handle, ctypes.byref(p), fd.data_ptr(), tmgb.TM_DTYPE_F32, big, 128, 128, lid, out.data_ptr(), stream)
    assert rc == tmgb.TM_ERR_INVALID_ARG and "scratch" in tmgb.tm_last_error()
    ctx.unload_library(lid)
    ctx.close()
