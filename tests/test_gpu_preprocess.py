"""Preprocessing of Section 3.1 on the GPU against the FP64 oracle:
- direct-beam centres (iterated centre of mass in a disc): bit-exact for u16 and f32 frames,
  and close to the true beam of frames whose beam was moved;
- the low-intensity threshold before gamma: the polar transform within the usual tolerance,
  for the tabulated u16 values, u16 values beyond the table, and f32 frames;
- the whole path on patterns with moved beams, indexed about the centres found, with the
  threshold and the pre-filter: hits equal the oracle's up to stated near-ties.
"""
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
    c.check()
    c.close()


def _t(a):
    import torch
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def moved():
    """FCC patterns whose content (beam included) is moved by whole pixels."""
    ts = synth.kinematic_library("fcc", step_deg=3.0)
    rng = synth.make_rng(6)
    scan = synth.render_scan(rng, ts, 64, 256, 256, n_theta=360)
    shift = rng.integers(-4, 5, size=(64, 2))
    frames = np.stack([np.roll(f, (int(dy), int(dx)), axis=(0, 1)) for f, (dx, dy) in zip(scan.frames, shift)])
    return ts, frames, shift


def test_find_centres_bit_exact(ctx, moved):
    ts, frames, shift = moved
    c = ctx.find_centres(_t(frames), radius=6.0, iterations=3).cpu().numpy()
    c_ref = O.find_centres(frames, (127.5, 127.5), 6.0, 3)
    assert np.array_equal(c, c_ref)
    assert np.all(np.abs(c - (127.5 + shift)) < 0.5)              # the moved beam is found
    c2 = ctx.find_centres(_t(frames), radius=9.5, iterations=1, cx=120.25, cy=131.0).cpu().numpy()
    assert np.array_equal(c2, O.find_centres(frames, (120.25, 131.0), 9.5, 1))
    _, scan, _ = synth.tiny_workload(n_side=4)                      # f32 frames: the same order of sums
    c3 = ctx.find_centres(_t(scan.frames), radius=5.0, iterations=2).cpu().numpy()
    assert np.array_equal(c3, O.find_centres(scan.frames, (63.5, 63.5), 5.0, 2))


def _check_threshold_polar(ctx, frames, n_r, n_theta, threshold, **kw):
    P_ref = O.polar(frames, n_r, n_theta, threshold=threshold, **kw)
    polar, norm, radial = ctx.polar_transform(_t(frames), n_r, n_theta, threshold=threshold, **kw)
    P = polar.cpu().numpy().astype(np.float64)
    scale = np.maximum(np.abs(P_ref).max(axis=(1, 2)), 1e-30)[:, None, None] + abs(kw.get("subtract", 0.0))
    assert np.all(np.abs(P - P_ref) <= 1e-6 * scale)
    assert np.allclose(norm.cpu().numpy(), np.sqrt((P_ref ** 2).sum(axis=(1, 2))), rtol=2e-6, atol=1e-30)


def test_threshold_polar_matches_oracle(ctx, moved):
    ts, frames, shift = moved
    _check_threshold_polar(ctx, frames[:8], 128, 360, 2.0)                 # tabulated u16 values
    _check_threshold_polar(ctx, frames[:8], 128, 360, 2.5, gamma=1.0, subtract=0.3)
    big = np.minimum(frames[:4].astype(np.int64) * 700, 65535).astype(np.uint16)
    _check_threshold_polar(ctx, big, 128, 360, 5000.0)                     # u16 values beyond the table
    _, scan, _ = synth.tiny_workload(n_side=2)
    _check_threshold_polar(ctx, scan.frames, 60, 180, 0.7)                 # f32, a threshold with no exact float


def test_centred_thresholded_index_matches_oracle(ctx, moved):
    ts, frames, shift = moved
    lib = O.prepare_library(ts, 128, 360)
    lid = ctx.load_library(ts, 128, 360)
    dev = _t(frames)
    c = ctx.find_centres(dev, radius=6.0, iterations=3)
    h = tmgb.hits_to_numpy(ctx.index(dev, lid, top_n=5, prefilter=0.5, centres=c, threshold=1.0))[0]
    ref = O.index(frames, lib, prefilter_fraction=0.5, N=5, centres=c.cpu().numpy().astype(np.float64),
                  threshold=1.0)
    compare_hits(h, ref, lib)
    ctx.unload_library(lid)


# ------------------------------------------------------------------ background removal and blur

def _noisy_frames(rng, n, H, W, dtype):
    """Patterns on a broad diffuse background (the case the difference of Gaussians is for)."""
    yy, xx = np.mgrid[0:H, 0:W]
    back = 20.0 * np.exp(-((xx - W / 2) ** 2 + (yy - H / 2) ** 2) / (2 * (W / 3) ** 2))
    f = rng.poisson(back[None] + 1.0, size=(n, H, W)).astype(np.float64)
    for p in range(n):
        for _ in range(6):
            y, x = rng.integers(8, H - 8), rng.integers(8, W - 8)
            f[p, y - 1:y + 2, x - 1:x + 2] += rng.integers(20, 200)
    return f.astype(dtype)


@pytest.mark.parametrize("dog,blur", [((1.0, 4.0), 0.0), (None, 1.5), ((1.0, 6.0), 1.2), (None, 0.0), ((0.7, 2.3), 9.0)])
def test_background_removal_and_blur_match_oracle(ctx, dog, blur):
    """Difference of Gaussians and blur on the GPU (FP32 sums) against the FP64 oracle: within
    3e-5 of the frames' largest value (two passes of up to 2 * 4 * 9 + 1 terms each, twice,
    at 2^-24 per term), for u16 and f32 frames, a frame narrower than the blur's radius
    included."""
    rng = np.random.default_rng(17)
    for shape, dtype in (((6, 96, 80), np.uint16), ((4, 64, 64), np.float32), ((2, 40, 24), np.float32)):
        f = _noisy_frames(rng, *shape, dtype)
        ref = O.preprocess(f, dog=dog, blur=blur)
        out = ctx.preprocess(_t(f), dog=dog, blur=blur).cpu().numpy().astype(np.float64)
        assert out.shape == ref.shape
        assert np.all(np.abs(out - ref) <= 3e-5 * float(f.max())), (shape, np.abs(out - ref).max())
        if dog is not None:
            assert np.all(out >= 0.0)


def test_index_after_background_removal(ctx):
    """The whole path on preprocessed frames: the tiny scan on a diffuse background, the
    background removed and blurred on the GPU and indexed, against the oracle's own
    preprocessing and index; the GPU's top-1 template is the oracle's, or within 1e-4 of
    the oracle's best Q (the two preprocessings differ by FP32 rounding), on >= 98 %."""
    ts, scan, _ = synth.tiny_workload(n_side=8)
    rng = np.random.default_rng(5)
    H, W = scan.frames.shape[1:]
    yy, xx = np.mgrid[0:H, 0:W]
    back = 3.0 * np.exp(-((xx - W / 2) ** 2 + (yy - H / 2) ** 2) / (2 * 30.0 ** 2))
    frames = (scan.frames + back[None] + rng.random(scan.frames.shape) * 0.2).astype(np.float32)
    lib = O.prepare_library(ts, 60, 180)
    lid = ctx.load_library(ts, 60, 180)
    pre = ctx.preprocess(_t(frames), dog=(1.0, 5.0), blur=1.0)
    h = tmgb.hits_to_numpy(ctx.index(pre, lid, top_n=5))[0]
    # the oracle indexes float32 frames, as the GPU path does: its preprocessing rounded to them
    ref = O.index(O.preprocess(frames, dog=(1.0, 5.0), blur=1.0).astype(np.float32), lib, N=5)
    ok = 0
    for p in range(frames.shape[0]):
        k = int(h["template_index"][p, 0])
        qb = ref["score"][p, 0]
        ok += int(k == ref["template"][p, 0] or abs(ref["q_best"][p, k] - qb) <= 1e-4 * abs(qb))
    assert ok >= 0.98 * frames.shape[0], ok
    ctx.unload_library(lid)
