"""Template simulation over an orientation grid on the GPU (Section 2.1) against the FP64
oracle: the kept reflections, their order and their values bit for bit (both sides round
every operation in the same order); a library made from the device's templates indexes
exactly like one made from the oracle's; an orientation with more reflections than the
kernel's buffer is reported, not truncated."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_07347_gb300 import synth
from paper_2111_07347_gb300 import tmgb

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


def _inputs(name, system, step, g_max=1.2):
    st = synth.STRUCTURES[name]
    g, F2, gn = synth._reciprocal_points(st, g_max)
    dirs = synth.beam_directions(system, step)
    R = np.stack([synth._orientation_matrix(d) for d in dirs])
    return g, F2, gn, R


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("name,system,step,max_spots", [("fcc", "cubic", 2.0, 150), ("hcp", "hexagonal", 3.0, 150),
                                                        ("tetragonal", "tetragonal", 3.0, 150),
                                                        ("hcp", "hexagonal", 5.0, 4)])
def test_kinematic_spots_bit_exact(ctx, name, system, step, max_spots):
    g, F2, gn, R = _inputs(name, system, step)
    lam, s_max = synth.WAVELENGTH_200KV, 0.02
    counts, spots = ctx.kinematic_spots(_dev(g), _dev(F2), _dev(gn), _dev(R), lam, s_max, max_spots)
    c_ref, s_ref = O.kinematic_spots(g, F2, gn, R, lam, s_max, max_spots)
    counts, spots = counts.cpu().numpy(), spots.cpu().numpy()
    assert np.array_equal(counts, c_ref)
    for d in range(len(counts)):
        assert np.array_equal(spots[d, :counts[d]], s_ref[d, :counts[d]]), d


def test_device_library_indexes_like_host_library(ctx):
    import torch
    g, F2, gn, R = _inputs("fcc", "cubic", 3.0)
    lam, s_max = synth.WAVELENGTH_200KV, 0.02
    ts_dev = ctx.kinematic_templates(g, F2, gn, R, lam, s_max, 150)
    c_ref, s_ref = O.kinematic_spots(g, F2, gn, R, lam, s_max, 150)
    flat = np.concatenate([s_ref[d, :c_ref[d]] for d in range(len(c_ref))])
    ts_host = synth.TemplateSet(np.concatenate([[0], np.cumsum(c_ref)]).astype(np.int64), flat[:, 0].copy(),
                                flat[:, 1].copy(), flat[:, 2].copy(), coords="xy", px_per_unit=100.0, mirror=True)
    rng = synth.make_rng(11)
    scan = synth.render_scan(rng, synth.kinematic_library("fcc", step_deg=3.0), 96, 256, 256, n_theta=360)
    frames = torch.from_numpy(scan.frames.view(np.int16)).cuda().view(torch.uint16)
    la = ctx.load_library(ts_dev, 128, 360)
    lb = ctx.load_library(ts_host, 128, 360)
    ha = tmgb.hits_to_numpy(ctx.index(frames, la, top_n=5, prefilter=0.5))[0]
    hb = tmgb.hits_to_numpy(ctx.index(frames, lb, top_n=5, prefilter=0.5))[0]
    # the device's templates are the oracle's bit for bit, so are the libraries and the hits
    for f in ("template_index", "shift", "score", "mirror"):
        assert np.array_equal(ha[f], hb[f]), f
    ctx.unload_library(la)
    ctx.unload_library(lb)


def test_kinematic_overflow_is_reported(ctx):
    g, F2, gn, R = _inputs("fcc", "cubic", 10.0, g_max=3.5)
    assert g.shape[0] > 512
    counts, _ = ctx.kinematic_spots(_dev(g), _dev(F2), _dev(gn), _dev(R[:3]), synth.WAVELENGTH_200KV, 50.0, 20)
    assert np.all(counts.cpu().numpy() == -1)
    with pytest.raises(tmgb.TmError):
        ctx.kinematic_templates(g, F2, gn, R[:3], synth.WAVELENGTH_200KV, 50.0, 20)


def test_orientation_vectors_and_deviation_match_oracle(ctx):
    """Orientation-map vectors and Eq. 2 on the GPU against the oracle (FP64 with the same
    operation order; cos, sin and acos from the math libraries, so within 1e-12), for random
    hits over the FCC grid's orientations, mirror copies and missing hits included."""
    import torch
    g, F2, gn, R = _inputs("fcc", "cubic", 3.0)
    K0 = R.shape[0]
    rng = np.random.default_rng(8)
    n, top_n = 500, 3
    tmpl = rng.integers(0, 2 * K0, size=n)
    tmpl[::37] = -1
    ang = (rng.integers(0, 360, size=n) * 1.0 + rng.random(n)).astype(np.float32)
    hits = np.zeros((n, top_n, 5), dtype=np.int32)
    hits[:, 0, 0] = tmpl
    hits[:, 0, 1] = ang.astype(np.int32)
    hits[:, 0, 3] = ang.view(np.int32)
    hits[:, 0, 4] = (tmpl >= K0).astype(np.int32)
    hits[:, 1:, 0] = 5                                                   # rows 1.. are ignored
    hd = torch.from_numpy(hits).cuda()
    rd = _dev(R)
    for axis in ((0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, 0.6, 0.8)):
        v = ctx.orientation_vectors(hd, rd, K0, axis).cpu().numpy()
        ref = O.orientation_vectors(tmpl, ang, R, K0, axis)
        assert np.array_equal(np.isnan(v), np.isnan(ref))
        ok = ~np.isnan(ref)
        assert np.allclose(v[ok], ref[ok], rtol=0, atol=1e-12)
    va = rng.standard_normal((n, 3))
    vb = va + 0.3 * rng.standard_normal((n, 3))
    vb[::11] = va[::11] * 2.5                                            # parallel
    vb[::13] = -va[::13]                                                 # antiparallel
    va[::17] = np.nan
    d = ctx.angular_deviation(_dev(va), _dev(vb)).cpu().numpy()
    dref = O.angular_deviation(va, vb)
    assert np.array_equal(np.isnan(d), np.isnan(dref))
    ok = ~np.isnan(dref)
    assert np.allclose(d[ok], dref[ok], rtol=0, atol=1e-9)
