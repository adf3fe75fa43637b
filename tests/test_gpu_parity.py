"""GPU parity: every stage of the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs (tolerances in tests/_compare.py: rel 1e-5 on Q, identical indices
except stated near-ties)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_07347_gb300 import synth
from paper_2111_07347_gb300 import tmgb
from tests._compare import compare_hits, compare_scores

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


def _t(a):
    import torch
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(a).cuda()


def _np(t):
    import torch
    if t.dtype == torch.uint16:
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def tiny():
    ts, scan, prm = synth.tiny_workload()
    lib = O.prepare_library(ts, 60, 180)
    ref = O.index(scan.frames, lib, N=5)
    return ts, scan, lib, ref


@pytest.fixture(scope="module")
def fcc():
    ts, scan, prm = synth.single_phase_workload(n_patterns=96)
    lib = O.prepare_library(ts, 128, 360)
    return ts, scan, lib


# ------------------------------------------------------------------ stage 1: polar

def _check_polar(ctx, frames, n_r, n_theta, gamma=0.5, subtract=0.0, dr=1.0, centres=None):
    P_ref = O.polar(frames, n_r, n_theta, dr, gamma, subtract,
                    centres=None if centres is None else centres.astype(np.float64))
    polar, norm, radial = ctx.polar_transform(_t(frames), n_r, n_theta, dr, gamma, subtract,
                                              centres=None if centres is None else _t(centres))
    P = _np(polar).astype(np.float64)
    # each sample is a convex combination of four float gamma values (correctly rounded
    # sqrt / powf) with weights within a few ulps: error <= 8 ulp of the largest tap; the
    # per-pattern maximum bounds every tap
    scale = np.maximum(np.abs(P_ref).max(axis=(1, 2)), 1e-30)[:, None, None] + abs(subtract)
    err = np.abs(P - P_ref)
    assert np.all(err <= 1e-6 * scale), (err.max(), np.unravel_index(np.argmax(err / scale), err.shape))
    nref = np.sqrt((P_ref ** 2).sum(axis=(1, 2)))
    assert np.allclose(_np(norm), nref, rtol=2e-6, atol=1e-30)
    rref = P_ref.sum(axis=2)
    rs = np.abs(P_ref).sum(axis=2)
    # row sums: the per-sample bound summed over the row plus float summation of n_theta terms
    rerr = np.abs(_np(radial) - rref)
    rtol = 1e-6 * scale[:, :, 0] * n_theta + 1e-6 * rs
    assert np.all(rerr <= rtol), (rerr.max(), np.unravel_index(np.argmax(rerr / rtol), rerr.shape))
    return P_ref


def test_polar_tiny_f32(ctx, tiny):
    ts, scan, lib, ref = tiny
    _check_polar(ctx, scan.frames, 60, 180)


def test_polar_u16_256_and_options(ctx, fcc):
    ts, scan, lib = fcc
    _check_polar(ctx, scan.frames[:24], 128, 360)
    _check_polar(ctx, scan.frames[:8], 128, 360, gamma=1.0, subtract=0.3)
    _check_polar(ctx, scan.frames[:8], 100, 90, gamma=0.7, dr=1.25)


def test_polar_per_pattern_centres(ctx, fcc):
    """Each pattern resampled about its own beam centre (fractional, off the frame centre)."""
    ts, scan, lib = fcc
    rng = np.random.default_rng(8)
    n = 16
    centres = (np.array([127.5, 127.5]) + rng.uniform(-6.0, 6.0, size=(n, 2))).astype(np.float32)
    centres[0] = (127.5, 127.5)
    centres[1] = (100.0, 140.25)
    _check_polar(ctx, scan.frames[:n], 128, 360, centres=centres)


def test_polar_ragged_and_tiny_grids(ctx):
    rng = np.random.default_rng(3)
    f = rng.poisson(3.0, size=(5, 37, 53)).astype(np.float32)
    _check_polar(ctx, f, 30, 7)
    _check_polar(ctx, f, 1, 1)
    _check_polar(ctx, f, 26, 1000)


# ------------------------------------------------------------------ library

def test_library_export_matches_oracle(ctx, fcc, tiny):
    for ts, lib, n_r, n_theta in [(fcc[0], fcc[2], 128, 360), (tiny[0], tiny[2], 60, 180)]:
        lid = ctx.load_library(ts, n_r, n_theta)
        h = ctx.library_export(lid)
        assert np.array_equal(h["offsets"], lib.off)
        assert np.array_equal(h["r"], lib.ri) and np.array_equal(h["t"], lib.ti)
        assert np.allclose(h["intensity"], lib.I, rtol=6e-8, atol=0)
        ctx.unload_library(lid)


# ------------------------------------------------------------------ stage 3: correlate

def test_correlate_scores_tiny(ctx, tiny):
    ts, scan, lib, ref = tiny
    lid = ctx.load_library(ts, 60, 180)
    polar, norm, radial = ctx.polar_transform(_t(scan.frames[:64]), 60, 180)
    q, s = ctx.correlate(lid, polar, norm)
    compare_scores(_np(q), _np(s), ref["q_best"][:64], ref["s_best"][:64], ref["polar"], lib)
    ctx.unload_library(lid)


def test_correlate_scores_fcc_mirror(ctx, fcc):
    ts, scan, lib = fcc
    lid = ctx.load_library(ts, 128, 360)
    frames = scan.frames[:12]
    P_ref = O.polar(frames, 128, 360)
    q_ref, s_ref = O.scores(P_ref, lib)
    polar, norm, radial = ctx.polar_transform(_t(frames), 128, 360)
    q, s = ctx.correlate(lid, polar, norm)
    compare_scores(_np(q), _np(s), q_ref, s_ref, P_ref, lib)
    ctx.unload_library(lid)


# ------------------------------------------------------------------ stage 2: pre-filter

def _unpack(mask, K):
    m = _np(mask).view(np.uint32)
    bits = ((m[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(bool)
    return bits.reshape(m.shape[0], -1)[:, :K]


def test_prefilter_parity(ctx, fcc):
    ts, scan, lib = fcc
    lid = ctx.load_library(ts, 128, 360)
    frames = scan.frames[:32]
    P_ref = O.polar(frames, 128, 360)
    for f in (0.5, 0.1, 1.0):
        act_ref, sc_ref = O.prefilter(P_ref, lib, f)
        polar, norm, radial = ctx.polar_transform(_t(frames), 128, 360)
        mask, score = ctx.prefilter(lid, radial, f)
        assert np.allclose(_np(score), sc_ref, rtol=1e-5, atol=1e-6)
        act = _unpack(mask, lib.K)
        keep = O.keep_count(f, lib.K)
        assert np.all(act.sum(axis=1) == keep)
        # differences only between templates whose scores tie with the threshold to 1e-5
        for p in range(frames.shape[0]):
            diff = np.flatnonzero(act[p] != act_ref[p])
            if diff.size:
                thr = np.sort(sc_ref[p])[::-1][keep - 1]
                assert np.all(np.abs(sc_ref[p, diff] - thr) <= 1e-5 * max(abs(thr), 1e-3)), (p, diff)
    ctx.unload_library(lid)


def _topk_mask(score, keep):
    """The keep largest FP32 scores of each row, ties to the lower index (values ordered as
    their bit patterns order them, -0 below +0)."""
    u = np.ascontiguousarray(score, dtype=np.float32).view(np.uint32).astype(np.int64)
    key = np.where(u & 0x80000000, 0xFFFFFFFF - u, u | 0x80000000)
    out = np.zeros(score.shape, bool)
    idx = np.arange(score.shape[1])
    for p in range(score.shape[0]):
        out[p, np.lexsort((idx, -key[p]))[:keep]] = True
    return out


def test_prefilter_selection_is_exact(ctx, fcc):
    """Keeping a template is an integer decision taken on the kernel's own FP32 scores: the
    mask is the top-keep of those scores, ties to the lower index, bit for bit; also for a
    blank frame (every score 0) and for a library whose templates all come in equal pairs."""
    ts, scan, lib = fcc
    lid = ctx.load_library(ts, 128, 360)
    K = ctx.library_info(lid)["n_templates"]
    frames = scan.frames[:40].copy()
    frames[5] = 0
    polar, norm, radial = ctx.polar_transform(_t(frames), 128, 360)
    for f in (0.5, 0.1, 0.97, 1e-4):
        mask, score = ctx.prefilter(lid, radial, f)
        sc = _np(score)
        assert np.all(sc[5] == 0)
        assert np.array_equal(_unpack(mask, K), _topk_mask(sc, O.keep_count(f, K))), f
    ctx.unload_library(lid)
    rt = synth.random_templates(synth.make_rng(4), 77)
    cnt = np.diff(rt.offsets)
    twice = np.repeat(np.arange(rt.n_templates), 2)
    sl = [np.arange(rt.offsets[k], rt.offsets[k + 1]) for k in twice]
    dup = synth.TemplateSet(offsets=np.concatenate([[0], np.cumsum(cnt[twice])]).astype(np.int64),
                            a=np.concatenate([rt.a[i] for i in sl]), b=np.concatenate([rt.b[i] for i in sl]),
                            intensity=np.concatenate([rt.intensity[i] for i in sl]))
    lid = ctx.load_library(dup, 60, 180)
    _, tscan, _ = synth.tiny_workload(n_side=4)
    polar, norm, radial = ctx.polar_transform(_t(tscan.frames), 60, 180)
    for f in (0.5, 0.3, 0.02):
        mask, score = ctx.prefilter(lid, radial, f)
        sc = _np(score)
        assert np.array_equal(sc[:, 0::2], sc[:, 1::2])
        assert np.array_equal(_unpack(mask, 2 * rt.n_templates), _topk_mask(sc, O.keep_count(f, 2 * rt.n_templates)))
    ctx.unload_library(lid)


# ------------------------------------------------------------------ whole path

def _hits(ctx, frames, lids, **kw):
    out = ctx.index(_t(frames), lids, **kw)
    return tmgb.hits_to_numpy(out)


def test_index_tiny_full(ctx, tiny):
    """The small workload in full: 256 patterns, 300 templates, 60 x 180, top-5."""
    ts, scan, lib, ref = tiny
    lid = ctx.load_library(ts, 60, 180)
    h = _hits(ctx, scan.frames, lid, top_n=5)[0]
    st = compare_hits(h, ref, lib)
    assert st["top1_same"] >= 0.99 * st["patterns"]
    ctx.unload_library(lid)


def test_index_fcc_prefilter(ctx, fcc):
    """Single phase, 256 x 256 u16 frames, 128 x 360, mirrors, pre-filter keeps 50 %.

    Templates whose FP64 pre-filter score lies within 1e-5 of the keep threshold may
    survive on one side only.  Where such a template would enter the oracle's top-N over
    the survivors plus those templates, the expected answer is not unique and the GPU's
    rows are checked for validity instead (every template eligible, every score equal to
    the oracle's Q for it); elsewhere the rows must match the oracle exactly."""
    ts, scan, lib = fcc
    lid = ctx.load_library(ts, 128, 360)
    N = 5
    ref = O.index(scan.frames, lib, prefilter_fraction=0.5, N=N)
    q_all, s_all = O.scores(ref["polar"], lib)
    _, sc = O.prefilter(ref["polar"], lib, 0.5)
    keep = O.keep_count(0.5, lib.K)
    h = _hits(ctx, scan.frames, lid, top_n=N, prefilter=0.5)[0]
    exact = []
    for p in range(scan.frames.shape[0]):
        thr = np.sort(sc[p])[::-1][keep - 1]
        amb = np.abs(sc[p] - thr) <= 1e-5 * max(abs(thr), 1e-3)
        elig = ref["active"][p] | amb
        tk, _, _ = O.top_n(q_all[p:p + 1], s_all[p:p + 1], N + 1, elig[None])
        if not np.any(amb[tk[0][tk[0] >= 0]]):
            exact.append(p)
            continue
        q_top = q_all[p][elig].max()
        for j in range(N):
            k = int(h["template_index"][p, j])
            assert k >= 0 and elig[k], (p, j, k)
            assert abs(h["score"][p, j] - q_all[p, k]) <= 1e-5 * max(abs(q_all[p, k]), 1e-3 * abs(q_top))
    assert len(exact) >= 0.9 * scan.frames.shape[0]
    compare_hits(h, ref, lib, patterns=exact)
    ctx.unload_library(lid)


def test_index_options_and_edges(ctx):
    rng = synth.make_rng(0, stream=7)
    ts = synth.random_templates(rng, 40, spots=(3, 12), r_range=(4.0, 30.0))
    ts.mirror = True
    scan = synth.render_scan(rng, ts, 20, 64, 72, n_theta=120, dtype=np.float32)
    frames = scan.frames
    for kw in [dict(top_n=3), dict(top_n=64), dict(top_n=100, subtract=0.4), dict(top_n=7, gamma=1.0),
               dict(top_n=5, unit=True), dict(top_n=2, prefilter=0.25)]:
        unit = kw.pop("unit", False)
        lib = O.prepare_library(ts, 32, 120, unit_intensity=unit)
        lid = ctx.load_library(ts, 32, 120, unit_intensity=unit)
        N = kw["top_n"]
        ref = O.index(frames, lib, gamma=kw.get("gamma", 0.5), subtract=kw.get("subtract", 0.0),
                      prefilter_fraction=kw.get("prefilter", 1.0), N=N)
        h = _hits(ctx, frames, lid, **kw)[0]
        compare_hits(h, ref, lib)
        ctx.unload_library(lid)


def test_index_per_pattern_centres(ctx, tiny):
    ts, scan, lib, ref = tiny
    rng = np.random.default_rng(9)
    n = 48
    centres = (np.array([63.5, 63.5]) + rng.uniform(-2.0, 2.0, size=(n, 2))).astype(np.float32)
    lid = ctx.load_library(ts, 60, 180)
    out = ctx.index(_t(scan.frames[:n]), lid, top_n=5, centres=_t(centres))
    h = tmgb.hits_to_numpy(out)[0]
    r = O.index(scan.frames[:n], lib, N=5, centres=centres.astype(np.float64))
    compare_hits(h, r, lib)
    ctx.unload_library(lid)


def test_index_zero_frames_and_single_pattern(ctx, tiny):
    ts, scan, lib, ref = tiny
    lid = ctx.load_library(ts, 60, 180)
    z = np.zeros((3, 128, 128), dtype=np.float32)
    h = _hits(ctx, z, lid, top_n=4)[0]
    # image norm 0: Q = 0 for every template, ranked by template index, shift 0
    assert np.all(h["template_index"] == np.arange(4)) and np.all(h["score"] == 0) and np.all(h["shift"] == 0)
    h1 = _hits(ctx, scan.frames[5:6], lid, top_n=5)[0]
    compare_hits(h1, {k: (v[5:6] if isinstance(v, np.ndarray) else v) for k, v in ref.items()}, lib)
    ctx.unload_library(lid)


def test_index_empty_batch(ctx, tiny):
    import torch
    ts, scan, lib, ref = tiny
    lid = ctx.load_library(ts, 60, 180)
    out = ctx.index(torch.zeros((0, 128, 128), dtype=torch.float32, device="cuda"), lid, top_n=5)
    assert out.shape == (1, 0, 5, 5)
    ctx.unload_library(lid)


def test_index_multi_library_equals_single(ctx):
    rng = synth.make_rng(2)
    a = synth.kinematic_library("fcc", step_deg=3.0)
    b = synth.kinematic_library("tetragonal", step_deg=3.0)
    scan = synth.render_scan(rng, b, 24, 256, 256, n_theta=360)
    la, lb = ctx.load_library(a, 128, 360), ctx.load_library(b, 128, 360)
    both = _hits(ctx, scan.frames, [la, lb], top_n=5)
    ha = _hits(ctx, scan.frames, la, top_n=5)[0]
    hb = _hits(ctx, scan.frames, lb, top_n=5)[0]
    assert np.array_equal(both[0], ha) and np.array_equal(both[1], hb)
    refb = O.index(scan.frames, O.prepare_library(b, 128, 360), N=5)
    compare_hits(hb, refb, O.prepare_library(b, 128, 360))
    ctx.unload_library(la)
    ctx.unload_library(lb)


def test_index_deterministic_alone_and_in_batch(ctx, tiny):
    ts, scan, lib, ref = tiny
    lid = ctx.load_library(ts, 60, 180)
    full = _hits(ctx, scan.frames, lid, top_n=5)[0]
    again = _hits(ctx, scan.frames, lid, top_n=5)[0]
    part = _hits(ctx, scan.frames[100:117], lid, top_n=5)[0]
    assert np.array_equal(full, again)
    assert np.array_equal(full[100:117], part)
    ctx.unload_library(lid)


def test_index_single_phase_full_size_sampled(ctx):
    """The single-phase scan at full size (16384 frames of 256 x 256, as the benchmark runs
    it) indexed in one call; 48 sampled patterns checked against the oracle."""
    ts, scan, prm = synth.single_phase_workload()
    lib = O.prepare_library(ts, 128, 360)
    lid = ctx.load_library(ts, 128, 360)
    h = _hits(ctx, scan.frames, lid, top_n=5, prefilter=1.0)[0]
    pick = np.sort(np.random.default_rng(0).choice(scan.frames.shape[0], 48, replace=False))
    ref = O.index(scan.frames[pick], lib, N=5)
    compare_hits(h[pick], ref, lib)
    ctx.unload_library(lid)


def test_index_graph_replay_equals_direct(ctx, tiny):
    """With the graph flag on a created stream, the second identical call is captured into a
    CUDA graph and later calls replay it; every result equals the direct call's."""
    import torch
    ts, scan, lib, ref = tiny
    lid = ctx.load_library(ts, 60, 180)
    f = _t(scan.frames)
    direct = _hits(ctx, scan.frames, lid, top_n=5)[0]
    s = torch.cuda.Stream()
    out = torch.empty((1, f.shape[0], 5, 5), dtype=torch.int32, device="cuda")
    with torch.cuda.stream(s):
        for _ in range(4):
            out.zero_()
            ctx.index(f, lid, top_n=5, out=out, stream=s, graph=True)
            s.synchronize()
            assert np.array_equal(tmgb.hits_to_numpy(out)[0], direct)
    assert ctx.last_stats["launches"] >= 2
    ctx.unload_library(lid)


def test_autotune_keeps_results(ctx, fcc, tmp_path, monkeypatch):
    """The autotuner only changes the sparse kernel's block size: results are identical."""
    ts, scan, lib = fcc
    monkeypatch.setenv("TMGB_TUNE_CACHE", str(tmp_path / "tune.txt"))
    c2 = tmgb.Context(0)
    lid = c2.load_library(ts, 128, 360)
    before = _hits(c2, scan.frames, lid, top_n=5, prefilter=0.5)
    best = c2.autotune(_t(scan.frames), lid, top_n=5, prefilter=0.5)
    assert best in (128, 256, 512)
    after = _hits(c2, scan.frames, lid, top_n=5, prefilter=0.5)
    assert np.array_equal(before, after)
    c2.close()
    assert (tmp_path / "tune.txt").read_text().split()[1] == str(best)


def test_refined_angles_match_oracle_and_reduce_error(ctx, tiny):
    """TM_INDEX_REFINE: templates, shifts and scores unchanged; the sub-step angle equals the
    oracle's parabola vertex (evaluated at the GPU's own hits) within the propagation of the
    Q tolerance; on the tiny scan (2 degree polar step, continuous true angles) it lowers the
    angle error of correctly indexed patterns."""
    ts, scan, lib, ref = tiny
    lid = ctx.load_library(ts, 60, 180)
    plain = _hits(ctx, scan.frames, lid, top_n=5)[0]
    fine = _hits(ctx, scan.frames, lid, top_n=5, refine=True)[0]
    for f in ("template_index", "shift", "score", "mirror"):
        assert np.array_equal(plain[f], fine[f])
    a_ref = O.refine_angles(ref["polar"], lib, fine["template_index"].astype(np.int64), fine["shift"].astype(np.int64))
    step = 360.0 / 180
    nP = np.sqrt((ref["polar"] ** 2).sum(axis=(1, 2)))
    for p in range(scan.frames.shape[0]):
        for j in range(5):
            k, s = int(fine["template_index"][p, j]), int(fine["shift"][p, j])
            d = nP[p] * lib.norm[k]
            q = [sum(lib.I[i] * ref["polar"][p, lib.ri[i], (lib.ti[i] + s + ds) % 180]
                     for i in range(lib.off[k], lib.off[k + 1])) / d for ds in (-1, 0, 1)]
            curv = abs(q[0] - 2 * q[1] + q[2])
            tol = step * (min(0.5, 5e-5 * abs(q[1]) / max(curv, 1e-30)) + 1e-5)
            assert abs(fine["angle_deg"][p, j] - a_ref[p, j]) <= tol, (p, j, fine["angle_deg"][p, j], a_ref[p, j])
    ok = fine["template_index"][:, 0] == scan.template
    true_deg = np.degrees(scan.angle) % 360.0

    def err(a):
        return np.abs((a - true_deg + 180.0) % 360.0 - 180.0)

    e_plain, e_fine = err(plain["angle_deg"][:, 0])[ok], err(fine["angle_deg"][:, 0])[ok]
    assert e_fine.mean() < e_plain.mean(), (e_fine.mean(), e_plain.mean())
    ctx.unload_library(lid)


def _topn_from_scores(q, s, active, N):
    """Top-N by (Q desc, template asc) over the active templates of each pattern."""
    n, K = q.shape
    tk = np.full((n, N), -1, np.int64)
    ts_ = np.full((n, N), -1, np.int64)
    tq = np.full((n, N), -np.inf, np.float32)
    for p in range(n):
        idx = np.flatnonzero(active[p])
        order = idx[np.lexsort((idx, -q[p, idx].astype(np.float64)))][:N]
        tk[p, :len(order)], ts_[p, :len(order)], tq[p, :len(order)] = order, s[p, order], q[p, order]
    return tk, ts_, tq


@pytest.mark.parametrize("which,prefilter,subtract", [("fcc", 0.5, 0.0), ("fcc", 1.0, 0.3), ("hcp", 0.5, 0.0),
                                                    ("hcp", 1.0, 0.0), ("hcp", 1.0, 0.3)])
def test_bound_pruning_is_exact(ctx, which, prefilter, subtract):
    """The fused top-N skips templates whose bound cannot reach the running N-th best; its hits
    equal, bit for bit, the top-N taken from every template's score computed without skipping
    (tm_correlate) on the same polar images and the same pre-filter mask."""
    ts = synth.kinematic_library(which, step_deg=1.0)
    rng = synth.make_rng(9)
    scan = synth.render_scan(rng, ts, 48, 256, 256, n_theta=360)
    lid = ctx.load_library(ts, 128, 360)
    K = ctx.library_info(lid)["n_templates"]
    f = _t(scan.frames)
    ctx.profile_enable(True)
    hits = tmgb.hits_to_numpy(ctx.index(f, lid, top_n=5, prefilter=prefilter, subtract=subtract))[0]
    _, counters = ctx.profile_read(counters=True)
    ctx.profile_enable(False)
    polar, norm, radial = ctx.polar_transform(f, 128, 360, subtract=subtract)
    mask = None
    active = np.ones((48, K), bool)
    if prefilter < 1.0:
        mask, _ = ctx.prefilter(lid, radial, prefilter)
        bits = np.unpackbits(mask.cpu().numpy().view(np.uint8), bitorder="little").reshape(48, -1)
        active = bits[:, :K].astype(bool)
    q, s = ctx.correlate(lid, polar, norm, mask=mask)
    tk, tsh, tq = _topn_from_scores(q.cpu().numpy(), s.cpu().numpy(), active, 5)
    assert np.array_equal(hits["template_index"], tk)
    assert np.array_equal(hits["shift"], tsh)
    assert np.array_equal(hits["score"], tq)
    # the executed multiply-adds: at most every surviving template's spots x shifts, and at
    # least those of the templates in the top-N (they are always scored)
    exp = ctx.library_export(lid)
    work_k = np.diff(exp["offsets"]).astype(np.int64) * (360 // exp["order"].astype(np.int64))
    full = int((active.astype(np.int64) @ work_k).sum())
    held = int(work_k[tk[tk >= 0]].sum())
    assert held <= counters["sparse_macs"] <= full, (held, counters["sparse_macs"], full)
    ctx.unload_library(lid)


@pytest.mark.parametrize("tile", [2, 4])
def test_tiled_bound_pass_is_exact(ctx, tile, tmp_path, monkeypatch):
    """Patterns bounded together in tiles (the unmasked pruned top-N; the tile forced through the
    tuning cache a new context reads back) give, bit for bit, the top-N taken from every
    template's score computed without skipping, for one library and for two in one call, with
    a partial last tile."""
    import torch
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TMGB_TUNE_CACHE", str(cache))
    libs = [synth.kinematic_library("hcp", step_deg=1.0), synth.kinematic_library("fcc", step_deg=1.0)]
    rng = synth.make_rng(21)
    scan = synth.render_scan(rng, libs[0], 50, 256, 256, n_theta=360)
    f = _t(scan.frames)
    for sets in ([0], [0, 1]):
        c1 = tmgb.Context(0)
        ids = [c1.load_library(libs[i], 128, 360) for i in sets]
        c1.autotune(f, ids, top_n=5)
        c1.close()
        # force the tile on the cached shape (key threads seeds tile ms)
        lines = [ln.split() for ln in cache.read_text().splitlines() if ln.strip()]
        key, threads, seeds = lines[-1][0], lines[-1][1], lines[-1][2]
        cache.write_text(f"{key} {threads} {seeds} {tile} 0.0\n")
        c2 = tmgb.Context(0)
        ids = [c2.load_library(libs[i], 128, 360) for i in sets]
        hits = tmgb.hits_to_numpy(c2.index(f, ids, top_n=5))
        c2.check()
        polar, norm, _ = c2.polar_transform(f, 128, 360)
        for li, lid in enumerate(ids):
            K = c2.library_info(lid)["n_templates"]
            q, s_ = c2.correlate(lid, polar, norm)
            tk, tsh, tq = _topn_from_scores(q.cpu().numpy(), s_.cpu().numpy(), np.ones((50, K), bool), 5)
            assert np.array_equal(hits[li]["template_index"], tk), (sets, li)
            assert np.array_equal(hits[li]["shift"], tsh), (sets, li)
            assert np.array_equal(hits[li]["score"], tq), (sets, li)
        c2.close()
        cache.unlink()
    torch.cuda.synchronize()
