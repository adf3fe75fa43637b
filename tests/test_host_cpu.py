"""CPU tests of the CUDA library's host side: it loads, exports every declared symbol, and
puts templates on the polar grid exactly as the oracle does (integer work: bit-exact)."""
import math
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_07347_gb300 import synth
from paper_2111_07347_gb300 import tmgb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_07347_gb300 import build
    build.build()
    return tmgb.library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tmgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(tm_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(tmgb.exported_symbols()) | {"tm_index_params_default"}


def test_create_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tmgb.TmError) as e:
        tmgb.tm_create(0)
    assert e.value.code in (tmgb.TM_ERR_CUDA, tmgb.TM_ERR_INVALID_ARG, tmgb.TM_ERR_UNSUPPORTED)


def _same(h, ref):
    assert np.array_equal(h["offsets"], ref.off)
    assert np.array_equal(h["r"], ref.ri)
    assert np.array_equal(h["t"], ref.ti)
    assert np.allclose(h["intensity"], ref.I, rtol=6e-8, atol=0)
    assert np.allclose(h["norm"], ref.norm, rtol=6e-8, atol=0)


@pytest.mark.parametrize("n_r,n_theta,dr", [(60, 180, 1.0), (32, 90, 2.0), (61, 7, 1.0)])
def test_prepare_random_templates_matches_oracle(lib, n_r, n_theta, dr):
    ts, _, _ = synth.tiny_workload(n_side=1)
    h = tmgb.tm_library_prepare_host(ts, n_r, n_theta, dr)
    _same(h, O.prepare_library(ts, n_r, n_theta, dr))


@pytest.mark.parametrize("unit", [False, True])
def test_prepare_kinematic_mirror_matches_oracle(lib, unit):
    ts = synth.kinematic_library("hcp", step_deg=2.0)
    h = tmgb.tm_library_prepare_host(ts, 128, 360, unit_intensity=unit)
    ref = O.prepare_library(ts, 128, 360, unit_intensity=unit)
    _same(h, ref)
    assert h["info"]["mirror"] == 1 and h["info"]["n_templates"] == 2 * ts.n_templates


def test_prepare_drops_out_of_grid_and_merges(lib):
    ts = synth.TemplateSet(np.array([0, 5]), np.array([3.0, 3.2, 9.6, 4.0, 0.2]),
                           np.array([0.0, 0.001, 1.0, -math.pi / 2, 2.0]), np.array([1.0, 2.0, 3.0, 4.0, 5.0]))
    h = tmgb.tm_library_prepare_host(ts, 8, 4)
    _same(h, O.prepare_library(ts, 8, 4))
    assert h["info"]["n_spots"] == 3          # (3,0) merged, 9.6 -> 10 dropped, (4,3), (0,*)


def test_rotational_order_is_a_true_period(lib):
    """A template reported with order n has Q(s + n_theta/n) == Q(s) for every pattern
    (checked with the oracle's Q table), and order 1 templates are not periodic."""
    rng = np.random.default_rng(1)
    base = np.array([4.0, 6.0, 6.0])
    th = np.array([0.2, 1.0, 2.5])
    # template 0: 3-fold copy; template 1: 2-fold; template 2: generic
    r = np.concatenate([np.tile(base, 3), np.tile(base, 2), base])
    t = np.concatenate([np.concatenate([th + i * 2 * math.pi / 3 for i in range(3)]),
                        np.concatenate([th + i * math.pi for i in range(2)]), th])
    I = np.concatenate([np.tile([1.0, 2.0, 3.0], 3), np.tile([1.0, 2.0, 3.0], 2), [1.0, 2.0, 3.0]])
    ts = synth.TemplateSet(np.array([0, 9, 15, 18]), r, t, I)
    h = tmgb.tm_library_prepare_host(ts, 8, 36)
    ref = O.prepare_library(ts, 8, 36)
    _same(h, ref)
    assert list(h["order"]) == [3, 2, 1]
    full = O.scores_full(rng.random((2, 8, 36)), ref)
    for k, n in enumerate(h["order"]):
        per = 36 // n
        assert np.allclose(full[:, k], np.roll(full[:, k], per, axis=1), atol=1e-14) == (n > 1) or n == 1


@pytest.mark.parametrize("bad", ["n_r", "theta", "dr", "offsets", "nan"])
def test_prepare_rejects_bad_descriptor(lib, bad):
    ts = synth.TemplateSet(np.array([0, 2]), np.array([3.0, 4.0]), np.array([0.0, 1.0]), np.array([1.0, 1.0]))
    kw = dict(n_r=8, n_theta=36, dr=1.0)
    if bad == "n_r":
        kw["n_r"] = 0
    elif bad == "theta":
        kw["n_theta"] = 5000
    elif bad == "dr":
        kw["dr"] = -1.0
    elif bad == "offsets":
        ts.offsets = np.array([0, 3])
        ts.a = np.array([3.0, 4.0, 5.0])
        ts.b = np.array([0.0, 1.0, 2.0])
        ts.intensity = np.array([1.0, 1.0, 1.0])
        ts.offsets = np.array([1, 3])
    elif bad == "nan":
        ts.a = np.array([3.0, np.nan])
    with pytest.raises(tmgb.TmError) as e:
        tmgb.tm_library_prepare_host(ts, **kw)
    assert e.value.code == tmgb.TM_ERR_INVALID_ARG


def _round_nb(nb):
    return nb if nb <= 4 else 6 if nb <= 6 else 8 if nb <= 8 else 12 if nb <= 12 else 16 if nb <= 16 \
        else 24 if nb <= 24 else 32


def _pitch(n_theta, layout):
    """Row pitch of the sparse kernel's shared-memory rows.  dual: two copies of each row (the
    second shifted by one column), n_theta + 64 NB2 columns rounded up to even; wrap-free:
    n_theta + 32 NB; wrapped: n_theta + 32 and at least 32 NB (NB2, NB the rounded 64- and
    32-wide block counts)."""
    if layout == "dual":
        p = n_theta + 64 * _round_nb((n_theta + 63) // 64)
        return p + (p & 1)
    nb = _round_nb((n_theta + 31) // 32)
    return n_theta + 32 * nb if layout == "wf" else max(n_theta + 32, 32 * nb)


@pytest.mark.parametrize("which", ["random", "fcc", "hcp", "odd"])
def test_sparse_layout_reads_stay_in_bounds(lib, which):
    """Replay the sparse kernel's shared-memory indexing on the CPU for every spot, lane and
    shift block, in all three row layouts: the spot words decode to the spot's angle column
    and its row among the library's distinct radii (wrapped layout) or to its precomputed
    offsets (dual and wrap-free layouts); every address stays inside the rows; the value read
    is the polar sample at (t + s) mod n_theta for the lane's shift s, given how each layout
    fills its rows (column c of a row holds P'[c mod n_theta]; the second dual copy holds
    P'[(c + 1) mod n_theta])."""
    if which == "random":
        ts, _, _ = synth.tiny_workload(n_side=1)
        n_r, n_theta = 60, 180
    elif which == "odd":
        ts, _, _ = synth.tiny_workload(n_side=1)
        n_r, n_theta = 61, 77
    else:
        ts = synth.kinematic_library(which, step_deg=3.0)
        n_r, n_theta = 128, 360
    h = tmgb.tm_library_prepare_host(ts, n_r, n_theta)
    radii = np.unique(h["r"])
    n_rad = max(1, radii.size)
    word = h["packed"].astype(np.int64) & 0xFFFFFFFF
    t = word & 0x7FF
    row = (word >> 11) & 0x1FFF
    w = word >> 24
    assert np.array_equal(radii[row], h["r"])
    assert np.array_equal(t, h["t"])
    assert np.array_equal(w, (n_theta - h["t"] + 31) // 32)
    w2 = h["packed2"].astype(np.int64) & 0xFFFFFFFF
    off_d, off_w = w2 & 0xFFFF, w2 >> 16
    pd, pw = _pitch(n_theta, "dual"), _pitch(n_theta, "wf")
    dual_ok, wf_ok = 2 * n_rad * pd <= 65535, n_rad * pw <= 65535
    if dual_ok:
        assert np.array_equal(off_d, np.where(t & 1, n_rad + row, row) * pd + (t & ~1))
    if wf_ok:
        assert np.array_equal(off_w, row * pw + t)
    lanes = np.arange(32)
    for layout in ("dual", "wf", "wrap"):
        if (layout == "dual" and not dual_ok) or (layout == "wf" and not wf_ok):
            continue
        pitch = _pitch(n_theta, layout)
        rows = 2 * n_rad if layout == "dual" else n_rad
        bw = 64 if layout == "dual" else 32
        for k in range(h["info"]["n_templates"]):
            S = n_theta // h["order"][k]
            nb = _round_nb((S + bw - 1) // bw)
            for i in range(h["offsets"][k], h["offsets"][k + 1]):
                for b in range(nb):
                    if layout == "dual":
                        for e in (0, 1):
                            addr = off_d[i] + 2 * lanes + 64 * b + e          # float index
                            r_, col = addr // pitch, addr % pitch
                            assert np.all(addr < rows * pitch) and np.all(r_ < rows), (k, i, b)
                            assert off_d[i] % 2 == 0 and np.all(r_ == r_[0])
                            src_row = r_[0] % n_rad
                            assert src_row == row[i]
                            val_col = (col + (1 if r_[0] >= n_rad else 0)) % n_theta
                            assert np.array_equal(val_col, (t[i] + 2 * lanes + 64 * b + e) % n_theta)
                    else:
                        if layout == "wf":
                            col = off_w[i] - row[i] * pitch + 32 * b + lanes
                        else:
                            col = t[i] + 32 * b - (n_theta if b >= w[i] else 0) + lanes
                        assert np.all((col >= 0) & (col < pitch)), (layout, k, i, b)
                        assert row[i] * pitch + col.max() < rows * pitch
                        # column c of a row holds P'[c mod n_theta]
                        assert np.array_equal(col % n_theta, (t[i] + 32 * b + lanes) % n_theta)
        # pruning windows: the spot word decodes (FP32 row division, as in the kernel) to the
        # spot's row and column; the window maxima cw[row][j], j = (t + h ww) / 32 for the
        # three windows h, lie inside [n_rad][nchw] and their ncov chunks cover the window
        ww = (n_theta + 2) // 3
        ncov = (ww + 31) // 32 + 1
        nchw = ((n_theta - 1 + 2 * ww) >> 5) + 1
        inv = np.float32(1.0) / np.float32(pitch)
        for i in range(len(word)):
            if layout == "wrap":
                r_dec, t_dec = row[i], t[i]
            else:
                off = off_d[i] if layout == "dual" else off_w[i]
                rr = int((np.float32(off) + np.float32(0.5)) * inv)
                r_dec, t_dec = rr, off - rr * pitch
                if layout == "dual" and rr >= n_rad:
                    r_dec, t_dec = rr - n_rad, t_dec + 1
            assert r_dec == row[i] and t_dec == t[i], (layout, i)
            for hw in range(3):
                s0 = t_dec + hw * ww
                j = s0 >> 5
                assert 0 <= j < nchw and r_dec * nchw + j < n_rad * nchw, (layout, i, hw)
                assert 32 * j <= s0 and s0 + ww <= 32 * (j + ncov)
        assert 3 * ww >= n_theta


def _polar_launch(n_theta, staged=True, max_threads=768):
    """Thread shape of the polar kernel: row groups of cols = 32 ceil(n_theta / 32) threads,
    R = min(4, 768 / cols) groups when the frame is staged, else one group of at most 768."""
    cols = (n_theta + 31) // 32 * 32
    if staged and cols <= max_threads:
        R = max(1, min(4, max_threads // cols))
        return cols, R
    return min(cols, max_threads), 1


@pytest.mark.parametrize("n_r,n_theta,staged", [(128, 360, True), (60, 180, True), (30, 7, True), (1, 1, True),
                                                (61, 77, True), (26, 1000, False), (128, 360, False),
                                                (130, 361, True)])
def test_polar_thread_mapping_covers_grid(n_r, n_theta, staged):
    """Replay the polar kernel's work split on the CPU: a warp samples 8 angles (lane & 7) by
    4 rows (lane >> 3); thread (group g, warp-in-group wg, lane) takes columns
    8 wg + (lane & 7) + i cols / 4 and rows (lane >> 3) + 4 g + m 4 R.  Every sample of the
    n_r x n_theta grid is taken exactly once; in each pass over the columns every warp of a
    row's group (g = (j / 4) mod R) writes that row's partial sum exactly once, from an even
    lane of the row's group of eight, which the radial sums then add over the group's warps."""
    cols, R = _polar_launch(n_theta, staged)
    threads = cols * R
    seen = np.zeros((n_r, n_theta), dtype=np.int64)
    part = {}
    for tid in range(threads):
        lane, warp = tid & 31, tid >> 5
        g, t_in = tid // cols, tid % cols
        k0, kstep = 8 * (t_in >> 5) + (lane & 7), cols >> 2
        row0, rstep = (lane >> 3) + 4 * g, 4 * R
        wrows = -(-(n_r - 4 * g) // rstep) if 4 * g < n_r else 0
        mine = -(-(n_r - row0) // rstep) if row0 < n_r else 0
        assert mine <= wrows
        for kk in range(0, n_theta, kstep):
            k = kk + k0
            for b in range(0, wrows, 4):
                nu = mine - b
                j0 = row0 + rstep * b
                if k < n_theta and nu > 0:
                    for u in range(min(4, nu)):
                        seen[j0 + rstep * u, k] += 1
                kl = lane & 7
                u = ((kl >> 2) & 1) * 2 + ((kl >> 1) & 1)
                if kl % 2 == 0 and u < nu:
                    key = (kk, j0 + rstep * u, warp)
                    assert key not in part and j0 + rstep * u < n_r
                    part[key] = True
    assert np.all(seen == 1)
    wpg = cols // 32
    for j in range(n_r):
        g0 = (j >> 2) % R
        for w in range(g0 * wpg, (g0 + 1) * wpg):
            for kk in range(0, n_theta, cols >> 2):
                assert (kk, j, w) in part, (j, w, kk)


@pytest.mark.parametrize("field,value,needle", [("pixel_mask", 0x1001, "pixel_mask"),
                                                 ("threshold", -1.0, "threshold"),
                                                 ("path", tmgb.TM_PATH_BF16_RESCORE, "FP32 sparse"),
                                                 ("prefilter_fraction", 0.5, "FP32 sparse")])
def test_noalloc_rejects_bad_params_before_launch(lib, field, value, needle):
    """The allocation-free entry point validates its parameters on the host, before any
    device work (here with no context and no GPU): a misaligned mask, a negative threshold,
    the BF16 path and a pre-filter are refused with TM_ERR_INVALID_ARG."""
    import ctypes
    f = lib.tm_index_patterns_noalloc
    p = tmgb.make_params(top_n=5)
    setattr(p, field, value)
    rc = f(None, ctypes.byref(p), None, tmgb.TM_DTYPE_U16, 4, 256, 256, 0, None, None)
    assert rc == tmgb.TM_ERR_INVALID_ARG
    assert needle in tmgb.tm_last_error()


@pytest.mark.parametrize("which", ["random", "fcc", "hcp"])
def test_sorted_bound_entries_cover_every_spot(which):
    """The second copy of the pruning-window entries that the unmasked top-N pass reads. The
    order must be a permutation of the templates by spot count, most first, ties by library
    index. For spot i of the template at position 32 w + l the kernel reads entry
    word_start[w] + 32 i + l. That entry must stay below the next word's start and hold the
    spot's intensity bits and window-table entries, recomputed here from the spot's radius row
    and angle column. Every table index must lie inside the rows x chunks table, and every
    other entry must be zero."""
    if which == "random":
        ts, _, _ = synth.tiny_workload(n_side=1)
        n_r, n_theta = 60, 180
    else:
        ts = synth.kinematic_library(which, step_deg=3.0)
        n_r, n_theta = 128, 360
    h = tmgb.tm_library_prepare_host(ts, n_r, n_theta)
    e = tmgb.tm_library_bound_entries_host(ts, n_r, n_theta)
    off = h["offsets"]
    K = off.size - 1
    cnt = np.diff(off)
    nw = (K + 31) // 32
    order, ws, ent = e["order"], e["word_start"], e["entries"]
    assert order.size == 32 * nw and ws.size == nw
    perm = order[:K]
    assert np.array_equal(perm, np.lexsort((np.arange(K), -cnt)))
    radii = np.unique(h["r"])
    rows = np.searchsorted(radii, h["r"]).astype(np.int64)
    t = h["t"].astype(np.int64)
    ww = (n_theta + 2) // 3
    nchw = ((n_theta - 1 + 2 * ww) >> 5) + 1
    j0 = rows * nchw + (t >> 5)
    d1 = ((t + ww) >> 5) - (t >> 5)
    d2 = ((t + 2 * ww) >> 5) - (t >> 5)
    assert (j0 + d2 < radii.size * nchw).all()
    word = j0 | (d1 << 16) | (d2 << 24)
    ibits = h["intensity"].view(np.int32)
    ends = np.append(ws[1:], ent.shape[0])
    seen = np.zeros(ent.shape[0], bool)
    for pos in range(K):
        w, lane = divmod(pos, 32)
        k = perm[pos]
        idx = ws[w] + 32 * np.arange(cnt[k]) + lane
        assert (idx < ends[w]).all()
        assert np.array_equal(ent[idx, 0], ibits[off[k]:off[k + 1]])
        assert np.array_equal(ent[idx, 1].astype(np.int64) & 0xFFFFFFFF, word[off[k]:off[k + 1]])
        seen[idx] = True
    assert not ent[~seen].any()
