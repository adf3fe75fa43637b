"""Pins for the FP64 oracle: closed forms, invariants, brute force and the paper's worked
example.  None of these compares the oracle with itself; each would fail on a plausible
mistake (dropped term, wrong sign or index, swapped axes, wrong tie rule)."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_07347_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_lib(rng, K=6, n_r=12, n_theta=24, spots=(2, 5), mirror=False):
    ts = synth.random_templates(rng, K, spots=spots, r_range=(1.0, n_r - 1.5))
    ts.mirror = mirror
    return ts, O.prepare_library(ts, n_r, n_theta, 1.0, mirror=mirror)


# ------------------------------------------------------------------ Eq. 1 itself

def test_brute_force_tiny_all_shifts():
    """Q(k, s) from the dense template image and np.roll, written out per (k, s), equals the
    oracle's sparse loop; argmax / lowest-shift / lowest-template rules hold."""
    rng = np.random.default_rng(7)
    n_r, n_theta = 8, 8
    ts = synth.random_templates(rng, 3, spots=(1, 4), r_range=(0.0, 7.4))
    lib = O.prepare_library(ts, n_r, n_theta)
    P = rng.random((2, n_r, n_theta))
    full = O.scores_full(P, lib)
    for p in range(2):
        nP = math.sqrt(sum(P[p, j, k] ** 2 for j in range(n_r) for k in range(n_theta)))
        for k in range(lib.K):
            T = np.zeros((n_r, n_theta))
            for i in range(lib.off[k], lib.off[k + 1]):
                T[lib.ri[i], lib.ti[i]] += lib.I[i]
            nT = math.sqrt(float((T * T).sum()))
            for s in range(n_theta):
                num = 0.0
                for j, t in itertools.product(range(n_r), range(n_theta)):
                    num += T[j, t] * P[p, j, (t + s) % n_theta]
                assert abs(full[p, k, s] - num / (nP * nT)) < 1e-12
    q, sb = O.scores(P, lib)
    for p in range(2):
        for k in range(lib.K):
            assert q[p, k] == pytest.approx(full[p, k].max(), abs=1e-15)
            assert sb[p, k] == int(np.argmax(full[p, k]))


def test_q_equals_one_for_rolled_template():
    """Cauchy-Schwarz: Q <= 1 with equality iff P is proportional to the template image
    shifted by m columns; the oracle must return (k, m) with Q = 1."""
    rng = np.random.default_rng(11)
    ts, lib = _small_lib(rng, K=8, n_r=16, n_theta=36, spots=(3, 7))
    for k, m in [(0, 0), (3, 5), (7, 35)]:
        T = lib.dense(k)
        P = 2.5 * np.roll(T, m, axis=1)[None]          # P[r, t + m] = T[r, t]
        q, s = O.scores(P, lib)
        assert abs(q[0, k] - 1.0) < 1e-12
        assert s[0, k] == m
        assert np.all(q[0] <= 1.0 + 1e-12)
        tk, tsh, tq = O.top_n(q, s, 3)
        assert tk[0, 0] == k and tsh[0, 0] == m


def test_q_bound_and_sign():
    rng = np.random.default_rng(3)
    ts, lib = _small_lib(rng, K=10, n_r=10, n_theta=20)
    P = rng.normal(size=(4, 10, 20))
    q, _ = O.scores(P, lib)
    assert np.all(q <= 1 + 1e-12) and np.all(q >= -1 - 1e-12)
    q2, _ = O.scores(-P, lib)
    full = O.scores_full(P, lib)
    assert np.allclose(q2, -full.min(axis=2), atol=1e-14)


def test_linearity_gamma_one():
    """With gamma = 1 and no subtraction, scaling the frame leaves Q unchanged."""
    ts, scan, prm = synth.tiny_workload(n_side=2)
    lib = O.prepare_library(ts, 60, 180)
    P1 = O.polar(scan.frames, 60, 180, gamma=1.0)
    P2 = O.polar(scan.frames * np.float32(3.0), 60, 180, gamma=1.0)
    q1, s1 = O.scores(P1, lib)
    q2, s2 = O.scores(P2, lib)
    assert np.allclose(q1, q2, rtol=1e-12, atol=1e-14)
    assert np.array_equal(s1, s2)


# ------------------------------------------------------------------ polar transform

def test_polar_constant_and_gamma_subtract():
    f = np.full((1, 32, 32), 9.0, dtype=np.float32)
    P = O.polar(f, 14, 40, gamma=1.0)
    assert np.allclose(P, 9.0, atol=1e-12)
    P = O.polar(f, 14, 40, gamma=0.5, subtract=0.25)
    assert np.allclose(P, 3.0 - 0.25, atol=1e-12)


def test_polar_linear_ramp_is_exact():
    """Bilinear interpolation reproduces a linear function: P(r, theta) =
    a (cx + r cos theta) + b (cy + r sin theta) + d  (x = column, y = row)."""
    H, W = 40, 48
    a, b, d = 0.75, -1.25, 100.0
    yy, xx = np.mgrid[0:H, 0:W]
    f = (a * xx + b * yy + d).astype(np.float32)[None]
    n_r, n_theta = 18, 72
    P = O.polar(f, n_r, n_theta, gamma=1.0)
    cx, cy = (W - 1) / 2, (H - 1) / 2
    for j in range(n_r):
        for k in range(n_theta):
            th = 2 * math.pi * k / n_theta
            want = a * (cx + j * math.cos(th)) + b * (cy + j * math.sin(th)) + d
            assert abs(P[0, j, k] - want) < 1e-9


def test_polar_centre_and_gamma_order():
    """r = 0 samples the centre: with the default centre ((W-1)/2, (H-1)/2) it is the mean of
    the four central pixels after gamma (gamma first, then resampling)."""
    f = np.zeros((1, 6, 6), dtype=np.float32)
    f[0, 2, 2], f[0, 2, 3], f[0, 3, 2], f[0, 3, 3] = 1.0, 4.0, 9.0, 16.0
    P = O.polar(f, 2, 12, gamma=0.5)
    assert np.allclose(P[0, 0], (1 + 2 + 3 + 4) / 4.0, atol=1e-12)


def test_polar_zero_outside_frame():
    f = np.ones((1, 8, 8), dtype=np.float32)
    P = O.polar(f, 5, 4, gamma=1.0)       # r = 4, theta = 0: x = 7.5 -> half the taps outside
    assert abs(P[0, 4, 0] - 0.5) < 1e-12
    assert abs(P[0, 4, 2] - 0.5) < 1e-12  # theta = pi: x = -0.5


def test_rotation_equivariance_rot90():
    """np.rot90 with the default centre rolls the polar image by n_theta/4 columns, so the
    best template and its Q are unchanged and the shift moves by -n_theta/4."""
    ts, scan, prm = synth.tiny_workload(n_side=3)
    lib = O.prepare_library(ts, 60, 180)
    f = scan.frames
    fr = np.ascontiguousarray(np.rot90(f, k=1, axes=(1, 2)))
    P, Pr = O.polar(f, 60, 180), O.polar(fr, 60, 180)
    assert np.allclose(Pr, np.roll(P, -45, axis=2), atol=1e-9)
    q, s = O.scores(P, lib)
    qr, sr = O.scores(Pr, lib)
    assert np.allclose(q, qr, rtol=1e-10, atol=1e-13)
    b = np.argmax(q, axis=1)
    br = np.argmax(qr, axis=1)
    assert np.array_equal(b, br)
    rows = np.arange(len(b))
    assert np.array_equal(sr[rows, br], (s[rows, b] - 45) % 180)


def test_mirror_flip_equivariance():
    """A vertical flip (y -> H-1-y) reflects the pattern across y = 0, so template k scores on
    the flipped frame what its mirror k +- K0 scores on the original, at shift -s."""
    rng = synth.make_rng(0)
    ts = synth.random_templates(rng, 40)
    ts.mirror = True
    scan = synth.render_scan(rng, ts, 6, 128, 128, n_theta=180, dtype=np.float32)
    lib = O.prepare_library(ts, 60, 180, mirror=True)
    K0 = lib.K0
    f = scan.frames
    ff = np.ascontiguousarray(f[:, ::-1, :])
    q, s = O.scores(O.polar(f, 60, 180), lib)
    qf, sf = O.scores(O.polar(ff, 60, 180), lib)
    perm = np.concatenate([np.arange(K0, 2 * K0), np.arange(K0)])
    assert np.allclose(qf, q[:, perm], rtol=1e-9, atol=1e-12)
    b = np.argmax(q, axis=1)
    bf = np.argmax(qf, axis=1)
    assert np.array_equal(bf, perm[b])
    rows = np.arange(len(b))
    assert np.array_equal(sf[rows, bf], (-s[rows, b]) % 180)


# ------------------------------------------------------------------ library preparation

def test_round_spot_rules():
    assert O.round_spot(2.5, 0.0, 360, 1.0) == (3, 0)       # half-way rounds up
    assert O.round_spot(2.49, 0.0, 360, 1.0) == (2, 0)
    assert O.round_spot(5.0, math.pi, 180, 1.0) == (5, 90)
    assert O.round_spot(5.0, -1e-9, 360, 1.0) == (5, 0)     # wraps to [0, 2pi) then rounds to 360 -> 0
    assert O.round_spot(5.0, -math.pi / 2, 4, 1.0) == (5, 3)
    assert O.round_spot(7.0, 0.0, 8, 2.0) == (4, 0)          # dr = 2 px


def test_golden_angle_step():
    """Section 2.2 worked example: a polar image 360 pixels wide gives a 1 degree in-plane step."""
    rows = [ln.split("#")[0].split() for ln in open(os.path.join(GOLDEN, "angle_step.txt"))]
    rows = [r for r in rows if r]
    for n_theta, step_deg in rows:
        n_theta, step_deg = int(n_theta), float(step_deg)
        # a template spot at angle step_deg degrees rounds to column 1
        assert O.round_spot(10.0, math.radians(step_deg), n_theta, 1.0) == (10, 1)
        ts = synth.TemplateSet(np.array([0, 1]), np.array([10.0]), np.array([0.0]), np.array([1.0]))
        lib = O.prepare_library(ts, 12, n_theta)
        P = np.roll(lib.dense(0), 1, axis=1)[None]
        tk, tsh, tq = O.top_n(*O.scores(P, lib), 1)
        assert tsh[0, 0] * 360.0 / n_theta == pytest.approx(step_deg)


def test_prepare_merge_drop_mirror_unit():
    ts = synth.TemplateSet(
        offsets=np.array([0, 4]),
        a=np.array([0.10, 0.101, 0.05, 2.0]),        # 1/A; px_per_unit 100 -> 10, 10.1, 5, 200 px
        b=np.array([0.0, 0.0, 0.05, 0.0]),
        intensity=np.array([2.0, 3.0, 5.0, 7.0]),
        coords="xy", px_per_unit=100.0, mirror=True)
    lib = O.prepare_library(ts, 64, 360)
    assert lib.K == 2 and lib.K0 == 1
    sp0 = sorted(zip(lib.ri[:lib.off[1]], lib.ti[:lib.off[1]], lib.I[:lib.off[1]]))
    # first two spots merge at (10, 0); (5, 5) at 45 deg -> (7, 45); 200 px dropped
    assert sp0 == [(7, 45, 5.0), (10, 0, 5.0)]
    sp1 = sorted(zip(lib.ri[lib.off[1]:], lib.ti[lib.off[1]:], lib.I[lib.off[1]:]))
    assert sp1 == [(7, 315, 5.0), (10, 0, 5.0)]            # mirror: ky -> -ky
    assert lib.norm[0] == pytest.approx(math.sqrt(50.0))
    assert lib.radial[0, 10] == 5.0 and lib.radial[0, 7] == 5.0
    libu = O.prepare_library(ts, 64, 360, unit_intensity=True)
    sp = sorted(zip(libu.ri[:libu.off[1]], libu.ti[:libu.off[1]], libu.I[:libu.off[1]]))
    assert sp == [(7, 45, 1.0), (10, 0, 2.0)]


# ------------------------------------------------------------------ pre-filter and top-N

def test_prefilter_identity_and_cosine():
    rng = np.random.default_rng(5)
    ts, lib = _small_lib(rng, K=9, n_r=10, n_theta=20, mirror=True)
    P = rng.random((3, 10, 20))
    act, sc = O.prefilter(P, lib, 1.0)
    assert act.all()
    # a polar image whose azimuthal sum equals R_T[k] scores cosine 1 for k (and its mirror)
    k = 4
    Pk = np.repeat((lib.radial[k] / 20.0)[:, None], 20, axis=1)[None]
    act, sc = O.prefilter(Pk, lib, 0.1)
    assert sc[0, k] == pytest.approx(1.0, abs=1e-12)
    assert sc[0, k + lib.K0] == sc[0, k]
    assert act.sum() == O.keep_count(0.1, lib.K) == 2
    assert act[0, k] and act[0, k + lib.K0]
    act, _ = O.prefilter(Pk, lib, 0.05)                   # keep 1: tie -> lower index
    assert act[0, k] and not act[0, k + lib.K0]


def test_top_n_order_ties_and_padding():
    q = np.array([[0.5, 0.9, 0.9, 0.1, 0.9 * (1 + 1e-13)]])
    s = np.array([[1, 2, 3, 4, 5]], dtype=np.int32)
    tk, tsh, tq = O.top_n(q, s, 4)
    assert list(tk[0]) == [1, 2, 4, 0]                     # ties within 1e-12 -> lower index
    act = np.array([[True, False, False, True, False]])
    tk, tsh, tq = O.top_n(q, s, 4, act)
    assert list(tk[0]) == [0, 3, -1, -1] and np.isneginf(tq[0, 2])


def test_shift_tie_lowest():
    """A template invariant under a half turn ties at s and s + n_theta/2: lowest wins."""
    ts = synth.TemplateSet(np.array([0, 2]), np.array([5.0, 5.0]), np.array([0.3, 0.3 + math.pi]),
                           np.array([1.0, 1.0]))
    lib = O.prepare_library(ts, 8, 36)
    P = np.roll(lib.dense(0), 25, axis=1)[None]
    q, s = O.scores(P, lib)
    assert s[0, 0] == 25 - 18 and abs(q[0, 0] - 1) < 1e-12


# ------------------------------------------------------------------ dense forms

def test_dense_and_dft_equal_sparse():
    rng = np.random.default_rng(9)
    ts, lib = _small_lib(rng, K=5, n_r=12, n_theta=30, spots=(2, 8))
    P = rng.random((1, 12, 30))
    full = O.scores_full(P, lib)[0]
    assert np.allclose(O.dense_scores(P[0], lib), full, atol=1e-12)
    assert np.allclose(O.dft_scores(P[0], lib), full, atol=1e-12)


# ------------------------------------------------------------------ ground truth (informative)

def test_tiny_workload_recovers_truth():
    ts, scan, prm = synth.tiny_workload()
    lib = O.prepare_library(ts, 60, 180)
    r = O.index(scan.frames, lib, N=5)
    assert np.mean(r["template"][:, 0] == scan.template) > 0.95
    ex = scan.exact
    m = np.round(scan.angle[ex] / (2 * math.pi / 180)).astype(int) % 180
    err = np.abs(((r["shift"][ex, 0] - m) + 90) % 180 - 90)
    assert np.mean(err <= 1) > 0.95


# ------------------------------------------------------------------ two-stage indexing (Section 4.3)

def test_frame_sum_closed_forms():
    n = 37
    f = np.broadcast_to(np.arange(n, dtype=np.uint16)[:, None, None], (n, 3, 4)).copy()
    assert np.array_equal(O.frame_sum(f), np.full((3, 4), n * (n - 1) / 2))
    g = np.full((n, 2, 2), 0.25, dtype=np.float32)
    g[5] = 1.5
    assert np.array_equal(O.frame_sum(g), np.full((2, 2), 0.25 * (n - 1) + 1.5))


def test_morphology_closed_forms():
    B = np.zeros((9, 9), bool)
    B[4, 4] = True
    D = O.dilate(B)
    assert D.sum() == 9 and D[3:6, 3:6].all()                    # a point grows to the 3 x 3 square
    assert np.array_equal(O.erode(D), B)                          # and shrinks back
    assert not O.erode(B).any()                                   # an isolated point is eroded
    full = np.ones((5, 5), bool)
    E = O.erode(full)                                             # outside counts as unset
    assert E.sum() == 9 and E[1:4, 1:4].all()
    blk = np.zeros((11, 11), bool)
    blk[2:7, 3:8] = True
    assert np.array_equal(O.dilate(O.erode(blk)), blk)            # opening keeps a 5 x 5 block


def test_matrix_mask_removes_specks_and_covers_tails():
    n = 10
    sums = np.zeros((21, 21))
    sums[2, 2] = 100.0 * n                                        # one-pixel speck (noise)
    sums[9:12, 9:12] = 50.0 * n                                   # a 3 x 3 intense reflection
    sums[15, 15] = 0.5 * n                                        # below the threshold
    M = O.matrix_mask(sums, n, threshold=1.0, n_open=1, n_dilate=2)
    assert M.dtype == np.uint8
    masked = M == 0
    assert masked.sum() == 49 and masked[7:14, 7:14].all()        # 3 x 3 opened, dilated twice -> 7 x 7
    assert M[2, 2] == 1 and M[15, 15] == 1
    # exactly at the threshold: sum > threshold * n is strict
    s2 = np.zeros((3, 3))
    s2[1, 1] = 2.0 * n
    assert O.matrix_mask(s2, n, threshold=2.0, n_open=0, n_dilate=0).all()
    f = np.full((2, 21, 21), 7, dtype=np.uint16)
    fm = O.apply_mask(f, M)
    assert fm.dtype == np.uint16 and fm[:, 10, 10].sum() == 0 and np.all(fm[:, 0, 0] == 7)


# ------------------------------------------------------------------ preprocessing: centring, threshold (Section 3.1)

def test_find_centres_symmetric_blob_and_shift():
    f = np.zeros((2, 32, 40), dtype=np.uint16)
    # a blob symmetric about (x, y) = (17, 12): its centre of mass is exactly that point
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            f[0, 12 + dy, 17 + dx] = 10 - 2 * (abs(dx) + abs(dy))
    f[1] = np.roll(f[0], (3, -4), axis=(0, 1))                      # moved by (dx, dy) = (-4, 3)
    c = O.find_centres(f, (15.0, 14.0), radius=6.0, iterations=3)
    assert np.array_equal(c, np.array([[17.0, 12.0], [13.0, 15.0]], dtype=np.float32))
    z = np.zeros((1, 8, 8), dtype=np.float32)                        # nothing in the disc: estimate kept
    assert np.array_equal(O.find_centres(z, (3.5, 2.25), 2.0, 4), np.array([[3.5, 2.25]], dtype=np.float32))


def test_find_centres_disc_membership():
    f = np.zeros((1, 9, 9), dtype=np.uint16)
    f[0, 4, 4] = 1
    f[0, 4, 7] = 1                                                   # distance 3 from (4, 4)
    assert np.array_equal(O.find_centres(f, (4.0, 4.0), 2.9, 1)[0], np.float32([4.0, 4.0]))
    assert np.array_equal(O.find_centres(f, (4.0, 4.0), 3.0, 1)[0], np.float32([5.5, 4.0]))


def test_threshold_sets_low_pixels_to_zero():
    f = np.full((1, 16, 16), 9, dtype=np.uint16)
    f[0, :, :8] = 3
    P0 = O.polar(f, 6, 8, gamma=1.0)
    P1 = O.polar(f, 6, 8, gamma=1.0, threshold=5.0)
    P2 = O.polar(np.where(f < 5, 0, f).astype(np.uint16), 6, 8, gamma=1.0)
    assert np.array_equal(P1, P2) and not np.array_equal(P0, P1)
    assert np.array_equal(O.polar(f, 6, 8, threshold=3.0), O.polar(f, 6, 8))   # strict: 3 < 3 is false


# ------------------------------------------------------------------ sub-step in-plane angle

def test_refine_angles_vertex_of_a_parabola():
    """A polar image whose single row is a sampled parabola in theta around a non-integer
    maximum: a one-spot template's Q(s) follows it, so the refined angle is the true vertex."""
    nt = 36
    ts = synth.TemplateSet(np.array([0, 1]), np.array([3.0]), np.array([0.0]), np.array([2.0]))
    lib = O.prepare_library(ts, 5, nt)
    P = np.zeros((1, 5, nt))
    x0 = 10.3                                                     # vertex, in columns
    cols = np.arange(nt)
    P[0, 3] = 50.0 - (cols - x0) ** 2
    P[0, 3] = np.maximum(P[0, 3], 1.0)
    a = O.refine_angles(P, lib, np.array([[0]]), np.array([[10]]))
    assert abs(a[0, 0] - x0 * 10.0) < 1e-9                         # 360 / 36 = 10 degrees per column
    # at a flat or inverted neighbourhood the step itself is kept; padding stays NaN
    P2 = np.ones((1, 5, nt))
    a2 = O.refine_angles(P2, lib, np.array([[0, -1]]), np.array([[7, -1]]))
    assert a2[0, 0] == 70.0 and np.isnan(a2[0, 1])
    # the offset is clipped to half a step
    P3 = np.zeros((1, 5, nt))
    P3[0, 3, 9], P3[0, 3, 10], P3[0, 3, 11] = 1.0, 1.0, 0.0        # vertex pulled beyond half a step
    a3 = O.refine_angles(P3, lib, np.array([[0]]), np.array([[10]]))
    assert a3[0, 0] == 95.0


# ------------------------------------------------------------------ background removal and blur

def test_gaussian_filter_matches_scipy():
    """The separable filter with the edge pixel repeated equals scipy's Gaussian filter in
    'nearest' mode with the same truncation (radius = floor(4 sigma + 1/2)), including a
    radius larger than the frame."""
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(21)
    x = rng.random((2, 23, 31)) * 100.0
    for sigma in (0.6, 1.0, 2.5, 7.0, 12.0):
        ref = np.stack([nd.gaussian_filter(f, sigma, mode="nearest", truncate=4.0) for f in x])
        assert np.allclose(O.gaussian_filter(x, sigma), ref, rtol=0, atol=1e-11)


def test_gaussian_filter_closed_forms():
    """A unit impulse far from the edges becomes the outer product of the normalised 1-D
    Gaussian exp(-i^2 / (2 sigma^2)); a constant image stays constant; a linear ramp stays
    the ramp where the kernel does not reach the edges."""
    sigma = 1.7
    r = int(math.floor(4.0 * sigma + 0.5))
    g = np.array([math.exp(-i * i / (2.0 * sigma * sigma)) for i in range(-r, r + 1)])
    g /= g.sum()
    w = O.gaussian_weights(sigma)
    assert w.shape == g.shape and np.allclose(w, g, rtol=1e-13, atol=0)
    img = np.zeros((41, 45))
    img[20, 22] = 1.0
    out = O.gaussian_filter(img, sigma)
    assert np.allclose(out[20 - r:21 + r, 22 - r:23 + r], np.outer(g, g), rtol=0, atol=1e-16)
    assert abs(out.sum() - 1.0) < 1e-12
    assert np.allclose(O.gaussian_filter(np.full((9, 12), 3.25), 2.0), 3.25, rtol=0, atol=1e-13)
    yy, xx = np.mgrid[0:40, 0:44]
    ramp = 0.5 * xx - 0.25 * yy + 3.0
    out = O.gaussian_filter(ramp, sigma)
    assert np.allclose(out[r:-r, r:-r], ramp[r:-r, r:-r], rtol=0, atol=1e-12)


def test_difference_of_gaussians_removes_smooth_background():
    """The difference of Gaussians is 0 on a constant or linear background (away from the
    edges), never negative, and keeps a sharp spot standing on a broad background."""
    yy, xx = np.mgrid[0:64, 0:64]
    back = 50.0 + 0.3 * xx + 0.1 * yy
    d = O.dog_background(back, 1.0, 4.0)
    assert np.all(d >= 0.0) and np.max(np.abs(d[16:-16, 16:-16])) < 1e-9
    spot = back.copy()
    spot[32, 30] += 200.0
    d = O.dog_background(spot, 1.0, 4.0)
    assert d[32, 30] > 10.0 and np.argmax(d) == 32 * 64 + 30
    f = np.random.default_rng(3).poisson(5.0, size=(2, 20, 24)).astype(np.uint16)
    assert np.array_equal(O.preprocess(f), f.astype(np.float64))              # nothing asked: the frames
    assert np.allclose(O.preprocess(f, dog=(1.0, 3.0), blur=1.5),
                       O.gaussian_filter(O.dog_background(f, 1.0, 3.0), 1.5), rtol=0, atol=1e-12)


# ------------------------------------------------------------------ template simulation

def test_kinematic_zone_axis_closed_form():
    """FCC seen down [001] (identity orientation): the kept reflections are the zero layer's
    allowed ones (h, k both even, l = 0, |F|^2 = 16 for the four-atom basis) whose excitation
    error k - sqrt(k^2 + |g|^2) lies within s_max, each with I = 16 (1 - |s| / s_max); no
    reflection of the layers l = +-1 (|s| ~ 1/a >> s_max) is kept."""
    st = synth.STRUCTURES["fcc"]
    g, F2, gn = synth._reciprocal_points(st, 1.2)
    lam, s_max = synth.WAVELENGTH_200KV, 0.02
    counts, spots = O.kinematic_spots(g, F2, gn, np.eye(3)[None], lam, s_max, 500)
    k = 1.0 / lam
    a = st["a"]
    exp = []
    for h in range(-6, 7):
        for kk in range(-6, 7):
            if (h, kk) == (0, 0) or h % 2 or kk % 2:
                continue
            gx, gy = h / a, kk / a
            if math.hypot(gx, gy) > 1.2:
                continue
            s = k - math.sqrt(k * k + gx * gx + gy * gy)
            if abs(s) <= s_max:
                exp.append((gx, gy, 16.0 * (1.0 - abs(s) / s_max)))
    got = spots[0, :counts[0]]
    assert counts[0] == len(exp) > 0
    key = lambda r: (round(r[0], 9), round(r[1], 9))
    e = sorted(exp, key=key)
    o = sorted(map(tuple, got), key=key)
    for (x0, y0, i0), (x1, y1, i1) in zip(e, o):
        assert abs(x0 - x1) < 1e-12 and abs(y0 - y1) < 1e-12 and abs(i0 - i1) < 1e-9
    assert np.all(np.diff(got[:, 2]) <= 0)                                   # strongest first


def test_kinematic_on_the_ewald_sphere_and_truncation():
    """A point placed exactly on the Ewald sphere has s = 0 and keeps its full |F|^2; one at
    s = s_max / 2 keeps half; max_spots keeps the strongest in order."""
    lam, s_max = synth.WAVELENGTH_200KV, 0.02
    k = 1.0 / lam
    pts, f2 = [], []
    for a_, s_target, w in ((0.5, 0.0, 4.0), (0.7, s_max / 2, 2.0), (0.9, -s_max / 2, 8.0), (0.3, 0.05, 1.0)):
        # |v + k z| = k - s  ->  v = (a, 0, -k + sqrt((k - s)^2 - a^2))
        pts.append((a_, 0.0, -k + math.sqrt((k - s_target) ** 2 - a_ * a_)))
        f2.append(w)
    g = np.array(pts)
    f2 = np.array(f2)
    gn = np.linalg.norm(g, axis=1)
    counts, spots = O.kinematic_spots(g, f2, gn, np.eye(3)[None], lam, s_max, 10)
    assert counts[0] == 3                                                    # the s = 0.05 point is out
    inten = spots[0, :3, 2]
    assert np.allclose(sorted(inten), sorted([4.0, 1.0, 4.0]), rtol=0, atol=1e-8)
    c1, s1 = O.kinematic_spots(g, f2, gn, np.eye(3)[None], lam, s_max, 2)
    assert c1[0] == 2 and np.array_equal(s1[0, :2], spots[0, :2])


def test_kinematic_matches_the_scan_generator():
    """The orientation-grid simulation equals the (independently written, vectorised)
    generator of the synthetic scans for FCC, HCP and tetragonal lattices."""
    for name, system in (("fcc", "cubic"), ("hcp", "hexagonal"), ("tetragonal", "tetragonal")):
        st = synth.STRUCTURES[name]
        g, F2, gn = synth._reciprocal_points(st, 1.2)
        dirs = synth.beam_directions(system, 4.0)
        R = np.stack([synth._orientation_matrix(d) for d in dirs])
        counts, spots = O.kinematic_spots(g, F2, gn, R, synth.WAVELENGTH_200KV, 0.02, 150)
        ts = synth.kinematic_library(name, step_deg=4.0)
        assert np.array_equal(np.diff(ts.offsets), counts)
        flat = np.concatenate([spots[d, :counts[d]] for d in range(len(counts))])
        assert np.allclose(flat[:, 0], ts.a, rtol=0, atol=1e-13)
        assert np.allclose(flat[:, 1], ts.b, rtol=0, atol=1e-13)
        assert np.allclose(flat[:, 2], ts.intensity, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ orientation maps (Eq. 2)

def test_orientation_vectors_special_cases():
    """Identity orientation at phi = 0 gives the sample axis itself; a rotation about the
    beam leaves the beam axis's vector unchanged and turns X into the direction at -phi;
    a mirror copy flips the y component; a 90 deg tilt about x maps the beam axis to the
    crystal's -y ... all against the matrices written out by hand."""
    I = np.eye(3)[None]
    z = O.orientation_vectors(np.array([0]), np.array([0.0]), I, 1, (0, 0, 1))
    assert np.array_equal(z[0], [0.0, 0.0, 1.0])
    v = O.orientation_vectors(np.array([0, 0]), np.array([37.0, 90.0]), I, 1, (0, 0, 1))
    assert np.allclose(v, [[0, 0, 1], [0, 0, 1]], atol=1e-15)
    x = O.orientation_vectors(np.array([0]), np.array([90.0]), I, 1, (1, 0, 0))
    assert np.allclose(x[0], [0.0, -1.0, 0.0], atol=1e-15)                     # Rz(90)^T X
    y = O.orientation_vectors(np.array([1]), np.array([0.0]), I, 1, (0, 1, 0))   # mirror copy of 0
    assert np.allclose(y[0], [0.0, -1.0, 0.0], atol=0)
    c, s = math.cos(math.radians(90)), math.sin(math.radians(90))
    Rx = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])[None]                     # rows: beam axes in crystal coords
    w = O.orientation_vectors(np.array([0, -1]), np.array([0.0, 0.0]), Rx, 1, (0, 0, 1))
    assert np.allclose(w[0], Rx[0].T @ np.array([0, 0, 1.0]), atol=1e-15) and np.all(np.isnan(w[1]))


def test_angular_deviation_eq2():
    """Eq. 2: parallel 0, orthogonal 90, antiparallel 180 degrees, independent of length;
    a known angle between two unit vectors; missing vectors give NaN."""
    va = np.array([[1.0, 0, 0], [0, 2.0, 0], [1.0, 1.0, 0], [0, 0, 3.0], [math.cos(0.3), math.sin(0.3), 0], [np.nan] * 3])
    vb = np.array([[5.0, 0, 0], [0, 0, 1.0], [-1.0, -1.0, 0], [0, 0, 1.0], [1.0, 0, 0], [1.0, 0, 0]])
    d = O.angular_deviation(va, vb)
    assert np.allclose(d[:5], [0.0, 90.0, 180.0, 0.0, math.degrees(0.3)], atol=1e-9) and np.isnan(d[5])
