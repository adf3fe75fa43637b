"""FP64 oracle of the indexing path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this module.  It shares no code with the CUDA path (``paper_2111_07347_gb300``)
and imports nothing from it; the seeded generators in
``paper_2111_07347_gb300.synth`` feed both sides.

Steps, in the paper's order (Section 2.2):

* ``prepare_library``  -- template spots to the polar grid: radius and angle rounded
  to the nearest pixel (Section 2.2, "rounded to the nearest integer"), spots beyond
  the grid dropped, spots landing on one pixel merged by summing intensity (the
  rendered template image of Eq. 1), mirror templates made by reflecting spots across
  y = 0 (Section 2.2 / Fig. 2 caption), optional unit intensities (Section 4.3),
  template norms sqrt(sum T^2) (Eq. 1 denominator) and azimuthal sums (Section 2.2,
  pre-filter).
* ``polar``            -- gamma/subtract then bilinear polar resampling (C loops).
* ``scores``           -- per template maximum of Eq. 1 over all azimuthal shifts with
  wraparound and the lowest shift attaining it (C loops).
* ``prefilter``        -- azimuthally integrated image and templates correlated by one
  matrix-vector product; the best fraction kept (Section 2.2, Fig. 3).
* ``top_n``            -- templates ranked by their best Q (Section 2.2: "sorted and
  the top N best matching templates can be queried").
* ``find_centres`` -- the direct beam's centre per pattern (centre of mass in a disc), and
  ``polar(threshold=...)`` -- low-intensity pixels set to zero (Section 3.1's preprocessing).
* ``frame_sum`` / ``matrix_mask`` / ``apply_mask`` -- the two-stage indexing of Section 4.3:
  mean of all patterns, thresholded, cleaned by erosions and dilations, and the masked
  patterns indexed again.
* ``gaussian_filter`` / ``dog_background`` / ``preprocess`` -- the diffuse background
  removed by a difference of Gaussians and the result smoothed by a Gaussian blur
  (Section 3.1's preprocessing; parameters are the caller's).
* ``kinematic_spots`` -- templates simulated over an orientation grid (Section 2.1:
  reflections near the Ewald sphere by their excitation error, a linear relrod shape,
  |F|^2 for the intensity, the strongest kept), the step before the library.
* ``orientation_vectors`` / ``angular_deviation`` -- the crystal direction along a sample
  axis for each pattern's best template and in-plane angle (the vectors of inverse pole
  figure maps) and the angle between two maps' vectors (Eq. 2).
* ``dense_scores`` / ``dft_scores`` -- Q(k, s) for every shift written as the dense
  circulant contraction and as its angular-DFT factorisation (Section 2.2, the
  complexity discussion naming the FFT cross-correlation alternative), both in FP64.

Ties: a relative window of 1e-12 decides equality; among equals the lowest shift and
the lowest template index win.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

TIE_REL = 1e-12
_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def build(force: bool = False) -> str:
    """Compile tm_oracle.c into liboracle.so beside it (gcc, -O2, OpenMP, no fast-math)."""
    src = os.path.join(_HERE, "tm_oracle.c")
    out = os.path.join(_HERE, "liboracle.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-o", out + ".tmp", src, "-lm"])
        os.replace(out + ".tmp", out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, d = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.oracle_polar.argtypes = [P, i32, i64, i32, i32, P, d, d, d, d, i32, i32, d, P]
        lib.oracle_scores.argtypes = [P, i64, i32, i32, P, P, P, P, P, i64, P, P, P]
        lib.oracle_scores_full.argtypes = [P, i64, i32, i32, P, P, P, P, P, i64, P]
        lib.oracle_num_threads.restype = i32
        _LIB = lib
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_lib().oracle_num_threads())


# ----------------------------------------------------------------------------------
# Library preparation (Section 2.1 template lists -> polar grid of Section 2.2)
# ----------------------------------------------------------------------------------

class Library:
    """Rounded, merged templates on the polar grid (expanded: mirrors at k >= K0)."""

    def __init__(self, off, ri, ti, inten, K0, mirror, n_r, n_theta, dr):
        self.off, self.ri, self.ti, self.I = off, ri, ti, inten
        self.K0, self.mirror = K0, mirror
        self.K = off.shape[0] - 1
        self.n_r, self.n_theta, self.dr = n_r, n_theta, dr
        self.norm = np.array([math.sqrt(float(np.sum(inten[off[k]:off[k + 1]] ** 2)))
                              for k in range(self.K)], dtype=np.float64)
        self.radial = np.zeros((self.K, n_r), dtype=np.float64)
        for k in range(self.K):
            for i in range(off[k], off[k + 1]):
                self.radial[k, ri[i]] += inten[i]

    def dense(self, k: int) -> np.ndarray:
        """Template k rendered as a dense polar image T[r, theta]."""
        T = np.zeros((self.n_r, self.n_theta))
        for i in range(self.off[k], self.off[k + 1]):
            T[self.ri[i], self.ti[i]] += self.I[i]
        return T


def round_spot(r_px: float, theta: float, n_theta: int, dr: float):
    """Nearest polar pixel of a spot: r_i = floor(r/dr + 1/2), t_i = floor(u + 1/2) mod
    n_theta with u = theta' / (2 pi / n_theta) and theta' = theta reduced to [0, 2 pi)."""
    th = math.fmod(theta, 2.0 * math.pi)
    if th < 0.0:
        th += 2.0 * math.pi
    step = 2.0 * math.pi / n_theta
    t = int(math.floor(th / step + 0.5)) % n_theta
    r = int(math.floor(r_px / dr + 0.5))
    return r, t


def prepare_library(ts, n_r: int, n_theta: int, dr: float = 1.0, mirror: bool | None = None,
                    unit_intensity: bool = False) -> Library:
    """Template set -> Library on the (n_r, n_theta, dr) grid.

    Spots given as (kx, ky) are converted with r = hypot(x, y), theta = atan2(y, x) after
    scaling to pixels; a mirror copy reflects y -> -y (theta -> -theta) before rounding.
    With ``unit_intensity`` every input spot gets intensity 1 before merging."""
    mirror = ts.mirror if mirror is None else mirror
    K0 = ts.n_templates
    copies = (False, True) if mirror else (False,)
    off = [0]
    ri_all, ti_all, I_all = [], [], []
    for m in copies:
        for k in range(K0):
            merged = {}
            order = []
            for i in range(int(ts.offsets[k]), int(ts.offsets[k + 1])):
                a, b = float(ts.a[i]), float(ts.b[i])
                if ts.coords == "xy":
                    x, y = a * ts.px_per_unit, b * ts.px_per_unit
                    if m:
                        y = -y
                    r_px, th = math.hypot(x, y), math.atan2(y, x)
                else:
                    r_px, th = a, (-b if m else b)
                r, t = round_spot(r_px, th, n_theta, dr)
                if r < 0 or r >= n_r:
                    continue
                w = 1.0 if unit_intensity else float(ts.intensity[i])
                if (r, t) not in merged:
                    merged[(r, t)] = 0.0
                    order.append((r, t))
                merged[(r, t)] += w
            for key in order:
                ri_all.append(key[0]); ti_all.append(key[1]); I_all.append(merged[key])
            off.append(len(ri_all))
    return Library(np.asarray(off, dtype=np.int64), np.asarray(ri_all, dtype=np.int32),
                   np.asarray(ti_all, dtype=np.int32), np.asarray(I_all, dtype=np.float64),
                   K0, mirror, n_r, n_theta, dr)


# ----------------------------------------------------------------------------------
# Pattern side
# ----------------------------------------------------------------------------------

def polar(frames: np.ndarray, n_r: int, n_theta: int, dr: float = 1.0, gamma: float = 0.5,
          subtract: float = 0.0, centre=None, centres: np.ndarray | None = None,
          threshold: float = 0.0) -> np.ndarray:
    """Gamma/subtract then bilinear polar resampling: [n][H][W] -> [n][n_r][n_theta] FP64.
    Default centre ((W-1)/2, (H-1)/2); ``centres`` [n][2] overrides per pattern.  A positive
    ``threshold`` first sets pixels below it to zero (Section 3.1: low-intensity pixels set to
    zero before the gamma correction)."""
    frames = np.ascontiguousarray(frames)
    if threshold > 0.0:
        frames = np.where(frames < threshold, 0, frames).astype(frames.dtype)
    if frames.dtype == np.uint16:
        dt = 0
    elif frames.dtype == np.float32:
        dt = 1
    else:
        raise TypeError("frames must be uint16 or float32")
    n, H, W = frames.shape
    cx, cy = ((W - 1) / 2.0, (H - 1) / 2.0) if centre is None else centre
    out = np.empty((n, n_r, n_theta), dtype=np.float64)
    c = None if centres is None else np.ascontiguousarray(centres, dtype=np.float64)
    _lib().oracle_polar(_ptr(frames), dt, n, H, W, _ptr(c), float(cx), float(cy), float(gamma),
                        float(subtract), n_r, n_theta, float(dr), _ptr(out))
    return out


def scores(P: np.ndarray, lib: Library, active: np.ndarray | None = None):
    """Per (pattern, template): max over shifts of Eq. 1 and the lowest shift attaining it."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    n = P.shape[0]
    q = np.empty((n, lib.K), dtype=np.float64)
    s = np.empty((n, lib.K), dtype=np.int32)
    act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
    _lib().oracle_scores(_ptr(P), n, lib.n_r, lib.n_theta, _ptr(lib.off), _ptr(lib.ri),
                         _ptr(lib.ti), _ptr(lib.I), _ptr(lib.norm), lib.K, _ptr(act),
                         _ptr(q), _ptr(s))
    return q, s


def scores_full(P: np.ndarray, lib: Library) -> np.ndarray:
    """Q for every (pattern, template, shift): [n][K][n_theta]."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    n = P.shape[0]
    q = np.empty((n, lib.K, lib.n_theta), dtype=np.float64)
    _lib().oracle_scores_full(_ptr(P), n, lib.n_r, lib.n_theta, _ptr(lib.off), _ptr(lib.ri),
                              _ptr(lib.ti), _ptr(lib.I), _ptr(lib.norm), lib.K, _ptr(q))
    return q


def radial_profile(P: np.ndarray) -> np.ndarray:
    """Azimuthal integral of each polar image: [n][n_r]."""
    return P.sum(axis=2)


def keep_count(fraction: float, K: int) -> int:
    """Number of templates the pre-filter keeps: ceil(fraction * K), all when fraction >= 1."""
    if fraction >= 1.0:
        return K
    return max(1, int(math.ceil(fraction * K)))


def prefilter(P: np.ndarray, lib: Library, fraction: float):
    """Cosine correlation of azimuthal sums; keep the ceil(fraction K) best templates per
    pattern, ties to the lower index.  Returns (active [n][K] bool, score [n][K])."""
    RP = radial_profile(P)
    RT = lib.radial
    num = RP @ RT.T
    nP = np.sqrt(np.sum(RP * RP, axis=1))
    nT = np.sqrt(np.sum(RT * RT, axis=1))
    den = nP[:, None] * nT[None, :]
    sc = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    n, K = sc.shape
    keep = keep_count(fraction, K)
    active = np.zeros((n, K), dtype=bool)
    ks = np.arange(K)
    for p in range(n):
        order = np.lexsort((ks, -sc[p]))
        active[p, order[:keep]] = True
    return active, sc


def top_n(q_best: np.ndarray, s_best: np.ndarray, N: int, active: np.ndarray | None = None):
    """Greedy top-N per pattern: repeatedly take the best remaining Q and, among the
    entries within the relative tie window of it, the lowest template index.
    Returns (template [n][N] int64, shift [n][N], score [n][N]); missing rows: -1, -1, -inf."""
    n, K = q_best.shape
    tk = np.full((n, N), -1, dtype=np.int64)
    ts = np.full((n, N), -1, dtype=np.int64)
    tq = np.full((n, N), -np.inf)
    for p in range(n):
        q = q_best[p].copy()
        if active is not None:
            q[~active[p]] = -np.inf
        for j in range(N):
            best = np.max(q)
            if best == -np.inf:
                break
            thr = best - TIE_REL * abs(best)
            k = int(np.flatnonzero(q >= thr)[0])
            tk[p, j], ts[p, j], tq[p, j] = k, s_best[p, k], best
            q[k] = -np.inf
    return tk, ts, tq


def index(frames: np.ndarray, lib: Library, gamma: float = 0.5, subtract: float = 0.0,
          prefilter_fraction: float = 1.0, N: int = 5, centre=None, centres: np.ndarray | None = None,
          threshold: float = 0.0):
    """The whole path for a batch of frames; returns a dict of FP64 results.  ``centres``
    [n][2] gives each pattern's own beam centre."""
    P = polar(frames, lib.n_r, lib.n_theta, lib.dr, gamma, subtract, centre, centres, threshold)
    active = None
    if prefilter_fraction < 1.0:
        active, _ = prefilter(P, lib, prefilter_fraction)
    q, s = scores(P, lib, active)
    tk, tsh, tq = top_n(q, s, N, active)
    return dict(polar=P, q_best=q, s_best=s, active=active, template=tk, shift=tsh, score=tq,
                angle_deg=np.where(tsh >= 0, tsh * (360.0 / lib.n_theta), np.nan),
                mirror=np.where(tk >= 0, tk >= lib.K0 if lib.mirror else False, False))


# ----------------------------------------------------------------------------------
# Dense forms of the same correlation (the contraction the tensor-core path computes)
# ----------------------------------------------------------------------------------

def dense_scores(P: np.ndarray, lib: Library) -> np.ndarray:
    """C[k, s] = sum_{r,theta} T_k[r, theta] P[r, (theta + s) mod n_theta] with every
    template rendered dense, for one polar image P [n_r][n_theta]; returns Q[k][s]."""
    n_theta = lib.n_theta
    nP = math.sqrt(float(np.sum(P * P)))
    out = np.zeros((lib.K, n_theta))
    # circulant stack: Pc[s] = P rolled so Pc[s][r, theta] = P[r, (theta + s) mod n_theta]
    Pc = np.stack([np.roll(P, -s, axis=1) for s in range(n_theta)])          # [s][r][theta]
    flat = Pc.reshape(n_theta, -1)
    for k in range(lib.K):
        T = lib.dense(k).reshape(-1)
        d = nP * lib.norm[k]
        out[k] = (flat @ T) / d if d > 0 else 0.0
    return out


def dft_scores(P: np.ndarray, lib: Library) -> np.ndarray:
    """The same Q[k][s] through the angular DFT: with X^[r, m] = sum_theta X[r, theta]
    e^{-2 pi i m theta / n}, C[k, s] = (1/n) sum_m e^{+2 pi i m s / n} sum_r
    conj(T^_k[r, m]) P^[r, m] (correlation theorem along theta, then a sum over r)."""
    n_theta = lib.n_theta
    nP = math.sqrt(float(np.sum(P * P)))
    Ph = np.fft.fft(P, axis=1)
    out = np.zeros((lib.K, n_theta))
    for k in range(lib.K):
        Th = np.fft.fft(lib.dense(k), axis=1)
        G = np.sum(np.conj(Th) * Ph, axis=0)                   # [m]
        C = np.fft.ifft(G).real
        d = nP * lib.norm[k]
        out[k] = C / d if d > 0 else 0.0
    return out


# ----------------------------------------------------------------------------------
# Two-stage (masked) indexing, Section 4.3: the matrix reflections are removed with a
# mask made from the average of all patterns, thresholded, then cleaned by erosions and
# dilations; the masked patterns are indexed against the precipitate library.
# ----------------------------------------------------------------------------------

def frame_sum(frames: np.ndarray) -> np.ndarray:
    """Per-pixel sum over the frames, in FP64, frames added in order p = 0, 1, ... (exact for
    integer frames; the order is fixed for float frames).  frames [n][H][W] -> [H][W]."""
    s = np.zeros(frames.shape[1:], dtype=np.float64)
    for p in range(frames.shape[0]):
        s += frames[p].astype(np.float64)
    return s


def _shifted(B: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """B moved so that out[y, x] = B[y + dy, x + dx], False outside the image."""
    H, W = B.shape
    out = np.zeros_like(B)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    out[ys:ye, xs:xe] = B[ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def erode(B: np.ndarray) -> np.ndarray:
    """Binary erosion by the 3 x 3 square: a pixel stays set when all nine pixels of its
    neighbourhood are set (pixels outside the image count as unset)."""
    out = np.ones_like(B, dtype=bool)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out &= _shifted(B.astype(bool), dy, dx)
    return out


def dilate(B: np.ndarray) -> np.ndarray:
    """Binary dilation by the 3 x 3 square: a pixel is set when any pixel of its
    neighbourhood is set."""
    out = np.zeros_like(B, dtype=bool)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out |= _shifted(B.astype(bool), dy, dx)
    return out


def matrix_mask(sums: np.ndarray, n: int, threshold: float, n_open: int, n_dilate: int) -> np.ndarray:
    """Mask of the pixels to keep (uint8 1 = keep).  Pixels whose mean over the n patterns
    exceeds ``threshold`` (sum > threshold * n, in FP64) are the intense matrix reflections;
    ``n_open`` erosions then ``n_open`` dilations remove noise-like features smaller than the
    structuring element, ``n_dilate`` further dilations cover the tails of the peaks; the
    kept pixels are the complement."""
    B = sums > float(threshold) * float(n)
    for _ in range(n_open):
        B = erode(B)
    for _ in range(n_open + n_dilate):
        B = dilate(B)
    return (~B).astype(np.uint8)


def apply_mask(frames: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Masked patterns: pixels outside the mask set to zero (before gamma and subtraction)."""
    return frames * mask.astype(frames.dtype)[None]


# ----------------------------------------------------------------------------------
# Direct-beam centring (Section 3.1: "the direct beam in each image was centered"): the
# centre used for the polar transform is found per pattern.
# ----------------------------------------------------------------------------------

def find_centres(frames: np.ndarray, centre, radius: float, iterations: int) -> np.ndarray:
    """Per pattern, the intensity-weighted centre of mass of the pixels within ``radius`` of
    the current estimate (starting at ``centre`` = (cx, cy)), repeated ``iterations`` times.
    FP64, pixels visited row by row (y, then x ascending) over the disc's bounding box,
    distances compared as (dx*dx) + (dy*dy) <= radius*radius; a disc with zero total
    intensity keeps the estimate.  Returns [n][2] float32 (the index call's centre type)."""
    n, H, W = frames.shape
    out = np.empty((n, 2), dtype=np.float32)
    r2 = float(radius) * float(radius)
    for p in range(n):
        f = frames[p]
        cx, cy = float(centre[0]), float(centre[1])
        for _ in range(iterations):
            y_lo, y_hi = max(0, math.ceil(cy - radius)), min(H - 1, math.floor(cy + radius))
            x_lo, x_hi = max(0, math.ceil(cx - radius)), min(W - 1, math.floor(cx + radius))
            s0 = sx = sy = 0.0
            for y in range(y_lo, y_hi + 1):
                dy = y - cy
                for x in range(x_lo, x_hi + 1):
                    dx = x - cx
                    if dx * dx + dy * dy <= r2:
                        v = float(f[y, x])
                        s0 += v
                        sx += float(x) * v
                        sy += float(y) * v
            if s0 > 0.0:
                cx, cy = sx / s0, sy / s0
        out[p] = (cx, cy)
    return out


# ----------------------------------------------------------------------------------
# Background removal and smoothing (the preprocessing of Section 3.1: the diffuse
# background removed with a difference of Gaussians, the result smoothed by a Gaussian
# blur).  The paper gives neither the sigmas nor the edge rule; the reading here: a 1-D
# Gaussian of standard deviation sigma on the integer offsets |i| <= radius, radius =
# floor(truncate * sigma + 1/2), normalised to sum 1; applied along rows, then along
# columns, with the edge pixel repeated outside the frame; the difference of Gaussians is
# G(sigma_min) * x - G(sigma_max) * x with negative values set to 0.
# ----------------------------------------------------------------------------------

def gaussian_weights(sigma: float, truncate: float = 4.0) -> np.ndarray:
    """Weights w[i + radius], i = -radius..radius, of the 1-D Gaussian (FP64, sum 1)."""
    radius = int(math.floor(truncate * sigma + 0.5))
    w = np.array([math.exp(-0.5 * (i / sigma) ** 2) for i in range(-radius, radius + 1)])
    return w / w.sum()


def _filter_axis(x: np.ndarray, w: np.ndarray, axis: int) -> np.ndarray:
    """out[.., j, ..] = sum_i w[i] x[.., clamp(j + i - radius), ..] along one axis, the
    terms added in the order i = 0, 1, ... (plain loops over the offsets)."""
    radius = (w.shape[0] - 1) // 2
    n = x.shape[axis]
    out = np.zeros_like(x, dtype=np.float64)
    idx = np.arange(n)
    for i in range(w.shape[0]):
        src = np.clip(idx + i - radius, 0, n - 1)
        out += w[i] * np.take(x, src, axis=axis)
    return out


def gaussian_filter(img: np.ndarray, sigma: float, truncate: float = 4.0) -> np.ndarray:
    """Gaussian smoothing of [..][H][W] images, rows (along W) first, then columns."""
    w = gaussian_weights(sigma, truncate)
    x = np.asarray(img, dtype=np.float64)
    return _filter_axis(_filter_axis(x, w, x.ndim - 1), w, x.ndim - 2)


def dog_background(img: np.ndarray, sigma_min: float, sigma_max: float, truncate: float = 4.0) -> np.ndarray:
    """Difference of Gaussians, G(sigma_min) * x - G(sigma_max) * x, negative values set to 0."""
    return np.maximum(gaussian_filter(img, sigma_min, truncate) - gaussian_filter(img, sigma_max, truncate), 0.0)


def preprocess(frames: np.ndarray, dog=None, blur: float = 0.0, truncate: float = 4.0) -> np.ndarray:
    """frames [n][H][W] -> float64: the difference of Gaussians (dog = (sigma_min, sigma_max),
    or None), then a Gaussian blur of standard deviation `blur` (0: none)."""
    x = np.asarray(frames, dtype=np.float64)
    if dog is not None:
        x = dog_background(x, dog[0], dog[1], truncate)
    if blur > 0.0:
        x = gaussian_filter(x, blur, truncate)
    return x


# ----------------------------------------------------------------------------------
# Template simulation over an orientation grid (Section 2.1: for each orientation the
# reciprocal lattice is rotated into the beam frame, reflections whose excitation error is
# within s_max are kept with the intensity |F|^2 (1 - |s|/s_max) of a linear relrod shape,
# projected onto the detector plane; Section 4.1 ignores atomic scattering, so |F|^2 comes
# from unit scattering factors -- any |F|^2 may be given).  The most intense max_spots are
# kept, ties by the smaller |g|, then the lower point index.
# ----------------------------------------------------------------------------------

def kinematic_spots(g: np.ndarray, f2: np.ndarray, gnorm: np.ndarray, rot: np.ndarray, wavelength: float,
                    s_max: float, max_spots: int):
    """g [G][3] reciprocal lattice points (1/Angstrom, crystal frame), f2 [G] |F|^2, gnorm
    [G] |g|, rot [D][3][3] orientation matrices (row j = beam-frame axis j in crystal
    coordinates; z along the beam).  Per orientation and point, in double precision with
    every operation rounded in this order: the beam-frame components
    x_j = (R[j][0] g_0 + R[j][1] g_1) + R[j][2] g_2, t = x_2 + k with k = 1 / wavelength,
    s = k - sqrt((x_0 x_0 + x_1 x_1) + t t); kept when |s| <= s_max and
    I = f2 (1 - |s| / s_max) > 0.  Returns (counts [D], spots [D][max_spots][3] = (x_0, x_1, I)
    in the order: I descending, |g| ascending, point index ascending)."""
    G, D = g.shape[0], rot.shape[0]
    k = 1.0 / wavelength
    counts = np.zeros(D, dtype=np.int32)
    spots = np.zeros((D, max_spots, 3), dtype=np.float64)
    for d in range(D):
        R = [[float(rot[d, j, m]) for m in range(3)] for j in range(3)]
        cand = []
        for i in range(G):
            g0, g1, g2 = float(g[i, 0]), float(g[i, 1]), float(g[i, 2])
            x = [(R[j][0] * g0 + R[j][1] * g1) + R[j][2] * g2 for j in range(3)]
            t = x[2] + k
            s = k - math.sqrt((x[0] * x[0] + x[1] * x[1]) + t * t)
            if abs(s) <= s_max:
                inten = float(f2[i]) * (1.0 - abs(s) / s_max)
                if inten > 0.0:
                    cand.append((-inten, float(gnorm[i]), i, x[0], x[1], inten))
        cand.sort()
        cand = cand[:max_spots]
        counts[d] = len(cand)
        for r, c in enumerate(cand):
            spots[d, r] = (c[3], c[4], c[5])
    return counts, spots


# ----------------------------------------------------------------------------------
# Orientation maps and their angular deviation (Section 4.1: inverse pole figure maps along
# the sample axes; Eq. 2: the angle between the vectors two maps hold in a pixel).  Reading:
# template b has the orientation matrix R_b (rows: the beam-frame axes in crystal
# coordinates, as its simulation used); its mirror copy reflects the beam-frame y axis
# (M = diag(1, -1, 1)); a hit at in-plane angle phi shows the template rotated by phi about
# the beam, so the pattern's orientation is O = Rz(phi) M R_b, and the crystal direction along
# the sample axis e is v = O^T e.
# ----------------------------------------------------------------------------------

def orientation_vectors(template: np.ndarray, angle_deg: np.ndarray, rot: np.ndarray, K0: int, axis) -> np.ndarray:
    """template [n] expanded indices (mirror copies at >= K0; < 0: no hit -> NaN), angle_deg
    [n] (float32 values, used as doubles), rot [K0][3][3], axis e [3] -> v [n][3] float64.
    Per pattern, with each operation rounded in this order: c = cos(phi), s = sin(phi) with
    phi = angle * (pi / 180); u = Rz(phi)^T e = (c e0 + s e1, -s e0 + c e1, e2); u1 negated for a
    mirror copy; v_j = (R[0][j] u0 + R[1][j] u1) + R[2][j] u2."""
    n = template.shape[0]
    out = np.full((n, 3), np.nan)
    e0, e1, e2 = float(axis[0]), float(axis[1]), float(axis[2])
    for p in range(n):
        k = int(template[p])
        if k < 0:
            continue
        mirror = k >= K0
        b = k - K0 if mirror else k
        phi = float(angle_deg[p]) * (math.pi / 180.0)
        c, s = math.cos(phi), math.sin(phi)
        u0 = c * e0 + s * e1
        u1 = -s * e0 + c * e1
        u2 = e2
        if mirror:
            u1 = -u1
        R = rot[b]
        for j in range(3):
            out[p, j] = (float(R[0, j]) * u0 + float(R[1, j]) * u1) + float(R[2, j]) * u2
    return out


def angular_deviation(va: np.ndarray, vb: np.ndarray) -> np.ndarray:
    """Eq. 2 per pattern, in degrees: |acos(va . vb / (|va| |vb|))| (the cosine clipped to
    [-1, 1]); NaN where either vector is missing."""
    n = va.shape[0]
    out = np.full(n, np.nan)
    for p in range(n):
        a, b = va[p], vb[p]
        if np.any(np.isnan(a)) or np.any(np.isnan(b)):
            continue
        dot = (float(a[0]) * float(b[0]) + float(a[1]) * float(b[1])) + float(a[2]) * float(b[2])
        na = math.sqrt((float(a[0]) ** 2 + float(a[1]) ** 2) + float(a[2]) ** 2)
        nb = math.sqrt((float(b[0]) ** 2 + float(b[1]) ** 2) + float(b[2]) ** 2)
        cosv = max(-1.0, min(1.0, dot / (na * nb)))
        out[p] = abs(math.degrees(math.acos(cosv)))
    return out


# ----------------------------------------------------------------------------------
# In-plane angle below the polar step (Section 2.2: the resolution of phi_1 is the polar
# transform's angular step; Section 5 names a better phi_1 optimisation as future work).
# ----------------------------------------------------------------------------------

def refine_angles(P: np.ndarray, lib: Library, template: np.ndarray, shift: np.ndarray) -> np.ndarray:
    """Sub-step in-plane angle of top-N hits: Q at the shifts s - 1, s, s + 1 (mod n_theta) of
    each hit's template, the vertex of the parabola through them, delta = (Q- - Q+) /
    (2 (Q- - 2 Q0 + Q+)) when the curvature Q- - 2 Q0 + Q+ is negative (else 0), clipped to
    [-1/2, 1/2]; angle = (s + delta) 360 / n_theta degrees.  P [n][n_r][n_theta];
    template, shift [n][N] (-1 padding -> NaN)."""
    n, N = template.shape
    out = np.full((n, N), np.nan)
    nt = lib.n_theta
    for p in range(n):
        nP = math.sqrt(float(np.sum(P[p] * P[p])))
        for j in range(N):
            k, s = int(template[p, j]), int(shift[p, j])
            if k < 0:
                continue
            d = nP * lib.norm[k]
            q = []
            for ds in (-1, 0, 1):
                acc = 0.0
                for i in range(lib.off[k], lib.off[k + 1]):
                    acc += lib.I[i] * P[p, lib.ri[i], (lib.ti[i] + s + ds) % nt]
                q.append(acc / d if d > 0 else 0.0)
            curv = q[0] - 2.0 * q[1] + q[2]
            delta = (q[0] - q[2]) / (2.0 * curv) if curv < 0.0 else 0.0
            out[p, j] = (s + min(0.5, max(-0.5, delta))) * 360.0 / nt
    return out
