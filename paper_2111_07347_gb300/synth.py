"""Seeded synthetic inputs: template sets and rendered 4D-STEM scans.

This module draws data only. It contains no step of the indexing method (no gamma
transform, polar resampling, template rounding, correlation index or ranking), so
both the CUDA path and the FP64 oracle can consume what it returns without sharing
any of the method's arithmetic.

Stand-ins for the paper's datasets (Section 3: Cu-Ag and irradiated steel scans,
not available here):

* ``random_templates``   -- random sparse templates (radius/angle/intensity lists).
* ``kinematic_library``  -- kinematic templates of a crystal over a beam-direction
  grid of the Laue-group fundamental triangle, with unit atomic scattering factors
  and a linear relrod shape function (Section 2.1, the options used in Section 4.1).
* ``render_scan``        -- diffraction frames: a template rotated in plane by a
  random angle, drawn as Gaussian spots, plus a direct beam and an exponential
  diffuse background, with Poisson counting noise.

Every draw comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED = 211107347

#: 200 kV relativistic electron wavelength in Angstrom.
WAVELENGTH_200KV = 0.025079


def make_rng(config_index: int, stream: int = 0) -> np.random.Generator:
    """Generator for a workload: seed = SEED + config_index + 100 * stream."""
    return np.random.Generator(np.random.PCG64(SEED + config_index + 100 * stream))


@dataclasses.dataclass
class TemplateSet:
    """Sparse templates as a CSR list of spots (Section 2.1: each template is a list
    of reflections with coordinates and intensities; the in-plane angle is zero).

    coords == "polar": ``a`` = radius in pixels, ``b`` = angle in radians.
    coords == "xy":    ``a`` = kx, ``b`` = ky in reciprocal Angstrom; ``px_per_unit``
                       converts reciprocal Angstrom to detector pixels.
    """

    offsets: np.ndarray          # int64 [K0 + 1]
    a: np.ndarray                # float64 [S]
    b: np.ndarray                # float64 [S]
    intensity: np.ndarray        # float64 [S]
    coords: str = "polar"
    px_per_unit: float = 1.0
    mirror: bool = False         # whether the set is meant to be used with mirror templates
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_templates(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_expanded(self) -> int:
        return self.n_templates * (2 if self.mirror else 1)

    def spot_counts(self) -> np.ndarray:
        return np.diff(self.offsets)


# ----------------------------------------------------------------------------------
# Random templates
# ----------------------------------------------------------------------------------

def random_templates(rng: np.random.Generator, n_templates: int = 300,
                     spots: tuple[int, int] = (8, 40), r_range: tuple[float, float] = (6.0, 60.0),
                     sigma_log: float = 1.0) -> TemplateSet:
    """Random sparse templates: n_spots ~ U{lo..hi}, r ~ U[r0, r1] px, theta ~ U[0, 2pi),
    intensity ~ lognormal(0, sigma_log)."""
    counts = rng.integers(spots[0], spots[1] + 1, size=n_templates)
    offsets = np.zeros(n_templates + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    s = int(offsets[-1])
    r = rng.uniform(r_range[0], r_range[1], size=s)
    th = rng.uniform(0.0, 2.0 * math.pi, size=s)
    inten = rng.lognormal(0.0, sigma_log, size=s)
    return TemplateSet(offsets, r, th, inten, coords="polar", mirror=False,
                       meta={"kind": "random", "spots": spots, "r_range": r_range})


# ----------------------------------------------------------------------------------
# Kinematic templates (data tool; stands in for the paper's diffsims libraries)
# ----------------------------------------------------------------------------------

STRUCTURES = {
    # cubic FCC, 4-atom basis
    "fcc": dict(system="cubic", a=4.05, c=4.05,
                basis=[(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)]),
    # hexagonal close packed, 2-atom basis
    "hcp": dict(system="hexagonal", a=3.21, c=5.21,
                basis=[(1 / 3, 2 / 3, 0.25), (2 / 3, 1 / 3, 0.75)]),
    # primitive tetragonal, one atom at the origin (basis not given by the workload)
    "tetragonal": dict(system="tetragonal", a=3.6, c=5.1, basis=[(0, 0, 0)]),
}


def _direct_lattice(system: str, a: float, c: float) -> np.ndarray:
    if system == "hexagonal":
        return np.array([[a, 0, 0], [-a / 2, a * math.sqrt(3) / 2, 0], [0, 0, c]], dtype=np.float64)
    return np.array([[a, 0, 0], [0, a, 0], [0, 0, c]], dtype=np.float64)


def _reciprocal_points(struct: dict, g_max: float):
    """All reciprocal lattice vectors g (Cartesian, 1/Angstrom, no 2pi) with 0 < |g| <= g_max
    and their |F|^2 for unit atomic scattering factors."""
    A = _direct_lattice(struct["system"], struct["a"], struct["c"])
    B = np.linalg.inv(A).T                      # rows b_i with a_i . b_j = delta_ij
    hmax = [int(math.ceil(g_max * np.linalg.norm(A[i]))) + 1 for i in range(3)]
    hs = np.arange(-hmax[0], hmax[0] + 1)
    ks = np.arange(-hmax[1], hmax[1] + 1)
    ls = np.arange(-hmax[2], hmax[2] + 1)
    H, K, L = np.meshgrid(hs, ks, ls, indexing="ij")
    hkl = np.stack([H.ravel(), K.ravel(), L.ravel()], axis=1).astype(np.float64)
    g = hkl @ B
    gn = np.linalg.norm(g, axis=1)
    keep = (gn > 0) & (gn <= g_max)
    hkl, g, gn = hkl[keep], g[keep], gn[keep]
    basis = np.array(struct["basis"], dtype=np.float64)
    phase = 2.0 * math.pi * (hkl @ basis.T)
    F = np.exp(1j * phase).sum(axis=1)
    F2 = (F * np.conj(F)).real
    nz = F2 > 1e-9
    return g[nz], F2[nz], gn[nz]


def beam_directions(system: str, step_deg: float = 0.5) -> np.ndarray:
    """Unit beam directions on the fundamental triangle of the Laue group, on a grid of
    about ``step_deg`` spacing (rings of constant polar angle, azimuth step scaled by
    1/sin).  cubic: [001]-[101]-[111] (z >= x >= y >= 0); hexagonal: [0001]-[2-1-10]-[10-10]
    (azimuth 0..30 deg); tetragonal: [001]-[100]-[110] (azimuth 0..45 deg)."""
    step = math.radians(step_deg)
    az_max = {"cubic": math.pi / 4, "hexagonal": math.pi / 6, "tetragonal": math.pi / 4}[system]
    dirs = [(0.0, 0.0, 1.0)]
    n_pol = int(round((math.pi / 2) / step))
    for i in range(1, n_pol + 1):
        pol = i * step
        sp, cp = math.sin(pol), math.cos(pol)
        n_az = max(1, int(math.floor(az_max * sp / step + 1e-9)))
        for j in range(n_az + 1):
            az = az_max * j / n_az
            x, y, z = sp * math.cos(az), sp * math.sin(az), cp
            if system == "cubic" and not (z >= x - 1e-12):
                continue
            dirs.append((x, y, z))
    return np.array(dirs, dtype=np.float64)


def _orientation_matrix(d: np.ndarray) -> np.ndarray:
    """Rotation taking crystal-frame vectors to the frame whose z axis is the beam
    direction d, with in-plane angle phi1 = 0 (Bunge (0, Phi, phi2))."""
    Phi = math.acos(max(-1.0, min(1.0, d[2])))
    phi2 = math.atan2(d[0], d[1])
    c2, s2, cP, sP = math.cos(phi2), math.sin(phi2), math.cos(Phi), math.sin(Phi)
    # Bunge g(phi1=0, Phi, phi2): its rows are the sample axes written in crystal
    # coordinates, so g maps a crystal-frame vector to sample-frame components.
    g = np.array([[c2, -s2, 0.0],
                  [s2 * cP, c2 * cP, -sP],
                  [s2 * sP, c2 * sP, cP]], dtype=np.float64)
    # g @ d == (0, 0, 1): rows are the sample axes expressed in crystal coordinates.
    return g


def kinematic_library(structure: str, step_deg: float = 0.5, g_max: float = 1.2,
                      s_max: float = 0.02, max_spots: int = 150,
                      wavelength: float = WAVELENGTH_200KV, px_per_unit: float = 100.0,
                      directions: np.ndarray | None = None) -> TemplateSet:
    """Kinematic templates of ``structure`` for every beam direction of the grid.

    For each direction the reciprocal lattice (|g| <= g_max) is rotated so the beam is
    along z, the excitation error s_g = k - |g + k z| (k = 1/wavelength) is taken, spots
    with |s_g| <= s_max are kept with intensity |F|^2 (1 - |s_g|/s_max) (unit atomic
    scattering factors, linear relrod), projected onto (kx, ky) and the ``max_spots``
    most intense kept (ties: smaller |g| first).  Coordinates are in 1/Angstrom;
    ``px_per_unit`` is the detector calibration (100 px per 1/Angstrom = 0.01 1/A per px).
    """
    st = STRUCTURES[structure]
    g, F2, gn = _reciprocal_points(st, g_max)
    dirs = beam_directions(st["system"], step_deg) if directions is None else directions
    k = 1.0 / wavelength
    offs = [0]
    xa, xb, xi = [], [], []
    for d in dirs:
        R = _orientation_matrix(d)
        gs = g @ R.T
        sg = k - np.sqrt(gs[:, 0] ** 2 + gs[:, 1] ** 2 + (gs[:, 2] + k) ** 2)
        sel = np.abs(sg) <= s_max
        inten = F2[sel] * (1.0 - np.abs(sg[sel]) / s_max)
        kx, ky, gg = gs[sel, 0], gs[sel, 1], gn[sel]
        pos = inten > 0
        inten, kx, ky, gg = inten[pos], kx[pos], ky[pos], gg[pos]
        order = np.lexsort((gg, -inten))[:max_spots]
        xa.append(kx[order]); xb.append(ky[order]); xi.append(inten[order])
        offs.append(offs[-1] + order.shape[0])
    return TemplateSet(np.asarray(offs, dtype=np.int64), np.concatenate(xa), np.concatenate(xb),
                       np.concatenate(xi), coords="xy", px_per_unit=px_per_unit, mirror=True,
                       meta={"kind": "kinematic", "structure": structure, "step_deg": step_deg,
                             "g_max": g_max, "s_max": s_max, "max_spots": max_spots,
                             "n_directions": int(dirs.shape[0])})


# ----------------------------------------------------------------------------------
# Pattern renderer
# ----------------------------------------------------------------------------------

@dataclasses.dataclass
class Scan:
    frames: np.ndarray           # [P][H][W] uint16 or float32
    template: np.ndarray         # int64 [P], expanded index (mirror copies at k >= K0)
    angle: np.ndarray            # float64 [P], in-plane rotation applied, radians
    exact: np.ndarray            # bool [P], angle is an exact multiple of 2pi/n_theta
    centre: tuple


def _spot_pixels(ts: TemplateSet):
    """Spot positions in pixels relative to the beam, before rotation (x right, y down)."""
    if ts.coords == "polar":
        return ts.a * np.cos(ts.b), ts.a * np.sin(ts.b)
    return ts.a * ts.px_per_unit, ts.b * ts.px_per_unit


def render_scan(rng: np.random.Generator, ts: TemplateSet, n_patterns: int, H: int, W: int,
                n_theta: int, dtype=np.uint16, electrons: float = 2000.0,
                shares=(0.4, 0.4, 0.2), spot_sigma: float = 1.5, beam_sigma: float = 2.0,
                bg_scale: float | None = None, exact_every: int = 8, chunk: int = 1024,
                templates: np.ndarray | None = None, angles: np.ndarray | None = None) -> Scan:
    """Render ``n_patterns`` frames.  Pattern p shows template k_p ~ U{0..K-1} (K counts
    mirror copies when ``ts.mirror``; a mirror copy reflects ky -> -ky) rotated in plane by
    phi_p ~ U[0, 2pi); every ``exact_every``-th pattern uses phi = m 2pi/n_theta exactly.

    The expected image has three parts with the given shares of ``electrons``: Gaussian
    spots (sigma = spot_sigma, weight proportional to intensity), a Gaussian direct beam
    (sigma = beam_sigma) at the centre ((W-1)/2, (H-1)/2), and a radially exponential
    background exp(-rho/rho0), rho0 = W/8.  Counting noise is Poisson: the counts of each
    part are Poisson and each electron lands at a point drawn from its part's density and
    is binned to the pixel whose centre is nearest (pixel (i, j) is centred on x = j,
    y = i).  Electrons falling outside the frame are lost.  ``templates`` / ``angles`` fix the
    template and in-plane angle of every pattern instead.
    """
    K0 = ts.n_templates
    K = ts.n_expanded
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    rho0 = W / 8.0 if bg_scale is None else bg_scale
    if templates is None:
        tk = rng.integers(0, K, size=n_patterns)
    else:
        tk = np.asarray(templates, dtype=np.int64)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n_patterns)
    exact = np.zeros(n_patterns, dtype=bool)
    if angles is not None:                     # given in-plane angles (no exact subset)
        phi = np.asarray(angles, dtype=np.float64).copy()
    elif exact_every:
        exact[::exact_every] = True
        m = rng.integers(0, n_theta, size=int(exact.sum()))
        phi[exact] = m * (2.0 * math.pi / n_theta)

    sx, sy = _spot_pixels(ts)
    inten = ts.intensity
    csum = np.concatenate([[0.0], np.cumsum(inten)])
    tot = csum[ts.offsets[1:]] - csum[ts.offsets[:-1]]

    out = np.zeros((n_patterns, H, W), dtype=dtype)
    for c0 in range(0, n_patterns, chunk):
        c1 = min(n_patterns, c0 + chunk)
        n = c1 - c0
        base = tk[c0:c1] % K0
        mir = tk[c0:c1] >= K0
        ph = phi[c0:c1]
        n_sp = rng.poisson(electrons * shares[0], size=n)
        n_bm = rng.poisson(electrons * shares[1], size=n)
        n_bg = rng.poisson(electrons * shares[2], size=n)
        # spot electrons: choose a spot by intensity, then a Gaussian offset
        owner = np.repeat(np.arange(n), n_sp)
        bk = base[owner]
        has = tot[bk] > 0
        owner, bk = owner[has], bk[has]
        u = rng.random(owner.shape[0])
        target = csum[ts.offsets[bk]] + u * tot[bk]
        si = np.searchsorted(csum, target, side="right") - 1
        si = np.clip(si, ts.offsets[bk], ts.offsets[bk + 1] - 1)
        px, py = sx[si], sy[si]
        py = np.where(mir[owner], -py, py)
        c, s = np.cos(ph[owner]), np.sin(ph[owner])
        x_sp = cx + c * px - s * py + rng.normal(0.0, spot_sigma, owner.shape[0])
        y_sp = cy + s * px + c * py + rng.normal(0.0, spot_sigma, owner.shape[0])
        # direct beam
        own_b = np.repeat(np.arange(n), n_bm)
        x_bm = cx + rng.normal(0.0, beam_sigma, own_b.shape[0])
        y_bm = cy + rng.normal(0.0, beam_sigma, own_b.shape[0])
        # background: planar density exp(-rho/rho0) -> rho ~ Gamma(2, rho0)
        own_g = np.repeat(np.arange(n), n_bg)
        rho = rng.gamma(2.0, rho0, own_g.shape[0])
        ang = rng.uniform(0.0, 2.0 * math.pi, own_g.shape[0])
        x_bg = cx + rho * np.cos(ang)
        y_bg = cy + rho * np.sin(ang)

        xs = np.concatenate([x_sp, x_bm, x_bg])
        ys = np.concatenate([y_sp, y_bm, y_bg])
        ow = np.concatenate([owner, own_b, own_g])
        col = np.floor(xs + 0.5).astype(np.int64)
        row = np.floor(ys + 0.5).astype(np.int64)
        ok = (col >= 0) & (col < W) & (row >= 0) & (row < H)
        flat = (ow[ok] * H + row[ok]) * W + col[ok]
        counts = np.bincount(flat, minlength=n * H * W).reshape(n, H, W)
        if np.issubdtype(np.dtype(dtype), np.integer):
            counts = np.minimum(counts, np.iinfo(dtype).max)
        out[c0:c1] = counts.astype(dtype)
    return Scan(out, tk, phi, exact, (cx, cy))


# ----------------------------------------------------------------------------------
# Workload presets (sizes of the paper-shaped scans)
# ----------------------------------------------------------------------------------

def tiny_workload(n_side: int = 16, n_templates: int = 300):
    """16x16 scan of 128x128 float32 frames, 300 random templates (8-40 spots,
    r in [6, 60] px), polar grid 60 x 180, top-5, no mirrors."""
    rng = make_rng(0)
    ts = random_templates(rng, n_templates)
    scan = render_scan(rng, ts, n_side * n_side, 128, 128, n_theta=180, dtype=np.float32)
    return ts, scan, dict(n_r=60, n_theta=180, dr=1.0, gamma=0.5, top_n=5, prefilter=1.0)


def single_phase_workload(n_patterns: int = 16384, structure: str = "fcc", step_deg: float = 0.5,
                          max_spots: int = 150, stream: int = 0):
    """128x128 scan of 256x256 uint16 frames, kinematic FCC library at 0.5 deg with
    <= 150 spots, polar 128 x 360, prefilter keeps 50%.  ``stream`` selects an independent
    scan drawn from the same library (one per GPU when the scan is sharded)."""
    rng = make_rng(1, stream)
    ts = kinematic_library(structure, step_deg=step_deg, max_spots=max_spots)
    scan = render_scan(rng, ts, n_patterns, 256, 256, n_theta=360, dtype=np.uint16)
    return ts, scan, dict(n_r=128, n_theta=360, dr=1.0, gamma=0.5, top_n=5, prefilter=0.5)


def two_phase_workload(n_patterns: int = 4096, stream: int = 0, matrix_share: float = 0.5,
                       precipitate_fraction: float = 0.5):
    """The two-stage (masked) indexing workload shaped after Section 4.3: every pattern shows
    one matrix orientation (a single grain: FCC, one template and in-plane angle for the whole
    scan) with 2000 electrons; a fraction of the patterns also shows a precipitate template
    (HCP, random template and angle per pattern) with 500 electrons in its spots only.  The
    paper's G-phase precipitate library is not available; the HCP kinematic library stands
    in for it.  Returns (matrix TemplateSet, precipitate TemplateSet, frames u16 [n][256][256],
    dict of the truth)."""
    rng = make_rng(5, stream)
    fcc = kinematic_library("fcc")
    hcp = kinematic_library("hcp")
    k_m = int(rng.integers(0, fcc.n_expanded))
    phi_m = float(rng.uniform(0.0, 2.0 * math.pi))
    mat = render_scan(rng, fcc, n_patterns, 256, 256, n_theta=360,
                      shares=(matrix_share, (1.0 - matrix_share) * 0.7, (1.0 - matrix_share) * 0.3),
                      templates=np.full(n_patterns, k_m), angles=np.full(n_patterns, phi_m))
    pre = render_scan(rng, hcp, n_patterns, 256, 256, n_theta=360, electrons=500.0, shares=(1.0, 0.0, 0.0))
    has = rng.random(n_patterns) < precipitate_fraction
    frames = mat.frames.astype(np.int64)
    frames[has] += pre.frames[has]
    frames = np.minimum(frames, 65535).astype(np.uint16)
    truth = dict(matrix_template=k_m, matrix_angle=phi_m, has_precipitate=has,
                 precipitate_template=pre.template, precipitate_angle=pre.angle)
    return fcc, hcp, frames, truth


#: Kinematic settings of the batched three-phase workload.  Its spot counts must span
#: 20-250 per template; at the single-phase settings (|g| <= 1.2 1/A, |s| <= 0.02 1/A,
#: 0.01 1/A per pixel) the three phases give 2.8 / 6.7 / 12 spots on average, because the
#: reciprocal lattice within 1.2 1/A holds few points and the thin relrod against the Ewald
#: curvature keeps few of them.  Here the detector calibration is 0.02 1/A per pixel, so the
#: 128-pixel polar grid reaches |g| = 2.54 1/A, every template keeps the reflections up to
#: that radius, and the relrod reaches 0.05 1/A (a thinner specimen): FCC 24-77, HCP
#: 51-160, tetragonal 110-244 spots, the most intense 250 kept; no template falls below 20,
#: so none is dropped.
MULTIPHASE_KINEMATICS = dict(g_max=2.54, s_max=0.05, max_spots=250, px_per_unit=50.0)
MULTIPHASE_STRUCTURES = ("fcc", "hcp", "tetragonal")


def multiphase_libraries(step_deg: float = 0.5, min_spots: int = 20):
    """The three phase libraries of the batched workload (FCC a = 4.05 A, HCP a = 3.21 A
    c = 5.21 A, tetragonal a = 3.6 A c = 5.1 A at 200 kV over their fundamental triangles at
    ``step_deg``), with MULTIPHASE_KINEMATICS.  Templates with fewer than ``min_spots`` spots
    are dropped (their count is in ``meta["dropped"]``)."""
    out = []
    for s in MULTIPHASE_STRUCTURES:
        ts = kinematic_library(s, step_deg=step_deg, **MULTIPHASE_KINEMATICS)
        cnt = ts.spot_counts()
        keep = np.nonzero(cnt >= min_spots)[0]
        dropped = int(cnt.shape[0] - keep.shape[0])
        if dropped:
            sel = np.concatenate([np.arange(ts.offsets[k], ts.offsets[k + 1]) for k in keep])
            offs = np.zeros(keep.shape[0] + 1, dtype=np.int64)
            np.cumsum(cnt[keep], out=offs[1:])
            ts = TemplateSet(offs, ts.a[sel], ts.b[sel], ts.intensity[sel], coords=ts.coords,
                             px_per_unit=ts.px_per_unit, mirror=ts.mirror, meta=dict(ts.meta))
        ts.meta.update(dropped=dropped, min_spots=min_spots)
        out.append(ts)
    return out


def multiphase_workload(n_unique: int = 8192, stream: int = 0, step_deg: float = 0.5):
    """Frames of the batched three-phase scan (256 x 256 u16, polar 128 x 360): pattern p
    shows a random template of phase truth[p] (phases drawn uniformly), rendered as
    ``render_scan`` does with the libraries' own calibration.  Every pattern is indexed
    against all three libraries (top-5 per phase).  Returns (libraries, frames, truth phase,
    truth template, parameters)."""
    libs = multiphase_libraries(step_deg)
    rng = make_rng(2, stream)
    phase = rng.integers(0, len(libs), size=n_unique)
    frames = np.zeros((n_unique, 256, 256), dtype=np.uint16)
    tmpl = np.zeros(n_unique, dtype=np.int64)
    for i, ts in enumerate(libs):
        idx = np.nonzero(phase == i)[0]
        if idx.shape[0]:
            sc = render_scan(rng, ts, idx.shape[0], 256, 256, n_theta=360)
            frames[idx] = sc.frames
            tmpl[idx] = sc.template
    return libs, frames, phase, tmpl, dict(n_r=128, n_theta=360, dr=1.0, gamma=0.5, top_n=5, prefilter=1.0)


def large_map_workload(n_unique: int = 16384, stream: int = 0, step_deg: float = 0.5):
    """Distinct frames of the large single map (512 x 512 scan of 256 x 256 u16 frames, HCP
    a = 3.21 A c = 5.21 A at 0.5 deg with mirrors, at most 250 spots, polar 128 x 360, top-5);
    the full map repeats these ``n_unique`` frames.  Returns (library, scan, parameters)."""
    rng = make_rng(4, stream)
    ts = kinematic_library("hcp", step_deg=step_deg, max_spots=250)
    scan = render_scan(rng, ts, n_unique, 256, 256, n_theta=360, dtype=np.uint16)
    return ts, scan, dict(n_r=128, n_theta=360, dr=1.0, gamma=0.5, top_n=5, prefilter=1.0)
