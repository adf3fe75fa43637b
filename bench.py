#!/usr/bin/env python
#!/usr/bin/env python
"""Throughput of the template-matching indexing path on one GB300 (or N, sharded).

Headline workload (one step): the large single map -- 512 x 512 = 262144 diffraction frames
of 256 x 256 uint16 (16384 distinct rendered frames repeated on the device; 2.1 GB of distinct
frames, 34 GB per step, larger than the 129 MB L2, so no flush), kinematic HCP (a = 3.21 A,
c = 5.21 A, 200 kV) templates over the hexagonal fundamental triangle at 0.5 deg with mirrors
(at most 250 spots), polar grid 128 r x 360 theta, gamma 0.5, top-5 -- indexed through the
library's public call (tm_index_patterns) by the FP32 sparse path and by the BF16 tensor-core
pre-score + FP32 rescore path.  `value` is the faster path whose top-1 matches the FP64
oracle on >= 99.5 % of a seeded subset of the distinct frames (Wilson 95 % interval given).
Also measured: the batched three-phase scan (65536 frames against FCC, HCP and tetragonal
libraries of 20-250 spots per template, one call, top-5 per phase) and the single-phase scan
(16384 frames, FCC with the radial pre-filter keeping 50 %), both paths each; the serving
loop; the two-stage masked workflow; preprocessing; template simulation.

`--impl reference` times the FP64 CPU oracle on the host cores on bounded samples of the
headline workload (there is no other reference implementation of this paper).

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "patterns/s indexed, BF16-TC vs FP32 sparse at ≥99.5% top-1 match; p99 line ms"
N_R, N_THETA, TOP_N = 128, 360, 5
E2E_CHUNK = 4096                  # patterns per chunk of the host-buffer entry point (tm_index_patterns_host)
# tensor-core work per (pattern, scored template): 2 x 180 shifts x (182 + 180) frequency terms
DENSE_FLOPS_PER_PAIR = 2 * 180 * (182 + 180)
# rescore_k: candidates of the BF16 pre-score rescored exactly; the configured 64 where it meets the
# top-1 bar, 256 on the FCC library, whose 2-spot templates have hundreds of near-ties
LARGE_MAP = dict(total=262144, unique=16384, rescore_k=64)
MULTIPHASE = dict(total=65536, unique=8192, rescore_k=64)
SINGLE_PHASE = dict(total=16384, prefilter=0.5, rescore_k=256)
WORKLOAD = ("large single map: 262144 x 256x256 u16 frames (16384 distinct, repeated), HCP 0.5 deg (+mirrors, "
            "<= 250 spots), polar 128x360, top-5; BF16 tensor-core pre-score + FP32 rescore vs FP32 sparse")
try:
    MEASURED = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
except Exception:
    MEASURED = {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paths", default="fp32,bf16", help="paths to time (fp32, bf16)")
    ap.add_argument("--workloads", default="large_map,multiphase,single_phase",
                    help="workloads to run; the first is the headline")
    ap.add_argument("--oracle-patterns", type=int, default=4096,
                    help="distinct frames of the headline workload checked against the FP64 oracle")
    ap.add_argument("--oracle-multiphase", type=int, default=192, help="patterns of the three-phase scan checked")
    ap.add_argument("--path-seconds", type=float, default=20.0,
                    help="timed steps of a slow path are reduced (to no fewer than 3) to fit this many seconds")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop latency run")
    ap.add_argument("--serving-seconds", type=float, default=30.0, help="seconds per offered-load level")
    ap.add_argument("--no-two-stage", action="store_true", help="skip the two-stage (masked) indexing run")
    ap.add_argument("--no-preprocess", action="store_true", help="skip the background-removal and blur timing")
    ap.add_argument("--total", type=int, default=0, help="patterns per step (0: the workload's; smaller for profiling)")
    ap.add_argument("--distinct", type=int, default=0, help="distinct rendered frames (0: the workload's)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner: the default shape, or the one a TMGB_TUNE_CACHE file holds")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def wilson(k: int, n: int, z: float = 1.96):
    """Wilson score interval of a binomial proportion k / n."""
    if n == 0:
        return [0.0, 1.0]
    p = k / n
    d = 1 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return [max(0.0, c - h), min(1.0, c + h)]


# ------------------------------------------------------------------ clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[4:]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, flags in rows:
            for nm, v in zip(names[1:], flags[1:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ helpers

def to_device_u16(a: np.ndarray, device):
    import torch
    return torch.from_numpy(a.view(np.int16)).to(device).view(torch.uint16)


def pinned_u16(a: np.ndarray):
    """Pinned host copy of a uint16 array: (torch uint16 view, numpy uint16 view)."""
    import torch
    t = torch.from_numpy(a.view(np.int16)).pin_memory()
    return t.view(torch.uint16), t.numpy().view(np.uint16)


def kernel_sha(path: str) -> str:
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_from_profiles(kernel_file: str, key: str, units: float):
    """DRAM bytes of one launch that processes `units` units of work, from the committed ncu
    summary `profiles/traffic.txt` (lines: kernel, sha256[:16] of its source file, bytes per unit,
    unit, capture), if it was taken on this source; None otherwise."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(p):
            f = line.split()
            if len(f) >= 4 and not f[0].startswith("#") and f[0] == key and f[1] == kernel_sha(kernel_file):
                return float(f[2]) * units
    except OSError:
        pass
    return None


# ------------------------------------------------------------------ the FP64 oracle on samples

def oracle_index(ts_list, frames: np.ndarray, prefilter: float = 1.0, chunk: int = 512):
    """The FP64 oracle, as it stands, on `frames` against each library: per library a dict of
    the top-N rows and every template's best Q; the wall time of the oracle calls."""
    from oracle import oracle as O
    libs = [O.prepare_library(ts, N_R, N_THETA) for ts in ts_list]
    refs = [dict(template=[], shift=[], score=[], q_best=[]) for _ in libs]
    t = time.perf_counter()
    for c0 in range(0, frames.shape[0], chunk):
        for li, lib in enumerate(libs):
            r = O.index(frames[c0:c0 + chunk], lib, prefilter_fraction=prefilter, N=TOP_N)
            for k in refs[li]:
                refs[li][k].append(r[k])
    dt = time.perf_counter() - t
    refs = [{k: np.concatenate(v) for k, v in r.items()} for r in refs]
    return libs, refs, dt, O.num_threads()


def top1_agrees(h, ref) -> np.ndarray:
    """Per pattern: the GPU's top-1 row is the oracle's (template and shift), or a template whose
    exact best Q lies within the score tolerance (1e-5 relative) of the oracle's best (a near-tie)."""
    n = h.shape[0]
    ok = np.zeros(n, dtype=bool)
    for i in range(n):
        k0 = int(h["template_index"][i, 0])
        qt = ref["score"][i, 0]
        t = 1e-5 * max(abs(qt), 1e-30)
        same = k0 == ref["template"][i, 0] and h["shift"][i, 0] == ref["shift"][i, 0]
        near = k0 >= 0 and np.isfinite(ref["q_best"][i, k0]) and abs(ref["q_best"][i, k0] - qt) <= t
        ok[i] = same or near
    return ok


def match_record(ok: np.ndarray) -> dict:
    k, n = int(ok.sum()), int(ok.shape[0])
    return {"matched": k, "patterns": n, "rate": k / max(1, n), "wilson95": wilson(k, n)}


def recall_record(ctx, lid, frames_np, ref, device, ks=(64, 256)) -> dict:
    """BF16 pre-score of every template for the sampled frames (tm_prescore): recall@k = share
    of patterns whose oracle top-1 (or a template within 1e-5 of its exact Q) is among the k best
    pre-scores; the pre-score error |Q~ - Q| relative to the pattern's exact top-1 Q."""
    import torch
    fr = to_device_u16(frames_np, device)
    polar, norm, radial = ctx.polar_transform(fr, N_R, N_THETA)
    pre = ctx.prescore(lid, polar, norm).cpu().numpy().astype(np.float64)
    del polar, norm, radial, fr
    torch.cuda.empty_cache()
    q = ref["q_best"]
    top = ref["score"][:, 0]
    good = np.abs(q - top[:, None]) <= 1e-5 * np.maximum(np.abs(top[:, None]), 1e-30)
    out = {}
    order = np.argsort(-pre, axis=1, kind="stable")
    for k in ks:
        hit = np.take_along_axis(good, order[:, :k], axis=1).any(axis=1)
        out[f"recall@{k}"] = float(hit.mean())
    err = np.abs(pre - q) / np.maximum(np.abs(top[:, None]), 1e-30)
    fin = np.isfinite(err)                  # templates without a finite Q (no spot on the grid) left out
    err = err[fin]
    out["prescore_err_rel_top1"] = {"median": float(np.median(err)), "p99": float(np.percentile(err, 99)),
                                    "max": float(err.max()), "pairs_left_out": int((~fin).sum())}
    return out


# ------------------------------------------------------------------ two-stage (masked) indexing

def simulation_bench(ctx, stream) -> dict:
    """Template simulation on the device (Section 2.1) over the 0.5 deg orientation grids of
    the FCC and HCP libraries: orientations per second, inputs resident on the device."""
    import torch
    from paper_2111_07347_gb300 import synth
    out = {}
    for name, system in (("fcc", "cubic"), ("hcp", "hexagonal")):
        st = synth.STRUCTURES[name]
        g, F2, gn = synth._reciprocal_points(st, 1.2)
        dirs = synth.beam_directions(system, 0.5)
        R = np.stack([synth._orientation_matrix(d) for d in dirs])
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
        gd, fd, nd, rd = t(g), t(F2), t(gn), t(R)
        ctx.kinematic_spots(gd, fd, nd, rd, synth.WAVELENGTH_200KV, 0.02, 150, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            counts, _ = ctx.kinematic_spots(gd, fd, nd, rd, synth.WAVELENGTH_200KV, 0.02, 150, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        out[name] = {"orientations": int(R.shape[0]), "points": int(g.shape[0]), "ms": ms,
                     "orientations_per_s": R.shape[0] / (ms / 1e3),
                     "spots": int(counts.sum().item())}
    return out


def preprocess_bench(ctx, stream, frames_d, steps: int) -> dict:
    """Section 3.1's background removal (difference of Gaussians, sigmas 1 and 4 px) and blur
    (1 px) of the scan's frames, as tm_preprocess runs them before indexing.  HBM bytes: the
    u16 frames read and the float frames written, plus the intermediates of the passes (the
    row pass writes two float images, the column pass reads them)."""
    import torch
    n, H, W = frames_d.shape
    out = torch.empty((n, H, W), dtype=torch.float32, device=frames_d.device)
    kw = dict(dog=(1.0, 4.0), blur=1.0)
    for _ in range(2):
        ctx.preprocess(frames_d, out=out, stream=stream, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.preprocess(frames_d, out=out, stream=stream, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    px = n * H * W
    # rows (u16 in, 2 floats out) + columns (2 floats in, 1 out) + blur rows (1 in, 1 out) + columns (1 in, 1 out)
    bytes_ = px * (2 + 8 + 8 + 4 + 4 + 4 + 4 + 4)
    peak = MEASURED.get("hbm_gbs") or 6800.0
    del out
    return {"ms_per_step": ms, "frames_per_s": n / (ms / 1e3), "sigmas": "difference of Gaussians 1 / 4 px, blur 1 px",
            "hbm_gbs": bytes_ / (ms / 1e3) / 1e9, "hbm_frac": bytes_ / (ms / 1e3) / 1e9 / peak,
            "algorithmic_bytes_per_step": bytes_}


def two_stage_bench(ctx, stream, steps: int, n_total: int = 16384, unique: int = 2048) -> dict:
    """The masked indexing of Section 4.3 on the two-phase scan (single-grain FCC matrix, HCP
    precipitates in half of the patterns): per step the per-pixel sums over the scan, the
    mask (threshold 1 count per pattern, one opening, two dilations) and the FP32 indexing of
    the masked patterns against the precipitate library (unit intensities, subtraction 0.4).
    The scan is `unique` rendered frames repeated on the device."""
    import torch
    from paper_2111_07347_gb300 import synth
    fcc, hcp, frames, truth = synth.two_phase_workload(unique)
    base = torch.from_numpy(frames.view(np.int16)).cuda()
    dev = base.repeat(n_total // unique, 1, 1).view(torch.uint16)
    lh = ctx.load_library(hcp, N_R, N_THETA, unit_intensity=True)
    out = torch.empty((1, n_total, TOP_N, 5), dtype=torch.int32, device="cuda")
    sums = torch.empty((256, 256), dtype=torch.float64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def step(rec):
        if rec:
            ev[0].record(stream)
        ctx.frame_sum(dev, out=sums)
        if rec:
            ev[1].record(stream)
        mask = ctx.matrix_mask(sums, n_total, 1.0, n_open=1, n_dilate=2)
        if rec:
            ev[2].record(stream)
        ctx.index(dev, lh, top_n=TOP_N, subtract=0.4, mask=mask, out=out)
        if rec:
            ev[3].record(stream)
        return mask

    for _ in range(2):
        step(False)
    torch.cuda.synchronize()
    t = np.zeros(3)
    for _ in range(steps):
        mask = step(True)
        torch.cuda.synchronize()
        t += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])]
    t /= steps
    ms = float(t.sum())
    masked = int((mask == 0).sum().item())
    ctx.unload_library(lh)
    return {"patterns_per_s": n_total / (ms / 1e3), "ms_per_step": ms, "sum_ms": float(t[0]), "mask_ms": float(t[1]),
            "index_ms": float(t[2]), "sum_gbs": n_total * 256 * 256 * 2 / (t[0] / 1e3) / 1e9,
            "masked_pixels": masked, "patterns": n_total, "library": f"HCP 0.5 deg, {hcp.n_expanded} templates",
            "workload": "two-phase scan (FCC single grain + HCP precipitates in half the patterns), "
                        f"{unique} rendered 256x256 u16 frames repeated to {n_total}"}


# ------------------------------------------------------------------ serving loop (scan lines and maps)

def serve_bench(ctx, lib_ids, line_pool: np.ndarray, map_pool, path_kw: dict, seconds: float = 30.0,
                line_rate: float = 40.0, seed: int = 2111_07347 + 103):
    """The serving workload: FCC + HCP libraries resident; two Poisson streams.  Scan lines
    (64-512 patterns from a pinned host pool, as a detector delivers them) arrive at
    `line_rate` per second; whole maps (side uniform in {64, 128, 256, 512}, frames already on the
    device) arrive at the rate that brings the offered load to 25 / 50 / 80 % of the capacity,
    which is measured first with a saturating burst of maps.  Each level runs `seconds`.  Latency
    = result ready - arrival (a late submission counts from its intended arrival); the admission
    wait and the device time of copies and kernels come from the server's per-request timeline."""
    from paper_2111_07347_gb300 import tmgb
    rng = np.random.default_rng(seed)
    srv = tmgb.Server(ctx, slots=4, tile_patterns=512, max_libs=len(lib_ids), max_top_n=TOP_N, priority_slots=1,
                      hbm_budget_bytes=1 << 30)
    n_line, n_map = line_pool.shape[0], map_pool.shape[0]
    sides = [64, 128, 256, 512]

    def submit_line(n):
        a = int(rng.integers(0, n_line - n + 1))
        return srv.submit(line_pool[a:a + n], lib_ids, top_n=TOP_N, priority=1, **path_kw)

    def submit_map(side):
        n = side * side
        a = int(rng.integers(0, n_map - n + 1))
        return srv.submit(map_pool[a:a + n], lib_ids, top_n=TOP_N, priority=0, **path_kw)

    # capacity: a saturating burst of maps
    t0 = time.perf_counter()
    burst = [submit_map(256) for _ in range(8)]
    for t in burst:
        srv.wait(t, timeout_ms=600000)
    cap = 8 * 65536 / (time.perf_counter() - t0)
    mean_line = (64 + 512) / 2
    mean_map = float(np.mean([s_ * s_ for s_ in sides]))
    out = {"capacity_patterns_per_s": cap, "slots": 4, "priority_slots": 1, "tile_patterns": 512,
           "line_rate_per_s": line_rate, "seconds_per_level": seconds,
           "maps": "sides 64, 128, 256, 512 (device-resident frames)", "lines": "64-512 patterns, pinned host frames"}
    for load in (0.25, 0.5, 0.8):
        map_rate = max(0.0, (load * cap - line_rate * mean_line) / mean_map)
        arrivals = []
        t = 0.0
        while True:
            t += rng.exponential(1.0 / line_rate)
            if t >= seconds:
                break
            arrivals.append((t, "line", int(rng.integers(64, 513))))
        t = 0.0
        while map_rate > 0:
            t += rng.exponential(1.0 / map_rate)
            if t >= seconds:
                break
            arrivals.append((t, "map", int(rng.choice(sides))))
        arrivals.sort()
        start = time.perf_counter()
        tickets = []
        for at, kind, size in arrivals:
            now = time.perf_counter() - start
            if now < at:
                time.sleep(at - now)
            lag_ms = max(0.0, (time.perf_counter() - start - at) * 1e3)
            tk = submit_line(size) if kind == "line" else submit_map(size)
            tickets.append((kind, size if kind == "line" else size * size, tk, lag_ms))
        lat = {"line": [], "map": []}
        tl = {"admit": [], "queue": [], "h2d": [], "kernels": [], "d2h": []}
        pats, first, last = 0, None, None
        for kind, n, tk, lag in tickets:
            res, st = srv.wait(tk, timeout_ms=600000)
            lat[kind].append(lag + st["done_ms"] - st["submit_ms"])
            if kind == "line":
                tl["admit"].append(lag + st["admit_ms"] - st["submit_ms"])
                tl["queue"].append(st["first_dispatch_ms"] - st["admit_ms"])
                tl["h2d"].append(st["h2d_ms"])
                tl["kernels"].append(st["kernels_ms"])
                tl["d2h"].append(st["d2h_ms"])
            pats += n
            first = st["submit_ms"] if first is None else min(first, st["submit_ms"])
            last = st["done_ms"] if last is None else max(last, st["done_ms"])
        rec = {"offered_load": load, "lines": len(lat["line"]), "maps": len(lat["map"]),
               "throughput_patterns_per_s": pats / max(1e-9, (last - first) / 1e3)}
        for kind in ("line", "map"):
            if lat[kind]:
                rec[f"{kind}_p50_ms"] = float(np.percentile(lat[kind], 50))
                rec[f"{kind}_p99_ms"] = float(np.percentile(lat[kind], 99))
        if lat["line"]:
            rec["line_p999_ms"] = float(np.percentile(lat["line"], 99.9))
            rec["line_timeline_mean_ms"] = {k: float(np.mean(v)) for k, v in tl.items()}
        out[f"load_{int(load * 100)}"] = rec
    srv.close()
    return out


# ------------------------------------------------------------------ reference arm: the oracle

def run_reference(args):
    rank, local, world = dist_env()
    if rank != 0:
        return 0
    from paper_2111_07347_gb300 import synth
    from oracle import oracle as O
    ts, scan, _ = synth.large_map_workload(n_unique=4096)
    lib = O.prepare_library(ts, N_R, N_THETA)
    per_step = 32
    # size the step so that warmup + steps stay within about two minutes
    t = time.perf_counter()
    O.index(scan.frames[:per_step], lib, N=TOP_N)
    dt = time.perf_counter() - t
    budget = 120.0 / max(1, args.steps + args.warmup)
    per_step = int(max(8, min(4096, per_step * budget / max(dt, 1e-3))))
    n = scan.frames.shape[0]
    for i in range(args.warmup):
        a = (i * per_step) % max(1, n - per_step)
        O.index(scan.frames[a:a + per_step], lib, N=TOP_N)
    times = []
    for i in range(args.steps):
        a = ((args.warmup + i) * per_step) % max(1, n - per_step)
        t = time.perf_counter()
        O.index(scan.frames[a:a + per_step], lib, N=TOP_N)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "patterns/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "patterns_per_step": per_step, "note": "bounded sample per step"},
            "cpu_baseline": {"value": value, "unit": "patterns/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{per_step} patterns per step of the large map's frames, FP64 oracle, "
                                       "whole path (polar, Q at every shift, top-5)"},
            "e2e": {"value": value, "unit": "patterns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

class Timer:
    """Device time of repeated steps on `stream` (CUDA events), with the contract's warm-up,
    clock sampling during the timed region and a max over ranks."""

    def __init__(self, args, stream, local, world):
        self.args, self.stream, self.local, self.world = args, stream, local, world

    def run(self, step, calls_per_step=1, ctx=None, headline=True):
        import torch
        args = self.args
        t = time.perf_counter()
        step()
        torch.cuda.synchronize()
        first = time.perf_counter() - t
        # three warm-up steps at least; the workloads after the headline take exactly three
        warm = max(3, args.warmup) if headline else 3
        for _ in range(warm - 1):
            step()
        torch.cuda.synchronize()
        if ctx is not None:
            ctx.check()
        steps = args.steps
        if first * steps > args.path_seconds:
            steps = max(3, int(args.path_seconds / max(first, 1e-9)))
        launches = ctx.last_stats["launches"] * calls_per_step if ctx is not None else 0
        clocks = ClockSampler(self.local)
        clocks.start()
        time.sleep(0.3)
        if self.world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(steps):
            step()
        e1.record(self.stream)
        torch.cuda.synchronize()
        if self.world > 1:
            torch.distributed.barrier()
        clk = clocks.stop()
        if ctx is not None:
            ctx.check()
        ms = e0.elapsed_time(e1) / steps
        if self.world > 1:
            tt = torch.tensor([ms], device=torch.device("cuda", self.local))
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            ms = float(tt.item())
        return {"ms": ms, "steps": steps, "warmup": warm, "clocks": clk, "launches_per_step": launches}

    def profile(self, ctx, step, steps=3):
        """Stage times and the sparse kernel's executed multiply-adds from a second pass of the
        same steps with stage timing on (events between the stages; not the timing of record)."""
        import torch
        ctx.profile_enable(True)
        for _ in range(steps):
            step()
        torch.cuda.synchronize()
        prof, counters = ctx.profile_read(counters=True)
        ctx.profile_enable(False)
        ctx.check()
        return prof, counters, steps


def sparse_roofline(prof, counters, prof_steps, macs_step, clk, sm, patterns_step):
    """Shared-memory roofline of sparse_kernel: one 4-byte operand per FP32 multiply-add.  frac is
    the executed work (the multiply-adds the kernel ran, counted while profiling) over the peak;
    the algorithmic fraction counts every template the definition scores, including those the
    exact bound pruning skips."""
    sp_ms, sp_l = prof.get("sparse", (0.0, 0))
    if not sp_l:
        return None
    per_launch_ms = sp_ms / sp_l
    lps = max(1, sp_l // prof_steps)
    fm = clk.get("sm_mhz") or 2070.0
    peak = 128.0 * sm * fm * 1e6 / 1e9
    ex = counters.get("sparse_macs", 0) / sp_l
    alg = macs_step / lps
    ex_gbs = 4.0 * ex / (per_launch_ms / 1e3) / 1e9
    alg_gbs = 4.0 * alg / (per_launch_ms / 1e3) / 1e9
    return {"bound": "smem", "kernel": "sparse_kernel", "achieved": ex_gbs, "peak": peak, "unit": "GB/s",
            "frac": ex_gbs / peak, "traffic": traffic_from_profiles(
                os.path.join(ROOT, "paper_2111_07347_gb300", "csrc", "k_sparse.cu"), "sparse_kernel",
                patterns_step / lps),
            "work": "4 B of shared memory per FP32 multiply-add executed (one polar sample per spot x shift "
                    "of every template the kernel scores)",
            "macs_executed_per_launch": ex, "macs_algorithmic_per_launch": alg,
            "skipped_share": 1.0 - ex / alg if alg else None,
            "algorithmic_achieved": alg_gbs, "algorithmic_frac": alg_gbs / peak,
            "peak_basis": f"128 B/clk/SM x {sm} SMs x {fm:.0f} MHz (median SM clock sampled in the run)",
            "launch_ms": per_launch_ms}


def dense_roofline(prof, prof_steps, pairs_step):
    d_ms, d_l = prof.get("dense", (0.0, 0))
    if not d_l:
        return None
    per_launch_ms = d_ms / d_l
    lps = max(1, d_l // prof_steps)
    flops = DENSE_FLOPS_PER_PAIR * pairs_step / lps
    achieved = flops / (per_launch_ms / 1e3) / 1e12
    peak = MEASURED.get("bf16_tflops_sustained") or 1700.0
    return {"bound": "tensor", "kernel": "dense_kernel", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic_from_profiles(
                os.path.join(ROOT, "paper_2111_07347_gb300", "csrc", "k_dense.cu"), "dense_kernel", pairs_step / lps),
            "work": f"{DENSE_FLOPS_PER_PAIR} flop per (pattern, scored template): inverse DFT over "
                    "182 even + 180 odd frequency terms for 180 shifts",
            "peak_basis": "measured sustained cuBLAS bf16 (MEASURED_PEAKS.json)", "launch_ms": per_launch_ms}


def polar_roofline(prof, prof_steps, n, kept_rows):
    """HBM roofline of polar_kernel per launch: the frame read once, the kept rows written, the
    azimuthal sums and the norm."""
    pol_ms, pol_l = prof.get("polar", (0.0, 0))
    if not pol_l:
        return None
    ms = pol_ms / pol_l
    per_launch = n * prof_steps / pol_l
    hbm_bytes = per_launch * (256 * 256 * 2 + kept_rows * N_THETA * 4 + N_R * 4 + 4)
    gbs = hbm_bytes / (ms / 1e3) / 1e9
    peak = MEASURED.get("hbm_gbs") or 6800.0
    tr = traffic_from_profiles(os.path.join(ROOT, "paper_2111_07347_gb300", "csrc", "k_polar.cu"), "polar_kernel",
                               per_launch)
    return {"bound": "hbm", "kernel": "polar_kernel", "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak, "algorithmic_bytes_per_launch": hbm_bytes, "traffic": tr,
            "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)", "launch_ms": ms,
            "ms_per_step": pol_ms / prof_steps}


def sparse_work(ctx, lids, frames_d, prefilter):
    """Multiply-adds (spots x shifts) of every template the definition scores per step, and the
    number of (pattern, template) pairs scored, from the libraries' shapes and, with the
    pre-filter, its masks."""
    import torch
    dev = frames_d.device
    n = frames_d.shape[0]
    macs, pairs = 0.0, 0.0
    for lid in lids:
        exp = ctx.library_export(lid)
        spots_k = np.diff(exp["offsets"]).astype(np.float64)
        wk = spots_k * (N_THETA // exp["order"])
        if prefilter >= 1.0:
            macs += n * float(wk.sum())
            pairs += n * float(wk.shape[0])
            continue
        K = wk.shape[0]
        work_k = torch.from_numpy(wk).to(dev)
        for c0 in range(0, n, 4096):
            polar, norm, radial = ctx.polar_transform(frames_d[c0:c0 + 4096], N_R, N_THETA)
            mask, _ = ctx.prefilter(lid, radial, prefilter)
            bits = ((mask.view(torch.int32).unsqueeze(-1) >> torch.arange(32, device=dev, dtype=torch.int32)) & 1)
            active = bits.reshape(mask.shape[0], -1)[:, :K].to(torch.float64)
            macs += float((active @ work_k).sum().item())
            pairs += float(active.sum().item())
            del polar, norm, radial, mask, bits, active
    torch.cuda.synchronize()
    return macs, pairs


def bench_workload(args, ctx, timer, name, libs_ts, lids, frames_d, frames_np_unique, sample_idx, prefilter,
                   oracle_n, local, dev, world, want_paths, rank, rescore_k, subsets=None, headline=True):
    """Both paths on one workload: device-timed patterns/s, stages, rooflines, and top-1 against
    the FP64 oracle on sampled distinct frames."""
    import torch
    from paper_2111_07347_gb300 import tmgb
    n = frames_d.shape[0]
    L = len(lids)
    subsets = subsets or {}
    sm = torch.cuda.get_device_properties(local).multi_processor_count
    kws = {"fp32": dict(top_n=TOP_N, prefilter=prefilter, path=tmgb.TM_PATH_FP32_SPARSE),
           "bf16": dict(top_n=TOP_N, prefilter=prefilter, path=tmgb.TM_PATH_BF16_RESCORE, rescore_k=rescore_k)}
    out = torch.empty((L, n, TOP_N, 5), dtype=torch.int32, device=dev)
    macs_step, pairs_step = sparse_work(ctx, lids, frames_d, prefilter)
    # the sparse kernel's shape (block size x seeds per warp on 2048 frames, then the patterns
    # bounded together on up to 16384) chosen by the library's autotuner for these libraries, on
    # the first frames of the scan (outside every timed region)
    tune_n = 256 if name == "multiphase" else 16384
    t0 = time.perf_counter()
    tuned_threads = None if args.no_autotune else ctx.autotune(frames_d[:tune_n], lids, top_n=TOP_N, prefilter=prefilter)
    tune_s = time.perf_counter() - t0
    res, hits = {}, {}
    for nm in want_paths:
        kw = kws[nm]
        # a path slower than a few seconds per full step is timed on the first `sub` patterns
        # (whole passes over the distinct frames, so the per-pattern work is the step's own)
        sub = subsets.get(nm, n)
        fr, ot = frames_d[:sub], out[:, :sub]

        def step(kw=kw, fr=fr, ot=ot):
            ctx.index(fr, lids, out=ot, **kw)
        try:
            r = timer.run(step, ctx=ctx, headline=headline)
        except tmgb.TmError as e:
            res[nm] = {"unsupported": str(e)}
            continue
        prof, counters, ps = timer.profile(ctx, step, steps=min(3 if sub == n else 1, r["steps"]))
        r["stages"] = {k: {"ms_per_step": v[0] / ps * n / sub, "launches_per_step": v[1] / ps}
                       for k, v in prof.items()}
        r["prof"], r["counters"], r["prof_steps"] = prof, counters, ps
        r["patterns_timed"] = sub
        r["ms_timed"] = r["ms"]
        r["ms"] = r["ms"] * n / sub                      # per full step of n patterns
        r["patterns_per_s"] = world * n / (r["ms"] / 1e3)
        res[nm] = r
        if sub < n:
            ctx.index(frames_d, lids, out=out, **kw)     # the whole scan, for the oracle comparison
        hits[nm] = tmgb.hits_to_numpy(out[:, torch.from_numpy(sample_idx).to(dev)])
    kept_rows = len(set().union(*[set(np.unique(ctx.library_export(l)["r"]).tolist()) for l in lids]))
    rec = {"patterns": n, "libraries": [ctx.library_info(l)["n_templates"] for l in lids],
           "spots_per_template": [round(ctx.library_info(l)["n_spots"] / ctx.library_info(l)["n_templates"], 2)
                                  for l in lids],
           "autotune": {"frames": tune_n, "block_threads": tuned_threads, "seconds": tune_s},
           "prefilter": prefilter, "rescore_k": rescore_k, "macs_per_step_sparse": macs_step,
           "pairs_per_step": pairs_step, "paths": {}}
    match, recall, oracle_info = {}, {}, None
    if rank == 0 and oracle_n and hits:
        sub = frames_np_unique[sample_idx % frames_np_unique.shape[0]]
        olibs, refs, dt, cores = oracle_index(libs_ts, sub, prefilter)
        oracle_info = {"patterns": int(sub.shape[0]), "seconds": dt, "cores": cores,
                       "patterns_per_s": sub.shape[0] / dt}
        for nm, h in hits.items():
            per = [match_record(top1_agrees(h[li], refs[li])) for li in range(L)]
            allok = np.concatenate([top1_agrees(h[li], refs[li]) for li in range(L)])
            match[nm] = {"all": match_record(allok), "per_library": per}
        if "bf16" in hits and L == 1:
            recall = recall_record(ctx, lids[0], sub, refs[0], dev, ks=(64, 256))
    for nm, r in res.items():
        if "unsupported" in r:
            rec["paths"][nm] = r
            continue
        frac_sub = r["patterns_timed"] / n
        roof = (dense_roofline(r["prof"], r["prof_steps"], pairs_step * frac_sub) if nm == "bf16"
                else sparse_roofline(r["prof"], r["counters"], r["prof_steps"], macs_step * frac_sub, r["clocks"], sm,
                                     r["patterns_timed"]))
        rec["paths"][nm] = {"patterns_per_s": r["patterns_per_s"], "ms_per_step": r["ms"], "steps": r["steps"],
                            "patterns_timed": r["patterns_timed"], "ms_per_timed_step": r["ms_timed"],
                            "warmup": r["warmup"], "clocks": r["clocks"], "stages": r["stages"],
                            "roofline": roof, "launches_per_step": r["launches_per_step"],
                            "polar_roofline": polar_roofline(r["prof"], r["prof_steps"], r["patterns_timed"], kept_rows),
                            "top1_vs_oracle": match.get(nm)}
        if nm == "fp32" and r["counters"].get("sparse_macs"):
            rec["paths"][nm]["sparse_macs_executed_per_step"] = (r["counters"]["sparse_macs"] / r["prof_steps"] /
                                                                 frac_sub)
    if "fp32" in rec["paths"] and "bf16" in rec["paths"] and "ms_per_step" in rec["paths"]["bf16"] \
            and "ms_per_step" in rec["paths"]["fp32"]:
        rec["speedup_bf16_vs_fp32"] = rec["paths"]["fp32"]["ms_per_step"] / rec["paths"]["bf16"]["ms_per_step"]
    if recall:
        rec["paths"]["bf16"]["candidates"] = recall
    if oracle_info:
        rec["oracle_sample"] = oracle_info
    rec["correlations_per_step"] = pairs_step * N_THETA
    del out
    return rec, res


def run_ours(args):
    import torch
    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2111_07347_gb300 import build, synth, tmgb
    build.build()
    ctx = tmgb.Context(local)
    stream = torch.cuda.current_stream()
    timer = Timer(args, stream, local, world)
    want_paths = [x.strip() for x in args.paths.split(",") if x.strip()]
    wls = [w.strip() for w in args.workloads.split(",") if w.strip()]
    line = {"metric": METRIC, "unit": "patterns/s", "n_gpus": world, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "workloads": {}}
    head_done = False
    for wi, wl in enumerate(wls):
        if wl == "large_map":
            ts, scan, _ = synth.large_map_workload(n_unique=args.distinct or LARGE_MAP["unique"], stream=rank)
            uniq = scan.frames
            libs_ts = [ts]
            total = args.total or LARGE_MAP["total"]
            prefilter = 1.0
            oracle_n = args.oracle_patterns
            rk = LARGE_MAP["rescore_k"]
        elif wl == "multiphase":
            libs_ts, uniq, phase, _, _ = synth.multiphase_workload(n_unique=args.distinct or MULTIPHASE["unique"],
                                                                   stream=rank)
            total = args.total or MULTIPHASE["total"]
            prefilter = 1.0
            oracle_n = args.oracle_multiphase
            rk = MULTIPHASE["rescore_k"]
        elif wl == "single_phase":
            ts, scan, _ = synth.single_phase_workload(n_patterns=args.distinct or SINGLE_PHASE["total"], stream=rank)
            uniq = scan.frames
            libs_ts = [ts]
            total = args.total or SINGLE_PHASE["total"]
            prefilter = SINGLE_PHASE["prefilter"]
            oracle_n = 512
            rk = SINGLE_PHASE["rescore_k"]
        else:
            raise SystemExit(f"unknown workload {wl}")
        if total < uniq.shape[0]:                            # a smaller scan (profiling)
            uniq = np.ascontiguousarray(uniq[:total])
            if wl == "multiphase":
                phase = phase[:total]
        base = to_device_u16(uniq, dev)
        frames_d = base.repeat(total // uniq.shape[0], 1, 1) if total > uniq.shape[0] else base
        del base
        lids = [ctx.load_library(t, N_R, N_THETA) for t in libs_ts]
        pick = np.sort(np.random.default_rng(5).choice(uniq.shape[0], min(uniq.shape[0], oracle_n), replace=False)) \
            if oracle_n else np.zeros(0, dtype=np.int64)
        # sampled positions spread over the whole scan (position p holds distinct frame p mod unique)
        reps = total // uniq.shape[0]
        sample_idx = pick + uniq.shape[0] * np.random.default_rng(6).integers(0, reps, size=pick.shape[0])
        # the FP32 sparse path on the three-phase scan takes tens of seconds per step: it is timed
        # on 4096 of the distinct frames
        subsets = {"fp32": min(4096, total)} if wl == "multiphase" else {}
        rec, res = bench_workload(args, ctx, timer, wl, libs_ts, lids, frames_d, uniq, sample_idx, prefilter,
                                  oracle_n, local, dev, world, want_paths, rank, rk, subsets, headline=not head_done)
        if wl == "multiphase" and rank == 0 and rec.get("paths"):
            rec["phase_share"] = [float((phase == i).mean()) for i in range(3)]
            rec["dropped_templates"] = [t.meta.get("dropped", 0) for t in libs_ts]
        if not head_done:
            head_done = True
            ok = [nm for nm in res if "ms" in res[nm] and (rec["paths"][nm].get("top1_vs_oracle") or {}).get(
                "all", {}).get("wilson95", [0])[0] >= 0.995]
            cand = ok or [nm for nm in res if "ms" in res[nm]]
            head = min(cand, key=lambda nm: res[nm]["ms"])
            r = res[head]
            line.update({"value": world * total / (r["ms"] / 1e3), "ms_per_step": r["ms"], "steps": r["steps"],
                         "warmup": r["warmup"], "dtype": "bf16" if head == "bf16" else "f32",
                         "clocks": r["clocks"], "gpu_launches": int(r["launches_per_step"] * r["steps"]),
                         "roofline": rec["paths"][head]["roofline"], "paths": rec["paths"],
                         "speedup_bf16_vs_fp32": rec.get("speedup_bf16_vs_fp32"),
                         "correlations_per_s": world * rec["correlations_per_step"] / (r["ms"] / 1e3),
                         "config": {"workload": WORKLOAD if wl == "large_map" else wl, "patterns_per_gpu": total,
                                    "distinct_frames": int(uniq.shape[0]), "frame": "256x256 u16",
                                    "templates": rec["libraries"], "spots_per_template": rec["spots_per_template"],
                                    "polar": f"{N_R}x{N_THETA}", "prefilter": prefilter, "top_n": TOP_N,
                                    "path": head, "rescore_k": rk,
                                    "top1_rule": "headline path: Wilson 95 % lower bound of top-1 agreement with "
                                                 "the FP64 oracle >= 99.5 %",
                                    "l2": "distinct frames (2.1 GB) and each step's 34 GB larger than L2; no flush"}})
            if rec.get("oracle_sample") and rank == 0 and world == 1 and not args.no_cpu_baseline:
                o = rec["oracle_sample"]
                line["cpu_baseline"] = {"value": o["patterns_per_s"], "unit": "patterns/s", "cores": o["cores"],
                                        "kind": "oracle",
                                        "sample": f"{o['patterns']} distinct frames of the scan (seeded uniform "
                                                  f"subset), whole path (polar, Q at every shift, top-5), "
                                                  f"{o['seconds']:.1f} s"}
            line["top1_vs_oracle"] = {nm: rec["paths"][nm].get("top1_vs_oracle") for nm in rec["paths"]}
            # ---- end to end through the host-buffer entry point (tm_index_patterns_host): each step
            # copies all of the step's frames from pinned host memory (the distinct frames, once per
            # repeat of the map) and reads every hit back into pinned host memory
            host, host_np = pinned_u16(uniq)
            host_out = torch.empty((len(lids), uniq.shape[0], TOP_N, 5), dtype=torch.int32).pin_memory()
            kw = dict(top_n=TOP_N, prefilter=prefilter,
                      path=tmgb.TM_PATH_BF16_RESCORE if head == "bf16" else tmgb.TM_PATH_FP32_SPARSE,
                      rescore_k=rk)

            def e2e_step():
                for _ in range(reps):
                    ctx.index_host(host, lids, out=host_out, chunk=E2E_CHUNK, **kw)
            e2e_step()
            if world > 1:
                torch.distributed.barrier()
            e2e_steps = max(2, min(args.steps // 2, int(args.path_seconds / max(1e-3, r["ms"] / 1e3 * 1.5))))
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                e2e_step()
            e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
            if world > 1:
                tt = torch.tensor([e2e_ms], device=dev)
                torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
                e2e_ms = float(tt.item())
            line["e2e"] = {"value": world * total / (e2e_ms / 1e3), "unit": "patterns/s", "ms_per_step": e2e_ms,
                           "path": head, "api": "tm_index_patterns_host", "calls_per_step": reps,
                           "chunk_patterns": E2E_CHUNK, "steps": e2e_steps,
                           "h2d_bytes_per_step": int(uniq.nbytes) * reps,
                           "d2h_bytes_per_step": int(host_out.numel() * 4) * reps}
            del host, host_np, host_out
            if wl == "large_map":
                line["pool_frames"] = uniq                      # the serving run's scan-line frames
        line["workloads"][wl] = rec
        for lid in lids:
            ctx.unload_library(lid)
        del frames_d
        torch.cuda.empty_cache()

    pool = line.pop("pool_frames", None)
    if not args.no_serving:
        if pool is None:
            _, scan, _ = synth.large_map_workload(n_unique=16384)
            pool = scan.frames
        fcc = synth.kinematic_library("fcc")
        hcp = synth.kinematic_library("hcp")
        lf, lh = ctx.load_library(fcc, N_R, N_THETA), ctx.load_library(hcp, N_R, N_THETA)
        host, host_np = pinned_u16(pool)
        map_pool = to_device_u16(pool, dev).repeat(LARGE_MAP["total"] // pool.shape[0], 1, 1)
        serving = serve_bench(ctx, [lf, lh], host_np, map_pool, {"path": tmgb.TM_PATH_FP32_SPARSE},
                              seconds=args.serving_seconds)
        line["serving"] = serving
        line["p99_line_ms"] = serving["load_50"].get("line_p99_ms")
        line["serving_workload"] = ("FCC + HCP resident; Poisson scan lines (64-512 patterns, 40/s, host frames) and "
                                    "Poisson maps (64^2-512^2, device frames) at 25/50/80 % of capacity")
        ctx.unload_library(lf)
        ctx.unload_library(lh)
        del host, host_np, map_pool
        torch.cuda.empty_cache()
    if not args.no_two_stage:
        line["two_stage"] = two_stage_bench(ctx, stream, max(2, args.steps // 2))
    if not args.no_preprocess:
        _, scan, _ = synth.single_phase_workload(n_patterns=16384)
        frames_d = to_device_u16(scan.frames, dev)
        line["preprocess"] = preprocess_bench(ctx, stream, frames_d, max(2, args.steps // 2))
        line["template_simulation"] = simulation_bench(ctx, stream)
        del frames_d
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
