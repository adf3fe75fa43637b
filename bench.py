#!/usr/bin/env python
"""Throughput of the template-matching indexing path on one GB300 (or N, sharded).

Workload (one step): the single-phase scan -- 128 x 128 = 16384 diffraction frames of
256 x 256 uint16, kinematic FCC (a = 4.05 A, 200 kV) templates over the cubic
fundamental triangle at 0.5 deg with mirrors, polar grid 128 r x 360 theta, gamma 0.5,
radial pre-filter keeping 50 %, top-5 -- indexed through the library's public call
(tm_index_patterns).  Frames are device-resident when the timed region starts; the
2.1 GB of frames per step is larger than the 129 MB L2, so no flush is needed.

`--impl reference` times the FP64 CPU oracle on the host cores on bounded samples of
the same workload (there is no other reference implementation of this paper).

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
WORKLOAD = ("single-phase scan: 16384 x 256x256 u16 frames, FCC 0.5 deg (+mirrors), polar 128x360, "
            "prefilter 50%, top-5; BF16 tensor-core pre-score + FP32 rescore of the top-256 vs FP32 sparse")
N_R, N_THETA, TOP_N, PREFILTER, RESCORE_K = 128, 360, 5, 0.5, 256
E2E_CHUNK = 2048                  # patterns per chunk of the host-buffer entry point (tm_index_patterns_host)
MATCH_SAMPLE = 512
# tensor-core work per (pattern, scored template): 2 x 180 shifts x (182 + 180) frequency terms
DENSE_FLOPS_PER_PAIR = 2 * 180 * (182 + 180)
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
    ap.add_argument("--patterns", type=int, default=16384)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paths", default="fp32,bf16", help="paths to time (fp32, bf16)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop latency run")
    ap.add_argument("--no-two-stage", action="store_true", help="skip the two-stage (masked) indexing run")
    ap.add_argument("--no-preprocess", action="store_true", help="skip the background-removal and blur timing")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


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


def traffic_from_profiles(kernel_file: str, key: str):
    """DRAM bytes per full-size launch from the committed ncu summary `profiles/traffic.txt`
    (lines: kernel, sha256[:16] of its source file, bytes, note), if it was taken on this
    source; None otherwise."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(p):
            f = line.split()
            if len(f) >= 3 and not f[0].startswith("#") and f[0] == key and f[1] == kernel_sha(kernel_file):
                return float(f[2])
    except OSError:
        pass
    return None


def cpu_baseline(ts, scan, seconds: float) -> dict:
    """The FP64 oracle, as it stands, on a bounded sample of the same workload."""
    from oracle import oracle as O
    lib = O.prepare_library(ts, N_R, N_THETA)
    n0 = 32
    t = time.perf_counter()
    O.index(scan.frames[:n0], lib, prefilter_fraction=PREFILTER, N=TOP_N)
    dt = time.perf_counter() - t
    n = int(min(scan.frames.shape[0], max(n0, n0 * seconds / max(dt, 1e-3))))
    t = time.perf_counter()
    O.index(scan.frames[:n], lib, prefilter_fraction=PREFILTER, N=TOP_N)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "patterns/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"first {n} patterns of the scan, whole path (polar, pre-filter, Q, top-5), {dt:.1f} s"}


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

def serve_bench(ctx, lib_ids, pool: np.ndarray, path_kw: dict, seconds: float = 2.5, seed: int = 2111_07347 + 103):
    """Poisson arrivals against device-resident libraries: 80 % scan lines of 64-512
    patterns (frame rate 1-10 kHz: a line arrives when its last frame is acquired), 20 %
    maps of 64^2 or 128^2 patterns (the frame pool holds 16384 frames, so the 256^2 and
    512^2 maps of the workload are left out).  Capacity is measured first with a saturating
    burst; offered load is then 25 / 50 / 80 % of it.  Latency = completion - arrival."""
    from paper_2111_07347_gb300 import tmgb
    rng = np.random.default_rng(seed)
    n_pool = pool.shape[0]
    srv = tmgb.Server(ctx, slots=4, tile_patterns=512, max_libs=len(lib_ids), max_top_n=TOP_N, priority_slots=1)

    def submit(n, prio):
        a = int(rng.integers(0, n_pool - n + 1))
        return srv.submit(pool[a:a + n], lib_ids, top_n=TOP_N, priority=prio, **path_kw)

    # capacity: a saturating burst of 16 maps of 128^2
    t0 = time.perf_counter()
    ts = [submit(16384, 0) for _ in range(6)]
    for t in ts:
        srv.wait(t, timeout_ms=600000)
    cap = 6 * 16384 / (time.perf_counter() - t0)
    mean_line, mean_map = (64 + 512) / 2, (64 * 64 + 128 * 128) / 2
    mean_req = 0.8 * mean_line + 0.2 * mean_map
    out = {"capacity_patterns_per_s": cap, "slots": 4, "priority_slots": 1, "tile_patterns": 512,
           "maps": "64^2 and 128^2 only (frame pool of 16384)"}
    for load in (0.25, 0.5, 0.8):
        lam = load * cap / mean_req
        t_next = time.perf_counter()
        end = t_next + seconds
        tickets = []
        while t_next < end:
            now = time.perf_counter()
            if now < t_next:
                time.sleep(min(t_next - now, 0.002))
                continue
            if rng.random() < 0.8:
                n = int(rng.integers(64, 513))
                tickets.append(("line", n, submit(n, 1)))
            else:
                side = int(rng.choice([64, 128]))
                tickets.append(("map", side * side, submit(side * side, 0)))
            t_next += rng.exponential(1.0 / lam)
        lat = {"line": [], "map": []}
        pats = 0
        first, last = None, None
        for kind, n, t in tickets:
            res, st = srv.wait(t, timeout_ms=600000)
            lat[kind].append(st["done_ms"] - st["submit_ms"])
            pats += n
            first = st["submit_ms"] if first is None else min(first, st["submit_ms"])
            last = st["done_ms"] if last is None else max(last, st["done_ms"])
        rec = {"requests": len(tickets), "throughput_patterns_per_s": pats / max(1e-9, (last - first) / 1e3)}
        for kind in ("line", "map"):
            if lat[kind]:
                rec[f"{kind}_p50_ms"] = float(np.percentile(lat[kind], 50))
                rec[f"{kind}_p99_ms"] = float(np.percentile(lat[kind], 99))
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
    ts, scan, _ = synth.single_phase_workload(n_patterns=4096)
    lib = O.prepare_library(ts, N_R, N_THETA)
    per_step = 128
    # size the step so that warmup + steps stay within about two minutes
    t = time.perf_counter()
    O.index(scan.frames[:per_step], lib, prefilter_fraction=PREFILTER, N=TOP_N)
    dt = time.perf_counter() - t
    budget = 120.0 / max(1, args.steps + args.warmup)
    per_step = int(max(16, min(4096, per_step * budget / max(dt, 1e-3))))
    off = 0
    for _ in range(args.warmup):
        O.index(scan.frames[off:off + per_step], lib, prefilter_fraction=PREFILTER, N=TOP_N)
    times = []
    for i in range(args.steps):
        a = (i * per_step) % max(1, scan.frames.shape[0] - per_step)
        t = time.perf_counter()
        O.index(scan.frames[a:a + per_step], lib, prefilter_fraction=PREFILTER, N=TOP_N)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "patterns/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "patterns_per_step": per_step, "note": "bounded sample per step"},
            "cpu_baseline": {"value": value, "unit": "patterns/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{per_step} patterns per step, FP64 oracle, whole path"},
            "e2e": {"value": value, "unit": "patterns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

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
    ts, scan, _ = synth.single_phase_workload(n_patterns=args.patterns, stream=rank)
    n = scan.frames.shape[0]
    frames_d = to_device_u16(scan.frames, dev)
    ctx = tmgb.Context(local)
    lid = ctx.load_library(ts, N_R, N_THETA)
    info = ctx.library_info(lid)
    stream = torch.cuda.current_stream()

    kw_fp32 = dict(top_n=TOP_N, prefilter=PREFILTER, path=tmgb.TM_PATH_FP32_SPARSE)
    kw_bf16 = dict(top_n=TOP_N, prefilter=PREFILTER, path=tmgb.TM_PATH_BF16_RESCORE, rescore_k=RESCORE_K)
    outs = {"fp32": torch.empty((1, n, TOP_N, 5), dtype=torch.int32, device=dev),
            "bf16": torch.empty((1, n, TOP_N, 5), dtype=torch.int32, device=dev)}

    def run_path(name, kw, frames):
        ctx.index(frames, lid, out=outs[name], **kw)

    # exact sparse work of one step: survivors x spots x shifts evaluated
    exp = ctx.library_export(lid)
    spots_k = np.diff(exp["offsets"]).astype(np.float64)
    work_k = torch.from_numpy(spots_k * (N_THETA // exp["order"])).to(dev)
    polar, norm, radial = ctx.polar_transform(frames_d, N_R, N_THETA)
    mask, _ = ctx.prefilter(lid, radial, PREFILTER)
    bits = ((mask.view(torch.int32).unsqueeze(-1) >> torch.arange(32, device=dev, dtype=torch.int32)) & 1)
    active = bits.reshape(n, -1)[:, :info["n_templates"]].to(torch.float64)
    macs_step = float((active @ work_k).sum().item())
    survivors_step = float(active.sum().item())
    del polar, norm, radial, mask, bits, active
    torch.cuda.synchronize()

    def timed(name, kw):
        for _ in range(max(3, args.warmup)):
            run_path(name, kw, frames_d)
        torch.cuda.synchronize()
        ctx.check()
        launches = ctx.last_stats["launches"]
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            run_path(name, kw, frames_d)
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = clocks.stop()
        ctx.check()
        # the stage breakdown and the work counters from a second pass of the same steps
        # with stage timing on (events between the stages; not the timing of record)
        ctx.profile_enable(True)
        for _ in range(args.steps):
            run_path(name, kw, frames_d)
        torch.cuda.synchronize()
        prof, counters = ctx.profile_read(counters=True)
        prof = dict(prof, _counters=counters)
        ctx.profile_enable(False)
        ctx.check()
        ms = e0.elapsed_time(e1) / args.steps
        if world > 1:
            t = torch.tensor([ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        return ms, prof, clk, launches

    want = [x.strip() for x in args.paths.split(",") if x.strip()]
    res = {nm: timed(nm, kw) for nm, kw in (("fp32", kw_fp32), ("bf16", kw_bf16)) if nm in want}

    # top-1 agreement with the FP64 oracle on a sample of the scan (both paths)
    match = {}
    if rank == 0:
        from oracle import oracle as O
        pick = np.sort(np.random.default_rng(5).choice(n, min(n, MATCH_SAMPLE), replace=False))
        olib = O.prepare_library(ts, N_R, N_THETA)
        ref = O.index(scan.frames[pick], olib, prefilter_fraction=PREFILTER, N=TOP_N)
        for name in res:
            h = tmgb.hits_to_numpy(outs[name])[0][pick]
            ok = 0
            for i in range(len(pick)):
                k0 = int(h["template_index"][i, 0])
                qt = ref["score"][i, 0]
                t = 1e-5 * max(abs(qt), 1e-30)
                same = (k0 == ref["template"][i, 0] and h["shift"][i, 0] == ref["shift"][i, 0])
                near = k0 >= 0 and np.isfinite(ref["q_best"][i, k0]) and abs(ref["q_best"][i, k0] - qt) <= t
                ok += int(same or near)
            match[name] = ok / len(pick)
    # headline: the faster path that meets the 99.5 % top-1 bar on the sample
    ok_paths = [nm for nm in res if match.get(nm, 0.0) >= 0.995] or list(res)
    head = min(ok_paths, key=lambda nm: res[nm][0])
    ms, prof, clk, launches_per_step = res[head]
    value = world * n / (ms / 1e3)

    # ---- end to end through the host-buffer entry point (tm_index_patterns_host): pinned host
    # frames -> device (chunked, copies overlapping the previous chunk's kernels) -> hits back
    # in pinned host memory; host wall clock around the synchronous call
    host, host_np = pinned_u16(scan.frames)
    host_out = torch.empty((1, n, TOP_N, 5), dtype=torch.int32).pin_memory()
    e2e_steps = max(2, args.steps // 2)
    kw_head = kw_bf16 if head == "bf16" else kw_fp32

    def e2e_step():
        ctx.index_host(host, lid, out=host_out, chunk=E2E_CHUNK, **kw_head)

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = {"value": world * n / (e2e_ms / 1e3), "unit": "patterns/s", "ms_per_step": e2e_ms, "path": head,
           "api": "tm_index_patterns_host", "chunk_patterns": E2E_CHUNK,
           "h2d_bytes_per_step": int(scan.frames.nbytes), "d2h_bytes_per_step": int(host_out.numel() * 4)}

    sm = torch.cuda.get_device_properties(local).multi_processor_count
    f_mhz = clk.get("sm_mhz") or 2070.0

    def roof_sparse(prof_, clk_):
        sp_ms, sp_l = prof_.get("sparse", (0.0, 0))
        per_launch_ms = sp_ms / max(1, sp_l)
        lps = max(1, sp_l // args.steps)
        fm = clk_.get("sm_mhz") or 2070.0
        achieved = 4.0 * macs_step / lps / (per_launch_ms / 1e3) / 1e9
        peak = 128.0 * sm * fm * 1e6 / 1e9
        # the bound pruning skips templates that cannot enter the top-N, so the algorithmic
        # rate may pass the shared-memory peak; the executed multiply-adds (counted by the
        # kernel while profiling, shifts padded to whole blocks) give the data path's own load
        ex_macs = prof_.get("_counters", {}).get("sparse_macs", 0)
        ex_achieved = 4.0 * ex_macs / max(1, sp_l) / (per_launch_ms / 1e3) / 1e9 if ex_macs else None
        return {"bound": "smem", "kernel": "sparse_kernel", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic_from_profiles(
                    os.path.join(ROOT, "paper_2111_07347_gb300", "csrc", "k_sparse.cu"), "sparse_kernel"),
                "algorithmic": "4 B of shared memory per FP32 multiply-add (one polar sample per spot x shift)",
                "peak_basis": f"128 B/clk/SM x {sm} SMs x {fm:.0f} MHz (median SM clock sampled in the run)",
                "launch_ms": per_launch_ms,
                "executed": {"macs_per_launch": ex_macs / max(1, sp_l), "achieved": ex_achieved,
                             "frac": ex_achieved / peak if ex_achieved else None,
                             "skipped_share": 1.0 - ex_macs / max(1, sp_l) * lps / macs_step if ex_macs else None}}

    def roof_dense(prof_):
        d_ms, d_l = prof_.get("dense", (0.0, 0))
        per_launch_ms = d_ms / max(1, d_l)
        lps = max(1, d_l // args.steps)
        flops = DENSE_FLOPS_PER_PAIR * survivors_step / lps
        achieved = flops / (per_launch_ms / 1e3) / 1e12
        peak = MEASURED.get("bf16_tflops_sustained") or 1700.0
        return {"bound": "tensor", "kernel": "dense_kernel", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_from_profiles(
                    os.path.join(ROOT, "paper_2111_07347_gb300", "csrc", "k_dense.cu"), "dense_kernel"),
                "algorithmic": f"{DENSE_FLOPS_PER_PAIR} flop per (pattern, surviving template): inverse DFT over "
                               "182 even + 180 odd frequency terms for 180 shifts",
                "peak_basis": "measured sustained cuBLAS bf16 (MEASURED_PEAKS.json)", "launch_ms": per_launch_ms}

    roofline = roof_dense(prof) if head == "bf16" else roof_sparse(prof, clk)
    stages = {nm: {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                   for k, v in res[nm][1].items() if not k.startswith("_")} for nm in res}
    pol_ms = res[head][1].get("polar", (0.0, 1))[0] / args.steps
    # polar stage against HBM: frames read, the library's rows stored (the norm and the
    # azimuthal sums cover every row but only the used rows are written), sums and norms
    kept_rows = int(np.unique(ctx.library_export(lid)["r"]).size)
    hbm_bytes = n * (256 * 256 * 2 + kept_rows * N_THETA * 4 + N_R * 4 + 4)
    if pol_ms:
        pol_gbs = hbm_bytes / (pol_ms / 1e3) / 1e9
        pol_peak = MEASURED.get("hbm_gbs") or 6800.0
        pol_traffic = traffic_from_profiles(os.path.join(ROOT, "paper_2111_07347_gb300", "csrc", "k_polar.cu"),
                                            "polar_kernel")
        stages[head].setdefault("polar", {}).update(
            {"hbm_gbs": pol_gbs, "roofline": {"bound": "hbm", "kernel": "polar_kernel", "achieved": pol_gbs,
                                              "peak": pol_peak, "unit": "GB/s", "frac": pol_gbs / pol_peak,
                                              "algorithmic_bytes_per_launch": hbm_bytes,
                                              "traffic": pol_traffic * n / 16384 if pol_traffic else None,
                                              "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)"}})

    line = {"metric": METRIC, "value": value, "unit": "patterns/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if head == "bf16" else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "patterns_per_gpu": n, "frame": "256x256 u16",
                       "templates": info["n_templates"], "spots": info["n_spots"], "polar": f"{N_R}x{N_THETA}",
                       "prefilter": PREFILTER, "top_n": TOP_N, "path": head, "rescore_k": RESCORE_K,
                       "l2": "inputs (2.1 GB of frames per step) larger than L2; no flush"},
            "paths": {nm: {"patterns_per_s": world * n / (res[nm][0] / 1e3), "ms_per_step": res[nm][0],
                           "top1_match_vs_oracle": match.get(nm), "clocks_sm_mhz": res[nm][2].get("sm_mhz"),
                           "roofline": roof_dense(res[nm][1]) if nm == "bf16" else roof_sparse(res[nm][1], res[nm][2])}
                      for nm in res},
            "speedup_bf16_vs_fp32": (res["fp32"][0] / res["bf16"][0]) if len(res) == 2 else None,
            "top1_match_sample": MATCH_SAMPLE,
            "correlations_per_s": world * survivors_step * N_THETA / (ms / 1e3),
            "macs_per_step_sparse": macs_step, "survivors_per_step": survivors_step,
            "roofline": roofline, "stages": stages, "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps), "clocks": clk}
    if not args.no_serving:
        hcp = synth.kinematic_library("hcp")
        lid_h = ctx.load_library(hcp, N_R, N_THETA)
        pool = host_np
        serving = serve_bench(ctx, [lid, lid_h], pool, {k: v for k, v in kw_head.items() if k not in ("top_n",)})
        line["serving"] = serving
        line["p99_line_ms"] = serving["load_50"].get("line_p99_ms")
        line["serving_workload"] = "FCC + HCP resident, Poisson arrivals, 80 % lines 64-512 / 20 % maps"
    if not args.no_two_stage:
        line["two_stage"] = two_stage_bench(ctx, stream, max(2, args.steps // 2))
    if not args.no_preprocess:
        line["preprocess"] = preprocess_bench(ctx, stream, frames_d, max(2, args.steps // 2))
        line["template_simulation"] = simulation_bench(ctx, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(ts, scan, args.cpu_seconds)
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
