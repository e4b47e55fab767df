"""Benchmark: path segments/s of the surfel path tracer on one GB300.

One step = one pass of the whole hot path over the workload: surfel
preprocess + LBVH build (sort, hierarchy, collapse) + path-traced render
(primary segments, then per-bounce trace/shade/compact waves, then the
deterministic accumulation).  Default workload: the large final render
(6M-surfel three-room layout, 1920x1080, 1024 spp, 5 bounces, Russian
roulette from bounce 2), one 64-sample slice of the frame per step: step k
renders samples [64 (k mod 16), 64 (k mod 16) + 64) with their own Philox
counters, so 16 consecutive steps render the whole 1024-sample frame.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large|medium|tiny] [--slice-spp S]
  python bench.py --workload serving [--requests R]   (continuous-batching server)
  python bench.py --workload diff|mis                 (differentiable single bounce / emitter sampling)
  python bench.py --workload stage1|bake [--views V]  (Eq. 7 / Eq. 10 optimisation loops)
  python bench.py --impl reference ...    (the FP64 CPU oracle on a bounded sample)

Prints one JSON line (rank 0).  With N > 1 every rank renders its own
samples (independent paths; no collective on the data path).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "path segments/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="large",
                    choices=["tiny", "medium", "diff", "large", "serving", "stage1", "bake", "mis", "lod"])
    ap.add_argument("--views", type=int, default=8, help="stage1/bake: training views")
    ap.add_argument("--requests", type=int, default=16, help="serving: requests in the stream")
    ap.add_argument("--queue-log2", type=int, default=27, help="serving: log2 of the paths one wave holds")
    ap.add_argument("--stream", default="mixed", choices=["mixed", "small"],
                    help="serving: the mixed stream (256x256..1920x1080, 16/64/256 spp) or small requests only "
                         "(256x256, 16 spp)")
    ap.add_argument("--spp", type=int, default=None, help="override samples per pixel (of the frame)")
    ap.add_argument("--slice-spp", type=int, default=None,
                    help="samples per step (default: 64 for the large render, the whole frame otherwise)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--adjoint-retrace", action="store_true",
                    help="diff: the adjoint re-traces every secondary segment instead of reading the forward's cache")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--lod-cell", default="0.05",
                    help="lod: grid cell edge of the surfel groups (m); a comma-separated list sweeps")
    ap.add_argument("--lod-from", default="2",
                    help="lod: first bounce that traces the merged surfels; a comma-separated list sweeps")
    return ap.parse_args()


def rank_seed(rank: int) -> int:
    """Render seed of a rank: every rank draws its own samples (independent
    paths), so N ranks together render N times one rank's work."""
    return 1000003 * rank


def max_over_ranks(t_local: float, world: int, device=None) -> float:
    """The step time of the whole job: the slowest rank's (all-reduce MAX)."""
    if world <= 1:
        return t_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_rank_step: int, steps: int, t_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank_step * steps / t_max


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# the sources that define the bounce kernel (its traffic summary is valid
# while these are unchanged)
# the bounce kernel's sources and the BVH builder's (the tree shapes its traffic)
BOUNCE_SOURCES = ("render.cu", "trace.cuh", "wave.cuh", "common.cuh", "bvh.cu", "bvh_tree.cu")


def source_digest() -> str:
    h = hashlib.sha256()
    for name in BOUNCE_SOURCES:
        with open(os.path.join(ROOT, "paper_2601_23065_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    h.update(os.environ.get("EAGPT_NVCC_FLAGS", "").encode())
    return h.hexdigest()[:16]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def load_traffic(workload: str):
    """DRAM bytes per secondary segment of the bounce kernel from the
    committed ncu summary (dram__bytes_read.sum + dram__bytes_write.sum of one
    captured launch / its segments), if it was taken on the current kernel
    sources; None otherwise."""
    p = os.path.join(ROOT, "profiles", f"k_bounce_{workload}_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_digest") != source_digest():
        return None
    return d.get("dram_bytes_per_segment")


def cpu_sample_spp(wl) -> int:
    """Samples per pixel of the oracle's bounded sample: the frame's first
    samples (same Philox counters as the GPU's)."""
    return min(wl.spp, 2 if wl.scene_fn.__name__ == "large_layout" else 16)


def host_cpu() -> str:
    """The host CPU's model name and the cores this process may run on."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    import platform
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        n = os.cpu_count() or 0
    return f"{model or platform.machine()}, {n} cores available"


def cpu_baseline(wl, scene, seconds: float):
    """The FP64 oracle on a bounded pixel sample of the same workload."""
    import numpy as np

    import oracle as O
    rng = np.random.default_rng(123)
    n_threads = O.default_threads()
    osc = O.OracleScene(scene)
    npix = wl.camera.width * wl.camera.height
    spp = cpu_sample_spp(wl)
    # grow the sample until ~`seconds` of CPU work (at least 2 pixels per thread)
    m = 2 * n_threads
    total_segs, total_t, total_pix = 0, 0.0, 0
    while True:
        pix = rng.choice(npix, m, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        out = O.render(osc, wl.camera, pix, "pt", spp, max_bounces=wl.max_bounces, rr_start=wl.rr_start,
                       seed=0, params=O.Params(fp32_eps=0.0), n_threads=n_threads)
        dt = time.perf_counter() - t0
        total_segs += int(out["segments"].sum())
        total_t += dt
        total_pix += m
        if total_t >= seconds or m >= 4096:
            break
        m = int(min(4096, max(m * 2, m * seconds / max(dt, 1e-3) / 2)))
    return {"value": total_segs / total_t, "unit": METRIC, "cores": n_threads, "kind": "oracle", "cpu": host_cpu(),
            "sample": f"{total_pix} random pixels x {spp} spp (the frame's first samples) of the same workload "
                      f"({total_segs} segments in {total_t:.1f} s, brute force over {scene.n} surfels, FP64)"}


def run_reference(args, rank, world):
    """--impl reference: the oracle as it stands, timed on the host cores.
    Each step renders 2 x threads random pixels (so every thread has work) at
    the oracle sample's samples per pixel."""
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    from paper_2601_23065_gb300 import scenes as S
    if args.workload in ("stage1", "bake"):
        field = 0 if args.workload == "stage1" else 1
        spp = args.spp or (256 if field == 0 else 1)
        cam = fit_views(1)[0]
        c = fit_cpu_baseline(S.diff_room(), cam, field, spp, args.cpu_seconds)
        line = {"metric": "Stage-1 iterations/s" if field == 0 else "light-baking iterations/s",
                "value": c["value"], "unit": c["unit"], "impl": "reference", "n_gpus": world, "steps": 1,
                "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": args.workload}, "cpu_baseline": c,
                "e2e": {"value": c["value"], "unit": c["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    lod = args.workload == "lod"
    wl = S.workload("large" if lod else args.workload)
    if args.spp:
        wl.spp = args.spp
    scene = wl.scene_fn()
    osc = O.OracleScene(scene)
    n_threads = O.default_threads()
    spp = cpu_sample_spp(wl)
    npix = wl.camera.width * wl.camera.height
    rng = np.random.default_rng(321)
    if lod:
        # the oracle's own merge of the same groups (untimed set-up), then its
        # level-of-detail render
        from oracle import lod as OL
        lod_cell = float(str(args.lod_cell).split(",")[0])
        lod_from = int(str(args.lod_from).split(",")[0])
        merged = O.OracleScene(OL.to_scene(OL.merge(scene, LOD_ORIGIN, lod_cell, with_members=False),
                                           S.SurfelScene))

    def one(m):
        pix = rng.choice(npix, m, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        if lod:
            out = O.render_lod(osc, merged, lod_from, wl.camera, pix, spp, max_bounces=wl.max_bounces,
                               rr_start=wl.rr_start, seed=0, params=O.Params(fp32_eps=0.0), n_threads=n_threads)
        else:
            out = O.render(osc, wl.camera, pix, "pt", spp, max_bounces=wl.max_bounces, rr_start=wl.rr_start,
                           seed=0, params=O.Params(fp32_eps=0.0), n_threads=n_threads)
        return int(out["segments"].sum()), time.perf_counter() - t0

    for _ in range(max(0, args.warmup)):
        one(n_threads)
    segs, secs = 0, 0.0
    for _ in range(args.steps):
        a, b = one(2 * n_threads)
        segs += a
        secs += b
    v = segs / secs
    sample = (f"{args.steps} steps x {2 * n_threads} random pixels x {spp} spp (the frame's first samples) of the "
              f"same workload ({segs} segments in {secs:.1f} s, brute force over {scene.n} surfels, FP64)")
    line = {"metric": METRIC, "value": v, "unit": METRIC, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": ({"workload": wl.name, "scale_factor": wl.scale_factor} if not lod else
                       {"workload": f"large final render with level of detail: {wl.name}; bounce segments k >= "
                                    f"{lod_from} trace the surfels merged over {lod_cell} m cells",
                        "scale_factor": wl.scale_factor, "lod_cell_m": lod_cell, "lod_from": lod_from}),
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": n_threads, "kind": "oracle", "cpu": host_cpu(),
                             "sample": sample},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Serving room (3M surfels, scales x0.436 of the medium room's law): a
    seeded request stream (renders of 256x256..1920x1080, 16/64/256 spp, 1-5
    bounces, 10 % edits) served (a) by plain sequential launches, (b) by the
    continuous-batching server with every request submitted at once (closed
    loop: throughput and latency under a full queue), (c) by the server at
    Poisson arrival rates of 0.8x and 1.2x the plain capacity.  Reports
    throughput (pixel samples/s), p50/p99 latency, and whether every served
    image equals its plain render bit for bit."""
    import numpy as np
    import torch

    from paper_2601_23065_gb300 import api, build
    from paper_2601_23065_gb300 import scenes as S

    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    host = S.serving_room()
    wl = S.workload("serving")
    if args.stream == "small":
        reqs = S.serving_requests(host, args.requests, seed=13, spp_choices=[16], res_choices=[(256, 256)])
    else:
        reqs = S.serving_requests(host, args.requests, seed=13)
    n_render = sum(1 for r in reqs if r["type"] == "render")
    samples = sum(r["camera"].width * r["camera"].height * r["spp"] for r in reqs if r["type"] == "render")
    queue_paths = 1 << args.queue_log2

    def resolve_edit(ds, r):
        idx = torch.from_numpy(r["idx"]).to(dev) if "idx" in r else api.select(ds, "sphere", r["sphere"])
        per = torch.from_numpy(r["per_index"]).to(dev) if "per_index" in r else None
        return idx, per

    # (a) plain launches, one request after the other
    ds = api.DeviceScene.from_host(host, device=dev)
    bvh = api.BVH(ds)
    rend = api.Renderer(device=dev)
    for _ in range(max(1, args.warmup)):
        rend.path_traced(ds, bvh, S.horizontal_camera(256, 256), 4, 2)
    # the edits' selection and the image comparison also run once untimed
    # (their kernels load on first use)
    api.select(ds, "sphere", [0.0, 0.0, 0.0, 0.1])
    torch.equal(torch.zeros(4, device=dev), torch.zeros(4, device=dev))
    torch.cuda.synchronize(dev)
    plain_out, plain_lat, t0 = [], [], time.perf_counter()
    for r in reqs:
        if r["type"] == "render":
            o = rend.path_traced(ds, bvh, r["camera"], r["spp"], r["max_bounces"], rr_start=2, seed=r["seed"])
            plain_out.append(o["rgb"].clone())
            torch.cuda.synchronize(dev)
            plain_lat.append(time.perf_counter() - t0)  # completion time when all arrive at t = 0
        else:
            idx, per = resolve_edit(ds, r)
            api.apply_edit(ds, bvh, r["op"], idx, value=r.get("value", ()), per_index=per)
    torch.cuda.synchronize(dev)
    t_plain = time.perf_counter() - t0
    mu = n_render / t_plain
    del ds, bvh, rend
    torch.cuda.empty_cache()

    def serve(arrivals):
        """Submits the stream at the given arrival offsets (None: all at
        once) and returns its throughput, latencies and bitwise check."""
        ds = api.DeviceScene.from_host(host, device=dev)
        bvh = api.BVH(ds)
        srv = api.Server(ds, bvh, queue_paths=queue_paths, max_active=16)
        # untimed warm-up, as the plain launches had: one small render through
        # the server (its kernels load on first use)
        for _ in range(max(1, args.warmup)):
            wid, _out = srv.submit_render(S.horizontal_camera(256, 256), 4, 2)
            srv.wait(wid, 600.0)
        torch.cuda.synchronize(dev)
        st0 = srv.stats()
        ids = []
        start = time.perf_counter()
        for n, r in enumerate(reqs):
            if arrivals is not None:
                delay = start + arrivals[n] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            if r["type"] == "render":
                ids.append(("render", srv.submit_render(r["camera"], r["spp"], r["max_bounces"], rr_start=2,
                                                        seed=r["seed"])))
            else:
                idx, per = resolve_edit(ds, r) if "idx" in r else (None, None)
                if idx is None:
                    # the selection runs on the scene the edit will apply to:
                    # wait for the edits before it, then select on the server's
                    # current scene
                    for kind, x in ids:
                        if kind == "edit":
                            srv.wait(x, 600.0)
                    cur = api.capi.Scene()
                    api.capi.check(api.capi.lib().eagpt_server_scene(srv.h, ctypes.byref(cur), None))
                    view = api.DeviceScene.__new__(api.DeviceScene)
                    view.n, view.version = ds.n, cur.version
                    view.t = {"pos": torch.empty(0, device=dev)}
                    view.c = lambda cur=cur: cur
                    idx = api.select(view, "sphere", r["sphere"])
                ids.append(("edit", srv.submit_edit(r["op"], idx, value=r.get("value", ()), per_index=per)))
        lat, equal, t_first, t_last = [], True, None, None
        outs = []
        for kind, x in ids:
            if kind == "render":
                rid, out = x
                info = srv.wait(rid, 1800.0)
                assert info["state"] == "done", info
                lat.append(info["t_done"] - info["t_submit"])
                t_first = info["t_submit"] if t_first is None else min(t_first, info["t_submit"])
                t_last = info["t_done"] if t_last is None else max(t_last, info["t_done"])
                outs.append(out)
            else:
                srv.wait(x, 1800.0)
        # the images are compared once the whole stream is done: work on the
        # caller's thread (a first use of a library kernel loads its module)
        # would otherwise stall the server's launches inside the measured span
        torch.cuda.synchronize(dev)
        for out, ref in zip(outs, plain_out):
            equal &= bool(torch.equal(out, ref))
        st = srv.stats()
        span = max(1e-9, t_last - t_first)
        res = {"throughput": samples / span, "seconds": span, "p50_s": float(np.percentile(lat, 50)),
               "p99_s": float(np.percentile(lat, 99)), "mean_s": float(np.mean(lat)), "equal_to_plain": equal,
               "segments_per_s_busy": (st["segments"] - st0["segments"]) / max(st["busy_s"] - st0["busy_s"], 1e-9),
               "waves": st["waves"] - st0["waves"],
               "edits": st["edits"], "rebuilds": st["rebuilds"]}
        srv.close()
        del ds, bvh
        torch.cuda.empty_cache()
        return res

    closed = serve(None)
    results = {}
    for load in (0.8, 1.2):
        rng = np.random.default_rng(int(load * 100))
        results[f"load_{load}"] = serve(np.cumsum(rng.exponential(1.0 / (load * mu), len(reqs))))
    plain = {"throughput": samples / t_plain, "capacity_req_per_s": mu, "seconds": t_plain,
             "p50_s": float(np.percentile(plain_lat, 50)), "p99_s": float(np.percentile(plain_lat, 99)),
             "mean_s": float(np.mean(plain_lat))}
    line = {"metric": "pixel samples/s (serving, all requests submitted at once)", "value": closed["throughput"],
            "unit": "pixel samples/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving room 3M surfels, seeded request stream", "scale_factor": wl.scale_factor,
                       "stream": args.stream, "requests": len(reqs), "renders": n_render, "pixel_samples": samples,
                       "queue_paths": queue_paths, "max_active": 16},
            "plain": plain, "closed_loop": closed, "speedup_vs_plain": closed["throughput"] / plain["throughput"],
            "poisson": results}
    print(json.dumps(line), flush=True)


# bytes counted per BVH node visit in the byte model (a binary node's two child
# boxes and links; one BVH4 node of 128 B replaces about two of them)
NODE_BYTES = 64


def fit_views(n_views, width=540, height=360):
    """Training views inside the 1M-surfel room: cameras on a ring of radius
    1 m around the centre, looking outward and slightly down (the paper
    optimises at 540x360)."""
    import math

    from paper_2601_23065_gb300 import scenes as S
    cams = []
    for k in range(n_views):
        a = 2 * math.pi * k / n_views
        c = (math.cos(a), math.sin(a), 0.2)
        f = (math.cos(a + 0.4), math.sin(a + 0.4), -0.15)
        cams.append(S.look_at_camera(width, height, 75.0, c, f, (0.0, 0.0, 1.0)))
    return cams


def fit_cpu_baseline(scene, cam, field, spp, seconds):
    """The oracle's step (render + PQ-L1 + gradient of the field) on a
    bounded random-pixel sample of one view, scaled to iterations/s of the
    full view."""
    import numpy as np

    import oracle as O
    from oracle import optim as OP
    rng = np.random.default_rng(321)
    osc = O.OracleScene(scene)
    npix = cam.width * cam.height
    n_threads = O.default_threads()
    m, total_t, total_pix = 2, 0.0, 0
    while True:
        pix = rng.choice(npix, m, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        if field == 0:
            img = O.render(osc, cam, pix, "single", spp, seed=1, params=O.Params(fp32_eps=0.0),
                           n_threads=n_threads)["rgb"]
            _, dL = OP.pq_l1(img, img * 0.9, 100.0)
            O.single_bounce_grad(osc, cam, pix, dL.reshape(-1, 3), spp, seed=1, n_threads=n_threads)
        else:
            img = O.primary(osc, cam, pix, mode=0, n_threads=n_threads)[0][:, 4:7]
            _, dL = OP.pq_l1(img, img * 0.9, 100.0)
            O.radiance_grad(osc, cam, pix, dL.reshape(-1, 3), n_threads=n_threads)
        dt = time.perf_counter() - t0
        total_t += dt
        total_pix += m
        if total_t >= seconds or m >= 4096:
            break
        m = int(min(4096, max(m * 2, m * seconds / max(dt, 1e-3) / 2)))
    per_iter = total_t / total_pix * npix
    what = f"single bounce {spp} spp + full FP64 adjoint" if field == 0 else "0-bounce + FP64 adjoint"
    return {"value": 1.0 / per_iter, "unit": "iterations/s", "cores": n_threads, "kind": "oracle", "cpu": host_cpu(),
            "sample": f"{total_pix} random pixels of one {cam.width}x{cam.height} view ({what}, brute force "
                      f"over {scene.n} surfels) in {total_t:.1f} s, scaled to the full view"}


def run_fit(args):
    """Stage 1 (Eq. 7, albedo through the single-bounce render) or light
    baking (Eq. 10, radiance through the 0-bounce render) on the 1M-surfel
    room with 540x360 training views.  One step = one optimisation
    iteration (render, PQ-L1 loss and gradient, shading adjoint, Adam,
    BVH shade-record update) through the native loop."""
    import numpy as np
    import torch

    from paper_2601_23065_gb300 import api, build, capi
    from paper_2601_23065_gb300 import scenes as S

    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    L = capi.lib()
    field = "albedo" if args.workload == "stage1" else "radiance"
    spp = args.spp or (256 if field == "albedo" else 1)
    host = S.diff_room()
    cams = fit_views(args.views)
    ds = api.DeviceScene.from_host(host, device=dev)
    bvh = api.BVH(ds)
    r = api.Renderer(device=dev)
    # targets: the room's own images (Stage 1: single bounce with its albedo;
    # baking: path-traced, 4 bounces), then the field is reset to a start value
    if field == "albedo":
        targets = [api.single_bounce_incident(ds, bvh, c, 64, seed=9, renderer=r)["rgb"].clone() for c in cams]
        ds.t["albedo"].fill_(0.5)
    else:
        targets = [r.path_traced(ds, bvh, c, 64, 4, rr_start=2, seed=9)["rgb"].clone() for c in cams]
    bvh = api.BVH(ds)
    fit = api.ShadingFit(ds, bvh, cams, targets, field, spp=spp, seed=1)
    # counters of one step's segments (same cameras, same samples)
    st = r.path_traced(ds, bvh, cams[0], spp, 1, rr_start=1 << 20, seed=2, want_stats=True)["stats"].cpu().numpy()
    prim, sec = int(st[0]), int(st[1])
    p_blend, p_nodes, p_tests = int(st[8]), int(st[9]), int(st[10])
    s_blend, s_nodes, s_tests = int(st[3]), int(st[4]), int(st[5])
    warm_losses = fit.run(max(3, args.warmup)).cpu().tolist()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = L.eagpt_launch_count()
    capi.check(L.eagpt_profile_begin())
    # the steps run as one native loop (how an optimisation runs); the scene
    # and its BVH (about 0.5 GB) exceed the L2, so no flush is needed between
    # steps
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    lo = fit.run(args.steps)
    b.record()
    b.synchronize()
    losses = lo.cpu().tolist()
    prof = capi.profile_end()
    launches = L.eagpt_launch_count() - launches0
    clk = clocks.stop()
    api.sync_status()
    ms = a.elapsed_time(b) / args.steps
    value = 1e3 / ms
    peak, peak_kind = load_peaks()
    total_kernel_ms = sum(v[1] for v in prof.values())
    kname = max(prof.items(), key=lambda kv: kv[1][1])[0]
    kl, kms = prof[kname]
    if kname == "k_bounce":
        unit_bytes = 96 * sec + NODE_BYTES * s_nodes + 64 * s_tests + 32 * s_blend
    elif kname in ("k_radiance", "k_primary", "k_shade_adjoint"):
        # one primary segment per pixel: 12 B out (image or gradient read) +
        # node, test and blended-record bytes; the adjoint adds 12 B of
        # atomics per blended hit
        extra = 12 * p_blend if kname == "k_shade_adjoint" else 0
        unit_bytes = 12 * prim + NODE_BYTES * p_nodes + 64 * p_tests + 32 * p_blend + extra
    else:
        unit_bytes = None
    per_launch_ms = kms / max(1, kl)
    launches_per_step = kl / max(1, args.steps)
    achieved = unit_bytes / launches_per_step / (per_launch_ms * 1e-3) / 1e9 if unit_bytes else None
    npix = cams[0].width * cams[0].height
    segs = prim + (sec if field == "albedo" else prim)
    line = {"metric": "Stage-1 iterations/s" if field == "albedo" else "light-baking iterations/s",
            "value": value, "unit": "iterations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": ("Stage 1 (Eq. 7): albedo, single bounce" if field == "albedo" else
                                    "light baking (Eq. 10): radiance, 0-bounce") +
                       f", 1M-surfel room, {len(cams)} views {cams[0].width}x{cams[0].height}, spp {spp}",
                       "surfels": host.n, "views": len(cams), "pixels_per_step": npix, "spp": spp,
                       "segments_per_step": segs, "segments_per_s": segs * value,
                       "loss_first_last": [losses[0], losses[-1]],
                       "loss_at_start": warm_losses[0],
                       "l2": "steps in one native loop; scene and BVH (~0.5 GB) exceed the L2"},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None, "traffic": None,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "share_of_kernel_time": kms / total_kernel_ms if total_kernel_ms else None},
            "cpu_baseline": fit_cpu_baseline(host, cams[0], 0 if field == "albedo" else 1, spp,
                                             args.cpu_seconds) if not args.no_cpu_baseline else None,
            "gpu_launches": int(launches), "clocks": clk,
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items())}}
    print(json.dumps(line), flush=True)


def run_diff(args):
    """The differentiable single-bounce workload (1M surfels, 800x800,
    16 spp): one step = LBVH build + single-bounce forward (Eq. 6) + the
    hand-written adjoint for L = sum w . image with w ~ U[-1, 1] (seed 11),
    gradients for every surfel parameter.  The forward keeps each sample's
    secondary R and T for the adjoint (``--adjoint-retrace``: the adjoint
    re-traces them).  value = the render's segments (primary and secondary),
    each differentiated, per second of the whole step; the adjoint's own
    traversals are reported in the config."""
    import numpy as np
    import torch

    from paper_2601_23065_gb300 import api, build, capi
    from paper_2601_23065_gb300 import scenes as S

    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    L = capi.lib()
    wl = S.workload("diff")
    spp = args.spp or wl.spp
    host = wl.scene_fn()
    cam = wl.camera
    ds = api.DeviceScene.from_host(host, device=dev)
    r = api.Renderer(device=dev)
    w = torch.from_numpy(np.random.default_rng(11).uniform(-1, 1, (cam.height, cam.width, 3)).astype(np.float32)).to(dev)
    grads = {k: torch.zeros_like(ds.t[k]) for k in api.GRAD_FIELDS}
    need = L.eagpt_render_backward_workspace_bytes(ctypes.byref(api.camera(cam)), spp)
    bws = torch.empty(need, dtype=torch.uint8, device=dev)

    cached = not args.adjoint_retrace

    def step(seed):
        bvh = api.BVH(ds)
        fwd = r.single_bounce(ds, bvh, cam, spp, seed=seed, want_cache=cached)
        for g in grads.values():
            g.zero_()
        api.single_bounce_backward(ds, bvh, cam, spp, seed, w, grads=grads, workspace=bws, cache=fwd.get("cache"))
        return fwd["rgb"]

    # the same rays as a path-traced render with one bounce and no roulette
    st = r.path_traced(ds, api.BVH(ds), cam, spp, 1, rr_start=1 << 20, seed=3, want_stats=True)["stats"].cpu().numpy()
    prim, sec = int(st[0]), int(st[1])
    s_blend, s_nodes, s_tests = int(st[3]), int(st[4]), int(st[5])
    hit_prim = int(st[2] // max(1, spp))
    fwd_segs = prim + sec
    # adjoint traversals: primary records once, every hit primary twice,
    # every secondary segment once (twice when it re-traces the values)
    bwd_segs = prim + (1 if cached else 2) * sec + 2 * hit_prim
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        step(3)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = L.eagpt_launch_count()
    capi.check(L.eagpt_profile_begin())
    times = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        step(3)
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    prof = capi.profile_end()
    launches = L.eagpt_launch_count() - launches0
    clk = clocks.stop()
    api.sync_status()
    ms = sum(times) / len(times)
    value = fwd_segs / (ms * 1e-3)
    total_kernel_ms = sum(v[1] for v in prof.values())
    kname = max(prof.items(), key=lambda kv: kv[1][1])[0]
    peak, peak_kind = load_peaks()
    achieved = None
    if kname == "k_bwd_secondary":
        # per secondary segment: the primary record it is rebuilt from (48 B),
        # the cached R and T (16 B) and one traversal, or two traversals
        # (values, then the adjoint), and 16 gradient atomics (64 B) per
        # blended hit
        trav = NODE_BYTES * s_nodes + 64 * s_tests + 32 * s_blend
        step_bytes = 48 * sec + (16 * sec + trav if cached else 2 * trav) + 64 * s_blend
        achieved = step_bytes / (prof[kname][1] / args.steps * 1e-3) / 1e9
    line = {"metric": METRIC + " (single-bounce forward + adjoint)", "value": value, "unit": METRIC, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "surfels": host.n, "width": cam.width, "height": cam.height, "spp": spp,
                       "forward_segments": fwd_segs, "adjoint_traced_segments": bwd_segs,
                       "traced_segments_per_s": (fwd_segs + bwd_segs) / (ms * 1e-3),
                       "adjoint": "re-traces the secondary values" if not cached else "reads the forward's per-sample cache",
                       "step": "LBVH build + single-bounce forward + adjoint (all parameters)",
                       "l2": "flushed between steps (512 MB write)"},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None, "traffic": None,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "share_of_kernel_time": prof[kname][1] / total_kernel_ms if total_kernel_ms else None},
            "cpu_baseline": None, "gpu_launches": int(launches), "clocks": clk,
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items())}}
    print(json.dumps(line), flush=True)


def run_mis(args):
    """Emitter sampling with MIS against plain path tracing on the medium room
    (200k surfels, 512x512, 4 bounces, RR from 2; 16 spp unless --spp): path
    segments/s of each (emitter samples are segments too), the per-pixel
    variance of each estimated from two renders with different seeds
    (E[(a - b)^2] / 2, averaged over pixels and channels), and the
    efficiency ratio (variance x time of plain) / (variance x time of MIS)."""
    import torch

    from paper_2601_23065_gb300 import api, build, capi
    from paper_2601_23065_gb300 import scenes as S

    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    L = capi.lib()
    wl = S.workload("medium")
    spp = args.spp or 16
    host = wl.scene_fn()
    cam = wl.camera
    ds = api.DeviceScene.from_host(host, device=dev)
    bvh = api.BVH(ds)
    r = api.Renderer(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    for name, prm in (("plain", api.params()), ("mis", api.params(flags=capi.FLAG_EMITTER_SAMPLING))):
        st = r.path_traced(ds, bvh, cam, spp, wl.max_bounces, rr_start=wl.rr_start, seed=1, prm=prm,
                           want_stats=True)["stats"].cpu().numpy()
        segs = int(st[0]) + int(st[1])
        for _ in range(max(3, args.warmup)):
            r.path_traced(ds, bvh, cam, spp, wl.max_bounces, rr_start=wl.rr_start, seed=1, prm=prm)
        torch.cuda.synchronize(dev)
        times, imgs = [], []
        for k in range(max(2, args.steps)):
            flush.fill_(float(k))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            out = r.path_traced(ds, bvh, cam, spp, wl.max_bounces, rr_start=wl.rr_start, seed=1 + 7919 * k, prm=prm)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
            if k < 2:
                imgs.append(out["rgb"].double().clone())
        api.sync_status()
        ms = sum(times) / len(times)
        var = float(((imgs[0] - imgs[1]) ** 2).mean() / 2.0)
        res[name] = {"ms_per_render": ms, "segments_per_render": segs, "segments_per_s": segs / (ms * 1e-3),
                     "variance": var, "mean": float(imgs[0].mean())}
    eff = (res["plain"]["variance"] * res["plain"]["ms_per_render"]) / max(
        1e-300, res["mis"]["variance"] * res["mis"]["ms_per_render"])
    line = {"metric": "path segments/s (emitter sampling + MIS)", "value": res["mis"]["segments_per_s"],
            "unit": "path segments/s", "n_gpus": 1, "steps": max(2, args.steps), "warmup": max(3, args.warmup),
            "ms_per_step": res["mis"]["ms_per_render"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"medium room 200k surfels 512x512 {spp}spp 4 bounces RR>=2, emitter sampling + MIS",
                       "l2": "flushed between renders (512 MB write)"},
            "plain": res["plain"], "mis": res["mis"], "efficiency_vs_plain": eff}
    print(json.dumps(line), flush=True)


def frame_slices(frame_spp: int, slice_spp: int):
    """(first sample, samples) of each slice of a frame of frame_spp samples."""
    out, first = [], 0
    while first < frame_spp:
        n = min(slice_spp, frame_spp - first)
        out.append((first, n))
        first += n
    return out


# Bytes the method moves per secondary segment (the byte model of the
# roofline): the ray read (48 B) and the ray or slot write (48 B), 64 B per BVH
# node visit, 64 B per surfel record tested and 32 B per shade record blended.
def alg_bytes_per_segment(nodes, tests, blended):
    return 48.0 + 48.0 + 64.0 * nodes + 64.0 * tests + 32.0 * blended


# The part no BVH can avoid: the ray in and out and, per blended hit, its
# trace and shade records (64 + 32 B).
def floor_bytes_per_segment(blended):
    return 96.0 + 96.0 * blended


def run_render(args, rank, world, local):
    """The path-traced render workloads (large | medium | tiny)."""
    import numpy as np
    import torch

    from paper_2601_23065_gb300 import api, build
    from paper_2601_23065_gb300 import capi
    from paper_2601_23065_gb300 import scenes as S

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    wl = S.workload(args.workload)
    frame_spp = args.spp or wl.spp
    slice_spp = min(args.slice_spp or (64 if args.workload == "large" else frame_spp), frame_spp)
    slices = frame_slices(frame_spp, slice_spp)
    host_scene = wl.scene_fn()
    cam = wl.camera
    seed_base = rank_seed(rank)  # each rank renders its own samples
    ds = api.DeviceScene.from_host(host_scene, device=dev)
    r = api.Renderer(device=dev)
    stream = torch.cuda.current_stream(dev)
    L = capi.lib()
    img = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device=dev)

    def step(k):
        first, n = slices[k % len(slices)]
        bvh = api.BVH(ds, stream=stream)
        r.path_traced(ds, bvh, cam, n, wl.max_bounces, rr_start=wl.rr_start, seed=seed_base, stream=stream,
                      first_sample=first, out=img)
        return bvh

    # untimed: the counting variant on the first slice gives the per-segment
    # work (BVH nodes, surfel tests, blended hits) of the byte model
    first0, n0 = slices[0]
    cnt = r.path_traced(ds, api.BVH(ds, stream=stream), cam, n0, wl.max_bounces, rr_start=wl.rr_start,
                        seed=seed_base, first_sample=first0, want_stats=True)["stats"].cpu().numpy()
    api.sync_status()
    c_sec = max(1, int(cnt[1]))
    per_seg = {"nodes": int(cnt[4]) / c_sec, "tests": int(cnt[5]) / c_sec, "blended": int(cnt[3]) / c_sec,
               "rounds": int(cnt[6]) / c_sec}
    prim_per_pixel_nodes = int(cnt[9]) / max(1, int(cnt[0]))

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(dev)

    # timed region
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = L.eagpt_launch_count()
    capi.check(L.eagpt_profile_begin())
    barrier()
    torch.cuda.synchronize(dev)
    times, prim_segs, sec_segs = [], 0, 0
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between steps (outside the step's events)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(k)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
        p, q = r.segments(stream)  # this step's exact segment counts (read after its events)
        prim_segs += p
        sec_segs += q
    torch.cuda.synchronize(dev)
    barrier()
    prof = capi.profile_end()
    launches = L.eagpt_launch_count() - launches0
    clk = clocks.stop()
    api.sync_status()

    ms = sum(times) / len(times)
    t_max = max_over_ranks(sum(times) / 1e3, world, dev)
    segs_local = prim_segs + sec_segs
    segs_job = segs_local
    if world > 1:
        t = torch.tensor([float(segs_local)], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t)
        segs_job = float(t.item())
    value = segs_job / t_max
    npix = cam.width * cam.height
    paths_local = npix * sum(slices[k % len(slices)][1] for k in range(args.steps))

    # roofline of the dominant kernel (the fused trace/shade/compact bounce)
    bounce = prof.get("k_bounce", (0, 0.0))
    total_kernel_ms = sum(v[1] for v in prof.values())
    peak, peak_kind = load_peaks()
    bounce_launches = max(1, bounce[0])
    ms_per_launch = bounce[1] / bounce_launches
    segs_per_launch = sec_segs / bounce_launches
    model_b = alg_bytes_per_segment(per_seg["nodes"], per_seg["tests"], per_seg["blended"])
    floor_b = floor_bytes_per_segment(per_seg["blended"])

    def gbs(bytes_per_seg):
        return bytes_per_seg * segs_per_launch / (ms_per_launch * 1e-3) / 1e9 if ms_per_launch else None

    achieved = gbs(model_b)
    dram_b = load_traffic(args.workload)
    traffic = dram_b * segs_per_launch if dram_b else None
    l2_resident = args.workload in ("medium", "tiny")
    roofline = {"bound": "l2" if l2_resident else "hbm", "kernel": "k_bounce", "achieved": achieved,
                "peak": None if l2_resident else peak, "unit": "GB/s",
                "frac": None if (l2_resident or not achieved) else achieved / peak,
                "traffic": traffic,
                "model": "algorithmic bytes per secondary segment = 48 (ray in) + 48 (ray or slot out) + 64 per BVH "
                         "node visit + 64 per surfel test + 32 per blended hit; per-segment counts from the counting "
                         "variant on the first slice",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                "bytes_per_launch": model_b * segs_per_launch, "ms_per_launch": ms_per_launch,
                "launches": bounce[0], "share_of_kernel_time": bounce[1] / total_kernel_ms if total_kernel_ms else None,
                "floor": {"what": "96 + 96 per blended hit (ray in/out, trace + shade record of every blended hit)",
                          "bytes_per_segment": floor_b, "achieved": gbs(floor_b),
                          "frac": (gbs(floor_b) / peak) if (ms_per_launch and not l2_resident) else None},
                "dram": ({"bytes_per_segment": dram_b, "achieved": gbs(dram_b), "frac": gbs(dram_b) / peak,
                          "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of a captured bounce launch, "
                                    "per segment (profiles/)"} if dram_b else None),
                "per_secondary_segment": per_seg, "bytes_per_segment": model_b,
                "primary_nodes_per_pixel": prim_per_pixel_nodes, "max_stack": int(cnt[7])}
    if l2_resident:
        roofline["note"] = ("scene and BVH fit in the 129 MB L2: L2/latency-bound, achieved is the byte model's "
                            "bandwidth equivalent, not an HBM fraction")

    # end to end through the public API with host buffers: the scene copied
    # from pinned host memory, BVH build, render, the image copied back
    pinned = {k: torch.from_numpy(getattr(host_scene, k)).pin_memory() for k in api.FIELDS}
    dev_t = {k: torch.empty_like(v, device=dev) for k, v in pinned.items()}
    out_host = torch.empty((cam.height, cam.width, 3), dtype=torch.float32).pin_memory()
    h2d = sum(v.numel() * 4 for v in pinned.values())
    d2h = out_host.numel() * 4
    e2e_t, e2e_segs = 0.0, 0
    for k in range(min(args.steps, 4)):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for kk in api.FIELDS:
            dev_t[kk].copy_(pinned[kk], non_blocking=True)
        dsk = api.DeviceScene(dev_t)
        bvh = api.BVH(dsk, stream=stream)
        first, n = slices[k % len(slices)]
        r.path_traced(dsk, bvh, cam, n, wl.max_bounces, rr_start=wl.rr_start, seed=seed_base, stream=stream,
                      first_sample=first, out=img)
        out_host.copy_(img, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_t += time.perf_counter() - t0
        p, q = r.segments(stream)
        e2e_segs += p + q
    e2e_val = world * e2e_segs / e2e_t

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, host_scene, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl.name, "surfels": host_scene.n, "scale_factor": wl.scale_factor,
                           "width": cam.width, "height": cam.height, "frame_spp": frame_spp,
                           "spp_per_step": slice_spp,
                           "step": (f"LBVH build + path-traced render of samples [{slice_spp}*(k mod {len(slices)}), "
                                    f"+{slice_spp}) of the {frame_spp}-sample frame (own Philox counters; "
                                    f"{len(slices)} steps cover the frame)"),
                           "max_bounces": wl.max_bounces, "rr_start": wl.rr_start,
                           "segments": prim_segs + sec_segs, "primary_segments": prim_segs,
                           "secondary_segments": sec_segs, "paths": paths_local,
                           "rays_per_s": world * paths_local / t_max,
                           "l2": "flushed between steps (512 MB write)",
                           "parallelism": f"replicas x{world} (independent samples per rank)"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "steps": min(args.steps, 4)},
                "gpu_launches": int(launches), "clocks": clk,
                "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items())}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# grid corner that puts the walls of the large layout in mid-cell (5 and 2.5 cm cells)
LOD_ORIGIN = (-7.6125, -2.1125, -1.6125)


def run_lod(args, local=0):
    """Level of detail on the large final render: plain steps and merged
    steps (the bounce segments from lod_from on trace the merged surfels)
    timed in the same process on the same 64-sample slices; each merged step
    also rebuilds the merged surfels and their BVH.  --lod-cell and
    --lod-from take comma-separated lists: the first pair is the line's
    value, every pair is reported under "sweep".  Accuracy is read after the
    timed spans on the first slice: the image mean, and the RMS difference of
    32x32-pixel block means (relative to the image mean) against the plain
    render, beside the same figure for two plain renders of different seeds
    (the Monte Carlo noise floor of that comparison)."""
    import numpy as np
    import torch

    from paper_2601_23065_gb300 import api, build
    from paper_2601_23065_gb300 import capi
    from paper_2601_23065_gb300 import scenes as S

    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = S.workload("large")
    frame_spp = args.spp or wl.spp
    slice_spp = min(args.slice_spp or 64, frame_spp)
    slices = frame_slices(frame_spp, slice_spp)
    host_scene = wl.scene_fn()
    cam = wl.camera
    ds = api.DeviceScene.from_host(host_scene, device=dev)
    r = api.Renderer(device=dev)
    stream = torch.cuda.current_stream(dev)
    L = capi.lib()
    img = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    cells = [float(v) for v in str(args.lod_cell).split(",")]
    froms = [int(v) for v in str(args.lod_from).split(",")]
    pairs = [(h, f) for h in cells for f in froms]

    def plain_step(k):
        first, n = slices[k % len(slices)]
        bvh = api.BVH(ds, stream=stream)
        r.path_traced(ds, bvh, cam, n, wl.max_bounces, rr_start=wl.rr_start, seed=0, stream=stream,
                      first_sample=first, out=img)

    def lod_step(h, f):
        def step(k):
            first, n = slices[k % len(slices)]
            bvh = api.BVH(ds, stream=stream)
            lod = api.LevelOfDetail(ds, LOD_ORIGIN, h, stream=stream)
            r.path_traced_lod(ds, bvh, lod, f, cam, n, wl.max_bounces, rr_start=wl.rr_start, seed=0,
                              stream=stream, first_sample=first, out=img)
        return step

    def timed(step):
        for k in range(args.warmup):
            step(k)
        torch.cuda.synchronize(dev)
        times, segs = [], 0
        for k in range(args.steps):
            flush.fill_(float(k))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(k)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            p, q = r.segments(stream)
            segs += p + q
        return segs / (sum(times) / 1e3), sum(times) / len(times)

    def per(c):
        sec = max(1, int(c[1]))
        return {"nodes": int(c[4]) / sec, "tests": int(c[5]) / sec, "blended": int(c[3]) / sec,
                "secondary_segments": int(c[1])}

    def blocks(x, b=32):
        H, W = (x.shape[0] // b) * b, (x.shape[1] // b) * b
        return x[:H, :W].reshape(H // b, b, W // b, b, 3).mean((1, 3))

    first0, n0 = slices[0]

    def first_slice(render, seed=0):
        out = render(seed)
        api.sync_status()
        return out["stats"].cpu().numpy().copy(), out["rgb"].cpu().numpy().astype(np.float64)

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = L.eagpt_launch_count()
    v_plain, ms_plain = timed(plain_step)
    timed_pairs = [timed(lod_step(h, f)) for h, f in pairs]
    launches = L.eagpt_launch_count() - launches0
    clk = clocks.stop()
    api.sync_status()

    bvh = api.BVH(ds, stream=stream)
    cf, fimg = first_slice(lambda sd: r.path_traced(ds, bvh, cam, n0, wl.max_bounces, rr_start=wl.rr_start, seed=sd,
                                                    first_sample=first0, want_stats=True))
    _, fimg2 = first_slice(lambda sd: r.path_traced(ds, bvh, cam, n0, wl.max_bounces, rr_start=wl.rr_start, seed=sd,
                                                    first_sample=first0, want_stats=True), seed=1)
    mean_f = float(fimg.mean())
    noise = float(np.sqrt(np.mean((blocks(fimg2) - blocks(fimg)) ** 2)) / mean_f)
    sweep = []
    for (h, f), (v, ms) in zip(pairs, timed_pairs):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lod = api.LevelOfDetail(ds, LOD_ORIGIN, h, stream=stream)
        b.record(stream)
        b.synchronize()
        build_ms = a.elapsed_time(b)
        cl, limg = first_slice(lambda sd: r.path_traced_lod(ds, bvh, lod, f, cam, n0, wl.max_bounces,
                                                            rr_start=wl.rr_start, seed=sd, first_sample=first0,
                                                            want_stats=True))
        sweep.append({"lod_cell_m": h, "lod_from": f, "merged_surfels": lod.scene.n, "value": v, "ms_per_step": ms,
                      "speedup": v / v_plain, "merge_and_bvh_ms": build_ms,
                      "per_secondary_segment": per(cl),
                      "image_mean_rel_diff": float((limg.mean() - mean_f) / mean_f),
                      "block_rel_rmse": float(np.sqrt(np.mean((blocks(limg) - blocks(fimg)) ** 2)) / mean_f)})
    head = sweep[0]
    line = {"metric": METRIC, "value": head["value"], "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"large final render with level of detail: {wl.name}; bounce segments k >= "
                                   f"{head['lod_from']} trace the surfels merged over {head['lod_cell_m']} m cells",
                       "surfels": host_scene.n, "merged_surfels": head["merged_surfels"],
                       "scale_factor": wl.scale_factor, "lod_cell_m": head["lod_cell_m"],
                       "lod_from": head["lod_from"], "lod_origin": LOD_ORIGIN, "spp_per_step": slice_spp,
                       "frame_spp": frame_spp,
                       "step": "LBVH build + merge + merged LBVH build + render of one 64-sample slice",
                       "l2": "flushed between steps (512 MB write)"},
            "plain": {"value": v_plain, "ms_per_step": ms_plain, "step": "LBVH build + render of the same slices",
                      "per_secondary_segment": per(cf)},
            "speedup": head["speedup"],
            "accuracy": {"what": "first 64-sample slice: image mean and RMS of 32x32 block-mean differences against "
                                 "the plain render, relative to the plain image mean",
                         "plain_mean": mean_f, "noise_floor_block_rel_rmse": noise},
            "sweep": sweep, "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.workload == "lod" and args.impl == "native":
        if rank == 0:  # a one-GPU comparison; other ranks have nothing to do
            run_lod(args, local)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload in ("stage1", "bake") and args.impl == "native":
        run_fit(args)
        return
    if args.workload == "diff" and args.impl == "native":
        run_diff(args)
        return
    if args.workload == "mis" and args.impl == "native":
        run_mis(args)
        return
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        return
    run_render(args, rank, world, local)


if __name__ == "__main__":
    main()
