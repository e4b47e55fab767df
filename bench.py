"""Benchmark: path segments/s of the surfel path tracer on one GB300.

One step = one pass of the whole hot path over the workload: surfel
preprocess + LBVH build (sort, hierarchy, refit) + path-traced render (primary
segments, then per-bounce trace/shade/compact waves, then the deterministic
accumulation).  Default workload: the medium room (200k surfels, 512x512,
64 spp, up to 4 bounces, Russian roulette from bounce 2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload medium|large|tiny]
  python bench.py --impl reference ...    (the FP64 CPU oracle on a bounded sample)

Prints one JSON line (rank 0).  With N > 1 every rank renders its own share
of the samples (independent paths; no collective on the data path).
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
    ap.add_argument("--workload", default="medium", choices=["tiny", "medium", "diff", "large", "serving"])
    ap.add_argument("--requests", type=int, default=16, help="serving: requests in the stream")
    ap.add_argument("--spp", type=int, default=None, help="override samples per pixel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


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
def source_digest() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2601_23065_gb300", "csrc", "*"))):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def load_traffic(workload: str):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", f"k_bounce_{workload}_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_digest") != source_digest():
        return None
    return d.get("dram_bytes_per_launch")


def cpu_baseline(wl, scene, seconds: float):
    """The FP64 oracle on a bounded pixel sample of the same workload."""
    import numpy as np

    import oracle as O
    rng = np.random.default_rng(123)
    n_threads = O.default_threads()
    osc = O.OracleScene(scene)
    npix = wl.camera.width * wl.camera.height
    # grow the sample until ~`seconds` of CPU work
    m = 2
    total_segs, total_t, total_pix = 0, 0.0, 0
    while True:
        pix = rng.choice(npix, m, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        out = O.render(osc, wl.camera, pix, "pt", wl.spp, max_bounces=wl.max_bounces, rr_start=wl.rr_start,
                       seed=0, params=O.Params(fp32_eps=0.0), n_threads=n_threads)
        dt = time.perf_counter() - t0
        total_segs += int(out["segments"].sum())
        total_t += dt
        total_pix += m
        if total_t >= seconds or m >= 4096:
            break
        m = int(min(4096, max(m * 2, m * seconds / max(dt, 1e-3) / 2)))
    return {"value": total_segs / total_t, "unit": METRIC, "cores": n_threads, "kind": "oracle",
            "sample": f"{total_pix} random pixels x {wl.spp} spp of the same workload "
                      f"({total_segs} segments in {total_t:.1f} s, brute force over {scene.n} surfels, FP64)"}


def run_reference(args, rank, world):
    """--impl reference: the oracle as it stands, timed on the host cores."""
    if rank != 0:
        return
    from paper_2601_23065_gb300 import scenes as S
    wl = S.workload(args.workload)
    if args.spp:
        wl.spp = args.spp
    scene = wl.scene_fn()
    for _ in range(max(0, args.warmup)):
        cpu_baseline(wl, scene, 0.5)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(wl, scene, args.cpu_seconds / max(1, args.steps)))
    v = statistics.mean(x["value"] for x in vals)
    line = {"metric": METRIC, "value": v, "unit": METRIC, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Serving room (3M surfels): a seeded request stream (renders of
    256x256..1920x1080, 16/64/256 spp, 1-5 bounces, 10 % edits) served (a)
    by plain sequential launches, (b) by the continuous-batching server at
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
    reqs = S.serving_requests(host, args.requests, seed=13)
    n_render = sum(1 for r in reqs if r["type"] == "render")
    samples = sum(r["camera"].width * r["camera"].height * r["spp"] for r in reqs if r["type"] == "render")

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
    torch.cuda.synchronize(dev)
    plain_out, t0 = [], time.perf_counter()
    for r in reqs:
        if r["type"] == "render":
            o = rend.path_traced(ds, bvh, r["camera"], r["spp"], r["max_bounces"], rr_start=2, seed=r["seed"])
            plain_out.append(o["rgb"].clone())
        else:
            idx, per = resolve_edit(ds, r)
            api.apply_edit(ds, bvh, r["op"], idx, value=r.get("value", ()), per_index=per)
    torch.cuda.synchronize(dev)
    t_plain = time.perf_counter() - t0
    mu = n_render / t_plain
    del ds, bvh, rend
    torch.cuda.empty_cache()

    results = {}
    for load in (0.8, 1.2):
        ds = api.DeviceScene.from_host(host, device=dev)
        bvh = api.BVH(ds)
        srv = api.Server(ds, bvh, queue_paths=1 << 24, max_active=16)
        rng = np.random.default_rng(int(load * 100))
        arrivals = np.cumsum(rng.exponential(1.0 / (load * mu), len(reqs)))
        ids = []
        start = time.perf_counter()
        for r, ta in zip(reqs, arrivals):
            delay = start + ta - time.perf_counter()
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
        lat, equal, t_end = [], True, start
        k = 0
        for kind, x in ids:
            if kind == "render":
                rid, out = x
                info = srv.wait(rid, 1200.0)
                lat.append(info["t_done"] - info["t_submit"])
                t_end = max(t_end, info["t_done"])
                torch.cuda.synchronize(dev)
                equal &= bool(torch.equal(out, plain_out[k]))
                k += 1
            else:
                srv.wait(x, 1200.0)
        st = srv.stats()
        first_submit = start + arrivals[0]
        span = max(1e-9, time.perf_counter() - first_submit)
        results[f"load_{load}"] = {"throughput": samples / span, "p50_s": float(np.percentile(lat, 50)),
                                   "p99_s": float(np.percentile(lat, 99)), "equal_to_plain": equal,
                                   "segments_per_s_busy": st["segments"] / max(st["busy_s"], 1e-9),
                                   "waves": st["waves"], "edits": st["edits"], "rebuilds": st["rebuilds"]}
        srv.close()
        del ds, bvh
        torch.cuda.empty_cache()
    line = {"metric": "pixel samples/s (serving)", "value": results["load_1.2"]["throughput"],
            "unit": "pixel samples/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving room 3M surfels, Poisson request stream", "requests": len(reqs),
                       "renders": n_render, "pixel_samples": samples},
            "plain": {"throughput": samples / t_plain, "capacity_req_per_s": mu, "seconds": t_plain},
            "served": results}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.workload == "serving":
        run_serving(args)
        return
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        return

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
    if args.spp:
        wl.spp = args.spp
    host_scene = wl.scene_fn()
    cam = wl.camera
    seed_base = 1000003 * rank  # each rank renders its own samples
    ds = api.DeviceScene.from_host(host_scene, device=dev)
    r = api.Renderer(device=dev)
    stream = torch.cuda.current_stream(dev)
    L = capi.lib()

    def step(seed):
        bvh = api.BVH(ds, stream=stream)
        out = r.path_traced(ds, bvh, cam, wl.spp, wl.max_bounces, rr_start=wl.rr_start, seed=seed, stream=stream)
        return bvh, out

    # untimed: counters of the work one step does (same seeds as timed)
    bvh0 = api.BVH(ds, stream=stream)
    cnt = r.path_traced(ds, bvh0, cam, wl.spp, wl.max_bounces, rr_start=wl.rr_start, seed=seed_base,
                        want_stats=True)["stats"].cpu().numpy()
    api.sync_status()
    prim_segs, sec_segs = int(cnt[0]), int(cnt[1])
    segs_per_step = prim_segs + sec_segs
    paths = int(cnt[2])
    del bvh0

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    for w in range(args.warmup):
        step(seed_base)
    torch.cuda.synchronize(dev)

    # timed region
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = L.eagpt_launch_count()
    capi.check(L.eagpt_profile_begin())
    barrier()
    torch.cuda.synchronize(dev)
    times = []
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between steps (outside the step's events)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(seed_base)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    torch.cuda.synchronize(dev)
    barrier()
    prof = capi.profile_end()
    launches = L.eagpt_launch_count() - launches0
    clk = clocks.stop()
    api.sync_status()

    ms = sum(times) / len(times)
    t_local = sum(times) / 1e3
    if world > 1:
        t = torch.tensor([t_local], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    else:
        t_max = t_local
    value = world * segs_per_step * args.steps / t_max

    # roofline of the dominant kernel (the fused trace/shade/compact bounce)
    kern = max(prof.items(), key=lambda kv: kv[1][1])
    bounce = prof.get("k_bounce", (0, 0.0))
    total_kernel_ms = sum(v[1] for v in prof.values())
    peak, peak_kind = load_peaks()
    # counters of the secondary segments: blended hits, nodes, surfel tests
    cnt2 = r.path_traced(ds, api.BVH(ds), cam, wl.spp, wl.max_bounces, rr_start=wl.rr_start, seed=seed_base,
                         want_stats=True)["stats"].cpu().numpy()
    blended, nodes, tests, rounds = int(cnt2[3]), int(cnt2[4]), int(cnt2[5]), int(cnt2[6])
    # per-segment algorithmic bytes: 48 B ray read + 48 B ray/slot write +
    # 64 B per node + 64 B per surfel test + 32 B per blended shade record
    bounce_launches_per_step = bounce[0] / max(1, args.steps)
    bounce_ms_per_launch = bounce[1] / max(1, bounce[0])
    # bytes of the bounce launches only (secondary segments)
    alg_bytes_bounce_launch = (96 * sec_segs + 64 * nodes + 64 * tests + 32 * blended) / max(
        1.0, bounce_launches_per_step)
    achieved = alg_bytes_bounce_launch / (bounce_ms_per_launch * 1e-3) / 1e9 if bounce_ms_per_launch else None
    traffic = load_traffic(args.workload)
    roofline = {"bound": "hbm", "kernel": "k_bounce", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                "bytes_per_launch": alg_bytes_bounce_launch, "ms_per_launch": bounce_ms_per_launch,
                "share_of_kernel_time": bounce[1] / total_kernel_ms if total_kernel_ms else None,
                "per_secondary_segment": {"nodes": nodes / max(1, sec_segs), "tests": tests / max(1, sec_segs),
                                          "blended": blended / max(1, sec_segs),
                                          "rounds": rounds / max(1, sec_segs)}}

    # end to end through the public API with host buffers
    pinned = {k: torch.from_numpy(getattr(host_scene, k)).pin_memory() for k in api.FIELDS}
    dev_t = {k: torch.empty_like(v, device=dev) for k, v in pinned.items()}
    out_host = torch.empty((cam.height, cam.width, 3), dtype=torch.float32).pin_memory()
    h2d = sum(v.numel() * 4 for v in pinned.values())
    d2h = out_host.numel() * 4
    e2e_times = []
    for k in range(max(1, args.steps)):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for kk in api.FIELDS:
            dev_t[kk].copy_(pinned[kk], non_blocking=True)
        dsk = api.DeviceScene(dev_t)
        bvh = api.BVH(dsk, stream=stream)
        out = r.path_traced(dsk, bvh, cam, wl.spp, wl.max_bounces, rr_start=wl.rr_start, seed=seed_base)
        out_host.copy_(out["rgb"], non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_times.append(time.perf_counter() - t0)
    e2e_val = world * segs_per_step / (sum(e2e_times) / len(e2e_times))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, host_scene, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": wl.name, "surfels": host_scene.n, "width": cam.width, "height": cam.height,
                           "spp": wl.spp, "max_bounces": wl.max_bounces, "rr_start": wl.rr_start,
                           "segments_per_step": segs_per_step, "primary_segments": prim_segs,
                           "secondary_segments": sec_segs, "paths_per_step": paths,
                           "rays_per_s": world * paths * args.steps / t_max,
                           "step": "LBVH build + path-traced render",
                           "l2": "flushed between steps (512 MB write)",
                           "parallelism": f"replicas x{world} (independent samples per rank)"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": int(launches), "clocks": clk,
                "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items())}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
