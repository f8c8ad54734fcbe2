"""Benchmark: batched ray-cast depth+segmentation rendering on GB300.

Workload (default): 1024 synthetic obstacle rooms (10 x 10 x 4 m, 20-40
obstacles each, ~18.8k triangles per env), one 270x480 pinhole depth+seg
camera per env (87 deg hfov, 0.2-10 m), sensor poses walking for 100 steps.
One step = one render of every env (132.7 M rays) with that step's poses.

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mrays/s at 1024 envs x 270x480 depth+seg vs plain; p50/p99 served latency"
UNIT = "Mrays/s"
# other workloads of the method, measured with the same harness (--workload)
WORKLOADS = {
    "rooms": {"envs": 1024, "metric": METRIC},
    "forest": {"envs": 256, "metric": "Mrays/s at 256 LiDAR forests x 64x512 range+seg"},
    "serving": {"envs": 8192, "metric": "served Mrays/s, 8192 rooms of 1k-200k triangles, mixed sensors; p50/p99 ms"},
    "precision": {"envs": 4096, "metric": "Mrays/s at 4096 rooms x 135x240 per BVH node format; depth error vs FP64"},
    "dynamic": {"envs": 1024, "metric": "ms per obstacle-pose update (refit vs rebuild), 1024 rooms; render Mrays/s"},
    "features": {"envs": 1024, "metric": "Mrays/s at 1024 rooms per sensor feature (hit channels, stereo, projection models)"},
}
PAPER_MRAYS = 340.5  # Table II, 1024 envs x 270x480 (RTX 3090; context)
PROFILE_DIR = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rooms", choices=sorted(WORKLOADS))
    ap.add_argument("--envs", type=int, default=None, help="environments per GPU (workload default)")
    ap.add_argument("--width", type=int, default=None, help="camera columns (rooms only)")
    ap.add_argument("--height", type=int, default=None, help="camera rows (rooms only)")
    ap.add_argument("--walk", type=int, default=100, help="length of the sensor-pose random walk")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--build-flags", type=int, default=0, help="ags_scene_build flags")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--no-serving", action="store_true", help="skip the served-latency measurement")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="Poisson arrivals per load in --workload serving (seconds)")
    ap.add_argument("--no-sub-records", action="store_true",
                    help="skip the forest and node-format records of the default line")
    args = ap.parse_args()
    if args.envs is None:
        args.envs = WORKLOADS[args.workload]["envs"]
    if args.workload == "rooms":
        args.width = args.width or 480
        args.height = args.height or 270
    return args


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the render kernel's and BVH builders' code, comments and blank space left out (a comment edit
    does not invalidate counters taken from the same code)."""
    import re
    h = hashlib.sha256()
    for f in ("trace.cu", "trace_kernel.cuh", "internal.cuh", "build.cu", "ploc.cu", "radix_sort.cu"):
        with open(os.path.join(ROOT, "paper_2503_01471_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled_counters(workload, kernel):
    """(DRAM bytes, warp instructions) per launch of the render kernel from the committed ncu summary, if its
    row matches this workload, this kernel instance and the current kernel and builder sources; else None."""
    try:
        names = sorted(f for f in os.listdir(PROFILE_DIR) if f.startswith("k_trace_") and f.endswith("_traffic.md"))
        for name in names:
            with open(os.path.join(PROFILE_DIR, name)) as fh:
                for line in fh:
                    cells = [c.strip() for c in line.strip().strip("|").split("|")]
                    if len(cells) == 7 and cells[0] == workload and cells[1] == kernel \
                            and cells[2] == kernel_source_hash():
                        return float(cells[5]), float(cells[6])
    except (OSError, ValueError):
        pass
    return None


def clocks_rejected(c) -> bool:
    """A timed region whose clock record shows a hardware or thermal slowdown, or SM clocks well below
    their maximum with no reason given (a clock lock left behind), is not a valid measurement. A power
    cap alone is kept (normal for a dense load)."""
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(c.get("reasons") or []):
        return True
    sm, mx = c.get("sm_mhz"), c.get("sm_max_mhz")
    return bool(sm and mx and sm < 0.85 * mx and not c.get("reasons"))


def issue_peak_g(sm_count: int, sm_max_mhz: float) -> float:
    """Warp-instruction issue limit of the device in G/s: every SM has 4 schedulers, each issuing at most one
    warp instruction per cycle, at the maximum SM clock."""
    return sm_count * 4 * sm_max_mhz / 1e3


def sm_max_mhz(clocks) -> float:
    """The maximum SM clock: as sampled by nvidia-smi during the run, else the measured peaks file."""
    if clocks and clocks.get("sm_max_mhz"):
        return float(clocks["sm_max_mhz"])
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"])
    except Exception:
        return 2070.0


def rooflines(counters, ms_step, b_ray, rays, hbm, peak_kind, sm_count, mhz, nodes_per_ray, tris_per_ray,
              node_bytes):
    """The lead roofline of the render kernel and the algorithmic-bytes one beside it.

    The BVHs and triangles of an environment stay in L1/L2 while all SMs work on it, so what bounds the kernel
    is instruction issue, not DRAM: the lead block is the issue roofline (warp instructions per launch from the
    committed ncu capture of this kernel and these sources, per second, against SMs x 4 x max clock), with the
    DRAM traffic of that capture beside it. The algorithmic block is the B_ray roofline: the bytes of nodes and
    triangles a ray fetches, per second, against the HBM copy bandwidth; it exceeds 1 because those bytes are
    served mostly from L1/L2."""
    algo_gbs = b_ray * rays / (ms_step * 1e-3) / 1e9
    algorithmic = {"bound": "hbm", "achieved": algo_gbs, "peak": hbm, "unit": "GB/s", "frac": algo_gbs / hbm,
                   "peak_kind": peak_kind + " hbm_gbs (copy)",
                   "achieved_is": "algorithmic bytes served (node and triangle fetches per ray, mostly from L1/L2)",
                   "bytes_per_ray": b_ray, "nodes_per_ray": nodes_per_ray, "tris_per_ray": tris_per_ray,
                   "node_bytes": node_bytes}
    peak_g = issue_peak_g(sm_count, mhz)
    if counters is None:
        return dict(algorithmic, traffic=None, kernel="k_trace"), None
    dram_gbs = counters[0] / (ms_step * 1e-3) / 1e9
    achieved = counters[1] / (ms_step * 1e-3) / 1e9
    lead = {"bound": "alu", "achieved": achieved, "peak": peak_g, "unit": "G warp instructions/s",
            "frac": achieved / peak_g, "traffic": counters[0], "kernel": "k_trace",
            "peak_kind": f"{sm_count} SMs x 4 schedulers x 1 warp instruction/cycle x {mhz:.0f} MHz (max SM clock)",
            "instructions_per_launch": counters[1], "dram_gbs": dram_gbs, "dram_frac": dram_gbs / hbm,
            "dram_peak_kind": peak_kind + " hbm_gbs (copy)", "algorithmic": algorithmic}
    return lead, algorithmic


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- oracle (CPU) timing
def run_oracle(batch, spec, poses_step, envs, rays_per_env, seed=7):
    import oracle as O
    s = O.Sensor(type=int(spec.type), width=int(spec.width), height=int(spec.height),
                 hfov=float(np.float32(spec.hfov)), min_range=float(np.float32(spec.min_range)),
                 max_range=float(np.float32(spec.max_range)), vfov_min=float(np.float32(spec.vfov_min)),
                 vfov_max=float(np.float32(spec.vfov_max)), near_mode=int(spec.near_mode))
    rng = np.random.default_rng(seed)
    n_pix = spec.width * spec.height
    work = []
    for e in envs:
        vs, ix, ps, sg = batch.env_submeshes(int(e))
        tris, tseg = O.world_triangles(vs, ix, ps, sg)
        rays = np.sort(rng.choice(n_pix, min(rays_per_env, n_pix), replace=False)).astype(np.int64)
        work.append((tris, tseg, np.asarray(poses_step[e], np.float64), rays))
    t0 = time.perf_counter()
    n = tests = 0
    for tris, tseg, pose, rays in work:
        O.render(tris, tseg, s, pose, rays)
        n += rays.shape[0]
        tests += rays.shape[0] * tris.shape[0]
    dt = time.perf_counter() - t0
    run_oracle.last_tests = tests
    return n, dt, O.num_threads()


def cpu_baseline(batch, spec, poses, budget_s=12.0):
    """Oracle Mrays/s on a bounded sample of the workload (~10-30 s of CPU work)."""
    E = batch.n_envs
    envs = [0, E // 2, E - 1] if E >= 3 else list(range(E))
    n, dt, cores = run_oracle(batch, spec, poses[0], envs, 64)
    per_ray = dt / max(n, 1)
    k = int(max(64, min(spec.width * spec.height, budget_s / per_ray / len(envs))))
    n, dt, cores = run_oracle(batch, spec, poses[0], envs, k, seed=8)
    rays_per_step = E * spec.width * spec.height
    return {"value": n / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} random rays ({k} from each of envs {envs}) at step 0, FP64 brute force "
                      f"over every triangle of the env, {dt:.1f} s",
            "ray_tri_tests_per_s": run_oracle.last_tests / dt,
            "full_step_s_extrapolated": rays_per_step * dt / max(n, 1)}


# ---------------------------------------------------------------- serving
def serving_specs():
    from paper_2503_01471_gb300 import scenes as S
    return [S.pinhole(240, 135), S.pinhole(480, 270), S.lidar(512, 64)]


def serving_measure(ags, ctx, scene, n_envs, poses_step, specs, loads=(0.5, 1.0), duration=0.5, seq_max=2000,
                    burst=20000, seed=5, use_graph=True, sequential=True):
    """Continuous-batching server under a burst (capacity) and Poisson arrivals at fractions of it, and the
    sequential one-request-at-a-time launch on the same traces (first seq_max requests). use_graph: each
    stream replays its captured batch graph (else three calls per batch)."""
    rng = np.random.default_rng(seed)
    rays = np.array([sp.width * sp.height for sp in specs])

    def trace(n, rate):
        env = rng.integers(0, n_envs, n)
        sp = rng.integers(0, len(specs), n)
        reqs = ags.make_requests(env, sp, poses_step[env])
        arrival = np.cumsum(rng.exponential(1.0 / rate, n)) if rate else np.zeros(n)
        return reqs, arrival

    def pct(x, q):
        return float(np.percentile(x, q)) if len(x) else None

    server = ags.ags_server_create(ctx, scene, specs, max_slots=512, max_inflight=4, arena_bytes=4 << 30,
                                   use_graph=use_graph)
    try:
        reqs, arr = trace(burst, None)
        out = ags.ags_server_replay(server, reqs, arr)
        span = float(out["t_done"].max() - out["t_submit"].min())
        cap = burst / span
        res = {"capacity_req_per_s": cap, "capacity_mrays_per_s": float(rays[reqs["spec"]].sum()) / span / 1e6,
               "sensors": [f"{'camera' if sp.type == 0 else 'lidar'} {sp.height}x{sp.width}" for sp in specs],
               "max_slots": 512, "max_inflight": 4, "use_graph": use_graph, "seconds_per_load": duration,
               "loads": []}
        for f in loads:
            rate = f * cap
            n = max(100, int(rate * duration))
            reqs, arr = trace(n, rate)
            out = ags.ags_server_replay(server, reqs, arr)
            lat = (out["t_done"] - out["t_submit"]) * 1e3
            m = min(seq_max, n)
            slat = np.zeros(0)
            if sequential:
                seq = ags.ags_replay_sequential(ctx, scene, specs, reqs[:m], arr[:m])
                slat = (seq["t_done"] - seq["t_submit"]) * 1e3
            by_sensor = [{"sensor": res["sensors"][k], "requests": int((reqs["spec"] == k).sum()),
                          "p50_ms": pct(lat[reqs["spec"] == k], 50), "p99_ms": pct(lat[reqs["spec"] == k], 99)}
                         for k in range(len(specs))]
            res["loads"].append({"load": f, "req_per_s": rate, "requests": n, "p50_ms": pct(lat, 50),
                                 "p99_ms": pct(lat, 99), "mrays_per_s": float(rays[reqs["spec"]].sum()) /
                                 float(out["t_done"].max() - out["t_submit"].min()) / 1e6,
                                 "by_sensor": by_sensor,
                                 "sequential": {"requests": int(slat.shape[0]), "p50_ms": pct(slat, 50),
                                                "p99_ms": pct(slat, 99)}})
        if not sequential:
            return res
        # a load the sequential launch can sustain: half its own capacity, same trace for both
        reqs, arr = trace(300, None)
        seq = ags.ags_replay_sequential(ctx, scene, specs, reqs, arr)
        seq_cap = 300 / float(seq["t_done"].max() - seq["t_submit"].min())
        rate = 0.5 * seq_cap
        n = max(200, min(2000, int(rate * 2 * duration)))
        reqs, arr = trace(n, rate)
        out = ags.ags_server_replay(server, reqs, arr)
        seq = ags.ags_replay_sequential(ctx, scene, specs, reqs, arr)
        lat = (out["t_done"] - out["t_submit"]) * 1e3
        slat = (seq["t_done"] - seq["t_submit"]) * 1e3
        res["sequential_capacity_req_per_s"] = seq_cap
        res["at_half_sequential_capacity"] = {
            "req_per_s": rate, "requests": n, "batched": {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99)},
            "sequential": {"p50_ms": pct(slat, 50), "p99_ms": pct(slat, 99)}}
        st = ags.ags_server_stats(server)
        res["batches"] = st["batches"]
    finally:
        ags.ags_server_destroy(server)
    return res


def bench_serving(args, rank, world, local):
    """Serving workload: rooms of 1k-200k triangles, mixed camera and LiDAR requests."""
    import torch

    import paper_2503_01471_gb300 as ags
    from paper_2503_01471_gb300 import build as B
    from paper_2503_01471_gb300 import scenes as S

    B.build()
    torch.cuda.set_device(local)
    batch, poses = S.serving_rooms(args.envs)
    ctx = ags.ags_context_create(local)
    t0 = time.perf_counter()
    scene = ags.ags_scene_build(ctx, batch, args.build_flags)
    build_s = time.perf_counter() - t0
    n_tris = int(batch.env_tri_counts().sum())
    specs = serving_specs()
    with ClockSampler(torch.cuda.current_device()) as clk:
        res = serving_measure(ags, ctx, scene, batch.n_envs, poses[0], specs,
                              loads=(0.5, 0.75, 1.0, 1.25, 1.5), duration=args.serve_seconds)
        res["without_graph"] = serving_measure(ags, ctx, scene, batch.n_envs, poses[0], specs, loads=(0.5, 1.0),
                                               duration=args.serve_seconds, use_graph=False, sequential=False)
    line = {"metric": WORKLOADS["serving"]["metric"], "value": res["capacity_mrays_per_s"], "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving: {batch.n_envs} rooms, triangles log-uniform 1k-200k "
                                   f"({n_tris / 1e6:.1f} M resident), Poisson arrivals",
                       "tris": n_tris, "bvh_bytes": ags.ags_scene_stats(scene)[2]},
            "serving": res, "clocks": clk.summary(), "build_ms": build_s * 1e3}
    print(json.dumps(line), flush=True)
    ags.ags_scene_destroy(scene)
    ags.ags_context_destroy(ctx)


# ---------------------------------------------------------------- precision
def bench_precision(args, rank, world, local):
    """Node formats (float32, float16, 8-bit child bounds) on the same scenes: rays/s, bytes per ray,
    bit-exactness of the outputs across formats, and depth error against the FP64 oracle."""
    import torch

    import oracle as O
    import paper_2503_01471_gb300 as ags
    from paper_2503_01471_gb300 import build as B
    from paper_2503_01471_gb300 import scenes as S

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    batch, spec, poses = S.obstacle_rooms(args.envs, steps=args.walk, width=240, height=135)
    E = batch.n_envs
    ctx = ags.ags_context_create(local)
    poses_d = torch.as_tensor(poses).to(dev)
    depth = torch.empty((E, spec.height, spec.width), dtype=torch.float32, device=dev)
    seg = torch.empty((E, spec.height, spec.width), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rays = E * spec.width * spec.height
    formats = {"fp32": ags.AGS_BVH_FP32, "fp16": ags.AGS_BVH_FP16, "q8": ags.AGS_BVH_Q8}
    res, ref = {}, None
    for name, flag in formats.items():
        scene = ags.ags_scene_build(ctx, batch, flag | args.build_flags)
        cfg = ags.ags_autotune(ctx, scene, spec, poses_d[0], depth, seg, 2).as_dict()
        for i in range(args.warmup):
            ags.ags_render(ctx, scene, spec, poses_d[i % poses_d.shape[0]], depth, seg, stream)
        st, en = torch.cuda.Event(True), torch.cuda.Event(True)
        torch.cuda.synchronize(dev)
        st.record(stream)
        for i in range(args.steps):
            ags.ags_render(ctx, scene, spec, poses_d[(args.warmup + i) % poses_d.shape[0]], depth, seg, stream)
        en.record(stream)
        torch.cuda.synchronize(dev)
        ags.ags_stream_status(ctx, stream)
        ms = st.elapsed_time(en) / args.steps
        r_c, n_c, t_c = ags.ags_render_count(ctx, scene, spec, poses_d[0])
        nb = ags.ags_scene_node_bytes(scene)
        b_ray = (n_c * nb + t_c * 48) / r_c + 8.0
        ags.ags_render(ctx, scene, spec, poses_d[0], depth, seg, stream)
        ags.ags_stream_status(ctx, stream)
        out = (depth.cpu().numpy(), seg.cpu().numpy())
        if ref is None:
            ref = out
        res[name] = {"mrays_per_s": rays / ms / 1e3, "ms_per_step": ms, "node_bytes": nb,
                     "bvh_bytes": ags.ags_scene_stats(scene)[2], "bytes_per_ray": b_ray,
                     "nodes_per_ray": n_c / r_c, "tris_per_ray": t_c / r_c, "launch_config": cfg,
                     "bit_identical_to_fp32": bool(np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]))}
        ags.ags_scene_destroy(scene)
    # depth error against the FP64 oracle (outputs are the same for every format)
    rng = np.random.default_rng(11)
    s_or = O.Sensor(type=0, width=spec.width, height=spec.height, hfov=float(np.float32(spec.hfov)),
                    min_range=float(np.float32(spec.min_range)), max_range=float(np.float32(spec.max_range)))
    abs_e, rel_e, counted, n_s, loose = [], [], 0, 0, 0
    for e in rng.choice(E, min(E, 96), replace=False):
        vs, ix, ps, sg = batch.env_submeshes(int(e))
        tris, tseg = O.world_triangles(vs, ix, ps, sg)
        rr = np.sort(rng.choice(spec.width * spec.height, 256, replace=False)).astype(np.int64)
        resu = O.render(tris, tseg, s_or, poses[0][e].astype(np.float64), rr)
        d = ref[0][e].reshape(-1)[rr].astype(np.float64)
        g = ref[1][e].reshape(-1)[rr]
        ok, cnt = O.check(resu, d, g, s_or.max_range)
        if not ok.all():
            raise RuntimeError(f"precision bench: env {e}: {int((~ok).sum())} rays outside the oracle's outcomes")
        hit = (~cnt) & (resu["seg"] >= 0)
        abs_e.append(np.abs(d - resu["v"])[hit])
        rel_e.append((np.abs(d - resu["v"]) / resu["v"])[hit])
        counted += int(cnt.sum())
        loose += int((~cnt & (resu["seg"] >= 0) & (np.abs(d - resu["v"]) > O.tol(resu["v"]))).sum())
        n_s += rr.shape[0]
    a = np.concatenate(abs_e)
    r = np.concatenate(rel_e)
    err = {"sampled_rays": n_s, "single_outcome_hits": int(a.shape[0]), "counted": counted,
           "beyond_tolerance": loose, "max_abs_m": float(a.max()), "p999_abs_m": float(np.percentile(a, 99.9)),
           "max_rel": float(r.max()), "p999_rel": float(np.percentile(r, 99.9)),
           "tolerance": "1e-5*d + 1e-6 m"}
    line = {"metric": WORKLOADS["precision"]["metric"], "value": res["q8"]["mrays_per_s"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": f"obstacle rooms, {E} envs x 135x240 camera",
                                            "tris": int(batch.env_tri_counts().sum())},
            "formats": res, "depth_error_vs_fp64": err}
    print(json.dumps(line), flush=True)
    ags.ags_context_destroy(ctx)


# ---------------------------------------------------------------- dynamic obstacles
def bench_dynamic(args, rank, world, local):
    """Obstacles moving every step: refit vs rebuild cost, and how the refitted tree's render speed drifts."""
    import torch

    import paper_2503_01471_gb300 as ags
    from paper_2503_01471_gb300 import build as B
    from paper_2503_01471_gb300 import scenes as S

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    batch, spec, poses = S.obstacle_rooms(args.envs, steps=args.walk, width=480, height=270)
    E = batch.n_envs
    ctx = ags.ags_context_create(local)
    p = torch.as_tensor(poses[0]).to(dev)
    depth = torch.empty((E, spec.height, spec.width), dtype=torch.float32, device=dev)
    seg = torch.empty((E, spec.height, spec.width), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rays = E * spec.width * spec.height

    def render_ms(scene, reps=5):
        ags.ags_render(ctx, scene, spec, p, depth, seg, stream)
        st, en = torch.cuda.Event(True), torch.cuda.Event(True)
        torch.cuda.synchronize(dev)
        st.record(stream)
        for _ in range(reps):
            ags.ags_render(ctx, scene, spec, p, depth, seg, stream)
        en.record(stream)
        torch.cuda.synchronize(dev)
        return st.elapsed_time(en) / reps

    rng = np.random.default_rng(31)
    movable = np.ones(batch.poses.shape[0], bool)
    movable[batch.env_sub[:-1]] = False
    refit = ags.ags_scene_build(ctx, batch)
    rebuilt = ags.ags_scene_build(ctx, batch)
    two = ags.ags_scene_build(ctx, batch, ags.AGS_BUILD_INSTANCED)
    auto = ags.ags_scene_build(ctx, batch)
    cur = batch.poses.copy()
    rows = []
    t_refit, t_rebuild, t_two, t_auto = [], [], [], []
    auto_rebuilds = 0

    def cost_ratio(scene):
        now, built = ags.ags_scene_tree_cost(ctx, scene)
        return now / built if built > 0 else None
    for step in range(args.steps + 1):
        if step > 0:  # obstacles drift: 5 cm and 0.05 rad per step
            cur[movable, :3] += rng.normal(0, 0.05, (movable.sum(), 3)).astype(np.float32)
            dq = rng.normal(0, 0.025, (movable.sum(), 4)).astype(np.float32)
            q = cur[movable, 3:] + dq
            cur[movable, 3:] = q / np.linalg.norm(q, axis=1, keepdims=True)
            t0 = time.perf_counter()
            ags.ags_scene_update_poses(ctx, refit, cur, ags.AGS_UPDATE_REFIT)
            t_refit.append((time.perf_counter() - t0) * 1e3)
            t0 = time.perf_counter()
            ags.ags_scene_update_poses(ctx, rebuilt, cur, ags.AGS_UPDATE_REBUILD)
            t_rebuild.append((time.perf_counter() - t0) * 1e3)
            t0 = time.perf_counter()
            ags.ags_scene_update_poses(ctx, two, cur, ags.AGS_UPDATE_REBUILD)
            t_two.append((time.perf_counter() - t0) * 1e3)
            built_before = ags.ags_scene_tree_cost(ctx, auto)[1]
            t0 = time.perf_counter()
            ags.ags_scene_update_poses(ctx, auto, cur, ags.AGS_UPDATE_AUTO)
            t_auto.append((time.perf_counter() - t0) * 1e3)
            auto_rebuilds += int(ags.ags_scene_tree_cost(ctx, auto)[1] != built_before)
        if step in (0, 1, args.steps // 2, args.steps):
            rows.append({"step": step, "refit_mrays_per_s": rays / render_ms(refit) / 1e3,
                         "rebuild_mrays_per_s": rays / render_ms(rebuilt) / 1e3,
                         "two_level_mrays_per_s": rays / render_ms(two) / 1e3,
                         "auto_mrays_per_s": rays / render_ms(auto) / 1e3,
                         "refit_tree_cost_ratio": cost_ratio(refit), "auto_tree_cost_ratio": cost_ratio(auto),
                         "auto_rebuilds_so_far": auto_rebuilds})
    line = {"metric": WORKLOADS["dynamic"]["metric"], "value": float(np.median(t_refit)), "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"obstacle rooms, {E} envs, 270x480 camera; every obstacle moves each step",
                       "tris": int(batch.env_tri_counts().sum())},
            "refit_ms": {"median": float(np.median(t_refit)), "max": float(np.max(t_refit))},
            "rebuild_ms": {"median": float(np.median(t_rebuild)), "max": float(np.max(t_rebuild))},
            "two_level_update_ms": {"median": float(np.median(t_two)), "max": float(np.max(t_two))},
            "auto_update_ms": {"median": float(np.median(t_auto)), "max": float(np.max(t_auto)),
                               "rebuilds": auto_rebuilds, "rebuild_ratio": 1.25},
            "render_after_updates": rows}
    print(json.dumps(line), flush=True)
    for sc in (refit, rebuilt, two, auto):
        ags.ags_scene_destroy(sc)
    ags.ags_context_destroy(ctx)


# ---------------------------------------------------------------- sensor features
def bench_features(args, rank, world, local):
    """Cost of the extra sensor features on the 1024-room scene: hit channels, stereo shadows, a fisheye
    ray table, a dome LiDAR and the 848x480 navigation-task camera, each against the plain render."""
    import torch

    import paper_2503_01471_gb300 as ags
    from paper_2503_01471_gb300 import build as B
    from paper_2503_01471_gb300 import scenes as S

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    batch, spec, poses = S.obstacle_rooms(args.envs, steps=args.walk, width=480, height=270)
    E = batch.n_envs
    ctx = ags.ags_context_create(local)
    scene = ags.ags_scene_build(ctx, batch)
    poses_d = torch.as_tensor(poses).to(dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, rays):
        for i in range(args.warmup):
            fn(i)
        st, en = torch.cuda.Event(True), torch.cuda.Event(True)
        torch.cuda.synchronize(dev)
        st.record(stream)
        for i in range(args.steps):
            fn(args.warmup + i)
        en.record(stream)
        torch.cuda.synchronize(dev)
        ags.ags_stream_status(ctx, stream)
        ms = st.elapsed_time(en) / args.steps
        return {"mrays_per_s": rays / ms / 1e3, "ms_per_step": ms}

    def buffers(sp, chans=False):
        H, W = sp.height, sp.width
        b = {"d": torch.empty((E, H, W), device=dev), "s": torch.empty((E, H, W), dtype=torch.int32, device=dev)}
        if chans:
            b.update(face=torch.empty((E, H, W), dtype=torch.int32, device=dev),
                     bary=torch.empty((E, H, W, 2), device=dev), normal=torch.empty((E, H, W, 3), device=dev),
                     point=torch.empty((E, H, W, 3), device=dev))
        return b

    out = {}
    walk = poses_d.shape[0]
    rays = E * spec.width * spec.height
    b = buffers(spec, True)
    ch = {k: b[k] for k in ("face", "bary", "normal", "point")}
    out["camera_270x480"] = timed(lambda i: ags.ags_render(ctx, scene, spec, poses_d[i % walk], b["d"], b["s"], stream),
                                  rays)
    out["camera_270x480_channels"] = timed(
        lambda i: ags.ags_render_ex(ctx, scene, spec, poses_d[i % walk], b["d"], b["s"], stream=stream, **ch), rays)
    out["camera_270x480_stereo"] = timed(
        lambda i: ags.ags_render_ex(ctx, scene, spec, poses_d[i % walk], b["d"], b["s"], baseline=(0.0, -0.095, 0.0),
                                    stream=stream), rays)
    out["camera_270x480_channels_stereo"] = timed(
        lambda i: ags.ags_render_ex(ctx, scene, spec, poses_d[i % walk], b["d"], b["s"], baseline=(0.0, -0.095, 0.0),
                                    stream=stream, **ch), rays)
    del b, ch
    fs = S.ray_table_spec(480, 270, 0.2, 10.0)
    table = torch.as_tensor(S.fisheye_table(480, 270, 180.0)).to(dev)
    b = buffers(fs)
    out["fisheye_180_270x480_table"] = timed(
        lambda i: ags.ags_render_ex(ctx, scene, fs, poses_d[i % walk], b["d"], b["s"], ray_table=table, stream=stream),
        rays)
    del b
    dome = S.dome_lidar(512, 64, 0.2, 12.0)
    b = buffers(dome)
    out["dome_lidar_64x512"] = timed(lambda i: ags.ags_render(ctx, scene, dome, poses_d[i % walk], b["d"], b["s"], stream),
                                     E * 64 * 512)
    del b
    nav = S.pinhole(848, 480, 87.0, 0.2, 10.0)
    b = buffers(nav)
    out["camera_480x848"] = timed(lambda i: ags.ags_render(ctx, scene, nav, poses_d[i % walk], b["d"], b["s"], stream),
                                  E * 848 * 480)
    del b
    line = {"metric": WORKLOADS["features"]["metric"], "value": out["camera_270x480"]["mrays_per_s"], "unit": UNIT,
            "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
            "data": "synthetic", "config": {"workload": f"obstacle rooms, {E} envs; each feature on the same scene",
                                            "tris": int(batch.env_tri_counts().sum())},
            "features": out}
    print(json.dumps(line), flush=True)
    ags.ags_scene_destroy(scene)
    ags.ags_context_destroy(ctx)


# ---------------------------------------------------------------- sub-records of the default line
def timed_renders(ags, ctx, scene, spec, poses_d, depth, seg, stream, steps, warmup, min_seconds=0.5):
    """ms per render over at least `steps` renders after `warmup`, CUDA events on the render stream, clocks
    sampled. Short renders are repeated until the timed region lasts about min_seconds, so that the clock
    record (sampled every 100 ms) covers it."""
    import torch
    walk = poses_d.shape[0]
    st, en = torch.cuda.Event(True), torch.cuda.Event(True)
    st.record(stream)
    for i in range(warmup):
        ags.ags_render(ctx, scene, spec, poses_d[i % walk], depth, seg, stream)
    en.record(stream)
    torch.cuda.synchronize()
    per = st.elapsed_time(en) / max(warmup, 1)
    steps = int(min(5000, max(steps, math.ceil(min_seconds * 1e3 / max(per, 1e-3)))))
    st, en = torch.cuda.Event(True), torch.cuda.Event(True)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        st.record(stream)
        for i in range(steps):
            ags.ags_render(ctx, scene, spec, poses_d[(warmup + i) % walk], depth, seg, stream)
        en.record(stream)
        torch.cuda.synchronize()
    ags.ags_stream_status(ctx, stream)
    return st.elapsed_time(en) / steps, dict(clk.summary(), timed_steps=steps)


def forest_record(ags, ctx, dev, stream, steps, warmup, envs=64, cells=64, check_rays=256):
    """A bounded run of the LiDAR-forest workload: 64 forests (50-200 trees of 2k-10k triangles), the 64x512
    LiDAR, references split at a fixed 64 cells (the forest setting the build tuner keeps; no tuning here),
    the default launch shape, and a sample of beams checked against the FP64 oracle."""
    import torch

    import oracle as O
    from paper_2503_01471_gb300 import scenes as S
    batch, spec, poses = S.lidar_forests(envs, steps=max(steps + warmup, 4))
    t0 = time.perf_counter()
    scene = ags.ags_scene_build(ctx, batch, ags.AGS_SPLIT_CELLS(cells))
    build_s = time.perf_counter() - t0
    try:
        poses_d = torch.as_tensor(poses).to(dev)
        E = batch.n_envs
        depth = torch.empty((E, spec.height, spec.width), device=dev)
        seg = torch.empty((E, spec.height, spec.width), dtype=torch.int32, device=dev)
        ms, clocks = timed_renders(ags, ctx, scene, spec, poses_d, depth, seg, stream, steps, warmup)
        r_c, n_c, t_c = ags.ags_render_count(ctx, scene, spec, poses_d[0])
        ags.ags_render(ctx, scene, spec, poses_d[0], depth, seg, stream)
        ags.ags_stream_status(ctx, stream)
        d, g = depth.cpu().numpy(), seg.cpu().numpy()
        s_or = O.Sensor(type=1, width=spec.width, height=spec.height, hfov=float(np.float32(spec.hfov)),
                        min_range=float(np.float32(spec.min_range)), max_range=float(np.float32(spec.max_range)),
                        vfov_min=float(np.float32(spec.vfov_min)), vfov_max=float(np.float32(spec.vfov_max)))
        rng = np.random.default_rng(13)
        n_ok = n_cnt = 0
        for e in (0, E - 1):
            vs, ix, ps, sg = batch.env_submeshes(e)
            tris, tseg = O.world_triangles(vs, ix, ps, sg)
            rr = np.sort(rng.choice(spec.width * spec.height, check_rays // 2, replace=False)).astype(np.int64)
            res = O.render(tris, tseg, s_or, poses[0][e].astype(np.float64), rr)
            ok, cnt = O.check(res, d[e].reshape(-1)[rr], g[e].reshape(-1)[rr], s_or.max_range)
            if not ok.all():
                raise RuntimeError(f"forest record: env {e}: {int((~ok).sum())} beams outside the oracle's outcomes")
            n_ok += int(ok.sum())
            n_cnt += int(cnt.sum())
        rays = E * spec.width * spec.height
        return {"workload": f"LiDAR forests, {E} envs (50-200 trees of 2k-10k triangles), 64x512 LiDAR, "
                            f"references split at {cells} cells",
                "mrays_per_s": rays / ms / 1e3, "ms_per_step": ms, "steps": clocks.get("timed_steps", steps),
                "warmup": warmup,
                "tris": int(batch.env_tri_counts().sum()), "bvh_bytes": ags.ags_scene_stats(scene)[2],
                "build_ms": build_s * 1e3, "nodes_per_ray": n_c / r_c, "tris_per_ray": t_c / r_c,
                "bytes_per_ray": (n_c * ags.ags_scene_node_bytes(scene) + t_c * 48) / r_c + 8.0,
                "launch_config": ags.ags_get_launch_config(ctx, scene, spec), "clocks": clocks,
                "oracle_check": {"beams": n_ok, "counted": n_cnt, "envs": [0, E - 1],
                                 "rule": "uncounted beams within 1e-5*d + 1e-6 m of the FP64 range, exact segment"}}
    finally:
        ags.ags_scene_destroy(scene)


def precision_record(ags, ctx, dev, stream, batch, spec, poses, poses_d, steps, warmup, n_envs_checked=48,
                     rays_per_env=256):
    """Node formats on the benchmark's own scene: float32, float16 and 8-bit child bounds (rounded outward),
    each timed at the benchmark's sensor shape and compared bit for bit with float32; and the depth error of
    the (common) output against the FP64 oracle on a sample of rays."""
    import torch

    import oracle as O
    E = batch.n_envs
    depth = torch.empty((E, spec.height, spec.width), device=dev)
    seg = torch.empty((E, spec.height, spec.width), dtype=torch.int32, device=dev)
    out, ref = {}, None
    for name, flag in (("fp32", 0), ("fp16", ags.AGS_BVH_FP16), ("q8", ags.AGS_BVH_Q8)):
        scene = ags.ags_scene_build(ctx, batch, flag)
        try:
            ms, clocks = timed_renders(ags, ctx, scene, spec, poses_d, depth, seg, stream, steps, warmup)
            ags.ags_render(ctx, scene, spec, poses_d[0], depth, seg, stream)
            ags.ags_stream_status(ctx, stream)
            o = (depth.cpu().numpy(), seg.cpu().numpy())
            if ref is None:
                ref = o
            out[name] = {"mrays_per_s": E * spec.width * spec.height / ms / 1e3, "ms_per_step": ms,
                         "node_bytes": ags.ags_scene_node_bytes(scene), "bvh_bytes": ags.ags_scene_stats(scene)[2],
                         "bit_identical_to_fp32": bool(np.array_equal(o[0], ref[0]) and np.array_equal(o[1], ref[1])),
                         "clocks_sm_mhz": clocks.get("sm_mhz")}
        finally:
            ags.ags_scene_destroy(scene)
    s_or = O.Sensor(type=0, width=spec.width, height=spec.height, hfov=float(np.float32(spec.hfov)),
                    min_range=float(np.float32(spec.min_range)), max_range=float(np.float32(spec.max_range)))
    rng = np.random.default_rng(17)
    abs_e, rel_e, n_s, counted = [], [], 0, 0
    for e in rng.choice(E, min(E, n_envs_checked), replace=False):
        vs, ix, ps, sg = batch.env_submeshes(int(e))
        tris, tseg = O.world_triangles(vs, ix, ps, sg)
        rr = np.sort(rng.choice(spec.width * spec.height, rays_per_env, replace=False)).astype(np.int64)
        res = O.render(tris, tseg, s_or, poses[0][e].astype(np.float64), rr)
        d = ref[0][e].reshape(-1)[rr].astype(np.float64)
        g = ref[1][e].reshape(-1)[rr]
        ok, cnt = O.check(res, d, g, s_or.max_range)
        if not ok.all():
            raise RuntimeError(f"precision record: env {e}: {int((~ok).sum())} rays outside the oracle's outcomes")
        hit = (~cnt) & (res["seg"] >= 0)
        abs_e.append(np.abs(d - res["v"])[hit])
        rel_e.append((np.abs(d - res["v"]) / res["v"])[hit])
        counted += int(cnt.sum())
        n_s += rr.shape[0]
    a, r = np.concatenate(abs_e), np.concatenate(rel_e)
    return {"workload": f"the benchmark scene ({E} obstacle rooms, {spec.height}x{spec.width} camera) per node format",
            "formats": out,
            "depth_error_vs_fp64": {"sampled_rays": n_s, "single_outcome_hits": int(a.shape[0]), "counted": counted,
                                    "max_abs_m": float(a.max()), "p999_abs_m": float(np.percentile(a, 99.9)),
                                    "max_rel": float(r.max()), "p999_rel": float(np.percentile(r, 99.9)),
                                    "tolerance": "1e-5*d + 1e-6 m (every uncounted ray within it)"}}


# ---------------------------------------------------------------- workload
def make_workload(args, rank, world=1):
    from paper_2503_01471_gb300 import scenes as S
    from paper_2503_01471_gb300 import shard
    envs = shard.weak_shard(args.envs, rank, max(world, rank + 1))
    ids = list(envs) if rank else None
    if args.workload == "forest":
        return S.lidar_forests(args.envs, steps=args.walk, envs=ids)
    return S.obstacle_rooms(args.envs, steps=args.walk, width=args.width, height=args.height, envs=ids)


def workload_name(args, spec, E):
    if args.workload == "forest":
        return f"LiDAR forests, {E} envs (50-200 trees of 2k-10k triangles), {spec.height}x{spec.width} LiDAR"
    return f"obstacle rooms, {E} envs x {spec.height}x{spec.width} depth+seg camera"


def bench_reference(args, rank, world):
    if rank != 0:
        return
    batch, spec, poses = make_workload(args, 0)
    E = batch.n_envs
    rays_per_step = 1024
    times = []
    for it in range(args.warmup + args.steps):
        e = (it * 131) % E
        n, dt, cores = run_oracle(batch, spec, poses[it % poses.shape[0]], [e], rays_per_step, seed=it)
        if it >= args.warmup:
            times.append((n, dt, run_oracle.last_tests))
    n_tot = sum(t[0] for t in times)
    t_tot = sum(t[1] for t in times)
    value = n_tot / t_tot / 1e6
    line = {
        "impl": "reference", "metric": WORKLOADS[args.workload]["metric"], "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args, spec, E), "envs": E, "width": spec.width, "height": spec.height},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: {rays_per_step} random rays of one env (env cycles), FP64 brute "
                                   f"force over every triangle",
                         "ray_tri_tests_per_s": sum(t[2] for t in times) / t_tot,
                         "full_step_s_extrapolated": E * spec.width * spec.height * t_tot / n_tot},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_ours(args, rank, world, local):
    import torch

    import paper_2503_01471_gb300 as ags
    from paper_2503_01471_gb300 import build as B

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    batch, spec, poses = make_workload(args, rank, world)
    E = batch.n_envs
    ctx = ags.ags_context_create(local)
    t0 = time.perf_counter()
    scene = ags.ags_scene_build(ctx, batch, args.build_flags)
    build_s = time.perf_counter() - t0
    n_tris = int(batch.env_tri_counts().sum())
    poses_d = torch.as_tensor(poses).to(dev)  # [walk, E, 7]
    depth = torch.empty((E, spec.height, spec.width), dtype=torch.float32, device=dev)
    seg = torch.empty((E, spec.height, spec.width), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rays_per_step = E * spec.width * spec.height
    walk = poses_d.shape[0]

    def step(i):
        ags.ags_render(ctx, scene, spec, poses_d[i % walk], depth, seg, stream)

    tuned = None
    split_cells = (args.build_flags >> 12) & 0xFF
    cluster_radius = 16 << ((args.build_flags >> 23) & 3)
    leaf_size = (args.build_flags >> 8) & 0xF or 2
    if not args.no_autotune:  # untimed set-up, like the scene build
        if args.workload == "forest":
            # long LiDAR rays through dense trees gain from finer reference splitting and a wider clustering
            # search; rooms keep the defaults
            split_cells = ags.ags_autotune_build(ctx, scene, spec, poses_d[0], depth, seg, (16, 32, 48, 64), 2)
            base = (args.build_flags & ~(0xFF << 12) & ~ags.AGS_CLUSTER_RADIUS(128)) | ags.AGS_SPLIT_CELLS(split_cells)
            cands = [base | ags.AGS_CLUSTER_RADIUS(r) for r in (32, 64)]
            cands += [base | ags.AGS_LEAF_SIZE(1) | ags.AGS_CLUSTER_RADIUS(r) for r in (16, 64)]
            best = ags.ags_autotune_build_flags(ctx, scene, spec, poses_d[0], depth, seg, cands, 3)
            cluster_radius = 16 << ((best >> 23) & 3)
            leaf_size = (best >> 8) & 0xF or 2
        tuned = ags.ags_autotune(ctx, scene, spec, poses_d[0], depth, seg, 2).as_dict()
    for i in range(args.warmup):
        step(i)
    ags.ags_stream_status(ctx, stream)

    # algorithmic bytes per ray (instrumented traversal, untimed)
    rays_c, nodes_c, tris_c = ags.ags_render_count(ctx, scene, spec, poses_d[0])
    node_b = ags.ags_scene_node_bytes(scene)
    b_ray = (nodes_c * node_b + tris_c * 48) / rays_c + 8.0 + 28.0 / (spec.width * spec.height)

    def timed_steps():
        """K steps between barriers and device syncs, CUDA events on the render stream, clocks sampled."""
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(torch.cuda.current_device()) as clk:
            start.record(stream)
            for i in range(args.steps):
                step(args.warmup + i)
            stop.record(stream)
            torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        ags.ags_stream_status(ctx, stream)
        ms = start.elapsed_time(stop)
        if dist is not None:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, clk.summary()

    ms, clocks = timed_steps()
    start = torch.cuda.Event(enable_timing=True)  # for the plain-launch and step-graph timings below
    stop = torch.cuda.Event(enable_timing=True)
    first_clocks = None
    bad = clocks_rejected(clocks)
    if dist is not None:
        f = torch.tensor([1.0 if bad else 0.0], device=dev)
        dist.all_reduce(f, op=dist.ReduceOp.MAX)
        bad = f.item() > 0
    if bad:  # a throttled or clock-locked run is measured once more
        first_clocks = clocks
        ms, clocks = timed_steps()
    ms_step = ms / args.steps
    value = rays_per_step * world / (ms_step * 1e-3) / 1e6

    # end to end through the C ABI with host buffers: pinned poses in, depth+seg out
    pin_pose = torch.empty((E, 7), dtype=torch.float32).pin_memory()
    pin_depth = torch.empty((E, spec.height, spec.width), dtype=torch.float32).pin_memory()
    pin_seg = torch.empty((E, spec.height, spec.width), dtype=torch.int32).pin_memory()
    host_poses = poses
    pin_pose.numpy()[:] = host_poses[0]
    ags.ags_render_host(ctx, scene, spec, pin_pose.numpy(), pin_depth.numpy(), pin_seg.numpy())  # warm staging
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.e2e_steps):
        pin_pose.numpy()[:] = host_poses[i % walk]
        ags.ags_render_host(ctx, scene, spec, pin_pose.numpy(), pin_depth.numpy(), pin_seg.numpy())
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    if dist is not None:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": rays_per_step * world / e2e_s / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": E * 7 * 4, "d2h_bytes_per_step": 2 * E * spec.width * spec.height * 4,
           "api": "ags_render_host (page-locked host buffers: poses copied in, the kernel writes depth+seg in place "
                  "over the host link; synchronous)"}

    # plain per-env launches (one ags_render_envs call per environment), same outputs
    plain = None
    if not args.no_plain:
        ids = torch.arange(E, dtype=torch.int32, device=dev)
        npix = spec.width * spec.height

        def plain_step(i):
            p = poses_d[i % walk]
            for e in range(E):
                ags.ags_render_envs(ctx, scene, spec, ids[e:e + 1], p[e:e + 1], depth[e:e + 1], seg[e:e + 1],
                                    stream)

        plain_step(0)
        torch.cuda.synchronize(dev)
        ps = max(1, min(3, args.steps))
        start.record(stream)
        for i in range(ps):
            plain_step(i)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        pms = start.elapsed_time(stop) / ps
        ags.ags_stream_status(ctx, stream)
        plain = {"value": rays_per_step * world / (pms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": pms,
                 "launches_per_step": E, "speedup_of_batched": (rays_per_step / (ms_step * 1e-3)) /
                 (rays_per_step / (pms * 1e-3))}

    # the same step loop replayed from a captured CUDA graph (poses refreshed in a fixed buffer)
    graph_pose = poses_d[0].clone()
    g = ags.ags_render_graph_create(ctx, scene, spec, graph_pose, depth, seg)
    try:
        for i in range(args.warmup):
            graph_pose.copy_(poses_d[i % walk])
            ags.ags_render_graph_launch(g, stream)
        torch.cuda.synchronize(dev)
        start.record(stream)
        for i in range(args.steps):
            graph_pose.copy_(poses_d[(args.warmup + i) % walk])
            ags.ags_render_graph_launch(g, stream)
        stop.record(stream)
        torch.cuda.synchronize(dev)
        gms = start.elapsed_time(stop) / args.steps
        ags.ags_stream_status(ctx, stream)
    finally:
        ags.ags_render_graph_destroy(g)
    step_graph = {"value": rays_per_step * world / (gms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": gms,
                  "api": "ags_render_graph_launch (tile-counter reset + k_trace captured once)"}

    hbm, peak_kind = peaks()
    workload = workload_name(args, spec, E)
    lc = ags.ags_get_launch_config(ctx, scene, spec)
    fmt = args.build_flags & 0xFF
    counters = profiled_counters(f"{args.workload}:{E}x{spec.height}x{spec.width}:cells{split_cells or 16}",
                                 f"k_trace<0, {lc['tile_w']}, {lc['rays_per_lane']}, 0, {fmt}, 0>")
    sm_count = ags.ags_context_device(ctx)["sm_count"]
    lead, algorithmic = rooflines(counters, ms_step, b_ray, rays_per_step, hbm, peak_kind, sm_count,
                                  sm_max_mhz(clocks), nodes_c / rays_c, tris_c / rays_c, node_b)
    line = {
        "metric": WORKLOADS[args.workload]["metric"], "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_MRAYS if (args.workload == "rooms" and E == 1024 and spec.width == 480
                                                and spec.height == 270) else None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "envs_per_gpu": E, "width": spec.width, "height": spec.height,
                   "tris_per_gpu": n_tris, "rays_per_step": rays_per_step * world, "walk_steps": walk,
                   "l2": "not flushed: per step the resident BVHs and the outputs exceed the 129 MB L2",
                   "bvh_bytes": ags.ags_scene_stats(scene)[2], "build_flags": args.build_flags,
                   "split_cells": split_cells or 16, "cluster_radius": cluster_radius, "leaf_size": leaf_size,
                   "parallelism": f"env-sharded x{world}, no collective on the data path"},
        "roofline": lead,
        "roofline_hbm_algorithmic": algorithmic,
        "clocks": clocks if first_clocks is None else dict(clocks, first_run_rejected=first_clocks),
        "e2e": e2e,
        "gpu_launches": args.steps,
        "launch_config": ags.ags_get_launch_config(ctx, scene, spec), "autotuned": tuned is not None,
        "build_ms": build_s * 1e3,
        "build_mtris_per_s": n_tris / build_s / 1e6,
    }
    line["step_graph"] = step_graph
    if plain is not None:
        line["plain"] = plain
    if args.workload == "rooms" and not args.no_serving:
        # served latency on the same resident scene, mixed camera and LiDAR requests
        line["serving"] = serving_measure(ags, ctx, scene, E, poses[0], serving_specs())
        line["serving"]["without_graph"] = serving_measure(ags, ctx, scene, E, poses[0], serving_specs(),
                                                           use_graph=False, sequential=False)
    if args.workload == "rooms" and not args.no_sub_records and rank == 0:
        # the other workloads' figures in the same run: a bounded LiDAR-forest run and the node formats
        sub_steps = max(3, min(args.steps, 10))
        line["forest"] = forest_record(ags, ctx, dev, stream, sub_steps, 3)
        line["precision"] = precision_record(ags, ctx, dev, stream, batch, spec, poses, poses_d, sub_steps, 3)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(batch, spec, poses)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ags.ags_scene_destroy(scene)
    ags.ags_context_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        bench_reference(args, rank, world)
        return
    if args.workload == "serving":
        if rank == 0:
            bench_serving(args, rank, world, local)
        return
    if args.workload == "precision":
        if rank == 0:
            bench_precision(args, rank, world, local)
        return
    if args.workload == "dynamic":
        if rank == 0:
            bench_dynamic(args, rank, world, local)
        return
    if args.workload == "features":
        if rank == 0:
            bench_features(args, rank, world, local)
        return
    bench_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
