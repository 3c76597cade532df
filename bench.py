"""Benchmark: frames/s of the fisheye variational stereo path on GB300.

Workload (default): one 1024 x 1024 Kannala-Brandt fisheye pair (f = 320 px,
190 deg FOV, k1..k4 seeded in +-0.05), 0.12 m baseline plus a seeded rotation
<= 2 deg, 20 textured planes/spheres at 0.5-20 m, noise sigma 0.01; 5 pyramid
levels, 10 warps x 100 primal-dual iterations per level, FP32.  A step is one
whole frame: pre-rotation, pyramids, per-level tensor, warps, primal-dual
iterations, clip/update, upsampling and triangulation.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Multi-GPU runs are independent replicas (one pair per rank, no collective on
the data path).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s & p99 latency, 1024² fisheye pair; primal-dual Gpix-iter/s vs plain"
PD_BYTES_PER_PX_ITER = 52.0   # unblocked FP32 traffic of one pixel-iteration (9 reads + 4 writes)
# DRAM bytes (read + write) of one level-0 k_pd launch of this workload on
# 64 x 64 footprints of 1024 threads at 7 iterations per launch (schedule
# choice 31), from one ncu capture of the current kernel (cold L2; the
# command and figures are in profiles/k_pd_level0_kb1024.md)
PD_L0_DRAM_BYTES_PER_LAUNCH = 47.7e6
PD_L0_PROFILED_CHOICE = 31
FOOTPRINTS = ["64x64 footprints, 512 threads", "32x32 footprints, 256 threads",
              "64x32 footprints", "64x64 footprints, 1024 threads",
              "32x32 footprints, 1024 threads", "32x32 footprints, 512 threads"]


def schedule_label(c):
    """fs_autotune's per-level choice in words (0 = cluster; 1..48 = depth
    1..8 on each of the six footprints; 49..55 = depth 9..15 on 32x32
    footprints of 1024 threads)."""
    if c == 0:
        return "cluster"
    if c > 8 * len(FOOTPRINTS):           # depths 9..15 on the 1024-thread 32x32 footprint
        return f"blocking x{c - 8 * len(FOOTPRINTS) + 8} ({FOOTPRINTS[4]})"
    return f"blocking x{(c - 1) % 8 + 1} ({FOOTPRINTS[(c - 1) // 8]})"


def workload_pair(name, seed):
    import synth
    if name == "plain_kb_1024":
        return synth.plain_kb(seed)
    if name == "plain_small_256":
        return synth.plain_small(seed)
    raise SystemExit(f"unknown workload {name}")


def level_pixels(W, H, levels):
    import oracle
    return [w * h for w, h in oracle.level_sizes(W, H, levels)]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank values over all ranks (replicas time
    the same number of steps; the job is as slow as its slowest rank)."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_rate(world, steps, max_ms):
    """Whole-job frames/s: every rank solves `steps` frames of its own pair."""
    return world * steps / (max_ms / 1000.0)


def replica_seed(seed, rank):
    """Each replica solves its own seeded pair (no data is shared)."""
    return seed + rank


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def l2_probe_gbs(stream, reps=50):
    """L2-resident copy bandwidth: an elementwise add over 32 MB in and 32 MB
    out (64 MB, inside the 129 MB L2), timed with CUDA events after warm-up.
    The measured HBM peak file has no L2 figure, so the bench measures one."""
    import torch
    n = 8 * 1024 * 1024
    with torch.cuda.stream(stream):
        x = torch.rand(n, device="cuda")
        y = torch.empty_like(x)
        for _ in range(5):
            torch.add(x, 1.0, out=y)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            torch.add(x, 1.0, out=y)
        e1.record(stream)
        stream.synchronize()
    return 2 * n * 4 * reps / (e0.elapsed_time(e1) / 1000.0) / 1e9


def cpu_baseline(pair, target_s=15.0):
    """The FP64 oracle on a bounded sample of the same frame: the finest
    level's primal-dual iterations of one warp, extrapolated per pixel-iteration."""
    import oracle
    from oracle.solve import level_data
    prm = oracle.Params(lam=pair["lam"], eps=pair["eps"])
    cam = oracle.calib_from_dict(pair["cam0"])
    H, W = pair["I0"].shape
    M = oracle.fov_mask(cam, W, H)
    lv = level_data(pair["I0"], M, prm)
    rng = np.random.default_rng(0)
    st = dict(u=np.zeros((H, W)), ubar=np.zeros((H, W)), p1=np.zeros((H, W)),
              p2=np.zeros((H, W)), Iu=np.where(M, rng.uniform(-0.1, 0.1, (H, W)), 0.0),
              rho0=np.where(M, rng.uniform(-0.05, 0.05, (H, W)), 0.0), u_w=np.zeros((H, W)))
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.pd_iteration(st, lv, prm)
        n += 1
        if time.perf_counter() - t0 > target_s:
            break
    dt = time.perf_counter() - t0
    return n * W * H / dt, n, dt


def render_rigs(seed, n_rigs=16, n_frames=3):
    """The serving workload's rigs: sizes drawn from 640 / 1024 / 1280 px,
    each its own seeded Kannala-Brandt calibration, relative pose and scene,
    n_frames consecutive frames of its smooth path."""
    import synth
    rng = np.random.default_rng(1000 + seed)
    sizes = [int(v) for v in rng.choice([640, 1024, 1280], size=n_rigs)]
    t0 = time.perf_counter()
    rigs = [synth.rig_sequence(10000 * (seed + 1) + i, W, W, n_frames=n_frames)
            for i, W in enumerate(sizes)]
    return rigs, sizes, time.perf_counter() - t0


def serve_leg(rigs, sizes, seed, seconds, rate, inflight, warm_mode=1, storage="f32"):
    """Serving: Poisson arrivals from the rigs through one fs_server; each
    rig's frames warm-start from its previous result (3 warps x 50
    iterations on the finest level, continuing from the last u and w for
    warm_mode 1, from the last disparity for 0; a rig's first frame is a
    cold 10 x 100 solve over its pyramid).  Each rig's frames are replayed
    forwards and backwards (0, 1, 2, 1, 0, ...) so the motion stays smooth.
    Returns the open-loop figures at the offered rate and the saturated
    throughput (every rig's queue kept full)."""
    import queue

    import torch

    from paper_1909_07545_gb300 import Server
    n_rigs, n_frames = len(rigs), len(rigs[0]["frames"])
    rng = np.random.default_rng(2000 + seed)
    srv = Server(budget_bytes=40 << 30, max_inflight=inflight, warps=3, iters=50,
                 cold_warps=10, cold_iters=100, warm_mode=warm_mode)
    ids = []
    frames = []
    outs = []
    ring = 4                           # result buffers per rig
    for q, W in zip(rigs, sizes):
        ids.append(srv.add_rig(q["cam0"], q["cam1"], q["R"], q["t"], W, W, q["levels"],
                               lam=q["lam"], huber_eps=q["eps"], storage=storage))
        frames.append([(torch.from_numpy(np.float32(a)).pin_memory(),
                        torch.from_numpy(np.float32(b)).pin_memory()) for a, b, _ in q["frames"]])
        outs.append([(torch.empty((W, W)).pin_memory(), torch.empty((W, W)).pin_memory())
                     for _ in range(ring)])
    cycle = list(range(n_frames)) + list(range(n_frames - 2, 0, -1))
    pos = [0] * n_rigs
    free = [queue.Queue() for _ in range(n_rigs)]
    for r in range(n_rigs):
        for k in range(ring):
            free[r].put(k)

    def submit(r):
        slot = free[r].get()
        I0, I1 = frames[r][cycle[pos[r] % len(cycle)]]
        pos[r] += 1
        d, z = outs[r][slot]
        return srv.submit(ids[r], I0, I1, d, z), r, slot

    done_q = queue.Queue()

    def waiter():
        while True:
            item = done_q.get()
            if item is None:
                return
            req, r, slot = item
            srv.wait(req)
            free[r].put(slot)

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    # warm-up: every rig's cold first frame, then two warm frames each
    for _ in range(3):
        for r in range(n_rigs):
            done_q.put(submit(r))
    srv.drain()
    srv.stats(reset=True)

    # open loop at the offered rate
    arr = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * seconds * 1.2) + 16))
    arr = arr[arr < seconds]
    which = rng.integers(0, n_rigs, size=len(arr))
    start = time.perf_counter()
    stalls = 0
    for ta, r in zip(arr, which):
        now = time.perf_counter() - start
        if ta > now:
            time.sleep(ta - now)
        if free[int(r)].empty():
            stalls += 1
        done_q.put(submit(int(r)))
    srv.drain()
    open_loop = srv.stats(reset=True)

    # saturated: keep every rig's ring full for a fixed number of requests
    n_sat = 8 * n_rigs
    t1 = time.perf_counter()
    for i in range(n_sat):
        done_q.put(submit(i % n_rigs))
    srv.drain()
    sat = srv.stats(reset=True)
    sat_wall = time.perf_counter() - t1
    done_q.put(None)
    th.join()
    srv.close()
    px = {W: W * W for W in set(sizes)}
    mean_px = float(np.mean([px[W] for W in sizes]))
    return {
        "workload": f"{n_rigs} rigs (sizes {sorted(set(sizes))}: "
                    f"{[sizes.count(v) for v in sorted(set(sizes))]}), Kannala-Brandt 190 deg, "
                    f"warm start 3x50 on the finest level "
                    f"({'from the last u and w' if warm_mode == 1 else 'from the last disparity'}), "
                    f"{storage} storage",
        "offered_per_s": rate, "seconds": seconds, "max_inflight": inflight,
        "requests": int(open_loop["completed"]), "failed": int(open_loop["failed"]),
        "frames_per_s": open_loop["frames_per_s"], "p50_ms": open_loop["p50_ms"],
        "p99_ms": open_loop["p99_ms"], "max_ms": open_loop["max_ms"],
        "mean_ms": open_loop["mean_ms"], "submit_stalls": stalls,
        "cold": int(open_loop["cold"]), "evictions": int(open_loop["evictions"]),
        "resident_gb": open_loop["resident_bytes"] / 1e9,
        "saturated_frames_per_s": sat["frames_per_s"], "saturated_requests": n_sat,
        "saturated_wall_s": sat_wall,
        "gpix_iter_s_at_offered": open_loop["frames_per_s"] * mean_px * 150 / 1e9,
    }


def uneven_batch_leg(seed, stream, steps, warmup, storage="f16", per_size=16,
                     sizes=(512, 800, 1024, 1280)):
    """Batching: per_size pairs of each size, every pair its own seeded
    Kannala-Brandt calibration, relative pose and scene (the 1024 generator
    scaled), 4-6 pyramid levels (level count: coarsest level >= 40 px),
    10 warps x 100 iterations, 16-bit storage, each handle autotuned, all
    pairs in one fs_batch graph.  Returns frames/s per finest-level bound."""
    import torch

    import synth
    from paper_1909_07545_gb300 import Batch, Solver
    t0 = time.perf_counter()
    pairs = []
    for j, W in enumerate(sizes):
        for i in range(per_size):
            pairs.append(synth.plain_kb(100000 * (seed + 1) + 1000 * j + i, W=W, H=W,
                                        supersample=1, levels=synth.auto_levels(W)))
    render_s = time.perf_counter() - t0
    sols, I0s, I1s = [], [], []
    for p in pairs:
        W = p["I0"].shape[1]
        x = Solver(p["cam0"], p["cam1"], p["R"], p["t"], W, W, p["levels"], stream=stream,
                   lam=p["lam"], huber_eps=p["eps"], use_graph=1, storage=storage)
        x.autotune(p["iters"])
        sols.append(x)
        I0s.append(torch.as_tensor(np.float32(p["I0"]), device="cuda"))
        I1s.append(torch.as_tensor(np.float32(p["I1"]), device="cuda"))
    bt = Batch(sols, stream=stream)
    outs_d = [torch.empty_like(a) for a in I0s]
    outs_z = [torch.empty_like(a) for a in I0s]
    res = {}
    for k in (0, 1, 2, 4):
        bt.set_finest_limit(k)
        run = lambda: bt.solve(I0s, I1s, 10, 100, disps=outs_d, depths=outs_z)
        for _ in range(warmup):
            run()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            run()
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[f"finest{k}"] = {"frames_per_s": len(pairs) * 1000.0 / ms, "ms_per_batch": ms}
    bt.close()
    for x in sols:
        x.close()
    px_iter = sum(sum(level_pixels(p["I0"].shape[1], p["I0"].shape[0], p["levels"])) * 1000
                  for p in pairs)
    best = max(r["frames_per_s"] for r in res.values())
    return {"workload": f"{len(pairs)} pairs, {per_size} each of {list(sizes)} px, "
                        f"Kannala-Brandt 190 deg, own calibration and pose each, "
                        f"4-6 levels x 10 warps x 100 iterations, {storage} storage, one graph",
            "by_finest_limit": res, "best_frames_per_s": best,
            "gpix_iter_s_best": px_iter * best / len(pairs) / 1e9, "render_s": render_s}


def run_reference(args, pair, rank):
    """--impl reference: the FP64 oracle on the host cores, per step a bounded
    sample of the frame (primal-dual iterations of the finest level)."""
    import oracle
    from oracle.solve import level_data
    if rank != 0:
        return
    prm = oracle.Params(lam=pair["lam"], eps=pair["eps"])
    cam = oracle.calib_from_dict(pair["cam0"])
    H, W = pair["I0"].shape
    M = oracle.fov_mask(cam, W, H)
    lv = level_data(pair["I0"], M, prm)
    st = dict(u=np.zeros((H, W)), ubar=np.zeros((H, W)), p1=np.zeros((H, W)),
              p2=np.zeros((H, W)), Iu=np.where(M, 0.05, 0.0), rho0=np.where(M, 0.01, 0.0),
              u_w=np.zeros((H, W)))
    per_step = 5
    for _ in range(args.warmup):
        for _ in range(per_step):
            oracle.pd_iteration(st, lv, prm)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            oracle.pd_iteration(st, lv, prm)
        times.append(time.perf_counter() - t0)
    pxit_frame = sum(level_pixels(W, H, pair["levels"])) * pair["warps"] * pair["iters"]
    rate = per_step * W * H / float(np.mean(times))      # px-iter/s
    fps = rate / pxit_frame
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 / fps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": pair["name"], "W": W, "H": H, "levels": pair["levels"],
                   "warps": pair["warps"], "iters": pair["iters"]},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": 1,
                         "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{per_step} primal-dual iterations of the finest "
                                   f"{W}x{H} level per step, extrapolated to a frame by "
                                   f"pixel-iterations ({pxit_frame:.3e} per frame)"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpix_iter_s": rate / 1e9,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="plain_kb_1024")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--block-iters", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip fs_autotune (default schedule per level)")
    ap.add_argument("--batch", type=int, default=4,
                    help="pairs per fs_batch for the batched-throughput figure (<= 1 skips)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the open-loop serving run (0 skips serving)")
    ap.add_argument("--serve-rate", type=float, default=600.0, help="offered requests/s")
    ap.add_argument("--serve-inflight", type=int, default=8)
    ap.add_argument("--serve-warm-mode", type=int, default=1, choices=[0, 1])
    ap.add_argument("--uneven-batch", action="store_true",
                    help="also time 64 pairs of 512/800/1024/1280 px in one batch graph")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        if rank == 0:
            run_reference(args, workload_pair(args.workload, args.seed), rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1909_07545_gb300 import Solver

    pair = workload_pair(args.workload, replica_seed(args.seed, rank))
    H, W = pair["I0"].shape
    L, warps, iters = pair["levels"], pair["warps"], pair["iters"]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = Solver(pair["cam0"], pair["cam1"], pair["R"], pair["t"], W, H, L, stream=stream,
                   lam=pair["lam"], huber_eps=pair["eps"], use_graph=1,
                   block_iters=args.block_iters)
        tuned = s.autotune(iters) if args.autotune else None
        # pixels inside each level's FOV mask (the pixels the method moves)
        mask_px = [int((s.read(l, "MASK") > 0.5).sum().item()) for l in range(L)]
        I0 = torch.as_tensor(np.float32(pair["I0"]), device="cuda")
        I1 = torch.as_tensor(np.float32(pair["I1"]), device="cuda")
        disp = torch.empty((H, W), device="cuda")
        depth = torch.empty((H, W), device="cuda")
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
        stream.synchronize()

        def step():
            s.solve(I0, I1, warps, iters, disp=disp, depth=depth)

        for _ in range(args.warmup):
            step()
        stream.synchronize()

        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        clocks = ClockSampler(local)
        clocks.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))                      # evict the frame's working set from L2
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t_wall = time.perf_counter() - t_wall
        clk = clocks.stop()
        step_ms = np.array([a.elapsed_time(b) for a, b in ev])
        total_ms, = reduce_max([float(step_ms.sum())], dist, "cuda")

        # primal-dual kernel timing (CUDA events around each warp's launches,
        # recorded by the library on this stream) over the same number of steps
        s.timing_enable(True)
        step()
        stream.synchronize()
        s.timing_read(reset=True)
        for i in range(args.steps):
            flush.fill_(float(i))
            step()
            s.timing_read(reset=False)
        per_level = s.timing_read(reset=True)
        s.timing_enable(False)

        # end to end through the host entry point (pinned buffers, copies inside)
        hI0 = torch.as_tensor(np.float32(pair["I0"])).pin_memory()
        hI1 = torch.as_tensor(np.float32(pair["I1"])).pin_memory()
        hD = torch.empty((H, W), dtype=torch.float32).pin_memory()
        hZ = torch.empty((H, W), dtype=torch.float32).pin_memory()
        s.solve_host(hI0, hI1, warps, iters, disp=hD, depth=hZ)
        e2e_steps = max(10, min(args.steps, 20))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            s.solve_host(hI0, hI1, warps, iters, disp=hD, depth=hZ)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        e2e_s, = reduce_max([e2e_s], dist, "cuda")
        pd_launches = sum(n for _, n, _ in per_level) // max(args.steps, 1)
        l2_gbs = l2_probe_gbs(stream)

        # a per-frame pose change: fs_set_pose recomputes the calibration field
        # (FP64 on host threads from the cached rays) and the trajectory fields
        s.set_pose(pair["R"], pair["t"])
        stream.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            s.set_pose(pair["R"], pair["t"])
        stream.synchronize()
        set_pose_ms = (time.perf_counter() - t0) / 5 * 1000.0
        s.close()

        # variants of the same frame: 16-bit storage, and batches of
        # independent handles solved concurrently through one fs_batch graph
        def timed(run, n):
            for _ in range(args.warmup):
                run()
            stream.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(n)]
            for i in range(n):
                flush.fill_(float(i))
                evs[i][0].record(stream)
                run()
                evs[i][1].record(stream)
            stream.synchronize()
            ms, = reduce_max([float(sum(a.elapsed_time(b) for a, b in evs))], dist, "cuda")
            return ms / n

        def make(storage):
            x = Solver(pair["cam0"], pair["cam1"], pair["R"], pair["t"], W, H, L, stream=stream,
                       lam=pair["lam"], huber_eps=pair["eps"], use_graph=1, storage=storage)
            if args.autotune:
                x.autotune(iters)
            return x

        variants = {}
        vsteps = max(3, min(args.steps, 10))
        for storage in ("f16", "bf16"):
            x = make(storage)
            run = lambda: x.solve(I0, I1, warps, iters, disp=disp, depth=depth)
            ms = timed(run, vsteps)
            x.timing_enable(True)
            run()
            stream.synchronize()
            x.timing_read(reset=True)
            for i in range(vsteps):
                flush.fill_(float(i))
                run()
                x.timing_read(reset=False)
            lv = x.timing_read(reset=True)
            variants[storage] = {"value": job_rate(world, 1, ms), "unit": "frames/s",
                                 "ms_per_frame": ms,
                                 "pd_per_level_ms": [m / vsteps for m, _, _ in lv]}
            x.close()
        # the paper's own regulariser, TGV-L1 (Eq. 10-11): same frame, FP32
        x = Solver(pair["cam0"], pair["cam1"], pair["R"], pair["t"], W, H, L, stream=stream,
                   lam=pair["lam"], huber_eps=pair["eps"], use_graph=1, regularizer="tgv")
        tgv_sched = x.autotune(iters) if args.autotune else None
        ms = timed(lambda: x.solve(I0, I1, warps, iters, disp=disp, depth=depth), vsteps)
        variants["tgv_f32"] = {"value": job_rate(world, 1, ms), "unit": "frames/s",
                               "ms_per_frame": ms,
                               "schedule_per_level": tgv_sched or "default (blocking 4)"}
        x.close()
        if args.batch > 1:
            from paper_1909_07545_gb300 import Batch
            for storage in ("f32", "f16"):
                sols = [make(storage) for _ in range(args.batch)]
                bt = Batch(sols, stream=stream)
                outs_d = [torch.empty((H, W), device="cuda") for _ in sols]
                outs_z = [torch.empty((H, W), device="cuda") for _ in sols]
                # k: pairs allowed on their finest level at once (0 = no bound)
                for k in (0, 1, 2):
                    bt.set_finest_limit(k)
                    ms = timed(lambda: bt.solve([I0] * len(sols), [I1] * len(sols), warps,
                                                iters, disps=outs_d, depths=outs_z), vsteps)
                    variants[f"batched_{storage}_finest{k}"] = {
                        "value": job_rate(world, len(sols), ms), "unit": "frames/s",
                        "pairs_per_batch": len(sols), "finest_limit": k, "ms_per_batch": ms}
                bt.close()
                for x in sols:
                    x.close()

    uneven = None
    if args.uneven_batch:
        uneven = uneven_batch_leg(replica_seed(args.seed, rank), stream, 3, 3)

    # serving: one server on rank 0's GPU (the figures are per GPU; replicas
    # would serve independent request streams)
    serving = serving_f16 = None
    if args.serve_seconds > 0 and rank == 0:
        rigs, sizes, render_s = render_rigs(args.seed)
        serving = serve_leg(rigs, sizes, args.seed, args.serve_seconds, args.serve_rate,
                            args.serve_inflight, args.serve_warm_mode)
        serving["render_s"] = render_s
        serving["gpus"] = 1
        # the same requests with FP16 storage (FP32 arithmetic)
        serving_f16 = serve_leg(rigs, sizes, args.seed, args.serve_seconds, args.serve_rate,
                                args.serve_inflight, args.serve_warm_mode, storage="f16")

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    pxit_frame = sum(level_pixels(W, H, L)) * warps * iters
    ms_per_step = total_ms / args.steps
    fps = job_rate(world, args.steps, total_ms)
    ms0, n0, px0 = per_level[0]
    achieved = PD_BYTES_PER_PX_ITER * px0 / (ms0 / 1000.0) / 1e9
    # the profiled traffic applies while level 0 runs the profiled schedule
    l0_choice = tuned[0] if tuned else None
    traffic = PD_L0_DRAM_BYTES_PER_LAUNCH if l0_choice == PD_L0_PROFILED_CHOICE else None
    peaks, src = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    pd_ms = sum(m for m, _, _ in per_level) / args.steps
    # launches per frame: 2 copy/pre-rotate, L-1 downsample, L tensor, 1 zero,
    # L-1 upsample, per level one warp, warps-1 fused clip + warp and one
    # clip, PD launches, 1 depth
    per_frame_other = 2 + (L - 1) + L + 1 + (L - 1) + (warps + 1) * L + 1
    line = {
        "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": pair["name"], "W": W, "H": H, "levels": L, "warps": warps,
                   "iters": iters, "camera": "kannala_brandt f=320 fov=190",
                   "l2": "flushed between steps (256 MB write)",
                   "pd_schedule_per_level": (
                       [schedule_label(c) for c in tuned]
                       if tuned else "default (cluster <= 128 px, blocking 6 / 8 above)"),
                   "autotuned": bool(tuned), "graph": True,
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99)),
                       "max": float(step_ms.max())},
        "gpix_iter_s": pxit_frame * fps / world / 1e9 * world,
        "gpix_iter_s_in_mask": sum(mask_px) * warps * iters * fps / 1e9,
        "pd": {"ms_per_frame": pd_ms, "share_of_step": pd_ms / ms_per_step,
               "per_level_ms": [m / args.steps for m, _, _ in per_level]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_note": "DRAM bytes per level-0 launch, ncu, cold L2",
                     "kernel": "k_pd level 0 (1024x1024), " + (
                         schedule_label(l0_choice) if l0_choice is not None else "default"),
                     "launches_per_frame": n0 // max(args.steps, 1),
                     "algorithmic_bytes_per_launch": PD_BYTES_PER_PX_ITER * px0 / max(n0, 1),
                     "peak_source": f"{src} hbm_gbs",
                     "algorithmic_bytes_per_px_iter": PD_BYTES_PER_PX_ITER},
        "gpu_launches": int(args.steps * (pd_launches + per_frame_other)),
        "clocks": clk,
        "wall_s": t_wall,
    }
    line["variants"] = variants
    line["set_pose_ms"] = set_pose_ms
    # the same level-0 figure against the L2 bandwidth the frame's working set
    # (about 60 MB at level 0) actually streams from
    line["roofline_l2"] = {"bound": "l2", "achieved": achieved, "peak": l2_gbs, "unit": "GB/s",
                           "frac": achieved / l2_gbs,
                           "peak_source": "measured in this run: elementwise add over "
                                          "32 MB in + 32 MB out, L2-resident"}
    if serving is not None:
        line["serving"] = serving
        line["serving_f16"] = {k: serving_f16[k] for k in
                               ("workload", "frames_per_s", "p50_ms", "p99_ms", "max_ms",
                                "saturated_frames_per_s", "requests", "failed")}
    if uneven is not None:
        line["uneven_batch"] = uneven
    line["e2e"] = {"value": world / e2e_s, "unit": "frames/s",
                   "h2d_bytes_per_step": 2 * W * H * 4, "d2h_bytes_per_step": 2 * W * H * 4}
    if not args.no_cpu_baseline:
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        rate, n, dt = cpu_baseline(pair, args.cpu_seconds)
        line["cpu_baseline"] = {
            "value": rate / pxit_frame, "unit": "frames/s", "cores": 1,
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} primal-dual iterations of the finest {W}x{H} level in {dt:.1f} s "
                      f"(FP64 numpy, one thread), extrapolated to a frame by pixel-iterations "
                      f"({pxit_frame:.3e} per frame)"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
