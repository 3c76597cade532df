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
import gc
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
# ncu DRAM bytes (read + write) of one level-0 primal-dual launch of this
# workload, per schedule choice, each from one capture of the current kernel
# (cold L2, the mean of two consecutive launches; commands and figures in
# profiles/k_pd_level0_kb1024.md and profiles/k_pd_tma_level0_kb1024.md).  A
# choice without a capture of the current kernel reports traffic null.
PD_L0_DRAM_BYTES_PER_LAUNCH = {7: 47.44e6, 31: 47.44e6, 61: 47.65e6}
# FP32 instructions of one pixel-iteration of the primal-dual step as written
# in pd_math.cuh, an FMA counted as one: dual 24 (2 differences, 7 products,
# 9 FMAs, the reciprocal square root, a min and 4 mask selects), divergence 3,
# primal 5 (FMA, difference, clamp, sum), relaxation 2
PD_FP32_INSTR_PER_PX_ITER = 34
# FP32 lanes of GB300: 152 SMs x 128 lanes, one instruction per lane and clock
FP32_LANES = 152 * 128
FOOTPRINTS = ["64x64 footprints, 512 threads", "32x32 footprints, 256 threads",
              "64x32 footprints", "64x64 footprints, 1024 threads",
              "32x32 footprints, 1024 threads", "32x32 footprints, 512 threads",
              "64x64 footprints 48 columns apart, 1024 threads, TMA-staged",
              "64x48 footprints, 768 threads"]
FOOTPRINT_SIZE = [(64, 64), (32, 32), (64, 32), (64, 64), (32, 32), (32, 32), (64, 64),
                  (64, 48)]
TMA_FOOTPRINT = 6          # index of the TMA-staged footprint (choices 56..63)
FIRST_TMA_CHOICE = 56
FIRST_768_CHOICE = 64      # 64x48 footprints of 768 threads (choices 64..71)


def interior(v, B):
    """Interior (columns, rows) of footprint v at blocking depth B: the TMA
    footprints own 48 columns (8-column margins for the copies' 16-byte
    alignment), the others FW - 2B."""
    FW, FH = FOOTPRINT_SIZE[v]
    return (48 if v == TMA_FOOTPRINT else FW - 2 * B), FH - 2 * B


def decode_choice(c):
    """(depth, footprint index) of a schedule choice 1..71 (0: cluster -> None)."""
    if c is None or c <= 0:
        return None
    if c >= FIRST_768_CHOICE:
        return c - FIRST_768_CHOICE + 1, 7
    if c >= FIRST_TMA_CHOICE:
        return c - FIRST_TMA_CHOICE + 1, TMA_FOOTPRINT
    if c > 48:
        return c - 48 + 8, 4
    return (c - 1) % 8 + 1, (c - 1) // 8


def schedule_label(c):
    """fs_autotune's per-level choice in words (0 = cluster; 1..48 = depth
    1..8 on each of the six footprints; 49..55 = depth 9..15 on 32x32
    footprints of 1024 threads; 56..63 = depth 1..8 on the TMA-staged
    footprints; 64..71 = depth 1..8 on 64x48 footprints of 768 threads)."""
    if c == 0:
        return "cluster"
    B, v = decode_choice(c)
    return f"blocking x{B} ({FOOTPRINTS[v]})"


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


def _oracle_frame(pair):
    """One whole frame of the FP64 oracle (a worker of the host-core legs);
    returns its solve time in seconds."""
    import oracle
    t0 = time.perf_counter()
    oracle.solve(pair["I0"], pair["I1"], pair["cam0"], pair["cam1"], pair["R"], pair["t"],
                 pair["levels"], pair["warps"], pair["iters"],
                 oracle.Params(lam=pair["lam"], eps=pair["eps"]))
    return time.perf_counter() - t0


def _one_thread():
    os.environ["OMP_NUM_THREADS"] = "1"


def baseline_pairs(n):
    """n independent 256^2 pairs of the smallest workload (3 levels, 5 warps x
    50 iterations), images rounded to float32 as the GPU receives them."""
    import synth
    out = []
    for k in range(n):
        p = synth.plain_small(k)
        p["I0"] = np.float32(p["I0"]).astype(np.float64)
        p["I1"] = np.float32(p["I1"]).astype(np.float64)
        out.append(p)
    return out


def oracle_pool(n):
    """A spawned pool of n one-thread oracle processes."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(n, initializer=_one_thread)


def cpu_baseline(pxit_target, one_thread_frames=4, pool_steps=2):
    """The FP64 oracle as it stands on this host's cores, on whole frames of
    the 256^2 workload (3 levels, 5 warps x 50 iterations): one thread
    (frames one after another in this process) and all cores (one process per
    core, each its own pair, frames at once).  Returns the measured 256^2
    figures and both rates converted to frames of the target workload by
    pixel-iterations (pxit_target per frame)."""
    n = os.cpu_count() or 1
    pairs = baseline_pairs(n)
    pxit = sum(level_pixels(256, 256, 3)) * 5 * 50
    t1 = [_oracle_frame(pairs[k % n]) for k in range(one_thread_frames)]
    one_fps = len(t1) / sum(t1)
    with oracle_pool(n) as pool:
        pool.map(_oracle_frame, pairs)                 # start-up and warm-up
        walls = []
        for _ in range(pool_steps):
            t0 = time.perf_counter()
            pool.map(_oracle_frame, pairs)
            walls.append(time.perf_counter() - t0)
    all_fps = n / float(np.mean(walls))
    scale = pxit / pxit_target
    return {
        "value": all_fps * scale, "unit": "frames/s", "cores": n, "kind": "oracle",
        "sample": f"whole frames of the 256x256 equidistant workload (3 levels, 5 warps x 50 "
                  f"iterations, {pxit:.3e} pixel-iterations each), FP64 numpy: {pool_steps} "
                  f"rounds of {n} frames at once, one process per core on its own pair; the "
                  f"value is converted to 1024x1024 frames by pixel-iterations "
                  f"({pxit_target:.3e} per frame)",
        "measured_256": {"all_cores_frames_per_s": all_fps, "cores": n,
                         "one_thread_frames_per_s": one_fps,
                         "one_thread_s_per_frame": float(np.mean(t1)),
                         "all_cores_round_s": float(np.mean(walls))},
        "one_thread": {"value": one_fps * scale, "unit": "frames/s", "cores": 1},
    }


def render_rigs(seed, n_rigs=16, n_frames=3):
    """The serving workload's rigs: sizes drawn from 640 / 1024 / 1280 px,
    each its own seeded Kannala-Brandt calibration, relative pose and scene,
    n_frames consecutive frames of its smooth path."""
    import multiprocessing as mp
    rng = np.random.default_rng(1000 + seed)
    sizes = [int(v) for v in rng.choice([640, 1024, 1280], size=n_rigs)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(n_rigs, os.cpu_count() or 1)) as pool:
        rigs = pool.map(_render_rig, [(10000 * (seed + 1) + i, W, n_frames)
                                      for i, W in enumerate(sizes)])
    return rigs, sizes, time.perf_counter() - t0


def _render_rig(args):
    import synth
    s, W, n_frames = args
    return synth.rig_sequence(s, W, W, n_frames=n_frames)


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
        return srv.submit(ids[r], I0, I1, d, z), slot

    # one waiter thread per rig returns the rig's result buffers as its
    # requests complete (a rig's requests run in order): a single waiter
    # taking requests in submission order would hold a rig's finished slot
    # behind another rig's slower request, and the generator, needing that
    # slot, would stall
    done_q = [queue.Queue() for _ in range(n_rigs)]

    def waiter(r):
        while True:
            item = done_q[r].get()
            if item is None:
                return
            req, slot = item
            try:
                srv.wait(req)
            except Exception:          # a failed request: the server counts it
                pass
            free[r].put(slot)

    ths = [threading.Thread(target=waiter, args=(r,), daemon=True) for r in range(n_rigs)]
    for th in ths:
        th.start()
    # warm-up: every rig's cold first frame, then two warm frames each
    for _ in range(3):
        for r in range(n_rigs):
            done_q[r].put(submit(r))
    srv.drain()
    srv.stats(reset=True)

    # open loop at the offered rate.  The generator runs with Python's
    # cyclic collector frozen and off: a collection pass over the process's
    # objects stops this thread for milliseconds, and the arrivals it holds
    # back would reach the server as one burst.  late = how long after its
    # scheduled arrival each request's submission returned (the generator's
    # own delay, which the server's latency figures do not include).
    arr = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * seconds * 1.2) + 16))
    arr = arr[arr < seconds]
    which = [int(r) for r in rng.integers(0, n_rigs, size=len(arr))]
    arr = [float(a) for a in arr]
    late = np.zeros(len(arr))
    gc.collect()
    gc.freeze()
    gc.disable()
    try:
        start = time.perf_counter()
        stalls = 0
        for k, (ta, r) in enumerate(zip(arr, which)):
            now = time.perf_counter() - start
            if ta > now:
                time.sleep(ta - now)
            if free[r].empty():
                stalls += 1
            done_q[r].put(submit(r))
            late[k] = time.perf_counter() - start - ta
        srv.drain()
    finally:
        gc.enable()
        gc.unfreeze()
    open_loop = srv.stats(reset=True)
    late_ms = 1e3 * late

    # saturated: keep every rig's ring full for a fixed number of requests
    # (64 per rig, about a second: long enough that the ramp-up and the
    # drain do not decide the rate)
    n_sat = 64 * n_rigs
    t1 = time.perf_counter()
    for i in range(n_sat):
        done_q[i % n_rigs].put(submit(i % n_rigs))
    srv.drain()
    sat = srv.stats(reset=True)
    sat_wall = time.perf_counter() - t1
    for q in done_q:
        q.put(None)
    for th in ths:
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
        "submit_late_ms": {"p50": float(np.percentile(late_ms, 50)),
                           "p99": float(np.percentile(late_ms, 99)),
                           "max": float(late_ms.max()) if len(late_ms) else 0.0},
        "cold": int(open_loop["cold"]), "evictions": int(open_loop["evictions"]),
        "resident_gb": open_loop["resident_bytes"] / 1e9,
        "saturated_frames_per_s": sat["frames_per_s"], "saturated_requests": n_sat,
        "saturated_wall_s": sat_wall,
        "gpix_iter_s_at_offered": open_loop["frames_per_s"] * mean_px * 150 / 1e9,
    }


def _render_uneven(args):
    import synth
    seed, j, i, W = args
    return synth.plain_kb(100000 * (seed + 1) + 1000 * j + i, W=W, H=W, supersample=1,
                          levels=synth.auto_levels(W))


def render_uneven(seed, per_size, sizes):
    """The batching workload's pairs, rendered by a spawned process pool."""
    import multiprocessing as mp
    jobs = [(seed, j, i, W) for j, W in enumerate(sizes) for i in range(per_size)]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        return pool.map(_render_uneven, jobs)


def uneven_batch_leg(seed, stream, steps, warmup, storage="f16", per_size=16,
                     sizes=(512, 800, 1024, 1280)):
    """Batching: per_size pairs of each size, every pair its own seeded
    Kannala-Brandt calibration, relative pose and scene (the 1024 generator
    scaled), 4-6 pyramid levels (level count: coarsest level >= 40 px),
    10 warps x 100 iterations, 16-bit storage, all pairs in one fs_batch
    graph, the schedule autotuned once per size.  Beside it, the plain path
    on the same pairs: FP32 storage, one pair after another, each through
    its own graph.  Returns frames/s of both (the batch per finest-level
    bound)."""
    import torch

    from paper_1909_07545_gb300 import Batch, Solver
    t0 = time.perf_counter()
    pairs = render_uneven(seed, per_size, sizes)
    render_s = time.perf_counter() - t0
    I0s = [torch.as_tensor(np.float32(p["I0"]), device="cuda") for p in pairs]
    I1s = [torch.as_tensor(np.float32(p["I1"]), device="cuda") for p in pairs]
    outs_d = [torch.empty_like(a) for a in I0s]
    outs_z = [torch.empty_like(a) for a in I0s]

    def handles(st, sched="auto", tuned=None):
        sols, tuned = [], dict(tuned or {})
        for p in pairs:
            W = p["I0"].shape[1]
            x = Solver(p["cam0"], p["cam1"], p["R"], p["t"], W, W, p["levels"], stream=stream,
                       lam=p["lam"], huber_eps=p["eps"], use_graph=1, storage=st,
                       pd_schedule=sched)
            if W not in tuned:
                tuned[W] = x.autotune(p["iters"])
            else:
                x.set_schedule(tuned[W])
            sols.append(x)
        return sols, tuned

    def timed(run):
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
        return e0.elapsed_time(e1) / steps

    sols, tuned = handles(storage)
    bt = Batch(sols, stream=stream)
    coarse = bt.autotune(100)          # the coarse levels' schedule for throughput
    res = {}
    for k in (0, 1, 2, 4):
        bt.set_finest_limit(k)
        ms = timed(lambda: bt.solve(I0s, I1s, 10, 100, disps=outs_d, depths=outs_z))
        res[f"finest{k}"] = {"frames_per_s": len(pairs) * 1000.0 / ms, "ms_per_batch": ms}
    bt.close()
    for x in sols:
        x.close()
    # the same batch in the persistent schedule: one launch for every level
    # and warp of all 64 pairs (the graph holds the pyramids, that launch and
    # the depths)
    psols, _ = handles(storage, "persistent", tuned)
    bt = Batch(psols, stream=stream)
    ms = timed(lambda: bt.solve(I0s, I1s, 10, 100, disps=outs_d, depths=outs_z))
    persistent = {"frames_per_s": len(pairs) * 1000.0 / ms, "ms_per_batch": ms}
    bt.close()
    for x in psols:
        x.close()
    plain, _ = handles("f32")

    def one_by_one():
        for x, a, b, d, z in zip(plain, I0s, I1s, outs_d, outs_z):
            x.solve(a, b, 10, 100, disp=d, depth=z)
    plain_ms = timed(one_by_one)
    for x in plain:
        x.close()
    px_iter = sum(sum(level_pixels(p["I0"].shape[1], p["I0"].shape[0], p["levels"])) * 1000
                  for p in pairs)
    best = max(r["frames_per_s"] for r in res.values())
    return {"workload": f"{len(pairs)} pairs, {per_size} each of {list(sizes)} px, "
                        f"Kannala-Brandt 190 deg, own calibration and pose each, "
                        f"4-6 levels x 10 warps x 100 iterations, {storage} storage, one graph",
            "by_finest_limit": res, "persistent": persistent,
            "best_frames_per_s": max(best, persistent["frames_per_s"]),
            "gpix_iter_s_best": px_iter * max(best, persistent["frames_per_s"]) / len(pairs) / 1e9,
            "plain_f32_one_by_one": {"frames_per_s": len(pairs) * 1000.0 / plain_ms,
                                     "ms_per_64": plain_ms},
            "schedule_per_size": {str(W): [schedule_label(c) for c in t]
                                  for W, t in tuned.items()},
            "batch_coarse_schedule": "each pair's own" if coarse < 0 else schedule_label(coarse),
            "render_s": render_s}


def oracle_sample_parity(d, workload, seed):
    """|d - oracle| at the stored oracle samples of this configuration
    (tests/golden/kb1024_oracle.json: 4096 seeded FOV pixels of the full-count
    solve, written from oracle/ and synth/ only, with the oracle's own
    response at each to five FP32-sized probes).  None for another workload."""
    if workload != "plain_kb_1024" or seed != 0:
        return None
    with open(os.path.join(ROOT, "tests", "golden", "kb1024_oracle.json")) as f:
        g = json.load(f)
    c = np.array(g["sample"], dtype=np.float64)
    y, x, dref, probe = c[:, 0].astype(int), c[:, 1].astype(int), c[:, 2], c[:, 3]
    err = np.abs(np.asarray(d, dtype=np.float64)[y, x] - dref)
    well = probe <= 1e-3
    return {"pixels": len(err), "mean": float(err.mean()),
            "q998": float(np.quantile(err, 0.998)), "max": float(err.max()),
            "n_over_5e-3": int((err > 5e-3).sum()),
            "well_conditioned": {"pixels": int(well.sum()), "max": float(err[well].max()),
                                 "mean": float(err[well].mean())},
            "oracle_probe": {"mean": float(probe.mean()),
                             "q998": float(np.quantile(probe, 0.998)),
                             "max": float(probe.max()),
                             "n_over_5e-3": int((probe > 5e-3).sum())}}


def batch_1024_leg(seed, stream, tuned, steps, warmup, n=8, storage="f16"):
    """n distinct 1024^2 pairs of the Kannala-Brandt workload in one fs_batch
    graph (FP16 storage, FP32 arithmetic), each handle on the tuned schedule
    of the single pair, at finest-level bounds 0, 1 and 2."""
    import torch

    from paper_1909_07545_gb300 import Batch, Solver
    pairs = [workload_pair("plain_kb_1024", seed + 100 + k) for k in range(n)]
    sols = []
    for p in pairs:
        x = Solver(p["cam0"], p["cam1"], p["R"], p["t"], 1024, 1024, p["levels"], stream=stream,
                   lam=p["lam"], huber_eps=p["eps"], use_graph=1, storage=storage)
        if tuned:
            x.set_schedule(tuned)
        sols.append(x)
    I0s = [torch.as_tensor(np.float32(p["I0"]), device="cuda") for p in pairs]
    I1s = [torch.as_tensor(np.float32(p["I1"]), device="cuda") for p in pairs]
    outs_d = [torch.empty_like(a) for a in I0s]
    outs_z = [torch.empty_like(a) for a in I0s]
    bt = Batch(sols, stream=stream)
    coarse = bt.autotune(100)          # the coarse levels' schedule for throughput
    res = {}
    for k in (0, 1, 2):
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
        res[f"finest{k}"] = {"frames_per_s": n * 1000.0 / ms, "ms_per_batch": ms}
    bt.close()
    for x in sols:
        x.close()
    return {"workload": f"{n} distinct 1024x1024 Kannala-Brandt pairs (seeds +100..), 5 levels "
                        f"x 10 warps x 100 iterations, {storage} storage, one graph",
            "by_finest_limit": res,
            "batch_coarse_schedule": "each pair's own" if coarse < 0 else schedule_label(coarse),
            "best_frames_per_s": max(r["frames_per_s"] for r in res.values())}


def run_reference(args, pair, rank):
    """--impl reference: the FP64 oracle as it stands on the host cores.  Each
    step is a bounded, whole piece of the work: one frame of the 256^2
    workload (3 levels, 5 warps x 50 iterations) on every core at once, one
    process per core on its own pair; ms_per_step is that measured time, and
    the value converts the rate to frames of the target workload by
    pixel-iterations."""
    if rank != 0:
        return
    H, W = pair["I0"].shape
    pxit_target = sum(level_pixels(W, H, pair["levels"])) * pair["warps"] * pair["iters"]
    n = os.cpu_count() or 1
    pairs = baseline_pairs(n)
    pxit = sum(level_pixels(256, 256, 3)) * 5 * 50
    with oracle_pool(n) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_frame, pairs)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_frame, pairs)
            times.append(time.perf_counter() - t0)
    step_s = float(np.mean(times))
    fps256 = n / step_s
    fps = fps256 * pxit / pxit_target
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * step_s, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": pair["name"], "W": W, "H": H, "levels": pair["levels"],
                   "warps": pair["warps"], "iters": pair["iters"],
                   "camera": "kannala_brandt f=320 fov=190"},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": n, "kind": "oracle",
                         "sample": f"per step, {n} whole frames of the 256x256 equidistant "
                                   f"workload (3 levels, 5 warps x 50 iterations) at once, one "
                                   f"process per core; converted to 1024x1024 frames by "
                                   f"pixel-iterations ({pxit:.3e} against {pxit_target:.3e})",
                         "measured_256_frames_per_s": fps256},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpix_iter_s": fps256 * pxit / 1e9,
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
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip fs_autotune (default schedule per level)")
    ap.add_argument("--batch", type=int, default=8,
                    help="distinct 1024^2 pairs in the FP16 batch leg (<= 1 skips it)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the open-loop FP32 serving run (0 skips serving)")
    ap.add_argument("--serve-f16-seconds", type=float, default=10.0,
                    help="length of the FP16-storage serving run (0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=600.0, help="offered requests/s")
    ap.add_argument("--serve-inflight", type=int, default=2)
    ap.add_argument("--serve-warm-mode", type=int, default=1, choices=[0, 1])
    ap.add_argument("--no-uneven-batch", dest="uneven_batch", action="store_false",
                    help="skip the 64 uneven pairs (512/800/1024/1280 px) in one batch graph")
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
        main_disp = disp.cpu().numpy()
        parity = oracle_sample_parity(main_disp, args.workload, replica_seed(args.seed, rank))
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
        # and the trajectory fields (float-float kernels on the handle's stream)
        s.set_pose(pair["R"], pair["t"])
        stream.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            s.set_pose(pair["R"], pair["t"])
        stream.synchronize()
        set_pose_ms = (time.perf_counter() - t0) / 5 * 1000.0
        s.close()

        # variants of the same frame: 16-bit storage, the TGV-L1 regulariser
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
                                 "pd_per_level_ms": [m / vsteps for m, _, _ in lv],
                                 "vs_oracle": oracle_sample_parity(
                                     disp.cpu().numpy(), args.workload,
                                     replica_seed(args.seed, rank))}
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
        # the persistent schedule: every level and warp in one launch over a
        # work list (footprints and depths from the same tuning)
        x = Solver(pair["cam0"], pair["cam1"], pair["R"], pair["t"], W, H, L, stream=stream,
                   lam=pair["lam"], huber_eps=pair["eps"], use_graph=1, pd_schedule="persistent")
        if tuned:
            x.set_schedule(tuned)
        ms = timed(lambda: x.solve(I0, I1, warps, iters, disp=disp, depth=depth), vsteps)
        variants["persistent_f32"] = {"value": job_rate(world, 1, ms), "unit": "frames/s",
                                      "ms_per_frame": ms,
                                      "bit_identical_to_main": bool(torch.equal(
                                          disp, torch.as_tensor(main_disp, device="cuda")))}
        x.close()
    # the batched path against the plain one at 1024 x 1024: 8 distinct pairs of the workload
    # (seeds seed+100 ..), FP16 storage, one fs_batch graph, against the
    # plain FP32 single-pair figure above
    batch1024 = None
    if args.batch > 1:
        batch1024 = batch_1024_leg(args.seed, stream, tuned, max(3, min(args.steps, 10)),
                                   args.warmup, n=args.batch)

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
        # the same request stream with FP16 storage (FP32 arithmetic), shorter
        if args.serve_f16_seconds > 0:
            serving_f16 = serve_leg(rigs, sizes, args.seed, args.serve_f16_seconds,
                                    args.serve_rate, args.serve_inflight, args.serve_warm_mode,
                                    storage="f16")

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    pxit_frame = sum(level_pixels(W, H, L)) * warps * iters
    ms_per_step = total_ms / args.steps
    fps = job_rate(world, args.steps, total_ms)
    ms0, n0, px0 = per_level[0]
    launch_s = ms0 / 1000.0 / max(n0, 1)                # mean level-0 launch duration
    l0_choice = tuned[0] if tuned else None
    dec = decode_choice(l0_choice)
    peaks, src = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    # Algorithmic bytes of one level-0 launch (the blocked figure of the
    # roofline model): one pass over every footprint, 52 B per pixel
    # (9 words read, 4 written), the footprints overlapping by
    # (FW / IW) x (FH / IH) with IW x IH interior pixels (interior()).
    if dec is not None:
        B, v = dec
        FW, FH = FOOTPRINT_SIZE[v]
        IW, IH = interior(v, B)
        overlap = FW / IW * FH / IH
    else:
        B, FW, FH, IW, IH, overlap = None, None, None, None, None, 1.0
    px_l0 = W * H
    bytes_launch = PD_BYTES_PER_PX_ITER * px_l0 * overlap
    achieved = bytes_launch / launch_s / 1e9
    compulsory = PD_BYTES_PER_PX_ITER * px_l0 / launch_s / 1e9
    traffic = PD_L0_DRAM_BYTES_PER_LAUNCH.get(l0_choice)
    iters_per_launch = px0 / max(n0, 1) / px_l0
    alu_achieved = PD_FP32_INSTR_PER_PX_ITER * px_l0 * iters_per_launch / launch_s
    alu_peak = FP32_LANES * (clk["sm_mhz"] if clk else 2070.0) * 1e6
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
                     "traffic_note": "ncu DRAM read + write bytes of one level-0 launch of "
                                     "this schedule, cold L2 (null: no capture of it)",
                     # the measured DRAM bytes over the same warm launch time: what
                     # the kernel actually draws from HBM (L2 serves the halo overlap)
                     "traffic_gbs": traffic / launch_s / 1e9 if traffic else None,
                     "traffic_frac": traffic / launch_s / 1e9 / peak if traffic else None,
                     "kernel": ("k_pd_tma" if dec is not None and dec[1] == TMA_FOOTPRINT
                                else "k_pd") + " level 0 (1024x1024), " + (
                         schedule_label(l0_choice) if l0_choice is not None else "default"),
                     "launches_per_frame": n0 // max(args.steps, 1),
                     "launch_us": launch_s * 1e6,
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "algorithmic_bytes_note": "52 B per level-0 pixel x footprint overlap "
                                               f"({FW}x{FH} footprints, depth {B}, "
                                               f"interior {IW}x{IH}: x{overlap:.3f})",
                     "peak_source": f"{src} hbm_gbs",
                     "compulsory_frac": compulsory / peak,
                     "compulsory_note": "one pass, 52 B per level-0 pixel per launch, no halo",
                     "alu": {"achieved": alu_achieved / 1e12, "peak": alu_peak / 1e12,
                             "unit": "T FP32 instr/s",
                             "frac": alu_achieved / alu_peak,
                             "halo_recompute": overlap,
                             "note": f"{PD_FP32_INSTR_PER_PX_ITER} FP32 instructions per "
                                     "level-0 pixel-iteration (the halo recomputation, "
                                     "x halo_recompute, not counted); peak = 152 SMs x 128 "
                                     "lanes x median SM clock"}},
        "gpu_launches": int(args.steps * (pd_launches + per_frame_other)),
        "clocks": clk,
        "wall_s": t_wall,
    }
    line["variants"] = variants
    if parity is not None:
        line["parity"] = parity
    line["set_pose_ms"] = set_pose_ms
    # the same level-0 figure against the L2 bandwidth the frame's working set
    # (about 60 MB at level 0) actually streams from
    line["roofline_l2"] = {"bound": "l2", "achieved": achieved, "peak": l2_gbs, "unit": "GB/s",
                           "frac": achieved / l2_gbs,
                           "peak_source": "measured in this run: elementwise add over "
                                          "32 MB in + 32 MB out, L2-resident"}
    if serving is not None:
        line["serving"] = serving
    if serving_f16 is not None:
        line["serving_f16"] = {k: serving_f16[k] for k in
                               ("workload", "seconds", "frames_per_s", "p50_ms", "p99_ms",
                                "max_ms", "saturated_frames_per_s", "requests", "failed")}
    if batch1024 is not None:
        line["batch_1024"] = batch1024
    if uneven is not None:
        line["uneven_batch"] = uneven
    line["e2e"] = {"value": world / e2e_s, "unit": "frames/s",
                   "h2d_bytes_per_step": 2 * W * H * 4, "d2h_bytes_per_step": 2 * W * H * 4}
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(pxit_frame)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
