#!/usr/bin/env python
"""Throughput of the vectorised object-MLP training step (vMAP, section 3.2).

Workload ("room50"): 50 object MLPs (hidden 32, rays per object log-uniform
in 32-600) plus one background MLP (hidden 128, 1,200 rays), 22 samples per
ray, every object present (the steady state after the last incremental
insertion). One step = ray picking + depth-guided sampling + encoding + MLP
forward + rendering + losses + backward + Adam for all 51 objects.

Headline: the FP32 path (the paper's precision: FP32 SIMT kernels), the
step replayed as a CUDA graph, launch shapes autotuned. Beside it, on the
same workload: the BF16 tensor-core path (tcgen05 GEMMs, FP32 accumulation,
master weights, moments, rendering and losses); each with a profiled
kernel-by-kernel pass (per-kernel time and the roofline of the dominant
kernel). Also: the precision-200 and 1,000-object workloads, and the time to
a held-out depth-L1 target of plain FP32 vs BF16 + batched vs BF16 + batched
+ warm start.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. Under torchrun every rank trains its own 51-object
scene (objects are independent, no collective on the data path: weak
scaling); rank 0 prints the aggregate.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "object-MLP train steps/s and sampled pts/s at 50 objs; time-to-depth-L1 vs FP32"
UNIT = "pts/s"
L2_FLUSH_BYTES = 512 << 20   # > 126 MB L2
FP32_LANES_PER_SM = 128      # FFMA lanes per SM (4 SMSPs x 32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="fp32",
                    help="fp32: the FP32 path, the paper's precision (default headline); bf16: tcgen05 BF16 "
                         "GEMMs with FP32 accumulation (reported beside it either way)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch kernel by kernel instead of graph replay")
    ap.add_argument("--prof-steps", type=int, default=200, help="steps of the profiled kernel-by-kernel pass")
    ap.add_argument("--fp32-steps", type=int, default=1,
                    help="0: skip the line of the other precision (BF16 beside an FP32 headline, or FP32 beside BF16)")
    ap.add_argument("--no-ttd", action="store_true", help="skip the time-to-depth-L1 comparison")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=12, help="oracle steps of the CPU baseline sample")
    ap.add_argument("--e2e-steps", type=int, default=1000)
    ap.add_argument("--window-s", type=float, default=2.0,
                    help="repeat the K-step timed window for at least this many seconds (clock sampling)")
    ap.add_argument("--min-windows", type=int, default=5)
    ap.add_argument("--no-workloads", action="store_true", help="skip the precision200 / many1000 lines")
    ap.add_argument("--sweep", action="store_true",
                    help="print the object-count / hidden-width sweep instead of the bench line")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def rank_seed(rank):
    """Each rank trains its own independent scene (the unit of sharding is an object)."""
    return 2 + 1000 * rank


def workload(rank):
    from paper_2302_01838_b300 import scenes
    return scenes.scene_room(seed=rank_seed(rank))


def samples_per_step(scene):
    return sum(o["rays"] * (o["n_surface"] + o["n_strat"]) for o in scene["objects"])


def flops_per_sample(H, part="all"):
    """Algorithmic flops of one sample's forward + backward MLP GEMMs:
    forward F = 93H + 3H^2 + 4H MACs, weight gradient F MACs, input gradient
    3H^2 + 4H MACs (layer 1 skipped); 2 flops per MAC. part = "fb" (forward
    and input gradients) or "dw" (weight gradients) splits the sum the way
    the width-128 paths (tensor-core and FP32) split their two kernels."""
    F = 93 * H + 3 * H * H + 4 * H
    fb, dw = 2 * (F + 3 * H * H + 4 * H), 2 * F
    return {"all": fb + dw, "fb": fb, "dw": dw}[part]


def kernel_flops(name, objs):
    """Algorithmic flops of one launch of a tile kernel on the workload."""
    H = int(name.split("<")[1].rstrip(">"))
    part = ("fb" if name.startswith(("k_wide_fb", "k_w32_fb")) else
            "dw" if name.startswith(("k_wide_dw", "k_w32_dw")) else "all")
    return sum(o["rays"] * (o["n_surface"] + o["n_strat"]) * flops_per_sample(H, part) for o in objs if o["H"] == H)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def source_hash(files):
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2302_01838_b300", "csrc")
    for fn in files:
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel, launches_scale=1.0):
    """DRAM bytes per launch from the committed ncu summary, if the counters
    were taken on the kernel's current source files (else None)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    e = t.get(kernel)
    if not e or e.get("source_hash") != source_hash(e.get("sources", [])):
        return None
    return int(e["bytes_per_launch"] * launches_scale)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        # nvidia-smi numbers the physical GPUs; map the process's device index
        # through CUDA_VISIBLE_DEVICES when that lists indices
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        self.index = ids[index] if index < len(ids) and all(v.isdigit() for v in ids) else index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(",") for l in self.file.read().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(scene, steps):
    """The FP64 oracle as it stands on this host's cores: `steps` full steps of
    the same 51-object workload."""
    import numpy as np
    from oracle import vmap_step as vs
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    cfg = vs.Config(seed=scene["seed"], B=np.asarray(scene["B"], np.float64))
    st = [vs.ObjectState(H=o["H"], pool=o["pool"], center=np.asarray(o["center"], np.float64),
                         scale=float(o["scale"]), n_surface=o["n_surface"], n_strat=o["n_strat"],
                         stream=k, params=o["init"]) for k, o in enumerate(scene["objects"])]
    R = [o["rays"] for o in scene["objects"]]
    t0 = time.perf_counter()
    for _ in range(steps):
        vs.train_step(cfg, st, R)
    dt = time.perf_counter() - t0
    return {"value": samples_per_step(scene) * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} full steps of the room50 workload (51 objects, {samples_per_step(scene)} "
                      f"samples/step), FP64 numpy, {dt:.1f} s"}


REF_BUDGET_S = 120.0          # wall time the reference arm's steps may take


def run_reference(args):
    """The FP64 oracle as it stands, on this host's cores, on the room50
    workload. Each step is a bounded sample of it: every object trains with
    the same fraction f of its rays (at least one), f chosen so that the
    warm-up and timed steps fit a couple of minutes; value = sampled points/s."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sc = workload(0)
    import numpy as np
    from oracle import vmap_step as vs
    cfg = vs.Config(seed=sc["seed"], B=np.asarray(sc["B"], np.float64))
    st = [vs.ObjectState(H=o["H"], pool=o["pool"], center=np.asarray(o["center"], np.float64),
                         scale=float(o["scale"]), n_surface=o["n_surface"], n_strat=o["n_strat"],
                         stream=k, params=o["init"]) for k, o in enumerate(sc["objects"])]
    full = samples_per_step(sc)
    ray_sample = lambda f: [max(1, int(round(o["rays"] * f))) for o in sc["objects"]]
    n_samples = lambda R: sum(r * (o["n_surface"] + o["n_strat"]) for r, o in zip(R, sc["objects"]))
    # calibrate the cost of a step on this host with a 5% ray sample (a copy of the state)
    import copy
    probe = ray_sample(0.05)
    tc = time.perf_counter()
    vs.train_step(cfg, copy.deepcopy(st), probe)
    per_sample = (time.perf_counter() - tc) / n_samples(probe)
    budget = REF_BUDGET_S / max(1, args.steps + args.warmup) / per_sample   # samples per step
    f = min(1.0, budget / full)
    R = ray_sample(f)
    sps = n_samples(R)
    for _ in range(args.warmup):
        vs.train_step(cfg, st, R)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vs.train_step(cfg, st, R)
    dt = time.perf_counter() - t0
    value = sps * args.steps / dt
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    sample = (f"{args.steps} steps of the room50 workload (51 objects), each object training "
              f"{f:.4f} of its rays ({sps} of {full} samples per step), FP64 numpy")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "room50: 50 objects (hidden 32, 32-600 rays) + background (hidden 128, "
                                  "1200 rays), 22 samples/ray; the FP64 oracle on a ray sample of each step",
                      "objects": len(sc["objects"]), "samples_per_step": sps, "ray_fraction": f},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def make_context(sc, precision, autotune, reps=3, extra=8, n_add=None):
    """A context sized for the whole scene holding its first n_add objects
    (all by default), launch shape autotuned on their batch."""
    from paper_2302_01838_b300.api import VMap
    from paper_2302_01838_b300.native import VMAP_BF16, VMAP_FP32
    objs = sc["objects"]
    n_add = len(objs) if n_add is None else n_add
    R = [o["rays"] for o in objs]
    prec = VMAP_BF16 if precision == "bf16" else VMAP_FP32
    vm = VMap(max_objects=len(objs) + extra, max_rays_total=2 * sum(R) + 8192,
              max_pool_rays=sum(o["pool"].shape[0] for o in objs) + 16, B=sc["B"], seed=sc["seed"], precision=prec)
    for k, o in enumerate(objs[:n_add]):
        vm.add_object(o["pool"], hidden=o["H"], center=o["center"], scale=float(o["scale"]),
                      n_surface=o["n_surface"], n_strat=o["n_strat"], init_params=o["init"], stream_id=k)
    if autotune:
        # the autotuner times whole steps; graph-replayed, as they are timed below
        vm.set_graph(True)
        vm.autotune(R[:n_add], reps=reps)
        vm.set_graph(False)
    return vm


def step_intervals(vm, R, steps, flush, loss):
    """Device milliseconds of each of `steps` steps (CUDA events on the
    context's stream), L2 flushed between steps (outside the intervals)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record()
        vm.step(R, loss)   # sample_rays + train_step as one launch sequence
        ev[i][1].record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def timed_windows(vm, R, K, flush, loss, min_s, min_windows, world=1):
    """Windows of exactly K steps, each bracketed by a barrier and a
    synchronize, repeated until min_s seconds and min_windows windows have
    passed (so the clock sampler sees the timed work); returns the device
    milliseconds of every window (max over ranks)."""
    import torch
    import torch.distributed as dist
    from paper_2302_01838_b300 import sharding
    out = []
    t0 = time.perf_counter()
    while len(out) < min_windows or time.perf_counter() - t0 < min_s:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ms = sum(step_intervals(vm, R, K, flush, loss))
        if world > 1:
            dist.barrier()
        out.append(sharding.max_over_ranks(ms) if world > 1 else ms)
        if len(out) >= 100000:
            break
    return out


def median(x):
    y = sorted(x)
    n = len(y)
    return 0.5 * (y[(n - 1) // 2] + y[n // 2])


def profile_pass(vm, R, steps, flush, loss):
    """Kernel by kernel (every launch bracketed by the library's CUDA events):
    {kernel: (launches, total device ms)}."""
    for _ in range(3):
        vm.step(R, loss)
    vm.profile_reset()
    vm.profile_enable(True)
    step_intervals(vm, R, steps, flush, loss)
    vm.profile_enable(False)
    return vm.profile()


def fp32_peak_tflops(props, peaks):
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    return props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12, sm_max


def roofline_of(prof, objs, precision, peaks, props, prof_steps):
    """Roofline of the dominant tile kernel: algorithmic flops per launch /
    its mean CUDA-event duration, against the measured BF16 burst peak
    (tensor-core kernels) or the FP32 FFMA peak (FP32 SIMT kernels)."""
    tiles = {k: v for k, v in prof.items() if k.startswith(("k_tile", "k_wide", "k_w32"))}
    dom = max(tiles, key=lambda k: tiles[k][1])
    flops = kernel_flops(dom, objs)
    n_l, dom_ms = tiles[dom]
    achieved = flops / (dom_ms / n_l * 1e-3) / 1e12
    if dom.startswith(("k_tile_bf16", "k_wide")):
        peak, bound = peaks.get("bf16_tflops", 1800.0), "tensor"
        note = "measured cuBLAS BF16 burst (MEASURED_PEAKS.json bf16_tflops)"
    else:
        peak, sm_max = fp32_peak_tflops(props, peaks)
        bound = "alu"
        note = f"FP32 FFMA: {props.multi_processor_count} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {sm_max:.0f} MHz"
    return {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic_for(dom), "peak_note": note, "flops_per_launch": flops,
            "avg_launch_ms": dom_ms / n_l,
            "timing": f"CUDA events around each launch, {prof_steps}-step kernel-by-kernel pass"}


def kernel_table(prof):
    total = sum(v[1] for v in prof.values())
    return {k: {"launches": n, "total_ms": round(t_, 4), "share": round(t_ / total, 4)} for k, (n, t_) in prof.items()}


def measure_workload(sc, precision, K, W, flush, args, peaks, props, clocks=False, admit=0):
    """One workload, one precision: autotuned launch shape, graph replay,
    median of repeated K-step windows; the dominant kernel's roofline from a
    kernel-by-kernel pass. admit > 0: the last `admit` objects are held back
    and admitted after the timed windows into the captured step (no
    re-capture), and a second set of windows is timed."""
    import torch
    objs = sc["objects"]
    R = [o["rays"] for o in objs]
    n_first = len(objs) - admit
    vm = make_context(sc, precision, not args.no_autotune, n_add=n_first)
    R0 = R[:n_first]
    loss = torch.empty(len(objs) + 8, device="cuda")
    prof = profile_pass(vm, R0, args.prof_steps, flush, loss)
    vm.set_graph(not args.no_graph)
    for _ in range(max(W, 3)):
        vm.step(R0, loss)
    sampler = ClockSampler(torch.cuda.current_device()) if clocks else None
    if sampler:
        sampler.start()
    win = timed_windows(vm, R0, K, flush, loss, args.window_s, args.min_windows)
    clk = sampler.stop() if sampler else None
    sps = sum(r * (o["n_surface"] + o["n_strat"]) for r, o in zip(R0, objs))
    ms = median(win) / K
    out = {"value": sps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps_per_s": 1e3 / ms,
           "steps": K, "windows": len(win), "samples_per_step": sps, "objects": n_first,
           "dtype": "f32" if precision == "fp32" else "bf16+f32",
           "launch_shape": vm.get_launch() if not args.no_autotune else None,
           "roofline": roofline_of(prof, objs[:n_first], precision, peaks, props, args.prof_steps),
           "kernels": kernel_table(prof), "clocks": clk, "frozen_objects": len(vm.sync_status())}
    if admit:
        for k in range(n_first, len(objs)):
            o = objs[k]
            vm.add_object(o["pool"], hidden=o["H"], center=o["center"], scale=float(o["scale"]),
                          n_surface=o["n_surface"], n_strat=o["n_strat"], init_params=o["init"], stream_id=k)
        for _ in range(3):
            vm.step(R, loss)
        win2 = timed_windows(vm, R, K, flush, loss, args.window_s / 2, args.min_windows)
        sps2 = sum(r * (o["n_surface"] + o["n_strat"]) for r, o in zip(R, objs))
        ms2 = median(win2) / K
        out["after_admission"] = {"objects": len(objs), "admitted": admit, "value": sps2 / (ms2 * 1e-3),
                                  "ms_per_step": ms2, "samples_per_step": sps2, "windows": len(win2),
                                  "note": "admitted between steps into the captured step (no re-capture)",
                                  "frozen_objects": len(vm.sync_status())}
    vm.close()
    return out


def time_to_depth(seed=100, n_train=1000, train_steps=2000, epochs=100, n_held=200, target=0.04,
                  max_steps=2000):
    """Reduced form of the warm-start experiment (paper_2302_01838_b300.warmstart):
    the hypernetwork learns from shapes trained 2,000 steps (converged: depth-L1
    < 1 cm or 2,000 steps); for each form, steps and CUDA-event train time
    until the mean held-out depth-L1 < target, and per object the first step
    and train time at which its own depth-L1 < 1 cm (training runs on to
    max_steps for that); the final depth-L1 also with the training sampler."""
    from paper_2302_01838_b300 import scenes, warmstart as ws
    t0 = time.time()
    X, T = ws.produce_dataset(n_train, seed, train_steps)
    hyp = ws.train_hypernet(X, T, epochs=epochs)
    prep = time.time() - t0
    held = scenes.scene_shapes(seed + 10 ** 6, n_held, offmask=ws.OFFMASK)
    out = {"target_m": target, "obj_target_m": 0.01, "heldout_objects": n_held, "train_shapes": n_train,
           "train_steps_per_shape": train_steps, "hypernet_epochs": epochs, "max_steps": max_steps,
           "prep_s": round(prep, 2)}
    for form in ("plain", "batched", "warm"):
        r = ws.time_to_target(held["objects"], held["B"], seed, form, hyper=hyp if form == "warm" else None,
                              target=target, max_steps=max_steps, run_to=max_steps, guided=True)
        rnd = lambda x, n=5: None if x is None else round(x, n)
        out[form] = {"reached": r["reached"], "steps": r["steps"], "train_ms": rnd(r["train_ms"], 2),
                     "depth_l1_m": rnd(r["depth_l1_at_stop"]),
                     "frac_below_1cm": r["obj_reached_frac"], "median_steps_to_1cm": r["obj_median_steps"],
                     "median_ms_to_1cm": rnd(r["obj_median_ms"], 2), "total_steps": r["total_steps"],
                     "total_ms": rnd(r["total_ms"], 2), "final_depth_l1_m": rnd(r["final_depth_l1"]),
                     "final_depth_l1_median_m": rnd(r["final_depth_l1_median"]),
                     "final_depth_l1_guided_m": rnd(r["final_depth_l1_guided"]),
                     "final_depth_l1_guided_median_m": rnd(r["final_depth_l1_guided_median"]),
                     "final_frac_below_1cm_guided": r["frac_below_1cm_guided"],
                     "final_depth_l1_train_views_m": rnd(r["final_depth_l1_train_views"]),
                     "final_depth_l1_train_views_median_m": rnd(r["final_depth_l1_train_views_median"])}
    out["forms"] = {"plain": "FP32, kernel by kernel, seeded random init",
                    "batched": "BF16 tensor cores, CUDA graphs, autotuned, seeded random init",
                    "warm": "as batched, init predicted by the set-encoder hypernetwork"}
    out["eval"] = ("depth_l1: 96 uniform midpoints between the ray's entry and exit of the object's box, "
                   "held-out view; guided: the training sampler's depth-guided samples (Eq. 1-2) on the same "
                   "held-out rays; train_views: the uniform render on 256 rays of the training views")
    return out


def run_sweep(args):
    """The paper's scaling axes (section 4.3, Fig. vectorised-training ablation):
    step time against the object count (120 rays, hidden 32) and against the
    hidden width (50 objects x 120 rays), BF16 and FP32. One JSON line."""
    import torch
    from paper_2302_01838_b300 import scenes
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")
    pts = []

    def scene_of(n, H):
        sc = scenes.scene_small(seed=9, n_objects=n, rays=120)
        rng = __import__("numpy").random.default_rng(99)
        for o in sc["objects"]:
            o["H"] = H
            o["init"] = scenes.init_weights(rng, H)
        return sc

    axes = [("objects", n, 32) for n in (1, 10, 50, 100, 200, 1000)] + \
           [("hidden", 50, H) for H in (16, 32, 64, 128)]
    for axis, n, H in axes:
        sc = scene_of(n, H)
        for prec in ("bf16", "fp32"):
            r = measure_workload(sc, prec, args.steps, args.warmup, flush, args, peaks, props)
            pts.append({"axis": axis, "objects": n, "hidden": H, "precision": prec,
                        "ms_per_step": r["ms_per_step"], "pts_per_s": r["value"],
                        "samples_per_step": r["samples_per_step"],
                        "roofline": {k: r["roofline"][k] for k in ("kernel", "bound", "achieved", "peak", "frac")}})
            print(json.dumps(pts[-1]), flush=True, file=sys.stderr)
    print(json.dumps({"sweep": "vectorised step time vs object count and hidden width (120 rays, 22 samples)",
                      "unit": "ms/step", "points": pts}), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2302_01838_b300 import scenes, sharding

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    sc = workload(rank)
    objs = sc["objects"]
    R = [o["rays"] for o in objs]
    K = len(objs)
    sps = samples_per_step(sc)
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    vm = make_context(sc, args.precision, not args.no_autotune)
    launch = vm.get_launch() if not args.no_autotune else None
    loss = torch.empty(K, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")

    # ---- profiled kernel-by-kernel pass: per-kernel device time ----------------
    prof = profile_pass(vm, R, args.prof_steps, flush, loss)
    launches_per_step = sum(n for n, _ in prof.values()) / args.prof_steps

    # ---- the timed region: windows of exactly K steps, repeated -----------------
    if not args.no_graph:
        vm.set_graph(True)
    for _ in range(max(args.warmup, 3)):
        vm.step(R, loss)
    clocks = ClockSampler(local)
    clocks.start()
    win = timed_windows(vm, R, args.steps, flush, loss, args.window_s, args.min_windows, world)
    clk = clocks.stop()
    ms_max = median(win)
    assert np.all(np.isfinite(loss.cpu().numpy())), "non-finite loss"
    assert vm.sync_status() == [], "objects frozen during the bench"

    # ---- end to end through the C ABI with host buffers --------------------
    rng = np.random.default_rng(rank_seed(rank))
    n_batches = 4
    host_batches = []
    for _ in range(n_batches):
        parts = [o["pool"][rng.integers(0, o["pool"].shape[0], o["rays"])] for o in objs]
        host_batches.append(torch.from_numpy(np.concatenate(parts)).pin_memory())
    loss_h = torch.empty(K, dtype=torch.float32).pin_memory()
    for i in range(3):
        vm.train_step_host(host_batches[i % n_batches], R, loss_h)
    torch.cuda.synchronize()
    e2e_s = 0.0
    for i in range(args.e2e_steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vm.train_step_host(host_batches[i % n_batches], R, loss_h)
        e2e_s += time.perf_counter() - t0
    e2e_s = sharding.max_over_ranks(e2e_s)
    vm.close()

    # ---- the same workload at the other precision, side by side ------------------
    other = "bf16" if args.precision == "fp32" else "fp32"
    side = None
    if args.fp32_steps > 0 and world == 1:
        side = measure_workload(sc, other, args.steps, args.warmup, flush, args, peaks, props, clocks=True)
        side["note"] = ("room50 on the BF16 tensor-core kernels (tcgen05, FP32 accumulation, master weights, "
                        "moments, rendering and losses): the precision extension, same windows"
                        if other == "bf16" else
                        "room50 on the FP32 SIMT kernels (the paper's precision), same windows")

    # ---- the other named workloads, BF16 ------------------------------------------
    workloads = {}
    if world == 1 and not args.no_workloads:
        workloads["precision200"] = measure_workload(scenes.scene_small(seed=3, n_objects=200, rays=120), "bf16",
                                                     args.steps, args.warmup, flush, args, peaks, props)
        workloads["precision200"]["config"] = "200 objects x 120 rays x 22 samples, hidden 32, BF16 tensor cores"
        workloads["many1000"] = measure_workload(scenes.scene_many(), "bf16", args.steps, args.warmup, flush, args,
                                                 peaks, props, admit=8)
        workloads["many1000"]["config"] = ("1,000 objects, hidden {16,32,64}, rays log-uniform 16-1,024, "
                                           "samples per ray {16,22,32}, BF16, one persistent launch per width "
                                           "class (chained: each starts on the SMs the previous one frees), "
                                           "graph-replayed; 8 objects admitted after the first windows")
        workloads["many1000_fp32"] = measure_workload(scenes.scene_many(), "fp32", args.steps, args.warmup, flush,
                                                      args, peaks, props)
        workloads["many1000_fp32"]["config"] = "the same 1,000 objects on the FP32 SIMT kernels, graph-replayed"

    if rank == 0:
        value = world * sps * args.steps / (ms_max * 1e-3)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16+f32",
            "data": "synthetic",
            "steps_per_s": 1e3 * args.steps / ms_max,
            "config": {"workload": "room50: 50 objects (hidden 32, 32-600 rays) + background (hidden 128, 1200 rays), "
                                   f"22 samples/ray, {args.precision.upper()}, all objects present",
                       "precision": args.precision, "graph": not args.no_graph, "launch_shape": launch,
                       "objects_per_gpu": K, "samples_per_step_per_gpu": sps,
                       "rays_per_step_per_gpu": sum(R), "l2": "flushed (512 MB write) between timed steps",
                       "timing": f"median of {len(win)} windows of {args.steps} steps (CUDA events per step, "
                                 f"summed per window), windows repeated for >= {args.window_s} s",
                       "parallelism": f"objects sharded, {world} independent scene(s), no collective"},
            "roofline": roofline_of(prof, objs, args.precision, peaks, props, args.prof_steps),
            "kernels": kernel_table(prof),
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "e2e": {"value": world * sps * args.e2e_steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(R) * 48), "d2h_bytes_per_step": int(K * 4),
                    "api": "vmap_train_step_host (pinned host rays in, host losses out, synchronous)"},
            "clocks": clk,
        }
        if side:
            out[other] = side
        if workloads:
            out["workloads"] = workloads
        if world == 1 and not args.no_ttd:
            out["time_to_depth_l1"] = time_to_depth()
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(sc, args.cpu_steps)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
