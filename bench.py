#!/usr/bin/env python
"""Throughput of the vectorised object-MLP training step (vMAP, section 3.2).

Workload ("room50"): 50 object MLPs (hidden 32, rays per object log-uniform
in 32-600) plus one background MLP (hidden 128, 1,200 rays), 22 samples per
ray, every object present (the steady state after the last incremental
insertion). One step = ray picking + depth-guided sampling + encoding + MLP
forward + rendering + losses + backward + Adam for all 51 objects.

Default path: BF16 tensor-core GEMMs with FP32 accumulation, master weights,
moments, rendering and losses, the step replayed as CUDA graphs, launch
shapes autotuned. The same line reports the plain FP32 path on the same
workload, a profiled kernel-by-kernel pass (per-kernel time and the roofline
of the dominant kernel), and the time to a held-out depth-L1 target of
plain FP32 vs BF16 + batched vs BF16 + batched + warm start.

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
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="bf16",
                    help="bf16: tcgen05 BF16 GEMMs, FP32 accumulation (default); fp32: plain FP32 SIMT path")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch kernel by kernel instead of graph replay")
    ap.add_argument("--prof-steps", type=int, default=200, help="steps of the profiled kernel-by-kernel pass")
    ap.add_argument("--fp32-steps", type=int, default=300, help="steps of the FP32 comparison (0: skip)")
    ap.add_argument("--no-ttd", action="store_true", help="skip the time-to-depth-L1 comparison")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=12, help="oracle steps of the CPU baseline sample")
    ap.add_argument("--e2e-steps", type=int, default=1000)
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
    the width-128 path splits its two kernels."""
    F = 93 * H + 3 * H * H + 4 * H
    fb, dw = 2 * (F + 3 * H * H + 4 * H), 2 * F
    return {"all": fb + dw, "fb": fb, "dw": dw}[part]


def kernel_flops(name, objs):
    """Algorithmic flops of one launch of a tile kernel on the workload."""
    H = int(name.split("<")[1].rstrip(">"))
    part = "fb" if name.startswith("k_wide_fb") else "dw" if name.startswith("k_wide_dw") else "all"
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
        self.index = index
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


def make_context(sc, precision, autotune, reps=3):
    from paper_2302_01838_b300.api import VMap
    from paper_2302_01838_b300.native import VMAP_BF16, VMAP_FP32
    objs = sc["objects"]
    R = [o["rays"] for o in objs]
    prec = VMAP_BF16 if precision == "bf16" else VMAP_FP32
    vm = VMap(max_objects=len(objs) + 8, max_rays_total=2 * sum(R),
              max_pool_rays=sum(o["pool"].shape[0] for o in objs) + 16, B=sc["B"], seed=sc["seed"], precision=prec)
    for k, o in enumerate(objs):
        vm.add_object(o["pool"], hidden=o["H"], center=o["center"], scale=float(o["scale"]),
                      n_surface=o["n_surface"], n_strat=o["n_strat"], init_params=o["init"], stream_id=k)
    if autotune:
        vm.autotune(R, reps=reps)
    return vm


def timed_steps(vm, R, steps, flush, loss):
    """Device milliseconds of `steps` steps, L2 flushed between steps (outside the intervals)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record()
        vm.step(R, loss)   # sample_rays + train_step as one launch sequence
        ev[i][1].record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev)


def time_to_depth(seed=100, n_train=1000, train_steps=1000, epochs=100, n_held=200, target=0.04):
    """Reduced form of the warm-start experiment (paper_2302_01838_b300.warmstart):
    steps and CUDA-event train time until the mean held-out depth-L1 < target."""
    from paper_2302_01838_b300 import scenes, warmstart as ws
    t0 = time.time()
    X, T = ws.produce_dataset(n_train, seed, train_steps)
    hyp = ws.train_hypernet(X, T, epochs=epochs)
    prep = time.time() - t0
    held = scenes.scene_shapes(seed + 10 ** 6, n_held, offmask=ws.OFFMASK)
    out = {"target_m": target, "heldout_objects": n_held, "train_shapes": n_train,
           "train_steps_per_shape": train_steps, "hypernet_epochs": epochs, "prep_s": round(prep, 2)}
    for form in ("plain", "batched", "warm"):
        r = ws.time_to_target(held["objects"], held["B"], seed, form, hyper=hyp if form == "warm" else None,
                              target=target)
        out[form] = {"reached": r["reached"], "steps": r["steps"], "train_ms": round(r["train_ms"], 2),
                     "depth_l1_m": round(r["final_depth_l1"], 5)}
    out["forms"] = {"plain": "FP32, kernel by kernel, seeded random init",
                    "batched": "BF16 tensor cores, CUDA graphs, autotuned, seeded random init",
                    "warm": "as batched, init predicted by the set-encoder hypernetwork"}
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2302_01838_b300 import sharding

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    sc = workload(rank)
    objs = sc["objects"]
    R = [o["rays"] for o in objs]
    K = len(objs)
    sps = samples_per_step(sc)
    vm = make_context(sc, args.precision, not args.no_autotune)
    launch = vm.get_launch() if not args.no_autotune else None
    loss = torch.empty(K, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")

    # ---- profiled kernel-by-kernel pass: per-kernel device time ----------------
    for _ in range(3):
        vm.step(R, loss)
    vm.profile_reset()
    vm.profile_enable(True)
    timed_steps(vm, R, args.prof_steps, flush, loss)
    vm.profile_enable(False)
    prof = vm.profile()
    launches_per_step = sum(n for n, _ in prof.values()) / args.prof_steps

    # ---- the timed region -------------------------------------------------------
    if not args.no_graph:
        vm.set_graph(True)
    for _ in range(max(args.warmup, 3)):
        vm.step(R, loss)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed_steps(vm, R, args.steps, flush, loss)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_max = sharding.max_over_ranks(ms)
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

    # ---- the plain FP32 path on the same workload --------------------------------
    fp32 = None
    if args.precision == "bf16" and args.fp32_steps > 0:
        v32 = make_context(sc, "fp32", not args.no_autotune)
        if not args.no_graph:
            v32.set_graph(True)
        for _ in range(3):
            v32.step(R, loss)
        ms32 = sharding.max_over_ranks(timed_steps(v32, R, args.fp32_steps, flush, loss))
        v32.close()
        fp32 = {"value": world * sps * args.fp32_steps / (ms32 * 1e-3), "unit": UNIT,
                "ms_per_step": ms32 / args.fp32_steps, "steps_per_s": 1e3 * args.fp32_steps / ms32,
                "steps": args.fp32_steps}

    if rank == 0:
        peaks = measured_peaks()
        props = torch.cuda.get_device_properties(local)
        sm_max = peaks.get("sm_max_mhz", 2032.0)
        fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        tiles = {k: v for k, v in prof.items() if k.startswith(("k_tile", "k_wide"))}
        dom = max(tiles, key=lambda k: tiles[k][1])
        flops = kernel_flops(dom, objs)
        n_l, dom_ms = tiles[dom]
        achieved = flops / (dom_ms / n_l * 1e-3) / 1e12
        tensor = dom.startswith(("k_tile_bf16", "k_wide"))
        if tensor:
            peak, bound = peaks.get("bf16_tflops", 1800.0), "tensor"
            peak_note = "measured cuBLAS BF16 burst (MEASURED_PEAKS.json bf16_tflops)"
        else:
            peak, bound = fp32_peak, "alu"
            peak_note = f"FP32 FFMA: {props.multi_processor_count} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz"
        total_prof = sum(v[1] for v in prof.values())
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
                       "parallelism": f"objects sharded, {world} independent scene(s), no collective"},
            "roofline": {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic_for(dom),
                         "peak_note": peak_note, "flops_per_launch": flops, "avg_launch_ms": dom_ms / n_l,
                         "timing": f"CUDA events around each launch, {args.prof_steps}-step kernel-by-kernel pass"},
            "kernels": {k: {"launches": n, "total_ms": round(t_, 4), "share": round(t_ / total_prof, 4)}
                        for k, (n, t_) in prof.items()},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "e2e": {"value": world * sps * args.e2e_steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(R) * 48), "d2h_bytes_per_step": int(K * 4),
                    "api": "vmap_train_step_host (pinned host rays in, host losses out, synchronous)"},
            "clocks": clk,
        }
        if fp32:
            out["fp32"] = fp32
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
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
