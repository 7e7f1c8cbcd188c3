"""Benchmark: hexapod scene-steps per second on one GB300 (and N replicas under torchrun).

Workload: 4,096 independent 18-DoF hexapods (352 mass points each, flat ground, mu = 0.8,
dt = 1 ms, joints re-targeted every 80 steps to seeded sinusoids).  One benchmark step is one
npx_world_step(1000) call: 1 s of simulated time for every scene, i.e. 4.096e6 scene-steps.
The default 10 timed steps are the workload's 10 s of simulated time.

Timing: CUDA events on the world's stream around every step; between timed steps a 256 MiB
buffer is written to flush the 129 MB L2 (not timed).  `value` is whole-job throughput with the
state resident in HBM; `e2e` is the same metric through the public C-ABI with host buffers:
every step uploads the full dynamic state from pinned host memory, steps, and reads the sensors
back.  The roofline object reports the step kernel's algorithmic flops per launch -- the
floating-point operations of the plain step, counted by the oracle's counting build
(oracle/opcount.h) on a sample of the same workload -- over its measured launch time, against the
FP32 FMA peak of the part.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SCENES = 4096
CHUNK = 1000
ARENA_RADIUS = 0.01      # m, the sphere around every mass point for robot-robot contact
WORKLOAD = "hexapod_18dof_4096_scenes_flat_dt1ms_K80"
METRIC = "hexapod scene-steps/s on 1 GB300 (plain vs surrogate at stated error) + % roofline"
UNIT = "scene-steps/s"

# FP32 peak of a GB300 (152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz max SM clock)
SMS, FP32_LANES, MAX_SM_GHZ = 152, 128, 2.07
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * MAX_SM_GHZ / 1e3

# DRAM bytes (read + write) of one 1,000-step step-kernel launch, by workload and launch shape
# (lanes per scene, warps per block, blocks), from ncu (profiles/step_kernel_*_dram.md); reported
# only for a captured shape, and to be re-taken whenever the kernel changes
STEP_TRAFFIC = {
    (WORKLOAD, 8, 7, 147): 32_006_400,
    (WORKLOAD, 16, 14, 147): 31_901_440,
    ("hexapod_rough_terrain_16384_scenes", 16, 4, 456): 225_079_808,
    ("hexapod_rough_terrain_16384_scenes", 16, 2, 912): 224_312_320,
    ("hexapod_rough_terrain_16384_scenes", 16, 1, 1824): 225_149_696,
}


def counted_flops_per_scene_step(batch, n_scenes: int, n_steps: int, warm_steps: int) -> dict:
    """Algorithmic flops of the plain step: the operations the FP64 oracle's counting build
    performs (additions, multiplications, divisions, square roots, transcendental calls) on
    n_scenes scenes of the workload over n_steps after warm_steps, per scene-step, with the
    share of each part of the step."""
    from oracle.oracle import FLOP_KINDS, count_ops
    r = count_ops(batch.subset(np.arange(n_scenes)), n_steps, warm_steps=warm_steps)
    ss = r["events"]["scene_steps"]
    parts = {k: sum(v[f] for f in FLOP_KINDS) / ss for k, v in r["ops"].items() if k != "other"}
    return {"flops_per_scene_step": r["flops"] / ss, "by_part": parts,
            "sample": f"{n_scenes} scenes x {n_steps} steps after {warm_steps} (oracle counting build)"}


def job_throughput(units_per_rank: float, rank_ms: float, dist=None, device="cpu"):
    """Whole-job throughput of N replicas: each rank processed units_per_rank in rank_ms; the job
    lasts as long as its slowest rank (max over ranks), so value = N * units_per_rank / max time.
    Returns (value per second, max time in ms)."""
    import torch
    ws = dist.get_world_size() if dist else 1
    t = float(rank_ms)
    if dist:
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return ws * units_per_rank / (t / 1e3), t


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs: sampled
    every 10 ms, each line stamped on arrival; the report keeps the samples that arrived inside
    the timed region (plus the sampling interval, for the reporting lag) and says how many."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def stop(self, t0: float = None, t1: float = None) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [r for t, r in self.rows if t0 is not None and t0 <= t <= t1 + 0.02]
        rows = inside if inside else [r for _, r in self.rows]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm), "samples_in_timed_region": len(inside),
                "sampling_ms": 10}


def cpu_oracle_sample(batch, n_scenes: int, n_steps: int, threads: int) -> dict:
    """The FP64 CPU oracle as it stands on a bounded sample of the workload."""
    from oracle.oracle import time_oracle
    sub = batch.subset(np.arange(n_scenes))
    r = time_oracle(sub, n_steps, threads)
    return r


def other_workloads(World, scenes, stream, device) -> dict:
    """Scene-steps/s of 1,000-step launches, state resident in HBM, CUDA events, on:
    - one single body for 10 s (the step's latency, us_per_step);
    - the uneven mixed batch (2 s simulated after a warm-up second);
    - the evolution-scale rollout on rough terrain (the whole 60 s from the initial state, after a
      warm-up second and a reset; its fitness is the horizontal distance each robot's CoG moved);
    - the benchmark's hexapods with a joint update at every step (K = 1, the worst case; 2 s);
    - the benchmark's hexapods with both friction refinements on (2 s);
    - the same number of hexapods colliding in arenas of four (2 s), with the same robots stepped
      alone beside it and how far the collisions moved them.
    Where given, the FP64 oracle is timed beside the line on a bounded sample of its workload."""
    import torch
    out = {}
    from paper_2411_05799_gb300.npx import FRIC_TILT, FRIC_WEIGHTED
    alone = {}
    threads = os.cpu_count() or 1
    # (name, batch, seconds simulated, friction options, arena size, oracle sample (scenes, steps))
    for name, make, secs, fric, arena, sample in (
            ("single_body_1_scene", lambda: scenes.single_body(), 10, 0, 1, (1, 10 * CHUNK)),
            ("uneven_mix_65536_scenes", lambda: scenes.uneven_batch(65536), 2, 0, 1, (64, CHUNK)),
            ("hexapod_rough_terrain_16384_scenes", lambda: scenes.cpg_batch(16384), 60, 0, 1, (16, 60 * CHUNK)),
            ("hexapod_4096_scenes_K1_joint_update_every_step", lambda: scenes.hexapod_batch(N_SCENES, K=1), 2,
             0, 1, (64, CHUNK)),
            ("hexapod_4096_scenes_friction_weighted_tilt", lambda: scenes.hexapod_batch(N_SCENES), 2,
             FRIC_WEIGHTED | FRIC_TILT, 1, None),
            ("hexapod_arenas_1024x4_scenes_alone", lambda: scenes.arena_batch(N_SCENES // 4, 4), 2, 0, 1, None),
            ("hexapod_arenas_1024x4_scenes", lambda: scenes.arena_batch(N_SCENES // 4, 4), 2, 0, 4, (64, 200))):
        b = make()
        w = World.from_batch(b, stream=stream.cuda_stream, device=device)
        if fric:
            w.set_friction_model(fric)
        if arena > 1:
            w.set_arenas(arena, ARENA_RADIUS)
        w.autotune(100)
        w.configure(chunk_steps=CHUNK)
        start = w.export_state()
        c0 = w.read()["cog"]
        w.step(CHUNK)
        w.import_state(start)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        w.step(secs * CHUNK)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        info = w.info()
        r = w.read()
        out[name] = {"value": b.n_scenes * secs * CHUNK / (ms / 1e3), "unit": UNIT, "steps": secs * CHUNK,
                     "ms": ms, "points": b.n_points, "lanes_per_scene": info["lanes_per_scene"],
                     "size_classes": info["size_classes"],
                     "warps_per_block": info["warps_per_block"],
                     "frozen_scenes": int((r["status"] != 0).sum())}
        if b.n_scenes == 1:
            out[name]["us_per_step"] = ms * 1e3 / (secs * CHUNK)     # latency of one scene's step
        if sample is not None:
            n_sc, n_st = sample
            th = min(threads, n_sc // arena)
            if arena > 1:
                # the colliding regime: 600 untimed steps first (the robots walk into each other)
                from oracle.oracle import Oracle
                o = Oracle(b.subset(np.arange(n_sc)), threads=th, arena=arena, arena_radius=ARENA_RADIUS)
                o.step(600)
                t0 = time.perf_counter()
                o.step(n_st)
                v_o = n_sc * n_st / (time.perf_counter() - t0)
                what = f"{n_sc} scenes ({n_sc // arena} arenas) x {n_st} steps after 600 untimed steps (FP64)"
            else:
                v_o = cpu_oracle_sample(b, n_sc, n_st, th)["scene_steps_per_s"]
                what = f"{n_sc} scenes x {n_st} steps of this workload (FP64)"
            out[name]["cpu_baseline"] = {"value": v_o, "unit": UNIT, "cores": th, "kind": "oracle", "sample": what}
        if name.endswith("_alone"):
            alone = {"cog": r["cog"].copy(), "value": out[name]["value"]}
            del out[name]
        elif arena > 1:
            d = np.linalg.norm(r["cog"][:, :2] - alone["cog"][:, :2], axis=1)
            out[name].update({"arena": arena, "contact_radius_m": ARENA_RADIUS,
                              "alone_value": alone["value"],
                              "cog_shift_by_collisions_m": {"what": "horizontal distance between each robot's CoG "
                                                                    "and its CoG stepped alone, after 2 s",
                                                            "median": float(np.median(d)),
                                                            "p90": float(np.percentile(d, 90))}})
        if name.startswith("hexapod_rough_terrain"):
            # roofline of the height-map kernel: counted algorithmic flops, and the DRAM traffic of
            # one 1,000-step launch (ncu) against the measured HBM bandwidth
            fl = counted_flops_per_scene_step(b, 16, CHUNK, CHUNK)
            launch_ms = ms / secs
            achieved = fl["flops_per_scene_step"] * b.n_scenes * CHUNK / (launch_ms / 1e3) / 1e12
            shape = (name, info["lanes_per_scene"], info["warps_per_block"], info["blocks"])
            traffic = STEP_TRAFFIC.get(shape)
            hbm = _measured_peaks().get("hbm_gbs")
            out[name]["roofline"] = {
                "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic, "kernel": "step_kernel_hm",
                "launch_ms": launch_ms, "flops_per_scene_step": fl["flops_per_scene_step"],
                "flops_by_part": fl["by_part"], "flops_source": fl["sample"],
                "peak_note": "FP32 FMA peak from unit counts and max SM clock (derived)",
                "hbm": None if traffic is None or not hbm else {
                    "achieved_gbs": traffic / (launch_ms / 1e3) / 1e9, "peak_gbs": hbm,
                    "frac": traffic / (launch_ms / 1e3) / 1e9 / hbm,
                    "peak_note": "MEASURED_PEAKS.json hbm_gbs, of measured"}}
        if secs == 60:
            d = np.linalg.norm(r["cog"][:, :2] - c0[:, :2], axis=1)
            # untimed replay of the same rollout (stepping is deterministic), sampled every 0.1 s:
            # a robot counts as launched when its CoG rose more than 0.2 m above its start height
            # (penalty-force spikes under fast gaits throw some robots), and the fitness is split
            w.import_state(start)
            w.configure(chunk_steps=100)
            rise = np.zeros(b.n_scenes)
            for _ in range(secs * CHUNK // 100):
                w.step(100)
                rise = np.maximum(rise, w.read()["cog"][:, 2] - c0[:, 2])
            same = bool(np.array_equal(w.read()["cog"], r["cog"]))
            launched = rise > 0.2

            def stats(m):
                x = d[m]
                return {"robots": int(m.sum()), "median": float(np.median(x)) if len(x) else None,
                        "p90": float(np.percentile(x, 90)) if len(x) else None,
                        "max": float(x.max()) if len(x) else None}
            out[name]["fitness_m"] = {"what": "horizontal distance of the robot CoG from its start after 60 s",
                                      "median": float(np.median(d)), "p90": float(np.percentile(d, 90)),
                                      "max": float(d.max()),
                                      "split": {"what": "robots whose CoG rose more than 0.2 m above its start "
                                                        "height at some 0.1 s sample (launched) and the rest",
                                                "stayed_low": stats(~launched), "launched": stats(launched),
                                                "replay_bit_identical": same}}
        w.close()
        del b
    return out


def simplify_leg(World, stream, device) -> dict:
    """simplifyMode (Sec. III-D): the hexapod built from a torso box and 18 cylinder segments,
    4,096 copies with seeded sinusoid targets, in each simplify mode; scene-steps/s of 1,000-step
    launches (2 s simulated after a warm-up second), points per scene beside it."""
    import torch
    from paper_2411_05799_gb300 import construct
    out = {}
    for mode in (0, 1, 2, 3):
        rb = construct.cylinder_hexapod(mode)
        z0 = -float(rb.batch(1).p0[:, 2].min()) + 0.01
        rng = np.random.default_rng(50)
        J = 18 * N_SCENES
        act = np.stack([rng.uniform(0, 0.5, J), rng.uniform(0.5, 2.0, J), rng.uniform(0, 2 * np.pi, J),
                        np.zeros(J)], 1)
        b = rb.batch(N_SCENES, origin=(0.0, 0.0, z0), act_params=act)
        w = World.from_batch(b, stream=stream.cuda_stream, device=device)
        w.autotune(100)
        w.configure(chunk_steps=CHUNK)
        w.step(CHUNK)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        w.step(2 * CHUNK)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[f"mode_{mode}"] = {"value": N_SCENES * 2 * CHUNK / (ms / 1e3), "unit": UNIT,
                               "points_per_scene": b.n_points // N_SCENES,
                               "frozen_scenes": int((w.read()["status"] != 0).sum())}
        w.close()
    return out


def gp_evolution_leg(scenes, stream, n_groups: int = 160, generations: int = 3) -> dict:
    """The paper's own workload (Sec. IV): machine-code controllers of the hexapod evolved by
    mutation, best 50 of 100 kept, two-minute evaluations; here n_groups populations side by side
    in one world.  Scene-steps/s over the evaluations and the best fitness per generation."""
    from paper_2411_05799_gb300 import evolution
    t0 = time.perf_counter()
    res = evolution.evolve(n_groups=n_groups, pop=100, keep=50, generations=generations,
                           eval_seconds=120.0, seed=11, stream=stream.cuda_stream)
    wall = time.perf_counter() - t0
    best = res["best_fitness"]
    out = {"workload": f"gp_hexapod_{n_groups}x100_robots_2min_evaluations", "unit": UNIT,
           "value": res["scene_steps"] / res["step_seconds"], "generations": generations,
           "populations": n_groups, "robots": n_groups * 100,
           "seconds_per_generation": res["step_seconds"] / generations, "wall_seconds": round(wall, 2),
           "best_fitness_m": {"median_over_populations": [float(np.median(b)) for b in best],
                              "max": [float(b.max()) for b in best]}}
    res["world"].close()
    return out


def _measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def surrogate_leg(World, scenes, stream, device, n_transitions: int, stride: int = 1) -> dict:
    """The learned surrogate: trained on n_transitions transitions (windows of `stride` steps) of
    the 4,096-hexapod workload, then stepping 65,536 hexapods (joint-update steps, the steps left
    before them and scenes whose foot contacts change over a window are taken by the plain step);
    its throughput beside the plain step's on the same scenes, its 50-step error against the FP64
    oracle on 256 held-out scenes, and its network's forward pass against the bf16 tensor peak.
    Windows longer than one step are also timed and evaluated with the rule that never falls back
    (`never_fall_back`): the throughput the network alone gives, at its own stated error."""
    import torch
    from oracle.oracle import Oracle
    from paper_2411_05799_gb300 import npx, surrogate
    S, PERIOD = 65536, 80
    res = surrogate.train(scenes.hexapod_batch(4096, seed_key=40), n_transitions=n_transitions,
                          passes=2, lr=1e-3, max_batch=S, stride=stride)
    sur = res["surrogate"]
    big = scenes.hexapod_batch(S, seed_key=5)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    out = {"workload": f"hexapod_18dof_{S}_scenes_flat_dt1ms_K80", "unit": UNIT, "stride": stride}

    def timed(fn, reps):
        ms = 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize(device)
            ms += e0.elapsed_time(e1)
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
        return ms, r

    # plain step on the same scenes (1,000-step chunks)
    w = World.from_batch(big, stream=stream.cuda_stream, device=device.index or 0)
    w.autotune(100)
    w.configure(chunk_steps=CHUNK)
    w.step(CHUNK)
    ms, _ = timed(lambda: w.step(CHUNK), 2)
    out["plain_value"] = S * 2 * CHUNK / (ms / 1e3)
    # surrogate steps: whole joint-update periods from the step after a joint update (n mod K = 1:
    # the windows, then the plain steps up to and through the next joint update), after one
    # warm-up period; for each fallback rule
    w.step((1 - w.info()["step"]) % PERIOD)

    def time_rule(bits):
        npx.surrogate_set_fallback(w, bits)
        sur.step(w, PERIOD)
        fb_total, reps, ms = 0, 4, 0.0
        for _ in range(reps):
            m, fb = timed(lambda: sur.step(w, PERIOD), 1)
            ms += m
            fb_total += fb
        return {"value": S * PERIOD * reps / (ms / 1e3), "ms_per_step": ms / (PERIOD * reps),
                "fallback_fraction": fb_total / (S * PERIOD * reps)}

    rules = {"any_change": 0} if stride == 1 else {"any_change": 0, "more_than_one": 1, "never": -1}
    timing = {name: time_rule(bits) for name, bits in rules.items()}
    out.update(timing["any_change"])
    out["frozen_scenes"] = int((w.read()["status"] != 0).sum())
    w.close()
    # the network's forward pass over all scenes: five BF16 GEMMs with fused epilogues
    x = torch.zeros(S, sur.n_in, device=device)
    y = torch.empty(S, sur.n_out, device=device)
    net_stream = torch.cuda.ExternalStream(sur.stream, device=device)
    sur.net.forward(x.data_ptr(), y.data_ptr(), S)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(net_stream)
    for _ in range(reps):
        sur.net.forward(x.data_ptr(), y.data_ptr(), S)
    e1.record(net_stream)
    torch.cuda.synchronize(device)
    fwd_ms = e0.elapsed_time(e1) / reps
    n_in, H, n_out = sur.n_in, surrogate.N_HIDDEN, sur.n_out
    flops = 2.0 * S * (n_in * H + (surrogate.N_LAYERS - 1) * H * H + H * n_out)
    peak = _measured_peaks().get("bf16_tflops")
    achieved = flops / (fwd_ms / 1e3) / 1e12
    out["roofline"] = {"bound": "tensor", "kernel": "gemm_tn_kernel (network forward, 5 launches)",
                       "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak if peak else None, "traffic": None,
                       "flops_per_scene_step": flops / S,
                       "peak_note": "MEASURED_PEAKS.json bf16_tflops (burst), of measured"}
    out["forward_ms"] = fwd_ms
    # 50-step error against the FP64 oracle, from a mid-gait state of 256 held-out scenes: the step
    # after a joint update (n mod K = 1), so that the 50 steps hold as many whole windows as fit
    test_b = scenes.hexapod_batch(256, seed_key=41)
    o = Oracle(test_b, threads=os.cpu_count() or 1)
    o.step(1041)
    ref = Oracle(test_b, threads=os.cpu_count() or 1)
    ref.copy_state_from(o)
    ref.step(50)
    def errors(dc, ang):
        if len(dc) == 0:
            return {"scenes": 0}
        return {"scenes": int(len(dc)), "cog_m_median": float(np.median(dc)),
                "cog_m_rms": float(np.sqrt(np.mean(dc ** 2))), "cog_m_p90": float(np.percentile(dc, 90)),
                "angle_rad_median": float(np.median(ang)), "angle_rad_rms": float(np.sqrt(np.mean(ang ** 2))),
                "angle_rad_p90": float(np.percentile(ang, 90))}

    def rollout_errors(bits):
        err = {}
        for name, fn in (("surrogate", lambda ww: sur.step(ww, 50)),
                         ("plain", lambda ww: ww.step(50))):
            ww = World.from_batch(test_b, stream=stream.cuda_stream, device=device.index or 0)
            ww.write_state(o.c.astype(np.float32), o.q.astype(np.float32), o.v.astype(np.float32),
                           o.L.astype(np.float32), o.theta.astype(np.float32),
                           o.kappa.astype(np.uint8), o.n)
            if name == "surrogate":
                npx.surrogate_set_fallback(ww, bits)
                npx.surrogate_fallback_counts(ww)        # counters from zero
            fb = fn(ww)
            r = ww.read()
            dc = np.linalg.norm(r["cog"] - ref.c, axis=1)
            qa, qb = r["quat"].astype(np.float64), ref.q
            ang = 2 * np.arctan2(np.linalg.norm(qa - qb, axis=1), np.linalg.norm(qa + qb, axis=1))
            ang = np.minimum(ang, 2 * np.pi - ang)
            err[name] = errors(dc, ang)
            if name == "surrogate":
                # scene-steps of the 50 that the plain step took (fallbacks), and the error of the
                # scenes the network carried through every window of the 50 steps apart from those
                # whose windows (some or all) the plain step redid
                err[name]["fallback_fraction"] = fb / (test_b.n_scenes * 50)
                stayed = npx.surrogate_fallback_counts(ww) == 0
                err[name]["stayed_on_network"] = errors(dc[stayed], ang[stayed])
                err[name]["fell_back_at_least_once"] = errors(dc[~stayed], ang[~stayed])
            ww.close()
        return err

    err = rollout_errors(0)
    out["error_50_steps_vs_fp64_oracle"] = err
    out["stated_error"] = {"what": "50-step CoG and orientation error against the FP64 oracle of the "
                                   "held-out scenes the network carried through every window",
                           **err["surrogate"]["stayed_on_network"]}
    if "more_than_one" in timing:
        # a looser rule: a window falls back only when two or more foot sensors change
        e1 = rollout_errors(1)
        out["fall_back_on_two_changes"] = {
            "what": "the same network with npx_surrogate_set_fallback(1): a window falls back when more "
                    "than one contact sensor changes over it",
            **timing["more_than_one"], "plain_value": out["plain_value"],
            "error_50_steps_vs_fp64_oracle": e1,
            "stated_error": {"what": "50-step CoG and orientation error against the FP64 oracle of the "
                                     "held-out scenes the network carried through every window",
                             **e1["surrogate"]["stayed_on_network"]}}
    if "never" in timing:
        # the looser rule: no window falls back, so every held-out scene is the network's
        e2 = rollout_errors(-1)
        out["never_fall_back"] = {
            "what": "the same network with npx_surrogate_set_fallback(-1): every window keeps the "
                    "network's prediction (sensors read at the predicted state)",
            **timing["never"], "plain_value": out["plain_value"],
            "error_50_steps_vs_fp64_oracle": e2,
            "stated_error": {"what": "50-step CoG and orientation error against the FP64 oracle of all "
                                     "held-out scenes (none falls back)", **e2["surrogate"]}}
    u = res["unexplained"]
    out["training"] = {"transitions": int(res["transitions"]), "adam_steps": int(res["adam_steps"]),
                       "seconds": round(res["seconds"], 2), "scenes": 4096,
                       "held_out_unexplained_variance": float(np.mean(u[-5:]))}
    return out


def bench_config(ws: int) -> dict:
    """The workload of one benchmark step, the same dict in both arms."""
    return {"workload": WORKLOAD, "scenes_per_gpu": N_SCENES, "steps_per_bench_step": CHUNK,
            "dt": 1e-3, "K": 80, "parallelism": f"replicas{ws}",
            "l2": "GPU arm: flushed between timed steps (256 MiB write); CPU arm: not applicable"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, as it stands, on all host cores, stepping the whole
    workload: every benchmark step advances all 4,096 hexapods by 1,000 steps (the simulation
    continues from step to step, as in the GPU arm), timed with a wall clock around each step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2411_05799_gb300 import scenes
    from oracle.oracle import Oracle
    from oracle.oracle import build as build_oracle
    build_oracle()
    threads = os.cpu_count() or 1
    o = Oracle(scenes.hexapod_batch(N_SCENES), threads=threads)
    for _ in range(args.warmup):
        o.step(CHUNK)
    secs = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cnt = o.step(CHUNK)
        secs.append(time.perf_counter() - t0)
        assert cnt["scene_steps"] == N_SCENES * CHUNK
    total = float(sum(secs))
    value = N_SCENES * CHUNK * args.steps / total
    sample = (f"the whole workload: all {N_SCENES} hexapods x {CHUNK} steps per benchmark step, "
              f"{threads} threads (FP64)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(ws),
            "frozen_scenes": int((o.status != 0).sum()),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    from paper_2411_05799_gb300 import scenes
    from paper_2411_05799_gb300.build import build
    from paper_2411_05799_gb300.npx import World

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    stream = torch.cuda.Stream(device=dev)
    batch = scenes.hexapod_batch(N_SCENES)
    world = World.from_batch(batch, stream=stream.cuda_stream, device=local)
    tune = world.autotune(200)
    world.configure(chunk_steps=CHUNK)
    info = world.info()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def l2_flush():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)

    for _ in range(args.warmup):
        world.step(CHUNK)
    world.sync()
    l2_flush()
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    launches0 = world.info()["kernel_launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    t_begin = time.perf_counter()
    for i in range(args.steps):
        ev[i][0].record(stream)
        world.step(CHUNK)
        ev[i][1].record(stream)
        l2_flush()
    torch.cuda.synchronize(dev)
    t_end = time.perf_counter()
    time.sleep(0.03)   # the samples of the region's last moments arrive
    clk = clocks.stop(t_begin, t_end)
    per_step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(per_step_ms))
    launches = world.info()["kernel_launches"] - launches0
    value, total_ms = job_throughput(N_SCENES * CHUNK * args.steps, total_ms, dist, dev)
    if dist:
        dist.barrier()
    status = world.read()["status"]

    # ---- end to end through the C-ABI with host buffers: every step writes the state read back
    # by the previous one (pinned host arrays), steps, and reads the state and the per-point contact
    # flags back -- the simulation continues as in the timed region above
    e2e_steps = max(1, min(args.steps, 5))
    io = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in world.read_buffers().items()}
    kap = torch.zeros(info["n_points"], dtype=torch.uint8).pin_memory().numpy()
    io = world.read(out=io)
    world.contacts(out=kap)
    h2d = sum(io[k].nbytes for k in ("cog", "quat", "vel", "angmom", "theta")) + kap.nbytes + 8
    d2h = sum(v.nbytes for v in io.values() if isinstance(v, np.ndarray)) + 8 + kap.nbytes
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        world.write_state(io["cog"], io["quat"], io["vel"], io["angmom"], io["theta"], kap, io["step"])
        world.step(CHUNK)
        io = world.read(out=io)
        world.contacts(out=kap)
    e2e_s = time.perf_counter() - t0
    e2e_val, _ = job_throughput(N_SCENES * CHUNK * e2e_steps, e2e_s * 1e3, dist, dev)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(ws),
            "launch": {"lanes_per_scene": info["lanes_per_scene"],
                       "warps_per_block": info["warps_per_block"], "blocks": info["blocks"],
                       "size_classes": info["size_classes"]},
            "frozen_scenes": int((status != 0).sum()),
            "gpu_launches": int(launches + args.steps),   # step-kernel launches + step-counter kernels
            "clocks": clk,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "steps": e2e_steps}}

    # ---- the other batched workloads: throughput of the same step on the uneven 65,536-scene
    # mix and on 16,384 hexapods walking on rough height fields (informational)
    if rank == 0 and not args.no_extra:
        line["other_workloads"] = other_workloads(World, scenes, stream, local)
    if rank == 0 and not args.no_surrogate:
        line["surrogate"] = surrogate_leg(World, scenes, stream, dev, args.surrogate_transitions,
                                          args.surrogate_stride)
        # the configuration's one-step reading: a network predicting the next step's state
        line["surrogate"]["stride_1"] = surrogate_leg(World, scenes, stream, dev, args.surrogate_transitions_1, 1)
    if not args.no_extra and rank == 0:
        line["gp_evolution"] = gp_evolution_leg(scenes, stream)
        line["simplify_modes"] = simplify_leg(World, stream, local)

    if rank == 0:
        # algorithmic flops per scene-step: the oracle's counted operations on a sample
        n_sc, n_st = 1024, 1000
        threads = os.cpu_count() or 1
        r = cpu_oracle_sample(batch, n_sc, n_st, threads)
        fl = counted_flops_per_scene_step(batch, 64, 2 * CHUNK, CHUNK)
        flops_per_ss = fl["flops_per_scene_step"]
        launch_ms = total_ms / max(1, launches)
        achieved = flops_per_ss * N_SCENES * CHUNK / (launch_ms / 1e3) / 1e12
        shape = (WORKLOAD, info["lanes_per_scene"], info["warps_per_block"], info["blocks"])
        line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                            "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                            "traffic": STEP_TRAFFIC.get(shape) if CHUNK == 1000 else None,
                            "kernel": "step_kernel", "launch_ms": launch_ms,
                            "flops_per_scene_step": flops_per_ss, "flops_by_part": fl["by_part"],
                            "flops_source": fl["sample"],
                            "peak_note": "FP32 FMA peak from unit counts and max SM clock (derived)"}
        r1 = cpu_oracle_sample(batch, 64, 1000, 1)     # the paper's setting: one CPU thread
        line["cpu_baseline"] = {"value": r["scene_steps_per_s"], "unit": UNIT, "cores": threads,
                                "kind": "oracle",
                                "sample": f"{n_sc} of {N_SCENES} hexapods x {n_st} steps (FP64)",
                                "single_thread": {"value": r1["scene_steps_per_s"], "unit": UNIT,
                                                  "sample": f"64 of {N_SCENES} hexapods x 1000 steps"}}
        print(json.dumps(line), flush=True)
    world.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_profile(args):
    """ncu drivers (print no benchmark line).
    step:      a few step-kernel launches of `--chunk` steps on the benchmark workload in a fixed
               launch shape;
    step_hm:   the same on the rough-terrain rollout (16,384 hexapods, 128 x 128 height maps);
    arena:     the same on 4,096 hexapods colliding in arenas of four (after 600 untimed steps of
               walking into each other);
    uneven:    the uneven 65,536-scene mix in its autotuned size classes, three chunks, the last
               inside the NVTX range "chunk";
    gemm:      the surrogate network's forward GEMMs over 65,536 rows (random weights), 3 passes;
    surrogate: a briefly trained surrogate stepping 65,536 hexapods from the step after a joint
               update for one joint-update period (4 steps at stride 1) with the fallback rule
               --fallback-bits, inside the NVTX range "period"."""
    import torch
    from paper_2411_05799_gb300 import scenes
    from paper_2411_05799_gb300.build import build
    from paper_2411_05799_gb300.npx import World
    build()
    torch.cuda.set_device(0)
    if args.profile == "uneven":
        world = World.from_batch(scenes.uneven_batch(65536))
        world.autotune(100)
        world.configure(chunk_steps=args.chunk)
        world.step(2 * args.chunk)
        world.sync()
        torch.cuda.nvtx.range_push("chunk")
        world.step(args.chunk)
        world.sync()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile": args.profile, **world.info(),
                          "status_nonzero": int((world.read()["status"] != 0).sum())}))
        world.close()
        return 0
    if args.profile in ("step", "step_hm", "arena"):
        batch = {"step": lambda: scenes.hexapod_batch(args.scenes or N_SCENES),
                 "step_hm": lambda: scenes.cpg_batch(args.scenes or 16384),
                 "arena": lambda: scenes.arena_batch(N_SCENES // 4, 4)}[args.profile]()
        world = World.from_batch(batch, configure=dict(lanes_per_scene=args.lps, warps_per_block=args.wpb,
                                                       chunk_steps=args.chunk))
        if args.profile == "arena":
            world.set_arenas(4, ARENA_RADIUS)
            world.configure(lanes_per_scene=args.lps, warps_per_block=args.wpb, chunk_steps=args.chunk)
            world.step(600)
        for _ in range(3):
            world.step(args.chunk)
        world.sync()
        print(json.dumps({"profile": args.profile, **world.info(),
                          "status_nonzero": int((world.read()["status"] != 0).sum())}))
        world.close()
        return 0
    from paper_2411_05799_gb300 import npx, surrogate
    S = 65536
    if args.profile == "gemm":
        stream = torch.cuda.Stream()
        net = npx.MLP(271, 247, n_hidden=surrogate.N_HIDDEN, n_hidden_layers=surrogate.N_LAYERS,
                      max_batch=S, stream=stream.cuda_stream)
        with torch.cuda.stream(stream):
            x = torch.randn(S, 271, device="cuda")
            y = torch.empty(S, 247, device="cuda")
            for _ in range(3):
                net.forward(x.data_ptr(), y.data_ptr(), S)
            stream.synchronize()
        print(json.dumps({"profile": "gemm", "rows": S, "finite": bool(torch.isfinite(y).all())}))
        return 0
    stride = args.surrogate_stride
    res = surrogate.train(scenes.hexapod_batch(4096, seed_key=40), n_transitions=65536 * 8,
                          passes=2, stat_periods=1, warm_steps=100, max_batch=S, stride=stride)
    sur = res["surrogate"]
    stream = torch.cuda.Stream()
    n = 4 if stride == 1 else 80      # stride 1: four steps; else one joint-update period
    with torch.cuda.stream(stream):
        w = World.from_batch(scenes.hexapod_batch(S, seed_key=5), stream=stream.cuda_stream)
        npx.surrogate_set_fallback(w, args.fallback_bits)
        w.step(321)
        stream.synchronize()
        torch.cuda.nvtx.range_push("period")
        fb = sur.step(w, n)
        stream.synchronize()
        torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile": "surrogate", "scenes": S, "steps": n, "stride": stride,
                      "fallback_bits": args.fallback_bits, "fallbacks": fb}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile", choices=["step", "step_hm", "arena", "uneven", "gemm", "surrogate"],
                    help="ncu driver (no bench line): step kernel (4,096 hexapods on flat ground, or "
                         "16,384 on rough height maps), network GEMMs or surrogate step")
    ap.add_argument("--lps", type=int, default=16)
    ap.add_argument("--scenes", type=int, default=0, help="step profiles: scenes (0: the workload's own)")
    ap.add_argument("--fallback-bits", type=int, default=0,
                    help="surrogate profile: fallback when more contact sensors change (-1: never)")
    ap.add_argument("--wpb", type=int, default=16)
    ap.add_argument("--chunk", type=int, default=100)
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-surrogate leg")
    ap.add_argument("--surrogate-transitions", type=int, default=100_000_000)
    ap.add_argument("--surrogate-stride", type=int, default=25,
                    help="steps per surrogate prediction (window between joint updates); 25: two "
                         "windows make the 50-step horizon")
    ap.add_argument("--surrogate-transitions-1", type=int, default=20_000_000,
                    help="training transitions of the one-step (stride 1) surrogate line")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
