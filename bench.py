"""Benchmark: env-steps/s of the batched physics step (8192-world humanoid).

One step = one environment step (push event + 4 physics substeps) of every world,
one persistent launch. Timing: W warm-up steps, then K steps each bracketed by
CUDA events on the launching stream, with a 256 MB L2 flush between timed steps
(outside the events). Under torchrun each rank runs the full workload on its own
GPU (worlds are independent: weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload humanoid8192]
    python bench.py --impl reference      # the FP64 oracle on the host cores
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s, 8192-world 35-DoF humanoid; served-rollout p50/p99 latency"
WORKLOADS = {
    "humanoid8192": ("humanoid", 8192, 4),
    "quadruped4096": ("quadruped", 4096, 4),
    "pendulum64": ("pendulum", 64, 1),
}
PREROLL = 100          # untimed env steps so the robots reach their contact-rich steady state
FP32_LANES_PER_SM, NSM = 128, 148


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("sm_max_mhz", 2032.0), p.get("hbm_gbs", 6400.0), "measured"
    except Exception:
        return 2032.0, 6400.0, "fallback"


def start_clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def read_clocks(path, dev_index):
    mhz, maxmhz, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9 or c[0] != str(dev_index):
                continue
            mhz.append(float(c[1]))
            maxmhz = max(maxmhz, float(c[2]))
            for n, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
    except Exception:
        pass
    return {"sm_mhz": float(np.median(mhz)) if mhz else None, "sm_max_mhz": maxmhz or None,
            "reasons": sorted(reasons), "samples": len(mhz)}


def cpu_baseline(spec, q, v, a, sc, ctrl, params, decimation, seed, nworld_sample, nsteps):
    """The FP64 oracle as it stands, threaded over worlds, on a bounded sample."""
    from oracle import Oracle
    o = Oracle(spec)
    W = nworld_sample
    q, v, a = q[:W].copy(), v[:W].copy(), a[:W].copy()
    from paper_2601_22074_b300.inputs import WorldParams
    p = WorldParams(params.friction_scale[:W], params.mass_scale[:W], params.kp[:W], params.kd[:W])
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    for s in range(nsteps):
        o.step_batch(q, v, a, ctrl[s % len(ctrl)][:W], decimation, params=p,
                     step_count=sc[:W] + s, seed=seed, world_id=np.arange(W, dtype=np.int32),
                     nthreads=threads)
    dt = time.perf_counter() - t0
    return {"value": W * nsteps / dt, "unit": "env-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{W} worlds x {nsteps} env steps (decimation {decimation}) from the "
                      f"GPU state after the pre-roll, FP64, {threads} threads"}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, same workload and metric."""
    from oracle import Oracle, build_oracle
    from paper_2601_22074_b300 import inputs as I
    build_oracle()
    name, W, dec = WORKLOADS[args.workload]
    spec = getattr(I, name)() if name != "pendulum" else I.pendulum(3)
    o = Oracle(spec)
    Ws = min(W, 256)
    q = np.zeros((Ws, spec.nq)); v = np.zeros((Ws, spec.nv)); a = np.zeros((Ws, spec.nv))
    for w in range(Ws):
        q[w], v[w] = o.reset(0, w)
    params = I.randomised_params(spec, W, 7)
    from paper_2601_22074_b300.inputs import WorldParams
    p = WorldParams(params.friction_scale[:Ws], params.mass_scale[:Ws], params.kp[:Ws], params.kd[:Ws])
    ctrl = I.ctrl_targets(spec, Ws, args.warmup + args.steps, 11)
    threads = os.cpu_count() or 1
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o.step_batch(q, v, a, ctrl[s], dec, params=p, step_count=np.full(Ws, s), seed=0,
                     nthreads=threads)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    val = Ws * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "env-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "worlds_per_step": Ws, "decimation": dec},
            "cpu_baseline": {"value": val, "unit": "env-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"{Ws} worlds per step, FP64, {threads} threads"},
            "e2e": {"value": val, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b3phys", choices=["b3phys", "reference"])
    ap.add_argument("--workload", default="humanoid8192", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--preroll", type=int, default=PREROLL)
    ap.add_argument("--worlds", type=int, default=0, help="override the world count (profiling)")
    ap.add_argument("--wpb", type=int, default=0, help="worlds (warps) per CTA; 0 = library default")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    from paper_2601_22074_b300 import build as B
    B.build()
    from paper_2601_22074_b300 import flops as F, inputs as I
    from paper_2601_22074_b300.batch import Batch, Model

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    name, W, dec = WORKLOADS[args.workload]
    W = args.worlds or W
    spec = getattr(I, name)() if name != "pendulum" else I.pendulum(3)
    model = Model(spec)
    batch = Batch(model, W, warps_per_block=args.wpb)
    seed = 1000 + rank
    batch.reset(seed)
    params = I.randomised_params(spec, W, 7 + rank)
    dev = batch.device
    batch.set_param(0, "friction_scale", torch.tensor(params.friction_scale, dtype=torch.float32, device=dev))
    batch.set_param(0, "mass_scale", torch.tensor(params.mass_scale, dtype=torch.float32, device=dev))
    if spec.nu:
        batch.set_param(0, "kp", torch.tensor(params.kp, dtype=torch.float32, device=dev))
        batch.set_param(0, "kd", torch.tensor(params.kd, dtype=torch.float32, device=dev))
    nctrl = args.preroll + args.warmup + args.steps
    ctrl_np = I.ctrl_targets(spec, W, nctrl, 11 + rank).astype(np.float32)
    ctrl = torch.tensor(ctrl_np, device=dev)
    stream = torch.cuda.current_stream()
    for t in range(args.preroll):
        batch.step(ctrl[t] if spec.nu else None, dec)
    torch.cuda.synchronize()
    # state for the CPU baseline: the pre-rolled GPU state
    q_pre = batch.get("qpos").view(W, spec.nq).double().cpu().numpy()
    v_pre = batch.get("qvel").view(W, spec.nv).double().cpu().numpy()
    a_pre = batch.get("qacc").view(W, spec.nv).double().cpu().numpy()
    sc_pre = batch.get("step_count").cpu().numpy().astype(np.int64)
    for t in range(args.preroll, args.preroll + args.warmup):
        batch.step(ctrl[t] if spec.nu else None, dec)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clk_path = os.path.join(tempfile.gettempdir(), f"b3p_clocks_{os.getpid()}.csv")
    sampler, clk_file = start_clock_sampler(clk_path)
    time.sleep(0.3)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_flops = []
    wall0 = time.perf_counter()
    for k in range(args.steps):
        t = args.preroll + args.warmup + k
        flush.zero_()
        ev[k][0].record(stream)
        batch.step(ctrl[t] if spec.nu else None, dec)
        ev[k][1].record(stream)
        st = batch.get("stats").view(W, 4).cpu().numpy()   # outside the events
        step_flops.append(F.env_step_flops(spec, st, dec))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(np.sum(ms))
    if dist:
        tm = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        total_ms = float(tm.item())
    value = world * W * args.steps / (total_ms / 1e3)
    status = batch.get("status").cpu().numpy()
    stats = batch.get("stats").view(W, 4).cpu().numpy()

    # end to end through the public API with host buffers
    nu = spec.nu
    h_ctrl = torch.empty((args.steps, W * max(nu, 1)), dtype=torch.float32, pin_memory=True)
    h_ctrl.copy_(torch.from_numpy(ctrl_np[args.preroll:args.preroll + args.steps].reshape(args.steps, -1))
                 if nu else torch.zeros_like(h_ctrl))
    h_out = torch.empty((2, W * spec.nq + W * spec.nv), dtype=torch.float32, pin_memory=True)
    d_ctrl = torch.empty(W * max(nu, 1), dtype=torch.float32, device=dev)
    q_flat = torch.empty(W * spec.nq, dtype=torch.float32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        d_ctrl.copy_(h_ctrl[k], non_blocking=True)
        batch.step(d_ctrl if nu else None, dec)
        qf = batch.get("qpos")
        vf = batch.get("qvel")
        h_out[k % 2, : W * spec.nq].copy_(qf, non_blocking=True)
        h_out[k % 2, W * spec.nq:].copy_(vf, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if dist:
        tm = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        e2e_ms = float(tm.item())
    if sampler:
        sampler.terminate()
        sampler.wait()
        clk_file.close()
    clocks = read_clocks(clk_path, local)

    if rank == 0:
        mhz, hbm, src = peaks()
        peak_tflops = NSM * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        achieved = float(np.mean(step_flops)) / (total_ms / args.steps / 1e3) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "model": name, "worlds_per_gpu": W,
                       "decimation": dec, "nq": spec.nq, "nv": spec.nv, "nu": spec.nu,
                       "preroll_env_steps": args.preroll, "launch": "one persistent launch per env step",
                       "l2": "256 MB write between timed steps (outside the events)",
                       "parallelism": f"replicas x{world}"},
            "physics_steps_per_s": value * dec,
            "wall_s": wall,
            "contacts_mean": float(stats[:, 0].mean()),
            "newton_iters_per_substep_mean": float(stats[:, 1].mean() / dec),
            "fp64_fallback_rate": float((stats[:, 2] > 0).mean()),
            "nan_worlds": int(np.sum(status & 1)),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved / peak_tflops, "traffic": None,
                         "peak_note": f"FP32 FMA peak 148 SMs x 128 lanes x 2 x {mhz:.0f} MHz ({src} max clock)",
                         "flops_per_env_step": float(np.mean(step_flops)) / W},
            "e2e": {"value": world * W * args.steps / (e2e_ms / 1e3), "unit": "env-steps/s",
                    "h2d_bytes_per_step": 4 * W * nu, "d2h_bytes_per_step": 4 * W * (spec.nq + spec.nv)},
            "gpu_launches": args.steps,
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(spec, q_pre, v_pre, a_pre, sc_pre,
                                                ctrl_np[args.preroll:].astype(np.float64), params,
                                                dec, seed, min(W, 1024), 20)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
