"""Benchmark: env-steps/s of the batched physics step (default: 8192-world humanoid).

One step = one environment step (push event + 4 physics substeps) of every world
in the batch, recorded once as a CUDA graph and replayed: either one persistent
launch, or the staged placement (one launch per stage over all worlds, 2 + 6 d
launches); the autotuner picks the placement and CTA shape first, untimed. Timing:
W warm-up steps, then K steps each bracketed by CUDA events on the launching stream,
with a 256 MB L2 flush between timed steps (outside the events). The roofline is
taken on the dominant kernel: with the staged placement, per-stage kernel times come
from events between the launches (b3p_step_profile) over extra flushed steps. Under
torchrun each rank runs the full workload on its own GPU (worlds are independent:
weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload humanoid8192]
    python bench.py --workload hetero9216       # 4 morphologies in one launch
    python bench.py --impl reference            # the FP64 oracle on the host cores

Both arms step the same workload state: the reference arm pre-rolls, on the host cores,
the same seeded worlds (reset seed, randomised parameters, targets) the GPU arm pre-rolls
on the device, and the two lines carry the same `config`. The GPU arm's cpu_baseline leg
times the oracle on a bounded sample of the GPU's pre-rolled worlds and checks the GPU's
first timed env step of those worlds against the oracle's (the `parity` key).
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
# name -> ([(morphology, worlds), ...], decimation)
WORKLOADS = {
    "humanoid8192": ([("humanoid", 8192)], 4),
    "quadruped4096": ([("quadruped", 4096)], 4),
    "pendulum64": ([("pendulum", 64)], 1),
    "manipulation1024": ([("manipulation", 1024)], 4),
    "hetero9216": ([("pendulum", 2048), ("quadruped", 4096), ("humanoid", 2048),
                    ("manipulation", 1024)], 4),
}
PREROLL = 100          # untimed env steps so the robots reach their contact-rich steady state
FP32_LANES_PER_SM = 128
PARITY_TOL = 1e-3      # contact-step tolerance of the parity tests (relative, floors below)
PARITY_FLOORS = {"qacc": 9.81, "qvel": 1.0, "qpos": 1.0}
SERVE_CURVE = (50.0, 100.0, 150.0, 200.0)   # offered loads of the serving curve, req/s
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel, from one ncu capture of the same bench command; valid only while the kernel
# sources hash to "source" (else the line reports null)
TRAFFIC = {"source": "d7fe1a0a10fc48e0",
           "bytes_per_launch": {"humanoid8192:solve": 34.47e6}}


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("b3p_step.cu", "b3p_internal.h"):
        with open(os.path.join(ROOT, "paper_2601_22074_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def make_spec(name):
    from paper_2601_22074_b300 import inputs as I
    return I.pendulum(3) if name == "pendulum" else getattr(I, name)()


def max_clock():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("sm_max_mhz", 2032.0), "measured"
    except Exception:
        return 2032.0, "fallback"


def workload_config(args, groups, dec, world):
    """The workload both arms step (identical in the two lines)."""
    return {"workload": args.workload, "groups": [list(g) for g in groups],
            "worlds_per_gpu": int(sum(w for _, w in groups)), "decimation": dec,
            "preroll_env_steps": args.preroll, "parallelism": f"replicas x{world}"}


def seeded_inputs(spec, W, g, rank, nctrl):
    """Per-world parameters and targets [nctrl, W, nu] of group g on rank `rank` (the same
    draws in both arms; a subset of worlds is a slice of the full draw)."""
    from paper_2601_22074_b300 import inputs as I
    p = I.randomised_params(spec, W, 7 + rank + 100 * g)
    c = I.ctrl_targets(spec, W, nctrl, 11 + rank + 100 * g).astype(np.float32)
    return p, c


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def slice_params(p, n):
    from paper_2601_22074_b300.inputs import WorldParams
    return WorldParams(f32(p.friction_scale[:n]), f32(p.mass_scale[:n]), f32(p.kp[:n]), f32(p.kd[:n]))


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


def oracle_sample_rate(groups, states, params, ctrls, dec, seed, per_group, nsteps, threads):
    """FP64 oracle env-steps/s over a bounded sample of each group's worlds."""
    from oracle import Oracle
    from paper_2601_22074_b300.inputs import WorldParams
    done, secs = 0, 0.0
    for (name, W), st, p, ctrl in zip(groups, states, params, ctrls):
        spec = make_spec(name)
        o = Oracle(spec)
        n = min(W, per_group)
        q, v, a, sc = (x[:n].copy() for x in st)
        ps = WorldParams(p.friction_scale[:n], p.mass_scale[:n], p.kp[:n], p.kd[:n])
        t0 = time.perf_counter()
        for s in range(nsteps):
            o.step_batch(q, v, a, ctrl[s % len(ctrl)][:n], dec, params=ps, step_count=sc + s,
                         seed=seed, world_id=np.arange(n, dtype=np.int32), nthreads=threads)
        secs += time.perf_counter() - t0
        done += n * nsteps
    return done / secs, done


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, same workload, state and metric:
    the first worlds of every group, reset from the GPU arm's seed and stepped through the
    GPU arm's pre-roll on the CPU, then timed over the same env steps."""
    from oracle import Oracle, build_oracle
    build_oracle()
    groups, dec = WORKLOADS[args.workload]
    threads = os.cpu_count() or 1
    per_group = max(16, 256 // len(groups))
    nctrl = args.preroll + args.warmup + args.steps
    seed = 1000
    states, params, ctrls = [], [], []
    t0 = time.perf_counter()
    for g, (name, W) in enumerate(groups):
        spec = make_spec(name)
        o = Oracle(spec)
        n = min(W, per_group)
        p, c = seeded_inputs(spec, W, g, 0, nctrl)
        ps = slice_params(p, n)
        c = c[:, :n].astype(np.float64)
        q = np.zeros((n, spec.nq))
        v = np.zeros((n, spec.nv))
        for w in range(n):
            q[w], v[w] = (f32(x) for x in o.reset(seed, w))
        a = np.zeros((n, spec.nv))
        sc = np.zeros(n, dtype=np.int64)
        for t in range(args.preroll):
            o.step_batch(q, v, a, c[t], dec, params=ps, step_count=sc + t, seed=seed,
                         world_id=np.arange(n, dtype=np.int32), nthreads=threads)
        states.append((q, v, a, sc + args.preroll))
        params.append(ps)
        ctrls.append(c[args.preroll:])
    preroll_s = time.perf_counter() - t0
    oracle_sample_rate(groups, states, params, ctrls, dec, seed, per_group, args.warmup, threads)
    rate, done = oracle_sample_rate(groups, states, params, ctrls, dec, seed, per_group, args.steps,
                                    threads)
    per_step = done // args.steps
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "env-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * per_step / rate, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, groups, dec, args.gpus),
            "cpu_baseline": {"value": rate, "unit": "env-steps/s", "cores": threads, "kind": "oracle",
                             "per_core": rate / threads,
                             "sample": f"{per_step} of the workload's worlds per env step (the first "
                                       f"{per_group} of each group), reset from the GPU arm's seed and "
                                       f"pre-rolled {args.preroll} env steps on the host cores "
                                       f"({preroll_s:.1f} s, untimed) under the GPU arm's targets and "
                                       f"parameters, then each env step timed from that state; FP64, "
                                       f"{threads} threads"},
            "e2e": {"value": rate, "unit": "env-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line))


def parity_of_step(groups, specs, states, params, ctrl_np, gpu_after, dec, seed, preroll, per_group):
    """Teacher-forced parity of one GPU env step: sampled worlds of every group stepped once
    by the oracle from the GPU's pre-rolled state; errors per world and field relative to
    max(|oracle|, floor), contact forces matched record by record (geom pair, position)."""
    from oracle import Oracle
    from scipy.optimize import linear_sum_assignment
    err = {k: [] for k in ("qacc", "qvel", "qpos", "force")}
    mism = compared = contacts = 0
    rng = np.random.default_rng(3)
    for g, ((name, W), spec) in enumerate(zip(groups, specs)):
        o = Oracle(spec)
        q0, v0, a0, sc0 = states[g]
        ps = params[g]
        qg, vg, ag, st, con, cnt = gpu_after[g]
        mtot = float(np.sum(spec.body_mass))
        for w in rng.choice(W, min(W, per_group), replace=False):
            r = o.step(q0[w], v0[w], a0[w], f32(ctrl_np[g][preroll, w]) if spec.nu else None, nsub=dec,
                       friction_scale=f32(ps.friction_scale[w]), mass_scale=f32(ps.mass_scale[w]),
                       kp=f32(ps.kp[w]) if spec.nu else None, kd=f32(ps.kd[w]) if spec.nu else None,
                       step_count=int(sc0[w]), seed=seed, world=int(w), want_contacts=True)
            if st[w, 0] != r["ncon"]:
                mism += 1
                continue
            gc_, oc = con[w, : cnt[w]], r["contacts"]
            fe = 0.0
            if r["ncon"]:
                kg = [tuple(x) for x in np.rint(gc_[:, :2]).astype(int)]
                ko = [tuple(x) for x in np.rint(oc[:, :2]).astype(int)]
                if sorted(kg) != sorted(ko):
                    mism += 1
                    continue
                fs = max(float(np.abs(oc[:, 21:24]).max()), mtot * 9.81)
                for key in set(kg):
                    ig = [i for i, k in enumerate(kg) if k == key]
                    io = [i for i, k in enumerate(ko) if k == key]
                    d = np.linalg.norm(gc_[ig, 5:8][:, None] - oc[io, 5:8][None], axis=2)
                    ri, ci = linear_sum_assignment(d)
                    for a_, b_ in zip(ri, ci):
                        fe = max(fe, float(np.abs(gc_[ig[a_], 21:24] - oc[io[b_], 21:24]).max()) / fs)
                err["force"].append(fe)
                contacts += int(r["ncon"])
            compared += 1
            for f, x in (("qacc", ag[w]), ("qvel", vg[w]), ("qpos", qg[w])):
                err[f].append(float(np.abs(x - r[f]).max() / max(np.abs(r[f]).max(), PARITY_FLOORS[f])))
    out = {k: [max(v), float(np.percentile(v, 99))] if v else None for k, v in err.items()}
    out.update({"worlds_compared": compared, "threshold_mismatches": mism, "contacts_compared": contacts,
                "tolerance": PARITY_TOL, "within_tolerance": all(v is None or v[0] <= PARITY_TOL
                                                                  for k, v in out.items()),
                "reference": "FP64 oracle, one env step from the GPU's pre-rolled state (teacher-forced); "
                             "force = per-contact world force, records matched by geom pair and position; "
                             "floors qacc 9.81, qvel 1, qpos 1, force m_total g"})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b3phys", choices=["b3phys", "reference"])
    ap.add_argument("--workload", default="humanoid8192", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--preroll", type=int, default=PREROLL)
    ap.add_argument("--worlds", type=int, default=0, help="override the world count (profiling)")
    ap.add_argument("--wpb", type=int, default=0, help="worlds (warps) per CTA; 0 = autotuned")
    ap.add_argument("--schedule", type=int, default=0,
                    help="with --wpb/--working-set: 0 natural order, 1 heaviest first")
    ap.add_argument("--lane-solve", type=int, default=0,
                    help="with --working-set 2/3 and --schedule 1: 1 = the solve one world per lane")
    ap.add_argument("--working-set", type=int, default=-1,
                    help="0 fused/shared, 1 fused/global, 2 staged, 3 grouped staged; default: autotuned")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="Poisson rollout requests for the serving leg (0: skip)")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-pool", type=int, default=8192, help="slot cap per morphology")
    ap.add_argument("--serve-working-set", type=int, default=3,
                    help="placement of the server's slot batch (3 grouped staged, 0 fused)")
    ap.add_argument("--serve-curve-requests", type=int, default=400,
                    help="requests per offered load of the serving curve")
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
    from paper_2601_22074_b300 import flops as F, inputs as I, tune as T
    from paper_2601_22074_b300.batch import Batch, Model

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    groups, dec = WORKLOADS[args.workload]
    if args.worlds:
        groups = [(n, args.worlds) for n, _ in groups]
    specs = [make_spec(n) for n, _ in groups]
    Ws = [w for _, w in groups]
    Wt = sum(Ws)
    models = [Model(s) for s in specs]
    tuned = None
    if args.wpb or args.no_tune or args.working_set >= 0:
        opts = dict(warps_per_block=args.wpb, blocks_per_sm=0, schedule=args.schedule,
                    working_set=max(args.working_set, 0), lane_solve=args.lane_solve)
    else:
        tuned = T.autotune(models, Ws, decimation=dec)
        opts = tuned["options"]
    # contact records are written back every env step (the state and contact readback)
    batch = Batch(models, Ws, write_contacts=True, **opts)
    seed = 1000 + rank
    batch.reset(seed)
    dev = batch.device
    params, ctrl_np = [], []
    nctrl = args.preroll + args.warmup + args.steps
    for g, (spec, W) in enumerate(zip(specs, Ws)):
        p, c = seeded_inputs(spec, W, g, rank, nctrl)
        params.append(p)
        batch.set_param(g, "friction_scale", torch.tensor(p.friction_scale, dtype=torch.float32, device=dev))
        batch.set_param(g, "mass_scale", torch.tensor(p.mass_scale, dtype=torch.float32, device=dev))
        if spec.nu:
            batch.set_param(g, "kp", torch.tensor(p.kp, dtype=torch.float32, device=dev))
            batch.set_param(g, "kd", torch.tensor(p.kd, dtype=torch.float32, device=dev))
        ctrl_np.append(c)
    nu_tot = sum(s.nu * w for s, w in zip(specs, Ws))
    ctrl = (torch.tensor(np.concatenate([c.reshape(nctrl, -1) for c in ctrl_np], axis=1), device=dev)
            if nu_tot else None)
    stream = torch.cuda.Stream()
    ctrl_buf = torch.zeros(max(nu_tot, 1), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for t in range(args.preroll):
            batch.step(ctrl[t] if nu_tot else None, dec)
    torch.cuda.synchronize()
    # the pre-rolled state feeds the CPU baseline
    states = []
    qf, vf, af, scf = batch.get("qpos"), batch.get("qvel"), batch.get("qacc"), batch.get("step_count")
    for g in range(len(specs)):
        states.append((batch.group_view(qf, "qpos", g).double().cpu().numpy(),
                       batch.group_view(vf, "qvel", g).double().cpu().numpy(),
                       batch.group_view(af, "qacc", g).double().cpu().numpy(),
                       batch.group_view(scf, "step_count", g).reshape(-1).cpu().numpy().astype(np.int64)))
    snap = batch.state_save()                          # the pre-rolled state, for the parity step
    # one env step recorded once as a CUDA graph; each step stages its targets into ctrl_buf
    batch.capture(ctrl_buf if nu_tot else None, 0, dec, 1, stream)
    with torch.cuda.stream(stream):
        for t in range(args.preroll, args.preroll + args.warmup):
            if nu_tot:
                ctrl_buf.copy_(ctrl[t])
            batch.replay(stream)
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
    step_flops, stats_last = [], []
    wall0 = time.perf_counter()
    for k in range(args.steps):
        t = args.preroll + args.warmup + k
        with torch.cuda.stream(stream):
            flush.zero_()
            if nu_tot:
                ctrl_buf.copy_(ctrl[t])
            ev[k][0].record(stream)
            batch.replay(stream)
            ev[k][1].record(stream)
        stream.synchronize()
        st_flat = batch.get("stats")                      # outside the events
        fl = 0.0
        for g, spec in enumerate(specs):
            st = batch.group_view(st_flat, "stats", g).cpu().numpy()
            fl += F.env_step_flops(spec, st, dec)
            if k == args.steps - 1:
                stats_last.append(st)
        step_flops.append(fl)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    total_ms = float(np.sum([a.elapsed_time(b) for a, b in ev]))
    if dist:
        tm = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        total_ms = float(tm.item())
    value = world * Wt * args.steps / (total_ms / 1e3)
    status = batch.get("status").cpu().numpy()
    stats = np.concatenate(stats_last)

    # end to end through the public API with host buffers: each step copies its targets from
    # pinned host memory into the captured graph's target buffer, replays the graph
    # (b3p_graph_launch) and reads qpos + qvel back into pinned host memory
    nq_tot = sum(s.nq * w for s, w in zip(specs, Ws))
    nv_tot = sum(s.nv * w for s, w in zip(specs, Ws))
    h_ctrl = torch.empty((args.steps, max(nu_tot, 1)), dtype=torch.float32, pin_memory=True)
    if nu_tot:
        h_ctrl.copy_(ctrl[args.preroll:args.preroll + args.steps].cpu())
    h_out = torch.empty((2, nq_tot + nv_tot), dtype=torch.float32, pin_memory=True)
    # the same L2 flush between steps as the device-timed loop, outside the events
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            ev2[k][0].record(stream)
            if nu_tot:
                ctrl_buf.copy_(h_ctrl[k], non_blocking=True)
            batch.replay(stream)
            h_out[k % 2, :nq_tot].copy_(batch.get("qpos"), non_blocking=True)
            h_out[k % 2, nq_tot:].copy_(batch.get("qvel"), non_blocking=True)
            ev2[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = float(np.sum([a.elapsed_time(b) for a, b in ev2]))
    if dist:
        tm = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        e2e_ms = float(tm.item())
    # per-stage kernel times of the staged placement: events between its launches
    staged = batch.options["working_set"] >= 2
    stage_ms = np.zeros(8)
    stage_n = np.zeros(8, dtype=np.int64)
    stage_fl = None
    if staged:
        from paper_2601_22074_b300 import _lib as LB
        stage_fl = {k: 0.0 for k in LB.STAGES}
        with torch.cuda.stream(stream):
            for k in range(min(args.steps, 10)):
                t = args.preroll + args.warmup + k % args.steps
                flush.zero_()
                if nu_tot:
                    ctrl_buf.copy_(ctrl[t])
                ms, n = batch.step_profile(ctrl_buf if nu_tot else None, dec)
                stage_ms += ms
                stage_n += n
                st_flat = batch.get("stats")
                for g, spec in enumerate(specs):
                    sf = F.stage_flops(spec, batch.group_view(st_flat, "stats", g).cpu().numpy(), dec)
                    for key in stage_fl:
                        stage_fl[key] += sf[key]
        torch.cuda.synchronize()
    # comparator: the plain per-stage path (one model group per launch sequence, no graph)
    plain_ms = []
    with torch.cuda.stream(stream):
        for k in range(args.warmup + min(args.steps, 10)):
            t = args.preroll + args.warmup + k % args.steps
            flush.zero_()
            if nu_tot:
                ctrl_buf.copy_(ctrl[t])
            a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_ev.record(stream)
            batch.step_plain(ctrl_buf if nu_tot else None, dec)
            b_ev.record(stream)
            if k >= args.warmup:
                plain_ms.append((a_ev, b_ev))
    torch.cuda.synchronize()
    plain_ms = [a.elapsed_time(b) for a, b in plain_ms]
    if sampler:
        sampler.terminate()
        sampler.wait()
        clk_file.close()
    clocks = read_clocks(clk_path, local)
    # the parity step: one env step (the same launches b3p_step records in the graph) from
    # the pre-rolled state with the first timed step's targets, read back for the check in
    # the cpu_baseline leg
    with torch.cuda.stream(stream):
        batch.state_restore(snap)
        if nu_tot:
            ctrl_buf.copy_(ctrl[args.preroll])
        batch.step(ctrl_buf if nu_tot else None, dec)
    torch.cuda.synchronize()
    gpu_after = []
    fl_all = {f: batch.get(f) for f in ("qpos", "qvel", "qacc", "stats")}
    con_all, cnt_all = batch.contacts()
    con_all, cnt_all = con_all.double().cpu().numpy(), cnt_all.cpu().numpy()
    slot = 0
    for g, (spec, W) in enumerate(zip(specs, Ws)):
        nc = max(models[g].ncon_max, 1)
        gpu_after.append(tuple(batch.group_view(fl_all[f], f, g).cpu().numpy().astype(
            np.float64 if f != "stats" else np.int64) for f in ("qpos", "qvel", "qacc", "stats")) + (
            con_all[slot:slot + W * nc].reshape(W, nc, -1),
            cnt_all[batch.world_start[g]:batch.world_start[g] + W]))
        slot += W * nc
    # the ALU roof: measured FP32 FMA throughput of this device and its SM count
    from paper_2601_22074_b300.batch import fp32_peak
    with torch.cuda.stream(stream):
        probe_flops, nsm = fp32_peak(5)
    torch.cuda.synchronize()

    if rank == 0:
        mhz, src = max_clock()
        nominal_tflops = nsm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        peak_tflops = probe_flops / 1e12
        step_achieved = float(np.mean(step_flops)) / (total_ms / args.steps / 1e3) / 1e12
        sorted_solve = staged and batch.options["schedule"] == 1
        grouped = batch.options["working_set"] == 3
        launches_per_step = ((3 * dec + 1 if grouped else 2 + 6 * dec) + (dec if sorted_solve else 0)) if staged else 1
        if staged:
            from paper_2601_22074_b300 import _lib as LB
            top = int(np.argmax(stage_ms))
            name = LB.STAGES[top]
            per_launch_ms = stage_ms[top] / stage_n[top]
            achieved = stage_fl[name] / stage_n[top] / (per_launch_ms / 1e3) / 1e12
            # the staged solve runs as solve_aux_kernel (Newton arrays, M, M's factor and the
            # motion axes in shared memory); the other per-stage launches as staged_kernel
            kernel = "solve_aux_kernel (solve stage)" if name == "solve" else f"staged_kernel<{top}> ({name} stage)"
            tb = TRAFFIC["bytes_per_launch"].get(f"{args.workload}:{name}")
            traffic = tb if (tb is not None and TRAFFIC["source"] == kernel_source_hash()
                             and not args.worlds) else None
            stages = {LB.STAGES[i]: {"launches": int(stage_n[i]), "ms_per_launch": float(stage_ms[i] / stage_n[i]),
                                     "share": float(stage_ms[i] / stage_ms.sum()),
                                     "gflop_per_launch": stage_fl[LB.STAGES[i]] / stage_n[i] / 1e9}
                      for i in range(8) if stage_n[i]}
        else:
            achieved, kernel, traffic, stages = step_achieved, "step_kernel (whole env step)", None, None
            per_launch_ms = total_ms / args.steps
        line = {
            "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(args, groups, dec, world),
            "launch": {"form": (f"staged: {launches_per_step} launches per env step over all worlds"
                                f"{' (consecutive per-world stages grouped)' if grouped else ''}"
                                f"{', solve heaviest first' if sorted_solve else ''}, replayed from a CUDA "
                                f"graph; contact records written back every env step") if staged else
                               "one persistent launch per env step, replayed from a CUDA graph",
                       "options": opts,
                       "shape": batch.launch_info(),
                       "autotune_ms_per_step": None if tuned is None else
                       [[o, round(m, 4)] for o, m in tuned["table"]],
                       "autotune_refined_ms_per_step": None if tuned is None else
                       [[o, round(m, 4)] for o, m in tuned.get("refined", [])],
                       "l2": "256 MB write between timed steps (outside the events)"},
            "physics_steps_per_s": value * dec,
            "wall_s": wall,
            "contacts_mean": float(stats[:, 0].mean()),
            "contacts_hist": np.bincount(stats[:, 0]).tolist(),
            "newton_iters_per_substep_mean": float(stats[:, 1].mean() / dec),
            "newton_iters_hist": np.bincount(stats[:, 1]).tolist(),   # per world, summed over the env step's substeps
            "fp64_fallback_rate": float((stats[:, 2] > 0).mean()),
            "nan_worlds": int(np.sum(status & 1)),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved / peak_tflops, "traffic": traffic,
                         "kernel": kernel, "ms_per_launch": per_launch_ms,
                         "peak_note": f"measured: FP32 FMA probe (b3p_fp32_peak, best of 5, eight independent "
                                      f"FMA chains per thread on all {nsm} SMs, SM count read from the "
                                      f"device) = {peak_tflops:.2f} TFLOP/s; nominal {nsm} SMs x 128 lanes x 2 x "
                                      f"{mhz:.0f} MHz ({src} max clock) = {nominal_tflops:.2f}",
                         "whole_step_achieved": step_achieved,
                         "whole_step_frac": step_achieved / peak_tflops,
                         "flops_per_env_step": float(np.mean(step_flops)) / Wt,
                         "stages": stages},
            "e2e": {"value": world * Wt * args.steps / (e2e_ms / 1e3), "unit": "env-steps/s",
                    "h2d_bytes_per_step": 4 * nu_tot, "d2h_bytes_per_step": 4 * (nq_tot + nv_tot),
                    "path": "pinned targets -> graph target buffer, b3p_graph_launch, qpos + qvel -> pinned; "
                            "L2 flushed between steps outside the events"},
            "gpu_launches": args.steps * launches_per_step,
            "comparators": {"plain": {
                "value": Wt / (np.mean(plain_ms) / 1e3), "unit": "env-steps/s",
                "ms_per_step": float(np.mean(plain_ms)),
                "form": f"per-stage kernels, one model group per launch sequence "
                        f"({len(specs)} x {2 + 6 * dec} launches per env step), no graph, "
                        f"state in a global workspace; same parity bar"}},
            "clocks": clocks,
        }
        if args.serve_requests:
            # served rollouts: Poisson arrivals over the four morphologies, the configured 200 req/s
            # with the full request count, and a curve of lighter loads (latency against load)
            import gc
            from paper_2601_22074_b300 import serve as SV
            serve_specs = [make_spec(n) for n in ("pendulum", "quadruped", "humanoid", "manipulation")]

            def serve_point(rate, nreq, warm):
                srv = SV.RolloutServer(serve_specs, args.serve_budget_gb * 1e9, decimation=4,
                                       max_worlds_per_group=args.serve_pool, run_thread=True,
                                       options=dict(working_set=args.serve_working_set))
                reqs = SV.poisson_requests(nreq, rate=rate, ngroup=4, seed=17)
                rep = SV.run_load(srv, reqs, warmup_s=warm)
                del srv
                gc.collect()
                offered = sum(r.nworld * r.horizon for r in reqs) / max(reqs[-1].arrival, 1e-9)
                rep["offered"] = offered
                return rep

            rep = serve_point(200.0, args.serve_requests, 1.0)
            # the server's capacity: requests far beyond what it serves (all queued within a
            # second), the highest served rate over any one-second window
            cap = serve_point(2000.0, 600, 0.0)
            capacity = cap["peak_env_steps_per_s"]
            rep["overloaded"] = rep["offered"] > 0.95 * capacity
            curve = []
            for rate in SERVE_CURVE:
                r = serve_point(rate, args.serve_curve_requests, 0.5)
                r["overloaded"] = r["offered"] > 0.95 * capacity
                curve.append({"offered_req_per_s": rate, "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
                              "served_world_env_steps_per_s": r["env_steps_per_s"],
                              "offered_world_env_steps_per_s": r["offered"], "overloaded": r["overloaded"],
                              "mean_queue_wait_ms": r["mean_queue_ms"], "requests": r["requests"],
                              "measured": r["measured"], "latency_growth": r["latency_growth"]})
            sustainable = [c["offered_req_per_s"] for c in curve if not c["overloaded"]]
            line["serving"] = {
                "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"], "unit": "ms",
                "env_steps_per_s": rep["env_steps_per_s"], "requests": rep["requests"],
                "completed": rep["completed"], "measured_after_1s": rep["measured"],
                "refused_busy": rep["busy"], "mean_queue_wait_ms": rep["mean_queue_ms"],
                "slots_per_morphology": rep["capacity"], "ticks": rep["ticks"],
                "offered_world_env_steps_per_s": rep["offered"], "overloaded": rep["overloaded"],
                "latency_growth": rep["latency_growth"],
                "elapsed_s": rep["elapsed_s"],
                "load": "Poisson 200 req/s; morphology uniform over pendulum/quadruped/humanoid/"
                        "manipulation; worlds log-uniform [1, 1024]; horizon U{50..500} env steps; "
                        f"HBM budget {args.serve_budget_gb:g} GB",
                "server": "native rollout server (b3p_server_*), its own thread ticking, "
                          f"{'grouped staged' if args.serve_working_set == 3 else 'working_set ' + str(args.serve_working_set)} "
                          "placement, 2 ticks in flight",
                "curve": curve,
                "capacity_world_env_steps_per_s": capacity,
                "capacity_note": "600 requests offered at 2000 req/s (queued within 0.3 s): the highest served "
                                 "world-env-steps/s over any one-second window",
                "highest_sustained_req_per_s": max(sustainable) if sustainable else None,
                "curve_note": f"{args.serve_curve_requests} requests per offered load, the first 0.5 s of "
                              "arrivals excluded; overloaded = offered world-env-steps/s above 95 % of the "
                              "measured capacity (the queue then grows for as long as requests arrive, so "
                              "latencies depend on the run's length); served world-env-steps/s is over the "
                              "whole run, drain included; latency_growth = median latency of the later half "
                              "of the arrivals over the earlier half's"}
        if not args.no_cpu_baseline:
            threads = os.cpu_count() or 1
            per_group = max(64, 1024 // len(groups))
            samples = [slice_params(p, min(W, per_group)) for p, W in zip(params, Ws)]
            rate, done = oracle_sample_rate(
                groups, states, samples, [c[args.preroll:].astype(np.float64) for c in ctrl_np], dec,
                seed, per_group, 20, threads)
            line["cpu_baseline"] = {
                "value": rate, "unit": "env-steps/s", "cores": threads, "kind": "oracle",
                "per_core": rate / threads,
                "sample": f"{done // 20} worlds x 20 env steps (decimation {dec}) from the GPU state "
                          f"after the pre-roll, FP64, {threads} threads"}
            # the same leg checks the GPU's env step from that state against the oracle's
            line["parity"] = parity_of_step(groups, specs, states, params, ctrl_np, gpu_after, dec, seed,
                                            args.preroll, max(48, 96 // len(groups)))
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
