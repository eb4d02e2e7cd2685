"""Teacher-forced comparison of the CUDA step with the FP64 oracle.

At every environment step the GPU state (qpos, qvel, qacc, step count)
is read back and the oracle takes one step from exactly those float32 values with
the same float32 controls and per-world parameters; the GPU's next state is then
compared field by field. Error per world and field:
    |x_gpu - x_oracle|_inf / max(|x_oracle|_inf, floor)
with floors qacc 9.81, qvel 1, qpos 1, contact force m_total g. A world step whose
last-substep contact count differs between the two sides (a contact at the
activation threshold) is counted as a threshold mismatch, not compared.

Contact records of the last substep are compared one by one: both sides' records are
grouped by geom pair and, within a pair, matched by position (the assignment of least
total distance), then each matched record's position, normal, penetration and world
force is compared, each with its own floor (positions 1 m, normals 1, penetration
0.1 m, forces m_total g, the force floor relative to the largest oracle contact
force of the world). A world step whose per-pair counts differ although the totals
agree is counted as a threshold mismatch too.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np
import torch

from oracle import Oracle
from paper_2601_22074_b300 import inputs as I
from paper_2601_22074_b300.batch import Batch, Model

FLOORS = {"qacc": 9.81, "qvel": 1.0, "qpos": 1.0}
# contact record columns (24 floats, the same layout on both sides): g1 g2 b1 b2 dist
# pos[3] frame[9] (normal first) mu f[3] (contact frame) f_world[3]
# floors: positions 1 m (the qpos floor); penetration 0.1 m -- it derives from qpos, whose bar
# is 1e-3 of 1 m, so this keeps the penetration check ten times stricter than the position
# bar it follows from; normals 1 (unit vectors)
CONTACT_FIELDS = {"cpos": (slice(5, 8), 1.0), "cnormal": (slice(8, 11), 1.0), "cdist": (slice(4, 5), 0.1)}
FIELDS = ("qacc", "qvel", "qpos", "force", "cpos", "cnormal", "cdist", "cforce")


def match_contacts(gpu: np.ndarray, orc: np.ndarray):
    """Index pairs (i_gpu, i_oracle) matching two contact sets of equal size: records are
    grouped by geom pair (columns 0, 1) and matched within a pair by position (least total
    distance). None when some pair has a different number of records on the two sides."""
    from scipy.optimize import linear_sum_assignment
    if len(gpu) != len(orc):
        return None
    kg = [(int(round(r[0])), int(round(r[1]))) for r in gpu]
    ko = [(int(round(r[0])), int(round(r[1]))) for r in orc]
    out = []
    for key in sorted(set(kg) | set(ko)):
        ig = [i for i, k in enumerate(kg) if k == key]
        io = [i for i, k in enumerate(ko) if k == key]
        if len(ig) != len(io):
            return None
        d = np.linalg.norm(gpu[ig, 5:8][:, None, :] - orc[io, 5:8][None, :, :], axis=2)
        rows, cols = linear_sum_assignment(d)
        out += [(ig[r], io[c]) for r, c in zip(rows, cols)]
    return out


def contact_errors(gpu: np.ndarray, orc: np.ndarray, mtot: float):
    """Per-field errors of one world step's contact records (max over the matched
    contacts), or None when the sets do not match pair by pair."""
    pairs = match_contacts(gpu, orc)
    if pairs is None:
        return None
    if not pairs:
        return {}
    ig = [i for i, _ in pairs]
    io = [j for _, j in pairs]
    g, o = gpu[ig], orc[io]
    out = {}
    for name, (cols, floor) in CONTACT_FIELDS.items():
        out[name] = float(np.max(np.abs(g[:, cols] - o[:, cols]).max(axis=1) /
                                 np.maximum(np.abs(o[:, cols]).max(axis=1), floor)))
    fscale = max(float(np.abs(o[:, 21:24]).max()), mtot * 9.81)
    out["cforce"] = float(np.abs(g[:, 21:24] - o[:, 21:24]).max() / fscale)
    return out


@dataclasses.dataclass
class Report:
    err: Dict[str, List[float]]
    mismatches: int = 0
    compared: int = 0
    contact_steps: int = 0
    fallbacks: int = 0
    iters: List[int] = dataclasses.field(default_factory=list)
    max_ncon: int = 0
    limit_steps: int = 0     # compared world steps that started with a violated joint limit
    contacts_compared: int = 0
    with_contacts: bool = True   # contact records were read back and compared

    def max(self, k):
        return max(self.err[k]) if self.err[k] else 0.0

    def p99(self, k):
        return float(np.percentile(self.err[k], 99)) if self.err[k] else 0.0

    def summary(self):
        return {k: (self.max(k), self.p99(k)) for k in self.err} | {
            "mismatch": self.mismatches, "compared": self.compared,
            "contact_steps": self.contact_steps, "contacts_compared": self.contacts_compared,
            "fallbacks": self.fallbacks}


def check(rep: Report, tol: float, max_mismatch: float = 0.02) -> dict:
    """Assert every compared field within tol (per-contact record fields included whenever
    contacts were compared) and threshold mismatches within max_mismatch of the world
    steps; prints and returns the max / p99 summary."""
    s = rep.summary()
    print(s)
    n = rep.compared + rep.mismatches
    assert rep.mismatches <= max_mismatch * n, s
    for k in FIELDS:
        assert rep.max(k) <= tol, (k, s)
    if rep.contact_steps and rep.with_contacts:
        assert rep.contacts_compared > 0 and len(rep.err["cforce"]) == rep.contact_steps, s
    return s


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def set_params(batch: Batch, group: int, p: I.WorldParams, nu: int):
    dev = batch.device
    batch.set_param(group, "friction_scale", torch.tensor(p.friction_scale, dtype=torch.float32, device=dev))
    batch.set_param(group, "mass_scale", torch.tensor(p.mass_scale, dtype=torch.float32, device=dev))
    if nu:
        batch.set_param(group, "kp", torch.tensor(p.kp, dtype=torch.float32, device=dev))
        batch.set_param(group, "kd", torch.tensor(p.kd, dtype=torch.float32, device=dev))
    torch.cuda.synchronize()


def read(batch: Batch, W: int, spec):
    q = batch.get("qpos").view(W, spec.nq).double().cpu().numpy()
    v = batch.get("qvel").view(W, spec.nv).double().cpu().numpy()
    a = batch.get("qacc").view(W, spec.nv).double().cpu().numpy()
    sc = batch.get("step_count").cpu().numpy().astype(np.int64)
    st = batch.get("status").cpu().numpy()
    stats = batch.get("stats").view(W, 4).cpu().numpy()
    return q, v, a, sc, st, stats


def ulp_move(x, k: int, rng) -> np.ndarray:
    """x (float32 values held as float64) with every component moved k float32 ulps up
    or down (random signs)."""
    x32 = np.asarray(x, dtype=np.float32)
    sgn = rng.choice([-1, 1], size=x32.shape)
    out = x32.copy()
    for _ in range(k):
        out = np.where(sgn > 0, np.nextafter(out, np.float32(np.inf)), np.nextafter(out, np.float32(-np.inf)))
    return out.astype(np.float64)


def world_err(x_gpu, x_orc, floor):
    return float(np.abs(x_gpu - x_orc).max() / max(np.abs(x_orc).max(), floor))


def teacher_forced(spec, W: int, nsteps: int, decimation: int, seed: int = 0,
                   sample: Optional[np.ndarray] = None, warm_steps: int = 0,
                   param_seed: int = 7, ctrl_seed: int = 11, lift: float = 0.0,
                   step_count_start: Optional[int] = None, contacts: bool = True,
                   pinch: bool = False, options: Optional[dict] = None, inertia_sigma: float = 0.0,
                   oracle_ctrl_fn=None, spread_ulps: int = 0, qpos0: Optional[np.ndarray] = None) -> Report:
    """oracle_ctrl_fn maps the submitted targets [T, W, nu] to the ones the oracle applies
    (an actuation-delay model; default: the same). spread_ulps > 0 also steps the oracle
    from the read-back state with every qpos and qvel component moved by that many FP32
    ulps (seeded random signs) and records the oracle's own movement as "spread_*" (the
    conditioning of the case, not a parity field)."""
    model = Model(spec)
    batch = Batch(model, W, write_contacts=contacts, **(options or {}))
    batch.reset(seed)
    torch.cuda.synchronize()
    params = I.randomised_params(spec, W, param_seed)
    set_params(batch, 0, params, spec.nu)
    inertia = None
    if inertia_sigma > 0:
        inertia = I.randomised_inertia(spec, W, param_seed + 1, inertia_sigma)
        batch.set_param(0, "body_inertia", torch.tensor(inertia.reshape(W, -1), dtype=torch.float32))
        torch.cuda.synchronize()
        inertia = f32(inertia)
    # the oracle sees the float32-rounded parameters the GPU holds
    p32 = I.WorldParams(f32(params.friction_scale), f32(params.mass_scale), f32(params.kp), f32(params.kd))
    ctrl = I.ctrl_targets(spec, W, warm_steps + nsteps, ctrl_seed)
    if pinch:  # hold the arm at its reset pose and close both fingers
        ctrl[:] = spec.qpos_reset[spec.act_qposadr()]
        ctrl[:, :, -2:] = -0.03
    ctrl_dev = torch.tensor(ctrl, dtype=torch.float32, device=batch.device)
    octrl = oracle_ctrl_fn(f32(ctrl)) if oracle_ctrl_fn is not None else ctrl
    prng = np.random.default_rng(1234)
    if qpos0 is not None:                    # a start state per world (float32 on the GPU)
        batch.set("qpos", torch.tensor(np.asarray(qpos0).reshape(-1), dtype=torch.float32))
    if lift:
        q = batch.get("qpos").view(W, spec.nq).clone()
        q[:, 2] += lift
        batch.set("qpos", q.reshape(-1))
    if step_count_start is not None:
        batch.set("step_count", torch.full((W,), step_count_start, dtype=torch.int32))
    for t in range(warm_steps):
        batch.step(ctrl_dev[t] if spec.nu else None, decimation)
    torch.cuda.synchronize()
    o = Oracle(spec)
    sel = np.arange(W) if sample is None else np.asarray(sample)
    mtot = float(np.sum(spec.body_mass))
    rep = Report(err={k: [] for k in FIELDS}, with_contacts=contacts)
    for t in range(warm_steps, warm_steps + nsteps):
        q0, v0, a0, sc0, _, _ = read(batch, W, spec)
        batch.step(ctrl_dev[t] if spec.nu else None, decimation)
        torch.cuda.synchronize()
        q1, v1, a1, _, st1, stats1 = read(batch, W, spec)
        if contacts:
            con, cnt = batch.contacts()
            con = con.view(W, max(model.ncon_max, 1), 24).double().cpu().numpy()
            cnt = cnt.cpu().numpy()
        for w in sel:
            def ostep(qq, vv, want):
                return o.step(qq, vv, a0[w], f32(octrl[t, w]) if spec.nu else None, nsub=decimation,
                              friction_scale=p32.friction_scale[w], mass_scale=p32.mass_scale[w],
                              kp=p32.kp[w] if spec.nu else None, kd=p32.kd[w] if spec.nu else None,
                              step_count=int(sc0[w]), seed=seed, world=int(w), want_contacts=want,
                              body_inertia=None if inertia is None else inertia[w])
            r = ostep(q0[w], v0[w], contacts)
            rep.fallbacks += int(stats1[w, 2])
            if stats1[w, 0] != r["ncon"]:
                rep.mismatches += 1
                continue
            cerr = None
            if contacts and r["ncon"]:
                cerr = contact_errors(con[w, : cnt[w]], r["contacts"], mtot)
                if cerr is None:            # same count, different pairs: threshold case
                    rep.mismatches += 1
                    continue
            rep.compared += 1
            rep.max_ncon = max(rep.max_ncon, int(r["ncon"]))
            if r["ncon"]:
                rep.contact_steps += 1
                rep.iters.append(int(stats1[w, 1]))
            if spec.jnt_limited is not None and o.limits(q0[w], v0[w])["nl"] > 0:
                rep.limit_steps += 1
            rep.err["qacc"].append(world_err(a1[w], r["qacc"], FLOORS["qacc"]))
            rep.err["qvel"].append(world_err(v1[w], r["qvel"], FLOORS["qvel"]))
            rep.err["qpos"].append(world_err(q1[w], r["qpos"], FLOORS["qpos"]))
            if spread_ulps:
                qp = ulp_move(q0[w], spread_ulps, prng)
                vp = ulp_move(v0[w], spread_ulps, prng)
                rp = ostep(qp, vp, False)
                for f in ("qacc", "qvel", "qpos"):
                    rep.err.setdefault("spread_" + f, []).append(world_err(rp[f], r[f], FLOORS[f]))
            if contacts and r["ncon"]:
                fg = con[w, : cnt[w], 21:24].sum(0)
                fo = r["contacts"][:, 21:24].sum(0)
                rep.err["force"].append(float(np.abs(fg - fo).max() / max(np.abs(fo).max(), mtot * 9.81)))
                for k, v in cerr.items():
                    rep.err[k].append(v)
                rep.contacts_compared += int(r["ncon"])
    return rep


def teacher_forced_mixed(specs, Ws, nsteps: int, decimation: int, samples: int, seed: int = 0,
                         warm_steps: int = 0, options: Optional[dict] = None) -> List[Report]:
    """teacher_forced for a batch of several morphologies in one launch sequence: sampled
    worlds of every group are compared with the oracle, one Report per group."""
    models = [Model(s) for s in specs]
    batch = Batch(models, list(Ws), write_contacts=True, **(options or {}))
    batch.reset(seed)
    torch.cuda.synchronize()
    params, p32s, ctrls = [], [], []
    for g, (spec, W) in enumerate(zip(specs, Ws)):
        p = I.randomised_params(spec, W, 7 + 100 * g)
        set_params(batch, g, p, spec.nu)
        params.append(p)
        p32s.append(I.WorldParams(f32(p.friction_scale), f32(p.mass_scale), f32(p.kp), f32(p.kd)))
        ctrls.append(I.ctrl_targets(spec, W, warm_steps + nsteps, 11 + 100 * g))
    nu_tot = sum(s.nu * w for s, w in zip(specs, Ws))
    ctrl_dev = (torch.tensor(np.concatenate([c.reshape(c.shape[0], -1) for c in ctrls], axis=1),
                             dtype=torch.float32, device=batch.device) if nu_tot else None)
    for t in range(warm_steps):
        batch.step(ctrl_dev[t] if nu_tot else None, decimation)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed + 1)
    sels = [rng.choice(W, min(samples, W), replace=False) for W in Ws]
    slot0 = np.cumsum([0] + [W * max(m.ncon_max, 1) for m, W in zip(models, Ws)])
    reps = [Report(err={k: [] for k in FIELDS}) for _ in specs]
    oracles = [Oracle(s) for s in specs]

    def read_all():
        out = {}
        for f in ("qpos", "qvel", "qacc", "step_count", "stats"):
            flat = batch.get(f)
            out[f] = [batch.group_view(flat, f, g).cpu().numpy() for g in range(len(specs))]
            if f == "step_count":
                out[f] = [x.reshape(-1) for x in out[f]]
        return out

    for t in range(warm_steps, warm_steps + nsteps):
        s0 = read_all()
        batch.step(ctrl_dev[t] if nu_tot else None, decimation)
        torch.cuda.synchronize()
        s1 = read_all()
        con, cnt = batch.contacts()
        con, cnt = con.double().cpu().numpy(), cnt.cpu().numpy()
        for g, (spec, W) in enumerate(zip(specs, Ws)):
            rep, o, p32 = reps[g], oracles[g], p32s[g]
            mtot = float(np.sum(spec.body_mass))
            nc = max(models[g].ncon_max, 1)
            gcon = con[slot0[g]:slot0[g + 1]].reshape(W, nc, 24)
            gcnt = cnt[batch.world_start[g]:batch.world_start[g] + W]
            for w in sels[g]:
                r = o.step(s0["qpos"][g][w].astype(np.float64), s0["qvel"][g][w].astype(np.float64),
                           s0["qacc"][g][w].astype(np.float64),
                           f32(ctrls[g][t, w]) if spec.nu else None, nsub=decimation,
                           friction_scale=p32.friction_scale[w], mass_scale=p32.mass_scale[w],
                           kp=p32.kp[w] if spec.nu else None, kd=p32.kd[w] if spec.nu else None,
                           step_count=int(s0["step_count"][g][w]), seed=seed, world=int(w),
                           want_contacts=True)
                st = s1["stats"][g][w]
                rep.fallbacks += int(st[2])
                if st[0] != r["ncon"]:
                    rep.mismatches += 1
                    continue
                cerr = None
                if r["ncon"]:
                    cerr = contact_errors(gcon[w, : gcnt[w]], r["contacts"], mtot)
                    if cerr is None:
                        rep.mismatches += 1
                        continue
                rep.compared += 1
                rep.max_ncon = max(rep.max_ncon, int(r["ncon"]))
                if r["ncon"]:
                    rep.contact_steps += 1
                for f in ("qacc", "qvel", "qpos"):
                    rep.err[f].append(world_err(s1[f][g][w].astype(np.float64), r[f], FLOORS[f]))
                if r["ncon"]:
                    fg = gcon[w, : gcnt[w], 21:24].sum(0)
                    fo = r["contacts"][:, 21:24].sum(0)
                    rep.err["force"].append(float(np.abs(fg - fo).max() / max(np.abs(fo).max(), mtot * 9.81)))
                    for k, v in cerr.items():
                        rep.err[k].append(v)
                    rep.contacts_compared += int(r["ncon"])
    return reps
