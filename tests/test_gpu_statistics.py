"""Long-horizon statistics, GPU (FP32) against the FP64 oracle, both free-running.

Contact dynamics and multi-link pendulums are chaotic: single trajectories part ways
after a few hundred steps, so the comparison is over ensembles. The same statistic is
computed from both ensembles by the same FP64 function (the oracle's kinematics and mass
matrix), and the two ensemble means must agree within a tolerance set by the spread of
the ensemble (stated per test).
"""
import numpy as np
import pytest
import torch

from paper_2601_22074_b300 import build, inputs as I
from paper_2601_22074_b300.batch import Batch, Model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _energy(o, spec, q, v):
    """Kinetic + potential energy of one world (FP64, oracle kinematics)."""
    M = o.mass_matrix(q)
    f = o.fk(q)
    pe = float(np.sum(np.asarray(spec.body_mass)[1:] * 9.81 * f["xipos"][1:, 2]))
    return 0.5 * float(v @ M @ v) + pe


def test_pendulum_energy_statistics_over_1000_steps():
    """C0: 64 three-link pendulums, h = 2 ms, 1000 steps from the seeded reset. Semi-implicit
    Euler drifts in energy at O(h) on both sides; the ensemble-mean drift and the ensemble
    mean of |qdot| over the last 500 steps agree within 3 standard errors."""
    from oracle import Oracle
    spec = I.pendulum(3)
    W, T = 64, 1000
    b = Batch(Model(spec), W, working_set=3, warps_per_block=4, schedule=1)   # the benchmark's launch
    b.reset(0)
    o = Oracle(spec)
    q = np.zeros((W, spec.nq))
    v = np.zeros((W, spec.nv))
    for w in range(W):
        q[w], v[w] = o.reset(0, w)
    a = np.zeros((W, spec.nv))
    qg = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
    assert np.abs(qg - q).max() < 1e-6
    e0 = np.array([_energy(o, spec, q[w], v[w]) for w in range(W)])
    speed_g, speed_o = [], []
    sc = np.zeros(W, dtype=np.int64)
    for t in range(T):
        b.step(None, 1)
        o.step_batch(q, v, a, None, 1, step_count=sc + t)
        if t >= T // 2 and t % 10 == 0:
            vg = b.get("qvel").view(W, spec.nv).double().cpu().numpy()
            speed_g.append(np.linalg.norm(vg, axis=1))
            speed_o.append(np.linalg.norm(v, axis=1))
    qg = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
    vg = b.get("qvel").view(W, spec.nv).double().cpu().numpy()
    dg = np.array([_energy(o, spec, qg[w], vg[w]) for w in range(W)]) - e0
    do = np.array([_energy(o, spec, q[w], v[w]) for w in range(W)]) - e0
    se = np.sqrt(dg.var() / W + do.var() / W) + 1e-9
    assert abs(dg.mean() - do.mean()) <= 3 * se + 1e-3 * np.abs(e0).mean(), (dg.mean(), do.mean(), se)
    sg, so = np.mean(speed_g, axis=0), np.mean(speed_o, axis=0)      # per-world time means
    se = np.sqrt(sg.var() / W + so.var() / W)
    assert abs(sg.mean() - so.mean()) <= 3 * se, (sg.mean(), so.mean(), se)


def _ensemble_stats(spec, W, T, seed_params=7, seed_ctrl=11, stats_fn=None):
    """GPU (the benchmark's launch) and FP64 oracle ensembles of W worlds, both free-running
    for T env steps (d = 4) from the seeded reset under the same targets and randomised
    parameters; returns per-statistic lists over the last T / 2 env steps."""
    from oracle import Oracle
    dec = 4
    b = Batch(Model(spec), W, working_set=3, warps_per_block=4, schedule=1)
    b.reset(0)
    p = I.randomised_params(spec, W, seed_params)
    dev = b.device
    b.set_param(0, "friction_scale", torch.tensor(p.friction_scale, dtype=torch.float32, device=dev))
    b.set_param(0, "mass_scale", torch.tensor(p.mass_scale, dtype=torch.float32, device=dev))
    b.set_param(0, "kp", torch.tensor(p.kp, dtype=torch.float32, device=dev))
    b.set_param(0, "kd", torch.tensor(p.kd, dtype=torch.float32, device=dev))
    p32 = I.WorldParams(*(np.asarray(x, dtype=np.float32).astype(np.float64)
                          for x in (p.friction_scale, p.mass_scale, p.kp, p.kd)))
    ctrl = I.ctrl_targets(spec, W, T, seed_ctrl).astype(np.float32)
    ctrl_dev = torch.tensor(ctrl, device=dev)
    o = Oracle(spec)
    q = np.zeros((W, spec.nq))
    v = np.zeros((W, spec.nv))
    for w in range(W):
        q[w], v[w] = o.reset(0, w)
    a = np.zeros((W, spec.nv))
    sc = np.zeros(W, dtype=np.int64)
    out_g, out_o = {}, {}
    for t in range(T):
        b.step(ctrl_dev[t].reshape(-1), dec)
        st = o.step_batch(q, v, a, ctrl[t].astype(np.float64), dec, params=p32, step_count=sc + t,
                          world_id=np.arange(W, dtype=np.int32))
        if t >= T // 2 and t % 5 == 0:
            qg = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
            vg = b.get("qvel").view(W, spec.nv).double().cpu().numpy()
            sg = b.get("stats").view(W, 4).cpu().numpy()
            for name, val in stats_fn(o, qg, vg, sg[:, 0]).items():
                out_g.setdefault(name, []).append(val)
            for name, val in stats_fn(o, q, v, st[:, 0]).items():
                out_o.setdefault(name, []).append(val)
    assert np.isfinite(q).all() and not np.any(b.get("status").cpu().numpy() & 1)
    return out_g, out_o


def _agree(out_g, out_o, W, rel=0.02):
    """Ensemble means of per-world time means within 3 standard errors plus `rel` of the
    oracle mean (the systematic FP32-vs-FP64 difference of a chaotic system)."""
    rows = {}
    for name in out_g:
        mg, mo = np.mean(out_g[name], axis=0), np.mean(out_o[name], axis=0)
        se = np.sqrt(mg.var() / W + mo.var() / W)
        rows[name] = (float(mg.mean()), float(mo.mean()), float(se))
        assert abs(mg.mean() - mo.mean()) <= 3 * se + rel * abs(mo.mean()), (name, rows[name])
    print(rows)
    return rows


def test_humanoid_statistics_over_200_env_steps():
    """C2 morphology: 64 humanoids, 200 env steps (800 substeps; the robots fall and lie on
    the plane with box-foot and capsule contacts). Base height, energy, contacts per world
    and |qdot| over the last 100 env steps agree between the GPU and oracle ensembles."""
    spec = I.humanoid()

    def fn(o, q, v, ncon):
        e = np.array([_energy(o, spec, q[w], v[w]) for w in range(len(q))])
        return {"base height": q[:, 2], "energy": e, "contacts": ncon.astype(np.float64),
                "|qdot|": np.linalg.norm(v, axis=1)}
    g, o = _ensemble_stats(spec, 64, 200, stats_fn=fn)
    _agree(g, o, 64)


def test_manipulation_statistics_over_200_env_steps():
    """Manipulation world (box-box cube-table and finger-cube contacts, dense Hessian): 64
    worlds, 200 env steps under random arm targets. Cube height, energy, contacts per world
    and |qdot| over the last 100 env steps agree between the GPU and oracle ensembles."""
    spec = I.manipulation()
    cube_q = spec.jnt_qposadr()[-1]          # the free cube is the last joint

    def fn(o, q, v, ncon):
        e = np.array([_energy(o, spec, q[w], v[w]) for w in range(len(q))])
        return {"cube height": q[:, cube_q + 2], "energy": e, "contacts": ncon.astype(np.float64),
                "|qdot|": np.linalg.norm(v, axis=1)}
    g, o = _ensemble_stats(spec, 64, 200, stats_fn=fn)
    _agree(g, o, 64)


def test_quadruped_contact_statistics_over_200_env_steps():
    """C1: 64 quadrupeds, 200 env steps (800 substeps) under the seeded targets and
    randomised parameters. Ensemble means over the last 100 env steps of base height,
    contacts per world and |qdot| agree within 3 standard errors (plus 2 % for the
    systematic FP32-vs-FP64 difference of a chaotic system)."""
    from oracle import Oracle
    spec = I.quadruped()
    W, T, dec = 64, 200, 4
    b = Batch(Model(spec), W, working_set=3, warps_per_block=4, schedule=1)   # the benchmark's launch
    b.reset(0)
    p = I.randomised_params(spec, W, 7)
    dev = b.device
    b.set_param(0, "friction_scale", torch.tensor(p.friction_scale, dtype=torch.float32, device=dev))
    b.set_param(0, "mass_scale", torch.tensor(p.mass_scale, dtype=torch.float32, device=dev))
    b.set_param(0, "kp", torch.tensor(p.kp, dtype=torch.float32, device=dev))
    b.set_param(0, "kd", torch.tensor(p.kd, dtype=torch.float32, device=dev))
    p32 = I.WorldParams(*(np.asarray(x, dtype=np.float32).astype(np.float64)
                          for x in (p.friction_scale, p.mass_scale, p.kp, p.kd)))
    ctrl = I.ctrl_targets(spec, W, T, 11).astype(np.float32)
    ctrl_dev = torch.tensor(ctrl, device=dev)
    o = Oracle(spec)
    q = np.zeros((W, spec.nq))
    v = np.zeros((W, spec.nv))
    for w in range(W):
        q[w], v[w] = o.reset(0, w)
    a = np.zeros((W, spec.nv))
    sc = np.zeros(W, dtype=np.int64)
    hg, ho, cg, co, vgs, vos = [], [], [], [], [], []
    for t in range(T):
        b.step(ctrl_dev[t].reshape(-1), dec)
        st = o.step_batch(q, v, a, ctrl[t].astype(np.float64), dec, params=p32, step_count=sc + t,
                          world_id=np.arange(W, dtype=np.int32))
        if t >= T // 2:
            qg = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
            vg = b.get("qvel").view(W, spec.nv).double().cpu().numpy()
            sg = b.get("stats").view(W, 4).cpu().numpy()
            hg.append(qg[:, 2]); ho.append(q[:, 2].copy())
            cg.append(sg[:, 0].astype(np.float64)); co.append(st[:, 0].astype(np.float64))
            vgs.append(np.linalg.norm(vg, axis=1)); vos.append(np.linalg.norm(v, axis=1))
    assert np.isfinite(q).all() and not np.any(b.get("status").cpu().numpy() & 1)
    for name, xg, xo in (("base height", hg, ho), ("contacts", cg, co), ("|qdot|", vgs, vos)):
        mg, mo = np.mean(xg, axis=0), np.mean(xo, axis=0)     # per-world time means
        se = np.sqrt(mg.var() / W + mo.var() / W)
        assert abs(mg.mean() - mo.mean()) <= 3 * se + 0.02 * abs(mo.mean()), (name, mg.mean(), mo.mean(), se)
