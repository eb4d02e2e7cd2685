"""CUDA step against the FP64 oracle, through the C ABI (needs a B300).

Tolerances (relative, per world and field, floors in tests/parity.py):
  contact-free steps 1e-4, contact steps 1e-3 (qacc, qvel, qpos, total contact force, and
  every contact record's position, normal, penetration and world force, records matched
  by geom pair and position).
Threshold mismatches (contact count differs at the activation boundary) must stay
rare and are reported separately.
"""
import numpy as np
import pytest
import torch

from paper_2601_22074_b300 import build, inputs as I
from paper_2601_22074_b300.batch import Batch, Model

pytestmark = pytest.mark.gpu

TOL_FREE, TOL_CONTACT = 1e-4, 1e-3
# the two placements of the step: one fused persistent launch with shared-memory working
# sets, and the staged launches the benchmark's autotuner picks on a B300
PLACEMENTS = [pytest.param({}, id="fused"), pytest.param(dict(working_set=2, warps_per_block=2), id="staged"),
              pytest.param(dict(working_set=3, warps_per_block=4, schedule=1), id="grouped"),
              pytest.param(dict(working_set=3, warps_per_block=4, schedule=1, lane_solve=1), id="lane")]
BENCH_LAUNCH = dict(working_set=3, warps_per_block=4, schedule=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _check(rep, tol, max_mismatch=0.02):
    from parity import check
    check(rep, tol, max_mismatch)


def test_pendulum_contact_free():
    from parity import teacher_forced
    rep = teacher_forced(I.pendulum(3), W=64, nsteps=100, decimation=1)
    assert rep.contact_steps == 0
    _check(rep, TOL_FREE, max_mismatch=0)


def test_humanoid_contact_free_airborne():
    from parity import teacher_forced
    rep = teacher_forced(I.humanoid(), W=32, nsteps=20, decimation=4, lift=5.0)
    assert rep.contact_steps == 0 and rep.compared == 32 * 20
    _check(rep, TOL_FREE, max_mismatch=0)


@pytest.mark.parametrize("options", PLACEMENTS[:3])
def test_spatial_chain_contact_free(options):
    """Hinges about tilted axes through off-origin anchors, a slide joint and rotated body
    frames: every term of the kinematics (the joints' relative transforms composed down the
    tree) and of the dynamics, against the oracle in each placement."""
    from parity import teacher_forced
    rep = teacher_forced(I.spatial_chain(), W=64, nsteps=40, decimation=4, options=options)
    assert rep.contact_steps == 0 and rep.compared == 64 * 40
    _check(rep, TOL_FREE, max_mismatch=0)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_quadruped_contact_steps(options):
    from parity import teacher_forced
    rep = teacher_forced(I.quadruped(), W=48, nsteps=25, decimation=4, warm_steps=20, options=options)
    assert rep.contact_steps > 100
    _check(rep, TOL_CONTACT)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_humanoid_contact_steps(options):
    from parity import teacher_forced
    rep = teacher_forced(I.humanoid(), W=48, nsteps=15, decimation=4, warm_steps=60, options=options)
    assert rep.contact_steps > 100
    _check(rep, TOL_CONTACT)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_manipulation_contact_steps(options):
    from parity import teacher_forced
    rep = teacher_forced(I.manipulation(), W=48, nsteps=20, decimation=4, warm_steps=20, options=options,
                         spread_ulps=1)
    assert rep.contact_steps > 100
    # the case's conditioning beside the GPU error: the oracle's own movement when its FP32
    # input state moves by one ulp per component
    print("oracle spread at 1 ulp:", {f: (rep.max("spread_" + f), rep.p99("spread_" + f))
                                      for f in ("qacc", "qvel", "qpos")})
    _check(rep, TOL_CONTACT)


@pytest.mark.parametrize("options", PLACEMENTS)
def test_manipulation_pinch_cross_tree_contacts(options):
    """Gripper lowered around the cube, arm held by stiff gains, fingers driven closed:
    sustained finger-cube (cross-tree, dense Hessian) and cube-table box-box contacts."""
    from parity import teacher_forced
    spec = I.manipulation(base_z=0.38, cube_x=0.469, arm_kp=500.0, arm_kd=1.0)
    rep = teacher_forced(spec, W=16, nsteps=10, decimation=4, warm_steps=30, pinch=True, options=options,
                         spread_ulps=1)
    assert rep.contact_steps >= 120 and rep.max_ncon >= 8
    print("oracle spread at 1 ulp:", {f: (rep.max("spread_" + f), rep.p99("spread_" + f))
                                      for f in ("qacc", "qvel", "qpos")})
    _check(rep, TOL_CONTACT)


def test_humanoid_full_size_sampled():
    """8192 worlds in the benchmark's launch configuration; 48 sampled worlds checked."""
    from parity import teacher_forced
    sample = np.random.default_rng(0).choice(8192, 48, replace=False)
    rep = teacher_forced(I.humanoid(), W=8192, nsteps=2, decimation=4, warm_steps=40,
                         sample=sample, options=BENCH_LAUNCH)
    _check(rep, TOL_CONTACT)


def test_humanoid_full_size_sampled_lane_solve():
    """8192 humanoids, the solve of worlds with up to 8 contacts one world per lane."""
    from parity import teacher_forced
    sample = np.random.default_rng(2).choice(8192, 48, replace=False)
    rep = teacher_forced(I.humanoid(), W=8192, nsteps=2, decimation=4, warm_steps=40,
                         sample=sample, options=dict(BENCH_LAUNCH, lane_solve=1))
    _check(rep, TOL_CONTACT)


def test_lane_solve_runs_and_agrees_with_the_warp_solve():
    """The lane solve is a different instruction stream (sums in dof order, M products
    through M's factor): results differ in FP32 rounding from the one-world-per-warp
    solve, so the lane path demonstrably ran, and agree within the contact tolerance; a
    mixed batch keeps the manipulation group (dense Hessian) on the warp solve."""
    specs = [I.pendulum(3), I.quadruped(), I.humanoid(), I.manipulation()]
    Ws = [32, 96, 96, 32]
    models = [Model(s) for s in specs]
    ctrls = [torch.tensor(I.ctrl_targets(s, w, 30, 4), dtype=torch.float32, device="cuda")
             for s, w in zip(specs, Ws)]
    out = []
    for lane in (0, 1):
        b = Batch(models, Ws, **dict(BENCH_LAUNCH, lane_solve=lane))
        b.reset(3)
        for t in range(30):
            b.step(torch.cat([c[t].reshape(-1) for c in ctrls]), 4)
        torch.cuda.synchronize()
        out.append(b)
    for f, floor in (("qacc", 9.81), ("qvel", 1.0)):
        x, y = out[0].get(f), out[1].get(f)
        for g, spec in enumerate(specs):
            xg, yg = out[0].group_view(x, f, g), out[1].group_view(y, f, g)
            if spec.name in ("quadruped", "humanoid") and f == "qacc":
                assert not torch.equal(xg, yg), spec.name        # a different solve ran
            if spec.name in ("pendulum", "manipulation"):
                assert torch.equal(xg, yg), spec.name            # untouched groups: bitwise
    st = out[1].get("stats")
    for g in (1, 2):
        assert int(out[1].group_view(st, "stats", g)[:, 0].max()) > 0   # contacts were solved


def test_lane_solve_needs_the_sorted_staged_placement():
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        Batch(Model(I.humanoid()), 8, working_set=0, lane_solve=1)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        Batch(Model(I.humanoid()), 8, working_set=3, schedule=0, lane_solve=1)


def test_quadruped_full_size_sampled():
    from parity import teacher_forced
    sample = np.random.default_rng(1).choice(4096, 48, replace=False)
    rep = teacher_forced(I.quadruped(), W=4096, nsteps=2, decimation=4, warm_steps=30,
                         sample=sample, options=BENCH_LAUNCH)
    _check(rep, TOL_CONTACT)


def test_hetero_full_size_sampled():
    """The four-morphology 9216-world batch (2048 pendulum, 4096 quadruped, 2048 humanoid,
    1024 manipulation) in the benchmark's launches; 24 sampled worlds per group checked."""
    from parity import teacher_forced_mixed
    specs = [I.pendulum(3), I.quadruped(), I.humanoid(), I.manipulation()]
    for opts in (BENCH_LAUNCH, dict(BENCH_LAUNCH, lane_solve=1)):
        reps = teacher_forced_mixed(specs, [2048, 4096, 2048, 1024], nsteps=2, decimation=4, samples=24,
                                    warm_steps=30, options=opts)
        for spec, rep in zip(specs, reps):
            _check(rep, TOL_CONTACT)
        assert sum(r.contact_steps for r in reps) > 40


def test_push_event_matches_oracle():
    """step count 200 = push period: the Philox planar kick is applied on both sides."""
    from parity import teacher_forced
    rep = teacher_forced(I.humanoid(), W=32, nsteps=1, decimation=4, lift=5.0,
                         step_count_start=200)
    _check(rep, TOL_FREE, max_mismatch=0)


def test_fp64_pivot_fallback_path():
    """A large pivot threshold forces the FP64 refactor; results still match."""
    from parity import teacher_forced
    spec = I.humanoid(pivot_tau=0.9)
    rep = teacher_forced(spec, W=16, nsteps=6, decimation=4, warm_steps=60)
    assert rep.fallbacks > 0
    _check(rep, TOL_CONTACT)


def test_reset_matches_oracle_and_is_seeded():
    from oracle import Oracle
    spec = I.pendulum(3)
    b = Batch(Model(spec), 256)
    b.reset(1234)
    q = b.get("qpos").view(256, 3).double().cpu().numpy()
    o = Oracle(spec)
    ref = np.stack([o.reset(1234, w)[0] for w in range(256)])
    np.testing.assert_allclose(q, ref, atol=2e-6)
    b.reset(1235)
    assert not np.allclose(b.get("qpos").view(256, 3).double().cpu().numpy(), ref)


def _run(spec, W, nsteps, seed=3, decimation=4):
    b = Batch(Model(spec), W)
    b.reset(seed)
    ctrl = torch.tensor(I.ctrl_targets(spec, W, nsteps, 5), dtype=torch.float32, device="cuda")
    for t in range(nsteps):
        b.step(ctrl[t] if spec.nu else None, decimation)
    torch.cuda.synchronize()
    return b, ctrl


def test_determinism_and_checkpoint_resume_bitwise():
    spec = I.humanoid()
    b1, ctrl = _run(spec, 256, 10)
    b2, _ = _run(spec, 256, 10)
    assert torch.equal(b1.get("qpos"), b2.get("qpos"))
    snap = b1.state_save()
    for t in range(5):
        b1.step(ctrl[t], 4)
    after = b1.get("qpos").clone()
    b1.state_restore(snap)
    for t in range(5):
        b1.step(ctrl[t], 4)
    torch.cuda.synchronize()
    assert torch.equal(b1.get("qpos"), after)


def test_graph_replay_matches_eager():
    spec = I.quadruped()
    W, n = 512, 6
    b1, ctrl = _run(spec, W, 0)
    b2, _ = _run(spec, W, 0)
    ctrl = torch.tensor(I.ctrl_targets(spec, W, n, 5), dtype=torch.float32, device="cuda")
    for t in range(n):
        b1.step(ctrl[t], 4)
    s = torch.cuda.Stream()
    b2.capture(ctrl, W * spec.nu, 4, n, s)
    b2.replay(s)
    s.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(b1.get("qpos"), b2.get("qpos"))
    assert torch.equal(b1.get("qvel"), b2.get("qvel"))


def test_mixed_batch_equals_separate_batches():
    """Each world's result is identical alone and in a heterogeneous batch."""
    specs = [I.pendulum(3), I.quadruped(), I.humanoid(), I.manipulation()]
    Ws = [64, 96, 80, 40]
    models = [Model(s) for s in specs]
    mixed = Batch(models, Ws)
    mixed.reset(9)
    ctrls = [torch.tensor(I.ctrl_targets(s, w, 4, 2), dtype=torch.float32, device="cuda")
             for s, w in zip(specs, Ws)]
    for t in range(4):
        flat = torch.cat([c[t].reshape(-1) for c in ctrls])
        mixed.step(flat, 4)
    torch.cuda.synchronize()
    qm = mixed.get("qpos")
    for g, (m, s, w) in enumerate(zip(models, specs, Ws)):
        alone = Batch(m, w)
        alone.reset(9)
        for t in range(4):
            alone.step(ctrls[g][t].reshape(-1) if s.nu else None, 4)
        torch.cuda.synchronize()
        assert torch.equal(mixed.group_view(qm, "qpos", g), alone.get("qpos").view(w, s.nq))


def test_nan_world_is_flagged_and_isolated():
    spec = I.quadruped()
    W = 64
    b = Batch(Model(spec), W)
    b.reset(0)
    v = b.get("qvel").view(W, spec.nv).clone()
    v[5, 7] = float("nan")
    b.set("qvel", v.reshape(-1))
    ctrl = torch.zeros(W * spec.nu, device="cuda")
    b.step(ctrl, 4)
    torch.cuda.synchronize()
    st = b.get("status").cpu().numpy()
    assert st[5] & 1
    assert not np.any(np.delete(st, 5) & 1)
    assert torch.isfinite(b.get("qpos").view(W, spec.nq)[np.delete(np.arange(W), 5)]).all()


@pytest.mark.parametrize("options", PLACEMENTS)
def test_history_ring_keeps_the_last_states_of_a_failing_world(options):
    """A ring of the last 3 env steps per world: it holds the states the step produced,
    oldest first, and a world whose velocity turns non-finite keeps its last finite
    states there (the replay record of a failed world)."""
    spec = I.quadruped()
    W, H = 16, 3
    b = Batch(Model(spec), W, history=H, **options)
    b.reset(4)
    ctrl = torch.tensor(I.ctrl_targets(spec, W, 8, 9), dtype=torch.float32, device="cuda")
    seen = []
    for t in range(6):
        if t == 4:
            v = b.get("qvel").view(W, spec.nv).clone()
            v[5, 7] = float("nan")
            b.set("qvel", v.reshape(-1))
        b.step(ctrl[t].reshape(-1), 4)
        torch.cuda.synchronize()
        seen.append(torch.cat([b.get("qpos").view(W, spec.nq), b.get("qvel").view(W, spec.nv)], dim=1).clone())
    rows, n = b.history(0, 2)
    assert n == H
    for k in range(H):
        assert torch.equal(rows[k], seen[3 + k][2])
    rows5, _ = b.history(0, 5)
    assert torch.isfinite(rows5[0]).all()          # the step before the planted NaN
    assert not torch.isfinite(rows5[2]).all()
    fresh = Batch(Model(spec), W, history=H, **options)
    fresh.reset(1)
    rows0, n0 = fresh.history(0, 0)
    assert n0 == 0


def test_dynamic_schedule_and_launch_shapes_give_identical_results():
    """Heaviest-first dynamic queue, static order, CTA shapes and working-set placement of
    the fused kernel: bitwise identical worlds. Staged execution (separately compiled
    per-stage kernels): within the contact tolerance."""
    specs = [I.pendulum(3), I.quadruped(), I.humanoid(), I.manipulation()]
    Ws = [32, 64, 48, 24]
    models = [Model(s) for s in specs]
    ctrls = [torch.tensor(I.ctrl_targets(s, w, 3, 4), dtype=torch.float32, device="cuda")
             for s, w in zip(specs, Ws)]
    out = []
    for opts in (dict(schedule=0, warps_per_block=4), dict(schedule=1, warps_per_block=2),
                 dict(schedule=1, warps_per_block=1), dict(schedule=1, working_set=1),
                 dict(schedule=0, warps_per_block=2, working_set=1), dict(working_set=2, warps_per_block=1),
                 dict(working_set=2, warps_per_block=2), dict(working_set=2, schedule=1), dict(working_set=2),
                 dict(working_set=3, warps_per_block=1), dict(working_set=3, warps_per_block=4, schedule=1)):
        b = Batch(models, Ws, **opts)
        b.reset(3)
        for t in range(3):
            b.step(torch.cat([c[t].reshape(-1) for c in ctrls]), 4)
        torch.cuda.synchronize()
        out.append((b.get("qpos"), b.get("qvel"), b.get("stats")))
    fused, staged, grouped = out[:5], out[5:9], out[9:]
    for o in fused[1:]:
        for x, y in zip(fused[0], o):
            assert torch.equal(x, y)
    for group in (staged, grouped):             # CTA shapes and solve order: same kernels, bitwise
        for o in group[1:]:
            for x, y in zip(group[0], o):
                assert torch.equal(x, y)
    for other in (staged[0], grouped[0]):       # separately compiled kernels: within tolerance
        for x, y in zip(fused[0][:2], other[:2]):
            err = (x.double() - y.double()).abs().max() / max(float(x.abs().max()), 1.0)
            assert float(err) <= TOL_CONTACT


def test_autotuner_returns_a_measured_choice():
    from paper_2601_22074_b300 import tune
    models = [Model(I.quadruped()), Model(I.humanoid())]
    r = tune.autotune(models, [256, 256], steps=1, warmup=2)
    assert r["options"] in [o for o, _ in r["table"]]
    assert len(r["table"]) == 30 and all(ms > 0 for _, ms in r["table"])


def test_step_profile_times_each_stage_and_steps_like_b3p_step():
    """Per-stage timing of the staged placement: one launch per stage per substep, every
    stage timed, and the state update bitwise equal to b3p_step's; fused placements are
    refused (their step is one kernel)."""
    from paper_2601_22074_b300 import _lib as LB
    specs = [I.quadruped(), I.humanoid()]
    Ws = [96, 64]
    models = [Model(s) for s in specs]
    ctrls = [torch.tensor(I.ctrl_targets(s, w, 4, 8), dtype=torch.float32, device="cuda")
             for s, w in zip(specs, Ws)]
    a, b = Batch(models, Ws, working_set=2), Batch(models, Ws, working_set=2)
    a.reset(9)
    b.reset(9)
    tot = np.zeros(LB.NSTAGES)
    for t in range(4):
        flat = torch.cat([c[t].reshape(-1) for c in ctrls])
        a.step(flat, 4)
        ms, n = b.step_profile(flat, 4)
        assert n.tolist() == [1, 4, 4, 4, 4, 4, 4, 1]
        assert np.all(ms > 0)
        tot += ms
    torch.cuda.synchronize()
    for f in ("qpos", "qvel", "qacc", "stats"):
        assert torch.equal(a.get(f), b.get(f)), f
    assert tot[LB.STAGES.index("solve")] > tot[LB.STAGES.index("integrate")]
    fused = Batch(models, Ws)
    fused.reset(9)
    with pytest.raises(RuntimeError, match="staged"):
        fused.step_profile(torch.cat([c[0].reshape(-1) for c in ctrls]), 4)


def test_plain_per_stage_path_matches_fused_step():
    """The no-fusion comparator (per-stage kernels, global workspace) reproduces the fused
    step within the contact tolerance on a mixed batch."""
    specs = [I.quadruped(), I.humanoid(), I.manipulation()]
    Ws = [64, 64, 32]
    models = [Model(s) for s in specs]
    ctrls = [torch.tensor(I.ctrl_targets(s, w, 6, 4), dtype=torch.float32, device="cuda")
             for s, w in zip(specs, Ws)]
    fused, plain = Batch(models, Ws), Batch(models, Ws)
    fused.reset(5)
    plain.reset(5)
    for t in range(6):
        flat = torch.cat([c[t].reshape(-1) for c in ctrls])
        fused.step(flat, 4)
        plain.step_plain(flat, 4)
        torch.cuda.synchronize()
        for f, floor in (("qacc", 9.81), ("qvel", 1.0), ("qpos", 1.0)):
            a, b = fused.get(f), plain.get(f)
            for g in range(len(specs)):
                x, y = fused.group_view(a, f, g).double(), plain.group_view(b, f, g).double()
                err = (x - y).abs().max(dim=1).values / torch.clamp(y.abs().max(dim=1).values, min=floor)
                assert float(err.max()) <= TOL_CONTACT, (t, f, g, float(err.max()))
        # re-synchronise: the comparator starts every step from the fused state
        for f in ("qpos", "qvel", "qacc"):
            plain.set(f, fused.get(f))
