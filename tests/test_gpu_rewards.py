"""Fused reward/termination launch and the contact-force history on the GPU, against
the oracle's restatements (oracle/rewards.py), and the whole per-env-step RL loop --
step, contact sensor with history, reward -- recorded in one CUDA graph."""
import numpy as np
import pytest
import torch

from paper_2601_22074_b300 import _lib as L, build, inputs as I
from paper_2601_22074_b300.batch import Batch, Model, RewardConfig

pytestmark = pytest.mark.gpu

WEIGHTS = [1.0, 0.5, -2.0, -0.05, -0.01, -10.0, -0.1, 1.0, -1.0, -2.5e-7]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _bodies_with(spec, gtype):
    return sorted({int(b) for t, b in zip(spec.geom_type, spec.geom_body) if t == gtype and b > 0})


def _setup(spec, W, feet, illegal, T, seed=3):
    b = Batch(Model(spec), W, write_contacts=True, working_set=3, warps_per_block=4, schedule=1)
    b.reset(seed)
    p = I.randomised_params(spec, W, 5)
    b.set_param(0, "kp", torch.tensor(p.kp, dtype=torch.float32, device="cuda"))
    b.set_param(0, "kd", torch.tensor(p.kd, dtype=torch.float32, device="cuda"))
    ctrl = torch.tensor(I.ctrl_targets(spec, W, T + 1, 9), dtype=torch.float32, device="cuda").reshape(T + 1, -1)
    cfg = RewardConfig(WEIGHTS, dt=spec.opt.timestep * 4, min_base_height=0.45 if spec.name == "humanoid" else 0.15,
                       max_tilt=0.8, max_episode_steps=T - 2, feet=feet, illegal=illegal)
    rng = np.random.default_rng(seed)
    cmd = torch.tensor(rng.uniform(-1, 1, (W, 3)), dtype=torch.float32, device="cuda")
    return b, ctrl, cfg, cmd


def _out(W):
    return dict(reward=torch.zeros(W, device="cuda"), terms=torch.zeros(W, L.REWARD_NTERMS, device="cuda"),
                episode=torch.zeros(W, L.REWARD_NTERMS, device="cuda"),
                done=torch.zeros(W, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("name", ["quadruped", "humanoid"])
def test_reward_terms_and_termination_match_oracle(name):
    from oracle import Oracle
    from oracle import rewards as RW
    spec = getattr(I, name)()
    feet = _bodies_with(spec, I.SPHERE if name == "quadruped" else I.BOX)
    illegal = [1]                                   # the base touching the ground ends the episode
    W, T = 48, 40
    b, ctrl, cfg, cmd = _setup(spec, W, feet, illegal, T)
    o = Oracle(spec)
    ids = torch.tensor(feet, dtype=torch.int32, device="cuda")
    state = torch.zeros(W, len(feet), 4, device="cuda")
    hist = torch.zeros(W, len(feet), 5, 3, device="cuda")
    out = _out(W)
    ocfg = dict(weight=cfg.weight, sigma_lin=cfg.sigma_lin, sigma_ang=cfg.sigma_ang,
                air_time_target=cfg.air_time_target, dt=cfg.dt, min_base_height=cfg.min_base_height,
                max_tilt=cfg.max_tilt, max_episode_steps=cfg.max_episode_steps)
    f32 = lambda x: np.asarray(x, dtype=np.float32).astype(np.float64)   # noqa: E731
    rings = np.zeros((W, len(feet), 5, 3))
    ep_orc = np.zeros((W, L.REWARD_NTERMS))
    worst, bit_mismatch, compared, done_seen, touchdowns = 0.0, 0, 0, 0, 0
    cm = cmd.double().cpu().numpy()
    for t in range(1, T + 1):
        b.step(ctrl[t], 4)
        force = b.contact_sensor(0, ids, state, threshold=1.0, dt=cfg.dt, history=hist)
        b.reward(0, cfg, cmd, ctrl[t], ctrl[t - 1], state, out)
        torch.cuda.synchronize()
        q = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
        v = b.get("qvel").view(W, spec.nv).double().cpu().numpy()
        a = b.get("qacc").view(W, spec.nv).double().cpu().numpy()
        sc = b.get("step_count").cpu().numpy()
        st = state.double().cpu().numpy()
        con, cnt = b.contacts()
        con = con.view(W, -1, 24).double().cpu().numpy()
        cnt = cnt.cpu().numpy()
        fr = force.double().cpu().numpy()
        a_now = ctrl[t].view(W, spec.nu).double().cpu().numpy()
        a_prev = ctrl[t - 1].view(W, spec.nu).double().cpu().numpy()
        rg, tg, dg = (out[k].double().cpu().numpy() for k in ("reward", "terms", "done"))
        for w in range(W):
            r, c, d = RW.reward(o, spec, q[w], v[w], a[w], f32(cm[w]), a_now[w], a_prev[w], st[w], feet, ocfg,
                                contacts=con[w, : cnt[w]], illegal=illegal, step_count=int(sc[w]))
            scale = 1.0 + abs(r)
            worst = max(worst, abs(rg[w] - r) / scale, float(np.abs(tg[w] - c).max()) / scale)
            compared += 1
            bit_mismatch += int(dg[w]) != d
            done_seen += d != 0
            ep_orc[w] += c
            touchdowns += int(np.sum((st[w, :, 0] > 0.5) & (st[w, :, 2] <= 1.5 * cfg.dt)))
            for k in range(len(feet)):
                RW.history_write(rings[w, k], int(sc[w]), fr[w, k])
    print(name, "reward/terms rel err", worst, "done mismatches", bit_mismatch, "of", compared,
          "done worlds", done_seen, "touchdowns", touchdowns)
    assert worst <= 1e-4
    assert bit_mismatch <= 0.01 * compared and done_seen > 0
    assert touchdowns > 0
    ep = out["episode"].double().cpu().numpy()
    assert np.abs(ep - ep_orc).max() <= 1e-4 * (1.0 + np.abs(ep_orc).max())
    np.testing.assert_array_equal(hist.double().cpu().numpy(), rings)   # the ring holds the sensor's forces


def test_step_sensor_and_reward_replay_from_one_cuda_graph():
    """The RL loop of one env step -- b3p_step, the contact sensor with its force history,
    the reward and termination launch -- captured once in a CUDA graph and replayed: every
    output equals the same calls made eagerly from the same state, bitwise."""
    spec = I.humanoid()
    feet = _bodies_with(spec, I.BOX)
    W, T = 64, 6
    runs = []
    for graph in (False, True):
        b, ctrl, cfg, cmd = _setup(spec, W, feet, [1], T + 2, seed=11)
        ids = torch.tensor(feet, dtype=torch.int32, device="cuda")
        state = torch.zeros(W, len(feet), 4, device="cuda")
        hist = torch.zeros(W, len(feet), 4, 3, device="cuda")
        force = torch.zeros(W, len(feet), 3, device="cuda")
        act = torch.zeros_like(ctrl[0])
        prev = torch.zeros_like(ctrl[0])
        out = _out(W)
        for t in range(10):                      # fall into contact first (eager)
            b.step(ctrl[0], 4)
        torch.cuda.synchronize()

        def body():
            b.step(act, 4)
            b.contact_sensor(0, ids, state, threshold=1.0, dt=cfg.dt, history=hist, out=force)
            b.reward(0, cfg, cmd, act, prev, state, out)

        g = None
        if graph:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            snap = b.state_save()
            with torch.cuda.graph(g, stream=s):
                body()
            b.state_restore(snap)
            state.zero_(); hist.zero_(); out["episode"].zero_()
            torch.cuda.synchronize()
        rec = []
        for t in range(T):
            prev.copy_(act)
            act.copy_(ctrl[t + 1])
            if graph:
                g.replay()
            else:
                body()
            torch.cuda.synchronize()
            rec.append([x.clone() for x in (b.get("qpos"), force, hist, out["reward"], out["terms"],
                                            out["episode"], out["done"])])
        runs.append(rec)
    for eager, replay in zip(*runs):
        for x, y in zip(eager, replay):
            assert torch.equal(x, y)


def test_reward_rejects_bad_arguments():
    spec = I.quadruped()
    b = Batch(Model(spec), 8, write_contacts=False)
    cmd = torch.zeros(8, 3, device="cuda")
    a = torch.zeros(8 * spec.nu, device="cuda")
    out = _out(8)
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):           # illegal contacts need contacts
        b.reward(0, RewardConfig(WEIGHTS, dt=0.02, illegal=[1]), cmd, a, a, None, out)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):           # body out of range
        b.reward(0, RewardConfig(WEIGHTS, dt=0.02, feet=[99]), cmd, a, a, torch.zeros(8, 1, 4, device="cuda"), out)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):           # actuated group without actions
        b.reward(0, RewardConfig(WEIGHTS, dt=0.02), cmd, None, None, None, out)
