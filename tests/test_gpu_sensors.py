"""Observation terms and the contact sensor on the GPU against the oracle's restatement
(oracle/sensors.py) on the same states and contacts."""
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


def _feet(spec):
    return sorted({int(spec.geom_body[g]) for g in range(spec.ngeom) if spec.geom_type[g] == I.BOX and spec.geom_body[g] > 0})


@pytest.mark.parametrize("options", [{}, dict(working_set=2), dict(working_set=3, warps_per_block=4, schedule=1)])
def test_observation_matches_oracle_on_gpu_states(options):
    from oracle import sensors as S
    specs = [I.quadruped(), I.humanoid(), I.manipulation()]
    Ws = [64, 48, 16]
    b = Batch([Model(s) for s in specs], Ws, **options)
    b.reset(2)
    ctrls = [torch.tensor(I.ctrl_targets(s, w, 30, 3), dtype=torch.float32, device="cuda") for s, w in zip(specs, Ws)]
    for t in range(30):
        flat = torch.cat([c[t].reshape(-1) for c in ctrls])
        b.step(flat, 4)
    torch.cuda.synchronize()
    q, v = b.get("qpos"), b.get("qvel")
    for g, (spec, W) in enumerate(zip(specs, Ws)):
        obs = b.observe(g, flat).double().cpu().numpy()
        qg = b.group_view(q, "qpos", g).double().cpu().numpy()
        vg = b.group_view(v, "qvel", g).double().cpu().numpy()
        cg = ctrls[g][29].double().cpu().numpy().reshape(W, -1)
        ref = np.stack([S.observe(spec, qg[w], vg[w], cg[w]) for w in range(W)])
        assert obs.shape == ref.shape
        err = np.abs(obs - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1.0)
        assert err.max() < 1e-5, (spec.name, err.max())


def test_contact_sensor_forces_and_air_time():
    """Humanoid feet: the sensor's net force equals the sum over the step's contact records
    (GPU records, and the oracle's records from the same state within the contact
    tolerance), and the air-time state follows the oracle's bookkeeping step by step."""
    from oracle import Oracle, sensors as S
    spec = I.humanoid()
    W, T, dt = 32, 40, 0.02
    b = Batch(Model(spec), W, write_contacts=True, working_set=2)
    b.reset(5)
    feet = torch.tensor(_feet(spec), dtype=torch.int32)
    assert len(feet) == 2
    state = torch.zeros((W, 2, 4), dtype=torch.float32, device="cuda")
    ref_state = np.zeros((W, 2, 4))
    ctrl = torch.tensor(I.ctrl_targets(spec, W, T, 6), dtype=torch.float32, device="cuda")
    o = Oracle(spec)
    touched = 0
    for t in range(T):
        q0 = b.get("qpos").view(W, spec.nq).double().cpu().numpy()
        v0 = b.get("qvel").view(W, spec.nv).double().cpu().numpy()
        a0 = b.get("qacc").view(W, spec.nv).double().cpu().numpy()
        sc = b.get("step_count").cpu().numpy()
        b.step(ctrl[t].reshape(-1), 4)
        f = b.contact_sensor(0, feet, state, threshold=1.0, dt=dt).double().cpu().numpy()
        con, cnt = b.contacts()
        con = con.view(W, -1, 24).double().cpu().numpy()
        cnt = cnt.cpu().numpy()
        for w in range(W):
            for k, body in enumerate(feet.tolist()):
                fk = S.body_force(con[w, : cnt[w]], body)
                np.testing.assert_allclose(f[w, k], fk, rtol=1e-5, atol=1e-4 * spec.body_mass.sum())
                ref_state[w, k] = S.air_time_update(ref_state[w, k], f[w, k], 1.0, dt)
                touched += int(ref_state[w, k, 0])
        if t % 8 == 7:   # oracle contacts from the same start state
            for w in range(0, W, 8):
                r = o.step(q0[w], v0[w], a0[w], ctrl[t, w].double().cpu().numpy(), nsub=4, step_count=int(sc[w]),
                           seed=5, world=w, want_contacts=True)
                if r["ncon"] != cnt[w]:
                    continue
                for k, body in enumerate(feet.tolist()):
                    fo = S.body_force(r["contacts"], body)
                    assert np.abs(f[w, k] - fo).max() <= 1e-3 * max(np.abs(fo).max(), spec.body_mass.sum() * 9.81)
    np.testing.assert_allclose(state.double().cpu().numpy(), ref_state, atol=1e-5)
    assert touched > W      # the feet do touch down
    assert np.any(ref_state[:, :, 3] > 0) or np.any(ref_state[:, :, 1] > 0)


def test_contact_sensor_needs_contact_records():
    spec = I.quadruped()
    b = Batch(Model(spec), 4)
    st = torch.zeros((4, 1, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        b.contact_sensor(0, torch.tensor([1]), st)
