"""Conditioning of the contact parity cases (CPU): how far the FP64 oracle's own env step
moves when its FP32 input state moves by one FP32 ulp per component. The GPU parity bar
(1e-3 relative on contact steps) is only meaningful if it sits well above this spread;
the GPU tests print the same spread beside the GPU error on the states they compare."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2601_22074_b300 import inputs as I
from parity import FLOORS, ulp_move, world_err


@pytest.mark.parametrize("name", ["manipulation", "humanoid", "quadruped"])
def test_one_ulp_input_spread_is_far_below_the_contact_bar(name):
    spec = getattr(I, name)()
    W = 24
    o = Oracle(spec)
    q, v, a = np.zeros((W, spec.nq)), np.zeros((W, spec.nv)), np.zeros((W, spec.nv))
    for w in range(W):
        q[w], v[w] = o.reset(0, w)
    p = I.randomised_params(spec, W, 7)
    ctrl = I.ctrl_targets(spec, W, 34, 11)
    sc = np.zeros(W, dtype=np.int64)
    for t in range(30):                     # into contact
        o.step_batch(q, v, a, ctrl[t], 4, params=p, step_count=sc + t)
    rng = np.random.default_rng(0)
    spread = {k: [] for k in ("qacc", "qvel", "qpos")}
    contacts = 0
    for t in range(30, 34):
        q32, v32 = (x.astype(np.float32).astype(np.float64) for x in (q, v))
        for w in range(W):
            kw = dict(nsub=4, friction_scale=p.friction_scale[w], mass_scale=p.mass_scale[w], kp=p.kp[w],
                      kd=p.kd[w], step_count=t, world=w)
            r = o.step(q32[w], v32[w], a[w], ctrl[t, w], **kw)
            rp = o.step(ulp_move(q32[w], 1, rng), ulp_move(v32[w], 1, rng), a[w], ctrl[t, w], **kw)
            contacts += r["ncon"] > 0
            for k in spread:
                spread[k].append(world_err(rp[k], r[k], FLOORS[k]))
        o.step_batch(q, v, a, ctrl[t], 4, params=p, step_count=sc + t)
    print(name, {k: (max(x), float(np.percentile(x, 99))) for k, x in spread.items()})
    assert contacts >= W
    assert max(max(x) for x in spread.values()) < 1e-4
