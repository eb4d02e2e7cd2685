"""Every workload and readout on the checked build of the library (per-world accessor
and update-list indices verified on the GPU; a failure is counted and the access
redirected, never performed): no index may fail. Runs in a child process, since one
process loads one build."""
import os
import subprocess
import sys

import pytest
import torch

from paper_2601_22074_b300 import build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes as C, sys
import numpy as np, torch
from paper_2601_22074_b300 import _lib as L, inputs as I
from paper_2601_22074_b300.batch import Batch, Model
lib = L.load()
lib.b3p_check_read.argtypes = [C.POINTER(C.c_uint)]
def run(specs, Ws, steps=6, **opts):
    b = Batch([Model(s) for s in specs], Ws, **opts)
    b.reset(1)
    ctrls = [torch.tensor(I.ctrl_targets(s, w, steps, 2), dtype=torch.float32, device="cuda") for s, w in zip(specs, Ws)]
    for t in range(steps):
        flat = torch.cat([c[t].reshape(-1) for c in ctrls]) if any(s.nu for s in specs) else None
        b.step(flat, 4)
    torch.cuda.synchronize()
    return b, flat
for opts in (dict(), dict(working_set=2, schedule=1, history=2), dict(working_set=1, schedule=1)):
    run([I.pendulum(3), I.quadruped(), I.humanoid(), I.manipulation()], [64, 64, 64, 32], **opts)
run([I.manipulation(base_z=0.38, cube_x=0.469, arm_kp=500.0, arm_kd=1.0)], [32], steps=20)
run([I.with_limits(I.humanoid(), 0.3), I.with_dcmotor(I.quadruped(), 15.0, 20.0, 8.0)], [32, 32], working_set=2)
run([I.with_delay(I.with_terrain(I.quadruped(), amplitude=0.05), 2), I.with_terrain(I.humanoid(), amplitude=0.05)],
    [32, 32], working_set=2, schedule=1)
b, flat = run([I.quadruped(), I.manipulation()], [16, 16], write_contacts=True, working_set=2, history=3)
b.observe(0, flat); b.observe(1, flat)
st = torch.zeros((16, 2, 4), dtype=torch.float32, device="cuda")
b.contact_sensor(0, torch.tensor([4, 7]), st, 1.0, 0.02)
b.raycast(0, 1, torch.zeros((8, 3)), torch.tensor([[0.0, 0.0, -1.0]] * 8))
b.raycast(1, 7, torch.zeros((8, 3)), torch.tensor([[0.0, 0.0, -1.0]] * 8), world_only=False)
b.diffik(1, 7, [0.0, 0.0, 0.05], torch.zeros((16, 3)), flat)
b.history(0, 3)
# grouped staging with the lane-per-world solve, boxes on bumps (convex grid vertices against
# box faces), the ray-cast hierarchy with hits and normals, the force-history sensor and the
# reward launch
run([I.pendulum(3), I.quadruped(), I.humanoid(), I.manipulation()], [32, 64, 64, 32], working_set=3, schedule=1,
    lane_solve=1)
import dataclasses
terrain = I.with_terrain(I.quadruped(), nrow=41, ncol=41, half=1.0, amplitude=0.12, seed=7).hfield_data
box = I.free_body(I.BOX, (0.12, 0.07, 0.04), mass=1.0, pos=(0.1, -0.2, 0.2))
gt = box.geom_type.copy(); gt[0] = I.HFIELD
box = dataclasses.replace(box, geom_type=gt, hfield_data=terrain, hfield_size=(1.0, 1.0))
run([box, I.with_terrain(I.humanoid(), amplitude=0.05)], [16, 16], steps=12, working_set=3, schedule=1)
hb, hflat = run([I.humanoid(), I.manipulation()], [16, 16], write_contacts=True, working_set=3, schedule=1)
rays = torch.randn(24, 3)
rays = rays / rays.norm(dim=1, keepdim=True)
for hier in (True, False):
    hb.raycast_hits(0, 30, torch.zeros((24, 3)), rays, world_only=False, hierarchy=hier)
    hb.raycast_hits(1, 10, torch.zeros((24, 3)), rays, world_only=False, hierarchy=hier)
from paper_2601_22074_b300.batch import RewardConfig
feet = [b_ for t_, b_ in zip(I.humanoid().geom_type, I.humanoid().geom_body) if t_ == I.BOX and b_ > 0]
hst = torch.zeros((16, len(feet), 4), dtype=torch.float32, device="cuda")
hist = torch.zeros((16, len(feet), 3, 3), dtype=torch.float32, device="cuda")
hb.contact_sensor(0, torch.tensor(feet), hst, 1.0, 0.02, history=hist)
out = dict(reward=torch.zeros(16, device="cuda"), terms=torch.zeros(16, 10, device="cuda"),
           episode=torch.zeros(16, 10, device="cuda"), done=torch.zeros(16, dtype=torch.int32, device="cuda"))
hb.reward(0, RewardConfig([1.0] * 10, dt=0.02, min_base_height=0.4, max_tilt=0.8, max_episode_steps=5, feet=feet,
                          illegal=[1]), torch.zeros((16, 3), device="cuda"), hflat, hflat, hst, out)
torch.cuda.synchronize()
out = (C.c_uint * 2)()
assert lib.b3p_check_read(out) == 0
print("CHECK", out[0], out[1])
'''


def test_checked_build_reports_no_index_failure():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = build.build_checked()
    env = dict(os.environ, B3P_LIB_PATH=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("CHECK")][-1]
    count, site = (int(x) for x in line.split()[1:])
    assert count == 0, f"{count} failed index checks, first at site {site}"
