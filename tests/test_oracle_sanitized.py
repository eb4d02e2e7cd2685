"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU, child process
with the sanitizer runtime preloaded): model compilation and steps of every morphology,
with contacts, box-box, limits, DC motors, terrain, per-world inertias and the readout
helpers, raise no report."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
from oracle import Oracle, ik
from paper_2601_22074_b300 import inputs as I
specs = [I.pendulum(3), I.quadruped(), I.humanoid(), I.manipulation(),
         I.with_limits(I.humanoid(), 0.3), I.with_dcmotor(I.quadruped(), 15.0, 20.0, 8.0),
         I.with_terrain(I.quadruped(), amplitude=0.05), I.manipulation(base_z=0.38, cube_x=0.469, arm_kp=500.0, arm_kd=1.0)]
for spec in specs:
    o = Oracle(spec)
    q, v = o.reset(0, 1)
    a = np.zeros(spec.nv)
    u = spec.qpos_reset[spec.act_qposadr()] if spec.nu else None
    inert = I.randomised_inertia(spec, 1, 0, 0.05)[0]
    for t in range(3):
        r = o.step(q, v, a, u, nsub=4, want_contacts=True, body_inertia=inert if t == 2 else None)
        q, v, a = r["qpos"], r["qvel"], r["qacc"]
    o.mass_matrix(q); o.limits(q, v); o.constraints(q, v)
    if spec.name.startswith("manipulation"):
        ik.diffik(o, spec, q, 7, [0, 0, 0.05], o.fk(q)["xpos"][7], None, 0.05)
W = 4
o = Oracle(specs[1])
qs = np.stack([specs[1].qpos_reset] * W); vs = np.zeros((W, specs[1].nv)); acc = np.zeros((W, specs[1].nv))
o.step_batch(qs, vs, acc, np.zeros((W, specs[1].nu)), 4, nthreads=2)
print("SANITIZED-OK")
'''


def test_oracle_runs_clean_under_asan_and_ubsan():
    from oracle import build_oracle_sanitized
    try:
        lib = build_oracle_sanitized()
    except Exception as e:          # no sanitizer runtime in this toolchain
        pytest.skip(f"sanitizer build unavailable: {e}")
    asan = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    env = dict(os.environ, ORACLE_LIB=lib, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "SANITIZED-OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr[-4000:]
