"""The staged launches' shared-memory scratch blocks (options.smem_scratch): arrays that no
later launch reads live in each launch's dynamic shared memory when that costs the launch no
residency, else in the working set. Both settings run the same arithmetic in the same order
for every world. The solve's block leaves the bits unchanged. The grouped smooth launch with
its block is a different kernel from the one without, and the compiler may fuse a product
into a sum in one and not in the other. So the default build is compared within FP32
rounding, and a build without fused multiply-add contraction must agree bit for bit. The
batch reports which blocks it uses (b3p_batch_launch_info)."""
import os
import subprocess
import sys

import pytest
import torch

from paper_2601_22074_b300 import build, inputs as I
from paper_2601_22074_b300.batch import Batch, Model

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PLACEMENTS = [dict(working_set=3, warps_per_block=4, schedule=1), dict(working_set=3, warps_per_block=2, schedule=0),
              dict(working_set=2, warps_per_block=4, schedule=1)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def run_pair(options, steps):
    """One batch with the blocks, one without, the same seeds and targets: (with, without)."""
    specs = [I.pendulum(3), I.quadruped(), I.humanoid(), I.manipulation()]
    Ws = [17, 64, 64, 40]
    parts = [torch.tensor(I.ctrl_targets(s, w, steps, 5), dtype=torch.float32).reshape(steps, w * s.nu)
             for s, w in zip(specs, Ws) if s.nu]
    ctrl = torch.cat(parts, dim=1).cuda().contiguous()
    models = [Model(s) for s in specs]
    on = Batch(models, Ws, write_contacts=True, **options)
    off = Batch(models, Ws, write_contacts=True, smem_scratch=1, **options)
    for b in (on, off):
        b.reset(21)
        for t in range(steps):
            b.step(ctrl[t], 4)
    torch.cuda.synchronize()
    return on, off


@pytest.mark.parametrize("options", PLACEMENTS, ids=["grouped-sorted", "grouped-natural", "staged-sorted"])
def test_scratch_blocks_agree_within_rounding(options):
    on, off = run_pair(options, 1)
    info_on, info_off = on.launch_info(), off.launch_info()
    # the humanoid's blocks cost no residency: the solve block is always used, the smooth
    # block in the grouped placement; none with smem_scratch 1
    assert info_on["solve_smem_bytes"] > 0
    assert (info_on["smooth_smem_bytes"] > 0) == (options["working_set"] == 3)
    assert info_off["solve_smem_bytes"] == 0 and info_off["smooth_smem_bytes"] == 0
    for f, floor in (("qpos", 1.0), ("qvel", 1.0), ("qacc", 9.81)):
        a, b = on.get(f), off.get(f)
        err = ((a - b).abs() / torch.clamp(b.abs(), min=floor)).max().item()
        # the contact-step parity bar: two FP32 roundings of a contact step differ as much
        # as the FP32 path differs from the oracle (qacc up to 4.2e-4 on manipulation)
        assert err < 1e-3, (f, err)
    assert torch.equal(on.get("status"), off.get("status"))
    n1, n2 = on.contacts()[1], off.contacts()[1]
    assert torch.equal(n1, n2) and int(n1.sum()) > 0
    if options["working_set"] == 2:   # no smooth block: the solve block alone changes no bit
        for f in ("qpos", "qvel", "qacc", "stats"):
            assert torch.equal(on.get(f), off.get(f)), f


CHILD = r'''
import sys, torch
sys.path.insert(0, "tests")
from test_gpu_smem_scratch import PLACEMENTS, run_pair
for options in PLACEMENTS:
    on, off = run_pair(options, 8)
    for f in ("qpos", "qvel", "qacc", "status", "stats"):
        assert torch.equal(on.get(f), off.get(f)), (options, f)
    (c1, n1), (c2, n2) = on.contacts(), off.contacts()
    assert torch.equal(n1, n2) and torch.equal(c1, c2), options
print("SAME")
'''


def test_scratch_blocks_bitwise_without_fma_contraction():
    lib = build.build_nofma()
    env = dict(os.environ, B3P_LIB_PATH=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "SAME" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]


def test_large_model_keeps_its_arrays_in_the_working_set():
    """Two 31-link chains (nv 62, nM 992): the solve's block would need 58.7 KB and the
    smooth launch's 33.2 KB per 4-world CTA, fewer resident CTAs than either launch reaches
    without them, so the batch uses neither. Its step is the working-set path's, and its
    state after each env step stays within the qpos bar of the oracle. (Its accelerations
    carry the FP32 conditioning of a 31-link chain: 4e-2 relative in every placement.)"""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity import teacher_forced
    spec = I.pendulum(31, nchain=2, noise=0.3)
    opts = dict(working_set=3, warps_per_block=4, schedule=1)
    info = Batch(Model(spec), 8, **opts).launch_info()
    assert info["solve_smem_bytes"] == 0 and info["smooth_smem_bytes"] == 0, info
    assert Batch(Model(I.humanoid()), 8, **opts).launch_info()["solve_smem_bytes"] > 0
    auto = teacher_forced(spec, W=24, nsteps=5, decimation=4, options=opts)
    off = teacher_forced(spec, W=24, nsteps=5, decimation=4, options=dict(opts, smem_scratch=1))
    assert auto.compared == off.compared == 24 * 5
    for f in ("qacc", "qvel", "qpos"):
        assert auto.max(f) == off.max(f), f
    assert auto.max("qpos") <= 1e-3


def test_fused_placement_reports_no_blocks():
    b = Batch(Model(I.quadruped()), 8)
    info = b.launch_info()
    assert info["smooth_smem_bytes"] == 0 and info["solve_smem_bytes"] == 0 and info["lane_smem_bytes"] == 0
    with pytest.raises(RuntimeError):
        Batch(Model(I.quadruped()), 8, smem_scratch=2)
