"""b3p_step_static_scratch: the step for callers that cannot allocate device memory.

Such callers (code handed a fixed set of input and output buffers by a framework
that owns all device memory, or a process whose device memory is fixed at start-up)
cannot give b3p_step the FP64 pivot-fallback workspace it takes from the batch
buffer. b3p_step_static_scratch uses a fixed array inside the library instead.
These tests call it through the C ABI and check it against b3p_step on two calls in
a row, with the fallback forced on so that the array is really used. This file is
collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2601_22074_b300 import _lib as L, build, inputs as I
from paper_2601_22074_b300.batch import Batch, Model

pytestmark = pytest.mark.gpu

TOL = 1e-3  # the contact-step tolerance of the parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _prepared(spec, W, nsteps):
    b = Batch(Model(spec), W)
    b.reset(5)
    p = I.randomised_params(spec, W, 3)
    b.set_param(0, "kp", torch.tensor(p.kp, dtype=torch.float32, device="cuda"))
    b.set_param(0, "kd", torch.tensor(p.kd, dtype=torch.float32, device="cuda"))
    ctrl = torch.tensor(I.ctrl_targets(spec, W, nsteps, 9), dtype=torch.float32, device="cuda")
    return b, ctrl


def _rel(x, ref, floor):
    x, ref = x.double(), ref.double()
    return float((x - ref).abs().max() / max(float(ref.abs().max()), floor))


def test_static_scratch_step_matches_regular_step_on_two_calls():
    spec = I.humanoid(pivot_tau=0.9)  # every Newton iteration refactors in FP64
    W, pre = 256, 40
    regular, ctrl = _prepared(spec, W, pre + 2)
    static, _ = _prepared(spec, W, pre + 2)
    for t in range(pre):                 # identical contact-rich starting states
        regular.step(ctrl[t], 4)
        static.step(ctrl[t], 4)
    torch.cuda.synchronize()
    lib = L.load()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        t = pre + call
        regular.step(ctrl[t], 4)
        rc = lib.b3p_step_static_scratch(static._h, C.c_void_p(ctrl[t].data_ptr()), 4,
                                         C.c_void_p(stream))
        L.check(rc, "b3p_step_static_scratch")
        torch.cuda.synchronize()
        assert _rel(static.get("qacc"), regular.get("qacc"), 9.81) <= TOL
        assert _rel(static.get("qvel"), regular.get("qvel"), 1.0) <= TOL
        assert _rel(static.get("qpos"), regular.get("qpos"), 1.0) <= TOL
        stats = static.get("stats").view(W, 4).cpu().numpy()
        assert stats[:, 2].sum() > 0      # the FP64 workspace was used on this call
        ref = regular.get("stats").view(W, 4).cpu().numpy()
        assert np.array_equal(stats[:, 0], ref[:, 0])   # same contacts


def _mixed(specs, Ws, nsteps):
    b = Batch([Model(s) for s in specs], Ws)
    b.reset(5)
    ctrls = []
    for g, (spec, W) in enumerate(zip(specs, Ws)):
        p = I.randomised_params(spec, W, 3 + g)
        if spec.nu:
            b.set_param(g, "kp", torch.tensor(p.kp, dtype=torch.float32, device="cuda"))
            b.set_param(g, "kd", torch.tensor(p.kd, dtype=torch.float32, device="cuda"))
            ctrls.append(I.ctrl_targets(spec, W, nsteps, 9 + g).reshape(nsteps, -1))
    ctrl = torch.tensor(np.concatenate(ctrls, axis=1), dtype=torch.float32, device="cuda")
    return b, ctrl


def test_static_scratch_mixed_batch_with_dense_hessian_matches_regular_step():
    """Three groups in one batch: the pendulum (no contacts), the humanoid (tree-sparse
    Hessian) and the manipulation world, whose finger-cube contacts join two kinematic
    trees (dense Hessian, nv (nv + 1) doubles per world). With the fallback forced, every
    group's slice of the fixed array is laid out after the previous group's, so a wrong
    per-group offset or dense size shows up as a difference from b3p_step."""
    specs = [I.pendulum(3), I.humanoid(pivot_tau=0.9), I.manipulation(pivot_tau=0.9)]
    Ws, pre, dec = [16, 128, 96], 30, 4
    regular, ctrl = _mixed(specs, Ws, pre + 2)
    static, _ = _mixed(specs, Ws, pre + 2)
    # the gripper closes on the cube so that cross-tree (dense) contacts occur
    nu_h = specs[1].nu * Ws[1]
    grip = ctrl[:, nu_h:].view(pre + 2, Ws[2], specs[2].nu)
    grip[:, :, :-2] = torch.tensor(specs[2].qpos_reset[specs[2].act_qposadr()][:-2], dtype=torch.float32)
    grip[:, :, -2:] = -0.03
    for t in range(pre):
        regular.step(ctrl[t], dec)
        static.step(ctrl[t], dec)
    torch.cuda.synchronize()
    lib = L.load()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        t = pre + call
        regular.step(ctrl[t], dec)
        rc = lib.b3p_step_static_scratch(static._h, C.c_void_p(ctrl[t].data_ptr()), dec,
                                         C.c_void_p(stream))
        L.check(rc, "b3p_step_static_scratch")
        torch.cuda.synchronize()
        for f, floor in (("qacc", 9.81), ("qvel", 1.0), ("qpos", 1.0)):
            a, r = static.get(f), regular.get(f)
            for g in range(3):
                assert _rel(static.group_view(a, f, g), regular.group_view(r, f, g), floor) <= TOL, (f, g)
        stats = static.get("stats")
        for g in (1, 2):
            st = static.group_view(stats, "stats", g).cpu().numpy()
            assert st[:, 2].sum() > 0, g          # this group used its slice of the array
        man = static.group_view(stats, "stats", 2).cpu().numpy()
        assert man[:, 0].max() >= 8               # finger-cube and cube-table contacts


def test_static_scratch_rejects_batches_beyond_its_size():
    spec = I.humanoid()
    m = Model(spec)
    per_world = m.nM + m.nv
    W = L.STATIC_SCRATCH_DOUBLES // per_world + 1
    b = Batch(m, W)
    b.reset(0)
    ctrl = torch.zeros(W * spec.nu, dtype=torch.float32, device="cuda")
    lib = L.load()
    rc = lib.b3p_step_static_scratch(b._h, C.c_void_p(ctrl.data_ptr()), 4,
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert L.ERRORS[rc] == "INVALID_ARG"
    assert "doubles" in lib.b3p_last_error().decode()


def test_static_scratch_refuses_global_working_set_batches():
    b = Batch(Model(I.pendulum(3)), 8, working_set=1)
    lib = L.load()
    rc = lib.b3p_step_static_scratch(b._h, None, 1, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert L.ERRORS[rc] == "UNSUPPORTED"
