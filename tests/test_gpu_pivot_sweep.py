"""Sweep of the FP64-fallback pivot threshold tau (an FP32 LTDL pivot d_k below
tau * H_kk re-factors that world's Newton Hessian in FP64): for tau from 1e-6 to 1e-2 on
the humanoid in the benchmark's launch, the step must match the FP64 oracle within the
contact-step tolerance; the fallback rate and the error are printed for each tau."""
import numpy as np
import pytest
import torch

from paper_2601_22074_b300 import build, inputs as I

pytestmark = pytest.mark.gpu

TOL_CONTACT = 1e-3
BENCH_LAUNCH = dict(working_set=3, warps_per_block=4, schedule=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def test_pivot_threshold_sweep_keeps_parity():
    from parity import teacher_forced
    rows = []
    for tau in (1e-6, 1e-5, 1e-4, 1e-3, 1e-2):
        rep = teacher_forced(I.humanoid(pivot_tau=tau), W=256, nsteps=8, decimation=4, warm_steps=60,
                             options=BENCH_LAUNCH)
        n = rep.compared + rep.mismatches
        rows.append((tau, rep.fallbacks / max(n, 1), rep.max("qacc"), rep.p99("qacc"), rep.max("qvel"),
                     rep.contact_steps, rep.mismatches))
        assert rep.mismatches <= 0.02 * n, (tau, rep.summary())
        for k in ("qacc", "qvel", "qpos", "force"):
            assert rep.max(k) <= TOL_CONTACT, (tau, k, rep.summary())
    print("\ntau      fallbacks/world-step  qacc max  qacc p99  qvel max  contact steps  mismatches")
    for r in rows:
        print(f"{r[0]:.0e}  {r[1]:20.4f}  {r[2]:.2e}  {r[3]:.2e}  {r[4]:.2e}  {r[5]:13d}  {r[6]:10d}")
