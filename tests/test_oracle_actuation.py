"""Pins of the oracle's served-target draw and actuation-delay model (CPU)."""
import numpy as np
from scipy import stats

from oracle.actuation import delayed_targets, served_targets
from paper_2601_22074_b300 import inputs as I


def test_served_targets_are_normal_around_the_reset_pose():
    """Box-Muller on Philox words: over many (world, step) draws the deviations from the
    reset pose are N(0, sigma^2) per actuator (Kolmogorov-Smirnov), the cosine and sine
    members of a pair are uncorrelated, and draws of different steps are independent."""
    spec = I.quadruped()
    sigma = 0.5
    reset = spec.qpos_reset[spec.act_qposadr()]
    x = np.array([served_targets(spec, 12345 + (7 << 32), w, s, sigma) - reset
                  for w in range(40) for s in range(40)]) / sigma
    assert x.shape == (1600, spec.nu)
    z = x.reshape(-1)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 4 / np.sqrt(z.size) and abs(z.var() - 1) < 0.08
    assert abs(np.corrcoef(x[:, 0], x[:, 1])[0, 1]) < 0.1
    a = np.array([served_targets(spec, 99, 0, s, 1.0) for s in range(400)])
    assert abs(np.corrcoef(a[:-1, 0], a[1:, 0])[0, 1]) < 0.15


def test_served_targets_depend_on_seed_world_and_step_only():
    spec = I.humanoid()
    a = served_targets(spec, 5, 3, 17, 0.3)
    assert np.array_equal(a, served_targets(spec, 5, 3, 17, 0.3))
    for other in (served_targets(spec, 6, 3, 17, 0.3), served_targets(spec, 5, 4, 17, 0.3),
                  served_targets(spec, 5, 3, 18, 0.3), served_targets(spec, 5 + (1 << 32), 3, 17, 0.3)):
        assert not np.allclose(a, other)
    reset = spec.qpos_reset[spec.act_qposadr()]
    assert np.array_equal(served_targets(spec, 5, 3, 17, 0.0), reset)   # sigma 0: the pose


def test_delay_shifts_targets_and_holds_the_reset_pose_first():
    """Hand-worked sequence: D = 2, submitted c0, c1, c2, c3 -> applied reset, reset, c0, c1."""
    spec = I.quadruped()
    reset = spec.qpos_reset[spec.act_qposadr()]
    c = np.arange(4 * 2 * spec.nu, dtype=np.float64).reshape(4, 2, spec.nu)
    out = delayed_targets(spec, c, 2)
    assert np.array_equal(out[0], np.tile(reset, (2, 1))) and np.array_equal(out[1], out[0])
    assert np.array_equal(out[2], c[0]) and np.array_equal(out[3], c[1])
    assert np.array_equal(delayed_targets(spec, c, 0), c)
