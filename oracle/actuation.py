"""PD targets drawn from a request's seed and the actuation delay, FP64 (TEST
INFRASTRUCTURE ONLY).

Plain restatements of two readings of the adopted model; the CUDA path computes them
in its own kernels and shares nothing with this module:
  * served targets (the rollout server's controls): the actuated joints' reset pose plus
    sigma times a standard normal per actuator and env step. Actuators u and u + 1 (u
    even) share one Philox-4x32-10 block (Salmon et al., SC'11) with counter
    {u / 2, rng id, 3, step count} and key {seed low word, seed high word}; its first two
    words give u1 = (w0 >> 8 + 1) / 2^24 in (0, 1] and u2 = (w1 >> 8) / 2^24 in [0, 1),
    and the Box-Muller transform (Box and Muller, 1958) gives the pair
    sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2), the cosine for u and the sine for u + 1;
  * actuation delay (section "Components": actuators with delay): the target applied
    at env step s is the one submitted at step s - D, and the actuated joints' reset
    pose while s < D.
"""
from __future__ import annotations

import math

import numpy as np

from .oracle import Oracle

PURPOSE_TARGETS = 3


def served_targets(spec, seed: int, rng_id: int, step_count: int, sigma: float) -> np.ndarray:
    """[nu] PD targets of one served world at one env step (FP64)."""
    reset = np.asarray(spec.qpos_reset, dtype=np.float64)[spec.act_qposadr()]
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    out = np.empty(spec.nu)
    for u in range(0, spec.nu, 2):
        w = Oracle.philox([u // 2, rng_id, PURPOSE_TARGETS, step_count], key)
        u1 = ((int(w[0]) >> 8) + 1) / 16777216.0
        u2 = (int(w[1]) >> 8) / 16777216.0
        r = math.sqrt(-2.0 * math.log(u1))
        out[u] = reset[u] + sigma * r * math.cos(2.0 * math.pi * u2)
        if u + 1 < spec.nu:
            out[u + 1] = reset[u + 1] + sigma * r * math.sin(2.0 * math.pi * u2)
    return out


def delayed_targets(spec, submitted: np.ndarray, delay: int) -> np.ndarray:
    """Applied targets [T, W, nu] for submitted targets [T, W, nu] under a delay of
    `delay` env steps counted from the reset (step 0)."""
    submitted = np.asarray(submitted, dtype=np.float64)
    if delay <= 0:
        return submitted.copy()
    reset = np.asarray(spec.qpos_reset, dtype=np.float64)[spec.act_qposadr()]
    out = np.empty_like(submitted)
    for s in range(submitted.shape[0]):
        out[s] = submitted[s - delay] if s >= delay else reset
    return out
