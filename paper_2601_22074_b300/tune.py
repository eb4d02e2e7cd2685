"""Autotuner for the step's placement and launch shape.

Every kernel runs one world per warp; what varies is the launch shape: worlds
(warps) per CTA, how many CTAs stay resident per SM, the schedule (static
grid-stride over worlds in group order, or a dynamic queue that hands out the
heaviest morphologies first) and where each world's working set lives (shared
memory, or a global region cached in L1/L2, which lifts the shared-memory cap on
resident worlds; or "staged": one launch per stage over all worlds, each stage
touching a small slice of every working set; or grouped staging, consecutive per-world
stages sharing a launch), and, for the sorted staged placements, whether the Newton
solve of worlds with few contacts runs one world per lane (32 worlds per warp). Results
are identical for every choice of CTA shape and order and agree within FP32 rounding
across placements and solve forms; only the time changes. `autotune` times each candidate on a scratch batch of the same
models and world counts and returns the fastest options.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import inputs as I
from .batch import Batch, Model

CANDIDATES = {
    "warps_per_block": (1, 2, 4),
    "blocks_per_sm": (0,),
    "schedule": (0, 1),
    "working_set": (0, 1, 2, 3),
    "lane_solve": (0, 1),
}


def _time_batch(batch: Batch, ctrl: Optional[torch.Tensor], decimation: int, steps: int,
                warmup: int) -> float:
    stream = torch.cuda.current_stream()
    for t in range(warmup):
        batch.step(ctrl[t % ctrl.shape[0]] if ctrl is not None else None, decimation)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for t in range(steps):
        batch.step(ctrl[(warmup + t) % ctrl.shape[0]] if ctrl is not None else None, decimation)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def autotune(models: Sequence[Model], nworld: Sequence[int], decimation: int = 4,
             steps: int = 3, warmup: int = 8, seed: int = 0,
             candidates: Optional[Dict[str, tuple]] = None, refine: int = 4,
             refine_warmup: int = 100, refine_steps: int = 10) -> Dict:
    """Return {"options": best options, "ms": best time, "table": [(options, ms)...],
    "refined": [(options, ms)...]}.

    Every candidate is timed over `steps` env steps after `warmup` untimed ones from the
    reset. The first env steps after a reset carry few contacts, and candidates within a
    few percent of each other there can rank the other way once the contacts have formed
    and the solve takes its share of the step. So up to `refine` candidates within 10 % of
    the best are timed again, over `refine_steps` env steps after `refine_warmup` untimed
    ones, and the best of those is returned."""
    cand = candidates or CANDIDATES
    specs = [m.spec for m in models]
    nctrl = max(warmup + steps, refine_warmup + refine_steps)
    ctrl = None
    if any(s.nu for s in specs):
        parts = [torch.tensor(I.ctrl_targets(s, w, nctrl, seed), dtype=torch.float32).reshape(nctrl, -1)
                 for s, w in zip(specs, nworld)]
        ctrl = torch.cat(parts, dim=1).cuda()
    table = []
    keys = list(cand)
    seen = set()
    for values in itertools.product(*(cand[k] for k in keys)):
        opts = dict(zip(keys, values))
        if opts.get("working_set", 0) >= 2:   # staged: CTA size and solve order (no residency cap)
            opts.update(blocks_per_sm=0)
        if opts.get("lane_solve", 0) and not (opts.get("working_set", 0) >= 2 and opts.get("schedule", 0) == 1):
            continue                          # the lane solve runs on the sorted staged placements only
        key = tuple(sorted(opts.items()))
        if key in seen:
            continue
        seen.add(key)
        b = Batch(list(models), list(nworld), **opts)
        b.reset(seed)
        ms = _time_batch(b, ctrl, decimation, steps, warmup)
        table.append((opts, ms))
        del b
        torch.cuda.empty_cache()
    best = min(table, key=lambda x: x[1])
    near = sorted((t for t in table if t[1] <= 1.1 * best[1]), key=lambda x: x[1])[:refine]
    refined = []
    if len(near) > 1:
        for opts, _ in near:
            b = Batch(list(models), list(nworld), **opts)
            b.reset(seed)
            refined.append((opts, _time_batch(b, ctrl, decimation, refine_steps, refine_warmup)))
            del b
            torch.cuda.empty_cache()
        best = min(refined, key=lambda x: x[1])
    return {"options": best[0], "ms": best[1], "table": table, "refined": refined}
