"""Per-stage cycle breakdown of the step kernel, from the tracing build.

    python -m paper_2601_22074_b300.trace [--workload humanoid] [--worlds 8192] [--steps 20]

Runs the workload on the B3P_TRACE variant of the library (libb3phys_trace.so) and
prints, per stage, the summed clock64() cycles of every world's warp and the share.
"""
import argparse
import ctypes as C
import json
import os
import sys

STAGES = ["load", "fk", "com", "rne", "crba", "ltdl_M+solve", "collide", "rows", "newton_warm",
          "newton_zones+grad", "newton_hessian", "newton_factor+solve", "newton_linesearch",
          "newton_final", "integrate", "store", "newton_solve", "newton_ls_prep"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="humanoid")
    ap.add_argument("--worlds", type=int, default=8192)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--preroll", type=int, default=100)
    ap.add_argument("--working-set", type=int, default=0, help="placement (0 fused ... 3 grouped)")
    ap.add_argument("--wpb", type=int, default=1, help="worlds per CTA")
    args = ap.parse_args()
    from . import build
    os.environ["B3P_LIB_PATH"] = build.build_trace()
    import numpy as np
    import torch
    from . import _lib as L, inputs as I
    from .batch import Batch, Model
    lib = L.load()
    lib.b3p_trace_read.argtypes = [C.POINTER(C.c_ulonglong), C.c_int, C.c_int]
    spec = I.pendulum(3) if args.workload == "pendulum" else getattr(I, args.workload)()
    W = args.worlds
    b = Batch(Model(spec), W, schedule=1, warps_per_block=args.wpb, working_set=args.working_set)
    b.reset(0)
    p = I.randomised_params(spec, W, 7)
    if spec.nu:
        b.set_param(0, "kp", torch.tensor(p.kp, dtype=torch.float32, device="cuda"))
        b.set_param(0, "kd", torch.tensor(p.kd, dtype=torch.float32, device="cuda"))
    ctrl = torch.tensor(I.ctrl_targets(spec, W, args.preroll + args.steps, 11), dtype=torch.float32,
                        device="cuda") if spec.nu else None
    for t in range(args.preroll):
        b.step(ctrl[t] if ctrl is not None else None, 4)
    torch.cuda.synchronize()
    buf = (C.c_ulonglong * len(STAGES))()
    lib.b3p_trace_read(buf, len(STAGES), 1)
    for t in range(args.steps):
        b.step(ctrl[args.preroll + t] if ctrl is not None else None, 4)
    torch.cuda.synchronize()
    lib.b3p_trace_read(buf, len(STAGES), 1)
    cyc = np.array(list(buf), dtype=np.float64)
    tot = cyc.sum()
    per = {s: {"cycles_per_world_step": cyc[i] / (W * args.steps), "share": cyc[i] / tot}
           for i, s in enumerate(STAGES)}
    print(json.dumps({"workload": args.workload, "worlds": W, "steps": args.steps,
                      "cycles_per_world_step": tot / (W * args.steps), "stages": per}))


if __name__ == "__main__":
    sys.exit(main())
