"""FP64 CPU oracle for the batched physics step (test infrastructure only).

Only tests/, `__graft_entry__.smoke()` and bench.py's cpu_baseline leg may import
this package. The product path (the CUDA library and its binding) never does.
"""
from .oracle import Oracle, build_oracle, build_oracle_sanitized, CON_STRIDE  # noqa: F401
