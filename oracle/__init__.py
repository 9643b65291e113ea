"""FP64 CPU oracle (test infrastructure only: imported by the tests, the smoke check and the benchmark's
CPU-baseline leg, never by the product path)."""
from .fem_oracle import *  # noqa: F401,F403
from . import mlp_oracle  # noqa: F401
