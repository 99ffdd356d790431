"""FP64 CPU oracle of the GD-PG penalized GLAM solver (test infrastructure only).

Only the test suite, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may
import this package; the product path never does.
"""
from .glam_oracle import *  # noqa: F401,F403
from .glam_oracle import BINOMIAL, GAMMA, GAUSSIAN, POISSON  # noqa: F401
