"""FP64 CPU oracle of the MLBA hot path — test infrastructure only.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's cpu_baseline and
reference legs may import this package.  It shares no code with the CUDA
library and never imports it.
"""
from .mlba_oracle import *  # noqa: F401,F403
from . import mlba_oracle  # noqa: F401
