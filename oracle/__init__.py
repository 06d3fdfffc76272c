"""FP64 CPU oracle (test infrastructure only; see mra_oracle.py)."""
from .mra_oracle import *  # noqa: F401,F403
