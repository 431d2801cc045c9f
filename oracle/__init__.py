"""CPU oracle (test infrastructure only): see oracle/mlpg_oracle.py."""
from .mlpg_oracle import *  # noqa: F401,F403
