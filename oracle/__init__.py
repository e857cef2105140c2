"""FP64 CPU oracle for sWLR (test infrastructure only; see fp64.py)."""
from .fp64 import *  # noqa: F401,F403
