"""FP64 CPU oracle of the multigrid F-cycle (test infrastructure only)."""
from .oracle import *  # noqa: F401,F403
from .oracle import Oracle, Problem, build, thomas  # noqa: F401
