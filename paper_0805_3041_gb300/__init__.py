"""GB300-native geometric multigrid F-cycle solver (Wallis 2008, "Methods toward
better Multigrid Solver Convergence").

The solver lives in a CUDA shared library behind the C ABI of ``include/mg.h``;
``binding.Solver`` marshals torch tensors into it.  ``inputs`` builds the
synthetic problems.  Importing the package does not load the library.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "Solver", "load"]


def __getattr__(name):
    if name in ("Solver", "load", "MGError"):
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
