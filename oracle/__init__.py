"""FP64 CPU oracle of the InfOli network step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import
this package.  The product library never does: it shares no code with it.
"""
from .oracle import *  # noqa: F401,F403
