"""FP64 CPU oracle of H = D G and H^T (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of ``bench.py`` may
import this package.  The product path never does.  See ``oracle.c`` for the definitions and
the readings of the paper it follows.
"""
from .oracle import *  # noqa: F401,F403
