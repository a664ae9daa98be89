"""Plain CPU oracle for the DET-LSH hot path (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may
import this package.  It shares no code with the CUDA path.
"""
from .oracle import *  # noqa: F401,F403
