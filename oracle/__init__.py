"""FP64 CPU oracle for the T2 Shuffling PICS solve (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline legs may
import this package.  The CUDA library neither imports nor links it.
"""
from .t2sh_oracle import *  # noqa: F401,F403
