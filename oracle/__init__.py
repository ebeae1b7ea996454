"""CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  It shares no code with the CUDA path:
neither imports the other.
"""
from .tpt_oracle import *  # noqa: F401,F403
