"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and reference arm) may import this package.  The product path never
imports it and shares no code with it.
"""

from .eer4d_oracle import *  # noqa: F401,F403
