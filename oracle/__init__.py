"""Plain FP64 CPU oracle for the carousel phase-retrieval hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import or run anything here.
It shares no code with the GPU library: it is a slow, literal restatement of
the method, used to prove the GPU results.
"""
from .cpra_oracle import *  # noqa: F401,F403
