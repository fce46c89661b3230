"""FP64 CPU oracle for the FDAS correlation path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import, call or link anything under ``oracle/``.  The
product (the CUDA library and its Python binding) shares no code with it.
"""
from .fdas_oracle import *  # noqa: F401,F403
from .fdas_oracle import build  # noqa: F401
