"""FP64 CPU oracle (test infrastructure only).

Plain C, compiled with gcc, loaded through ctypes.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it; the library under ``paper_1711_03836_gb300`` never imports it.
"""
from .oracle import *  # noqa: F401,F403
