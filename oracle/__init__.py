"""FP64 CPU oracle for the hash-encoded neural volume (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference legs import this package.  The GPU library never imports it.
The arithmetic lives in ``oracle.c``; ``ref`` marshals numpy arrays into it.
"""
from .ref import *  # noqa: F401,F403
