"""GB300 (sm_103a) neural-volume library: hash-encoded network training and
rendering kernels behind the C ABI of include/nv.h.

Importing the package loads nothing; ``paper_2207_11620_gb300.nv`` loads
libnv.so on first use and raises if it is missing.
"""
