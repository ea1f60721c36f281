"""B300-native batched HPS leaf static condensation (arXiv 2211.14969).

The compute path lives in the CUDA library ``libhps.so`` (C ABI, declared in
include/hps.h); ``paper_2211_14969_b300.hps`` is its thin Python binding.
``workloads`` holds the seeded synthetic problems.  Importing the package does
not load the library; the binding loads it on first use and raises if it is
missing.
"""
